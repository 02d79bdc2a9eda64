"""Thin ctypes binding of the C ABI in include/sn.h (argument marshalling only).

Every step of the transport path runs in libsn_gb300.so; PyTorch only supplies
device memory and the current CUDA stream.  If the library is missing this
module raises: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsn_gb300.so")

SN_OK, SN_EINVAL, SN_ENOMEM, SN_ECUDA, SN_ENOCONV, SN_ETIMEOUT, SN_ENAN, SN_ESTATE = range(8)
GE32R, GE32, ANN, ANN_GATED, GE64, OCTNET, ANN_FROZEN = 0, 1, 2, 3, 4, 5, 6
MODES = {"ge32r": GE32R, "ge32": GE32, "ann": ANN, "ann_gated": ANN_GATED, "ge64": GE64, "octnet": OCTNET,
         "ann_frozen": ANN_FROZEN}

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.c_void_p


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class Quadrature(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("ndir", ctypes.c_int32), ("omega", _dp), ("w", _dp)]


class XS(ctypes.Structure):
    _fields_ = [("ngroups", ctypes.c_int32), ("sigt", _dp), ("sigs", _dp), ("q", _dp),
                ("xfer", _dp), ("psi_inc", _dp)]


class Options(ctypes.Structure):
    _fields_ = [("fp64", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("ncell", ctypes.c_int64), ("ndir", ctypes.c_int32), ("ngroups", ctypes.c_int32),
                ("nplanes", ctypes.c_int32), ("dirs_per_octant", ctypes.c_int32),
                ("solves_per_sweep", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


class SnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


_LIB = None

# (name, restype, argtypes) of every exported entry point
_API = [
    ("sn_setup", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Mesh),
                                ctypes.POINTER(Quadrature), ctypes.POINTER(XS), ctypes.POINTER(Options),
                                ctypes.c_void_p]),
    ("sn_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("sn_get_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Info)]),
    ("sn_get_quadrature", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("sn_cell_solve_batch", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_void_p]),
    ("sn_cell_solve_batch_f64", ctypes.c_int, [_fp, _fp, ctypes.c_int64, ctypes.c_void_p]),
    ("sn_sweep", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int]),
    ("sn_source_iterate", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int,
                                         _fp, ctypes.POINTER(ctypes.c_int32), _dp, _dp, ctypes.c_int32]),
    ("sn_get_balance", ctypes.c_int, [ctypes.c_void_p, _dp]),
    ("sn_source", ctypes.c_int, [ctypes.c_void_p, _fp, _fp]),
    ("sn_harvest", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.POINTER(ctypes.c_int64)]),
    ("sn_set_profiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("sn_get_profile", ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    ("sn_wave_plan", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int64)]),
    ("sn_surrogate_prepare", ctypes.c_int, [_fp, ctypes.c_int64, _fp, _fp, ctypes.c_void_p]),
    ("sn_surrogate_init", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("sn_surrogate_set_weights", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    ("sn_surrogate_get_weights", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    ("sn_surrogate_set_gate", ctypes.c_int, [ctypes.c_void_p, ctypes.c_float]),
    ("sn_surrogate_grad", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_float), _dp]),
    ("sn_surrogate_fit", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_float, _dp]),
    ("sn_surrogate_eval", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, _dp]),
    ("sn_surrogate_train", ctypes.c_int, [ctypes.c_void_p, _fp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, _dp, _dp]),
    ("sn_surrogate_apply", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int64)]),
    ("sn_selftest_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    ("sn_surrogate_freeze_gate", ctypes.c_int, [ctypes.c_void_p, _fp]),
    ("sn_surrogate_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]),
    ("sn_adjoint_sweep", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_double, ctypes.c_int32, _fp, _fp, _fp,
                                        _fp, ctypes.POINTER(ctypes.c_int32)]),
    ("sn_response", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, _dp]),
    ("sn_surrogate_grad_noalloc", ctypes.c_int, [_fp, _fp, _fp, ctypes.c_int64, _fp, _fp, ctypes.c_void_p]),
    ("sn_set_scattering_order", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _dp]),
    ("sn_set_geometry", ctypes.c_int, [ctypes.c_void_p, _dp]),
    ("sn_octnet_init", ctypes.c_int, [ctypes.c_void_p, _dp, _dp, ctypes.c_uint64]),
    ("sn_octnet_set", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                     _dp, _dp]),
    ("sn_octnet_get", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    ("sn_octnet_prepare", ctypes.c_int, [ctypes.c_void_p, _fp, ctypes.c_int64, _fp, _fp]),
    ("sn_octnet_grad", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, ctypes.POINTER(ctypes.c_float), _dp]),
    ("sn_octnet_fit", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, _dp]),
    ("sn_octnet_eval", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, _dp, _dp]),
    ("sn_octnet_prune", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                                       ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    ("sn_octnet_apply", ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_int64]),
    ("sn_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("sn_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("sn_destroy", None, [ctypes.c_void_p]),
]


def lib():
    """Load libsn_gb300.so (raises if it was not built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsn_gb300.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _API:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def api_names():
    return [n for n, _, _ in _API]


def _check(st, h=None):
    if st != SN_OK:
        msg = lib().sn_last_error(h)
        raise SnError(st, msg.decode() if msg else "error")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype, shape_tail=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError("expected a contiguous %s tensor" % dtype)
    if shape_tail is not None and tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
        raise ValueError("bad trailing shape %s, want %s" % (tuple(t.shape), shape_tail))
    return ctypes.c_void_p(t.data_ptr())


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _batch(in27, out):
    """Row count n of one-cell problems in27 [n, 27] and their result out [n, 8]:
    ValueError unless both are 2-D with those widths, the same n and one device
    (the kernels read n x 27 and write n x 8 values)."""
    for name, t, w in (("in27", in27, 27), ("out", out, 8)):
        if not isinstance(t, torch.Tensor) or t.dim() != 2 or t.shape[1] != w:
            raise ValueError("%s must be [n, %d], got %s" % (name, w, tuple(getattr(t, "shape", ()))))
    if out.shape[0] != in27.shape[0]:
        raise ValueError("out has %d rows, in27 %d" % (out.shape[0], in27.shape[0]))
    if out.device != in27.device:
        raise ValueError("in27 on %s, out on %s" % (in27.device, out.device))
    return in27.shape[0]


def cell_solve_batch(in27, mode=GE32R, handle=None, out=None):
    """psi[N, 8] of N one-cell problems in27[N, 27] (FP32, CUDA)."""
    if out is None:
        out = torch.empty((in27.shape[0], 8), dtype=torch.float32, device=in27.device)
    n = _batch(in27, out)
    h = handle.h if handle is not None else None
    st = lib().sn_cell_solve_batch(h, _dev(in27, torch.float32, (27,)), _dev(out, torch.float32, (8,)),
                                   n, int(mode), _stream())
    _check(st, h)
    return out


def cell_solve_batch_f64(in27, out=None):
    if out is None:
        out = torch.empty((in27.shape[0], 8), dtype=torch.float64, device=in27.device)
    n = _batch(in27, out)
    st = lib().sn_cell_solve_batch_f64(_dev(in27, torch.float64, (27,)), _dev(out, torch.float64, (8,)),
                                       n, _stream())
    _check(st)
    return out


def wave_plan(nx, ny, nz, G, Do, nsm):
    """(units [n, 4], uplane [n, 4]) int32: the wavefront unit records a float handle
    of this box mesh builds on a GPU with nsm SMs (host only; n = 0 where the mesh is
    left to one launch per hyperplane)."""
    n = ctypes.c_int64()
    _check(lib().sn_wave_plan(nx, ny, nz, G, Do, nsm, None, None, 0, ctypes.byref(n)))
    units = np.zeros((n.value, 4), dtype=np.int32)
    uplane = np.zeros((n.value, 4), dtype=np.int32)
    if n.value:
        _check(lib().sn_wave_plan(nx, ny, nz, G, Do, nsm, units.ctypes.data_as(ctypes.c_void_p),
                                  uplane.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)))
    return units, uplane


NPARAM = 2312


def surrogate_prepare(in27):
    """(features [N, 27], targets [N, 8]) of one-cell problems, targets labelled by
    the library's FP32 elimination (canonical frame, divided by the input scale)."""
    n = in27.shape[0]
    feat = torch.empty((n, 27), dtype=torch.float32, device=in27.device)
    targ = torch.empty((n, 8), dtype=torch.float32, device=in27.device)
    _check(lib().sn_surrogate_prepare(_dev(in27, torch.float32, (27,)), n, _dev(feat, torch.float32, (27,)),
                                      _dev(targ, torch.float32, (8,)), _stream()))
    return feat, targ


def _rows(feat, targ):
    """Row count of a (features [n, 27], targets [n, 8]) pair; ValueError unless both
    are 2-D with those widths and the same n."""
    if feat.dim() != 2 or feat.shape[1] != 27 or targ.dim() != 2 or targ.shape[1] != 8:
        raise ValueError("features must be [n, 27] and targets [n, 8], got %s and %s"
                         % (tuple(feat.shape), tuple(targ.shape)))
    if feat.shape[0] != targ.shape[0]:
        raise ValueError("features have %d rows, targets %d" % (feat.shape[0], targ.shape[0]))
    return int(feat.shape[0])


def _octant_rows(feat, targ):
    """m of octant-grouped features [8m, 27] and targets [8m, 8] (8 equal blocks of m
    rows, octant 0 first); ValueError otherwise."""
    n = _rows(feat, targ)
    if n % 8:
        raise ValueError("features and targets must hold 8 equal octant blocks, got %d rows" % n)
    return n // 8


def surrogate_grad_noalloc(params, feat, targ, grad, loss):
    """Loss and gradient of Eq. (19) without any device allocation by the library:
    params [2312], feat [n, 27], targ [n, 8], grad [2312] (out) FP32 and loss [1]
    FP64 (out) are all caller-owned CUDA tensors on the current device; n <= 32768.
    The C entry point sees only pointers, so every size and the device are checked
    here, before anything is launched (ValueError / TypeError)."""
    n = _rows(feat, targ)
    if params.numel() != NPARAM or grad.numel() != NPARAM:
        raise ValueError("params and grad must hold %d values, got %d and %d"
                         % (NPARAM, params.numel(), grad.numel()))
    if loss.numel() < 1:
        raise ValueError("loss must hold at least one value")
    tensors = (params, feat, targ, grad, loss)
    if not all(isinstance(t, torch.Tensor) and t.is_cuda for t in tensors):
        raise TypeError("expected CUDA tensors")
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in tensors):
        raise ValueError("every tensor must be on the current CUDA device (cuda:%d)" % dev)
    _check(lib().sn_surrogate_grad_noalloc(_dev(params, torch.float32), _dev(feat, torch.float32, (27,)),
                                           _dev(targ, torch.float32, (8,)), n,
                                           _dev(grad, torch.float32), _dev(loss, torch.float64), _stream()))


OCTNET_NIN, OCTNET_NPARAM = 26, 288


def _f32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Problem:
    """A set-up transport problem (sn_setup) on the current CUDA device.

    ``wl`` is a workload dict (see paper_1906_04017_gb300.workloads); explicit
    quadrature may be given as (omega[ndir,3], w[ndir]).  fp64=True makes every
    flux buffer of the handle double precision (mode GE64)."""

    def __init__(self, wl, quadrature=None, fp64=False):
        self.fp64 = bool(fp64)
        self.dtype = torch.float64 if fp64 else torch.float32
        self.default_mode = GE64 if fp64 else GE32R
        self._keep = []
        nx, ny, nz = int(wl["nx"]), int(wl["ny"]), int(wl["nz"])
        mesh = Mesh(nx, ny, nz, float(wl["lx"]), float(wl["ly"]), float(wl["lz"]))
        if quadrature is None:
            quad = Quadrature(int(wl["order"]), 0, None, None)
        else:
            om = np.ascontiguousarray(quadrature[0], dtype=np.float64)
            w = np.ascontiguousarray(quadrature[1], dtype=np.float64)
            self._keep += [om, w]
            quad = Quadrature(0, w.shape[0], _dptr(om), _dptr(w))
        arrs = [np.ascontiguousarray(wl[k], dtype=np.float64) for k in ("sigt", "sigs", "q", "xfer", "psi_inc")]
        self._keep += arrs
        G = arrs[0].reshape(-1, nx * ny * nz).shape[0]
        xs = XS(G, *[_dptr(a) for a in arrs])
        h = ctypes.c_void_p()
        torch.cuda.init()
        self.device = torch.cuda.current_device()
        opts = Options(1 if fp64 else 0)
        st = lib().sn_setup(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(quad), ctypes.byref(xs),
                            ctypes.byref(opts), _stream())
        _check(st)
        self.h = h
        self._keep = []
        info = Info()
        _check(lib().sn_get_info(self.h, ctypes.byref(info)), self.h)
        self.ncell, self.ndir, self.G = info.ncell, info.ndir, info.ngroups
        self.nplanes, self.dirs_per_octant = info.nplanes, info.dirs_per_octant
        self.solves_per_sweep = info.solves_per_sweep
        self.device_bytes = info.device_bytes
        self.L, self.K = 0, 1

    def close(self):
        if getattr(self, "h", None):
            lib().sn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _flux(self, *ts, dtype=None, moments=True):
        """Device pointers of tensors in the handle's flux layout: [G, ncell, 8], or
        [G, K, ncell, 8] under anisotropic scattering where the call takes moments.
        The kernels index G x K x ncell x 8 values, so any other shape (every
        argument's shape is checked first), dtype or device is refused here, before
        any library call."""
        want = (self.G, self.ncell, 8) if (self.K == 1 or not moments) else (self.G, self.K, self.ncell, 8)
        for t in ts:
            if not isinstance(t, torch.Tensor) or tuple(t.shape) != want:
                raise ValueError("bad flux shape %s, want %s" % (tuple(getattr(t, "shape", ())), want))
        ps = []
        for t in ts:
            ps.append(_dev(t, self.dtype if dtype is None else dtype))
            if t.device.index != self.device:
                raise ValueError("tensor on %s, the problem on cuda:%d" % (t.device, self.device))
        return ps[0] if len(ps) == 1 else ps

    def _sync_stream(self):
        _check(lib().sn_set_stream(self.h, _stream()), self.h)

    def quadrature(self):
        om = np.zeros((self.ndir, 3))
        w = np.zeros(self.ndir)
        _check(lib().sn_get_quadrature(self.h, _dptr(om), _dptr(w)), self.h)
        return om, w

    def flux_tensor(self, device="cuda"):
        """Zero flux (or source) array of the handle's layout: [G, ncell, 8], or the
        moments [G, K, ncell, 8] under anisotropic scattering."""
        shape = (self.G, self.ncell, 8) if self.K == 1 else (self.G, self.K, self.ncell, 8)
        return torch.zeros(shape, dtype=self.dtype, device=device)

    def set_geometry(self, xyz=None):
        """General hexahedral cells: vertex coordinates [(nx+1)(ny+1)(nz+1), 3] (see
        workloads.deformed_vertices); None restores the box cells."""
        a = None if xyz is None else np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self._sync_stream()
        _check(lib().sn_set_geometry(self.h, None if a is None else _dptr(a)), self.h)

    def set_scattering_order(self, L, sigs_n=None):
        """Anisotropic scattering to Legendre order L (Eqs. (3)-(8)); sigs_n: sigma_{s,n}
        for n = 1..L, [L, G, ncell].  Flux and source arrays become moments
        [G, (L+1)^2, ncell, 8]."""
        a = None
        if L > 0:
            a = np.ascontiguousarray(sigs_n, dtype=np.float64).reshape(L, self.G, self.ncell)
        self._sync_stream()
        _check(lib().sn_set_scattering_order(self.h, int(L), None if a is None else _dptr(a)), self.h)
        self.L, self.K = int(L), (int(L) + 1) ** 2

    def sweep(self, S, phi=None, mode=None):
        """One sweep: phi[G, ncell, 8] from the isotropic nodal source S[G, ncell, 8]."""
        if phi is None:
            phi = torch.empty_like(S)
        pS, pphi = self._flux(S, phi)
        self._sync_stream()
        mode = self.default_mode if mode is None else mode
        _check(lib().sn_sweep(self.h, pS, pphi, int(mode)), self.h)
        return phi

    def source_iterate(self, phi=None, tol=1e-6, max_it=500, mode=None, use_graph=True, allow_noconv=False):
        """Source iteration in place on phi[G, ncell, 8]; returns a dict of results."""
        mode = self.default_mode if mode is None else mode
        if phi is None:
            phi = self.flux_tensor()
        pphi = self._flux(phi)
        self._sync_stream()
        it = ctypes.c_int32(0)
        cmax = ctypes.c_double(0)
        cmean = ctypes.c_double(0)
        st = lib().sn_source_iterate(self.h, float(tol), int(max_it), int(mode), pphi, ctypes.byref(it),
                                     ctypes.byref(cmax), ctypes.byref(cmean), 1 if use_graph else 0)
        if not (st == SN_ENOCONV and allow_noconv):
            _check(st, self.h)
        return dict(phi=phi, iters=it.value, change_max=cmax.value, change_mean=cmean.value,
                    converged=(st == SN_OK))

    def source(self, phi, S=None):
        """The isotropic nodal source S[G, ncell, 8] built from phi by the library."""
        if S is None:
            S = torch.empty_like(phi)
        pphi, pS = self._flux(phi, S)
        self._sync_stream()
        _check(lib().sn_source(self.h, pphi, pS), self.h)
        return S

    def harvest(self, S, cap, seed=0):
        """One elimination sweep from S that returns about `cap` of its solves as
        one-cell problems in27 [n, 27] (positive-octant frame)."""
        if int(cap) < 0:
            raise ValueError("cap must be non-negative")
        pS = self._flux(S, dtype=torch.float32, moments=False)
        self._sync_stream()
        out = torch.empty((int(cap), 27), dtype=torch.float32, device=S.device)
        n = ctypes.c_int64(0)
        _check(lib().sn_harvest(self.h, pS, _dev(out, torch.float32, (27,)), int(cap), int(seed), ctypes.byref(n)),
               self.h)
        return out[:n.value]

    def set_profiling(self, on=True):
        _check(lib().sn_set_profiling(self.h, 1 if on else 0), self.h)

    def profile(self, reset=True):
        """(summed sweep-kernel milliseconds, sweeps timed) since the last reset."""
        ms = ctypes.c_double(0)
        n = ctypes.c_int64(0)
        _check(lib().sn_get_profile(self.h, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0), self.h)
        return ms.value, n.value

    def balance(self):
        t = np.zeros(4)
        _check(lib().sn_get_balance(self.h, _dptr(t)), self.h)
        return t

    # ---- surrogate network (Sec. 3) ----
    def surrogate_init(self, seed=0):
        self._sync_stream()
        _check(lib().sn_surrogate_init(self.h, int(seed)), self.h)

    def surrogate_set_weights(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != NPARAM:
            raise ValueError("the surrogate has %d parameters, got %d" % (NPARAM, p.size))
        self._sync_stream()
        _check(lib().sn_surrogate_set_weights(self.h, _f32p(p)), self.h)

    def surrogate_weights(self):
        p = np.zeros(NPARAM, dtype=np.float32)
        _check(lib().sn_surrogate_get_weights(self.h, _f32p(p)), self.h)
        return p

    def surrogate_set_gate(self, tau):
        _check(lib().sn_surrogate_set_gate(self.h, float(tau)), self.h)

    def surrogate_grad(self, feat, targ):
        """(loss, gradient [2312]) of Eq. (19) at the current weights over all rows."""
        n = _rows(feat, targ)
        self._sync_stream()
        g = np.zeros(NPARAM, dtype=np.float32)
        loss = ctypes.c_double(0)
        _check(lib().sn_surrogate_grad(self.h, _dev(feat, torch.float32, (27,)), _dev(targ, torch.float32, (8,)),
                                       n, _f32p(g), ctypes.byref(loss)), self.h)
        return loss.value, g

    def surrogate_fit(self, feat, targ, steps, batch, lr):
        n = _rows(feat, targ)
        self._sync_stream()
        loss = ctypes.c_double(0)
        _check(lib().sn_surrogate_fit(self.h, _dev(feat, torch.float32, (27,)), _dev(targ, torch.float32, (8,)),
                                      n, int(steps), int(batch), float(lr), ctypes.byref(loss)), self.h)
        return loss.value

    def surrogate_eval(self, feat, targ):
        n = _rows(feat, targ)
        self._sync_stream()
        mae = ctypes.c_double(0)
        _check(lib().sn_surrogate_eval(self.h, _dev(feat, torch.float32, (27,)), _dev(targ, torch.float32, (8,)),
                                       n, ctypes.byref(mae)), self.h)
        return mae.value

    def surrogate_train(self, in27, n_test, steps, batch, lr, seed=0):
        """Label in27 with elimination, initialise, train with Adam; (train MAE, test MAE)."""
        self._sync_stream()
        a = ctypes.c_double(0)
        b = ctypes.c_double(0)
        _check(lib().sn_surrogate_train(self.h, _dev(in27, torch.float32, (27,)), in27.shape[0], int(n_test),
                                        int(steps), int(batch), float(lr), int(seed), ctypes.byref(a),
                                        ctypes.byref(b)), self.h)
        return a.value, b.value

    def surrogate_apply(self, in27, gated=True, out=None):
        """psi [N, 8] from the tensor-core network; returns (psi, number of gate fallbacks)."""
        if out is None:
            out = torch.empty((in27.shape[0], 8), dtype=torch.float32, device=in27.device)
        n = _batch(in27, out)
        self._sync_stream()
        nfb = ctypes.c_int64(0)
        _check(lib().sn_surrogate_apply(self.h, _dev(in27, torch.float32, (27,)), _dev(out, torch.float32, (8,)),
                                        n, 1 if gated else 0, ctypes.byref(nfb)), self.h)
        return out, nfb.value

    def surrogate_stats(self):
        """(fallbacks, timeouts) of the last surrogate sweep / iteration / apply."""
        a = ctypes.c_int64(0)
        b = ctypes.c_int64(0)
        _check(lib().sn_surrogate_stats(self.h, ctypes.byref(a), ctypes.byref(b)), self.h)
        return a.value, b.value

    def surrogate_freeze_gate(self, S):
        """Record the residual gate's decisions of one gated sweep from S [G, C, 8] for
        later ANN_FROZEN sweeps; returns the number of rows sent to elimination."""
        self._sync_stream()
        _check(lib().sn_surrogate_freeze_gate(self.h, _dev(S, torch.float32, (8,))), self.h)
        return self.surrogate_stats()[0]

    def selftest_wait(self, limit_cycles=100000):
        """Run the bounded-wait self-test (sn_selftest_wait); returns its status code
        (SN_ETIMEOUT when the withheld wait gave up as designed)."""
        self._sync_stream()
        return int(lib().sn_selftest_wait(self.h, int(limit_cycles)))

    # ---- the paper's per-octant networks (Sec. 3, Sec. 4) ----
    def octnet_init(self, lo, hi, seed=0):
        """Glorot-initialised networks with a-priori input ranges lo, hi [8, 26]."""
        lo = np.ascontiguousarray(lo, dtype=np.float64).reshape(8, OCTNET_NIN)
        hi = np.ascontiguousarray(hi, dtype=np.float64).reshape(8, OCTNET_NIN)
        self._sync_stream()
        _check(lib().sn_octnet_init(self.h, _dptr(lo), _dptr(hi), int(seed)), self.h)

    def octnet_set(self, params, mask=None, lo=None, hi=None):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(8, OCTNET_NPARAM)
        k = None if mask is None else np.ascontiguousarray(mask, dtype=np.float32).reshape(8, OCTNET_NPARAM)
        r = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(8, OCTNET_NIN) for a in (lo, hi)]
        self._sync_stream()
        _check(lib().sn_octnet_set(self.h, _f32p(p), None if k is None else _f32p(k),
                                   None if r[0] is None else _dptr(r[0]), None if r[1] is None else _dptr(r[1])),
               self.h)

    def octnet_get(self):
        """(params [8, 288], mask [8, 288]) FP32."""
        p = np.zeros((8, OCTNET_NPARAM), dtype=np.float32)
        k = np.zeros((8, OCTNET_NPARAM), dtype=np.float32)
        self._sync_stream()
        _check(lib().sn_octnet_get(self.h, _f32p(p), _f32p(k)), self.h)
        return p, k

    def octnet_prepare(self, in27):
        """(features [8m, 27], targets [8m, 8]) of octant-grouped one-cell problems in27 [8m, 27]."""
        n = in27.shape[0]
        if n % 8:
            raise ValueError("in27 must hold 8 equal octant blocks")
        feat = torch.empty((n, 27), dtype=torch.float32, device=in27.device)
        targ = torch.empty((n, 8), dtype=torch.float32, device=in27.device)
        self._sync_stream()
        _check(lib().sn_octnet_prepare(self.h, _dev(in27, torch.float32, (27,)), n // 8,
                                       _dev(feat, torch.float32, (27,)), _dev(targ, torch.float32, (8,))), self.h)
        return feat, targ

    def octnet_grad(self, feat, targ):
        """(loss [8], gradient [8, 288]) of Eq. (19) per octant at the current parameters."""
        g = np.zeros((8, OCTNET_NPARAM), dtype=np.float32)
        loss = np.zeros(8)
        m = _octant_rows(feat, targ)
        self._sync_stream()
        _check(lib().sn_octnet_grad(self.h, _dev(feat, torch.float32, (27,)), _dev(targ, torch.float32, (8,)),
                                    m, _f32p(g), _dptr(loss)), self.h)
        return loss, g

    def octnet_fit(self, feat, targ, steps, lr):
        loss = np.zeros(8)
        m = _octant_rows(feat, targ)
        self._sync_stream()
        _check(lib().sn_octnet_fit(self.h, _dev(feat, torch.float32, (27,)), _dev(targ, torch.float32, (8,)),
                                   m, int(steps), float(lr), _dptr(loss)), self.h)
        return loss

    def octnet_eval(self, feat, targ):
        """(mean absolute error [8], mean squared error [8]) per octant."""
        mae = np.zeros(8)
        mse = np.zeros(8)
        m = _octant_rows(feat, targ)
        self._sync_stream()
        _check(lib().sn_octnet_eval(self.h, _dev(feat, torch.float32, (27,)), _dev(targ, torch.float32, (8,)),
                                    m, _dptr(mae), _dptr(mse)), self.h)
        return mae, mse

    def octnet_prune(self, feat, targ, retrain_steps, lr, tol=1e-3, max_drops=272):
        """Connection dropping (Sec. 3); returns the drops kept per octant [8]."""
        d = (ctypes.c_int32 * 8)()
        m = _octant_rows(feat, targ)
        self._sync_stream()
        _check(lib().sn_octnet_prune(self.h, _dev(feat, torch.float32, (27,)), _dev(targ, torch.float32, (8,)),
                                     m, int(retrain_steps), float(lr), float(tol), int(max_drops), d),
               self.h)
        return np.array(list(d))

    def octnet_apply(self, in27, out=None):
        """psi [N, 8] of one-cell problems by the networks of their octants."""
        if out is None:
            out = torch.empty((in27.shape[0], 8), dtype=torch.float32, device=in27.device)
        n = _batch(in27, out)
        self._sync_stream()
        _check(lib().sn_octnet_apply(self.h, _dev(in27, torch.float32, (27,)), _dev(out, torch.float32, (8,)), n),
               self.h)
        return out

    # ---- discrete adjoint ----
    def adjoint(self, phi, resp, tol=1e-6, max_it=500, allow_noconv=False):
        """Gradients of R = resp . phi at the converged forward flux phi (device
        [G, ncell, 8]): dict(Lam [G, ncell, 8], grad_sigt, grad_sigs, grad_q [G, ncell]
        FP64, iters)."""
        pphi, presp = self._flux(phi, resp, dtype=torch.float32, moments=False)
        self._sync_stream()
        G, C = self.G, self.ncell
        Lam = torch.empty((G, C, 8), dtype=torch.float32, device=phi.device)
        gt = torch.empty((G, C), dtype=torch.float64, device=phi.device)
        gs = torch.empty_like(gt)
        gq = torch.empty_like(gt)
        it = ctypes.c_int32(0)
        st = lib().sn_adjoint_sweep(self.h, pphi, presp, float(tol), int(max_it), _dev(Lam, torch.float32, (C, 8)),
                                    _dev(gt, torch.float64), _dev(gs, torch.float64), _dev(gq, torch.float64),
                                    ctypes.byref(it))
        if not (st == SN_ENOCONV and allow_noconv):
            _check(st, self.h)
        return dict(Lam=Lam, grad_sigt=gt, grad_sigs=gs, grad_q=gq, iters=it.value, converged=(st == SN_OK))

    def response(self, phi, resp):
        """R = sum resp * phi (device [G, ncell, 8] tensors of the handle's dtype), FP64."""
        pphi, presp = self._flux(phi, resp, moments=False)
        self._sync_stream()
        R = ctypes.c_double(0.0)
        _check(lib().sn_response(self.h, pphi, presp, ctypes.byref(R)), self.h)
        return R.value


class DetectorResponse(torch.autograd.Function):
    """R(sigma_t, sigma_s, q) = sum resp * phi of the converged source iteration, as a
    differentiable function of the per-cell, per-group cross sections and source
    (tensors of the workload's [G, ...] shape); backward runs the discrete adjoint
    (sn_adjoint_sweep).  The other fields (mesh, quadrature order, transfer matrix,
    inflow) come from the workload dict ``wl``; ``resp`` is dR/dphi [G, ncell, 8].

        R = DetectorResponse.apply(sigt, sigs, q, wl, resp, tol, max_it)
    """

    @staticmethod
    def forward(ctx, sigt, sigs, q, wl, resp, tol=1e-6, max_it=500):
        w = dict(wl)
        for k, v in (("sigt", sigt), ("sigs", sigs), ("q", q)):
            w[k] = v.detach().to("cpu", torch.float64).numpy()
        P = Problem(w)
        try:
            fwd = P.source_iterate(tol=tol, max_it=max_it)
            r = resp.detach().to(device="cuda", dtype=torch.float32).reshape(P.G, P.ncell, 8).contiguous()
            R = P.response(fwd["phi"], r)
        except Exception:
            P.close()
            raise
        ctx.P, ctx.phi, ctx.r, ctx.tol, ctx.max_it = P, fwd["phi"], r, tol, max_it
        ctx.shapes = [(t.shape, t.dtype, t.device) for t in (sigt, sigs, q)]
        return torch.tensor(R, dtype=torch.float64, device=sigt.device)

    @staticmethod
    def backward(ctx, gR):
        P = ctx.P
        try:
            adj = P.adjoint(ctx.phi, ctx.r, tol=ctx.tol, max_it=ctx.max_it)
        finally:
            P.close()
            ctx.P = None
        out = []
        for key, (shape, dtype, device) in zip(("grad_sigt", "grad_sigs", "grad_q"), ctx.shapes):
            g = adj[key].to(device=device) * gR.to(device=device, dtype=torch.float64)
            out.append(g.reshape(shape).to(dtype))
        return out[0], out[1], out[2], None, None, None, None

"""FP64 oracle of the DFEM S_n transport solve (Tano & Ragusa, arXiv:1906.04017).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline and reference legs) may import this package.
The product library never calls it and shares no code with it.

The sweep, the per-cell assembly, the Gaussian elimination and the source
iteration live in plain C (``sn_oracle.c``, FP64, built by ``oracle/build.py``);
this module is the ctypes wrapper, plus the numpy FP64 oracles of the
surrogate network (``oracle.mlp``), of the paper's per-octant networks
(``oracle.octant_net``), of the discrete adjoint (``oracle.adjoint``) and the real
spherical harmonics of the anisotropic scattering source (``oracle.harmonics``).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(_build.build())
        _declare(_LIB)
    return _LIB


_dp = ctypes.POINTER(ctypes.c_double)


class Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("ndir", ctypes.c_int), ("omega", _dp), ("w", _dp),
        ("G", ctypes.c_int), ("sigt", _dp), ("sigs", _dp), ("q", _dp),
        ("xfer", _dp), ("psi_inc", _dp), ("hex", ctypes.c_void_p),
    ]

HEX_DOUBLES = 64 + 3 * 64 + 6 * 3 * 64     # or_hex: M, L[3], Fv[6][3]


class OctNet(ctypes.Structure):
    _fields_ = [("p", _dp), ("lo", _dp), ("hi", _dp)]


class Mlp(ctypes.Structure):
    _fields_ = [("p", _dp), ("bf16", ctypes.c_int)]


def _declare(L):
    L.or_ge.argtypes = [ctypes.c_int, _dp, _dp, _dp]
    L.or_lqn.argtypes = [ctypes.c_int, _dp, _dp]
    L.or_element.argtypes = [ctypes.c_double] * 3 + [_dp] * 4
    L.or_assemble.argtypes = [ctypes.c_double] * 3 + [_dp, ctypes.c_double, _dp, _dp, _dp, _dp]
    L.or_assemble_inflow_form.argtypes = [ctypes.c_double] * 3 + [_dp, ctypes.c_double, _dp]
    L.or_cell_solve.argtypes = [_dp, _dp]
    L.or_cell_solve_batch.argtypes = [ctypes.c_long, _dp, _dp]
    P = ctypes.POINTER(Problem)
    L.or_sweep_dir.argtypes = [P, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    L.or_sweep.argtypes = [P, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    L.or_source.argtypes = [P, _dp, _dp]
    L.or_source_iterate.argtypes = [P, ctypes.c_double, ctypes.c_int, _dp,
                                    ctypes.POINTER(ctypes.c_int), _dp, _dp, _dp]
    L.or_num_threads.argtypes = []
    L.or_hex_element.argtypes = [_dp, _dp]
    L.or_hex_elements.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
    L.or_source_moments.argtypes = [P, ctypes.c_int, _dp, _dp, _dp]
    L.or_sweep_moments.argtypes = [P, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp]
    L.or_source_iterate_moments.argtypes = [P, ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp,
                                            ctypes.POINTER(ctypes.c_int), _dp, _dp, _dp]
    N = ctypes.POINTER(OctNet)
    L.or_octnet_cell_batch.argtypes = [N, ctypes.c_long, _dp, _dp]
    L.or_sweep_octnet.argtypes = [P, N, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    Mp = ctypes.POINTER(Mlp)
    L.or_mlp_cell_batch.argtypes = [Mp, ctypes.c_long, _dp, _dp]
    L.or_sweep_mlp.argtypes = [P, Mp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    L.or_sweep_mlp_gated.argtypes = [P, Mp, ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_long)]
    L.or_adjoint.argtypes = [P, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp, _dp,
                             ctypes.POINTER(ctypes.c_int)]


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return lib().or_num_threads()


def ge_solve(A, b):
    """Gaussian elimination with partial pivoting (FP64) of one n x n system."""
    A = _f64(A).copy()
    b = _f64(b).copy()
    n = b.shape[0]
    x = np.zeros(n)
    if lib().or_ge(n, _p(A), _p(b), _p(x)) != 0:
        raise ZeroDivisionError("zero pivot")
    return x


def lqn(order):
    """Level-symmetric LQ_N directions [ndir,3] and weights [ndir] (sum 4 pi)."""
    n = order * (order + 2)
    om = np.zeros((n, 3))
    w = np.zeros(n)
    nd = lib().or_lqn(order, _p(om), _p(w))
    if nd < 0:
        raise ValueError("unsupported LQ_N order %r" % order)
    return om, w


def element(dx, dy, dz):
    """Element matrices (M, L[3], G[3], F[6]) of the Q1 box, by Gauss quadrature."""
    M = np.zeros((8, 8)); L = np.zeros((3, 8, 8)); G = np.zeros((3, 8, 8)); F = np.zeros((6, 8, 8))
    lib().or_element(dx, dy, dz, _p(M), _p(L), _p(G), _p(F))
    return M, L, G, F


def assemble(in27):
    """(A, b) of one one-cell problem in the outflow form of Eq. (14)."""
    x = _f64(in27)
    A = np.zeros((8, 8)); b = np.zeros(8)
    lib().or_assemble(x[3], x[4], x[5], _p(_f64(x[0:3])), x[6], _p(_f64(x[7:15])),
                      _p(_f64(x[15:27])), _p(A), _p(b))
    return A, b


def assemble_inflow_form(in27):
    x = _f64(in27)
    A = np.zeros((8, 8))
    lib().or_assemble_inflow_form(x[3], x[4], x[5], _p(_f64(x[0:3])), x[6], _p(A))
    return A


def cell_solve(in27):
    """Solve a batch of one-cell problems in27[N,27] -> psi[N,8] (FP64 GE)."""
    x = _f64(np.atleast_2d(in27))
    out = np.zeros((x.shape[0], 8))
    if lib().or_cell_solve_batch(x.shape[0], _p(x), _p(out)) != 0:
        raise ZeroDivisionError("zero pivot")
    return out


class _OctNetArrays:
    """FP64 copies of per-octant network parameters [8, 288] and input ranges [8, 26]
    kept alive beside their ctypes view."""

    def __init__(self, P, lo, hi):
        self.P, self.lo, self.hi = _f64(P).reshape(8, 288), _f64(lo).reshape(8, 26), _f64(hi).reshape(8, 26)
        self.c = OctNet(_p(self.P), _p(self.lo), _p(self.hi))


def octnet_cell(P, lo, hi, in27):
    """psi [N, 8] of the per-octant networks (the C oracle's evaluation) on in27 [N, 27]."""
    net = _OctNetArrays(P, lo, hi)
    x = _f64(np.atleast_2d(in27))
    out = np.zeros((x.shape[0], 8))
    lib().or_octnet_cell_batch(ctypes.byref(net.c), x.shape[0], _p(x), _p(out))
    return out


class _MlpArrays:
    """An FP64 copy of the surrogate's parameters [2312] kept alive beside its ctypes view."""

    def __init__(self, p, bf16):
        self.p = _f64(p).reshape(-1)
        assert self.p.size == 2312
        self.c = Mlp(_p(self.p), 1 if bf16 else 0)


def mlp_cell(p, in27, bf16=False):
    """psi [N, 8] of the surrogate network p [2312] (the C oracle's evaluation) on in27
    [N, 27]; bf16 applies the rounding steps of the tensor-core path."""
    net = _MlpArrays(p, bf16)
    x = _f64(np.atleast_2d(in27))
    out = np.zeros((x.shape[0], 8))
    lib().or_mlp_cell_batch(ctypes.byref(net.c), x.shape[0], _p(x), _p(out))
    return out


def hex_element(X):
    """(M [8,8], L [3,8,8], Fv [6,3,8,8]) of the trilinear cell with vertices X [8,3]
    (node n = a + 2b + 4c)."""
    X = _f64(X).reshape(8, 3)
    out = np.zeros(HEX_DOUBLES)
    lib().or_hex_element(_p(X), _p(out))
    return out[:64].reshape(8, 8), out[64:256].reshape(3, 8, 8), out[256:].reshape(6, 3, 8, 8)


class OracleProblem:
    """Holds the FP64 arrays of one problem and the ctypes view of them.

    Fields follow the workload dictionaries of ``paper_1906_04017_gb300.workloads``:
    nx, ny, nz, lx, ly, lz, order (or omega/w), sigt[G,ncell], sigs[G,ncell],
    q[G,ncell], xfer[G,G], psi_inc[G,6].
    """

    def __init__(self, wl, omega=None, w=None, xyz=None):
        """xyz: optional vertex coordinates [(nx+1)(ny+1)(nz+1), 3] of general
        hexahedral cells with the mesh's structured topology (box cells if None)."""
        self.nx, self.ny, self.nz = int(wl["nx"]), int(wl["ny"]), int(wl["nz"])
        self.ncell = self.nx * self.ny * self.nz
        self.dx = wl["lx"] / self.nx
        self.dy = wl["ly"] / self.ny
        self.dz = wl["lz"] / self.nz
        if omega is None:
            omega, w = lqn(int(wl["order"]))
        self.omega = _f64(omega)
        self.w = _f64(w)
        self.ndir = self.w.shape[0]
        self.sigt = _f64(wl["sigt"]).reshape(-1, self.ncell)
        self.G = self.sigt.shape[0]
        self.sigs = _f64(wl["sigs"]).reshape(self.G, self.ncell)
        self.q = _f64(wl["q"]).reshape(self.G, self.ncell)
        self.xfer = _f64(wl["xfer"]).reshape(self.G, self.G)
        self.psi_inc = _f64(wl["psi_inc"]).reshape(self.G, 6)
        self.hex = None
        if xyz is not None:
            self.xyz = _f64(xyz).reshape(-1, 3)
            self.hex = np.zeros(self.ncell * HEX_DOUBLES)
            lib().or_hex_elements(self.nx, self.ny, self.nz, _p(self.xyz), _p(self.hex))
        self.c = Problem(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.ndir,
                         _p(self.omega), _p(self.w), self.G, _p(self.sigt), _p(self.sigs),
                         _p(self.q), _p(self.xfer), _p(self.psi_inc),
                         None if self.hex is None else self.hex.ctypes.data)

    def sweep_dir(self, d, g, S, bx=None, by=None, bz=None):
        """psi[ncell,8] of direction d, group g, for the nodal source S[ncell,8].
        Returns (psi, tallies[4] = leakage, collision, source, inflow)."""
        S = _f64(S).reshape(self.ncell, 8)
        psi = np.zeros((self.ncell, 8))
        tal = np.zeros(4)
        bx, by, bz = [None if b is None else _f64(b) for b in (bx, by, bz)]
        if lib().or_sweep_dir(ctypes.byref(self.c), d, g, _p(S), _p(bx), _p(by), _p(bz),
                              _p(psi), _p(tal)) != 0:
            raise ZeroDivisionError("zero pivot")
        return psi, tal

    def sweep(self, S, groups=None, dirs=None, octnet=None, mlp=None, gate=None):
        """phi[G,ncell,8] = sum_d w_d psi_d for the isotropic source S[G,ncell,8].

        ``groups`` / ``dirs`` are (begin, end) ranges; phi is zero outside them.
        ``octnet`` = (P [8, 288], lo [8, 26], hi [8, 26]) replaces every per-cell
        solve by the octant networks (oracle.octant_net); ``mlp`` = (p [2312], bf16)
        by the workload's surrogate network (oracle.mlp, with the BF16 rounding steps
        if bf16); with ``gate`` = tau as well, a cell keeps the network's prediction
        only where its residual passes ||b - A psi|| <= tau ||b|| and is solved by
        elimination otherwise (the count is left in ``self.last_fallbacks``).
        Returns (phi, tallies[4])."""
        S = _f64(S).reshape(self.G, self.ncell, 8)
        g0, g1 = groups if groups else (0, self.G)
        d0, d1 = dirs if dirs else (0, self.ndir)
        phi = np.zeros((self.G, self.ncell, 8))
        tal = np.zeros(4)
        if mlp is not None and gate is not None:
            net = _MlpArrays(*mlp)
            nfb = ctypes.c_long(0)
            rc = lib().or_sweep_mlp_gated(ctypes.byref(self.c), ctypes.byref(net.c), float(gate), _p(S), _p(phi),
                                          g0, g1, d0, d1, _p(tal), ctypes.byref(nfb))
            self.last_fallbacks = int(nfb.value)
        elif mlp is not None:
            net = _MlpArrays(*mlp)
            rc = lib().or_sweep_mlp(ctypes.byref(self.c), ctypes.byref(net.c), _p(S), _p(phi), g0, g1, d0, d1,
                                    _p(tal))
        elif octnet is None:
            rc = lib().or_sweep(ctypes.byref(self.c), _p(S), _p(phi), g0, g1, d0, d1, _p(tal))
        else:
            net = _OctNetArrays(*octnet)
            rc = lib().or_sweep_octnet(ctypes.byref(self.c), ctypes.byref(net.c), _p(S), _p(phi), g0, g1, d0, d1,
                                       _p(tal))
        if rc != 0:
            raise ZeroDivisionError("zero pivot")
        return phi, tal

    # ---- anisotropic scattering (Eqs. (3)-(8)); see oracle.harmonics ----
    def _aniso(self, sigs_n):
        """sigma_{s,n} [L+1][G][ncell] with row 0 = the problem's sigma_s; K = (L+1)^2;
        scaled harmonics of the problem's directions [ndir][K]."""
        from . import harmonics
        s = _f64(sigs_n).reshape(-1, self.G, self.ncell)
        L = s.shape[0] - 1
        full = _f64(np.concatenate([self.sigs[None], s[1:]], 0)) if L > 0 else _f64(self.sigs[None])
        return L, (L + 1) ** 2, full, _f64(harmonics.yhat(self.omega, L))

    def source_moments(self, phi_m, sigs_n):
        L, K, full, _ = self._aniso(sigs_n)
        phi_m = _f64(phi_m).reshape(self.G, self.ncell, K, 8)
        S = np.zeros_like(phi_m)
        lib().or_source_moments(ctypes.byref(self.c), K, _p(full), _p(phi_m), _p(S))
        return S

    def sweep_moments(self, S_m, sigs_n, groups=None):
        """flux moments [G,ncell,K,8] of one sweep from source moments S_m [G,ncell,K,8]
        (groups: a (begin, end) range; zero outside it)."""
        L, K, full, Yh = self._aniso(sigs_n)
        S_m = _f64(S_m).reshape(self.G, self.ncell, K, 8)
        phi = np.zeros_like(S_m)
        tal = np.zeros(4)
        g0, g1 = groups if groups else (0, self.G)
        if lib().or_sweep_moments(ctypes.byref(self.c), K, _p(Yh), _p(S_m), _p(phi), g0, g1, _p(tal)) != 0:
            raise ZeroDivisionError("zero pivot")
        return phi, tal

    def source_iterate_moments(self, sigs_n, tol, maxit, phi0=None):
        """Source iteration with Legendre scattering moments sigs_n [L+1][G][ncell]
        (row 0 is ignored: the problem's sigma_s); flux moments [G, ncell, K, 8]."""
        L, K, full, Yh = self._aniso(sigs_n)
        phi = (np.zeros((self.G, self.ncell, K, 8)) if phi0 is None
               else _f64(phi0).reshape(self.G, self.ncell, K, 8).copy())
        it = ctypes.c_int(0)
        cmax = ctypes.c_double(0.0)
        cmean = ctypes.c_double(0.0)
        tal = np.zeros(4)
        rc = lib().or_source_iterate_moments(ctypes.byref(self.c), K, _p(full), _p(Yh), tol, maxit, _p(phi),
                                             ctypes.byref(it), ctypes.byref(cmax), ctypes.byref(cmean), _p(tal))
        if rc < 0:
            raise ZeroDivisionError("zero pivot")
        return dict(phi=phi, iters=it.value, change_max=cmax.value, change_mean=cmean.value, tallies=tal,
                    converged=(rc == 0))

    def source(self, phi):
        S = np.zeros((self.G, self.ncell, 8))
        lib().or_source(ctypes.byref(self.c), _p(_f64(phi).reshape(self.G, self.ncell, 8)), _p(S))
        return S

    def source_iterate(self, tol, maxit, phi0=None):
        """Source iteration; returns dict(phi, iters, change_max, change_mean, tallies, converged)."""
        phi = np.zeros((self.G, self.ncell, 8)) if phi0 is None else _f64(phi0).reshape(self.G, self.ncell, 8).copy()
        it = ctypes.c_int(0)
        cmax = ctypes.c_double(0.0)
        cmean = ctypes.c_double(0.0)
        tal = np.zeros(4)
        rc = lib().or_source_iterate(ctypes.byref(self.c), tol, maxit, _p(phi), ctypes.byref(it),
                                     ctypes.byref(cmax), ctypes.byref(cmean), _p(tal))
        if rc < 0:
            raise ZeroDivisionError("zero pivot")
        return dict(phi=phi, iters=it.value, change_max=cmax.value, change_mean=cmean.value,
                    tallies=tal, converged=(rc == 0))

    def adjoint(self, phi, resp, tol=1e-13, maxit=2000):
        """Discrete adjoint of R = resp . phi at the converged forward flux phi:
        dict(Lam [G,ncell,8] = sum_d lambda_d, grad_sigt, grad_sigs, grad_q [G,ncell], iters)."""
        phi = _f64(phi).reshape(self.G, self.ncell, 8)
        resp = _f64(resp).reshape(self.G, self.ncell, 8)
        Lam = np.zeros((self.G, self.ncell, 8))
        gt = np.zeros((self.G, self.ncell)); gs = np.zeros((self.G, self.ncell)); gq = np.zeros((self.G, self.ncell))
        it = ctypes.c_int(0)
        rc = lib().or_adjoint(ctypes.byref(self.c), _p(phi), _p(resp), tol, maxit, _p(Lam), _p(gt), _p(gs), _p(gq),
                              ctypes.byref(it))
        if rc < 0:
            raise ZeroDivisionError("zero pivot")
        return dict(Lam=Lam, grad_sigt=gt, grad_sigs=gs, grad_q=gq, iters=it.value, converged=(rc == 0))

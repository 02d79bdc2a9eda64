"""CPU-side checks of the C ABI: the library builds, loads and exports every entry
point include/sn.h declares; host-side validation rejects bad input before any
device work; the binding refuses to run without the library."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sn_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def libsn():
    from paper_1906_04017_gb300 import build
    return ctypes.CDLL(build.build())


def test_exports_every_declared_symbol(libsn):
    names = declared_symbols()
    assert "sn_setup" in names and "sn_sweep" in names
    for n in sorted(names):
        assert hasattr(libsn, n), n


def test_binding_covers_header():
    from paper_1906_04017_gb300 import sn
    assert declared_symbols() == set(sn.api_names())


def _setup_raw(mesh=(2, 2, 2, 1.0, 1.0, 1.0), order=4, G=1, sigt=1.0):
    from paper_1906_04017_gb300 import sn
    n = mesh[0] * mesh[1] * mesh[2]
    arrs = [np.full(G * n, sigt), np.zeros(G * n), np.zeros(G * n), np.eye(G).ravel(), np.zeros(6 * G)]
    xs = sn.XS(G, *[a.ctypes.data_as(sn._dp) for a in arrs])
    h = ctypes.c_void_p()
    st = sn.lib().sn_setup(ctypes.byref(h), ctypes.byref(sn.Mesh(*mesh)),
                           ctypes.byref(sn.Quadrature(order, 0, None, None)), ctypes.byref(xs), None, None)
    msg = sn.lib().sn_last_error(None)
    if st == 0:
        sn.lib().sn_destroy(h)
    return st, msg


@pytest.mark.parametrize("mesh,order,G,sigt", [
    ((0, 2, 2, 1.0, 1.0, 1.0), 4, 1, 1.0),
    ((2, 2, 2, -1.0, 1.0, 1.0), 4, 1, 1.0),
    ((2, 2, 2, 1.0, 1.0, 1.0), 5, 1, 1.0),
    ((2, 2, 2, 1.0, 1.0, 1.0), 16, 1, 1.0),
    ((2, 2, 2, 1.0, 1.0, 1.0), 4, 0, 1.0),
    ((2, 2, 2, 1.0, 1.0, 1.0), 4, 1, -0.5),
    ((2, 2, 2, 1.0, 1.0, 1.0), 4, 1, float("nan")),
    ((2048, 2, 2, 1.0, 1.0, 1.0), 4, 1, 1.0),
])
def test_setup_rejects_bad_input(mesh, order, G, sigt):
    from paper_1906_04017_gb300 import sn
    st, msg = _setup_raw(mesh, order, max(G, 1) if G else 1, sigt) if G else _setup_g0(mesh)
    assert st == sn.SN_EINVAL, (st, msg)
    assert msg


def _setup_g0(mesh):
    from paper_1906_04017_gb300 import sn
    xs = sn.XS(0, None, None, None, None, None)
    h = ctypes.c_void_p()
    st = sn.lib().sn_setup(ctypes.byref(h), ctypes.byref(sn.Mesh(*mesh)),
                           ctypes.byref(sn.Quadrature(4, 0, None, None)), ctypes.byref(xs), None, None)
    return st, sn.lib().sn_last_error(None)


def test_null_arguments():
    from paper_1906_04017_gb300 import sn
    L = sn.lib()
    assert L.sn_setup(None, None, None, None, None, None) == sn.SN_EINVAL
    assert L.sn_sweep(None, None, None, 0) == sn.SN_EINVAL
    assert L.sn_cell_solve_batch(None, None, None, -1, 0, None) == sn.SN_EINVAL
    assert L.sn_cell_solve_batch(None, None, None, 0, 0, None) == sn.SN_OK
    assert L.sn_cell_solve_batch(None, None, None, 4, sn.ANN, None) == sn.SN_EINVAL   # no handle, no network
    assert L.sn_status_string(sn.SN_ENAN) == b"non-finite flux"
    L.sn_destroy(None)


def test_no_gpu_is_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1906_04017_gb300 import sn
    st, msg = _setup_raw()
    assert st == sn.SN_ECUDA, (st, msg)


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_1906_04017_gb300 import sn
    monkeypatch.setattr(sn, "LIB_PATH", "/nonexistent/libsn_gb300.so")
    monkeypatch.setattr(sn, "_LIB", None)
    with pytest.raises(RuntimeError):
        sn.lib()


@pytest.mark.parametrize("case", ["targ_rows", "feat_width", "targ_width", "params_len", "grad_len", "loss_empty"])
def test_noalloc_wrapper_refuses_bad_sizes_before_launch(case, monkeypatch):
    """The allocation-free gradient's C entry point sees only pointers, so its
    binding checks every size first: a short target, gradient or parameter array
    would otherwise become an out-of-bounds access on the device.  Each bad size is
    refused with ValueError before the library is even loaded."""
    import torch
    from paper_1906_04017_gb300 import sn

    def no_launch():
        raise AssertionError("the library was reached")
    monkeypatch.setattr(sn, "lib", no_launch)
    n = 64
    t = {"params": torch.zeros(sn.NPARAM), "feat": torch.zeros(n, 27), "targ": torch.zeros(n, 8),
         "grad": torch.zeros(sn.NPARAM), "loss": torch.zeros(1, dtype=torch.float64)}
    bad = {"targ_rows": ("targ", torch.zeros(n - 1, 8)), "feat_width": ("feat", torch.zeros(n, 26)),
           "targ_width": ("targ", torch.zeros(n, 9)), "params_len": ("params", torch.zeros(sn.NPARAM - 1)),
           "grad_len": ("grad", torch.zeros(100)), "loss_empty": ("loss", torch.zeros(0, dtype=torch.float64))}
    k, v = bad[case]
    t[k] = v
    with pytest.raises(ValueError):
        sn.surrogate_grad_noalloc(t["params"], t["feat"], t["targ"], t["grad"], t["loss"])


def test_noalloc_wrapper_refuses_host_tensors(monkeypatch):
    """Right sizes, but host tensors: refused (TypeError) before the library is reached."""
    import torch
    from paper_1906_04017_gb300 import sn

    def no_launch():
        raise AssertionError("the library was reached")
    monkeypatch.setattr(sn, "lib", no_launch)
    with pytest.raises(TypeError):
        sn.surrogate_grad_noalloc(torch.zeros(sn.NPARAM), torch.zeros(8, 27), torch.zeros(8, 8),
                                  torch.zeros(sn.NPARAM), torch.zeros(1, dtype=torch.float64))


def _bare_problem(G=2, ncell=8, K=1):
    """A Problem with sizes but no handle: enough for the argument checks, which
    run before any stream or library call."""
    import torch
    from paper_1906_04017_gb300 import sn
    P = sn.Problem.__new__(sn.Problem)
    P.h = None
    P.G, P.ncell, P.K = G, ncell, K
    P.dtype, P.device, P.default_mode = torch.float32, 0, sn.GE32R
    return P


@pytest.mark.parametrize("call", ["sweep", "sweep_out", "source", "source_iterate", "response", "adjoint",
                                  "harvest"])
def test_problem_refuses_a_flux_of_the_wrong_shape(call):
    """The kernels index G x ncell x 8 values of every flux argument: a tensor one
    group short (or one cell short) is refused before any launch."""
    import torch
    P = _bare_problem()
    good = torch.zeros((2, 8, 8))
    for bad in (torch.zeros((1, 8, 8)), torch.zeros((2, 7, 8)), torch.zeros((16, 8))):
        run = {"sweep": lambda: P.sweep(bad), "sweep_out": lambda: P.sweep(good, phi=bad),
               "source": lambda: P.source(bad), "source_iterate": lambda: P.source_iterate(phi=bad),
               "response": lambda: P.response(good, bad), "adjoint": lambda: P.adjoint(bad, good),
               "harvest": lambda: P.harvest(bad, cap=4)}[call]
        with pytest.raises(ValueError):
            run()
    # the right shape gets past the shape check and stops at the device check
    with pytest.raises(TypeError, match="CUDA"):
        P.sweep(good)


def test_problem_flux_shape_follows_the_scattering_order():
    """Under anisotropic scattering sweeps take moments [G, K, ncell, 8]; the
    response and the adjoint stay isotropic [G, ncell, 8]."""
    import torch
    P = _bare_problem(K=4)
    with pytest.raises(ValueError):
        P.sweep(torch.zeros((2, 8, 8)))
    with pytest.raises(TypeError, match="CUDA"):
        P.sweep(torch.zeros((2, 4, 8, 8)))
    with pytest.raises(ValueError):
        P.response(torch.zeros((2, 4, 8, 8)), torch.zeros((2, 4, 8, 8)))
    with pytest.raises(ValueError):
        P.harvest(torch.zeros((2, 8, 8)), cap=-1)


@pytest.mark.parametrize("shapes", [((4, 27), (3, 8)), ((4, 27), (5, 8)), ((4, 27), (4, 7)), ((4, 26), (4, 8)),
                                    ((108,), (4, 8)), ((4, 27), (32,))])
def test_batch_wrappers_refuse_mismatched_rows(shapes):
    """An out with fewer rows than in27 would be written past its end: every batch
    entry point refuses it (and any other shape) before any library call."""
    import torch
    from paper_1906_04017_gb300 import sn
    in27, out = torch.zeros(shapes[0]), torch.zeros(shapes[1])
    P = _bare_problem()
    for run in (lambda: sn.cell_solve_batch(in27, out=out), lambda: sn.cell_solve_batch_f64(in27, out=out),
                lambda: P.surrogate_apply(in27, out=out), lambda: P.octnet_apply(in27, out=out)):
        with pytest.raises(ValueError):
            run()


@pytest.mark.parametrize("rows", [(16, 15), (16, 17), (12, 12)])
def test_octnet_wrappers_refuse_unequal_or_ragged_batches(rows):
    """Features and targets of the octant networks are 8 equal blocks of m rows: a
    target array with other rows than the features, or a row count that is not a
    multiple of 8, is refused before any library call."""
    import torch
    P = _bare_problem()
    feat, targ = torch.zeros((rows[0], 27)), torch.zeros((rows[1], 8))
    for run in (lambda: P.octnet_grad(feat, targ), lambda: P.octnet_fit(feat, targ, 1, 1e-3),
                lambda: P.octnet_eval(feat, targ), lambda: P.octnet_prune(feat, targ, 0, 0.0)):
        with pytest.raises(ValueError):
            run()


def test_weight_setters_refuse_wrong_sizes():
    """The C setters read a fixed number of host values: a shorter array is refused."""
    P = _bare_problem()
    with pytest.raises(ValueError):
        P.surrogate_set_weights(np.zeros(2311, dtype=np.float32))
    with pytest.raises(ValueError):
        P.octnet_set(np.zeros((8, 287), dtype=np.float32))
    with pytest.raises(ValueError):
        P.octnet_init(np.zeros((8, 25)), np.ones((8, 25)))

"""Pins of the surrogate-network oracle (Sec. 3, Eq. (15); Sec. 4, Eq. (19) and
the Adam optimiser): finite differences for the back-propagated gradient,
hand-computed loss values, Adam's closed-form first step, and the mirror
symmetry that lets one network serve every octant, checked against the
oracle's own physical-frame elimination."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1906_04017_gb300 import workloads as W


def smooth_batch(seed, n=6):
    """Random parameters and data with every residual and pre-activation away from
    the kinks of |.| and ReLU, so that central differences are exact to O(h^2)."""
    rng = np.random.default_rng(seed)
    for _ in range(1000):
        p = mlp.init_params(seed) * 2.0
        x = rng.uniform(-1, 1, (n, mlp.NIN))
        t = rng.uniform(-1, 1, (n, mlp.NOUT))
        o, a, _ = mlp.forward(p, x)
        d = t - o
        if np.abs(a).min() > 1e-3 and np.abs(d).min() > 1e-3 and np.abs(d.sum(1)).min() > 1e-3:
            return p, x, t
        seed += 1000
    raise RuntimeError("no smooth batch")


def test_gradient_matches_central_differences():
    p, x, t = smooth_batch(3)
    L, g = mlp.loss_grad(p, x, t)
    assert np.isclose(L, mlp.loss(p, x, t), rtol=1e-14)
    h = 1e-7
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss(p + e, x, t) - mlp.loss(p - e, x, t)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-9)


def test_loss_hand_values():
    """One sample, zero network (all outputs = b2 = 0): the loss is the mean |t| plus
    lambda |sum t| / (gamma_1 |sum t| + gamma_2)."""
    p = np.zeros(mlp.NPARAM)
    x = np.zeros((1, mlp.NIN))
    t = np.array([[1.0, -1.0, 0, 0, 0, 0, 0, 0]])
    assert mlp.loss(p, x, t) == pytest.approx(0.25)
    t = np.full((1, 8), 0.5)
    assert mlp.loss(p, x, t) == pytest.approx(0.5 + 0.2 * 4.0 / (10 * 4.0 + 0.01))
    # a perfect fit has zero loss
    W1, b1, W2, b2 = mlp.unpack(p)
    b2 = t[0].copy()
    assert mlp.loss(mlp.pack(W1, b1, W2, b2), x, t) == 0.0


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    opt = mlp.Adam(4, lr=0.01)
    p1 = opt.step(np.zeros(4), g)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_canonical_frame_commutes_with_elimination():
    """Mirroring a one-cell problem into the positive octant and solving it there
    gives the mirrored solution of the original problem (the DFEM system is
    symmetric under axis reflection)."""
    x = W.onecell_problems(3000, seed=11)
    psi = oracle.cell_solve(x)
    aom, h, sig, S, U, mask = mlp.canonical(x)
    xc = np.concatenate([aom, h, sig[:, None], S, U], 1)
    psic = oracle.cell_solve(xc)
    _, s, _ = mlp.features(x)
    assert np.allclose(mlp.targets(psi, x) * s[:, None], psic, rtol=1e-10, atol=1e-12)


def test_predict_is_octant_symmetric():
    p = mlp.init_params(5)
    x = W.onecell_problems(500, seed=2)
    x[:, 0:3] = np.abs(x[:, 0:3])
    out = mlp.predict(p, x)
    # flip Omega_x: reverse the node order along x in S, swap in-face order of y, z faces
    y = x.copy()
    y[:, 0] *= -1
    k = np.arange(8)
    y[:, 7:15] = x[:, 7:15][:, k ^ 1]
    t = np.arange(4)
    y[:, 19:23] = x[:, 19:23][:, t ^ 1]
    y[:, 23:27] = x[:, 23:27][:, t ^ 1]
    out2 = mlp.predict(p, y)
    assert np.allclose(out2, out[:, k ^ 1], rtol=1e-12, atol=1e-14)


def test_features_ranges_and_zero_scale():
    x = W.onecell_problems(2000, seed=4)
    x[:5, 7:27] = 0.0
    f, s, _ = mlp.features(x)
    assert np.all(s[:5] == 0) and np.all(f[:5, 7:] == 0)
    assert np.all(np.abs(f[:, 0:3]) <= 1.0)
    assert np.all((f[5:, 7:] >= 0) & (f[5:, 7:] <= 1.0))
    assert np.allclose(f[5:, 7:].max(axis=1), 1.0, rtol=1e-15)


def test_training_reduces_loss():
    x = W.onecell_problems(4096, seed=7)
    f, s, _ = mlp.features(x)
    t = mlp.targets(oracle.cell_solve(x), x)
    p0 = mlp.init_params(0)
    p1 = mlp.train(p0, f, t, steps=300, batch=256, lr=2e-3)
    assert mlp.loss(p1, f, t) < 0.5 * mlp.loss(p0, f, t)


def test_vanishing_input_scale_counts_as_zero():
    """An input scale at or below 1e-30 (a flux FP32 cannot hold) scales inputs and
    target by zero instead of producing an infinite 1/s."""
    x = W.onecell_problems(4, seed=2)
    x[:, 7:27] *= 1e-36
    feat, s, _ = mlp.features(x)
    assert np.all(np.isfinite(feat)) and np.all(feat[:, 7:27] == 0.0)
    assert np.all(mlp.targets(np.ones((4, 8)), x) == 0.0)


def bf16_ref(p, in27):
    """The numpy oracle with the BF16 path's rounding steps (shared with the GPU
    parity tests)."""
    from _parity import f32_roundtrip
    from test_gpu_surrogate import predict_bf16
    return predict_bf16(p, f32_roundtrip(in27))


@pytest.mark.parametrize("bf16", [False, True])
def test_c_and_numpy_evaluations_agree(bf16):
    """The C oracle's surrogate cell (used by the whole-mesh sweeps) equals the numpy
    oracle on every octant, with and without the BF16 rounding steps; an input scale
    at or below 1e-30 zeroes the flux features, so psi = s o stays of the order of s
    in both."""
    x = W.onecell_problems(3000, seed=5)
    x[:3, 7:27] *= 1e-36
    p = mlp.init_params(3)
    got = oracle.mlp_cell(p, x, bf16=bf16)
    want = bf16_ref(p, x) if bf16 else mlp.predict(p, x)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    assert np.all(np.isfinite(got)) and np.abs(got[:3]).max() < 1e-30
    assert len(np.unique(mlp.mirror_masks(x)[0] | (mlp.mirror_masks(x)[1] << 1) | (mlp.mirror_masks(x)[2] << 2))) == 8


@pytest.mark.parametrize("order, bf16", [(2, False), (4, True), (8, True)])
def test_c_network_sweep_matches_the_python_sweep(order, bf16):
    """The C oracle's sweep with the surrogate as cell solver against the pure-Python
    upwind sweep calling the numpy network (both FP64 sweeps)."""
    from _parity import network_sweep
    wl = W.random_small(3, 4, 2, order=order, G=2, seed=8, psi_inc=True)
    p = mlp.init_params(12) * 0.5
    S = np.random.default_rng(2).uniform(0.0, 1.0, (2, 24, 8))
    phi, _ = oracle.OracleProblem(wl).sweep(S, mlp=(p, bf16))
    ref = network_sweep(wl, S, (lambda z: bf16_ref(p, z)) if bf16 else (lambda z: mlp.predict(p, z)))
    assert np.abs(phi - ref).max() <= 1e-12 * np.abs(ref).max()


def test_c_gated_network_sweep_matches_the_python_sweep():
    """The residual gate in the C oracle's network sweep (keep the network's psi where
    ||b - A psi|| <= tau ||b|| for the cell's own system (14), else eliminate) against
    the pure-Python upwind sweep that applies the same test with numpy and solves the
    rejected cells with LAPACK: at a threshold that sends part of the cells to
    elimination the fluxes agree to round-off and the fallback counts are equal; tau
    = 0 gives the elimination sweep and a huge tau the ungated network sweep, bit for
    bit."""
    from _parity import network_sweep
    wl = W.random_small(3, 4, 2, order=4, G=2, seed=8, psi_inc=True)
    p = mlp.init_params(12) * 0.5
    S = np.random.default_rng(2).uniform(0.0, 1.0, (2, 24, 8))

    def gated(tau, record):
        def predict(x):
            psi = mlp.predict(p, x)
            A, b = oracle.assemble(x[0])
            r = np.linalg.norm(b - A @ psi[0]) / np.linalg.norm(b)
            record.append(r)
            return np.linalg.solve(A, b)[None] if r > tau else psi
        return predict

    first = []
    network_sweep(wl, S, gated(np.inf, first))
    tau = float(np.median(first))
    ratios = []
    ref = network_sweep(wl, S, gated(tau, ratios))
    rejected = int(sum(r > tau for r in ratios))
    assert 0.2 < rejected / len(ratios) < 0.8
    assert min(abs(r / tau - 1.0) for r in ratios) > 1e-9      # no decision at the threshold
    O = oracle.OracleProblem(wl)
    phi, _ = O.sweep(S, mlp=(p, False), gate=tau)
    assert O.last_fallbacks == rejected
    assert np.abs(phi - ref).max() <= 1e-11 * np.abs(ref).max()
    ge, _ = O.sweep(S)
    g0, _ = O.sweep(S, mlp=(p, False), gate=0.0)
    assert np.array_equal(g0, ge) and O.last_fallbacks == len(ratios)
    un, _ = O.sweep(S, mlp=(p, True))
    ginf, _ = O.sweep(S, mlp=(p, True), gate=1e300)
    assert np.array_equal(ginf, un) and O.last_fallbacks == 0


def test_bf16_rounding_is_nearest_even():
    """The rounding step itself: values exactly halfway between two BF16 numbers go
    to the even one, others to the nearest."""
    from test_gpu_surrogate import bf16
    one = 1.0
    ulp = 2.0 ** -7                      # BF16 spacing in [1, 2)
    v = np.array([one + ulp / 2, one + 1.5 * ulp, one + 0.26 * ulp, one + 0.74 * ulp, -3.0])
    assert list(bf16(v)) == [one, one + 2 * ulp, one, one + ulp, -3.0]

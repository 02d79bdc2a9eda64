"""Pins of the FP64 oracle of the paper's per-octant networks (oracle.octant_net,
Sec. 3 Eqs. (15)-(18), Sec. 4 Eq. (19) and the connection dropping of Sec. 3)
against closed forms, limits, finite differences and brute force -- nothing here
re-types the oracle's own formulas."""
import numpy as np
import pytest

import oracle
from oracle import octant_net as on
from paper_1906_04017_gb300 import workloads as W
from _parity import network_sweep

LO, HI = W.octant_net_ranges()


def nets(seed, bias=0.3):
    rng = np.random.default_rng(seed)
    P = np.stack([on.glorot_init(seed * 8 + o) for o in range(8)])
    P[:, on.connection_mask() == 0] = rng.uniform(-bias, bias, (8, on.NPARAM - on.NCONN))
    return P


def test_input_scaling_closed_form():
    """Eq. (16) with alpha = 0.27 on [0, 10]: 5 -> (5 - 1.35) / 10, the ends map to
    -0.135 and 0.865 (a unit-wide interval), and the mirrored angle range [-1, 0]
    sends -0.5 to -0.365."""
    x = on.scale(np.array([0.0, 5.0, 10.0]), 0.0, 10.0)
    assert np.allclose(x, [-0.135, 0.365, 0.865], rtol=0, atol=1e-15)
    assert on.scale(np.array([-0.5]), -1.0, 0.0)[0] == pytest.approx(-0.365, abs=1e-15)


@pytest.mark.parametrize("j, name", [(0, "psi_x[0]"), (7, "psi_y[3]"), (11, "psi_z[3]"), (12, "mu"),
                                     (13, "eta"), (14, "q[0]"), (21, "q[7]"), (22, "sigma_t"), (25, "dz")])
def test_each_input_reaches_the_network_in_the_listed_order(j, name):
    """A network that reads input j alone through a near-linear tanh returns the
    scaled value of the quantity the list of Sec. 3 puts at position j."""
    x27 = W.octant_problems(4, seed=3)
    want = {"psi_x[0]": x27[:, 15], "psi_y[3]": x27[:, 22], "psi_z[3]": x27[:, 26], "mu": x27[:, 0],
            "eta": x27[:, 1], "q[0]": x27[:, 7], "q[7]": x27[:, 14], "sigma_t": x27[:, 6], "dz": x27[:, 5]}[name]
    eps = 1e-5
    P = np.zeros((8, on.NPARAM))
    W1, b1, W2, b2 = [np.zeros_like(a) for a in on.unpack(P[0])]
    W1[0, j] = eps
    W2[0, 0] = 1.0 / eps
    b2[0] = 50.0          # stay on the linear branch of Eq. (18)
    P[:] = on.pack(W1, b1, W2, b2)
    got = on.predict(P, x27, LO, HI)[:, 0] - 50.0
    o = on.octant_of(x27)
    lo, hi = LO[o, j], HI[o, j]
    ref = (want - 0.27 * 0.5 * (lo + hi)) / np.abs(hi - lo)
    assert np.allclose(got, ref, rtol=0, atol=1e-8)


def test_small_weights_give_the_affine_map():
    """|tanh(a) - a| <= |a|^3 / 3: with W1, b1 of size 1e-4 and outputs on the
    linear branch the network equals W2 (W1 x + b1) + b2 within that bound."""
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (32, on.NIN))
    W1 = rng.uniform(-1, 1, (on.NHID, on.NIN)) * 1e-4
    b1 = rng.uniform(-1, 1, on.NHID) * 1e-4
    W2 = rng.uniform(-1, 1, (on.NOUT, on.NHID))
    b2 = np.full(on.NOUT, 3.0)
    y = on.forward(on.pack(W1, b1, W2, b2), x, np.ones(32))[0]
    a = x @ W1.T + b1
    bound = (np.abs(a) ** 3 / 3.0) @ np.abs(W2).T + 1e-14
    assert np.all(np.abs(y - (a @ W2.T + b2)) <= bound)


def test_saturated_hidden_units_are_signs():
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (16, on.NIN))
    W1 = rng.uniform(-1, 1, (on.NHID, on.NIN)) * 1e4
    W2 = rng.uniform(-1, 1, (on.NOUT, on.NHID))
    b2 = np.full(on.NOUT, 10.0)
    y = on.forward(on.pack(W1, np.zeros(on.NHID), W2, b2), x, np.ones(16))[0]
    assert np.allclose(y, np.sign(x @ W1.T) @ W2.T + b2, rtol=0, atol=1e-12)


def test_negative_outputs_are_bounded_by_beta():
    """Eq. (18): far below zero the output tends to -beta, beta = 0.1 max |psi_inc|;
    at z = -1 it is beta (1/e - 1)."""
    x27 = W.octant_problems(8, seed=6)
    P = np.zeros((8, on.NPARAM))
    P[:, -on.NOUT:] = -60.0
    y = on.predict(P, x27, LO, HI)
    beta = 0.1 * np.abs(x27[:, 15:27]).max(axis=1)
    assert np.allclose(y, -beta[:, None], rtol=1e-15, atol=0)
    P[:, -on.NOUT:] = -1.0
    y = on.predict(P, x27, LO, HI)
    assert np.allclose(y, (beta * (np.exp(-1.0) - 1.0))[:, None], rtol=1e-14, atol=0)


def test_each_octant_uses_its_own_network():
    """Constant networks psi = o + 1: the rows of octant o (bit 0 mu < 0, bit 1
    eta < 0, bit 2 xi < 0) get o + 1, in the numpy and the C evaluation."""
    x27 = W.octant_problems(5, seed=7)
    P = np.zeros((8, on.NPARAM))
    for o in range(8):
        P[o, -on.NOUT:] = o + 1.0
    want = np.repeat(np.arange(1.0, 9.0), 5)[:, None] * np.ones(8)
    assert np.array_equal(on.predict(P, x27, LO, HI), want)
    assert np.array_equal(oracle.octnet_cell(P, LO, HI, x27), want)
    om = x27[:, 0:3]
    assert np.array_equal(on.octant_of(x27), (om[:, 0] < 0) + 2 * (om[:, 1] < 0) + 4 * (om[:, 2] < 0))


def test_c_and_numpy_evaluations_agree():
    x27 = W.octant_problems(64, seed=8)
    P = nets(1)
    assert np.abs(on.predict(P, x27, LO, HI) - oracle.octnet_cell(P, LO, HI, x27)).max() < 1e-13


def labelled(m, seed, o=0):
    x27 = W.octant_problems(m, seed=seed)[o * m:(o + 1) * m]
    x, b, _ = on.features(x27, LO, HI)
    return x, b, oracle.cell_solve(x27)


def test_gradient_matches_central_differences():
    """Back-propagation against FP64 central differences of Eq. (19), step 1e-6,
    on a batch of elimination-labelled one-cell problems."""
    x, b, t = labelled(48, seed=9, o=5)
    p = nets(2)[5]
    L, g = on.loss_grad(p, x, b, t)
    assert L == pytest.approx(on.loss(p, x, b, t), rel=1e-15)
    h = 1e-6
    fd = np.empty(on.NPARAM)
    for k in range(on.NPARAM):
        e = np.zeros(on.NPARAM)
        e[k] = h
        fd[k] = (on.loss(p + e, x, b, t) - on.loss(p - e, x, b, t)) / (2 * h)
    assert np.abs(fd - g).max() < 1e-6 * max(1.0, np.abs(g).max())


def test_gradient_on_the_negative_branch():
    """The ELU branch (Eq. (18) below zero) and the regulariser's sign: outputs
    pushed negative by b2, checked against central differences."""
    x, b, t = labelled(32, seed=10, o=2)
    p = nets(3)[2]
    p[-on.NOUT:] -= 1.5
    _, g = on.loss_grad(p, x, b, t)
    h = 1e-6
    for k in list(range(on.NPARAM - 72, on.NPARAM)) + [0, 25, 100, 207]:
        e = np.zeros(on.NPARAM)
        e[k] = h
        fd = (on.loss(p + e, x, b, t) - on.loss(p - e, x, b, t)) / (2 * h)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, np.abs(g).max())


def test_training_fits_a_teacher_network():
    """Targets made by a network of the same shape: full-batch Adam from another
    start lowers the loss of Eq. (19) tenfold."""
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, (256, on.NIN))
    b = rng.uniform(0.01, 0.1, 256)
    teacher = on.glorot_init(100)
    teacher[on.connection_mask() == 0] = rng.uniform(0.2, 0.5, on.NPARAM - on.NCONN)
    t = on.forward(teacher, x, b)[0]
    p0 = on.glorot_init(101)
    p1 = on.train(p0, x, b, t, steps=400, lr=1e-2)
    assert on.loss(p1, x, b, t) < 0.1 * on.loss(p0, x, b, t)


def test_masked_training_keeps_dropped_connections_at_zero():
    x, b, t = labelled(64, seed=12)
    p = nets(4)[0]
    mask = np.ones(on.NPARAM)
    mask[[3, 40, 230]] = 0.0
    q = on.train(p, x, b, t, steps=20, lr=1e-3, mask=mask)
    assert np.all(q[[3, 40, 230]] == 0.0)
    assert np.any(q[mask > 0] != p[mask > 0])


def test_pure_magnitude_pruning_drops_the_smallest_connections():
    """With no retraining and no error limit the procedure of Sec. 3 removes the k
    connections of smallest magnitude, never a bias."""
    x, b, t = labelled(32, seed=13)
    p = nets(5)[0]
    k = 37
    q, mask, dropped, _, _ = on.prune(p, x, b, t, retrain_steps=0, lr=0.0, tol=np.inf, max_drops=k)
    conn = np.flatnonzero(on.connection_mask() > 0)
    smallest = conn[np.argsort(np.abs(p[conn]), kind="stable")[:k]]
    assert sorted(dropped) == sorted(smallest.tolist())
    assert np.all(q[dropped] == 0.0) and np.all(mask[dropped] == 0.0)
    assert np.sum(mask == 0) == k


def test_pruning_stops_at_the_error_limit():
    """The kept network's training MSE is within (1 + tol) of the fully connected
    one's, and the next drop of the same procedure would exceed it."""
    x, b, t = labelled(128, seed=14)
    p = on.train(nets(6)[0], x, b, t, steps=300, lr=3e-3)
    tol = 0.05
    q, mask, dropped, mse0, mse = on.prune(p, x, b, t, retrain_steps=10, lr=1e-3, tol=tol, max_drops=60)
    assert mse <= (1 + tol) * mse0
    assert on.errors(q, x, b, t)[1] == pytest.approx(mse, rel=1e-12)
    if len(dropped) < 60:
        conn = np.flatnonzero((on.connection_mask() > 0) & (mask > 0))
        k = conn[np.argmin(np.abs(q[conn]))]
        m2 = mask.copy()
        m2[k] = 0.0
        assert on.errors(on.train(q, x, b, t, 10, 1e-3, m2), x, b, t)[1] > (1 + tol) * mse0


def test_network_sweep_in_c_matches_the_python_sweep():
    """The C oracle's sweep with the octant networks as cell solver against the
    pure-Python upwind sweep calling the numpy networks (3 x 2 x 2 mesh, LQ_4,
    two groups, inflow on every face)."""
    wl = W.random_small(3, 2, 2, order=4, G=2, seed=15, psi_inc=True)
    P = nets(7, bias=0.1)
    rng = np.random.default_rng(16)
    S = rng.uniform(0.0, 1.0, (2, 12, 8))
    got, _ = oracle.OracleProblem(wl).sweep(S, octnet=(P, LO, HI))
    ref = network_sweep(wl, S, lambda x: on.predict(P, x, LO, HI))
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()

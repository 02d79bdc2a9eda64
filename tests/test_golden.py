"""Pins against values the paper prints (fixtures under tests/golden/, each entry with
its citation): the parameters of Problems 1-4 (Sec. 4 tables) and their stated optical
sizes, the network's dimensions and constants (Secs. 3-4, Eqs. (15)-(19)), the error
metric's offset (Eq. (20)), and the bench's table of the paper's own results."""
import json
import math
import os
import sys

import numpy as np
import pytest
import torch

import oracle
from oracle import octant_net as ON
from paper_1906_04017_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
import bench  # noqa: E402


def golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


PROBLEMS = golden("paper_sec4_problems.json")
NETWORK = golden("paper_sec3_network.json")


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_paper_problems_match_the_printed_tables(k):
    """Cross sections, source, inflow faces, lengths and meshes of Problem k."""
    t = PROBLEMS["problems"][str(k)]
    for n in sorted(set(t["cells_per_axis"])):
        wl = W.paper_problem(k, n=n, order=2)
        assert (wl["nx"], wl["ny"], wl["nz"]) == (n, n, n)
        assert [wl["lx"], wl["ly"], wl["lz"]] == t["lengths"]
        assert np.all(wl["sigt"] == t["sigma_t"])
        assert np.all(wl["sigs"] == t["sigma_s"])
        assert np.all(wl["q"] == t["q"])
        # incident flux on the x-, y-, z- faces (faces 0, 2, 4), vacuum opposite
        assert list(wl["psi_inc"][0, [0, 2, 4]]) == t["psi_inc"]
        assert np.all(wl["psi_inc"][0, [1, 3, 5]] == 0.0)
    # the order study of Sec. 4 runs 100^3 cells: cell size 0.1 cm on the 10 cm cube
    wl = W.paper_problem(k, n=100, order=8)
    assert wl["lx"] / wl["nx"] == pytest.approx(0.1)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_printed_optical_sizes(k):
    """The domain spans the printed range of mean free paths: sigma_t times an edge at
    the low end, times the cube's diagonal at the high end (Problem 4 prints 170 for
    the diagonal's 173.2; the tolerance covers that rounding)."""
    t = PROBLEMS["problems"][str(k)]
    wl = W.paper_problem(k, n=10, order=2)
    sig = float(wl["sigt"][0, 0])
    edge = sig * wl["lx"]
    diag = sig * math.sqrt(wl["lx"] ** 2 + wl["ly"] ** 2 + wl["lz"] ** 2)
    lo, hi = t["mean_free_paths"]
    assert edge == pytest.approx(lo, rel=1e-12)
    assert diag == pytest.approx(hi, rel=0.025)


def test_network_dimensions_and_constants():
    """The per-octant network of the oracle is the printed one: 26 inputs, one hidden
    layer of 8, 8 outputs, alpha = 0.27, and the regulariser lambda = 0.2,
    gamma_1 = 10, gamma_2 = 0.01."""
    assert ON.NIN == NETWORK["inputs"]["value"]
    assert ON.NOUT == NETWORK["outputs"]["value"]
    assert NETWORK["hidden_layers"]["value"] == 1
    assert ON.NHID == NETWORK["hidden_neurons"]["value"]
    assert ON.ALPHA == NETWORK["alpha"]["value"]
    assert (ON.LAMBDA, ON.GAMMA1, ON.GAMMA2) == (
        NETWORK["loss"]["lambda"], NETWORK["loss"]["gamma_1"], NETWORK["loss"]["gamma_2"])
    # one weight matrix and one bias per layer
    assert ON.NPARAM == ON.NIN * ON.NHID + ON.NHID + ON.NHID * ON.NOUT + ON.NOUT
    p = ON.glorot_init(0)
    W1, b1, W2, b2 = ON.unpack(p)
    assert W1.shape == (ON.NHID, ON.NIN) and W2.shape == (ON.NOUT, ON.NHID)


def test_loss_regulariser_constants_enter_the_loss():
    """One hand-computed row of Eq. (19): targets psi, prediction psi + e at a single
    output; the loss is |e| / 8 + lambda |e| / (gamma_1 |sum psi| + gamma_2)."""
    rng = np.random.default_rng(1)
    feats = rng.uniform(0, 1, (1, ON.NIN))
    beta = np.array([0.1])
    p = ON.glorot_init(2)
    pred = ON.forward(p, feats, beta)[0]
    tgt = pred.copy()
    e = 0.3
    tgt[0, 2] -= e
    lam, g1, g2 = NETWORK["loss"]["lambda"], NETWORK["loss"]["gamma_1"], NETWORK["loss"]["gamma_2"]
    want = e / 8 + lam * e / (g1 * abs(tgt.sum()) + g2)
    assert ON.loss(p, feats, beta, tgt) == pytest.approx(want, rel=1e-12)


def test_training_defaults_follow_the_paper():
    """The bench trains the per-octant networks on 9e4 problems per octant (10% more for
    testing) for 5e4 Adam epochs at a learning rate inside the printed range."""
    import inspect
    d = {k: v.default for k, v in inspect.signature(bench.octnet_train).parameters.items()}
    assert d["m_train"] == NETWORK["training_set"]["value"]
    assert d["m_train"] + d["m_test"] == NETWORK["dataset_problems"]["value"]
    assert d["m_train"] / (d["m_train"] + d["m_test"]) == NETWORK["dataset_problems"]["train_fraction"]
    assert d["epochs"] == NETWORK["adam"]["epochs"]
    lo, hi = NETWORK["adam"]["lr_range"]
    assert lo <= d["lr"] <= hi


def test_error_metric_offset():
    """Eq. (20) with m = 1e-8: cells whose flux is zero in both solutions add nothing,
    the others add |phi - phi_ANN| / (|phi| + m); cell values are the means of the
    eight nodes."""
    m = PROBLEMS["error_offset_m"]["value"]
    ref = torch.zeros(1, 4, 8, dtype=torch.float64)
    ref[0, 0] = 2.0
    ref[0, 1] = 1e-8
    phi = ref.clone()
    phi[0, 0] = 1.5
    phi[0, 2] = 1e-6
    want = (0.5 / (2.0 + m) + 0.0 + 1e-6 / m + 0.0) / 4
    assert bench.eps_p(phi, ref) == pytest.approx(want, rel=1e-12)


def test_paper_reported_results_table():
    """The bench's paper column covers every case of the Sec. 4 tables it runs."""
    for k in (1, 2, 3, 4):
        for o in (2, 4, 6, 8):
            r = bench.paper_reported(k, 100, o)
            assert r is not None and 0.0 < r["eps_P_pct"] < 3.0
        for n in (10, 25, 50):
            assert bench.paper_reported(k, n, 8) is not None
    assert bench.paper_reported(1, 100, 8) == {"eps_P_pct": 1.59, "time_reduction_pct": 68.4}
    p4 = bench.paper_reported(4, 10, 8)
    assert (p4["ge_iters"], p4["ann_iters"]) == (15, 9)
    assert bench.paper_reported(1, 100, 12) is None
    assert bench.paper_reported(2, 30, 8) is None


def octant0_error(n, order):
    """Max over the nodes and the first-octant directions of |psi - exp(-sigma_t s)| in
    Problem 2, s the distance back along -Omega to the first of the three inflow planes
    (every such ray leaves through an inflow face, so the transport solution is exactly
    that exponential), and the largest attenuation 1 - exp(-sigma_t s) itself."""
    wl = W.paper_problem(2, n=n, order=order)
    P = oracle.OracleProblem(wl)
    om, _ = oracle.lqn(order)
    h = wl["lx"] / n
    sig = float(wl["sigt"][0, 0])
    i, j, k = W.cell_ijk(wl)
    err = dev = 0.0
    for d in np.flatnonzero((om > 0).all(axis=1)):
        psi, _ = P.sweep_dir(int(d), 0, np.zeros((P.ncell, 8)))
        for node in range(8):
            x = np.stack([(i + (node & 1)) * h, (j + ((node >> 1) & 1)) * h, (k + (node >> 2)) * h], axis=1)
            exact = np.exp(-sig * (x / om[d]).min(axis=1))
            err = max(err, float(np.abs(psi[:, node] - exact).max()))
            dev = max(dev, float(np.abs(1.0 - exact).max()))
    return err, dev


@pytest.mark.parametrize("order", [2, 8])
def test_problem2_attenuation_matches_the_transport_solution(order):
    """Problem 2 is a hundredth of a mean free path thin: the oracle's flux follows
    the exponential attenuation of the transport equation to well under a tenth of the
    attenuation itself (a dropped or sign-flipped collision term would miss by all of
    it), and the gap closes as the mesh is refined."""
    e10, dev = octant0_error(10, order)
    e20, _ = octant0_error(20, order)
    assert dev > 0.01
    assert e10 < 0.1 * dev
    assert e20 < 0.75 * e10

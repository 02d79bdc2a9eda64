"""GPU parity of the surrogate network (Sec. 3, Eq. (15); Sec. 4, Eq. (19), Adam)
against the FP64 oracle (oracle.mlp), through the C ABI: input construction and
elimination labels, the back-propagated gradient, Adam steps, and the tcgen05
BF16 inference with and without the residual gate."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_1906_04017_gb300 import workloads as W
from _parity import f32_roundtrip, network_sweep

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round FP32 values to BF16 (nearest, ties to even) and back, as the tensor cores see them."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def predict_bf16(p, in27):
    """The oracle's network evaluated with the rounding steps of the BF16 path:
    inputs, weights and hidden activations rounded to BF16, FP64 sums, FP32 biases."""
    W1, b1, W2, b2 = mlp.unpack(np.asarray(p, dtype=np.float32).astype(np.float64))
    x, s, mask = mlp.features(in27)
    x = bf16(x.astype(np.float32))
    h = np.maximum(x @ bf16(W1).T + b1, 0.0)
    h = bf16(h.astype(np.float32))
    o = h @ bf16(W2).T + b2
    k = np.arange(8)
    return np.take_along_axis(o * s[:, None], k[None, :] ^ mask[:, None], 1)


@pytest.fixture(scope="module")
def handle(sn):
    wl = W.random_small(2, 2, 2, order=2, G=1)
    P = sn.Problem(wl)
    yield P
    P.close()


def cuda(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def test_prepare_matches_oracle(sn):
    x = W.onecell_problems(50001, seed=21).astype(np.float32).astype(np.float64)
    feat, targ = sn.surrogate_prepare(cuda(x))
    f_ref, s, _ = mlp.features(x)
    t_ref = mlp.targets(oracle.cell_solve(x), x)
    assert np.abs(feat.cpu().numpy() - f_ref).max() < 2e-6
    t = targ.cpu().numpy()
    scale = np.maximum(np.abs(t_ref).max(axis=1), 1e-30)
    assert (np.abs(t - t_ref).max(axis=1) / scale).max() < 1e-5


def test_no_network_is_a_state_error(sn):
    wl = W.random_small(2, 2, 2, order=2, G=1)
    P = sn.Problem(wl)
    with pytest.raises(sn.SnError) as e:
        P.surrogate_apply(cuda(W.onecell_problems(4)))
    P.close()
    assert e.value.status == sn.SN_ESTATE


def clean_batch(n, seed, p):
    """Rows whose residuals and pre-activations stay away from the kinks of |.| and
    ReLU, so FP32 and FP64 agree on every sign in the sub-gradient."""
    x = W.onecell_problems(4 * n, seed=seed)
    f, _, _ = mlp.features(x)
    t = mlp.targets(oracle.cell_solve(x), x)
    f = f.astype(np.float32).astype(np.float64)
    t = t.astype(np.float32).astype(np.float64)
    o, a, _ = mlp.forward(p, f)
    d = t - o
    ok = (np.abs(a).min(1) > 1e-4) & (np.abs(d).min(1) > 1e-4) & (np.abs(d.sum(1)) > 1e-4)
    return f[ok][:n], t[ok][:n]


def test_gradient_matches_oracle(handle):
    p = mlp.init_params(3).astype(np.float32).astype(np.float64)
    f, t = clean_batch(3000, 5, p)
    handle.surrogate_set_weights(p)
    loss, g = handle.surrogate_grad(cuda(f), cuda(t))
    L, gref = mlp.loss_grad(p, f, t)
    assert abs(loss - L) < 1e-5 * L
    assert np.abs(g - gref).max() < 2e-5 * np.abs(gref).max()


def test_adam_steps_match_oracle(handle):
    p = mlp.init_params(4).astype(np.float32).astype(np.float64)
    f, t = clean_batch(2048, 9, p)
    handle.surrogate_set_weights(p)
    handle.surrogate_fit(cuda(f), cuda(t), steps=3, batch=512, lr=1e-3)
    got = handle.surrogate_weights().astype(np.float64)
    ref = mlp.train(p, f, t, steps=3, batch=512, lr=1e-3)
    # Adam's early steps move each weight by about lr * sign(gradient): compare the
    # weights whose gradient is not vanishingly small (a sign decided by round-off
    # there is not a defect)
    _, g0 = mlp.loss_grad(p, f[:512], t[:512])
    sel = np.abs(g0) > 1e-3 * np.abs(g0).max()
    assert sel.mean() > 0.8
    assert np.abs(got - ref)[sel].max() < 2e-6


def test_tensor_core_inference(handle):
    x = W.onecell_problems(100003, seed=31)
    x[:7, 7:27] = 0.0                          # zero input scale: psi = 0
    x32 = x.astype(np.float32)
    xd = x32.astype(np.float64)
    p = mlp.init_params(6)
    handle.surrogate_set_weights(p)
    psi, nfb = handle.surrogate_apply(cuda(x32), gated=False)
    psi = psi.cpu().numpy().astype(np.float64)
    assert nfb == 0
    assert np.all(psi[:7] == 0.0)
    ref = predict_bf16(p, xd)
    err = (np.abs(psi[7:] - ref[7:]) / np.abs(ref).max(axis=1)[7:, None]).max(axis=1)
    # the FP32 inputs and hidden sums can land on the other side of a BF16 rounding
    # boundary than the FP64 emulation (one BF16 ulp, 2^-8 relative, in one value):
    # nearly every row agrees to accumulation round-off, none by more than such flips
    assert np.percentile(err, 99.0) < 1e-4
    assert err.max() < 3e-2
    # and against the exact FP64 network: the BF16 rounding bound
    exact = mlp.predict(np.asarray(p, dtype=np.float32).astype(np.float64), xd)
    assert (np.abs(psi[7:] - exact[7:]) / np.abs(exact).max(axis=1)[7:, None]).max() < 5e-2


@pytest.mark.parametrize("n", [1, 128, 1000])
def test_gate_extremes(sn, handle, n):
    """tau = 0 rejects every prediction, so the result is the elimination's; a huge
    tau accepts every one, so the result is the network's."""
    x = cuda(W.onecell_problems(n, seed=n).astype(np.float32))
    handle.surrogate_set_weights(mlp.init_params(7))
    handle.surrogate_set_gate(0.0)
    psi, nfb = handle.surrogate_apply(x, gated=True)
    ge = sn.cell_solve_batch(x, sn.GE32R)
    assert nfb == n
    assert torch.allclose(psi, ge, rtol=1e-6, atol=1e-7)
    handle.surrogate_set_gate(1e30)
    psi2, nfb2 = handle.surrogate_apply(x, gated=True)
    psi3, _ = handle.surrogate_apply(x, gated=False)
    assert nfb2 == 0 and torch.equal(psi2, psi3)
    handle.surrogate_set_gate(1e-2)


def test_training_reduces_error(handle):
    x = cuda(W.onecell_problems(1 << 16, seed=41).astype(np.float32))
    tr, te = handle.surrogate_train(x, n_test=4096, steps=0, batch=4096, lr=1e-3, seed=1)
    tr2, te2 = handle.surrogate_train(x, n_test=4096, steps=600, batch=4096, lr=2e-3, seed=1)
    assert tr2 < 0.5 * tr and te2 < 0.5 * te


@pytest.mark.parametrize("order", [2, 4, 8, 12])
def test_ann_sweep_matches_oracle_network_sweep(sn, order):
    """The tensor-core surrogate sweep against the oracle's network swept in Python,
    for 1, 3, 10 and 21 directions per octant (128 down to 6 keys a tile)."""
    wl = W.random_small(3, 4, 2, order=order, G=2, seed=8, psi_inc=True)
    P = sn.Problem(wl)
    p = mlp.init_params(12) * 0.5
    P.surrogate_set_weights(p)
    rng = np.random.default_rng(2)
    S = rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32)
    phi = P.sweep(cuda(S), mode=sn.ANN).cpu().numpy()
    P.close()
    p64 = np.asarray(p, np.float32).astype(np.float64)
    ref = network_sweep(wl, S.astype(np.float64), lambda x: predict_bf16(p64, f32_roundtrip(x)))
    err = np.abs(phi - ref).max() / np.abs(ref).max()
    assert err < 2e-2
    exact = network_sweep(wl, S.astype(np.float64), lambda x: mlp.predict(p64, f32_roundtrip(x)))
    assert np.abs(phi - exact).max() / np.abs(exact).max() < 1e-1


def test_ann_sweep_gate_zero_is_elimination(sn):
    """tau = 0: every cell fails the gate, so the gated surrogate sweep is the
    elimination sweep, and every solve is counted as a fallback."""
    wl = W.random_small(6, 5, 7, order=6, G=3, seed=5, psi_inc=True)
    P = sn.Problem(wl)
    P.surrogate_set_weights(mlp.init_params(13))
    P.surrogate_set_gate(0.0)
    rng = np.random.default_rng(3)
    S = cuda(rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32))
    ann = P.sweep(S, mode=sn.ANN_GATED)
    fb, to = P.surrogate_stats()
    ge = P.sweep(S, mode=sn.GE32R)
    P.close()
    assert to == 0 and fb == P.solves_per_sweep
    assert torch.allclose(ann, ge, rtol=1e-6, atol=1e-7 * ge.abs().max().item())


def test_graph_replays_follow_gate_changes(sn):
    """Source-iteration graphs bake the gate threshold and the packed weights into
    their kernel arguments; changing either must re-capture them: with tau = 0 after
    a run at tau = 1e30 the gated iteration is the elimination iteration again."""
    wl = W.random_small(5, 6, 4, order=4, G=2, seed=6, psi_inc=True)
    P = sn.Problem(wl)
    P.surrogate_set_weights(mlp.init_params(14))
    P.surrogate_set_gate(1e30)
    P.source_iterate(tol=0.0, max_it=3, mode=sn.ANN_GATED, use_graph=True, allow_noconv=True)
    P.surrogate_set_gate(0.0)
    a = P.source_iterate(tol=0.0, max_it=3, mode=sn.ANN_GATED, use_graph=True, allow_noconv=True)["phi"]
    b = P.source_iterate(tol=0.0, max_it=3, mode=sn.GE32R, use_graph=True, allow_noconv=True)["phi"]
    P.close()
    assert torch.allclose(a, b, rtol=1e-6, atol=1e-7 * b.abs().max().item())


def test_harvest_returns_the_sweeps_one_cell_problems(sn):
    """At full rate the harvesting sweep writes every solve of the sweep as a one-cell
    problem in the positive-octant frame: directions from the first octant of the
    quadrature, the mesh spacing, the cell's sigma_t, inflow psi_inc on boundary
    faces; and solving them again reproduces the same elimination."""
    wl = W.random_small(4, 3, 5, order=4, G=2, seed=2, psi_inc=True)
    P = sn.Problem(wl)
    rng = np.random.default_rng(4)
    S = cuda(rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32))
    x = P.harvest(S, cap=P.solves_per_sweep, seed=1).cpu().numpy().astype(np.float64)
    assert x.shape[0] >= P.solves_per_sweep - 1
    om, _ = oracle.lqn(4)
    first = np.round(om[:3], 6)
    assert all(any(np.allclose(r, f, atol=1e-6) for f in first) for r in x[::97, 0:3])
    assert np.allclose(x[:, 3:6], [wl["lx"] / 4, wl["ly"] / 3, wl["lz"] / 5], rtol=1e-6)
    sig_set = np.unique(wl["sigt"].astype(np.float32).astype(np.float64))
    near = np.abs(x[:, 6][:, None] - sig_set[None, :]).min(axis=1)
    assert (near <= 1e-7 * x[:, 6]).all()
    ge = sn.cell_solve_batch(cuda(x), sn.GE32R).cpu().numpy()
    ref = oracle.cell_solve(x)
    assert (np.abs(ge - ref).max(axis=1) / np.abs(ref).max(axis=1)).max() < 1e-5
    # a 10% sample
    y = P.harvest(S, cap=P.solves_per_sweep // 10, seed=3)
    P.close()
    assert 0.85 * (P.solves_per_sweep // 10) <= y.shape[0] <= P.solves_per_sweep // 10


def test_ann_sweep_underflowing_flux_stays_finite(sn):
    """A hundred mean free paths of pure absorber (the paper's Problem 1 on 100^3
    cells of one mean free path): the flux underflows FP32 deep inside, the
    surrogate's input scale there counts as zero, and its flux stays finite
    everywhere (like the elimination's)."""
    wl = W.paper_problem(1, n=100, order=2)
    P = sn.Problem(wl)
    P.surrogate_set_weights(mlp.init_params(3))
    S = P.source(P.flux_tensor())
    ann = P.sweep(S, mode=sn.ANN)
    ge = P.sweep(S, mode=sn.GE32R)
    P.close()
    assert torch.isfinite(ann).all() and torch.isfinite(ge).all()
    assert (ge.abs() < 1e-30).any().item()        # the case is really there


def gate_ratios(in27, psi):
    """||b - A psi||_2 / ||b||_2 of each one-cell problem's own system (14), FP64 from
    the oracle's assembly (the ratio is unchanged by the canonical mirroring and the
    216/V scaling of the device's system)."""
    r = np.empty(in27.shape[0])
    for i in range(in27.shape[0]):
        A, b = oracle.assemble(in27[i])
        r[i] = np.linalg.norm(b - A @ psi[i]) / np.linalg.norm(b)
    return r


def test_mixed_gate_rows_follow_the_residual_test(sn, handle):
    """At a threshold that rejects about half of the rows: every row the CPU's
    residual test (FP64, the oracle's A and b, the network's own output) accepts
    carries the network's output, every row it rejects the elimination's, and the
    device's fallback count is the CPU's -- except rows within FP32 rounding of the
    threshold, which may go either way and are left out of the comparison."""
    x32 = W.onecell_problems(6000, seed=51).astype(np.float32)
    x = cuda(x32)
    handle.surrogate_set_weights(mlp.init_params(17))
    net, _ = handle.surrogate_apply(x, gated=False)
    net = net.cpu().numpy()
    ratio = gate_ratios(x32.astype(np.float64), net.astype(np.float64))
    tau = float(np.float32(np.median(ratio)))
    handle.surrogate_set_gate(tau)
    got, nfb = handle.surrogate_apply(x, gated=True)
    handle.surrogate_set_gate(1e-2)
    got = got.cpu().numpy()
    ge = sn.cell_solve_batch(x, sn.GE32R).cpu().numpy()
    near = np.abs(ratio / tau - 1.0) < 1e-4
    acc = (ratio <= tau) & ~near
    rej = (ratio > tau) & ~near
    assert 0.3 < rej.mean() < 0.7 and near.mean() < 0.01
    assert np.array_equal(got[acc], net[acc])
    assert np.allclose(got[rej], ge[rej], rtol=1e-6, atol=1e-7 * np.abs(ge).max())
    assert rej.sum() <= nfb <= rej.sum() + near.sum()


def test_mixed_gate_sweep_matches_oracle_gated_sweep(sn):
    """The gated surrogate sweep at a threshold that sends about half of the cells to
    elimination, against the oracle's gated network sweep (BF16 rounding steps, FP64
    residual test, FP64 elimination for the rejected cells).  A cell whose residual
    sits within rounding of the threshold may be decided the other way on the
    device, so the bar is that of the ungated network sweep; the fallback counts
    agree to a few cells, and the gated flux is much closer to the oracle's gated
    flux than to either pure form."""
    wl = W.random_small(5, 4, 3, order=4, G=2, seed=8, psi_inc=True)
    p = mlp.init_params(12) * 0.5
    p64 = np.asarray(p, np.float32).astype(np.float64)
    rng = np.random.default_rng(2)
    S = rng.uniform(0.0, 1.0, (2, 60, 8)).astype(np.float32)
    ratios = []

    def record(x):
        psi = predict_bf16(p64, f32_roundtrip(x))
        A, b = oracle.assemble(x[0])
        ratios.append(np.linalg.norm(b - A @ psi[0]) / np.linalg.norm(b))
        return psi
    network_sweep(wl, S.astype(np.float64), record)
    tau = float(np.float32(np.median(ratios)))
    O = oracle.OracleProblem(wl)
    ref, _ = O.sweep(S.astype(np.float64), mlp=(p64, True), gate=tau)
    ref_fb = O.last_fallbacks
    ge, _ = O.sweep(S.astype(np.float64))
    un, _ = O.sweep(S.astype(np.float64), mlp=(p64, True))
    P = sn.Problem(wl)
    P.surrogate_set_weights(p)
    P.surrogate_set_gate(tau)
    phi = P.sweep(cuda(S), mode=sn.ANN_GATED).cpu().numpy()
    fb, to = P.surrogate_stats()
    P.close()
    n = P.solves_per_sweep
    assert to == 0 and 0.2 * n < ref_fb < 0.8 * n
    assert abs(fb - ref_fb) <= 0.01 * n + 2
    scale = np.abs(ref).max()
    err = np.abs(phi - ref).max() / scale
    assert err < 2e-2
    assert err < 0.25 * min(np.abs(phi - ge).max(), np.abs(phi - un).max()) / scale


def bounded_weights(seed):
    """A network whose swept flux stays bounded on any mesh: 20 hidden units pass the
    20 flux features (S / s and the upwind values / s, all >= 0) through, each output
    is 0.9 times their mean, and small random terms sit everywhere else; psi <= about
    0.9 s, so no cell amplifies its inputs."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-0.01, 0.01, (64, 27))
    b1 = rng.uniform(-0.01, 0.01, 64)
    W2 = rng.uniform(-0.01, 0.01, (8, 64))
    b2 = rng.uniform(-0.01, 0.01, 8)
    for j in range(20):
        W1[j, 7 + j] = 1.0
    W2[:, :20] += 0.9 / 20
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2])


def test_ann_sweep_blocked_32_sampled_group(sn):
    """The tensor-core surrogate sweep at a stated workload size (blocked_32: 32^3
    cells, LQ_8, 4 groups; 10.5 M solves), ungated, with weights that keep the flux
    bounded; group 2 recomputed by the oracle's network sweep with the BF16 rounding
    steps.  The device rounds its FP32 inputs to BF16 where the oracle rounds FP64
    ones, so a feature may land one BF16 step away (2^-8 relative); with these
    weights one such step moves an output by at most 0.9/20 of that, and the bar
    is 1e-4 of the group maximum."""
    wl = W.blocked_32()
    P = sn.Problem(wl)
    p = bounded_weights(5)
    P.surrogate_set_weights(p)
    rng = np.random.default_rng(7)
    S = rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32)
    phi = P.sweep(cuda(S), mode=sn.ANN).cpu().numpy()
    fb, to = P.surrogate_stats()
    P.close()
    assert to == 0
    p64 = np.asarray(p, np.float32).astype(np.float64)
    ref, _ = oracle.OracleProblem(wl).sweep(S.astype(np.float64), groups=(2, 3), mlp=(p64, True))
    err = np.abs(phi[2] - ref[2]).max() / np.abs(ref[2]).max()
    print("blocked_32 ANN sweep vs oracle BF16 network sweep, group 2: max-norm rel err %.3e" % err)
    assert err < 1e-4        # measured 1.7e-5 on GB300


def long_key_mesh():
    """16^3 cells, LQ_8 (10 directions an octant), 128 groups: the central hyperplanes
    hold 8 * 192 * 128 = 196,608 keys, more than the persistent grid's thread slots
    (at most 4 CTAs of 128 threads on each SM), so there every key runs all 10 of its
    directions in one thread; the planes near the corners split theirs into 2-8
    chunks.  The surrogate kernel keeps two direction steps in flight and prefetches
    the inflow faces of the step after next, which only a key of 4 or more steps
    exercises."""
    wl = W.blocked(16, 2.5, 8, 128, 8, 4, seed=3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 8 * 192 * 128 > 4 * 128 * sms
    return wl


@pytest.mark.parametrize("mode", ["ungated", "gated"])
def test_ann_sweep_long_keys_match_oracle(sn, mode):
    """The surrogate sweep on long_key_mesh, groups 5 and 6 recomputed by the oracle's
    network sweep with the BF16 rounding steps (bounded weights, as in the blocked_32
    test).  Ungated: 1e-4 of the group maximum.  Gated at tau = 0.3 (the oracle sends
    about 43% of these rows to elimination): a row whose residual sits within a BF16
    input step of the threshold may be decided the other way on the device, and its
    downstream cells follow it, so the bar is on the mean nodal error (1e-3 of the
    group maximum) with the max-norm error held well below the distance to either
    pure form; the gate recorded by sn_surrogate_freeze_gate reproduces the gated
    flux bit for bit."""
    wl = long_key_mesh()
    P = sn.Problem(wl)
    p = bounded_weights(4)
    P.surrogate_set_weights(p)
    rng = np.random.default_rng(11)
    S64 = rng.uniform(0.0, 1.0, (P.G, P.ncell, 8))
    S = cuda(S64.astype(np.float32))
    p64 = np.asarray(p, np.float32).astype(np.float64)
    O = oracle.OracleProblem(wl)
    gs = slice(5, 7)
    Sr = S64.astype(np.float32).astype(np.float64)
    un, _ = O.sweep(Sr, groups=(5, 7), mlp=(p64, True))
    if mode == "ungated":
        phi = P.sweep(S, mode=sn.ANN).cpu().numpy()
        fb, to = P.surrogate_stats()
        P.close()
        assert to == 0
        err = np.abs(phi[gs] - un[gs]).max() / np.abs(un[gs]).max()
        print("long keys, ungated: max-norm rel err %.3e" % err)
        assert err < 1e-4
        return
    tau = 0.3
    ref, _ = O.sweep(Sr, groups=(5, 7), mlp=(p64, True), gate=tau)
    ref_frac = O.last_fallbacks / (2 * P.ncell * 80)
    ge, _ = O.sweep(Sr, groups=(5, 7))
    P.surrogate_set_gate(tau)
    gated = P.sweep(S, mode=sn.ANN_GATED).clone()
    fb, to = P.surrogate_stats()
    fb_freeze = P.surrogate_freeze_gate(S)
    frozen = P.sweep(S, mode=sn.ANN_FROZEN)
    fb_frozen = P.surrogate_stats()[0]
    n = P.solves_per_sweep
    P.close()
    assert to == 0 and 0.3 < ref_frac < 0.6 and 0.3 < fb / n < 0.6
    assert fb_freeze == fb == fb_frozen and torch.equal(frozen, gated)
    phi = gated.cpu().numpy()
    scale = np.abs(ref[gs]).max()
    d = np.abs(phi[gs] - ref[gs])
    far = min(np.abs(phi[gs] - ge[gs]).max(), np.abs(phi[gs] - un[gs]).max())
    print("long keys, gated tau 0.3: %.3f of rows to elimination (oracle, groups 5-6: %.3f); "
          "mean %.2e, max %.2e of the group maximum (pure forms: %.2e)"
          % (fb / n, ref_frac, d.mean() / scale, d.max() / scale, far / scale))
    assert d.mean() / scale < 1e-3
    assert d.max() < 0.25 * far


def test_frozen_gate_repeats_the_gated_sweep_and_converges(sn):
    """sn_surrogate_freeze_gate records the gate's decisions of one gated sweep; a
    frozen sweep from the same source takes the same solver in every row, so it gives
    the gated sweep's flux bit for bit and the same number of elimination rows; the
    frozen source iteration settles: its Eq. (21) mean change falls below 1e-4, the
    paper's stop for the network iteration (the network reads BF16-rounded inputs,
    so its sweep is piecewise constant in the flux and the change stalls at a noise
    floor instead of reaching the 1e-6 max-norm stop of elimination); changing the
    threshold drops the frozen decisions."""
    wl = W.random_small(6, 5, 7, order=6, G=3, seed=5, psi_inc=True)
    P = sn.Problem(wl)
    P.surrogate_set_weights(bounded_weights(3))
    rng = np.random.default_rng(3)
    S = cuda(rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32))
    n = P.solves_per_sweep
    tau, seen = None, []
    for t in 10.0 ** np.arange(-4.0, 1.01, 0.25):
        P.surrogate_set_gate(float(t))
        P.sweep(S, mode=sn.ANN_GATED)
        seen.append((float(t), P.surrogate_stats()[0] / n))
        if 0.2 < seen[-1][1] < 0.8:
            tau = float(t)
            break
    assert tau is not None, seen
    gated = P.sweep(S, mode=sn.ANN_GATED)
    fb_gated = P.surrogate_stats()[0]
    fb_freeze = P.surrogate_freeze_gate(S)
    frozen = P.sweep(S, mode=sn.ANN_FROZEN)
    fb_frozen = P.surrogate_stats()[0]
    assert fb_freeze == fb_gated == fb_frozen
    assert torch.equal(frozen, gated)
    phi = P.flux_tensor()
    for _ in range(50):
        r = P.source_iterate(phi=phi, tol=0.0, max_it=10, mode=sn.ANN_FROZEN, allow_noconv=True)
        if r["change_mean"] < 1e-4:
            break
    assert r["change_mean"] < 1e-4 and torch.isfinite(phi).all()
    P.surrogate_set_gate(tau * 2)
    with pytest.raises(sn.SnError) as e:
        P.sweep(S, mode=sn.ANN_FROZEN)
    P.close()
    assert e.value.status == sn.SN_ESTATE

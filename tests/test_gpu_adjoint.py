"""GPU parity of the discrete adjoint (gradients of a detector response with respect
to sigma_t, sigma_s and q) against the FP64 oracle adjoint, through the C ABI.
Bar: per-group max-norm relative error within 1e-4 (FP32 forward and adjoint
fluxes, FP64 gradient accumulation)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1906_04017_gb300 import workloads as W
from _parity import norm_err

pytestmark = pytest.mark.gpu


def corner_response(wl, n):
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    G = wl["sigt"].shape[0]
    vol = wl["lx"] / nx * wl["ly"] / ny * wl["lz"] / nz
    r = np.zeros((G, nx * ny * nz, 8))
    i, j, k = W.cell_ijk(wl)
    r[:, (i < n) & (j < n) & (k < n), :] = vol / 8.0
    return r


@pytest.mark.parametrize("shape,order,G,ncorner", [((5, 4, 3), 4, 2, 2), ((9, 7, 8), 6, 3, 3),
                                                   ((12, 12, 12), 8, 4, 4)])
def test_adjoint_matches_oracle(sn, shape, order, G, ncorner):
    wl = W.random_small(*shape, order=order, G=G, seed=sum(shape), psi_inc=True)
    r = corner_response(wl, ncorner)
    P = sn.Problem(wl)
    fwd = P.source_iterate(tol=1e-7, max_it=2000, allow_noconv=True)
    adj = P.adjoint(fwd["phi"], torch.from_numpy(r.astype(np.float32)).cuda(), tol=1e-7, max_it=2000,
                    allow_noconv=True)
    P.close()
    O = oracle.OracleProblem(wl)
    phi = O.source_iterate(1e-13, 5000)["phi"]
    ref = O.adjoint(phi, r, tol=1e-13, maxit=5000)
    assert norm_err(adj["Lam"].cpu().numpy(), ref["Lam"]) < 1e-4
    for key in ("grad_q", "grad_sigs", "grad_sigt"):
        got, want = adj[key].cpu().numpy(), ref[key]
        assert np.abs(got - want).max() < 1e-4 * np.abs(want).max(), key


def test_adjoint_checkpoint_blocks_cover_every_plane(sn):
    """A mesh whose hyperplane count is not a multiple of the checkpoint block
    (nplanes = 3 + 1 + 5 - 2 = 7, blocks of 3): dR/dsigma_t still matches."""
    wl = W.random_small(3, 1, 5, order=4, G=1, seed=3, psi_inc=True)
    r = corner_response(wl, 1)
    P = sn.Problem(wl)
    fwd = P.source_iterate(tol=1e-7, max_it=2000, allow_noconv=True)
    adj = P.adjoint(fwd["phi"], torch.from_numpy(r.astype(np.float32)).cuda(), tol=1e-7, max_it=2000,
                    allow_noconv=True)
    P.close()
    O = oracle.OracleProblem(wl)
    phi = O.source_iterate(1e-13, 5000)["phi"]
    ref = O.adjoint(phi, r, tol=1e-13, maxit=5000)
    got, want = adj["grad_sigt"].cpu().numpy(), ref["grad_sigt"]
    assert np.abs(got - want).max() < 1e-4 * np.abs(want).max()


def test_detector_response_autograd_matches_oracle(sn):
    """DetectorResponse (torch.autograd.Function over sn_source_iterate, sn_response
    and sn_adjoint_sweep): R and its gradients against the oracle."""
    wl = W.random_small(6, 5, 4, order=4, G=2, seed=11, psi_inc=True)
    r = corner_response(wl, 2)
    sigt, sigs, q = (torch.tensor(wl[k], dtype=torch.float64, requires_grad=True) for k in ("sigt", "sigs", "q"))
    R = sn.DetectorResponse.apply(sigt, sigs, q, wl, torch.from_numpy(r), 1e-6, 2000)
    R.backward()
    O = oracle.OracleProblem(wl)
    phi = O.source_iterate(1e-13, 5000)["phi"]
    ref = O.adjoint(phi, r, tol=1e-13, maxit=5000)
    R_ref = float((r * phi).sum())
    assert abs(R.item() - R_ref) < 1e-5 * abs(R_ref)
    for t, key in ((sigt, "grad_sigt"), (sigs, "grad_sigs"), (q, "grad_q")):
        want = ref[key]
        assert np.abs(t.grad.numpy() - want).max() < 1e-4 * np.abs(want).max(), key


def test_adjoint_matches_fp64_central_differences(sn):
    """FP32 adjoint gradients against central differences (relative step 1e-6) of R
    from FP64 GPU source iterations (SN_SOLVE_GE64), warm-started from the
    unperturbed flux, for parameters of every kind."""
    wl = W.random_small(5, 6, 4, order=4, G=2, seed=4, psi_inc=True)
    r = corner_response(wl, 2)
    P = sn.Problem(wl)
    fwd = P.source_iterate(tol=1e-6, max_it=2000)
    adj = P.adjoint(fwd["phi"], torch.from_numpy(r.astype(np.float32)).cuda(), tol=1e-6, max_it=2000)
    P.close()
    P64 = sn.Problem(wl, fp64=True)
    base = P64.source_iterate(tol=1e-13, max_it=5000)["phi"]
    P64.close()
    r64 = torch.from_numpy(r).cuda()

    def R_of(key, idx, val):
        w = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in wl.items()}
        w[key][idx] = val
        Q = sn.Problem(w, fp64=True)
        phi = base.clone()
        Q.source_iterate(phi=phi, tol=1e-13, max_it=5000)
        R = Q.response(phi, r64)
        Q.close()
        return R

    rng = np.random.default_rng(0)
    for key, gkey in (("sigt", "grad_sigt"), ("sigs", "grad_sigs"), ("q", "grad_q")):
        g = adj[gkey].cpu().numpy()
        # parameters whose gradient is at least 10% of the largest of their kind
        cand = np.argwhere(np.abs(g) >= 0.1 * np.abs(g).max())
        for gi, ci in cand[rng.choice(len(cand), min(4, len(cand)), replace=False)]:
            p = wl[key][gi, ci]
            h = 1e-6 * (p if p > 0 else 1.0)
            fd = (R_of(key, (gi, ci), p + h) - R_of(key, (gi, ci), p - h)) / (2 * h)
            assert abs(g[gi, ci] - fd) <= 1e-4 * abs(fd), (key, gi, ci, g[gi, ci], fd)


def test_adjoint_blocked_32_against_central_differences(sn):
    """The adjoint form at its stated size: blocked_32 (32^3 cells, LQ_8, 4 groups),
    R = group-summed scalar flux over the 4x4x4 low corner, gradients with respect to
    all 393,216 per-cell, per-group sigma_t, sigma_s and q by the FP32 adjoint; 32
    parameters drawn uniformly over every kind, group and cell, and 8 more from the
    cells within 6 cells of the detector's corner, each checked against FP64 central
    differences with relative step 1e-6 (absolute 1e-6 where the parameter is 0).
    Both perturbed FP64 source iterations start from the converged unperturbed flux
    and take the same 120 iterations (spectral radius <= 0.9, so the difference is
    converged to ~1e-6 of itself).

    Bar: |adjoint - FD| <= 1e-4 |FD| + 1e-5 max|g| + 1e-14 |R| / h, max|g| the largest
    adjoint gradient of the parameter's kind.  The second term is the accuracy of the
    FP32 adjoint itself: its source iteration stops at a 1e-6 change in the max norm,
    so every entry carries an absolute error of about tol / (1 - rho) <= 1e-5 of the
    largest one (far from the detector that is more than 1e-4 of the entry).  The
    third is the resolution of the difference: two FP64 values of R carry ~1e-15 R of
    rounding each, divided by the step h.  The 8 parameters near the detector are
    held to 1e-4 relative alone (measured: at most 2e-5)."""
    wl = W.blocked_32()
    nx = wl["nx"]
    G, C = wl["sigt"].shape[0], nx ** 3
    r = corner_response(wl, 4)
    P = sn.Problem(wl)
    fwd = P.source_iterate(tol=1e-6, max_it=2000)
    adj = P.adjoint(fwd["phi"], torch.from_numpy(r.astype(np.float32)).cuda(), tol=1e-6, max_it=2000)
    P.close()
    P64 = sn.Problem(wl, fp64=True)
    base = P64.source_iterate(tol=1e-13, max_it=5000)
    phi0 = base["phi"]
    r64 = torch.from_numpy(r).cuda()
    R0 = P64.response(phi0, r64)
    P64.close()
    rng = np.random.default_rng(2024)
    kinds = (("sigt", "grad_sigt"), ("sigs", "grad_sigs"), ("q", "grad_q"))
    gmax = {gk: float(adj[gk].abs().max().item()) for _, gk in kinds}
    i, j, k = W.cell_ijk(wl)
    near = np.flatnonzero((i < 6) & (j < 6) & (k < 6))
    worst, rows, strict = 0.0, [], 0
    for n in range(40):
        key, gkey = kinds[rng.integers(0, 3)]
        g = int(rng.integers(0, G))
        c = int(rng.integers(0, C)) if n < 32 else int(near[rng.integers(0, len(near))])
        p0 = float(wl[key][g, c])
        h = 1e-6 * (p0 if p0 > 0 else 1.0)
        Rs = []
        for v in (p0 + h, p0 - h):
            w = dict(wl)
            w[key] = wl[key].copy()
            w[key][g, c] = v
            Q = sn.Problem(w, fp64=True)
            phi = phi0.clone()
            Q.source_iterate(phi=phi, tol=0.0, max_it=120, allow_noconv=True)
            Rs.append(Q.response(phi, r64))
            Q.close()
        fd = (Rs[0] - Rs[1]) / (2 * h)
        ga = float(adj[gkey][g, c].item())
        bound = 1e-4 * abs(fd) + 1e-5 * gmax[gkey] + 1e-14 * abs(R0) / h
        worst = max(worst, abs(ga - fd) / bound)
        rows.append((key, g, c, p0, ga, fd, abs(ga - fd) / max(abs(fd), 1e-300)))
        if n >= 32:
            strict += 1
            assert abs(ga - fd) <= 1e-4 * abs(fd), rows[-1]
    for r in rows:
        print("%-4s g=%d c=%6d p=%.4g adjoint=% .6e fd=% .6e rel=%.2e" % r)
    print("blocked_32 adjoint vs FD: worst |adjoint - FD| / bound = %.3f, %d near the detector held to 1e-4 "
          "relative alone" % (worst, strict))
    assert worst <= 1.0

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

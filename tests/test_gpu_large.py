"""The large mixed workload (96^3 cells, LQ_12 = 168 directions, 16 groups, spheres
of high opacity): only scalar-flux arrays and wavefront face planes are resident
(no angular flux), the source iteration runs from a captured CUDA graph.  Checks
that hold at any size (particle balance, convergence) plus one group recomputed by
the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1906_04017_gb300 import workloads as W
from _parity import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spheres():
    return W.spheres_96()


def test_spheres_96_memory_has_no_angular_flux(sn, spheres):
    """The handle holds scalar-flux arrays (per-octant partials included) and the
    wavefront face planes, an order of magnitude below one full angular flux."""
    P = sn.Problem(spheres)
    angular = P.solves_per_sweep * 8 * 4          # bytes of a full FP32 angular flux
    held = P.device_bytes
    P.close()
    assert held < angular / 10


def test_spheres_96_source_iteration_converges_with_balance(sn, spheres):
    P = sn.Problem(spheres)
    r = P.source_iterate(tol=1e-6, max_it=400, use_graph=True)
    bal = P.balance()
    P.close()
    assert r["converged"]
    assert np.all(np.isfinite(r["phi"].cpu().numpy()))
    assert abs(bal[0] + bal[1] - bal[2] - bal[3]) < 1e-5 * (bal[2] + bal[3])


def test_spheres_96_sampled_group(sn, spheres):
    """One sweep of every group from a random source; the last group recomputed by
    the FP64 oracle (168 directions x 884,736 cells)."""
    P = sn.Problem(spheres)
    rng = np.random.default_rng(5)
    S = rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32)
    phi = P.sweep(torch.from_numpy(S).cuda()).cpu().numpy()
    P.close()
    g = P.G - 1
    ref, _ = oracle.OracleProblem(spheres).sweep(S.astype(np.float64), groups=(g, g + 1))
    assert rel_err(phi[g], ref[g]) < 1e-5

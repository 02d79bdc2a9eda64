"""GPU parity of the batched one-cell solve (Sec. 3 one-cell problem; per-cell
system (14)) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1906_04017_gb300 import workloads as W
from _parity import f32_roundtrip

pytestmark = pytest.mark.gpu


def per_problem_err(got, ref):
    return (np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).max()


def edge_problems(rng, n):
    """Directions on the octant boundaries (zero cosines), sigma_t = 0, tiny and
    large cells, negative inflow values."""
    x = W.onecell_problems(n, seed=99)
    axes = rng.integers(0, 3, n)
    x[np.arange(n), axes] = 0.0
    x[:, 0:3] /= np.linalg.norm(x[:, 0:3], axis=1, keepdims=True)
    x[: n // 4, 6] = 0.0
    x[n // 4: n // 2, 3:6] *= rng.uniform(0.01, 100.0, (n // 2 - n // 4, 1))
    x[n // 2:, 15:27] -= 0.5
    return x


@pytest.mark.parametrize("n", [1, 127, 129, 200003])
def test_ge32r_matches_oracle(sn, n):
    x = f32_roundtrip(W.onecell_problems(n, seed=n))
    ref = oracle.cell_solve(x)
    got = sn.cell_solve_batch(torch.from_numpy(x.astype(np.float32)).cuda(), sn.GE32R).cpu().numpy()
    assert per_problem_err(got, ref) < 1e-5


def test_ge32_without_refinement_is_close(sn):
    x = f32_roundtrip(W.onecell_problems(50000, seed=5))
    ref = oracle.cell_solve(x)
    got = sn.cell_solve_batch(torch.from_numpy(x.astype(np.float32)).cuda(), sn.GE32).cpu().numpy()
    assert per_problem_err(got, ref) < 1e-4


def test_f64_matches_oracle(sn):
    x = W.onecell_problems(100000, seed=8)
    ref = oracle.cell_solve(x)
    got = sn.cell_solve_batch_f64(torch.from_numpy(x).cuda()).cpu().numpy()
    assert per_problem_err(got, ref) < 1e-12


def test_edge_cases(sn):
    rng = np.random.default_rng(3)
    x = f32_roundtrip(edge_problems(rng, 40000))
    ref = oracle.cell_solve(x)
    got = sn.cell_solve_batch(torch.from_numpy(x.astype(np.float32)).cuda(), sn.GE32R).cpu().numpy()
    assert np.all(np.isfinite(got))
    assert per_problem_err(got, ref) < 1e-5
    got64 = sn.cell_solve_batch_f64(torch.from_numpy(x).cuda()).cpu().numpy()
    assert per_problem_err(got64, ref) < 1e-12


def test_empty_batch(sn):
    out = sn.cell_solve_batch(torch.zeros((0, 27), device="cuda"), sn.GE32R)
    assert out.shape == (0, 8)


def test_exchange_path_matches_oracle(sn):
    """sigma_t < 0: partial pivoting exchanges rows in most systems (lanes of a warp
    mixed between the diagonal path and the exchange path); the solutions still
    match the oracle's elimination.  The systems' condition numbers stay below ~20."""
    x = f32_roundtrip(W.exchange_problems(50021, seed=2))
    ref = oracle.cell_solve(x)
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    assert per_problem_err(sn.cell_solve_batch(xt, sn.GE32R).cpu().numpy(), ref) < 1e-5
    assert per_problem_err(sn.cell_solve_batch(xt, sn.GE32).cpu().numpy(), ref) < 1e-4
    got64 = sn.cell_solve_batch_f64(torch.from_numpy(x).cuda()).cpu().numpy()
    assert per_problem_err(got64, ref) < 1e-12

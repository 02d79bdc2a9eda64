"""Facts about the per-cell system (14) that the GPU elimination relies on, checked
with an independent LU (scipy, partial pivoting) on the oracle's assembled matrices.

For sigma_t >= 0 the symmetric part of the matrix is positive definite (upwind
coercivity: half the face masses of the six faces plus sigma_t times the mass
matrix), so elimination on the diagonal pivots is well defined and partial
pivoting makes no exchange; the GPU path eliminates on the diagonal first and
redoes with exchanges only where the pivoting test asks for them.  Negative
sigma_t (outside the physical range) is where exchanges do occur, so the GPU test
of that path has cases to work on."""
import numpy as np
import scipy.linalg as sl

import oracle
from paper_1906_04017_gb300 import workloads as W


def extreme_problems(n, seed):
    """Directions with zero cosines, cells from 1e-3 to 1e2 per axis (aspect ratios
    up to 1e5), sigma_t from 0 to 1e4."""
    rng = np.random.default_rng(seed)
    x = W.onecell_problems(n, seed=seed)
    om = rng.normal(size=(n, 3))
    third = n // 3
    om[np.arange(third), rng.integers(0, 3, third)] = 0.0
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    x[:, 0:3] = om
    x[:, 3:6] = 10.0 ** rng.uniform(-3, 2, (n, 3))
    x[:, 6] = 10.0 ** rng.uniform(-6, 4, n)
    x[::5, 6] = 0.0
    return x


def exchanges(A):
    P, _, _ = sl.lu(A)
    return not np.array_equal(P, np.eye(A.shape[0]))


def test_physical_systems_have_positive_definite_symmetric_part():
    for x in (W.onecell_problems(1500, seed=4), extreme_problems(1500, seed=5)):
        for i in range(len(x)):
            A, _ = oracle.assemble(x[i])
            lam = np.linalg.eigvalsh(0.5 * (A + A.T)).min()
            assert lam > 0.1 * np.abs(A).max()
            assert not exchanges(A)


def test_negative_sigma_needs_exchanges():
    x = W.exchange_problems(1000, seed=1)
    assert np.all(x[:, 6] < 0)
    n_ex = sum(exchanges(oracle.assemble(x[i])[0]) for i in range(len(x)))
    assert 0.2 * len(x) < n_ex < len(x)

"""Pins of the oracle's LQ_N quadrature (Sec. 2, Eqs. (8)-(9)) against closed-form
integrals over the unit sphere, symmetry and positivity."""
import itertools
import math

import numpy as np
import pytest

import oracle

ORDERS = [2, 4, 6, 8, 10, 12]


def sphere_monomial(a, b, c):
    """Exact integral of x^a y^b z^c over the unit sphere."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    g = math.gamma
    return 2.0 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)


@pytest.mark.parametrize("order", ORDERS)
def test_count_norm_positive(order):
    om, w = oracle.lqn(order)
    assert om.shape == (order * (order + 2), 3)
    assert np.all(w > 0)
    assert abs(w.sum() - 4 * np.pi) < 1e-13
    assert np.allclose(np.linalg.norm(om, axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("order", ORDERS)
def test_octant_and_permutation_symmetry(order):
    om, w = oracle.lqn(order)
    n8 = om.shape[0] // 8
    base = om[:n8]
    assert np.all(base > 0)
    for o in range(8):
        s = np.array([-1 if o & 1 else 1, -1 if o & 2 else 1, -1 if o & 4 else 1])
        assert np.array_equal(om[o * n8:(o + 1) * n8], base * s)
        assert np.array_equal(w[o * n8:(o + 1) * n8], w[:n8])
    # the point set of an octant is closed under axis permutations, weights too
    key = {tuple(np.round(p, 12)): wi for p, wi in zip(base, w[:n8])}
    for p, wi in zip(base, w[:n8]):
        for perm in itertools.permutations(range(3)):
            q = tuple(np.round(p[list(perm)], 12))
            assert q in key and abs(key[q] - wi) < 1e-14


@pytest.mark.parametrize("order", ORDERS)
def test_exact_sphere_moments(order):
    """All monomials of even degree <= order - 2 are integrated to round-off, and
    the pure power of degree `order` to the precision of the tabulated mu_1 (the
    condition that fixes mu_1); every odd monomial vanishes."""
    om, w = oracle.lqn(order)
    for deg in range(0, order + 3):
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                c = deg - a - b
                got = np.sum(w * om[:, 0] ** a * om[:, 1] ** b * om[:, 2] ** c)
                ref = sphere_monomial(a, b, c)
                if deg % 2 or a % 2 or b % 2:
                    assert abs(got) < 1e-13
                elif deg <= max(order - 2, 2):
                    assert abs(got - ref) < 1e-13 * 4 * np.pi, (order, a, b, c)
                elif deg == order and max(a, b, c) == deg:
                    assert abs(got - ref) < 5e-7 * ref, (order, a, b, c)


def test_unsupported_order():
    with pytest.raises(ValueError):
        oracle.lqn(16)

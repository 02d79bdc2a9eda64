"""Pins of the oracle's Q1 element matrices (Sec. 2, the streaming, interaction and
source terms that build Eq. (12)).

The oracle integrates with 2x2x2 Gauss points.  Here the same bilinear forms are
integrated exactly with sympy, and checked against the 1D Kronecker closed form;
the outflow form of Eq. (14) is checked against the inflow form that Green's
theorem gives."""
import numpy as np
import pytest

import oracle


def sympy_element(dx, dy, dz):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    hx, hy, hz = sp.Rational(dx), sp.Rational(dy), sp.Rational(dz)
    b = [lambda t, h: 1 - t / h, lambda t, h: t / h]
    u = [b[n & 1](x, hx) * b[(n >> 1) & 1](y, hy) * b[(n >> 2) & 1](z, hz) for n in range(8)]
    X = [x, y, z]
    H = [hx, hy, hz]

    def vol(f):
        return sp.integrate(f, (x, 0, hx), (y, 0, hy), (z, 0, hz))

    M = np.array([[float(vol(sp.expand(u[k] * u[j]))) for j in range(8)] for k in range(8)])
    L = np.array([[[float(vol(sp.expand(-u[j] * sp.diff(u[k], X[a])))) for j in range(8)]
                   for k in range(8)] for a in range(3)])
    F = np.zeros((6, 8, 8))
    for f in range(6):
        ax, side = f // 2, f % 2
        t = [X[i] for i in range(3) if i != ax]
        th = [H[i] for i in range(3) if i != ax]
        for k in range(8):
            for j in range(8):
                g = (u[k] * u[j]).subs(X[ax], H[ax] if side else 0)
                F[f, k, j] = float(sp.integrate(sp.expand(g), (t[0], 0, th[0]), (t[1], 0, th[1])))
    return M, L, F


@pytest.mark.parametrize("h", [("1/10", "7/5", "2/7")])
def test_element_vs_exact_integrals(h):
    hf = [float(eval(s)) for s in h]
    M, L, G, F = oracle.element(*hf)
    Me, Le, Fe = sympy_element(*h)
    scale = hf[0] * hf[1] * hf[2]
    assert np.allclose(M, Me, atol=1e-15 * scale, rtol=1e-13)
    assert np.allclose(L, Le, atol=1e-15, rtol=1e-13)
    assert np.allclose(F, Fe, atol=1e-15, rtol=1e-13)
    # G_a = -L_a^T  (both are int u_k d_a u_j)
    assert np.allclose(G, -np.transpose(L, (0, 2, 1)), atol=1e-14)


def test_kronecker_closed_form():
    """With node n = a + 2b + 4c the matrices factor into 1D 2x2 blocks:
    M = m_z (x) m_y (x) m_x with m(h) = h/6 [[2,1],[1,2]], and
    L_x = m_z (x) m_y (x) l, l = -int b_j b_k' = [[1/2, 1/2], [-1/2, -1/2]]."""
    dx, dy, dz = 0.3, 0.7, 1.9
    M, L, G, F = oracle.element(dx, dy, dz)
    m = lambda h: h / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
    l = np.array([[0.5, 0.5], [-0.5, -0.5]])
    e0 = np.array([[1.0, 0.0], [0.0, 0.0]])
    e1 = np.array([[0.0, 0.0], [0.0, 1.0]])
    K = lambda cz, cy, cx: np.kron(cz, np.kron(cy, cx))
    assert np.allclose(M, K(m(dz), m(dy), m(dx)), atol=1e-15)
    assert np.allclose(L[0], K(m(dz), m(dy), l), atol=1e-15)
    assert np.allclose(L[1], K(m(dz), l, m(dx)), atol=1e-15)
    assert np.allclose(L[2], K(l, m(dy), m(dx)), atol=1e-15)
    assert np.allclose(F[0], K(m(dz), m(dy), e0), atol=1e-15)
    assert np.allclose(F[1], K(m(dz), m(dy), e1), atol=1e-15)
    assert np.allclose(F[3], K(m(dz), e1, m(dx)), atol=1e-15)
    assert np.allclose(F[4], K(e0, m(dy), m(dx)), atol=1e-15)


def test_outflow_form_equals_inflow_form():
    rng = np.random.default_rng(1)
    for _ in range(200):
        x = np.zeros(27)
        v = rng.normal(size=3)
        x[0:3] = v / np.linalg.norm(v)
        x[3:6] = rng.uniform(0.05, 2.0, 3)
        x[6] = rng.lognormal(0, 2)
        A, _ = oracle.assemble(x)
        Ai = oracle.assemble_inflow_form(x)
        assert np.allclose(A, Ai, atol=1e-14 * np.abs(Ai).max())


def test_streaming_conserves():
    """Summing the test functions gives w = 1, whose gradient vanishes: every column
    of L_a sums to zero, and the column sums of M and F_f are the volume and face
    integrals of the basis functions."""
    dx, dy, dz = 0.4, 1.3, 0.9
    M, L, G, F = oracle.element(dx, dy, dz)
    assert np.allclose(L.sum(axis=1), 0.0, atol=1e-15)
    assert np.allclose(M.sum(axis=0), dx * dy * dz / 8)
    areas = [dy * dz, dy * dz, dx * dz, dx * dz, dx * dy, dx * dy]
    for f in range(6):
        col = F[f].sum(axis=0)
        assert np.isclose(col.sum(), areas[f])
        assert np.count_nonzero(np.abs(col) > 0) == 4

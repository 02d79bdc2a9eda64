"""Pins of the oracle's general hexahedral cells (trilinear maps; the shape change of
the cells of Sec. 2's closing remarks): the box limit, closed-form volumes and face
area vectors of parallelepipeds, Green's theorem between the streaming and face
matrices, an exactly reproduced linear solution on a deformed mesh, and balance."""
import numpy as np
import pytest

import oracle
from paper_1906_04017_gb300 import workloads as W


def unit_nodes():
    return np.array([[n & 1, (n >> 1) & 1, n >> 2] for n in range(8)], dtype=float)


def test_box_vertices_give_the_box_element():
    h = np.array([0.5, 0.7, 0.9])
    M, L, Fv = oracle.hex_element(unit_nodes() * h)
    Mb, Lb, Gb, Fb = oracle.element(*h)
    assert np.allclose(M, Mb, atol=1e-15)
    assert np.allclose(L, Lb, atol=1e-15)
    for f in range(6):
        a, side = f // 2, f % 2
        for c in range(3):
            want = (1.0 if side else -1.0) * Fb[f] if c == a else np.zeros((8, 8))
            assert np.allclose(Fv[f, c], want, atol=1e-15)


def test_parallelepiped_volume_and_face_area_vectors():
    """An affine cell x = x0 + B xi: volume |det B| (sum of M), and the summed face
    matrix of face f is its outward area vector (cross products of B's columns)."""
    rng = np.random.default_rng(0)
    B = np.eye(3) * [0.8, 1.1, 0.6] + rng.uniform(-0.15, 0.15, (3, 3))
    X = np.array([0.3, -0.2, 1.0]) + unit_nodes() @ B.T
    M, L, Fv = oracle.hex_element(X)
    assert M.sum() == pytest.approx(abs(np.linalg.det(B)), rel=1e-14)
    cols = [B[:, 0], B[:, 1], B[:, 2]]
    for f in range(6):
        a, side = f // 2, f % 2
        p, q = (a + 1) % 3, (a + 2) % 3
        area = np.cross(cols[p], cols[q]) * (1.0 if side else -1.0)
        got = np.array([Fv[f, c].sum() for c in range(3)])
        assert np.allclose(got, area, atol=1e-14)


def test_greens_theorem_on_a_deformed_cell():
    """L_a + L_a^T = -sum_f Fv[f][a] entry by entry (integration by parts of
    N_k N_j), and sum_k L_a[k][j] = 0 (the test function 1 has no gradient)."""
    rng = np.random.default_rng(1)
    X = unit_nodes() * [1.0, 0.8, 1.2] + rng.uniform(-0.12, 0.12, (8, 3))
    M, L, Fv = oracle.hex_element(X)
    for a in range(3):
        assert np.allclose(L[a] + L[a].T, -Fv[:, a].sum(axis=0), atol=1e-14)
        assert np.allclose(L[a].sum(axis=0), 0.0, atol=1e-14)
    assert np.all(np.linalg.eigvalsh(M) > 0)


def face_values(fun, xyz, wl, ax, side):
    """Nodal boundary values of fun on the face plane (ax, side), layout [cell of the
    face plane][4] with the in-face order of the sweep (x: b + 2c, y: a + 2c, z: a + 2b)."""
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)
    out = []
    if ax == 0:
        i = 0 if side == 0 else nx
        for k in range(nz):
            for j in range(ny):
                out.append([fun(xyz[vid(i, j + (t & 1), k + (t >> 1))]) for t in range(4)])
    elif ax == 1:
        j = 0 if side == 0 else ny
        for k in range(nz):
            for i in range(nx):
                out.append([fun(xyz[vid(i + (t & 1), j, k + (t >> 1))]) for t in range(4)])
    else:
        k = 0 if side == 0 else nz
        for j in range(ny):
            for i in range(nx):
                out.append([fun(xyz[vid(i + (t & 1), j + (t >> 1), k)]) for t in range(4)])
    return np.array(out, dtype=float)


def cell_vertex_values(fun, xyz, wl):
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)
    out = np.zeros((nx * ny * nz, 8))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = i + nx * (j + ny * k)
                for n in range(8):
                    out[c, n] = fun(xyz[vid(i + (n & 1), j + ((n >> 1) & 1), k + (n >> 2))])
    return out


@pytest.mark.parametrize("order", [4, 8])
def test_linear_solution_is_reproduced_on_a_deformed_mesh(order):
    """psi*(x) = alpha + beta . x lies in the isoparametric Q1 space of any trilinear
    cell, and so does Q = Omega . beta + sigma_t psi*: with that nodal source and psi*
    as inflow the DFEM sweep returns psi* at every node of every cell, exactly."""
    wl = W.random_small(3, 3, 3, order=order, G=1, seed=9)
    wl["sigs"][:] = 0.0
    xyz = W.deformed_vertices(wl, 0.08, seed=1)
    P = oracle.OracleProblem(wl, xyz=xyz)
    om, _ = oracle.lqn(order)
    alpha, beta = 0.7, np.array([0.3, -0.2, 0.45])
    psi_star = lambda x: alpha + beta @ x
    exact = cell_vertex_values(psi_star, xyz, wl)
    sig = wl["sigt"][0]
    for d in (0, len(om) // 3, len(om) - 1):
        o = om[d]
        S = exact * sig[:, None] + o @ beta
        bnd = [face_values(psi_star, xyz, wl, a, 0 if o[a] >= 0 else 1) for a in range(3)]
        psi, _ = P.sweep_dir(d, 0, S, *bnd)
        assert np.abs(psi - exact).max() < 1e-12 * np.abs(exact).max()


def test_deformed_mesh_balance():
    """Leakage + collisions = source + inflow, with the face and volume integrals from
    the cells' own matrices (w = 1 is the sum of the test functions)."""
    wl = W.random_small(4, 3, 3, order=6, G=2, seed=10, psi_inc=True)
    xyz = W.deformed_vertices(wl, 0.1, seed=2)
    P = oracle.OracleProblem(wl, xyz=xyz)
    rng = np.random.default_rng(3)
    S = rng.uniform(0.0, 1.0, (2, P.ncell, 8))
    _, tal = P.sweep(S)
    assert abs(tal[0] + tal[1] - tal[2] - tal[3]) < 1e-12 * (tal[2] + tal[3])


def test_small_deformation_is_close_to_the_box_solution():
    """A continuity check: vertices moved by 1e-7 of a cell change the flux by ~1e-7."""
    wl = W.random_small(3, 2, 2, order=4, G=1, seed=11, psi_inc=True)
    box = oracle.OracleProblem(wl).source_iterate(1e-14, 500)["phi"]
    hexp = oracle.OracleProblem(wl, xyz=W.deformed_vertices(wl, 1e-7, seed=4)).source_iterate(1e-14, 500)["phi"]
    same = oracle.OracleProblem(wl, xyz=W.box_vertices(wl)).source_iterate(1e-14, 500)["phi"]
    assert np.allclose(same, box, rtol=1e-12, atol=0)
    assert 0 < np.abs(hexp - box).max() < 1e-5 * np.abs(box).max()

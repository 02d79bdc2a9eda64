"""Pins of the oracle's per-cell solve and sweep (Sec. 2, Eqs. (10)-(14)).

Each check is fixed by the mathematics, not by the oracle's own formulas:
LAPACK for the elimination, a manufactured tri-linear solution that Q1 DFEM must
reproduce exactly, the infinite-medium constant solution, the streaming-only
constant solution, and particle balance."""
import numpy as np
import pytest

import oracle
from paper_1906_04017_gb300 import workloads as W


def rand_dir(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def test_ge_matches_lapack_random():
    rng = np.random.default_rng(0)
    worst = 0.0
    for n in (1, 2, 3, 5, 8, 11):
        for _ in range(300):
            A = rng.normal(size=(n, n)) + 0.1 * np.eye(n)
            b = rng.normal(size=n)
            x = oracle.ge_solve(A, b)
            ref = np.linalg.solve(A, b)
            cond = np.linalg.cond(A)
            worst = max(worst, np.abs(x - ref).max() / (np.abs(ref).max() * cond))
    assert worst < 1e-14


def test_ge_pivots():
    # a zero leading entry needs a row exchange
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.allclose(oracle.ge_solve(A, [2.0, 3.0]), [3.0, 2.0])
    with pytest.raises(ZeroDivisionError):
        oracle.ge_solve(np.zeros((3, 3)), np.ones(3))


def test_cell_solve_matches_lapack():
    x = W.onecell_problems(20000, seed=3)
    psi = oracle.cell_solve(x)
    for i in range(0, 20000, 97):
        A, b = oracle.assemble(x[i])
        ref = np.linalg.solve(A, b)
        assert np.allclose(psi[i], ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def trilinear(rng):
    c = rng.normal(size=8)

    def f(x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * x * z
                + c[6] * y * z + c[7] * x * y * z)

    def grad(x, y, z):
        return np.array([c[1] + c[4] * y + c[5] * z + c[7] * y * z,
                         c[2] + c[4] * x + c[6] * z + c[7] * x * z,
                         c[3] + c[5] * x + c[6] * y + c[7] * x * y])
    return f, grad


def node_xyz(i, j, k, h):
    return [((i + (n & 1)) * h[0], (j + ((n >> 1) & 1)) * h[1], (k + ((n >> 2) & 1)) * h[2]) for n in range(8)]


def face_points(ax, side, h, origin):
    """Positions of the 4 in-face nodes of face (ax, side), in-face order
    x-face t = b + 2c, y-face t = a + 2c, z-face t = a + 2b."""
    pts = []
    for t in range(4):
        lo, hi = t & 1, (t >> 1) & 1
        if ax == 0:
            a, b, c = side, lo, hi
        elif ax == 1:
            a, b, c = lo, side, hi
        else:
            a, b, c = lo, hi, side
        pts.append((origin[0] + a * h[0], origin[1] + b * h[1], origin[2] + c * h[2]))
    return pts


def test_manufactured_one_cell():
    """Q1 is closed under differentiation, so for a tri-linear psi* the source
    Omega.grad psi* + sigma_t psi* is tri-linear: with that nodal source and psi*
    on the inflow faces, the DFEM cell solve returns psi* exactly."""
    rng = np.random.default_rng(7)
    for _ in range(400):
        f, grad = trilinear(rng)
        om = rand_dir(rng)
        h = rng.uniform(0.05, 2.0, 3)
        sig = rng.lognormal(0, 1.5)
        x = np.zeros(27)
        x[0:3], x[3:6], x[6] = om, h, sig
        pts = node_xyz(0, 0, 0, h)
        x[7:15] = [om @ grad(*p) + sig * f(*p) for p in pts]
        for ax in range(3):
            side = 0 if om[ax] >= 0 else 1
            x[15 + 4 * ax:19 + 4 * ax] = [f(*p) for p in face_points(ax, side, h, (0, 0, 0))]
        psi = oracle.cell_solve(x)[0]
        exact = np.array([f(*p) for p in pts])
        assert np.allclose(psi, exact, rtol=1e-11, atol=1e-11 * np.abs(exact).max())


@pytest.mark.parametrize("shape", [(3, 4, 5), (6, 2, 3)])
def test_manufactured_sweep(shape):
    """The same manufactured solution through a whole-mesh sweep: upwind traces of
    a continuous psi* match, so the sweep reproduces psi* at every node."""
    rng = np.random.default_rng(11)
    nx, ny, nz = shape
    wl = W.random_small(nx, ny, nz, order=4, G=1, seed=2)
    P = oracle.OracleProblem(wl)
    h = (P.dx, P.dy, P.dz)
    for d in range(P.ndir):
        f, grad = trilinear(rng)
        om = P.omega[d]
        S = np.zeros((P.ncell, 8))
        exact = np.zeros((P.ncell, 8))
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    c = i + nx * (j + ny * k)
                    sig = P.sigt[0, c]
                    for n, p in enumerate(node_xyz(i, j, k, h)):
                        S[c, n] = om @ grad(*p) + sig * f(*p)
                        exact[c, n] = f(*p)
        bnd = []
        for ax, (na, nb) in enumerate([(ny, nz), (nx, nz), (nx, ny)]):
            side = 0 if om[ax] >= 0 else 1
            arr = np.zeros((na * nb, 4))
            n_ax = [nx, ny, nz][ax]
            for q in range(nb):
                for p in range(na):
                    o = [0, 0, 0]
                    t = [a for a in range(3) if a != ax]
                    o[ax] = (n_ax if side else 0) * h[ax] - side * h[ax]
                    o[t[0]] = p * h[t[0]]
                    o[t[1]] = q * h[t[1]]
                    arr[p + na * q] = [f(*pt) for pt in face_points(ax, side, h, o)]
            bnd.append(arr)
        psi, _ = P.sweep_dir(d, 0, S, *bnd)
        assert np.allclose(psi, exact, rtol=1e-10, atol=1e-10 * np.abs(exact).max())


def test_infinite_medium_constant():
    """Matched inflow and source: with q/(sigma_t - sigma_s) the same in every cell
    and psi_inc = q / (4 pi sigma_a) on every face, the solution is that constant."""
    rng = np.random.default_rng(5)
    wl = W.random_small(5, 4, 3, order=6, G=1, seed=9)
    n = 60
    c = 0.7
    sigt = rng.lognormal(0, 1, n)
    wl["sigt"][0] = sigt
    wl["sigs"][0] = c * sigt
    psi0 = 0.37
    wl["q"][0] = 4 * np.pi * psi0 * (1 - c) * sigt
    wl["psi_inc"][0, :] = psi0
    P = oracle.OracleProblem(wl)
    r = P.source_iterate(1e-14, 400)
    assert np.allclose(r["phi"], 4 * np.pi * psi0, rtol=1e-12)
    # and a single sweep from the exact scattering source
    S = P.source(np.full((1, n, 8), 4 * np.pi * psi0))
    phi, _ = P.sweep(S)
    assert np.allclose(phi, 4 * np.pi * psi0, rtol=1e-13)


def test_streaming_only_constant():
    """sigma_t = 0, no source, the same inflow on every face: psi is that constant."""
    wl = W.random_small(4, 3, 5, order=8, G=1, seed=1)
    wl["sigt"][:] = 0.0
    wl["sigs"][:] = 0.0
    wl["q"][:] = 0.0
    wl["psi_inc"][:] = 2.5
    P = oracle.OracleProblem(wl)
    phi, _ = P.sweep(np.zeros((1, P.ncell, 8)))
    assert np.allclose(phi, 4 * np.pi * 2.5, rtol=1e-13)


@pytest.mark.parametrize("seed", [0, 1])
def test_global_balance(seed):
    """Weight 1 = sum of test functions: over a sweep, boundary leakage + collisions
    = source + boundary inflow (interior face terms cancel pairwise)."""
    wl = W.random_small(5, 6, 4, order=8, G=2, seed=seed, psi_inc=True)
    P = oracle.OracleProblem(wl)
    rng = np.random.default_rng(seed)
    S = rng.uniform(0, 1, (P.G, P.ncell, 8))
    _, t = P.sweep(S)
    leak, coll, src, infl = t
    assert abs(leak + coll - src - infl) < 1e-13 * (src + infl)
    # converged source iteration: leakage + absorption = emission + inflow
    r = P.source_iterate(1e-13, 500)
    phi = r["phi"]
    M, _, _, _ = oracle.element(P.dx, P.dy, P.dz)
    vint = M.sum(axis=0)
    absorb = 0.0
    for g in range(P.G):
        # removal = sigma_t - (scattering that stays in the system: all of it here)
        absorb += np.sum((P.sigt[g] - P.sigs[g] * P.xfer[g].sum())[:, None] * phi[g] * vint[None, :])
    emit = np.sum(P.q * (P.dx * P.dy * P.dz))
    assert abs(r["tallies"][0] + absorb - emit - r["tallies"][3]) < 1e-10 * (emit + r["tallies"][3])


def test_superposition():
    wl = W.random_small(4, 4, 4, order=4, G=2, seed=3, psi_inc=True)
    P = oracle.OracleProblem(wl)
    rng = np.random.default_rng(3)
    S1 = rng.uniform(0, 1, (2, 64, 8))
    S2 = rng.uniform(-1, 1, (2, 64, 8))
    phi12, _ = P.sweep(S1 + S2)
    wl0 = dict(wl)
    wl0["psi_inc"] = np.zeros_like(wl["psi_inc"])
    P0 = oracle.OracleProblem(wl0)
    phi1, _ = P.sweep(S1)
    phi2, _ = P0.sweep(S2)
    assert np.allclose(phi12, phi1 + phi2, rtol=1e-12, atol=1e-13)


def test_mirror_symmetry():
    """Data symmetric under x -> Lx - x gives a flux with the same symmetry."""
    wl = W.random_small(6, 3, 4, order=6, G=1, seed=4)
    nx, ny, nz = 6, 3, 4
    for key in ("sigt", "sigs", "q"):
        a = wl[key].reshape(1, nz, ny, nx)
        a[:] = 0.5 * (a + a[..., ::-1])
        wl[key] = a.reshape(1, -1)
    wl["psi_inc"][0] = [0.3, 0.3, 0.1, 0.2, 0.0, 0.5]
    P = oracle.OracleProblem(wl)
    r = P.source_iterate(1e-13, 300)
    phi = r["phi"].reshape(nz, ny, nx, 2, 2, 2)          # node (c, b, a)
    mirrored = phi[:, :, ::-1, :, :, ::-1]
    assert np.allclose(phi, mirrored, rtol=1e-11, atol=1e-13)


def test_problem4_iteration_rate_is_the_scattering_ratio():
    """The paper's Problem 4 (sigma_s / sigma_t = 0.99 in a box a hundred mean free
    paths wide): almost nothing leaks, so the source iteration's error shrinks by
    about the scattering ratio each sweep (the infinite-medium rate)."""
    O = oracle.OracleProblem(W.paper_problem(4, n=10, order=2))
    phi, hist = None, []
    for _ in range(80):
        r = O.source_iterate(0.0, 1, phi0=phi)
        phi, _ = r["phi"], hist.append(r["change_mean"])
    rho = (hist[-1] / hist[-21]) ** (1.0 / 20)
    assert 0.975 < rho <= 0.99


def test_per_cell_balance_with_closed_form_integrals():
    """Testing the cell's weak form with w = 1 (the sum of its basis functions) gives
    the cell's particle balance: outflow + sigma_t int psi = int S + inflow.  Each
    integral is written here in closed form for the box cell (a trilinear function
    integrates to V/8 times its nodal sum, a bilinear face trace to A/4 times its
    four values), independently of the oracle's matrices."""
    x = W.onecell_problems(2000, seed=13)
    psi = oracle.cell_solve(x)
    worst = 0.0
    for r in range(x.shape[0]):
        om, h, sig = x[r, 0:3], x[r, 3:6], x[r, 6]
        S, up = x[r, 7:15], x[r, 15:27]
        V = h[0] * h[1] * h[2]
        area = (h[1] * h[2], h[0] * h[2], h[0] * h[1])
        out = inflow = 0.0
        for a in range(3):
            side = 1 if om[a] >= 0 else 0
            on_face = [n for n in range(8) if (n >> a) & 1 == side]
            out += abs(om[a]) * area[a] / 4 * psi[r, on_face].sum()
            inflow += abs(om[a]) * area[a] / 4 * up[4 * a:4 * a + 4].sum()
        lhs = out + sig * V / 8 * psi[r].sum()
        rhs = V / 8 * S.sum() + inflow
        worst = max(worst, abs(lhs - rhs) / (abs(rhs) + abs(lhs)))
    assert worst < 1e-13

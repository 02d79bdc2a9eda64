"""Seeded synthetic inputs of the DFEM S_n sweep, shared by the oracle tests and the GPU path.

This module draws random fields and one-cell problems and nothing else: it holds
none of the method's arithmetic (no quadrature, no element matrices, no solve).
Every field is generated on the host in FP64 with numpy's PCG64 and handed to
both sides, so the oracle and the CUDA library never have to agree on a random
number generator.

A workload is a dict with
  nx, ny, nz        cells per axis (uniform box cells)
  lx, ly, lz        box size
  order             LQ_N order of the level-symmetric quadrature
  sigt[G, ncell]    total cross section per group and cell
  sigs[G, ncell]    scattering cross section out of group g (per cell)
  q[G, ncell]       isotropic emission density (particles / volume), cell-constant
  xfer[G, G]        fraction of group g' scattering that lands in group g (row g')
  psi_inc[G, 6]     isotropic inflow on the faces x-, x+, y-, y+, z-, z+ (0 = vacuum)
Cells are numbered c = i + nx * (j + ny * k).

The shapes follow the paper's test problems (Sec. 4, the four problem tables)
and the five workload configurations the library is measured on:
  onecube_8  : unit cube, 8^3 cells, LQ_4, 1 group, sigma_t ~ U[0.5, 2],
               scattering ratio 0.5, q = 1 in the central 2^3 cells.
  blocked_64 : 10^3 box, 64^3 cells, LQ_8, 8 groups, sigma_t constant on
               8^3-cell blocks, lognormal(0, 1) per block and group, scattering
               ratio U[0.3, 0.9] per block, downscatter-only transfer, q = 1 in
               group 0 inside a random 16^3-cell sub-box.
  blocked_32 : the same generator at 32^3 cells on a 5^3 box (same cell size),
               LQ_8, 4 groups, 8^3-cell source box.
  spheres_96 : 10^3 box, 96^3 cells, LQ_12, 16 groups, background sigma_t 0.1,
               200 spheres (radius U[2, 8] cells, sigma_t lognormal(2, 0.5)),
               q = 1 in group 0 inside 8 of the spheres.
  paper_problem(k) : the paper's Problems 1-4 (10 cm cube, psi_inc = 1 on the
               x-, y-, z- faces).
"""
import numpy as np


def downscatter_xfer(G):
    """Lower-triangular (downscatter-only) group transfer: half of the scattering
    out of group g stays in g, the rest is spread evenly over the groups below it;
    the last group keeps all of it."""
    x = np.zeros((G, G))
    for g in range(G):
        if g == G - 1:
            x[g, g] = 1.0
        else:
            x[g, g] = 0.5
            x[g, g + 1:] = 0.5 / (G - 1 - g)
    return x


def _base(nx, ny, nz, lx, ly, lz, order, G):
    n = nx * ny * nz
    return dict(nx=nx, ny=ny, nz=nz, lx=float(lx), ly=float(ly), lz=float(lz), order=order,
                sigt=np.zeros((G, n)), sigs=np.zeros((G, n)), q=np.zeros((G, n)),
                xfer=downscatter_xfer(G), psi_inc=np.zeros((G, 6)))


def cell_ijk(wl):
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def onecube_8(seed=0):
    """Unit cube, 8^3 cells, LQ_4, 1 group (the small plain-method case)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    wl = _base(8, 8, 8, 1.0, 1.0, 1.0, 4, 1)
    wl["sigt"][0] = rng.uniform(0.5, 2.0, size=512)
    wl["sigs"][0] = 0.5 * wl["sigt"][0]
    i, j, k = cell_ijk(wl)
    centre = (i >= 3) & (i <= 4) & (j >= 3) & (j <= 4) & (k >= 3) & (k <= 4)
    wl["q"][0, centre] = 1.0
    wl["name"] = "onecube_8"
    return wl


def blocked(n=64, length=10.0, order=8, G=8, block=8, src=16, seed=0):
    """Blocked lognormal opacity field (the plain method at scale)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    wl = _base(n, n, n, length, length, length, order, G)
    nb = n // block
    blk_sigt = rng.lognormal(0.0, 1.0, size=(G, nb, nb, nb))
    blk_c = rng.uniform(0.3, 0.9, size=(nb, nb, nb))
    i, j, k = cell_ijk(wl)
    bi, bj, bk = i // block, j // block, k // block
    wl["sigt"][:] = blk_sigt[:, bk, bj, bi]
    wl["sigs"][:] = blk_c[bk, bj, bi][None, :] * wl["sigt"]
    o = rng.integers(0, n - src + 1, size=3)
    inside = ((i >= o[0]) & (i < o[0] + src) & (j >= o[1]) & (j < o[1] + src)
              & (k >= o[2]) & (k < o[2] + src))
    wl["q"][0, inside] = 1.0
    wl["name"] = "blocked_%d" % n
    return wl


def blocked_64(seed=0):
    return blocked(64, 10.0, 8, 8, 8, 16, seed)


def blocked_32(seed=0):
    return blocked(32, 5.0, 8, 4, 8, 8, seed)


def spheres(n=96, length=10.0, order=12, G=16, nsph=200, nsrc=8, seed=0):
    """Background sigma_t = 0.1 with random spheres of high opacity (large mixed form).

    Scattering ratio: 0.5 in the background, U[0.3, 0.9] per sphere (unstated in
    the workload description; this is the reading used)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    wl = _base(n, n, n, length, length, length, order, G)
    i, j, k = cell_ijk(wl)
    mat = np.full(i.shape, -1, dtype=np.int64)
    cen = rng.uniform(0.0, n, size=(nsph, 3))
    rad = rng.uniform(2.0, 8.0, size=nsph)
    sph_sigt = rng.lognormal(2.0, 0.5, size=(nsph, G))
    sph_c = rng.uniform(0.3, 0.9, size=nsph)
    x, y, z = i + 0.5, j + 0.5, k + 0.5
    for s in range(nsph):
        inside = (x - cen[s, 0]) ** 2 + (y - cen[s, 1]) ** 2 + (z - cen[s, 2]) ** 2 <= rad[s] ** 2
        mat[inside] = s
    bg = mat < 0
    wl["sigt"][:, bg] = 0.1
    wl["sigs"][:, bg] = 0.05
    ins = ~bg
    wl["sigt"][:, ins] = sph_sigt[mat[ins]].T
    wl["sigs"][:, ins] = sph_c[mat[ins]][None, :] * wl["sigt"][:, ins]
    present = np.unique(mat[ins])
    srcs = rng.choice(present, size=min(nsrc, present.size), replace=False)
    wl["q"][0, np.isin(mat, srcs)] = 1.0
    wl["name"] = "spheres_%d" % n
    return wl


def spheres_96(seed=0):
    return spheres(seed=seed)


def paper_problem(k, n=10, order=8):
    """The paper's Problems 1-4 (Sec. 4 tables): 10 cm cube, psi_inc = 1 on the
    x-, y-, z- faces, vacuum on the others, one group."""
    sigt, sigs, q = {1: (10.0, 0.0, 0.0), 2: (0.001, 0.0, 0.0),
                     3: (10.0, 0.0, 1.0), 4: (10.0, 9.9, 1.0)}[k]
    wl = _base(n, n, n, 10.0, 10.0, 10.0, order, 1)
    wl["sigt"][:] = sigt
    wl["sigs"][:] = sigs
    wl["q"][:] = q
    wl["psi_inc"][0, [0, 2, 4]] = 1.0
    wl["name"] = "paper_problem_%d" % k
    return wl


def random_small(nx, ny, nz, order=4, G=2, seed=0, psi_inc=False, lengths=None):
    """Small irregular meshes for parity tests (odd sizes give non-cubic hyperplanes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lx, ly, lz = lengths if lengths else (rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0))
    wl = _base(nx, ny, nz, lx, ly, lz, order, G)
    n = nx * ny * nz
    wl["sigt"][:] = rng.lognormal(0.0, 1.0, size=(G, n))
    wl["sigs"][:] = rng.uniform(0.2, 0.8, size=(1, n)) * wl["sigt"]
    wl["q"][:] = rng.uniform(0.0, 1.0, size=(G, n)) * (rng.uniform(size=(G, n)) < 0.3)
    if psi_inc:
        wl["psi_inc"][:] = rng.uniform(0.0, 1.0, size=(G, 6))
    wl["name"] = "random_%dx%dx%d" % (nx, ny, nz)
    return wl


def onecell_problems(n, seed=0):
    """Random one-cell problems in27[n, 27] = Omega(3), (dx, dy, dz), sigma_t,
    S(8), psi_up(12): direction uniform on the unit sphere, cell sizes U[0.1, 1],
    sigma_t lognormal(0, 1.5), nodal source U[0, 1], upwind face values U[0, 1]
    (the surrogate's training distribution)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n, 27))
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    out[:, 0:3] = v
    out[:, 3:6] = rng.uniform(0.1, 1.0, size=(n, 3))
    out[:, 6] = rng.lognormal(0.0, 1.5, size=n)
    out[:, 7:15] = rng.uniform(0.0, 1.0, size=(n, 8))
    out[:, 15:27] = rng.uniform(0.0, 1.0, size=(n, 12))
    return out


def exchange_problems(n, seed=0):
    """One-cell problems outside the physical range, built so that elimination with
    partial pivoting exchanges rows: flow in the first octant (canonical orientation
    equals the physical one), sigma_t = -U[0.2, 1] * sum_a |Omega_a| / h_a < 0, so the
    system loses its positive-definite symmetric part; other entries as in
    onecell_problems."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    out = onecell_problems(n, seed)
    out[:, 0:3] = np.abs(out[:, 0:3])
    tau = (out[:, 0:3] / out[:, 3:6]).sum(axis=1)
    out[:, 6] = -rng.uniform(0.2, 1.0, size=n) * tau
    return out


# Sampling box of the per-octant networks' one-cell problems (Sec. 4: uniform
# sampling of the incident fluxes, sources, total cross section, direction and cell
# shape).  The ranges cover the paper's Problems 1-4: psi_inc <= 1 on the boundary,
# sigma_t in {0.001, 10}, cells of 10 cm / (10..100).
OCTANT_NET_RANGES = {"psi": (0.0, 1.0), "angle": (0.0, 1.0), "q": (0.0, 1.0),
                     "sigt": (0.0, 10.0), "h": (0.1, 1.0)}


def octant_net_ranges(ranges=None):
    """(lo, hi) [8, 26] a-priori input ranges of the 8 networks, in their input
    order: psi_x(4), psi_y(4), psi_z(4), mu, eta, q(8), sigma_t, dx, dy, dz.  The
    angle range of octant o is mirrored to [-1, 0] on the axes where o has a
    negative cosine (bit 0: mu, bit 1: eta)."""
    r = dict(OCTANT_NET_RANGES if ranges is None else ranges)
    lo = np.empty((8, 26))
    hi = np.empty((8, 26))
    for o in range(8):
        spans = [r["psi"]] * 12 + [r["angle"]] * 2 + [r["q"]] * 8 + [r["sigt"]] + [r["h"]] * 3
        for j, (a, b) in enumerate(spans):
            if j in (12, 13) and (o >> (j - 12)) & 1:
                a, b = -b, -a
            lo[o, j], hi[o, j] = a, b
    return lo, hi


def octant_problems(m, seed=0, ranges=None):
    """8 * m one-cell problems in27 (layout of onecell_problems), rows
    [o * m, (o + 1) * m) in octant o (bit 0: Omega_x < 0, bit 1: Omega_y < 0,
    bit 2: Omega_z < 0): direction uniform on the octant's part of the unit sphere,
    every other input uniform on OCTANT_NET_RANGES."""
    r = dict(OCTANT_NET_RANGES if ranges is None else ranges)
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    out = np.empty((8 * m, 27))
    v = rng.normal(size=(8 * m, 3))
    v = np.abs(v) / np.linalg.norm(v, axis=1, keepdims=True)
    oct_ = np.repeat(np.arange(8), m)
    for a in range(3):
        v[:, a] *= np.where((oct_ >> a) & 1, -1.0, 1.0)
    out[:, 0:3] = v
    out[:, 3:6] = rng.uniform(*r["h"], size=(8 * m, 3))
    out[:, 6] = rng.uniform(*r["sigt"], size=8 * m)
    out[:, 7:15] = rng.uniform(*r["q"], size=(8 * m, 8))
    out[:, 15:27] = rng.uniform(*r["psi"], size=(8 * m, 12))
    return out


def box_vertices(wl):
    """Vertex coordinates [(nx+1)(ny+1)(nz+1), 3] of the workload's uniform box cells,
    vertex (i, j, k) at index i + (nx+1) (j + (ny+1) k)."""
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    x = np.linspace(0.0, wl["lx"], nx + 1)
    y = np.linspace(0.0, wl["ly"], ny + 1)
    z = np.linspace(0.0, wl["lz"], nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def deformed_vertices(wl, amp, seed=0):
    """The box vertices with every interior coordinate moved by U[-amp, amp] x the
    cell size along its axis; a vertex on a boundary plane stays on it (the domain
    remains the box), so the cells become general trilinear hexahedra."""
    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    v = box_vertices(wl)
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    i = np.tile(np.arange(nx + 1), (ny + 1) * (nz + 1))
    j = np.tile(np.repeat(np.arange(ny + 1), nx + 1), nz + 1)
    k = np.repeat(np.arange(nz + 1), (nx + 1) * (ny + 1))
    h = (wl["lx"] / nx, wl["ly"] / ny, wl["lz"] / nz)
    for a, (idx, n) in enumerate(((i, nx), (j, ny), (k, nz))):
        inner = (idx > 0) & (idx < n)
        v[inner, a] += rng.uniform(-amp, amp, size=int(inner.sum())) * h[a]
    return v


WORKLOADS = {"onecube_8": onecube_8, "blocked_64": blocked_64, "blocked_32": blocked_32,
             "spheres_96": spheres_96}

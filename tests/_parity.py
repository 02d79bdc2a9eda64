"""Shared helpers of the GPU parity tests.

The flux of a DFEM sweep crosses zero (the method allows negative nodal values)
and spans many decades, so a pointwise relative error is ill-posed at nodes
near zero.  The parity bar is the per-group max-norm relative error
||phi_g - ref_g||_inf / ||ref_g||_inf; pointwise relative errors are reported
only where |ref| is at least a fraction of the group maximum."""
import numpy as np


def norm_err(got, ref):
    """max over groups of ||got_g - ref_g||_inf / ||ref_g||_inf (arrays [G, ...] or [...])."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim < 3:
        got, ref = got[None], ref[None]
    worst = 0.0
    for g in range(ref.shape[0]):
        m = np.abs(ref[g]).max()
        d = np.abs(got[g] - ref[g]).max()
        worst = max(worst, d / m if m > 0 else d)
    return float(worst)


def point_err(got, ref, floor=1e-2):
    """max |got - ref| / |ref| over nodes with |ref| >= floor * group max."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim < 3:
        got, ref = got[None], ref[None]
    worst = 0.0
    for g in range(ref.shape[0]):
        m = np.abs(ref[g]).max()
        sel = np.abs(ref[g]) >= floor * m
        if sel.any():
            worst = max(worst, float((np.abs(got[g] - ref[g])[sel] / np.abs(ref[g])[sel]).max()))
    return worst


def rel_err(got, ref):
    """The parity measure used by the GPU tests (see the module docstring)."""
    return norm_err(got, ref)


def f32_roundtrip(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def network_sweep(wl, S, predict):
    """The sweep of Sec. 2 with every per-cell solve replaced by a one-cell solver
    (Sec. 4): cells in upwind order per direction, one-cell inputs in27 assembled
    from the upwind neighbours' outflow nodes or psi_inc, phi = sum_d w_d psi_d.
    predict(in27 [1, 27]) -> psi [1, 8] (physical node order).  Pure-Python loops:
    small meshes only."""
    import oracle

    nx, ny, nz = wl["nx"], wl["ny"], wl["nz"]
    h = (wl["lx"] / nx, wl["ly"] / ny, wl["lz"] / nz)
    om, w = oracle.lqn(wl["order"])
    G = wl["sigt"].shape[0]
    nc = nx * ny * nz
    phi = np.zeros((G, nc, 8))

    def node(ax, side, t):
        lo, hi = t & 1, (t >> 1) & 1
        abc = [lo, hi]
        abc.insert(ax, side)
        return abc[0] + 2 * abc[1] + 4 * abc[2]

    for g in range(G):
        for d in range(len(w)):
            o = om[d]
            psi = np.zeros((nc, 8))
            rng_axes = [range(n) if o[a] >= 0 else range(n - 1, -1, -1) for a, n in enumerate((nx, ny, nz))]
            for k in rng_axes[2]:
                for j in rng_axes[1]:
                    for i in rng_axes[0]:
                        c = i + nx * (j + ny * k)
                        x = np.zeros(27)
                        x[0:3], x[3:6], x[6] = o, h, wl["sigt"][g, c]
                        x[7:15] = S[g, c]
                        for a in range(3):
                            fin = 0 if o[a] >= 0 else 1
                            idx = [i, j, k]
                            idx[a] += -1 if fin == 0 else 1
                            if 0 <= idx[a] < (nx, ny, nz)[a]:
                                cu = idx[0] + nx * (idx[1] + ny * idx[2])
                                x[15 + 4 * a:19 + 4 * a] = [psi[cu, node(a, 1 - fin, t)] for t in range(4)]
                            else:
                                x[15 + 4 * a:19 + 4 * a] = wl["psi_inc"][g, 2 * a + fin]
                        psi[c] = predict(x[None, :])[0]
            phi[g] += w[d] * psi
    return phi

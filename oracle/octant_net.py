"""FP64 oracle of the paper's own surrogate: one small network per octant of
directions (Sec. 3, Eqs. (15)-(18); Sec. 4, the per-octant segmentation, the
loss of Eq. (19), Adam, and the connection-dropping of Sec. 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Inputs.  The independent quantities of the one-cell problem listed in Sec. 3,
in that order, in the problem's own (physical) frame:
  I[0:4]   psi_x^inc  upwind values on the inflow x-face (in-face order b + 2c)
  I[4:8]   psi_y^inc  (a + 2c)          I[8:12]  psi_z^inc  (a + 2b)
  I[12:14] mu, eta    the direction's x and y cosines (xi follows from the octant)
  I[14:22] q          nodal source density S (node order a + 2b + 4c)
  I[22]    sigma_t    I[23:26] dx, dy, dz
Octant o of a direction: bit 0 mu < 0, bit 1 eta < 0, bit 2 xi < 0; network o
serves the directions of octant o (Sec. 4).

Scaling (Eq. (16)): x_j = (I_j - alpha * m_j) / |I_j^max - I_j^min|, with m_j the
mean of I_j^min and I_j^max (the "norm" of Eq. (16) is defined as that mean) and
alpha = 0.27; the ranges are a-priori per input and per octant.

Network (Eqs. (15), (17), (18)): h = tanh(W1 x + b1), z = W2 h + b2,
psi_d = z_d if z_d >= 0, else beta (e^{z_d} - 1), beta = 0.1 * max |psi^inc| over
the cell's 12 upwind values.  The output is the angular flux itself (nodes in the
physical order), not a normalised value.

Loss (Eq. (19)): mean over the set of (1/8) sum_d |psi_d - psi^ANN_d| plus
lambda |sum_d (psi_d - psi^ANN_d)| / (gamma_1 |sum_d psi_d| + gamma_2) with
lambda = 0.2, gamma_1 = 10, gamma_2 = 0.01; the sub-gradient of |.| at 0 is 0.
Training: Adam (beta1 0.9, beta2 0.999, eps 1e-8), one full-batch step per epoch;
dropped connections are held at zero (the constraint function of Sec. 4).

Dropping connections (Sec. 3): drop the remaining connection (a weight of W1 or
W2; biases are not connections) of smallest magnitude, retrain, and keep the drop
while the training-set mean squared error stays within a factor (1 + tol) of the
fully connected network's, tol = 0.1 %; the first drop that exceeds it is undone
and the procedure stops.

Per-octant parameter vector (288): W1[8][26] row-major, b1[8], W2[8][8], b2[8].
"""
import numpy as np

from .mlp import Adam

NIN, NHID, NOUT = 26, 8, 8
NPARAM = NHID * NIN + NHID + NOUT * NHID + NOUT
NCONN = NHID * NIN + NOUT * NHID
ALPHA = 0.27
BETA_FRAC = 0.1
LAMBDA, GAMMA1, GAMMA2 = 0.2, 10.0, 0.01


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + NHID * NIN].reshape(NHID, NIN); o += NHID * NIN
    b1 = p[o:o + NHID]; o += NHID
    W2 = p[o:o + NOUT * NHID].reshape(NOUT, NHID); o += NOUT * NHID
    b2 = p[o:o + NOUT]
    return W1, b1, W2, b2


def pack(W1, b1, W2, b2):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2)])


def connection_mask():
    """1 on the entries of the parameter vector that are connections (W1, W2)."""
    return pack(np.ones((NHID, NIN)), np.zeros(NHID), np.ones((NOUT, NHID)), np.zeros(NOUT))


def glorot_init(seed=0):
    """Glorot-uniform weights (the initialisation of the network the paper builds
    on), zero biases."""
    rng = np.random.default_rng(seed)
    a1 = np.sqrt(6.0 / (NIN + NHID))
    a2 = np.sqrt(6.0 / (NHID + NOUT))
    return pack(rng.uniform(-a1, a1, (NHID, NIN)), np.zeros(NHID), rng.uniform(-a2, a2, (NOUT, NHID)),
                np.zeros(NOUT))


def octant_of(in27):
    om = np.atleast_2d(np.asarray(in27, dtype=np.float64))[:, 0:3]
    return ((om[:, 0] < 0).astype(np.int64) | ((om[:, 1] < 0).astype(np.int64) << 1)
            | ((om[:, 2] < 0).astype(np.int64) << 2))


def inputs(in27):
    """I [n, 26] of the one-cell problems in27 [n, 27] (layout of oracle.cell_solve)."""
    x = np.atleast_2d(np.asarray(in27, dtype=np.float64))
    I = np.empty((x.shape[0], NIN))
    I[:, 0:12] = x[:, 15:27]
    I[:, 12:14] = x[:, 0:2]
    I[:, 14:22] = x[:, 7:15]
    I[:, 22] = x[:, 6]
    I[:, 23:26] = x[:, 3:6]
    return I


def scale(I, lo, hi):
    """Eq. (16) with alpha = 0.27."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return (I - ALPHA * 0.5 * (lo + hi)) / np.abs(hi - lo)


def beta(in27):
    x = np.atleast_2d(np.asarray(in27, dtype=np.float64))
    return BETA_FRAC * np.abs(x[:, 15:27]).max(axis=1)


def elu(z, b):
    """Eq. (18): z for z >= 0, b (e^z - 1) below (b broadcast over the outputs)."""
    return np.where(z >= 0.0, z, b * np.expm1(np.minimum(z, 0.0)))


def forward(p, x, b):
    """One network on scaled inputs x [n, 26] with ELU scales b [n]:
    (psi [n, 8], hidden pre-activation, h, output pre-activation)."""
    W1, b1, W2, b2 = unpack(p)
    a = x @ W1.T + b1
    h = np.tanh(a)
    z = h @ W2.T + b2
    return elu(z, b[:, None]), a, h, z


def features(in27, lo, hi):
    """(x [n, 26], beta [n], octant [n]): each row scaled with its octant's ranges."""
    o = octant_of(in27)
    lo = np.asarray(lo, dtype=np.float64).reshape(8, NIN)
    hi = np.asarray(hi, dtype=np.float64).reshape(8, NIN)
    return scale(inputs(in27), lo[o], hi[o]), beta(in27), o


def predict(P, in27, lo, hi):
    """psi [n, 8] (physical node order) of the networks P [8, 288] on in27 [n, 27]."""
    P = np.asarray(P, dtype=np.float64).reshape(8, NPARAM)
    x, b, o = features(in27, lo, hi)
    out = np.empty((x.shape[0], NOUT))
    for k in range(8):
        sel = o == k
        if sel.any():
            out[sel] = forward(P[k], x[sel], b[sel])[0]
    return out


def loss(p, x, b, t):
    """Eq. (19) averaged over the set."""
    y = forward(p, x, b)[0]
    d = t - y
    mae = np.abs(d).mean(axis=1)
    reg = np.abs(d.sum(axis=1)) / (GAMMA1 * np.abs(t.sum(axis=1)) + GAMMA2)
    return float(np.mean(mae + LAMBDA * reg))


def loss_grad(p, x, b, t):
    """(loss, gradient [288]) of Eq. (19) by back-propagation through Eqs. (18), (17)."""
    W1, b1, W2, b2 = unpack(p)
    y, a, h, z = forward(p, x, b)
    n = x.shape[0]
    d = t - y
    den = GAMMA1 * np.abs(t.sum(axis=1)) + GAMMA2
    L = float(np.mean(np.abs(d).mean(axis=1) + LAMBDA * np.abs(d.sum(axis=1)) / den))
    gy = -(np.sign(d) / NOUT + LAMBDA * (np.sign(d.sum(axis=1)) / den)[:, None]) / n
    # d psi / d z: 1 above zero, b e^z below
    gz = gy * np.where(z >= 0.0, 1.0, b[:, None] * np.exp(np.minimum(z, 0.0)))
    gW2 = gz.T @ h
    gb2 = gz.sum(axis=0)
    ga = (gz @ W2) * (1.0 - h * h)
    gW1 = ga.T @ x
    gb1 = ga.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2)


def errors(p, x, b, t):
    """(mean absolute error, mean squared error) over rows and outputs."""
    d = t - forward(p, x, b)[0]
    return float(np.abs(d).mean()), float((d * d).mean())


def train(p, x, b, t, steps, lr, mask=None):
    """Full-batch Adam from a fresh optimiser state; entries with mask 0 stay 0."""
    p = np.array(p, dtype=np.float64)
    keep = np.ones(NPARAM) if mask is None else np.asarray(mask, dtype=np.float64)
    p *= keep
    opt = Adam(NPARAM, lr)
    for _ in range(steps):
        _, g = loss_grad(p, x, b, t)
        p = opt.step(p, g * keep) * keep
    return p


def prune(p, x, b, t, retrain_steps, lr, tol=1e-3, max_drops=None):
    """Connection dropping of Sec. 3 on one network.  Returns (params, mask, dropped
    connection indices in order, reference MSE, final MSE)."""
    p = np.array(p, dtype=np.float64)
    mask = np.ones(NPARAM)
    conn = connection_mask() > 0
    mse0 = errors(p, x, b, t)[1]
    mse = mse0
    dropped = []
    while max_drops is None or len(dropped) < max_drops:
        cand = np.flatnonzero(conn & (mask > 0))
        if cand.size == 0:
            break
        k = int(cand[np.argmin(np.abs(p[cand]))])
        m2 = mask.copy()
        m2[k] = 0.0
        p2 = train(p, x, b, t, retrain_steps, lr, m2)
        e2 = errors(p2, x, b, t)[1]
        if e2 > (1.0 + tol) * mse0:
            break
        p, mask, mse = p2, m2, e2
        dropped.append(k)
    return p, mask, dropped, mse0, mse

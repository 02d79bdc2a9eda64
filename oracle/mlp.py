"""FP64 oracle of the shallow-network surrogate (Sec. 3 and Sec. 4 of Tano & Ragusa).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The network follows Eq. (15): one hidden layer, h = f(W1 x + b1), o = W2 h + b2,
with the workload's shape 27 -> 64 (ReLU) -> 8.  The loss is Eq. (19): mean
absolute error plus lambda * |sum_d (psi_d - o_d)| / (gamma_1 |sum_d psi_d| +
gamma_2), lambda = 0.2, gamma_1 = 10, gamma_2 = 0.01 (the inner sum of the
denominator runs over the 8 nodes).  The optimiser is Adam.  The sub-gradient of
|.| at 0 is taken as 0.

Input construction (the analogue of the paper's input scaling, Eq. (16)): the
one-cell problem is first mirrored into the positive octant -- the DFEM system
of a direction with Omega_a < 0 is the system of |Omega_a| with the node order
reversed along axis a, so one network serves every octant -- and then
  x[0:3]  = 2 |Omega_a| - 1
  x[3:6]  = (log h_a + LOG_H_SHIFT) / LOG_H_SCALE
  x[6]    = log(max(sigma_t, SIG_FLOOR)) / LOG_SIG_SCALE
  x[7:15] = S_canonical / s,  x[15:27] = up_canonical / s,
  s = max(max|S|, max|up|)   (the "normalised by the inflow/source max" scale)
and the network predicts psi_canonical / s.  A problem with s = 0 has psi = 0; a scale
at or below 1e-30 is treated as 0 (inputs and target scaled by 0).

Parameter vector (2312 values): W1[64][27] row-major, b1[64], W2[8][64], b2[8].
"""
import numpy as np

NIN, NHID, NOUT = 27, 64, 8
NPARAM = NHID * NIN + NHID + NOUT * NHID + NOUT
LAMBDA, GAMMA1, GAMMA2 = 0.2, 10.0, 0.01
LOG_H_SHIFT, LOG_H_SCALE = 1.15, 1.15
LOG_SIG_SCALE, SIG_FLOOR = 4.5, 1e-6
# an input scale at or below this counts as zero (a flux that FP32 cannot hold)
SCALE_FLOOR = 1e-30


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


def init_params(seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)
    a1, a2 = 1.0 / np.sqrt(NIN), 1.0 / np.sqrt(NHID)
    return pack(rng.uniform(-a1, a1, (NHID, NIN)), rng.uniform(-a1, a1, NHID),
                rng.uniform(-a2, a2, (NOUT, NHID)), rng.uniform(-a2, a2, NOUT))


def mirror_masks(in27):
    om = np.asarray(in27)[:, 0:3]
    fx = (om[:, 0] < 0).astype(np.int64)
    fy = (om[:, 1] < 0).astype(np.int64)
    fz = (om[:, 2] < 0).astype(np.int64)
    return fx, fy, fz


def canonical(in27):
    """Mirror each one-cell problem into the positive octant.
    Returns (|Omega| [n,3], h [n,3], sigma_t [n], S_c [n,8], up_c [n,12], node mask [n])."""
    x = np.asarray(in27, dtype=np.float64)
    fx, fy, fz = mirror_masks(x)
    mask = fx | (fy << 1) | (fz << 2)
    k = np.arange(8)
    S = np.take_along_axis(x[:, 7:15], k[None, :] ^ mask[:, None], 1)
    t = np.arange(4)
    ux = np.take_along_axis(x[:, 15:19], t[None, :] ^ (fy | (fz << 1))[:, None], 1)
    uy = np.take_along_axis(x[:, 19:23], t[None, :] ^ (fx | (fz << 1))[:, None], 1)
    uz = np.take_along_axis(x[:, 23:27], t[None, :] ^ (fx | (fy << 1))[:, None], 1)
    return np.abs(x[:, 0:3]), x[:, 3:6], x[:, 6], S, np.concatenate([ux, uy, uz], 1), mask


def features(in27):
    """(x [n,27], s [n], mask [n]) of the input construction in the module docstring."""
    aom, h, sig, S, U, mask = canonical(in27)
    s = np.maximum(np.abs(S).max(1), np.abs(U).max(1))
    inv = np.where(s > SCALE_FLOOR, 1.0 / np.where(s > SCALE_FLOOR, s, 1.0), 0.0)
    x = np.empty((aom.shape[0], NIN))
    x[:, 0:3] = 2.0 * aom - 1.0
    x[:, 3:6] = (np.log(h) + LOG_H_SHIFT) / LOG_H_SCALE
    x[:, 6] = np.log(np.maximum(sig, SIG_FLOOR)) / LOG_SIG_SCALE
    x[:, 7:15] = S * inv[:, None]
    x[:, 15:27] = U * inv[:, None]
    return x, s, mask


def targets(psi, in27):
    """psi (physical node order) -> canonical psi / s, the network's target."""
    _, s, mask = features(in27)
    k = np.arange(8)
    pc = np.take_along_axis(np.asarray(psi, dtype=np.float64), k[None, :] ^ mask[:, None], 1)
    inv = np.where(s > SCALE_FLOOR, 1.0 / np.where(s > SCALE_FLOOR, s, 1.0), 0.0)
    return pc * inv[:, None]


def forward(p, x):
    """Eq. (15) with ReLU hidden units and linear outputs: returns (o, pre-activation, h)."""
    W1, b1, W2, b2 = unpack(p)
    a = x @ W1.T + b1
    h = np.maximum(a, 0.0)
    return h @ W2.T + b2, a, h


def predict(p, in27):
    """psi [n, 8] in physical node order from the network."""
    x, s, mask = features(in27)
    o, _, _ = forward(p, x)
    k = np.arange(8)
    return np.take_along_axis(o * s[:, None], k[None, :] ^ mask[:, None], 1)


def loss(p, x, t):
    """Eq. (19) averaged over the batch."""
    o, _, _ = forward(p, x)
    d = t - o
    mae = np.abs(d).mean(axis=1)
    reg = np.abs(d.sum(axis=1)) / (GAMMA1 * np.abs(t.sum(axis=1)) + GAMMA2)
    return float(np.mean(mae + LAMBDA * reg))


def loss_grad(p, x, t):
    """(loss, gradient [NPARAM]) of Eq. (19) by back-propagation."""
    W1, b1, W2, b2 = unpack(p)
    o, a, h = forward(p, x)
    n = x.shape[0]
    d = t - o
    mae = np.abs(d).mean(axis=1)
    den = GAMMA1 * np.abs(t.sum(axis=1)) + GAMMA2
    reg = np.abs(d.sum(axis=1)) / den
    L = float(np.mean(mae + LAMBDA * reg))
    # dL/do = -(1/n) [ sign(d)/8 + lambda sign(sum d) / den ]
    go = -(np.sign(d) / NOUT + LAMBDA * (np.sign(d.sum(axis=1)) / den)[:, None]) / n
    gW2 = go.T @ h
    gb2 = go.sum(axis=0)
    gh = go @ W2
    ga = gh * (a > 0)
    gW1 = ga.T @ x
    gb1 = ga.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2)


class Adam:
    """Adam (Kingma & Ba) with bias correction; beta1 0.9, beta2 0.999, eps 1e-8."""

    def __init__(self, n, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, p, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return p - self.lr * mh / (np.sqrt(vh) + self.eps)


def train(p, x, t, steps, batch, lr):
    """Plain mini-batch Adam: batch k takes rows [(k*batch) mod n, +batch) in order
    (wrapping), the schedule the GPU trainer uses."""
    opt = Adam(p.size, lr)
    n = x.shape[0]
    for k in range(steps):
        idx = (np.arange(batch) + k * batch) % n
        _, g = loss_grad(p, x[idx], t[idx])
        p = opt.step(p, g)
    return p

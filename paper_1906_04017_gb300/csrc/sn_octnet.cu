// sn_octnet.cu -- the paper's own surrogate: one 26 -> 8 (tanh) -> 8 (ELU) network per
// octant of directions (Sec. 3, Eqs. (15)-(18); Sec. 4), trained on one-cell problems
// labelled by the library's elimination with the loss of Eq. (19) and full-batch Adam,
// thinned by the connection dropping of Sec. 3, and evaluated in FP32 on the CUDA
// cores.  A network costs 272 multiply-adds a cell: at M = 8 hidden units there is no
// tile a tensor-core instruction could fill, and the weights of an octant (1.1 KB)
// sit in shared memory, read as broadcasts by every thread of the CTA.
//
// Parameters of octant o (288 FP32, physical frame): W1[8][26], b1[8], W2[8][8], b2[8];
// the inputs of the networks and their scaling are described in octnet.cuh.  The
// sweeps and sn_octnet_apply read the folded copies (octnet.cuh), rebuilt whenever the
// parameters change.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cell_problem.cuh"
#include "octnet.cuh"
#include "sn_internal.cuh"

namespace sn {

struct OctNet {
    float *p = nullptr;        // [8][288] parameters, dropped connections held at 0
    float *mask = nullptr;     // [8][288] 1 trainable, 0 dropped
    float *m = nullptr, *v = nullptr;   // Adam moments
    int64_t t = 0;             // Adam steps since the last reset
    float *shift = nullptr;    // [8][26] alpha (lo + hi) / 2
    float *inv_r = nullptr;    // [8][26] 1 / |hi - lo|
    float *fold = nullptr;     // [8][288] folded networks (canonical frame)
    float *gpart = nullptr;    // [8][B][288] per-CTA gradient partials
    double *lpart = nullptr;   // [8][B] loss partials
    double *epart = nullptr;   // [8][B][2] error partials
    int64_t part_blocks = 0;
    double *loss = nullptr;    // [8] Eq. (19) of the last gradient
    int *flag = nullptr;       // rows found outside their octant by prepare
    bool ranges = false;       // input ranges set
};

static OctNet *onet_of(sn_handle h) { return reinterpret_cast<OctNet *>(h->octnet); }

void free_octnet(sn_handle h)
{
    if (!h || !h->octnet) return;
    OctNet *n = onet_of(h);
    void *bufs[] = {n->p, n->mask, n->m, n->v, n->shift, n->inv_r, n->fold, n->gpart, n->lpart, n->epart, n->loss,
                    n->flag};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete n;
    h->octnet = nullptr;
    h->has_octnet = false;
}

static sn_status ensure_octnet(sn_handle h)
{
    if (h->octnet) return SN_OK;
    OctNet *n = new OctNet();
    h->octnet = n;
    const size_t P = sizeof(float) * 8 * kOnParam;
    SN_CK(h, cudaMalloc(&n->p, P));
    SN_CK(h, cudaMalloc(&n->mask, P));
    SN_CK(h, cudaMalloc(&n->m, P));
    SN_CK(h, cudaMalloc(&n->v, P));
    SN_CK(h, cudaMalloc(&n->fold, sizeof(float) * 8 * kOnFold));
    SN_CK(h, cudaMalloc(&n->shift, sizeof(float) * 8 * kOnIn));
    SN_CK(h, cudaMalloc(&n->inv_r, sizeof(float) * 8 * kOnIn));
    SN_CK(h, cudaMalloc(&n->loss, sizeof(double) * 8));
    SN_CK(h, cudaMalloc(&n->flag, sizeof(int)));
    return SN_OK;
}

// --------------------------------------------------------------------------------
// Training data.  Rows [o m, (o + 1) m) of in27 belong to octant o.  feat row: the 26
// scaled inputs (Eq. (16)) and beta; targ row: the FP32 elimination solution
// (GE32R, physical node order).
// --------------------------------------------------------------------------------
__device__ __forceinline__ int octant_of(const float *p)
{
    return (p[0] < 0.f) | ((p[1] < 0.f) << 1) | ((p[2] < 0.f) << 2);
}

__global__ void __launch_bounds__(128) octnet_prepare_kernel(const float *__restrict__ in27, int64_t m,
                                                             const float *__restrict__ shift,
                                                             const float *__restrict__ inv_r,
                                                             float *__restrict__ feat, float *__restrict__ targ,
                                                             int *__restrict__ flag)
{
    const int64_t n = 8 * m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float *p = in27 + 27 * i;
        const int o = octant_of(p);
        if (o != (int)(i / m)) atomicOr(flag, 1);
        float I[kOnIn];
#pragma unroll
        for (int t = 0; t < 12; ++t) I[t] = p[15 + t];
        I[12] = p[0];
        I[13] = p[1];
#pragma unroll
        for (int k = 0; k < 8; ++k) I[14 + k] = p[7 + k];
        I[22] = p[6];
        I[23] = p[3]; I[24] = p[4]; I[25] = p[5];
        float *f = feat + 27 * i;
        float bm = 0.f;
#pragma unroll
        for (int j = 0; j < kOnIn; ++j) f[j] = (I[j] - shift[kOnIn * o + j]) * inv_r[kOnIn * o + j];
#pragma unroll
        for (int t = 0; t < 12; ++t) bm = fmaxf(bm, fabsf(p[15 + t]));
        f[26] = kOnBetaFrac * bm;
        float psi[8];
        solve_in27<float, true>(p, psi);
#pragma unroll
        for (int k = 0; k < 8; ++k) targ[8 * i + k] = psi[k];
    }
}

// --------------------------------------------------------------------------------
// Loss (19) and its gradient for the 8 networks.  grid = (B, 8): CTA (b, o) takes the
// 128-row chunks b, b + B, ... of octant o; each thread forwards and back-propagates
// one row, then the CTA forms its partial gradient from the rows' activations and
// deltas in shared memory (3 of the 288 entries a thread, accumulated over chunks).
// --------------------------------------------------------------------------------
constexpr float kOnLambda = 0.2f, kOnGamma1 = 10.f, kOnGamma2 = 0.01f;
constexpr int kOnXs = 27, kOnHs = 9;

__device__ __forceinline__ float sgn1(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

// forward of a physical-frame network on scaled inputs x: hidden h, pre-activation z, output y
__device__ __forceinline__ void octnet_phys_forward(const float *__restrict__ P, const float (&x)[kOnIn], float beta,
                                                    float (&h)[kOnHid], float (&z)[kOnOut], float (&y)[kOnOut])
{
#pragma unroll
    for (int k = 0; k < kOnHid; ++k) {
        float a = P[kOnB1 + k];
#pragma unroll
        for (int j = 0; j < kOnIn; ++j) a = fmaf(P[kOnW1 + kOnIn * k + j], x[j], a);
        h[k] = octnet_tanh(a);
    }
#pragma unroll
    for (int t = 0; t < kOnOut; ++t) {
        float a = P[kOnB2 + t];
#pragma unroll
        for (int k = 0; k < kOnHid; ++k) a = fmaf(P[kOnW2 + kOnHid * t + k], h[k], a);
        z[t] = a;
        y[t] = a >= 0.f ? a : beta * (__expf(a) - 1.f);
    }
}

__global__ void __launch_bounds__(128) octnet_grad_kernel(const float *__restrict__ Pall,
                                                          const float *__restrict__ feat,
                                                          const float *__restrict__ targ, int64_t m, float inv_m,
                                                          float *__restrict__ gpart, double *__restrict__ lpart)
{
    __shared__ float sP[kOnParam];
    __shared__ float sX[128 * kOnXs], sH[128 * kOnHs], sGA[128 * kOnHs], sGZ[128 * kOnHs];
    __shared__ double sl[4];
    const int o = blockIdx.y, B = gridDim.x, t = threadIdx.x;
    for (int e = t; e < kOnParam; e += 128) sP[e] = Pall[kOnParam * o + e];
    float acc[3] = {0.f, 0.f, 0.f};
    double lsum = 0.0;
    const int64_t base = (int64_t)o * m;
    for (int64_t c0 = (int64_t)blockIdx.x * 128; c0 < m; c0 += (int64_t)B * 128) {
        __syncthreads();   // sP loaded; the previous chunk's rows consumed
        const int64_t i = c0 + t;
        float *xr = sX + t * kOnXs, *hr = sH + t * kOnHs, *gar = sGA + t * kOnHs, *gzr = sGZ + t * kOnHs;
        if (i < m) {
            const float *f = feat + 27 * (base + i);
            const float *tg = targ + 8 * (base + i);
            float x[kOnIn], h[kOnHid], z[kOnOut], y[kOnOut];
#pragma unroll
            for (int j = 0; j < kOnIn; ++j) { x[j] = f[j]; xr[j] = x[j]; }
            const float beta = f[26];
            octnet_phys_forward(sP, x, beta, h, z, y);
            float d[kOnOut], sd = 0.f, st = 0.f, mae = 0.f;
#pragma unroll
            for (int q = 0; q < kOnOut; ++q) {
                const float tt = tg[q];
                d[q] = tt - y[q];
                sd += d[q];
                st += tt;
                mae += fabsf(d[q]);
            }
            const float den = kOnGamma1 * fabsf(st) + kOnGamma2;
            lsum += (double)((mae / 8.f + kOnLambda * fabsf(sd) / den) * inv_m);
            float gz[kOnOut];
#pragma unroll
            for (int q = 0; q < kOnOut; ++q) {
                const float gy = -(sgn1(d[q]) / 8.f + kOnLambda * sgn1(sd) / den) * inv_m;
                // d theta / dz: 1 above zero, beta e^z = y + beta below
                gz[q] = gy * (z[q] >= 0.f ? 1.f : y[q] + beta);
                gzr[q] = gz[q];
            }
#pragma unroll
            for (int k = 0; k < kOnHid; ++k) {
                float gh = 0.f;
#pragma unroll
                for (int q = 0; q < kOnOut; ++q) gh = fmaf(gz[q], sP[kOnW2 + kOnHid * q + k], gh);
                gar[k] = gh * (1.f - h[k] * h[k]);
                hr[k] = h[k];
            }
        } else {
#pragma unroll
            for (int j = 0; j < kOnIn; ++j) xr[j] = 0.f;
#pragma unroll
            for (int k = 0; k < kOnHid; ++k) { hr[k] = 0.f; gar[k] = 0.f; gzr[k] = 0.f; }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int e = t + 128 * r;
            if (e >= kOnParam) break;
            float a = 0.f;
            if (e < kOnB1) {
                const int k = e / kOnIn, j = e - k * kOnIn;
                for (int s = 0; s < 128; ++s) a = fmaf(sGA[s * kOnHs + k], sX[s * kOnXs + j], a);
            } else if (e < kOnW2) {
                const int k = e - kOnB1;
                for (int s = 0; s < 128; ++s) a += sGA[s * kOnHs + k];
            } else if (e < kOnB2) {
                const int q = (e - kOnW2) / kOnHid, k = (e - kOnW2) % kOnHid;
                for (int s = 0; s < 128; ++s) a = fmaf(sGZ[s * kOnHs + q], sH[s * kOnHs + k], a);
            } else {
                const int q = e - kOnB2;
                for (int s = 0; s < 128; ++s) a += sGZ[s * kOnHs + q];
            }
            acc[r] += a;
        }
    }
    float *gp = gpart + ((int64_t)o * B + blockIdx.x) * kOnParam;
#pragma unroll
    for (int r = 0; r < 3; ++r)
        if (t + 128 * r < kOnParam) gp[t + 128 * r] = acc[r];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
    __syncthreads();
    if ((t & 31) == 0) sl[t >> 5] = lsum;
    __syncthreads();
    if (t == 0) lpart[(int64_t)o * B + blockIdx.x] = sl[0] + sl[1] + sl[2] + sl[3];
}

// One CTA per octant, one thread per parameter: sum the partials in a fixed order,
// optionally hand the gradient out, then (for the octants in `active`) one Adam step
// with dropped connections held at zero (the constraint of Sec. 4).
__global__ void __launch_bounds__(kOnParam) octnet_adam_kernel(float *__restrict__ P, float *__restrict__ M,
                                                               float *__restrict__ V, const float *__restrict__ mask,
                                                               const float *__restrict__ gpart,
                                                               const double *__restrict__ lpart, int B, float lr,
                                                               float bc1, float bc2, int active, int do_step,
                                                               float *__restrict__ gout, double *__restrict__ loss)
{
    const int o = blockIdx.x, e = threadIdx.x;
    const int64_t q = (int64_t)kOnParam * o + e;
    double g = 0.0;
    for (int b = 0; b < B; ++b) g += (double)gpart[((int64_t)o * B + b) * kOnParam + e];
    if (e == 0) {
        double l = 0.0;
        for (int b = 0; b < B; ++b) l += lpart[(int64_t)o * B + b];
        loss[o] = l;
    }
    const float gf = (float)g;
    if (gout) gout[q] = gf;
    if (!do_step || !((active >> o) & 1)) return;
    const float k = mask[q];
    const float gm = gf * k;
    const float mm = 0.9f * M[q] + 0.1f * gm;
    const float vv = 0.999f * V[q] + 0.001f * gm * gm;
    M[q] = mm;
    V[q] = vv;
    P[q] = (P[q] - lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f)) * k;
}

// Sums of |psi - psi^ANN| and of its square, per CTA of grid (B, 8).
__global__ void __launch_bounds__(128) octnet_eval_kernel(const float *__restrict__ Pall,
                                                          const float *__restrict__ feat,
                                                          const float *__restrict__ targ, int64_t m,
                                                          double *__restrict__ epart)
{
    __shared__ float sP[kOnParam];
    __shared__ double sa[4], sq[4];
    const int o = blockIdx.y, B = gridDim.x, t = threadIdx.x;
    for (int e = t; e < kOnParam; e += 128) sP[e] = Pall[kOnParam * o + e];
    double ab = 0.0, sqr = 0.0;
    const int64_t base = (int64_t)o * m;
    for (int64_t c0 = (int64_t)blockIdx.x * 128; c0 < m; c0 += (int64_t)B * 128) {
        // a barrier per chunk also keeps the weight reads inside the loop (hoisted,
        // they would need 288 registers)
        __syncthreads();
        const int64_t i = c0 + t;
        if (i >= m) continue;
        const float *f = feat + 27 * (base + i);
        float x[kOnIn], h[kOnHid], z[kOnOut], y[kOnOut];
#pragma unroll
        for (int j = 0; j < kOnIn; ++j) x[j] = f[j];
        octnet_phys_forward(sP, x, f[26], h, z, y);
        float a = 0.f, s2 = 0.f;
#pragma unroll
        for (int q = 0; q < kOnOut; ++q) {
            const float d = targ[8 * (base + i) + q] - y[q];
            a += fabsf(d);
            s2 = fmaf(d, d, s2);
        }
        ab += (double)a;
        sqr += (double)s2;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ab += __shfl_down_sync(0xffffffffu, ab, off);
        sqr += __shfl_down_sync(0xffffffffu, sqr, off);
    }
    if ((t & 31) == 0) { sa[t >> 5] = ab; sq[t >> 5] = sqr; }
    __syncthreads();
    if (t == 0) {
        double *ep = epart + ((int64_t)o * B + blockIdx.x) * 2;
        ep[0] = sa[0] + sa[1] + sa[2] + sa[3];
        ep[1] = sq[0] + sq[1] + sq[2] + sq[3];
    }
}

// Folded network of octant o (layout in octnet.cuh): one thread per folded entry.
// Input j of the physical network enters as (I_j - shift_j) inv_r_j, so its
// coefficient is W1[k][j] inv_r_j and the bias gains -W1[k][j] shift_j inv_r_j; the
// canonical value of a mirrored face value, source or output sits at the physical
// index XOR the axis mask, and |mu| = -mu on a flipped axis.
__global__ void __launch_bounds__(kOnFold) octnet_fold_kernel(const float *__restrict__ Pall,
                                                              const float *__restrict__ shift,
                                                              const float *__restrict__ inv_r,
                                                              float *__restrict__ fold)
{
    const int o = blockIdx.x, e = threadIdx.x;
    const float *P = Pall + kOnParam * o, *sh = shift + kOnIn * o, *ir = inv_r + kOnIn * o;
    const int fx = o & 1, fy = (o >> 1) & 1, fz = (o >> 2) & 1;
    float v;
    if (e < kOnFoldH) {
        const int k = e / 24, s = e % 24;
        const float *w = P + kOnW1 + kOnIn * k;
        if (s == 23) {
            double b = P[kOnB1 + k];
            for (int j = 0; j < kOnIn; ++j) b -= (double)w[j] * (double)sh[j] * (double)ir[j];
            v = (float)b;
        } else {
            int j;
            float sign = 1.f;
            if (s < 4) j = s ^ (fy | (fz << 1));
            else if (s < 8) j = 4 + ((s - 4) ^ (fx | (fz << 1)));
            else if (s < 12) j = 8 + ((s - 8) ^ (fx | (fy << 1)));
            else if (s < 20) j = 14 + ((s - 12) ^ o);
            else if (s == 20) { j = 12; sign = fx ? -1.f : 1.f; }
            else if (s == 21) { j = 13; sign = fy ? -1.f : 1.f; }
            else j = 22;
            v = sign * w[j] * ir[j];
        }
    } else if (e < kOnFoldW2) {
        const int k = (e - kOnFoldH) / 3, a = (e - kOnFoldH) % 3;
        v = P[kOnW1 + kOnIn * k + 23 + a] * ir[23 + a];
    } else if (e < kOnFoldB2) {
        const int tc = (e - kOnFoldW2) / kOnHid, k = (e - kOnFoldW2) % kOnHid;
        v = P[kOnW2 + kOnHid * (tc ^ o) + k];
    } else {
        v = P[kOnB2 + ((e - kOnFoldB2) ^ o)];
    }
    fold[kOnFold * o + e] = v;
}

// Batches of one-cell problems through the folded network of each problem's octant
// (the same evaluation the sweep runs), inputs staged through shared memory.
__global__ void __launch_bounds__(128) octnet_cells_kernel(const float *__restrict__ fold,
                                                           const float *__restrict__ in27, float *__restrict__ out,
                                                           int64_t n)
{
    __shared__ float stage[128 * 27];
    for (int64_t base = (int64_t)blockIdx.x * 128; base < n; base += (int64_t)gridDim.x * 128) {
        const int64_t cnt = n - base < 128 ? n - base : 128;
        __syncthreads();
        for (int64_t e = threadIdx.x; e < cnt * 27; e += 128) stage[e] = in27[base * 27 + e];
        __syncthreads();
        if (threadIdx.x < cnt) {
            const float *p = stage + threadIdx.x * 27;
            CanonCell<float> c;
            canonicalize(p, c);
            float psi[8];
            octnet_forward<true>(fold + kOnFold * c.mask, c.ux, c.uy, c.uz, c.S, fabsf(p[0]), fabsf(p[1]), c.sig,
                                 p[3], p[4], p[5], psi);
            mirror8(psi, c.mask);
            float *o = out + (base + threadIdx.x) * 8;
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = psi[k];
        }
    }
}

static int blocks_per_octant(int64_t m)
{
    const int64_t chunks = (m + 127) / 128;
    const int64_t cap = std::max<int64_t>(1, (int64_t)num_sms() * 6 / 8);
    return (int)std::max<int64_t>(1, std::min(chunks, cap));
}

static sn_status ensure_parts(sn_handle h, int B)
{
    OctNet *n = onet_of(h);
    if (n->part_blocks >= B) return SN_OK;
    if (n->gpart) cudaFree(n->gpart);
    if (n->lpart) cudaFree(n->lpart);
    if (n->epart) cudaFree(n->epart);
    n->gpart = nullptr;
    n->lpart = nullptr;
    n->epart = nullptr;
    n->part_blocks = 0;
    SN_CK(h, cudaMalloc(&n->gpart, sizeof(float) * 8 * (size_t)B * kOnParam));
    SN_CK(h, cudaMalloc(&n->lpart, sizeof(double) * 8 * (size_t)B));
    SN_CK(h, cudaMalloc(&n->epart, sizeof(double) * 16 * (size_t)B));
    n->part_blocks = B;
    return SN_OK;
}

static sn_status refold(sn_handle h, cudaStream_t st)
{
    OctNet *n = onet_of(h);
    octnet_fold_kernel<<<8, kOnFold, 0, st>>>(n->p, n->shift, n->inv_r, n->fold);
    SN_CK(h, cudaGetLastError());
    h->net_gen++;
    return SN_OK;
}

// gradient (and optionally one Adam step of the octants in `active`) over all rows
static sn_status grad_step(sn_handle h, const float *feat, const float *targ, int64_t m, float lr, bool step,
                           int active, float *gout, cudaStream_t st)
{
    OctNet *n = onet_of(h);
    const int B = blocks_per_octant(m);
    sn_status s = ensure_parts(h, B);
    if (s != SN_OK) return s;
    octnet_grad_kernel<<<dim3(B, 8), 128, 0, st>>>(n->p, feat, targ, m, 1.f / (float)m, n->gpart, n->lpart);
    float bc1 = 1.f, bc2 = 1.f;
    if (step) {
        n->t += 1;
        bc1 = (float)(1.0 - std::pow(0.9, (double)n->t));
        bc2 = (float)(1.0 - std::pow(0.999, (double)n->t));
    }
    octnet_adam_kernel<<<8, kOnParam, 0, st>>>(n->p, n->m, n->v, n->mask, n->gpart, n->lpart, B, lr, bc1, bc2,
                                                active, step ? 1 : 0, gout, n->loss);
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

static sn_status reset_adam(sn_handle h, cudaStream_t st)
{
    OctNet *n = onet_of(h);
    SN_CK(h, cudaMemsetAsync(n->m, 0, sizeof(float) * 8 * kOnParam, st));
    SN_CK(h, cudaMemsetAsync(n->v, 0, sizeof(float) * 8 * kOnParam, st));
    n->t = 0;
    return SN_OK;
}

// per-octant mean absolute and mean squared error (over rows and the 8 outputs)
static sn_status errors(sn_handle h, const float *feat, const float *targ, int64_t m, double *mae, double *mse,
                        cudaStream_t st)
{
    OctNet *n = onet_of(h);
    const int B = blocks_per_octant(m);
    sn_status s = ensure_parts(h, B);
    if (s != SN_OK) return s;
    octnet_eval_kernel<<<dim3(B, 8), 128, 0, st>>>(n->p, feat, targ, m, n->epart);
    SN_CK(h, cudaGetLastError());
    std::vector<double> ep(16 * (size_t)B);
    SN_CK(h, cudaMemcpyAsync(ep.data(), n->epart, sizeof(double) * ep.size(), cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    for (int o = 0; o < 8; ++o) {
        double a = 0.0, q = 0.0;
        for (int b = 0; b < B; ++b) {
            a += ep[((size_t)o * B + b) * 2];
            q += ep[((size_t)o * B + b) * 2 + 1];
        }
        if (mae) mae[o] = a / (8.0 * (double)m);
        if (mse) mse[o] = q / (8.0 * (double)m);
    }
    return SN_OK;
}

static sn_status set_ranges(sn_handle h, const double *lo, const double *hi, cudaStream_t st)
{
    std::vector<float> sh(8 * kOnIn), ir(8 * kOnIn);
    for (int e = 0; e < 8 * kOnIn; ++e) {
        const double a = lo[e], b = hi[e];
        if (!std::isfinite(a) || !std::isfinite(b) || a == b)
            return fail(h, SN_EINVAL, "octant networks: every input range needs finite, distinct ends");
        sh[e] = (float)((double)kOnAlpha * 0.5 * (a + b));
        ir[e] = (float)(1.0 / std::fabs(b - a));
    }
    OctNet *n = onet_of(h);
    SN_CK(h, cudaMemcpyAsync(n->shift, sh.data(), sizeof(float) * sh.size(), cudaMemcpyHostToDevice, st));
    SN_CK(h, cudaMemcpyAsync(n->inv_r, ir.data(), sizeof(float) * ir.size(), cudaMemcpyHostToDevice, st));
    SN_CK(h, cudaStreamSynchronize(st));
    n->ranges = true;
    return SN_OK;
}

static sn_status upload(sn_handle h, const std::vector<float> &p, const std::vector<float> &mask, cudaStream_t st)
{
    OctNet *n = onet_of(h);
    SN_CK(h, cudaMemcpyAsync(n->p, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice, st));
    SN_CK(h, cudaMemcpyAsync(n->mask, mask.data(), sizeof(float) * mask.size(), cudaMemcpyHostToDevice, st));
    SN_CK(h, cudaStreamSynchronize(st));
    return SN_OK;
}

static sn_status download(sn_handle h, std::vector<float> &p, std::vector<float> &mask, cudaStream_t st)
{
    OctNet *n = onet_of(h);
    p.resize(8 * kOnParam);
    mask.resize(8 * kOnParam);
    SN_CK(h, cudaMemcpyAsync(p.data(), n->p, sizeof(float) * p.size(), cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaMemcpyAsync(mask.data(), n->mask, sizeof(float) * mask.size(), cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    return SN_OK;
}

static sn_status need_octnet(sn_handle h, const char *who)
{
    if (!h) return fail(nullptr, SN_EINVAL, std::string(who) + ": NULL handle");
    if (!h->has_octnet) return fail(h, SN_ESTATE, std::string(who) + ": no octant networks (init or set first)");
    return SN_OK;
}

static sn_status check_rows(sn_handle h, const float *feat, const float *targ, int64_t m, const char *who)
{
    if (m < 1 || m > (1LL << 28)) return fail(h, SN_EINVAL, std::string(who) + ": rows per octant must be in 1..2^28");
    if (!feat || !targ) return fail(h, SN_EINVAL, std::string(who) + ": NULL pointer");
    return SN_OK;
}

sn_status launch_octnet_cells(sn_handle h, const float *in27, float *psi, int64_t n, cudaStream_t st)
{
    if (n <= 0) return SN_OK;
    int64_t grid = (n + 127) / 128;
    if (grid > (int64_t)num_sms() * 16) grid = (int64_t)num_sms() * 16;
    octnet_cells_kernel<<<(unsigned)grid, 128, 0, st>>>(onet_of(h)->fold, in27, psi, n);
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

const float *octnet_folded(sn_handle h) { return h->octnet ? onet_of(h)->fold : nullptr; }

}  // namespace sn

using namespace sn;

extern "C" {

sn_status sn_octnet_init(sn_handle h, const double *lo, const double *hi, uint64_t seed)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_octnet_init: NULL handle");
    if (!lo || !hi) return fail(h, SN_EINVAL, "sn_octnet_init: NULL ranges");
    const cudaStream_t st = h->stream;
    sn_status s = ensure_octnet(h);
    if (s == SN_OK) s = set_ranges(h, lo, hi, st);
    if (s != SN_OK) return s;
    // Glorot-uniform weights from a SplitMix64 stream, zero biases
    uint64_t x = seed;
    auto next = [&x]() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    std::vector<float> p(8 * kOnParam, 0.f), mask(8 * kOnParam, 1.f);
    const double a1 = std::sqrt(6.0 / (kOnIn + kOnHid)), a2 = std::sqrt(6.0 / (kOnHid + kOnOut));
    for (int o = 0; o < 8; ++o) {
        float *q = p.data() + kOnParam * o;
        for (int e = kOnW1; e < kOnB1; ++e) q[e] = (float)((2.0 * next() - 1.0) * a1);
        for (int e = kOnW2; e < kOnB2; ++e) q[e] = (float)((2.0 * next() - 1.0) * a2);
    }
    s = upload(h, p, mask, st);
    if (s == SN_OK) s = reset_adam(h, st);
    if (s == SN_OK) s = refold(h, st);
    if (s != SN_OK) return s;
    SN_CK(h, cudaStreamSynchronize(st));
    h->has_octnet = true;
    return SN_OK;
}

sn_status sn_octnet_set(sn_handle h, const float *params, const float *mask, const double *lo, const double *hi)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_octnet_set: NULL handle");
    if (!params) return fail(h, SN_EINVAL, "sn_octnet_set: NULL params");
    if (!lo != !hi) return fail(h, SN_EINVAL, "sn_octnet_set: give both range arrays or neither");
    const cudaStream_t st = h->stream;
    sn_status s = ensure_octnet(h);
    if (s != SN_OK) return s;
    if (lo) {
        s = set_ranges(h, lo, hi, st);
        if (s != SN_OK) return s;
    } else if (!onet_of(h)->ranges) {
        return fail(h, SN_ESTATE, "sn_octnet_set: no input ranges yet");
    }
    std::vector<float> p(params, params + 8 * kOnParam), k(8 * kOnParam, 1.f);
    for (int e = 0; e < 8 * kOnParam; ++e) {
        if (mask) {
            if (mask[e] != 0.f && mask[e] != 1.f) return fail(h, SN_EINVAL, "sn_octnet_set: mask entries are 0 or 1");
            k[e] = mask[e];
        }
        if (!std::isfinite(p[e])) return fail(h, SN_EINVAL, "sn_octnet_set: non-finite parameter");
        p[e] *= k[e];
    }
    s = upload(h, p, k, st);
    if (s == SN_OK) s = reset_adam(h, st);
    if (s == SN_OK) s = refold(h, st);
    if (s != SN_OK) return s;
    SN_CK(h, cudaStreamSynchronize(st));
    h->has_octnet = true;
    return SN_OK;
}

sn_status sn_octnet_get(sn_handle h, float *params, float *mask)
{
    sn_status s = need_octnet(h, "sn_octnet_get");
    if (s != SN_OK) return s;
    std::vector<float> p, k;
    s = download(h, p, k, h->stream);
    if (s != SN_OK) return s;
    if (params) std::copy(p.begin(), p.end(), params);
    if (mask) std::copy(k.begin(), k.end(), mask);
    return SN_OK;
}

sn_status sn_octnet_prepare(sn_handle h, const float *in27, int64_t m, float *feat, float *targ)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_octnet_prepare: NULL handle");
    if (!h->octnet || !onet_of(h)->ranges) return fail(h, SN_ESTATE, "sn_octnet_prepare: no input ranges yet");
    sn_status s = check_rows(h, feat, targ, m, "sn_octnet_prepare");
    if (s != SN_OK) return s;
    if (!in27) return fail(h, SN_EINVAL, "sn_octnet_prepare: NULL in27");
    const cudaStream_t st = h->stream;
    OctNet *n = onet_of(h);
    SN_CK(h, cudaMemsetAsync(n->flag, 0, sizeof(int), st));
    int64_t grid = (8 * m + 127) / 128;
    if (grid > (int64_t)num_sms() * 16) grid = (int64_t)num_sms() * 16;
    octnet_prepare_kernel<<<(unsigned)grid, 128, 0, st>>>(in27, m, n->shift, n->inv_r, feat, targ, n->flag);
    SN_CK(h, cudaGetLastError());
    int bad = 0;
    SN_CK(h, cudaMemcpyAsync(&bad, n->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    if (bad) return fail(h, SN_EINVAL, "sn_octnet_prepare: a row of block o is not in octant o");
    return SN_OK;
}

sn_status sn_octnet_grad(sn_handle h, const float *feat, const float *targ, int64_t m, float *grad, double *loss)
{
    sn_status s = need_octnet(h, "sn_octnet_grad");
    if (s == SN_OK) s = check_rows(h, feat, targ, m, "sn_octnet_grad");
    if (s != SN_OK) return s;
    const cudaStream_t st = h->stream;
    OctNet *n = onet_of(h);
    float *gdev = nullptr;
    SN_CK(h, cudaMalloc(&gdev, sizeof(float) * 8 * kOnParam));
    s = grad_step(h, feat, targ, m, 0.f, false, 0, gdev, st);
    std::vector<float> g(8 * kOnParam);
    std::vector<double> l(8);
    cudaError_t e = cudaSuccess;
    if (s == SN_OK) {
        e = cudaMemcpyAsync(g.data(), gdev, sizeof(float) * g.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(l.data(), n->loss, sizeof(double) * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFree(gdev);
    if (s != SN_OK) return s;
    SN_CK(h, e);
    if (grad) std::copy(g.begin(), g.end(), grad);
    if (loss) std::copy(l.begin(), l.end(), loss);
    return SN_OK;
}

sn_status sn_octnet_fit(sn_handle h, const float *feat, const float *targ, int64_t m, int32_t steps, float lr,
                        double *loss)
{
    sn_status s = need_octnet(h, "sn_octnet_fit");
    if (s == SN_OK) s = check_rows(h, feat, targ, m, "sn_octnet_fit");
    if (s != SN_OK) return s;
    if (steps < 0 || !(lr >= 0.f)) return fail(h, SN_EINVAL, "sn_octnet_fit: steps >= 0 and lr >= 0");
    const cudaStream_t st = h->stream;
    for (int k = 0; k < steps; ++k) {
        s = grad_step(h, feat, targ, m, lr, true, 0xff, nullptr, st);
        if (s != SN_OK) return s;
    }
    s = refold(h, st);
    if (s != SN_OK) return s;
    if (loss) SN_CK(h, cudaMemcpyAsync(loss, onet_of(h)->loss, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    return SN_OK;
}

sn_status sn_octnet_eval(sn_handle h, const float *feat, const float *targ, int64_t m, double *mae, double *mse)
{
    sn_status s = need_octnet(h, "sn_octnet_eval");
    if (s == SN_OK) s = check_rows(h, feat, targ, m, "sn_octnet_eval");
    if (s != SN_OK) return s;
    return errors(h, feat, targ, m, mae, mse, h->stream);
}

sn_status sn_octnet_prune(sn_handle h, const float *feat, const float *targ, int64_t m, int32_t retrain_steps,
                          float lr, double tol, int32_t max_drops, int32_t *dropped)
{
    sn_status s = need_octnet(h, "sn_octnet_prune");
    if (s == SN_OK) s = check_rows(h, feat, targ, m, "sn_octnet_prune");
    if (s != SN_OK) return s;
    if (retrain_steps < 0 || !(lr >= 0.f) || !(tol >= 0.0) || max_drops < 0)
        return fail(h, SN_EINVAL, "sn_octnet_prune: retrain_steps, lr, tol, max_drops >= 0");
    const cudaStream_t st = h->stream;
    double mse0[8], mse[8];
    s = errors(h, feat, targ, m, nullptr, mse0, st);
    if (s != SN_OK) return s;
    int active = 0xff, count[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (max_drops == 0) active = 0;
    std::vector<float> p, k, p_prev, k_prev;
    while (active) {
        s = download(h, p, k, st);
        if (s != SN_OK) return s;
        p_prev = p;
        k_prev = k;
        for (int o = 0; o < 8; ++o) {
            if (!((active >> o) & 1)) continue;
            // the remaining connection (W1 or W2 entry) of smallest magnitude, lowest index on ties
            int best = -1;
            float bv = 0.f;
            for (int e = 0; e < kOnParam; ++e) {
                const bool conn = e < kOnB1 || (e >= kOnW2 && e < kOnB2);
                const int q = kOnParam * o + e;
                if (!conn || k[q] == 0.f) continue;
                if (best < 0 || std::fabs(p[q]) < bv) { best = q; bv = std::fabs(p[q]); }
            }
            if (best < 0) { active &= ~(1 << o); continue; }
            p[best] = 0.f;
            k[best] = 0.f;
        }
        if (!active) break;
        s = upload(h, p, k, st);
        if (s == SN_OK) s = reset_adam(h, st);
        for (int it = 0; s == SN_OK && it < retrain_steps; ++it) s = grad_step(h, feat, targ, m, lr, true, active, nullptr, st);
        if (s == SN_OK) s = errors(h, feat, targ, m, nullptr, mse, st);
        if (s != SN_OK) return s;
        s = download(h, p, k, st);
        if (s != SN_OK) return s;
        bool undo = false;
        for (int o = 0; o < 8; ++o) {
            if (!((active >> o) & 1)) continue;
            if (mse[o] > (1.0 + tol) * mse0[o]) {
                std::copy(p_prev.begin() + kOnParam * o, p_prev.begin() + kOnParam * (o + 1), p.begin() + kOnParam * o);
                std::copy(k_prev.begin() + kOnParam * o, k_prev.begin() + kOnParam * (o + 1), k.begin() + kOnParam * o);
                active &= ~(1 << o);
                undo = true;
            } else if (++count[o] >= max_drops) {
                active &= ~(1 << o);
            }
        }
        if (undo) {
            s = upload(h, p, k, st);
            if (s != SN_OK) return s;
        }
    }
    s = reset_adam(h, st);
    if (s == SN_OK) s = refold(h, st);
    if (s != SN_OK) return s;
    SN_CK(h, cudaStreamSynchronize(st));
    if (dropped)
        for (int o = 0; o < 8; ++o) dropped[o] = count[o];
    return SN_OK;
}

sn_status sn_octnet_apply(sn_handle h, const float *in27, float *psi, int64_t n)
{
    sn_status s = need_octnet(h, "sn_octnet_apply");
    if (s != SN_OK) return s;
    if (n < 0) return fail(h, SN_EINVAL, "sn_octnet_apply: n < 0");
    if (n > 0 && (!in27 || !psi)) return fail(h, SN_EINVAL, "sn_octnet_apply: NULL pointer");
    return launch_octnet_cells(h, in27, psi, n, h->stream);
}

}  // extern "C"

// sn_ann.cu -- the shallow-network surrogate of the per-cell solve (Sec. 3 of Tano &
// Ragusa): training on one-cell problems labelled by the library's own elimination
// (Sec. 4: loss of Eq. (19), Adam), and BF16 inference on the tcgen05 tensor cores
// with a residual gate that sends failing cells back to elimination.
//
// Network: Eq. (15) with 27 inputs, 64 ReLU hidden units and 8 linear outputs.
// Parameters (2312, FP32 masters): W1[64][27], b1[64], W2[8][64], b2[8].
//
// Inference: a CTA of 128 threads owns a 128-row tile.  Each thread builds its
// row's 27 inputs, rounds them to BF16 and writes one row of the A operand in shared
// memory (with two columns of ones that carry b1); one thread issues tcgen05.mma
// (M=128, N=64, K=16, twice) with the accumulator in tensor memory; the four warps
// read their 32 TMEM lanes back (tcgen05.ld), apply ReLU, round to BF16 and store the
// hidden tile back into tensor memory (tcgen05.st), where the second layer reads its
// A operand (N=16, only 8 columns used); b2 is added in FP32.
//
// Shared-memory operands use the no-swizzle K-major core-matrix layout: a core
// matrix is 8 rows x 16 bytes, stored row after row; core matrices follow each other
// along K every 128 bytes (leading byte offset) and along M/N every K/8 * 128 bytes
// (stride byte offset).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "cell_problem.cuh"
#include "sn_internal.cuh"
#include "sweep_common.cuh"
#include "wave.cuh"

#include <cuda_bf16.h>

namespace sn {

// --------------------------------------------------------------------------------
// tcgen05 / mbarrier helpers (inline PTX)
// --------------------------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// One test of an mbarrier phase; the thread may be suspended in hardware for up to
// hint_ns nanoseconds while the phase is incomplete (it resumes when the phase
// completes), so a waiting warp does not spend issue slots spinning.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: false once `limit` SM cycles (by default 2^31,
// about 1 s) have passed without completion.  Each test may suspend the thread for up
// to SN_MBAR_HINT_NS nanoseconds; 0, a plain test in a spinning loop, measured faster
// for the surrogate sweep (4.57 against 4.83 ms on blocked_64 with a 100 us hint).
#ifndef SN_MBAR_HINT_NS
#define SN_MBAR_HINT_NS 0u
#endif
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit = (1LL << 31))
{
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity, SN_MBAR_HINT_NS)) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulate, cta_group::1
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one per thread), waited.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: no swizzle, K-major, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, k) in a K-major no-swizzle operand with kdim columns.
__host__ __device__ constexpr uint32_t umma_off(int row, int k, int kdim)
{
    return (uint32_t)((row >> 3) * (kdim / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

constexpr int kTile = 128;
constexpr int kK1 = 32;                        // 27 inputs, 2 bias columns, 3 zero
constexpr int kN2 = 16;                        // 8 outputs padded
constexpr uint32_t kW1Bytes = kNhid * kK1 * 2; // 4096
constexpr uint32_t kW2Bytes = kN2 * kNhid * 2; // 2048
constexpr uint32_t kXBytes = kTile * kK1 * 2;  // 8192
constexpr uint32_t kTmemCols = 64;   // layer 1: 0..63; hidden BF16 pairs: 0..31; layer 2: 32..47

struct Net {
    float *p = nullptr;        // [kNparam] FP32 master weights
    float *m = nullptr, *v = nullptr;
    int64_t t = 0;             // Adam steps taken
    unsigned char *w1p = nullptr;  // BF16 W1 in the operand layout
    unsigned char *w2p = nullptr;  // BF16 W2 (rows 8..15 zero)
    float *b1 = nullptr, *b2 = nullptr;   // [64], [16]
    bool dirty = true;         // packed copies stale
    float tau = 1e-2f;         // gate threshold
    float *gpart = nullptr;    // per-CTA gradient partials
    double *lpart = nullptr;
    int64_t gpart_blocks = 0;
    unsigned long long *counter = nullptr;   // [0] fallbacks, [1] error flags
    double *dacc = nullptr;    // scratch accumulator
    uint32_t *fb_queue = nullptr;   // gated sweep: rows rejected on the current hyperplane
    uint32_t *fb_count = nullptr;   // [nplanes] queue lengths
    uint32_t *mask = nullptr;       // frozen gate: one bit a row ((o C + c) G + g) Do + d, 1 = network
    int64_t mask_words = 0;
    uint64_t frozen_gen = 0;        // net_gen of the handle when the mask was recorded (0: none)
};

static Net *net_of(sn_handle h) { return reinterpret_cast<Net *>(h->net); }

void free_net(sn_handle h)
{
    if (!h || !h->net) return;
    Net *n = net_of(h);
    void *bufs[] = {n->p, n->m, n->v, n->w1p, n->w2p, n->b1, n->b2, n->gpart, n->lpart, n->counter, n->dacc,
                    n->fb_queue, n->fb_count, n->mask};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete n;
    h->net = nullptr;
    h->has_net = false;
}

static sn_status ensure_net(sn_handle h)
{
    if (h->net) return SN_OK;
    Net *n = new Net();
    h->net = n;
    SN_CK(h, cudaMalloc(&n->p, sizeof(float) * kNparam));
    SN_CK(h, cudaMalloc(&n->m, sizeof(float) * kNparam));
    SN_CK(h, cudaMalloc(&n->v, sizeof(float) * kNparam));
    SN_CK(h, cudaMalloc(&n->w1p, kW1Bytes));
    SN_CK(h, cudaMalloc(&n->w2p, kW2Bytes));
    SN_CK(h, cudaMalloc(&n->b1, sizeof(float) * kNhid));
    SN_CK(h, cudaMalloc(&n->b2, sizeof(float) * kN2));
    SN_CK(h, cudaMalloc(&n->counter, sizeof(unsigned long long) * 2));
    SN_CK(h, cudaMalloc(&n->dacc, sizeof(double) * 4));
    SN_CK(h, cudaMemsetAsync(n->m, 0, sizeof(float) * kNparam, h->stream));
    SN_CK(h, cudaMemsetAsync(n->v, 0, sizeof(float) * kNparam, h->stream));
    SN_CK(h, cudaMemsetAsync(n->counter, 0, sizeof(unsigned long long) * 2, h->stream));
    // fallback queue of the gated sweep: every row of the largest hyperplane's tiles
    int64_t max_cells = 0;
    for (int p = 0; p < h->nplanes; ++p) max_cells = std::max(max_cells, h->plane_off[p + 1] - h->plane_off[p]);
    const int64_t kpt = kTile / h->Do;
    const int64_t max_tiles = (max_cells * h->G + kpt - 1) / kpt;
    SN_CK(h, cudaMalloc(&n->fb_queue, sizeof(uint32_t) * (size_t)(8 * max_tiles * kTile)));
    SN_CK(h, cudaMalloc(&n->fb_count, sizeof(uint32_t) * (size_t)h->nplanes));
    return SN_OK;
}

// --------------------------------------------------------------------------------
// Training data: canonical features and elimination labels psi_c / s.
// --------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) prepare_kernel(const float *__restrict__ in27, int64_t n,
                                                      float *__restrict__ feat, float *__restrict__ targ)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float *p = in27 + 27 * i;
        CanonCell<float> c;
        canonicalize(p, c);
        const float s = input_scale(c.S, c.ux, c.uy, c.uz);
        const float inv = s > kScaleFloor ? 1.f / s : 0.f;
        float x[kNin];
        ann_features(fabsf(p[0]), fabsf(p[1]), fabsf(p[2]), p[3], p[4], p[5], c.sig, c.S, c.ux, c.uy, c.uz, inv, x);
#pragma unroll
        for (int k = 0; k < kNin; ++k) feat[kNin * i + k] = x[k];
        float psi[8];
        cell_solve_canonical<float, true>(c.t3x, c.t3y, c.t3z, c.sig, c.S, c.ux, c.uy, c.uz, psi);
#pragma unroll
        for (int k = 0; k < 8; ++k) targ[8 * i + k] = psi[k] * inv;
    }
}

// --------------------------------------------------------------------------------
// Loss (19) and its back-propagated gradient over a batch, FP32, one CTA per 128
// samples; partial gradients per CTA are summed in a fixed order by adam_kernel.
// Batch row i is dataset row (row0 + i) mod nrows.
// --------------------------------------------------------------------------------
constexpr float kLambda = 0.2f, kGamma1 = 10.f, kGamma2 = 0.01f;
constexpr int kXs = 28, kHs = 65, kOs = 9;    // shared-memory row strides

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(128) grad_kernel(const float *__restrict__ P, const float *__restrict__ feat,
                                                   const float *__restrict__ targ, int64_t nrows, int64_t row0,
                                                   int batch, float inv_batch, float *__restrict__ gpart,
                                                   double *__restrict__ lpart)
{
    extern __shared__ __align__(16) float sm[];
    float *sP = sm;                          // kNparam
    float *sX = sP + kNparam;                // [128][28]
    float *sH = sX + 128 * kXs;              // [128][65]
    float *sGA = sH + 128 * kHs;             // [128][65]
    float *sGO = sGA + 128 * kHs;            // [128][9]
    __shared__ double sl[4];
    for (int e = threadIdx.x; e < kNparam; e += blockDim.x) sP[e] = P[e];
    __syncthreads();
    const float *W1 = sP, *b1 = sP + kNhid * kNin, *W2 = b1 + kNhid, *b2 = W2 + kNout * kNhid;
    const int t = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * 128 + t;
    double lsum = 0.0;
    float *xr = sX + t * kXs, *hr = sH + t * kHs, *gar = sGA + t * kHs, *gor = sGO + t * kOs;
    if (i < batch) {
        const int64_t r = (row0 + i) % nrows;
        float x[kNin], tt[8], h[kNhid];
#pragma unroll
        for (int k = 0; k < kNin; ++k) { x[k] = feat[kNin * r + k]; xr[k] = x[k]; }
#pragma unroll
        for (int k = 0; k < 8; ++k) tt[k] = targ[8 * r + k];
#pragma unroll 4
        for (int j = 0; j < kNhid; ++j) {
            float a = b1[j];
#pragma unroll
            for (int k = 0; k < kNin; ++k) a = fmaf(W1[j * kNin + k], x[k], a);
            h[j] = fmaxf(a, 0.f);
            hr[j] = h[j];
        }
        float d[8], sd = 0.f, st = 0.f, mae = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float a = b2[q];
#pragma unroll
            for (int j = 0; j < kNhid; ++j) a = fmaf(W2[q * kNhid + j], h[j], a);
            d[q] = tt[q] - a;
            sd += d[q];
            st += tt[q];
            mae += fabsf(d[q]);
        }
        const float den = kGamma1 * fabsf(st) + kGamma2;
        lsum = (double)((mae / 8.f + kLambda * fabsf(sd) / den) * inv_batch);
        float go[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            go[q] = -(sgnf(d[q]) / 8.f + kLambda * sgnf(sd) / den) * inv_batch;
            gor[q] = go[q];
        }
#pragma unroll 4
        for (int j = 0; j < kNhid; ++j) {
            float gh = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) gh = fmaf(go[q], W2[q * kNhid + j], gh);
            gar[j] = h[j] > 0.f ? gh : 0.f;
        }
    } else {
        for (int k = 0; k < kNin; ++k) xr[k] = 0.f;
        for (int j = 0; j < kNhid; ++j) { hr[j] = 0.f; gar[j] = 0.f; }
        for (int q = 0; q < 8; ++q) gor[q] = 0.f;
    }
    __syncthreads();
    float *gp = gpart + (int64_t)blockIdx.x * kNparam;
    for (int e = t; e < kNparam; e += 128) {
        float acc = 0.f;
        if (e < kNhid * kNin) {
            const int j = e / kNin, k = e % kNin;
            for (int s = 0; s < 128; ++s) acc = fmaf(sGA[s * kHs + j], sX[s * kXs + k], acc);
        } else if (e < kNhid * kNin + kNhid) {
            const int j = e - kNhid * kNin;
            for (int s = 0; s < 128; ++s) acc += sGA[s * kHs + j];
        } else if (e < kNhid * kNin + kNhid + kNout * kNhid) {
            const int q = (e - kNhid * kNin - kNhid) / kNhid, j = (e - kNhid * kNin - kNhid) % kNhid;
            for (int s = 0; s < 128; ++s) acc = fmaf(sGO[s * kOs + q], sH[s * kHs + j], acc);
        } else {
            const int q = e - (kNhid * kNin + kNhid + kNout * kNhid);
            for (int s = 0; s < 128; ++s) acc += sGO[s * kOs + q];
        }
        gp[e] = acc;
    }
    // batch loss partial
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
    if ((t & 31) == 0) sl[t >> 5] = lsum;
    __syncthreads();
    if (t == 0) lpart[blockIdx.x] = sl[0] + sl[1] + sl[2] + sl[3];
}

constexpr size_t kGradSmem = sizeof(float) * (kNparam + 128 * kXs + 2 * 128 * kHs + 128 * kOs);

// Sum the partials (fixed order); optionally write the gradient, then Adam.
__global__ void adam_kernel(float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                            const float *__restrict__ gpart, int nblk, float lr, float bc1, float bc2,
                            float *__restrict__ gout, int do_step)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNparam) return;
    double g = 0.0;
    for (int b = 0; b < nblk; ++b) g += (double)gpart[(int64_t)b * kNparam + e];
    const float gf = (float)g;
    if (gout) gout[e] = gf;
    if (!do_step) return;
    const float m = 0.9f * M[e] + 0.1f * gf;
    const float v = 0.999f * V[e] + 0.001f * gf * gf;
    M[e] = m;
    V[e] = v;
    P[e] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
}

__global__ void sum_kernel(const double *__restrict__ part, int n, double *__restrict__ out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s;
    }
}

// mean |t - o| over a set (FP32 forward), partial sums per CTA into acc (atomic)
__global__ void __launch_bounds__(128) mae_kernel(const float *__restrict__ P, const float *__restrict__ feat,
                                                  const float *__restrict__ targ, int64_t n, double *acc)
{
    __shared__ float sP[kNparam];
    __shared__ double sl[4];
    for (int e = threadIdx.x; e < kNparam; e += blockDim.x) sP[e] = P[e];
    __syncthreads();
    const float *W1 = sP, *b1 = sP + kNhid * kNin, *W2 = b1 + kNhid, *b2 = W2 + kNout * kNhid;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float x[kNin], h[kNhid];
#pragma unroll
        for (int k = 0; k < kNin; ++k) x[k] = feat[kNin * i + k];
#pragma unroll 4
        for (int j = 0; j < kNhid; ++j) {
            float a = b1[j];
#pragma unroll
            for (int k = 0; k < kNin; ++k) a = fmaf(W1[j * kNin + k], x[k], a);
            h[j] = fmaxf(a, 0.f);
        }
        float e = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float a = b2[q];
#pragma unroll
            for (int j = 0; j < kNhid; ++j) a = fmaf(W2[q * kNhid + j], h[j], a);
            e += fabsf(targ[8 * i + q] - a);
        }
        s += (double)e;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(acc, sl[0] + sl[1] + sl[2] + sl[3]);
}

// FP32 masters -> BF16 operands in the tcgen05 layout.  W1 carries b1 in two columns
// (bf16(b1) and bf16(b1 - bf16(b1))) that meet the two columns of ones in X; b2 stays
// FP32 (added to the layer-2 accumulator).
__global__ void pack_kernel(const float *__restrict__ P, unsigned char *__restrict__ w1p,
                            unsigned char *__restrict__ w2p, float *__restrict__ b1, float *__restrict__ b2)
{
    const float *W1 = P, *B1 = P + kNhid * kNin, *W2 = B1 + kNhid, *B2 = W2 + kNout * kNhid;
    for (int e = threadIdx.x; e < kNhid * kK1; e += blockDim.x) {
        const int n = e / kK1, k = e % kK1;
        const float hi = __bfloat162float(__float2bfloat16_rn(B1[n]));
        const float v = k < kNin ? W1[n * kNin + k] : (k == kNin ? hi : (k == kNin + 1 ? B1[n] - hi : 0.f));
        *reinterpret_cast<__nv_bfloat16 *>(w1p + umma_off(n, k, kK1)) = __float2bfloat16_rn(v);
    }
    for (int e = threadIdx.x; e < kN2 * kNhid; e += blockDim.x) {
        const int n = e / kNhid, k = e % kNhid;
        const float v = n < kNout ? W2[n * kNhid + k] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(w2p + umma_off(n, k, kNhid)) = __float2bfloat16_rn(v);
    }
    for (int e = threadIdx.x; e < kNhid; e += blockDim.x) b1[e] = B1[e];
    for (int e = threadIdx.x; e < kN2; e += blockDim.x) b2[e] = e < kNout ? B2[e] : 0.f;
}

// --------------------------------------------------------------------------------
// tcgen05 inference.
//
// Both inference kernels run a 128-row tile as follows.  Each thread writes its row
// of X (27 features, then two columns of ones that carry b1 = bf16(b1) +
// bf16(b1 - bf16(b1)) through the first product, then zeros) in BF16 to shared
// memory; one thread issues layer 1 (M=128, N=64, K=32) into TMEM columns 0..63;
// each warp reads its 32 lanes back, applies ReLU, rounds to BF16 and writes the
// hidden tile H back into TMEM columns 0..31 (two BF16 per column); one thread
// issues layer 2 with A = H read from TMEM (M=128, N=16, K=64) into columns 32..47;
// each thread reads its 8 outputs and adds b2.  Shared memory holds only W1, W2
// and X, and TMEM 64 columns, so eight CTAs fit on an SM.
// --------------------------------------------------------------------------------
struct AnnArgs {
    const unsigned char *w1p, *w2p;
    const float *b2;
    float tau;
    unsigned long long *counter;   // [0] fallbacks, [1] timeouts
};

// Two FP32 values rounded to BF16 and packed, the first in the low half (lower address).
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&t);
}

// max(a, 0), max(b, 0) rounded to BF16 and packed, a in the low half.
__device__ __forceinline__ uint32_t pack_relu_bf16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(__uint_as_float(b)), "f"(__uint_as_float(a)));
    return d;
}

// The X row of thread `row` (features, bias ones, zero padding) as BF16, 4 x 16 bytes.
// Rows of idle threads are left as they are: a row of the product depends only on
// the same row of X, and idle rows' outputs are never used.
__device__ __forceinline__ void write_x_row(unsigned char *sx, int row, const float (&x)[kNin])
{
    float v[kK1];
#pragma unroll
    for (int k = 0; k < kNin; ++k) v[k] = x[k];
    v[kNin] = v[kNin + 1] = 1.f;
#pragma unroll
    for (int k = kNin + 2; k < kK1; ++k) v[k] = 0.f;
#pragma unroll
    for (int kg = 0; kg < kK1 / 8; ++kg) {
        uint4 u;
        u.x = pack_bf16x2(v[kg * 8 + 0], v[kg * 8 + 1]);
        u.y = pack_bf16x2(v[kg * 8 + 2], v[kg * 8 + 3]);
        u.z = pack_bf16x2(v[kg * 8 + 4], v[kg * 8 + 5]);
        u.w = pack_bf16x2(v[kg * 8 + 6], v[kg * 8 + 7]);
        *reinterpret_cast<uint4 *>(sx + umma_off(row, kg * 8, kK1)) = u;
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D[tmem] (+)= A[tmem] * B[smem]^T, BF16 inputs, FP32 accumulate, cta_group::1
__device__ __forceinline__ void umma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

// Layer 1 of the tile in X (issued by thread 0; completion arrives on the barrier).
__device__ __forceinline__ void mma_layer1(uint32_t sbase, uint32_t offx, uint32_t offw1, uint32_t tbase, uint32_t bar)
{
    constexpr uint32_t id1 = idesc_bf16(128, kNhid);
#pragma unroll
    for (int kk = 0; kk < kK1 / 16; ++kk)
        umma_bf16(tbase, sdesc(sbase + offx + kk * 256, 128, (kK1 / 8) * 128),
                  sdesc(sbase + offw1 + kk * 256, 128, (kK1 / 8) * 128), id1, kk > 0);
    umma_commit(bar);
}

// Layer 2 with A = H in TMEM columns 0..31, D in columns 32..47 (thread 0).
__device__ __forceinline__ void mma_layer2(uint32_t sbase, uint32_t offw2, uint32_t tbase, uint32_t bar)
{
    constexpr uint32_t id2 = idesc_bf16(128, kN2);
#pragma unroll
    for (int kk = 0; kk < kNhid / 16; ++kk)
        umma_bf16_ta(tbase + 32, tbase + 8 * kk, sdesc(sbase + offw2 + kk * 256, 128, (kNhid / 8) * 128), id2,
                     kk > 0);
    umma_commit(bar);
}

// This warp's lanes of the layer-1 accumulator -> ReLU -> BF16 pairs in columns 0..31.
__device__ __forceinline__ void hidden_to_tmem(uint32_t twarp)
{
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        uint32_t v[32], h[16];
        tmem_ld32(twarp + 32 * half, v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) h[j] = pack_relu_bf16x2(v[2 * j], v[2 * j + 1]);
        tmem_st16(twarp + 16 * half, h);
    }
    tmem_wait_st();
}

// Weights to shared memory, nbar mbarriers (8 bytes apart from offbar), ncols TMEM
// columns; returns the TMEM base.
__device__ __forceinline__ uint32_t ann_setup(unsigned char *smem, const AnnArgs &a, uint32_t offw1, uint32_t offw2,
                                              uint32_t offbar, int *misc, uint32_t ncols = kTmemCols, int nbar = 1)
{
    const uint4 *g1 = reinterpret_cast<const uint4 *>(a.w1p), *g2 = reinterpret_cast<const uint4 *>(a.w2p);
    uint4 *s1 = reinterpret_cast<uint4 *>(smem + offw1), *s2 = reinterpret_cast<uint4 *>(smem + offw2);
    for (int e = threadIdx.x; e < (int)(kW1Bytes / 16); e += blockDim.x) s1[e] = g1[e];
    for (int e = threadIdx.x; e < (int)(kW2Bytes / 16); e += blockDim.x) s2[e] = g2[e];
    if (threadIdx.x == 0) {
        misc[1] = 0;   // queue count
        misc[2] = 0;   // abort flag
        for (int b = 0; b < nbar; ++b) mbar_init(smem_u32(smem + offbar + 8 * b), 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x < 32) {
        tmem_alloc(smem_u32(misc), ncols);
        tmem_relinquish();
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *reinterpret_cast<volatile uint32_t *>(misc);
}

__device__ __forceinline__ void ann_teardown(uint32_t tbase, const AnnArgs &a, const int *misc,
                                             uint32_t ncols = kTmemCols)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && reinterpret_cast<const volatile int *>(misc)[2]) atomicAdd(a.counter + 1, 1ull);
    __syncwarp();
    if (threadIdx.x < 32) tmem_dealloc(tbase, ncols);
}

// Self-test of the bounded tensor-core waits (not in the paper): the set-up of a
// surrogate kernel (mbarrier, TMEM columns), then thread 0 waits on phase 0 of the
// mbarrier, which expects one arrival that nothing makes, for at most `limit` SM
// cycles.  It gives up, raises the CTA's abort flag, and the teardown counts the
// timed-out CTA and frees the TMEM exactly as after a failed wait in a sweep.
__global__ void __launch_bounds__(128) wait_selftest_kernel(AnnArgs a, long long limit)
{
    __shared__ __align__(8) unsigned long long bar_word;
    __shared__ __align__(16) int misc[4];
    const uint32_t bar = smem_u32(&bar_word);
    if (threadIdx.x == 0) {
        misc[2] = 0;
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x < 32) {
        tmem_alloc(smem_u32(misc), kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t *>(misc);
    const bool late = threadIdx.x == 0 && !mbar_wait_bounded(bar, 0u, limit);
    if (__syncthreads_or(late) && threadIdx.x == 0) misc[2] = 1;
    ann_teardown(tbase, a, misc);
}

// Independent one-cell problems (sn_surrogate_apply).  Rows the gate rejects are
// queued in shared memory and re-solved by elimination by the whole CTA.
constexpr uint32_t kCellOffW1 = 0, kCellOffW2 = kCellOffW1 + kW1Bytes, kCellOffX = kCellOffW2 + kW2Bytes;
constexpr uint32_t kCellOffStage = kCellOffX + kXBytes;                 // [128][27] floats
constexpr uint32_t kCellOffQueue = kCellOffStage + 4 * kTile * 27;      // [128] ints
constexpr uint32_t kCellOffBar = kCellOffQueue + 4 * kTile;
constexpr uint32_t kCellOffMisc = kCellOffBar + 8;                      // tmem slot, queue count, abort
constexpr uint32_t kCellSmem = kCellOffMisc + 16;

template <bool GATED>
__global__ void __launch_bounds__(128, 4) ann_cells_kernel(const float *__restrict__ in27, float *__restrict__ out,
                                                           int64_t n, AnnArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    int *misc = reinterpret_cast<int *>(smem + kCellOffMisc);
    const uint32_t tbase = ann_setup(smem, a, kCellOffW1, kCellOffW2, kCellOffBar, misc);
    const uint32_t sbase = smem_u32(smem), bar = sbase + kCellOffBar;
    const uint32_t twarp = tbase + ((uint32_t)(threadIdx.x & ~31) << 16);
    float *stage = reinterpret_cast<float *>(smem + kCellOffStage);
    int *queue = reinterpret_cast<int *>(smem + kCellOffQueue);
    float b2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) b2[q] = a.b2[q];
    uint32_t phase = 0;
    unsigned long long nfb = 0;
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
        const int cnt = (int)(n - base < kTile ? n - base : kTile);
        for (int e = threadIdx.x; e < cnt * 27; e += blockDim.x) stage[e] = in27[base * 27 + e];
        __syncthreads();
        const int t = threadIdx.x;
        CanonCell<float> c;
        float s = 0.f, x[kNin];
        if (t < cnt) {
            const float *p = stage + 27 * t;
            canonicalize(p, c);
            s = input_scale(c.S, c.ux, c.uy, c.uz);
            ann_features(fabsf(p[0]), fabsf(p[1]), fabsf(p[2]), p[3], p[4], p[5], c.sig, c.S, c.ux, c.uy, c.uz,
                         s > kScaleFloor ? 1.f / s : 0.f, x);
        }
        if (t < cnt) write_x_row(smem + kCellOffX, t, x);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) mma_layer1(sbase, kCellOffX, kCellOffW1, tbase, bar);
        // the issuing thread waits for the tensor cores; the others wait at the barrier
        bool late = t == 0 && !mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(late)) { if (t == 0) misc[2] = 1; break; }
        tc_fence_after();
        hidden_to_tmem(twarp);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) mma_layer2(sbase, kCellOffW2, tbase, bar);
        late = t == 0 && !mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(late)) { if (t == 0) misc[2] = 1; break; }
        tc_fence_after();
        uint32_t r[8];
        tmem_ld8(twarp + 32, r);
        tmem_wait_ld();
        float psi[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) psi[q] = s * (__uint_as_float(r[q]) + b2[q]);
        bool pass = true;
        if (GATED && t < cnt && s > 0.f) pass = gate_pass(c, psi, a.tau);
        if (t < cnt && pass) {
            mirror8(psi, c.mask);
            float *dst = out + (base + t) * 8;
#pragma unroll
            for (int q = 0; q < 8; ++q) dst[q] = psi[q];
        }
        if (GATED) {
            if (t < cnt && !pass) queue[atomicAdd(&misc[1], 1)] = t;
            __syncthreads();
            const int nq = misc[1];
            for (int q = t; q < nq; q += blockDim.x) {
                const int row = queue[q];
                float ge[8];
                solve_in27<float, true>(stage + 27 * row, ge);
                float *dst = out + (base + row) * 8;
#pragma unroll
                for (int k = 0; k < 8; ++k) dst[k] = ge[k];
            }
            if (t == 0) nfb += (unsigned long long)nq;
            __syncthreads();
            if (t == 0) misc[1] = 0;
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (GATED && threadIdx.x == 0 && nfb) atomicAdd(a.counter, nfb);
    ann_teardown(tbase, a, misc);
}

// --------------------------------------------------------------------------------
// Surrogate sweep: one hyperplane of every octant, the per-cell elimination of the
// wavefront replaced by the network (Sec. 4: "construction of the input vector and a
// feed-forward evaluation").  Same keys, face planes and flux reduction as
// sweep_plane_ge; a tile is 128 rows = keys_per_tile keys x Do directions (rows past
// that are idle MMA rows).  The CTA loops over tiles; the inputs of the next tile
// (inflow faces, source, sigma_t) are copied to shared memory with cp.async while
// the current tile runs through the tensor cores.  With the residual gate, rejected
// rows write nothing: they are appended to a per-hyperplane queue that
// ann_fallback_kernel re-solves by elimination before the next hyperplane starts.
// --------------------------------------------------------------------------------
struct AnnSweepArgs {
    int nx, ny, nz, G, Do, ncells_plane, keys_per_tile, ntiles;   // tiles per octant
    int C;
    FastDiv divG;
    const uint32_t *cells;
    const float *sigt, *S, *psi_inc;
    const DirData<float> *dir;
    const float4 *dir_abs;
    Vec4<float> *fx, *fy, *fz;
    float *phi_oct;
    double *leak;
    float vol12, hx, hy, hz;
    uint32_t *fb_queue;      // rejected rows: (tile << 10) | (octant << 7) | row
    uint32_t *fb_count;      // this hyperplane's queue length
    AnnArgs ann;
};

// Where one row of a tile sits: key (cell of the hyperplane, group) and direction d.
struct SweepRow {
    int g, cell, ip, jp, kp;
    int64_t ix, iy, iz;
};

__device__ __forceinline__ SweepRow sweep_row(const AnnSweepArgs &a, int o, uint32_t key, uint32_t pk, int d)
{
    SweepRow r;
    const uint32_t cidx = a.divG.div(key);
    r.g = (int)(key - cidx * (uint32_t)a.G);
    r.ip = pk & 1023; r.jp = (pk >> 10) & 1023; r.kp = pk >> 20;
    const int i = (o & 1) ? a.nx - 1 - r.ip : r.ip;
    const int j = (o & 2) ? a.ny - 1 - r.jp : r.jp;
    const int k = (o & 4) ? a.nz - 1 - r.kp : r.kp;
    r.cell = i + a.nx * (j + a.ny * k);
    const int GD = a.G * a.Do, gd = r.g * a.Do + d;
    r.ix = (int64_t)(o * a.ny * a.nz + r.jp + a.ny * r.kp) * GD + gd;
    r.iy = (int64_t)(o * a.nx * a.nz + r.ip + a.nx * r.kp) * GD + gd;
    r.iz = (int64_t)(o * a.nx * a.ny + r.ip + a.nx * r.jp) * GD + gd;
    return r;
}

// One row of the canonical problem read with plain loads (fallback kernel).
__device__ __forceinline__ void load_canon(const AnnSweepArgs &a, int o, const SweepRow &r, const DirData<float> &dd,
                                           CanonCell<float> &c)
{
    const int g = r.g;
    if (r.ip == 0) { const float v = a.psi_inc[6 * g + (o & 1)]; c.ux[0] = c.ux[1] = c.ux[2] = c.ux[3] = v; }
    else load4(c.ux, a.fx + r.ix);
    if (r.jp == 0) { const float v = a.psi_inc[6 * g + 2 + ((o >> 1) & 1)]; c.uy[0] = c.uy[1] = c.uy[2] = c.uy[3] = v; }
    else load4(c.uy, a.fy + r.iy);
    if (r.kp == 0) { const float v = a.psi_inc[6 * g + 4 + ((o >> 2) & 1)]; c.uz[0] = c.uz[1] = c.uz[2] = c.uz[3] = v; }
    else load4(c.uz, a.fz + r.iz);
    const int gc = g * a.C + r.cell;
    c.sig = a.sigt[gc];
    const Vec4<float> *Sp = reinterpret_cast<const Vec4<float> *>(a.S + (int64_t)gc * 8);
    float s0[4], s1[4];
    load4(s0, Sp);
    load4(s1, Sp + 1);
#pragma unroll
    for (int n = 0; n < 4; ++n) { c.S[n] = s0[n]; c.S[4 + n] = s1[n]; }
    mirror8(c.S, o);
    c.t3x = dd.t3x; c.t3y = dd.t3y; c.t3z = dd.t3z;
    c.mask = o;
}

// Outflow faces (or leakage) of a solved row.
__device__ __forceinline__ void store_outflow(const AnnSweepArgs &a, const SweepRow &r, const DirData<float> &dd,
                                              const float (&psi)[8], float &leak)
{
    if (r.ip < a.nx - 1) store4(a.fx + r.ix, psi[1], psi[3], psi[5], psi[7]);
    else leak += dd.w * a.vol12 * dd.t3x * (psi[1] + psi[3] + psi[5] + psi[7]);
    if (r.jp < a.ny - 1) store4(a.fy + r.iy, psi[2], psi[3], psi[6], psi[7]);
    else leak += dd.w * a.vol12 * dd.t3y * (psi[2] + psi[3] + psi[6] + psi[7]);
    if (r.kp < a.nz - 1) store4(a.fz + r.iz, psi[4], psi[5], psi[6], psi[7]);
    else leak += dd.w * a.vol12 * dd.t3z * (psi[4] + psi[5] + psi[6] + psi[7]);
}

// Shared-memory layout of the sweep kernel for kpt keys per tile.
struct SweepSmem {
    uint32_t w1, w2, x, face, ks, sig, rec, red, bar, misc, total;
};
__host__ __device__ inline SweepSmem sweep_smem(int kpt)
{
    SweepSmem m;
    m.w1 = 0;
    m.w2 = m.w1 + kW1Bytes;
    m.x = m.w2 + kW2Bytes;                  // X tile
    m.face = m.x + kXBytes;                 // [128 rows][12] inflow face values
    m.ks = m.face + kTile * 48;             // [kpt][8] source
    m.sig = m.ks + 32 * kpt;                // [kpt] sigma_t
    m.rec = (m.sig + 4 * kpt + 15) & ~15u;  // two sets of [kpt] key records
    m.red = m.rec + 2 * 32 * kpt;           // [128][9] w_d psi of the previous tile
    m.bar = m.red + kTile * 9 * 4;
    m.misc = m.bar + 8;                     // tmem slot, (unused), abort
    m.total = m.misc + 16;
    return m;
}

__device__ __forceinline__ float lg2_approx(float v)
{
    float r;
    asm("lg2.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float rcp_approx(float v)
{
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Tile loop of the surrogate sweep.  Per tile: (1) wait for the staged inputs and
// reduce the previous tile's w_d psi to its octant flux partial; (2) every row builds
// its features from the stage and the key records into X; (3) one thread issues
// layer 1, the key threads build the next tile's key records and start copying its
// sources and opacities; (4) each warp waits for layer 1 on its own, moves its lanes'
// hidden layer through TMEM; after one barrier all rows start copying the next
// tile's inflow faces and one thread issues layer 2; (5) each warp waits for layer 2
// and writes its outputs (gate, outflow faces, w_d psi).  Three CTA barriers a tile.
// DO > 0 fixes the directions per octant at compile time (DO = 0: the handle's value).
template <bool GATED, int DO>
__global__ void __launch_bounds__(128, GATED ? 6 : 8) sweep_plane_ann(AnnSweepArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    griddep_launch();
    const int Do = DO ? DO : a.Do;
    const int kpt = a.keys_per_tile;
    const SweepSmem L = sweep_smem(kpt);
    int *misc = reinterpret_cast<int *>(smem + L.misc);
    const uint32_t tbase = ann_setup(smem, a.ann, L.w1, L.w2, L.bar, misc);
    const uint32_t sbase = smem_u32(smem), bar = sbase + L.bar;
    const int t = threadIdx.x;
    const uint32_t twarp = tbase + ((uint32_t)(t & ~31) << 16);
    float *red = reinterpret_cast<float *>(smem + L.red);
    const int o = blockIdx.y;
    const int lk = t / Do, d = t - lk * Do;
    const bool lane_row = lk < kpt;
    const uint32_t nkeys = (uint32_t)a.ncells_plane * (uint32_t)a.G;
    DirData<float> dd = {0.f, 0.f, 0.f, 0.f};
    float xo0 = 0.f, xo1 = 0.f, xo2 = 0.f;
    if (lane_row) {
        dd = a.dir[d];
        const float4 ab = a.dir_abs[d];
        xo0 = 2.f * ab.x - 1.f; xo1 = 2.f * ab.y - 1.f; xo2 = 2.f * ab.z - 1.f;
    }
    float b2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) b2[q] = a.ann.b2[q];
    const float lhx = (logf(a.hx) + kLogHShift) / kLogHScale;
    const float lhy = (logf(a.hy) + kLogHShift) / kLogHScale;
    const float lhz = (logf(a.hz) + kLogHShift) / kLogHScale;
    const float lsig = 0.69314718f / kLogSigScale;      // ln 2 / 4.5: log2 -> feature
    const uint32_t sface = sbase + L.face + 48 * t;
    const float4 *fface = reinterpret_cast<const float4 *>(smem + L.face) + 3 * t;
    const float *fks = reinterpret_cast<const float *>(smem + L.ks) + 8 * lk;
    const float *fsig = reinterpret_cast<const float *>(smem + L.sig) + lk;
    const int psi_o[3] = {o & 1, 2 + ((o >> 1) & 1), 4 + ((o >> 2) & 1)};

    // key records of a tile (key threads only) and the copies of their sources
    auto key_record = [&](int tl, uint32_t pk, int parity) -> KeyRec {
        const uint32_t key = (uint32_t)tl * (uint32_t)kpt + (uint32_t)t;
        KeyRec r;
        if (tl < a.ntiles && key < nkeys) {
            make_key<DO>(a, o, key, pk, r);
        } else {
            r.bx = r.by = r.bz = 0; r.flags = 0; r.cell = r.g = 0; r.pad0 = r.pad1 = 0;
        }
        put_key(smem + L.rec + parity * 32 * kpt + 32 * t, r);
        return r;
    };
    auto key_copy = [&](const KeyRec &r) {
        if (!(r.flags & 0x80u)) return;
        const int64_t gc = (int64_t)r.g * a.C + r.cell;
        cp_async16(sbase + L.ks + 32 * t, a.S + gc * 8);
        cp_async16(sbase + L.ks + 32 * t + 16, a.S + gc * 8 + 4);
        cp_async4(sbase + L.sig + 4 * t, a.sigt + gc);
    };
    auto key_stage = [&](int tl, uint32_t pk, int parity) { key_copy(key_record(tl, pk, parity)); };
    // a row's inflow faces of the tile whose key records are in `parity`
    auto face_stage = [&](int parity) {
        if (!lane_row) return;
        const KeyRec r = get_key(smem + L.rec + parity * 32 * kpt + 32 * lk);
        if (!(r.flags & 0x80u)) return;
        if (!(r.flags & 1u)) cp_async16(sface, a.fx + r.bx + d);
        if (!(r.flags & 2u)) cp_async16(sface + 16, a.fy + r.by + d);
        if (!(r.flags & 4u)) cp_async16(sface + 32, a.fz + r.bz + d);
    };

    // set-up above and the first tile's key records read only what no hyperplane
    // writes; the copies of its inputs need the previous hyperplane (or fallback pass)
    // complete
    int tile = blockIdx.x;
    int par = 0;
    KeyRec r0 = {0, 0, 0, 0u, 0, 0, 0, 0};
    if (t < kpt) {
        const uint32_t key = (uint32_t)tile * (uint32_t)kpt + (uint32_t)t;
        const uint32_t pk = key < nkeys ? a.cells[a.divG.div(key)] : 0u;
        r0 = key_record(tile, pk, 0);
    }
    griddep_wait();
    if (t < kpt) key_copy(r0);
    __syncthreads();
    face_stage(0);
    cp_async_commit();
    uint32_t phase = 0;
    float leak = 0.f;
    unsigned long long nq_total = 0;
    // flux partial of the tile whose records are in `parity`: thread (key, node) sums
    // the key's directions
    auto reduce_tile = [&](int parity) {
        for (int e = t; e < 8 * kpt; e += kTile) {
            const int kk = e >> 3, n = e & 7;
            const KeyRec r = get_key(smem + L.rec + parity * 32 * kpt + 32 * kk);
            if (r.flags & 0x80u) {
                const float *base = red + (kk * Do) * 9 + n;
                float sum = 0.f;
                if (DO) {
#pragma unroll
                    for (int q = 0; q < DO; ++q) sum += base[q * 9];
                } else {
                    for (int q = 0; q < Do; ++q) sum += base[q * 9];
                }
                a.phi_oct[(((int64_t)o * a.C + r.cell) * a.G + r.g) * 8 + n] = sum;
            }
        }
    };
    bool late = false, done = true;
    int ntile_done = 0;
    for (; tile < a.ntiles; tile += gridDim.x, par ^= 1) {
        const int tn = tile + gridDim.x;
        uint32_t pk_n = 0;
        if (t < kpt) {
            const uint32_t key_n = (uint32_t)tn * (uint32_t)kpt + (uint32_t)t;
            if (tn < a.ntiles && key_n < nkeys) pk_n = a.cells[a.divG.div(key_n)];
        }
        cp_async_wait_all();
        if (__syncthreads_or(late)) { if (t == 0) misc[2] = 1; done = false; break; }
        if (ntile_done > 0) reduce_tile(par ^ 1);
        // (2) features
        const KeyRec kr = get_key(smem + L.rec + par * 32 * kpt + 32 * (lane_row ? lk : 0));
        const bool act = lane_row && (kr.flags & 0x80u);
        CanonCell<float> c;
        float s = 0.f;
        {
            float x[kNin];
            if (act) {
                const float4 fx4 = fface[0], fy4 = fface[1], fz4 = fface[2];
                const float *pi = a.psi_inc + 6 * kr.g;
                if (kr.flags & 1u) { c.ux[0] = c.ux[1] = c.ux[2] = c.ux[3] = pi[psi_o[0]]; }
                else { c.ux[0] = fx4.x; c.ux[1] = fx4.y; c.ux[2] = fx4.z; c.ux[3] = fx4.w; }
                if (kr.flags & 2u) { c.uy[0] = c.uy[1] = c.uy[2] = c.uy[3] = pi[psi_o[1]]; }
                else { c.uy[0] = fy4.x; c.uy[1] = fy4.y; c.uy[2] = fy4.z; c.uy[3] = fy4.w; }
                if (kr.flags & 4u) { c.uz[0] = c.uz[1] = c.uz[2] = c.uz[3] = pi[psi_o[2]]; }
                else { c.uz[0] = fz4.x; c.uz[1] = fz4.y; c.uz[2] = fz4.z; c.uz[3] = fz4.w; }
#pragma unroll
                for (int q = 0; q < 8; ++q) c.S[q] = fks[q ^ o];
                c.sig = *fsig;
                c.t3x = dd.t3x; c.t3y = dd.t3y; c.t3z = dd.t3z;
                c.mask = o;
                s = input_scale(c.S, c.ux, c.uy, c.uz);
                const float inv = s > kScaleFloor ? rcp_approx(s) : 0.f;
                x[0] = xo0; x[1] = xo1; x[2] = xo2;
                x[3] = lhx; x[4] = lhy; x[5] = lhz;
                x[6] = lg2_approx(fmaxf(c.sig, kSigFloor)) * lsig;
#pragma unroll
                for (int k = 0; k < 8; ++k) x[7 + k] = c.S[k] * inv;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    x[15 + q] = c.ux[q] * inv;
                    x[19 + q] = c.uy[q] * inv;
                    x[23 + q] = c.uz[q] * inv;
                }
            }
            if (act) write_x_row(smem + L.x, t, x);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // (3) layer 1; the next tile's key records and source copies
        if (t == 0) mma_layer1(sbase, L.x, L.w1, tbase, bar);
        if (t < kpt) key_stage(tn, pk_n, par ^ 1);
        // (4) each warp waits for layer 1 itself, hidden layer through TMEM
        if ((t & 31) == 0) late = !mbar_wait_bounded(bar, phase);
        __syncwarp();
        phase ^= 1u;
        tc_fence_after();
        hidden_to_tmem(twarp);
        tc_fence_before();
        if (__syncthreads_or(late)) { if (t == 0) misc[2] = 1; done = false; break; }
        tc_fence_after();
        if (t == 0) mma_layer2(sbase, L.w2, tbase, bar);
        face_stage(par ^ 1);
        cp_async_commit();
        // (5) each warp waits for layer 2 itself, outputs
        if ((t & 31) == 0) late = !mbar_wait_bounded(bar, phase);
        __syncwarp();
        phase ^= 1u;
        tc_fence_after();
        uint32_t r8[8];
        tmem_ld8(twarp + 32, r8);
        tmem_wait_ld();
        float psi[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) psi[q] = s * (__uint_as_float(r8[q]) + b2[q]);
        bool keep = act;
        if (GATED) {
            const bool reject = act && s != 0.f && !gate_pass(c, psi, a.ann.tau);
            keep = act && !reject;
            const unsigned m = __ballot_sync(0xffffffffu, reject);
            if (m) {
                const int lane = t & 31, leader = __ffs(m) - 1;
                uint32_t base = 0;
                if (lane == leader) base = atomicAdd(a.fb_count, (uint32_t)__popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (reject)
                    a.fb_queue[base + __popc(m & ((1u << lane) - 1u))] =
                        ((uint32_t)tile << 10) | ((uint32_t)o << 7) | (uint32_t)t;
                if (lane == 0) nq_total += (unsigned long long)__popc(m);
            }
        }
        float *rr = red + t * 9;
        if (keep) {
            if (!(kr.flags & 8u)) store4(a.fx + kr.bx + d, psi[1], psi[3], psi[5], psi[7]);
            else leak += dd.w * a.vol12 * dd.t3x * (psi[1] + psi[3] + psi[5] + psi[7]);
            if (!(kr.flags & 16u)) store4(a.fy + kr.by + d, psi[2], psi[3], psi[6], psi[7]);
            else leak += dd.w * a.vol12 * dd.t3y * (psi[2] + psi[3] + psi[6] + psi[7]);
            if (!(kr.flags & 32u)) store4(a.fz + kr.bz + d, psi[4], psi[5], psi[6], psi[7]);
            else leak += dd.w * a.vol12 * dd.t3z * (psi[4] + psi[5] + psi[6] + psi[7]);
#pragma unroll
            for (int n = 0; n < 8; ++n) rr[n ^ o] = dd.w * psi[n];
        } else {
#pragma unroll
            for (int n = 0; n < 8; ++n) rr[n] = 0.f;
        }
        ++ntile_done;
    }
    if (done) {
        cp_async_wait_all();
        if (__syncthreads_or(late)) {
            if (t == 0) misc[2] = 1;
        } else if (ntile_done > 0) {
            reduce_tile(par ^ 1);
        }
    }
    cp_async_wait_all();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) leak += __shfl_down_sync(0xffffffffu, leak, off);
    if ((t & 31) == 0 && leak != 0.f) atomicAdd(a.leak, (double)leak);
    if (GATED && (t & 31) == 0 && nq_total) atomicAdd(a.ann.counter, nq_total);
    ann_teardown(tbase, a.ann, misc);
}

// Elimination of the rows the gate rejected on this hyperplane: outflow faces,
// leakage, and w_d psi added to the tile's flux partial (atomics).
__global__ void __launch_bounds__(128, 4) ann_fallback_kernel(AnnSweepArgs a)
{
    griddep_launch();
    griddep_wait();
    const uint32_t n = *reinterpret_cast<volatile const uint32_t *>(a.fb_count);
    float leak = 0.f;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t qv = a.fb_queue[e];
        const int tile = (int)(qv >> 10), o = (int)((qv >> 7) & 7u), t = (int)(qv & 127u);
        const int lk = t / a.Do, d = t - lk * a.Do;
        const uint32_t key = (uint32_t)tile * (uint32_t)a.keys_per_tile + (uint32_t)lk;
        const uint32_t pk = a.cells[a.divG.div(key)];
        const SweepRow r = sweep_row(a, o, key, pk, d);
        const DirData<float> dd = a.dir[d];
        CanonCell<float> c;
        load_canon(a, o, r, dd, c);
        float psi[8];
        cell_solve_canonical<float, true>(c.t3x, c.t3y, c.t3z, c.sig, c.S, c.ux, c.uy, c.uz, psi);
        store_outflow(a, r, dd, psi, leak);
        float *dst = a.phi_oct + (((int64_t)o * a.C + r.cell) * a.G + r.g) * 8;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) atomicAdd(dst + (n2 ^ o), dd.w * psi[n2]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) leak += __shfl_down_sync(0xffffffffu, leak, off);
    if ((threadIdx.x & 31) == 0 && leak != 0.f) atomicAdd(a.leak, (double)leak);
}

static sn_status pack_if_dirty(sn_handle h, cudaStream_t st)
{
    Net *n = net_of(h);
    if (!n->dirty) return SN_OK;
    pack_kernel<<<1, 256, 0, st>>>(n->p, n->w1p, n->w2p, n->b1, n->b2);
    SN_CK(h, cudaGetLastError());
    n->dirty = false;
    return SN_OK;
}

static AnnArgs ann_args(sn_handle h)
{
    Net *n = net_of(h);
    AnnArgs a;
    a.w1p = n->w1p; a.w2p = n->w2p; a.b2 = n->b2; a.tau = n->tau; a.counter = n->counter;
    return a;
}

// After a synchronised surrogate sweep: SN_ETIMEOUT if any CTA gave up a wait.
sn_status check_ann_timeouts(sn_handle h)
{
    if (!h->net) return SN_OK;
    unsigned long long c[2] = {0, 0};
    SN_CK(h, cudaMemcpyAsync(c, net_of(h)->counter, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    SN_CK(h, cudaStreamSynchronize(h->stream));
    if (c[1]) return fail(h, SN_ETIMEOUT, "surrogate sweep: a tensor-core completion wait timed out");
    return SN_OK;
}

sn_status reset_ann_counters(sn_handle h, cudaStream_t st)
{
    if (!h->net) return SN_OK;
    SN_CK(h, cudaMemsetAsync(net_of(h)->counter, 0, sizeof(unsigned long long) * 2, st));
    return SN_OK;
}


// --------------------------------------------------------------------------------
// Surrogate key sweep: the schedule of the elimination key sweep (sn_sweep_keys.cu:
// one thread per key (octant, cell of the hyperplane, group) and chunk of directions,
// wavefront units, face planes [o][column][d][g], inflow vectors on the boundary)
// with the per-cell solve of (14) replaced by the network (Sec. 4: build the input
// vector, one feed-forward evaluation).  For each direction step the CTA's 128 rows
// (one a thread, TMEM lane = thread) go through the two tcgen05 layers together.
//   ANN_UNGATED  every row takes the network's output;
//   ANN_GATED    a row keeps it when ||b - A psi|| <= tau ||b|| for its system (14),
//                and with `record` the decision goes to the gate mask;
//   ANN_FROZEN   the gate mask decides (the decisions of a recorded gated sweep).
// The rows a step rejects are compacted, in thread order, to the first threads of
// the CTA and solved there by elimination (GE32R, the key sweep's solve), so only
// ceil(rejected / 32) warps run it; their outflow faces are stored by the solving
// thread and w_d psi_d handed back to the key's thread, which adds the network's and
// the elimination's rows to its flux partial in direction order: the flux is
// bit-reproducible for a given set of decisions.
// --------------------------------------------------------------------------------
enum { ANN_UNGATED = 0, ANN_GATED = 1, ANN_FROZEN = 2 };

struct AnnKeyArgs {
    int nx, ny, nz, G, Do, C;
    FastDiv divG;
    const float *sigt, *S;
    const float4 *dir;        // [Do] (3|Omega_x|/dx, 3|Omega_y|/dy, 3|Omega_z|/dz, w)
    const float4 *dir_abs;    // [Do] |Omega|
    float4 *face;             // x-planes | y-planes | z-planes | inflow vectors [G][6]
    uint32_t off_y, off_z, off_in;
    float *phi_oct;           // [8][C][G][8]
    float lhx, lhy, lhz;      // the cell-size inputs of the network
    AnnArgs ann;
    uint32_t *mask;           // gate decisions (ANN_GATED with record, ANN_FROZEN)
    int record;
    WaveCtl w;
};

// shared memory (bytes)
constexpr uint32_t kAkW1 = 0, kAkW2 = kAkW1 + kW1Bytes, kAkX = kAkW2 + kW2Bytes;   // two X tiles
constexpr uint32_t kAkStage = kAkX + 2 * kXBytes;       // [2][3][128] float4 inflow stages
constexpr uint32_t kAkSrc = kAkStage + 2 * 3 * kTile * 16;   // [128][8] canonical source of each key
constexpr uint32_t kAkKey = kAkSrc + kTile * 32;        // [128] sigma_t of each key
constexpr uint32_t kAkOff = kAkKey + kTile * 4;         // [128] uint4 (slots of d0, d0)
constexpr uint32_t kAkDir = kAkOff + kTile * 16;        // [64] float4 directions
constexpr uint32_t kAkDab = kAkDir + 64 * 16;           // [64] float4 |Omega|
constexpr uint32_t kAkQ = kAkDab + 64 * 16;             // [128] rejected rows: 12 faces, owner, d
constexpr int kAkQf = 14;                               // floats a rejected row
// [128][8] w_d psi of a step's rejected rows, by owner; at the end of a unit the same
// space holds the chunk partials of the flux (never both at once)
constexpr uint32_t kAkRes = kAkQ + kTile * kAkQf * 4;
constexpr uint32_t kAkRed = kAkRes;
constexpr uint32_t kAkDst = kAkRed + kTile * 32;        // [128] flux-partial index of each key
constexpr uint32_t kAkCnt = kAkDst + kTile * 4;         // [8] ints: warp counts, next unit, stop
constexpr uint32_t kAkBar = kAkCnt + 32;                // two mbarriers: layer 1, layer 2
constexpr uint32_t kAkMisc = kAkBar + 16;               // tmem slot, (unused), abort
constexpr uint32_t kAkB2 = kAkMisc + 16;                // [8] the output bias
constexpr uint32_t kAkSmem = kAkB2 + 32;
constexpr uint32_t kAkTmemCols = 2 * kTmemCols;         // two steps in flight

// Two direction steps are in flight per CTA: while the hidden layer and the outputs
// of step j run, step j+1's features are in its own X tile and its first layer in its
// own TMEM region (64 columns each), so one CTA barrier a step separates the phases:
//   features(j+1) -> X[(j+1)&1] | wait layer 1 (j) | hidden(j) -> TMEM region j&1 |
//   barrier | issue layer 2 (j), layer 1 (j+1) | wait layer 2 (j) | outputs(j)
template <int MODE>
__global__ void __launch_bounds__(kTile, MODE == ANN_UNGATED ? 4 : 3) sweep_ann_wave(AnnKeyArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    int *misc = reinterpret_cast<int *>(smem + kAkMisc);
    const uint32_t tbase = ann_setup(smem, a.ann, kAkW1, kAkW2, kAkBar, misc, kAkTmemCols, 2);
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t sbase = smem_u32(smem), barA = sbase + kAkBar, barB = barA + 8;
    const uint32_t twarp = tbase + ((uint32_t)(t & ~31) << 16);
    float4 *sdir = reinterpret_cast<float4 *>(smem + kAkDir), *sdab = reinterpret_cast<float4 *>(smem + kAkDab);
    float *ssrc = reinterpret_cast<float *>(smem + kAkSrc), *ssig = reinterpret_cast<float *>(smem + kAkKey);
    uint4 *soff = reinterpret_cast<uint4 *>(smem + kAkOff);
    float *sq = reinterpret_cast<float *>(smem + kAkQ), *sres = reinterpret_cast<float *>(smem + kAkRes);
    float *sred = reinterpret_cast<float *>(smem + kAkRed);
    int *sdst = reinterpret_cast<int *>(smem + kAkDst), *cnt = reinterpret_cast<int *>(smem + kAkCnt);
    const int Do = a.Do, G = a.G;
    for (int e = t; e < Do; e += kTile) {
        sdir[e] = a.dir[e];
        sdab[e] = a.dir_abs[e];
    }
    // the output bias from shared memory (registers are the gated modes' limit)
    float *b2 = reinterpret_cast<float *>(smem + kAkB2);
    if (t < 8) b2[t] = a.ann.b2[t];
    const float lsig_scale = 0.69314718f / kLogSigScale;   // log2 -> the sigma_t input
    uint32_t phA = 0, phB = 0;
    unsigned long long nfb = 0;
    bool late = false, stop = false;
    if (t == 0) cnt[4] = (int)atomicAdd(a.w.next, 1u);
    __syncthreads();
    while (!stop) {
        const int u = cnt[4];
        if (u >= a.w.nunits) break;
        __syncthreads();   // every thread has read the unit index
        const int4 ud = a.w.units[u];
        const int4 up = a.w.uplane[u];
        if (t == 0) cnt[4] = (int)atomicAdd(a.w.next, 1u);
        const int o = (ud.y >> 12) & 7, lch = (ud.y >> 15) & 7;
        const uint32_t c0 = up.x;
        const int nkeys = (int)up.y;
        const int KB = kTile >> lch, nch = 1 << lch;
        const int chunk = t >> (31 - __clz(KB)), lk = t & (KB - 1);
        const int key = ud.x + lk;
        const bool act = key < nkeys;
        const int d0 = chunk * Do / nch, d1 = (chunk + 1) * Do / nch;
        const int nsteps = (Do + nch - 1) / nch;

        // the key (inputs of the sweep and set-up tables only: before the wait)
        float sig = 0.f, smax = 0.f, lsig = 0.f;
        uint32_t ou0 = 0, ou1 = 0, ou2 = 0, inb = 0, bnd = 0, row0 = 0;
        int dst = -1;
        if (act) {
            const uint32_t cidx = a.divG.div((uint32_t)key);
            const int g = key - (int)cidx * G;
            const uint32_t pk = a.w.all_cells[c0 + cidx];
            const int ip = pk & 1023, jp = (pk >> 10) & 1023, kp = pk >> 20;
            const int i = (o & 1) ? a.nx - 1 - ip : ip;
            const int j = (o & 2) ? a.ny - 1 - jp : jp;
            const int k = (o & 4) ? a.nz - 1 - kp : kp;
            const int c = i + a.nx * (j + a.ny * k);
            const int gc = g * a.C + c;
            sig = __ldg(a.sigt + gc);
            const float4 s0 = __ldg(reinterpret_cast<const float4 *>(a.S) + 2 * (int64_t)gc);
            const float4 s1 = __ldg(reinterpret_cast<const float4 *>(a.S) + 2 * (int64_t)gc + 1);
            float Sc[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
            mirror8(Sc, o);      // canonical node n = physical n ^ o
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                ssrc[t * 8 + n] = Sc[n];
                smax = fmaxf(smax, fabsf(Sc[n]));
            }
            lsig = lg2_approx(fmaxf(sig, kSigFloor)) * lsig_scale;
            const uint32_t DG = (uint32_t)(Do * G), first = (uint32_t)(d0 * G + g);
            ou0 = (uint32_t)(o * a.ny * a.nz + jp + a.ny * kp) * DG + first;
            ou1 = a.off_y + (uint32_t)(o * a.nx * a.nz + ip + a.nx * kp) * DG + first;
            ou2 = a.off_z + (uint32_t)(o * a.nx * a.ny + ip + a.nx * jp) * DG + first;
            inb = a.off_in + 6u * (uint32_t)g;
            bnd = (ip == 0 ? 1u : 0u) | (jp == 0 ? 2u : 0u) | (kp == 0 ? 4u : 0u);
            dst = (o * a.C + c) * G + g;
            row0 = (uint32_t)dst * (uint32_t)Do + (uint32_t)d0;
        }
        ssig[t] = sig;
        soff[t] = make_uint4(ou0, ou1, ou2, (uint32_t)d0);
        sdst[t] = dst;
        if (t < 32) {
            const bool fine = wave_wait_deps_warp(a.w, ud.z, ud.w, up.z, up.w);
            if (t == 0) cnt[5] = fine ? 0 : 1;
        }
        __syncthreads();
        if (cnt[5]) break;

        constexpr uint32_t AX = kTile * 16, SP = 3 * AX;
        const uint32_t sb = sbase + kAkStage + 16 * t;
        // inflow faces of step jj (direction d0 + jj) into stage buffer jj & 1; the
        // face offsets ou* point at the current step's slots, `ahead` steps before jj
        auto issue = [&](int jj, int ahead) {
            const uint32_t step = (uint32_t)ahead * (uint32_t)G;
            const uint32_t nb = sb + (uint32_t)(jj & 1) * SP;
            cp_async16(nb, a.face + ((bnd & 1u) ? inb + (uint32_t)(o & 1) : ou0 + step));
            cp_async16(nb + AX, a.face + ((bnd & 2u) ? inb + 2u + (uint32_t)((o >> 1) & 1) : ou1 + step));
            cp_async16(nb + 2 * AX, a.face + ((bnd & 4u) ? inb + 4u + (uint32_t)((o >> 2) & 1) : ou2 + step));
        };
        // step jj's faces from its stage into registers, its scale, and (valid rows)
        // its X row in tile jj & 1
        auto features = [&](int jj, float (&f)[12], float &scale) {
            const float4 *stg = reinterpret_cast<const float4 *>(smem + kAkStage) + (jj & 1) * 3 * kTile + t;
            const float4 fx = stg[0], fy = stg[kTile], fz = stg[2 * kTile];
            f[0] = fx.x; f[1] = fx.y; f[2] = fx.z; f[3] = fx.w;
            f[4] = fy.x; f[5] = fy.y; f[6] = fy.z; f[7] = fy.w;
            f[8] = fz.x; f[9] = fz.y; f[10] = fz.z; f[11] = fz.w;
            scale = 0.f;
            if (!(act && d0 + jj < d1)) return;
            scale = smax;
#pragma unroll
            for (int q = 0; q < 12; ++q) scale = fmaxf(scale, fabsf(f[q]));
            const float inv = scale > kScaleFloor ? rcp_approx(scale) : 0.f;
            const float4 ab = sdab[d0 + jj];
            float x[kNin];
            x[0] = 2.f * ab.x - 1.f; x[1] = 2.f * ab.y - 1.f; x[2] = 2.f * ab.z - 1.f;
            x[3] = a.lhx; x[4] = a.lhy; x[5] = a.lhz;
            x[6] = lsig;
#pragma unroll
            for (int n = 0; n < 8; ++n) x[7 + n] = ssrc[t * 8 + n] * inv;
#pragma unroll
            for (int q = 0; q < 12; ++q) x[15 + q] = f[q] * inv;
            write_x_row(smem + kAkX + (uint32_t)(jj & 1) * kXBytes, t, x);
        };

        float phi[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) phi[n] = 0.f;
        float fc[12], fn[12], sc = 0.f, scn = 0.f;
        // prologue: step 0's faces and features, step 1's faces in flight, layer 1 (0)
        if (act && d0 < d1) issue(0, 0);
        cp_async_commit();
        if (act && d0 + 1 < d1) issue(1, 1);
        cp_async_commit();
        cp_async_wait_pending<1>();
        features(0, fc, sc);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) {
            mma_layer1(sbase, kAkX, kAkW1, tbase, barA);
        }
        for (int jst = 0; jst < nsteps; ++jst) {
            const int d = d0 + jst;
            const bool valid = act && d < d1;
            const uint32_t treg = (uint32_t)(jst & 1) * kTmemCols;   // this step's TMEM region
            const bool more = jst + 1 < nsteps;
            // step j+1: its faces have landed (step j+2's start copying), its features
            if (more) {
                if (act && d + 2 < d1) issue(jst + 2, 2);
                cp_async_commit();
                cp_async_wait_pending<1>();
                features(jst + 1, fn, scn);
            }
            // step j: layer 1 done -> hidden layer into its region
            if (lane == 0) late = !mbar_wait_bounded(barA, phA);
            __syncwarp();
            phA ^= 1u;
            tc_fence_after();
            hidden_to_tmem(twarp + treg);
            fence_async_smem();
            tc_fence_before();
            if (__syncthreads_or(late)) { stop = true; break; }
            tc_fence_after();
            if (t == 0) {
                mma_layer2(sbase, kAkW2, tbase + treg, barB);
                if (more) mma_layer1(sbase, kAkX + (uint32_t)((jst + 1) & 1) * kXBytes, kAkW1,
                                     tbase + (treg ^ kTmemCols), barA);
            }
            if (lane == 0) late = !mbar_wait_bounded(barB, phB);
            __syncwarp();
            phB ^= 1u;
            tc_fence_after();
            uint32_t r8[8];
            tmem_ld8(twarp + treg + 32, r8);
            tmem_wait_ld();
            float psi[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) psi[q] = sc * (__uint_as_float(r8[q]) + b2[q]);
            const float4 dd = valid ? sdir[d] : make_float4(0.f, 0.f, 0.f, 0.f);
            bool keep = valid;
            if (MODE == ANN_GATED && valid && sc != 0.f) {
                CanonCell<float> cc;
                cc.t3x = dd.x; cc.t3y = dd.y; cc.t3z = dd.z; cc.sig = sig; cc.mask = o;
#pragma unroll
                for (int n = 0; n < 8; ++n) cc.S[n] = ssrc[t * 8 + n];
#pragma unroll
                for (int q = 0; q < 4; ++q) { cc.ux[q] = fc[q]; cc.uy[q] = fc[4 + q]; cc.uz[q] = fc[8 + q]; }
                keep = gate_pass(cc, psi, a.ann.tau);
            }
            if (MODE == ANN_GATED && valid && a.record && keep) {
                const uint32_t r = row0 + (uint32_t)jst;
                atomicOr(a.mask + (r >> 5), 1u << (r & 31));
            }
            if (MODE == ANN_FROZEN && valid) {
                const uint32_t r = row0 + (uint32_t)jst;
                keep = (__ldg(a.mask + (r >> 5)) >> (r & 31)) & 1u;
            }
            if (keep) {
                a.face[ou0] = make_float4(psi[1], psi[3], psi[5], psi[7]);
                a.face[ou1] = make_float4(psi[2], psi[3], psi[6], psi[7]);
                a.face[ou2] = make_float4(psi[4], psi[5], psi[6], psi[7]);
#pragma unroll
                for (int n = 0; n < 8; ++n) phi[n] = fmaf(dd.w, psi[n], phi[n]);
            }
            if (MODE != ANN_UNGATED) {
                // rejected rows to the first threads of the CTA, in thread order
                const bool rej = valid && !keep;
                const unsigned m = __ballot_sync(0xffffffffu, rej);
                if (lane == 0) cnt[wid] = __popc(m);
                __syncthreads();
                int base = 0, total = 0;
#pragma unroll
                for (int w2 = 0; w2 < kTile / 32; ++w2) {
                    base += w2 < wid ? cnt[w2] : 0;
                    total += cnt[w2];
                }
                if (rej) {
                    float *e = sq + kAkQf * (base + __popc(m & ((1u << lane) - 1u)));
#pragma unroll
                    for (int q = 0; q < 12; ++q) e[q] = fc[q];
                    e[12] = __int_as_float(t);
                    e[13] = __int_as_float(d);
                }
                __syncthreads();
                if (t < total) {
                    const float *e = sq + kAkQf * t;
                    const int ow = __float_as_int(e[12]), de = __float_as_int(e[13]);
                    const float4 de4 = sdir[de];
                    float Sm[8];
#pragma unroll
                    for (int n = 0; n < 8; ++n) Sm[n] = ssrc[ow * 8 + n];
                    mh_axis<0>(Sm);
                    mh_axis<1>(Sm);
                    mh_axis<2>(Sm);
                    const float gx[4] = {e[0], e[1], e[2], e[3]}, gy[4] = {e[4], e[5], e[6], e[7]},
                                gz[4] = {e[8], e[9], e[10], e[11]};
                    float xg[8];
                    cell_solve_key<true>(de4.x, de4.y, de4.z, ssig[ow], Sm, gx, gy, gz, xg);
                    const uint4 of = soff[ow];
                    const uint32_t dG = (uint32_t)(de - (int)of.w) * (uint32_t)G;
                    a.face[of.x + dG] = make_float4(xg[1], xg[3], xg[5], xg[7]);
                    a.face[of.y + dG] = make_float4(xg[2], xg[3], xg[6], xg[7]);
                    a.face[of.z + dG] = make_float4(xg[4], xg[5], xg[6], xg[7]);
#pragma unroll
                    for (int n = 0; n < 8; ++n) sres[ow * 8 + n] = de4.w * xg[n];
                }
                if (t == 0) nfb += (unsigned long long)total;
                __syncthreads();
                if (rej) {
#pragma unroll
                    for (int n = 0; n < 8; ++n) phi[n] += sres[t * 8 + n];
                }
            }
            ou0 += (uint32_t)G;
            ou1 += (uint32_t)G;
            ou2 += (uint32_t)G;
#pragma unroll
            for (int q = 0; q < 12; ++q) fc[q] = fn[q];
            sc = scn;
        }
        if (!stop && __syncthreads_or(late)) stop = true;   // the last step's layer-2 wait
        if (stop) {
            if (t == 0) {
                misc[2] = 1;   // counted as a timed-out CTA by the teardown
                *reinterpret_cast<volatile double *>(a.w.abort) = 1.0;
            }
            break;
        }
        mirror8(phi, o);   // physical node order
        if (lch == 0) {
            if (act) {
                float4 *p = reinterpret_cast<float4 *>(a.phi_oct) + 2 * (int64_t)dst;
                p[0] = make_float4(phi[0], phi[1], phi[2], phi[3]);
                p[1] = make_float4(phi[4], phi[5], phi[6], phi[7]);
            }
        } else {
            float4 *r = reinterpret_cast<float4 *>(sred + (chunk * KB + lk) * 8);
            r[0] = make_float4(phi[0], phi[1], phi[2], phi[3]);
            r[1] = make_float4(phi[4], phi[5], phi[6], phi[7]);
            __syncthreads();
            for (int e = t; e < KB * 8; e += kTile) {
                const int kk = e >> 3, n = e & 7;
                const int dk = sdst[kk];
                if (dk < 0) continue;
                float sum = sred[kk * 8 + n];
                for (int q = 1; q < nch; ++q) sum += sred[(q * KB + kk) * 8 + n];
                a.phi_oct[(int64_t)dk * 8 + n] = sum;
            }
        }
        __syncthreads();   // every store of this unit has been issued
        if (t == 0) wave_done(a.w, u);
    }
    cp_async_wait_all();
    if (MODE != ANN_UNGATED && t == 0 && nfb) atomicAdd(a.ann.counter, nfb);
    ann_teardown(tbase, a.ann, misc, kAkTmemCols);
}

// The surrogate key sweep of every hyperplane (one persistent launch) and the
// boundary-leakage sum; false if the handle has no unit tables.
static sn_status launch_sweep_ann_keys(sn_handle h, const float *S, float *phi_oct, int mode, bool record,
                                       cudaStream_t st)
{
    Net *net = net_of(h);
    const WaveTables *wt = static_cast<const WaveTables *>(h->wave);
    AnnKeyArgs a = {};
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.G = h->G; a.Do = h->Do; a.C = (int)h->ncell;
    a.divG = FastDiv((uint32_t)h->G);
    a.sigt = (const float *)h->sigt;
    a.S = S;
    a.dir = reinterpret_cast<const float4 *>(h->dir);
    a.dir_abs = h->dir_abs;
    a.face = reinterpret_cast<float4 *>(h->face);
    a.off_y = (uint32_t)h->face_x;
    a.off_z = (uint32_t)(h->face_x + h->face_y);
    a.off_in = (uint32_t)h->face_in;
    a.phi_oct = phi_oct;
    a.lhx = (logf((float)h->dx) + kLogHShift) / kLogHScale;
    a.lhy = (logf((float)h->dy) + kLogHShift) / kLogHScale;
    a.lhz = (logf((float)h->dz) + kLogHShift) / kLogHScale;
    a.ann = ann_args(h);
    a.mask = net->mask;
    a.record = record ? 1 : 0;
    a.w = wave_ctl(h);
    void (*kern)(AnnKeyArgs) = mode == ANN_UNGATED ? sweep_ann_wave<ANN_UNGATED>
                               : mode == ANN_GATED ? sweep_ann_wave<ANN_GATED> : sweep_ann_wave<ANN_FROZEN>;
    SN_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAkSmem));
    // CTAs an SM: the kernel's register bound (4 ungated, 3 with the elimination's
    // registers), its shared memory (plus the 1 KB the driver reserves a CTA) within
    // 228 KB, and 128 of the SM's 512 TMEM columns each (the occupancy query does not
    // see the carveout set below and answers 1)
    int per_sm = mode == ANN_UNGATED ? 4 : 3;
    per_sm = std::min(per_sm, (int)((228 * 1024) / (kAkSmem + 1024)));
    per_sm = std::max(1, std::min(per_sm, (int)(512 / kAkTmemCols)));
    // The unified L1 / shared array: the whole of it as shared memory for the ungated
    // kernel (4 CTAs of 55 KB), and no more than its 3 CTAs take for the gated modes,
    // whose elimination spills a few registers: their local-memory traffic then stays in
    // L1 (with the whole array as shared memory it went to L2; the frozen sweep at half
    // the rows to elimination took 11.1 ms that way on blocked_64, 10.6 ms this way).
    int carve = (int)cudaSharedmemCarveoutMaxShared;
    if (mode != ANN_UNGATED)
        carve = std::min(100, (int)((100 * (int64_t)per_sm * (kAkSmem + 1024) + 228 * 1024 - 1) / (228 * 1024)));
    SN_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    SN_CK(h, cudaMemsetAsync(wt->flags, 0, sizeof(uint32_t) * (size_t)(wt->nunits + 1), st));
    if (record) SN_CK(h, cudaMemsetAsync(net->mask, 0, sizeof(uint32_t) * (size_t)net->mask_words, st));
    if (h->prof) SN_CK(h, cudaEventRecord(h->ev_sweep[0], st));
    kern<<<per_sm * num_sms(), kTile, kAkSmem, st>>>(a);
    SN_CK(h, cudaGetLastError());
    if (h->prof) {
        SN_CK(h, cudaEventRecord(h->ev_sweep[1], st));
        h->prof_pending = true;
    }
    return launch_leak_keys(h, st);
}

bool ann_frozen(sn_handle h)
{
    return h->net && net_of(h)->mask && net_of(h)->frozen_gen == h->net_gen;
}

sn_status launch_sweep_ann(sn_handle h, const float *S, float *phi_oct, int ann_mode, cudaStream_t st)
{
    sn_status s = pack_if_dirty(h, st);
    if (s != SN_OK) return s;
    if (key_sweep_ok(h) && h->wave)
        return launch_sweep_ann_keys(h, S, phi_oct, ann_mode, false, st);
    if (ann_mode == ANN_FROZEN) return fail(h, SN_EINVAL, "frozen gate: needs the key sweep");
    const bool gated = ann_mode == ANN_GATED;
    Net *net = net_of(h);
    AnnSweepArgs a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.G = h->G; a.Do = h->Do; a.C = (int)h->ncell;
    a.divG = FastDiv((uint32_t)h->G);
    a.keys_per_tile = kTile / h->Do;
    a.sigt = (const float *)h->sigt; a.S = S; a.psi_inc = (const float *)h->psi_inc;
    a.dir = (const DirData<float> *)h->dir;
    a.dir_abs = h->dir_abs;
    a.fx = (Vec4<float> *)h->face;
    a.fy = a.fx + h->face_x;
    a.fz = a.fy + h->face_y;
    a.phi_oct = phi_oct;
    a.leak = h->acc + ACC_LEAK;
    a.vol12 = (float)(h->dx * h->dy * h->dz / 12.0);
    a.hx = (float)h->dx; a.hy = (float)h->dy; a.hz = (float)h->dz;
    a.fb_queue = net->fb_queue;
    a.ann = ann_args(h);
    const SweepSmem L = sweep_smem(a.keys_per_tile);
    // CTAs per SM: shared memory (plus the 1 KB the driver reserves per CTA) within the
    // SM's 228 KB, 64 TMEM columns each (at most 8), and the kernels' register bounds
    auto pick = [&](auto kern, int &per_sm) -> sn_status {
        SN_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
        SN_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
        per_sm = std::min((int)((228 * 1024) / (L.total + 1024)), (int)(512 / kTmemCols));
        if (gated) per_sm = std::min(per_sm, 6);
        per_sm = std::max(per_sm, 1);
        return SN_OK;
    };
    void (*kern)(AnnSweepArgs) = nullptr;
    if (gated)
        kern = h->Do == 10 ? sweep_plane_ann<true, 10> : h->Do == 21 ? sweep_plane_ann<true, 21> : sweep_plane_ann<true, 0>;
    else
        kern = h->Do == 10 ? sweep_plane_ann<false, 10> : h->Do == 21 ? sweep_plane_ann<false, 21> : sweep_plane_ann<false, 0>;
    int per_sm = 1;
    s = pick(kern, per_sm);
    if (s != SN_OK) return s;
    if (gated) SN_CK(h, cudaMemsetAsync(net->fb_count, 0, sizeof(uint32_t) * (size_t)h->nplanes, st));
    // persistent CTAs per octant: as many as fit on the SMs
    const int cap = std::max(1, num_sms() * per_sm / 8);
    const int fb_grid = num_sms() * 4;
    if (h->prof) SN_CK(h, cudaEventRecord(h->ev_sweep[0], st));
    for (int p = 0; p < h->nplanes; ++p) {
        const int64_t n = h->plane_off[p + 1] - h->plane_off[p];
        a.cells = h->plane_cells + h->plane_off[p];
        a.ncells_plane = (int)n;
        a.ntiles = (int)((n * h->G + a.keys_per_tile - 1) / a.keys_per_tile);
        a.fb_count = net->fb_count + p;
        const dim3 grid((unsigned)(a.ntiles < cap ? a.ntiles : cap), 8);
        // later hyperplanes (and the fallback passes) overlap their launch and set-up
        // with the previous kernel's drain
        SN_CK(h, launch_k(p > 0, kern, grid, dim3(kTile), L.total, st, a));
        if (gated) SN_CK(h, launch_k(true, ann_fallback_kernel, dim3(fb_grid), dim3(128), 0, st, a));
    }
    SN_CK(h, cudaGetLastError());
    if (h->prof) {
        SN_CK(h, cudaEventRecord(h->ev_sweep[1], st));
        h->prof_pending = true;
    }
    return SN_OK;
}

static sn_status need_net(sn_handle h, const char *who)
{
    if (!h) return fail(nullptr, SN_EINVAL, std::string(who) + ": NULL handle");
    if (!h->has_net) return fail(h, SN_ESTATE, std::string(who) + ": no network (train, init or set weights first)");
    return SN_OK;
}

static sn_status apply_cells(sn_handle h, const float *in27, float *psi, int64_t n, bool gated, int64_t *n_fallback,
                             cudaStream_t st)
{
    Net *net = net_of(h);
    sn_status s = pack_if_dirty(h, st);
    if (s != SN_OK) return s;
    SN_CK(h, cudaMemsetAsync(net->counter, 0, sizeof(unsigned long long) * 2, st));
    if (n > 0) {
        int64_t grid = (n + kTile - 1) / kTile;
        const int64_t cap = (int64_t)num_sms() * 4;
        if (grid > cap) grid = cap;
        const AnnArgs a = ann_args(h);
        if (gated) {
            SN_CK(h, cudaFuncSetAttribute(ann_cells_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCellSmem));
            ann_cells_kernel<true><<<(unsigned)grid, kTile, kCellSmem, st>>>(in27, psi, n, a);
        } else {
            SN_CK(h, cudaFuncSetAttribute(ann_cells_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCellSmem));
            ann_cells_kernel<false><<<(unsigned)grid, kTile, kCellSmem, st>>>(in27, psi, n, a);
        }
        SN_CK(h, cudaGetLastError());
    }
    unsigned long long c[2] = {0, 0};
    SN_CK(h, cudaMemcpyAsync(c, net->counter, sizeof(c), cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    if (c[1]) return fail(h, SN_ETIMEOUT, "surrogate: a tensor-core completion wait timed out");
    if (n_fallback) *n_fallback = (int64_t)c[0];
    return SN_OK;
}

// ---------------------------------------------------------------------------------
// Allocation-free gradient of the training loss.
//
// sn_surrogate_grad needs a handle (created with device allocations) and allocates a
// temporary gradient buffer on every call.  Some callers cannot do that: code that
// issues its work while a stream is being captured in global capture mode (where
// cudaMalloc is refused), code whose device memory is a fixed pool handed out in
// advance, and latency-bound loops that must not pay for the device-wide
// synchronisation a cudaMalloc/cudaFree pair can cause.  This variant takes every
// input and output as caller-owned device memory and keeps the per-block partial
// gradients in the fixed array below instead of allocated scratch.
//
// The array lives in every GPU that loads the library until the process exits:
// kNoAllocMaxBlocks * 2312 floats + kNoAllocMaxBlocks doubles = 2.37 MB, which caps a
// call at kNoAllocMaxBlocks * 128 = 32768 rows.  Every call uses it from the start,
// so calls that overlap on the GPU (different streams, or different host threads on
// one device) race on it; calls queued on one stream are ordered and safe.  Each call
// writes all the partials it later reads, so no part of the array has to start at
// zero.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and sets the gradient kernel's
// shared-memory attribute; make that first call before any stream capture begins.
// The address is kept for the life of the process: a device reset (cudaDeviceReset,
// or a reset of the primary context) reloads the module and invalidates it, so after
// a reset this entry point must not be called again in the same process.
// ---------------------------------------------------------------------------------
constexpr int kNoAllocMaxBlocks = 256;
static __device__ __align__(256) float g_noalloc_gpart[kNoAllocMaxBlocks * kNparam];
static __device__ __align__(256) double g_noalloc_lpart[kNoAllocMaxBlocks];

static std::mutex g_noalloc_mutex;
static float *g_noalloc_gpart_ptr[64];
static double *g_noalloc_lpart_ptr[64];

static sn_status noalloc_scratch(float **gpart, double **lpart)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(nullptr, SN_ECUDA, "sn_surrogate_grad_noalloc: device index above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_gpart_ptr[dev]) {
        void *pg = nullptr, *pl = nullptr;
        e = cudaGetSymbolAddress(&pg, g_noalloc_gpart);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(gradient partials)");
        e = cudaGetSymbolAddress(&pl, g_noalloc_lpart);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(loss partials)");
        e = cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaFuncSetAttribute");
        g_noalloc_lpart_ptr[dev] = static_cast<double *>(pl);
        g_noalloc_gpart_ptr[dev] = static_cast<float *>(pg);
    }
    *gpart = g_noalloc_gpart_ptr[dev];
    *lpart = g_noalloc_lpart_ptr[dev];
    return SN_OK;
}

}  // namespace sn

extern "C" sn_status sn_surrogate_grad_noalloc(const float *params, const float *feat, const float *targ, int64_t n,
                                                float *grad, double *loss, void *stream)
{
    using namespace sn;
    if (!params || !feat || !targ || !grad || !loss)
        return fail(nullptr, SN_EINVAL, "sn_surrogate_grad_noalloc: NULL pointer");
    if (n < 1 || n > (int64_t)kNoAllocMaxBlocks * 128)
        return fail(nullptr, SN_EINVAL, "sn_surrogate_grad_noalloc: n must be in 1..32768 (fixed scratch of 256 "
                                        "blocks of 128 rows)");
    float *gpart = nullptr;
    double *lpart = nullptr;
    sn_status s = noalloc_scratch(&gpart, &lpart);
    if (s != SN_OK) return s;
    const cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)((n + 127) / 128);
    grad_kernel<<<nblk, 128, kGradSmem, st>>>(params, feat, targ, n, 0, (int)n, 1.f / (float)n, gpart, lpart);
    adam_kernel<<<(kNparam + 255) / 256, 256, 0, st>>>(nullptr, nullptr, nullptr, gpart, nblk, 0.f, 1.f, 1.f, grad, 0);
    sum_kernel<<<1, 32, 0, st>>>(lpart, nblk, loss);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "sn_surrogate_grad_noalloc");
    return SN_OK;
}

namespace sn {

// Host-side uniform initialisation (SplitMix64 stream), +-1/sqrt(fan_in).
static void init_params(std::vector<float> &p, uint64_t seed)
{
    uint64_t x = seed;
    auto next = [&x]() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    p.resize(kNparam);
    const double a1 = 1.0 / std::sqrt((double)kNin), a2 = 1.0 / std::sqrt((double)kNhid);
    int e = 0;
    for (int i = 0; i < kNhid * kNin + kNhid; ++i) p[e++] = (float)((2.0 * next() - 1.0) * a1);
    for (int i = 0; i < kNout * kNhid + kNout; ++i) p[e++] = (float)((2.0 * next() - 1.0) * a2);
}

static sn_status upload_params(sn_handle h, const float *host)
{
    sn_status s = ensure_net(h);
    if (s != SN_OK) return s;
    Net *n = net_of(h);
    SN_CK(h, cudaMemcpyAsync(n->p, host, sizeof(float) * kNparam, cudaMemcpyHostToDevice, h->stream));
    SN_CK(h, cudaMemsetAsync(n->m, 0, sizeof(float) * kNparam, h->stream));
    SN_CK(h, cudaMemsetAsync(n->v, 0, sizeof(float) * kNparam, h->stream));
    SN_CK(h, cudaStreamSynchronize(h->stream));
    n->t = 0;
    n->dirty = true;
    h->has_net = true;
    h->net_gen++;
    return SN_OK;
}

static sn_status ensure_gpart(sn_handle h, int64_t blocks)
{
    Net *n = net_of(h);
    if (n->gpart_blocks >= blocks) return SN_OK;
    if (n->gpart) cudaFree(n->gpart);
    if (n->lpart) cudaFree(n->lpart);
    n->gpart = nullptr;
    n->lpart = nullptr;
    n->gpart_blocks = 0;
    SN_CK(h, cudaMalloc(&n->gpart, sizeof(float) * kNparam * blocks));
    SN_CK(h, cudaMalloc(&n->lpart, sizeof(double) * blocks));
    n->gpart_blocks = blocks;
    return SN_OK;
}

// one gradient evaluation (and optionally one Adam step) on `batch` rows from row0
static sn_status grad_step(sn_handle h, const float *feat, const float *targ, int64_t nrows, int64_t row0, int batch,
                           float lr, bool step, float *gout, cudaStream_t st)
{
    Net *n = net_of(h);
    const int nblk = (batch + 127) / 128;
    sn_status s = ensure_gpart(h, nblk);
    if (s != SN_OK) return s;
    SN_CK(h, cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem));
    grad_kernel<<<nblk, 128, kGradSmem, st>>>(n->p, feat, targ, nrows, row0, batch, 1.f / (float)batch, n->gpart,
                                              n->lpart);
    float bc1 = 1.f, bc2 = 1.f;
    if (step) {
        n->t += 1;
        bc1 = (float)(1.0 - std::pow(0.9, (double)n->t));
        bc2 = (float)(1.0 - std::pow(0.999, (double)n->t));
        n->dirty = true;
        h->net_gen++;
    }
    adam_kernel<<<(kNparam + 255) / 256, 256, 0, st>>>(n->p, n->m, n->v, n->gpart, nblk, lr, bc1, bc2, gout,
                                                       step ? 1 : 0);
    sum_kernel<<<1, 32, 0, st>>>(n->lpart, nblk, n->dacc);
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

static sn_status mean_abs_err(sn_handle h, const float *feat, const float *targ, int64_t n, double *mae,
                              cudaStream_t st)
{
    Net *net = net_of(h);
    SN_CK(h, cudaMemsetAsync(net->dacc + 1, 0, sizeof(double), st));
    if (n > 0) {
        int64_t grid = (n + 127) / 128;
        if (grid > (int64_t)num_sms() * 8) grid = (int64_t)num_sms() * 8;
        mae_kernel<<<(unsigned)grid, 128, 0, st>>>(net->p, feat, targ, n, net->dacc + 1);
        SN_CK(h, cudaGetLastError());
    }
    double v = 0.0;
    SN_CK(h, cudaMemcpyAsync(&v, net->dacc + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    *mae = n > 0 ? v / (8.0 * (double)n) : 0.0;
    return SN_OK;
}

static sn_status launch_prepare(sn_handle h, const float *in27, int64_t n, float *feat, float *targ, cudaStream_t st)
{
    if (n <= 0) return SN_OK;
    int64_t grid = (n + 127) / 128;
    if (grid > (int64_t)num_sms() * 16) grid = (int64_t)num_sms() * 16;
    prepare_kernel<<<(unsigned)grid, 128, 0, st>>>(in27, n, feat, targ);
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

static sn_status fit_loop(sn_handle h, const float *feat, const float *targ, int64_t nrows, int steps, int batch,
                          float lr, double *last_loss, cudaStream_t st)
{
    Net *n = net_of(h);
    for (int k = 0; k < steps; ++k) {
        const int64_t row0 = ((int64_t)k * batch) % nrows;
        sn_status s = grad_step(h, feat, targ, nrows, row0, batch, lr, true, nullptr, st);
        if (s != SN_OK) return s;
    }
    if (last_loss) {
        SN_CK(h, cudaMemcpyAsync(last_loss, n->dacc, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    SN_CK(h, cudaStreamSynchronize(st));
    return SN_OK;
}

}  // namespace sn

using namespace sn;

extern "C" {

sn_status sn_surrogate_prepare(const float *in27, int64_t n, float *feat, float *targ, void *stream)
{
    if (n < 0) return fail(nullptr, SN_EINVAL, "sn_surrogate_prepare: n < 0");
    if (n > 0 && (!in27 || !feat || !targ)) return fail(nullptr, SN_EINVAL, "sn_surrogate_prepare: NULL pointer");
    return launch_prepare(nullptr, in27, n, feat, targ, (cudaStream_t)stream);
}

sn_status sn_surrogate_init(sn_handle h, uint64_t seed)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_surrogate_init: NULL handle");
    std::vector<float> p;
    init_params(p, seed);
    return upload_params(h, p.data());
}

sn_status sn_surrogate_set_weights(sn_handle h, const float *params)
{
    if (!h || !params) return fail(h, SN_EINVAL, "sn_surrogate_set_weights: NULL argument");
    for (int i = 0; i < kNparam; ++i)
        if (!std::isfinite(params[i])) return fail(h, SN_EINVAL, "sn_surrogate_set_weights: non-finite weight");
    return upload_params(h, params);
}

sn_status sn_surrogate_get_weights(sn_handle h, float *params)
{
    sn_status s = need_net(h, "sn_surrogate_get_weights");
    if (s != SN_OK) return s;
    if (!params) return fail(h, SN_EINVAL, "sn_surrogate_get_weights: NULL argument");
    SN_CK(h, cudaMemcpyAsync(params, net_of(h)->p, sizeof(float) * kNparam, cudaMemcpyDeviceToHost, h->stream));
    SN_CK(h, cudaStreamSynchronize(h->stream));
    return SN_OK;
}

sn_status sn_surrogate_set_gate(sn_handle h, float tau)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_surrogate_set_gate: NULL handle");
    if (!(tau >= 0.f) || !std::isfinite(tau)) return fail(h, SN_EINVAL, "sn_surrogate_set_gate: tau must be >= 0");
    sn_status s = ensure_net(h);
    if (s != SN_OK) return s;
    net_of(h)->tau = tau;
    h->net_gen++;
    return SN_OK;
}

sn_status sn_surrogate_grad(sn_handle h, const float *feat, const float *targ, int64_t n, float *grad,
                            double *loss)
{
    sn_status s = need_net(h, "sn_surrogate_grad");
    if (s != SN_OK) return s;
    if (n < 1 || n > (1 << 24) || !feat || !targ || !grad) return fail(h, SN_EINVAL, "sn_surrogate_grad: bad argument");
    Net *net = net_of(h);
    float *dg = nullptr;
    SN_CK(h, cudaMalloc(&dg, sizeof(float) * kNparam));
    s = grad_step(h, feat, targ, n, 0, (int)n, 0.f, false, dg, h->stream);
    if (s == SN_OK) {
        cudaError_t e = cudaMemcpyAsync(grad, dg, sizeof(float) * kNparam, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, net->dacc, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) s = cuda_fail(h, e, "sn_surrogate_grad");
    }
    cudaFree(dg);
    return s;
}

sn_status sn_surrogate_fit(sn_handle h, const float *feat, const float *targ, int64_t nrows, int32_t steps,
                           int32_t batch, float lr, double *last_loss)
{
    sn_status s = need_net(h, "sn_surrogate_fit");
    if (s != SN_OK) return s;
    if (nrows < 1 || steps < 0 || batch < 1 || batch > (1 << 22) || !(lr >= 0.f) || !feat || !targ)
        return fail(h, SN_EINVAL, "sn_surrogate_fit: bad argument");
    return fit_loop(h, feat, targ, nrows, steps, batch, lr, last_loss, h->stream);
}

sn_status sn_surrogate_eval(sn_handle h, const float *feat, const float *targ, int64_t n, double *mae)
{
    sn_status s = need_net(h, "sn_surrogate_eval");
    if (s != SN_OK) return s;
    if (n < 0 || !mae || (n > 0 && (!feat || !targ))) return fail(h, SN_EINVAL, "sn_surrogate_eval: bad argument");
    return mean_abs_err(h, feat, targ, n, mae, h->stream);
}

sn_status sn_surrogate_train(sn_handle h, const float *in27, int64_t n, int64_t n_test, int32_t steps, int32_t batch,
                             float lr, uint64_t seed, double *train_mae, double *test_mae)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_surrogate_train: NULL handle");
    if (n < 2 || n_test < 1 || n_test >= n || !in27 || steps < 0 || batch < 1 || batch > (1 << 22) || !(lr > 0.f))
        return fail(h, SN_EINVAL, "sn_surrogate_train: bad argument");
    const cudaStream_t st = h->stream;
    float *feat = nullptr, *targ = nullptr;
    SN_CK(h, cudaMalloc(&feat, sizeof(float) * kNin * n));
    cudaError_t e = cudaMalloc(&targ, sizeof(float) * 8 * n);
    if (e != cudaSuccess) {
        cudaFree(feat);
        return cuda_fail(h, e, "cudaMalloc");
    }
    sn_status s = launch_prepare(h, in27, n, feat, targ, st);
    if (s == SN_OK) s = sn_surrogate_init(h, seed);
    const int64_t ntr = n - n_test;
    if (s == SN_OK) s = fit_loop(h, feat, targ, ntr, steps, batch, lr, nullptr, st);
    if (s == SN_OK && train_mae) s = mean_abs_err(h, feat, targ, ntr, train_mae, st);
    if (s == SN_OK && test_mae) s = mean_abs_err(h, feat + kNin * ntr, targ + 8 * ntr, n_test, test_mae, st);
    cudaStreamSynchronize(st);
    cudaFree(feat);
    cudaFree(targ);
    return s;
}

sn_status sn_surrogate_apply(sn_handle h, const float *in27, float *psi, int64_t n, int32_t gated, int64_t *n_fallback)
{
    sn_status s = need_net(h, "sn_surrogate_apply");
    if (s != SN_OK) return s;
    if (n < 0 || (n > 0 && (!in27 || !psi))) return fail(h, SN_EINVAL, "sn_surrogate_apply: bad argument");
    return apply_cells(h, in27, psi, n, gated != 0, n_fallback, h->stream);
}

sn_status sn_selftest_wait(sn_handle h, int64_t limit_cycles)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_selftest_wait: NULL handle");
    if (limit_cycles < 1 || limit_cycles > (1LL << 31))
        return fail(h, SN_EINVAL, "sn_selftest_wait: limit_cycles must be in 1..2^31");
    sn_status s = ensure_net(h);
    if (s != SN_OK) return s;
    Net *n = net_of(h);
    AnnArgs a;
    a.w1p = n->w1p; a.w2p = n->w2p; a.b2 = n->b2; a.tau = n->tau; a.counter = n->counter;
    s = reset_ann_counters(h, h->stream);
    if (s != SN_OK) return s;
    wait_selftest_kernel<<<1, 128, 0, h->stream>>>(a, (long long)limit_cycles);
    SN_CK(h, cudaGetLastError());
    return check_ann_timeouts(h);
}

sn_status sn_surrogate_freeze_gate(sn_handle h, const float *S)
{
    sn_status s = need_net(h, "sn_surrogate_freeze_gate");
    if (s != SN_OK) return s;
    if (!S) return fail(h, SN_EINVAL, "sn_surrogate_freeze_gate: NULL source");
    if (!key_sweep_ok(h) || !h->wave)
        return fail(h, SN_EINVAL, "sn_surrogate_freeze_gate: needs an FP32 handle on box cells with isotropic "
                                  "scattering (the key sweep)");
    const uint64_t rows = 8ull * (uint64_t)h->ncell * (uint64_t)h->G * (uint64_t)h->Do;
    if (rows >= (1ull << 32)) return fail(h, SN_EINVAL, "sn_surrogate_freeze_gate: more than 2^32 rows");
    Net *n = net_of(h);
    if (!n->mask) {
        n->mask_words = (int64_t)((rows + 31) / 32);
        SN_CK(h, cudaMalloc(&n->mask, sizeof(uint32_t) * (size_t)n->mask_words));
        h->device_bytes += (int64_t)sizeof(uint32_t) * n->mask_words;
    }
    const cudaStream_t st = h->stream;
    s = pack_if_dirty(h, st);
    if (s != SN_OK) return s;
    SN_CK(h, cudaMemsetAsync(h->acc, 0, sizeof(double) * ACC_COUNT, st));
    s = reset_ann_counters(h, st);
    if (s != SN_OK) return s;
    s = launch_sweep_ann_keys(h, S, static_cast<float *>(h->phi_oct), ANN_GATED, true, st);
    if (s != SN_OK) return s;
    SN_CK(h, cudaMemcpyAsync(h->acc_host, h->acc, sizeof(double) * ACC_COUNT, cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    if (h->acc_host[ACC_ABORT] != 0.0) return fail(h, SN_ETIMEOUT, "sn_surrogate_freeze_gate: a bounded wait gave up");
    s = check_ann_timeouts(h);
    if (s != SN_OK) return s;
    n->frozen_gen = h->net_gen;
    return SN_OK;
}

sn_status sn_surrogate_stats(sn_handle h, int64_t *fallbacks, int64_t *timeouts)
{
    sn_status s = need_net(h, "sn_surrogate_stats");
    if (s != SN_OK) return s;
    unsigned long long c[2] = {0, 0};
    SN_CK(h, cudaMemcpyAsync(c, net_of(h)->counter, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    SN_CK(h, cudaStreamSynchronize(h->stream));
    if (fallbacks) *fallbacks = (int64_t)c[0];
    if (timeouts) *timeouts = (int64_t)c[1];
    return SN_OK;
}

sn_status sn_cell_solve_batch(sn_handle h, const float *in27, float *psi, int64_t n, sn_solve_mode mode, void *stream)
{
    if (n < 0) return fail(h, SN_EINVAL, "sn_cell_solve_batch: n < 0");
    if (mode == SN_SOLVE_GE32R || mode == SN_SOLVE_GE32) {
        if (n == 0) return SN_OK;
        if (!in27 || !psi) return fail(h, SN_EINVAL, "sn_cell_solve_batch: NULL pointer");
        sn_status s = launch_cells_f32(in27, psi, n, mode == SN_SOLVE_GE32R, (cudaStream_t)stream);
        if (s != SN_OK && h) h->err = sn_last_error(nullptr);
        return s;
    }
    if (mode == SN_SOLVE_ANN || mode == SN_SOLVE_ANN_GATED) {
        sn_status s = need_net(h, "sn_cell_solve_batch");
        if (s != SN_OK) return s;
        if (n > 0 && (!in27 || !psi)) return fail(h, SN_EINVAL, "sn_cell_solve_batch: NULL pointer");
        return apply_cells(h, in27, psi, n, mode == SN_SOLVE_ANN_GATED, nullptr, (cudaStream_t)stream);
    }
    if (mode == SN_SOLVE_OCTNET) {
        if (!h) return fail(nullptr, SN_EINVAL, "sn_cell_solve_batch: SN_SOLVE_OCTNET needs a handle");
        if (!h->has_octnet) return fail(h, SN_ESTATE, "sn_cell_solve_batch: no octant networks");
        if (n > 0 && (!in27 || !psi)) return fail(h, SN_EINVAL, "sn_cell_solve_batch: NULL pointer");
        return launch_octnet_cells(h, in27, psi, n, (cudaStream_t)stream);
    }
    return fail(h, SN_EINVAL, "sn_cell_solve_batch: unknown mode");
}

}  // extern "C"

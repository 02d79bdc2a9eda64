// sn_adjoint.cu -- the discrete adjoint of the source-iteration solve: gradients of a
// detector response R = r . phi with respect to the per-cell, per-group sigma_t,
// sigma_s and q (not in the paper; it follows from the discrete system of Sec. 2).
//
// With L the upwind sweep operator of all (direction, group) pairs, Phi psi = phi,
// B the scattering source and Q the external source, (L - B Phi) psi = Q and the
// adjoint solves (L - B Phi)^T lambda = Phi^T r.  Transposing the upwind DFEM
// operator of a direction gives the operator of the opposite direction (the outflow
// form of A(Omega)^T is A(-Omega), and the face couplings transpose onto the
// reversed upwind pattern), so lambda_d = w_d mu_{-d}, where mu solves an ordinary
// vacuum-boundary sweep with the nodal source chi = M^{-1} x,
// x = r + B^T lambda.  The adjoint scalar flux Lam = sum_d lambda_d is then exactly
// what the forward sweep kernel accumulates.  Gradients:
//   dR/dq[g,c]        = (1/4pi) Lam_gc^T M 1 = (V/8)/(4pi) sum_n Lam_gc,n
//   dR/dsigma_s[g',c] = (1/4pi) sum_g xfer[g'][g] Lam_gc^T M phi_g'c
//   dR/dsigma_t[g,c]  = -sum_d lambda_dgc^T M psi_dgc
// The last one pairs every forward angular flux with the adjoint one of the same
// direction; the adjoint sweep meets the cells in the reverse hyperplane order, so
// the forward face planes are checkpointed every K hyperplanes and each block of K
// hyperplanes is recomputed (storing its angular fluxes) just before the adjoint
// pass consumes it -- the full angular flux is never stored.
#include <cmath>
#include <vector>

#include "ge8.cuh"
#include "sn_internal.cuh"

namespace sn {

struct Adj {
    float *chi = nullptr, *Sadj = nullptr, *Sfwd = nullptr, *lam_b = nullptr, *zero_inc = nullptr;
    void *face2 = nullptr;       // forward face planes of the recompute
    char *ckpt = nullptr;        // nblk copies of the face planes
    float *psi_blk = nullptr;    // angular fluxes of one block of hyperplanes
    double *acc2 = nullptr;      // scratch accumulators of the recompute sweeps
    int K = 0, nblk = 0;
    size_t face_bytes = 0;
};

void free_adjoint(sn_handle h)
{
    if (!h || !h->adj) return;
    Adj *a = reinterpret_cast<Adj *>(h->adj);
    void *bufs[] = {a->chi, a->Sadj, a->Sfwd, a->lam_b, a->zero_inc, a->face2, a->ckpt, a->psi_blk, a->acc2};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete a;
    h->adj = nullptr;
}

static sn_status ensure_adjoint(sn_handle h)
{
    if (h->adj) return SN_OK;
    Adj *a = new Adj();
    h->adj = a;
    const size_t GC8 = (size_t)h->G * h->ncell * 8;
    SN_CK(h, cudaMalloc(&a->chi, sizeof(float) * GC8));
    SN_CK(h, cudaMalloc(&a->Sadj, sizeof(float) * GC8));
    SN_CK(h, cudaMalloc(&a->Sfwd, sizeof(float) * GC8));
    SN_CK(h, cudaMalloc(&a->lam_b, sizeof(float) * GC8));
    SN_CK(h, cudaMalloc(&a->zero_inc, sizeof(float) * 6 * h->G));
    SN_CK(h, cudaMemsetAsync(a->zero_inc, 0, sizeof(float) * 6 * h->G, h->stream));
    SN_CK(h, cudaMalloc(&a->acc2, sizeof(double) * ACC_COUNT));
    a->face_bytes = sizeof(float4) * (size_t)(h->face_x + h->face_y + h->face_z);
    SN_CK(h, cudaMalloc(&a->face2, a->face_bytes));
    a->K = (int)std::ceil(std::sqrt((double)h->nplanes));
    a->nblk = (h->nplanes + a->K - 1) / a->K;
    SN_CK(h, cudaMalloc(&a->ckpt, a->face_bytes * a->nblk));
    int64_t cap = 0;
    for (int b = 0; b < a->nblk; ++b) {
        const int s0 = b * a->K, s1 = std::min(h->nplanes, s0 + a->K);
        cap = std::max(cap, h->plane_off[s1] - h->plane_off[s0]);
    }
    SN_CK(h, cudaMalloc(&a->psi_blk, sizeof(float) * 8 * (size_t)cap * 8 * h->G * h->Do));
    h->device_bytes += (int64_t)(sizeof(float) * (4 * GC8 + 8 * (size_t)cap * 8 * h->G * h->Do) +
                                 a->face_bytes * (a->nblk + 1));
    return SN_OK;
}

// chi = M^{-1} r per cell: M = V/216 (Mh x Mh x Mh), Mh^{-1} = [[2,-1],[-1,2]]/3.
__global__ void chi_kernel(const float *__restrict__ r, float *__restrict__ chi, int n_gc, float scale)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_gc; e += gridDim.x * blockDim.x) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = r[8 * e + k];
#pragma unroll
        for (int bit = 0; bit < 3; ++bit) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (k & (1 << bit)) continue;
                const float a = v[k], b = v[k | (1 << bit)];
                v[k] = (2.f * a - b) * (1.f / 3.f);
                v[k | (1 << bit)] = (2.f * b - a) * (1.f / 3.f);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) chi[8 * e + k] = scale * v[k];
    }
}

// Adjoint nodal source: S_adj[g'] = chi[g'] + (sigs[g']/4pi) sum_g xfer[g'][g] Lam[g].
__global__ void adj_source_kernel(const float *__restrict__ chi, const float *__restrict__ lam,
                                  const float *__restrict__ sigs, const float *__restrict__ xfer,
                                  float *__restrict__ S, int C, int G)
{
    const float inv4pi = (float)(1.0 / (4.0 * kPi));
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < G * C * 8; e += gridDim.x * blockDim.x) {
        const int gp = e / (C * 8), ce = e - gp * C * 8, c = ce >> 3;
        float acc = 0.f;
        for (int g = 0; g < G; ++g) acc = fmaf(xfer[gp * G + g], lam[(int64_t)g * C * 8 + ce], acc);
        S[e] = chi[e] + sigs[(int64_t)gp * C + c] * inv4pi * acc;
    }
}

// dR/dq and dR/dsigma_s from the adjoint and forward scalar fluxes, one thread per (g', c).
__global__ void grad_qs_kernel(const float *__restrict__ lam, const float *__restrict__ phi,
                               const float *__restrict__ xfer, double *__restrict__ gq,
                               double *__restrict__ gs, int C, int G, double vol)
{
    const double inv4pi = 1.0 / (4.0 * kPi);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < G * C; e += gridDim.x * blockDim.x) {
        const int gp = e / C, c = e - gp * C;
        const float *L = lam + (int64_t)e * 8;
        double sl = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) sl += (double)L[k];
        gq[e] = sl * (vol / 8.0) * inv4pi;
        float mp[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) mp[k] = phi[(int64_t)e * 8 + k];
        mh_axis<0>(mp);
        mh_axis<1>(mp);
        mh_axis<2>(mp);
        double s = 0.0;
        for (int g = 0; g < G; ++g) {
            const float f = xfer[gp * G + g];
            if (f == 0.f) continue;
            const float *Lg = lam + ((int64_t)g * C + c) * 8;
            float dot = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) dot = fmaf(Lg[k], mp[k], dot);
            s += (double)f * (double)dot;
        }
        gs[e] = s * (vol / 216.0) * inv4pi;
    }
}

static unsigned grid_for(int64_t n, int per)
{
    int64_t g = (n + per - 1) / per;
    const int64_t cap = (int64_t)num_sms() * 16;
    return (unsigned)(g < cap ? (g > 0 ? g : 1) : cap);
}

// R = sum resp * phi over groups, cells and nodes, FP64 products and accumulation.
template <typename T>
__global__ void __launch_bounds__(256) response_kernel(const T *__restrict__ phi, const T *__restrict__ resp,
                                                       int64_t n, double *out)
{
    __shared__ double sh[8];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma((double)phi[i], (double)resp[i], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x % 32 == 0) sh[threadIdx.x / 32] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)blockDim.x / 32; ++w) s += sh[w];
        atomicAdd(out, s);
    }
}

}  // namespace sn

using namespace sn;

extern "C" {

sn_status sn_response(sn_handle h, const void *phi, const void *resp, double *R)
{
    if (!h || !phi || !resp || !R) return fail(h, SN_EINVAL, "sn_response: NULL argument");
    if (h->K > 1) return fail(h, SN_EINVAL, "sn_response: isotropic scattering only");
    const cudaStream_t st = h->stream;
    const int64_t n = (int64_t)h->G * h->ncell * 8;
    int64_t grid = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    SN_CK(h, cudaMemsetAsync(h->acc + ACC_RESP, 0, sizeof(double), st));
    if (h->fp64)
        response_kernel<double><<<(unsigned)grid, 256, 0, st>>>((const double *)phi, (const double *)resp, n,
                                                                 h->acc + ACC_RESP);
    else
        response_kernel<float><<<(unsigned)grid, 256, 0, st>>>((const float *)phi, (const float *)resp, n,
                                                               h->acc + ACC_RESP);
    SN_CK(h, cudaGetLastError());
    SN_CK(h, cudaMemcpyAsync(h->acc_host + ACC_RESP, h->acc + ACC_RESP, sizeof(double), cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    *R = h->acc_host[ACC_RESP];
    return SN_OK;
}


sn_status sn_adjoint_sweep(sn_handle h, const float *phi, const float *resp, double tol, int32_t max_it, float *Lam,
                           double *dR_dsigt, double *dR_dsigs, double *dR_dq, int32_t *iters)
{
    if (!h || !phi || !resp || !Lam || !dR_dsigt || !dR_dsigs || !dR_dq)
        return fail(h, SN_EINVAL, "sn_adjoint_sweep: NULL argument");
    if (h->K > 1 || h->geom) return fail(h, SN_EINVAL, "sn_adjoint_sweep: isotropic scattering on box cells only");
    if (h->fp64) return fail(h, SN_EINVAL, "sn_adjoint_sweep: needs an FP32 handle");
    if (max_it < 1 || !(tol >= 0.0)) return fail(h, SN_EINVAL, "sn_adjoint_sweep: max_it >= 1, tol >= 0");
    sn_status s = ensure_adjoint(h);
    if (s != SN_OK) return s;
    Adj *a = reinterpret_cast<Adj *>(h->adj);
    const cudaStream_t st = h->stream;
    const int C = (int)h->ncell, G = h->G;
    const double vol = h->dx * h->dy * h->dz;
    const size_t GC8 = (size_t)G * C * 8;

    chi_kernel<<<grid_for((int64_t)G * C, 256), 256, 0, st>>>(resp, a->chi, G * C, (float)(216.0 / vol));
    SN_CK(h, cudaMemsetAsync(Lam, 0, sizeof(float) * GC8, st));

    // adjoint source iteration: vacuum sweeps of the adjoint source
    AdjPass pa;
    pa.mode = 0;
    pa.S = a->Sadj;
    pa.psi_inc = a->zero_inc;
    pa.face = h->face;
    pa.phi_oct = (float *)h->phi_oct;
    pa.leak = h->acc + ACC_LEAK;
    float *buf[2] = {Lam, a->lam_b};
    int cur = 0, it = 0;
    sn_status rc = SN_ENOCONV;
    for (it = 0; it < max_it; ++it) {
        adj_source_kernel<<<grid_for((int64_t)GC8, 256), 256, 0, st>>>(a->chi, buf[cur], (const float *)h->sigs,
                                                                      (const float *)h->xfer, a->Sadj, C, G);
        SN_CK(h, cudaMemsetAsync(h->acc, 0, sizeof(double) * ACC_COUNT, st));
        s = launch_planes_adjoint(h, pa, 0, h->nplanes, st);
        if (s != SN_OK) return s;
        s = launch_reduce(h, buf[cur], buf[1 - cur], a->Sadj, nullptr, true, st);
        if (s != SN_OK) return s;
        SN_CK(h, cudaMemcpyAsync(h->acc_host, h->acc, sizeof(double) * ACC_COUNT, cudaMemcpyDeviceToHost, st));
        SN_CK(h, cudaStreamSynchronize(st));
        cur = 1 - cur;
        const double *ac = h->acc_host;
        if (ac[ACC_FLAG] != 0.0) return fail(h, SN_ENAN, "sn_adjoint_sweep: non-finite adjoint flux");
        const double cm = ac[ACC_PMAX] > 0 ? ac[ACC_DMAX] / ac[ACC_PMAX] : 0.0;
        if (cm <= tol) {
            rc = SN_OK;
            ++it;
            break;
        }
    }
    if (cur == 1) SN_CK(h, cudaMemcpyAsync(Lam, a->lam_b, sizeof(float) * GC8, cudaMemcpyDeviceToDevice, st));
    if (iters) *iters = it;

    // dR/dq, dR/dsigma_s
    grad_qs_kernel<<<grid_for((int64_t)G * C, 128), 128, 0, st>>>(Lam, phi, (const float *)h->xfer, dR_dq, dR_dsigs,
                                                                  C, G, vol);
    SN_CK(h, cudaGetLastError());

    // dR/dsigma_t: checkpointed forward recompute paired with the final adjoint sweep
    s = launch_source(h, phi, a->Sfwd, st);
    if (s != SN_OK) return s;
    adj_source_kernel<<<grid_for((int64_t)GC8, 256), 256, 0, st>>>(a->chi, Lam, (const float *)h->sigs,
                                                                  (const float *)h->xfer, a->Sadj, C, G);
    SN_CK(h, cudaMemsetAsync(dR_dsigt, 0, sizeof(double) * (size_t)G * C, st));
    AdjPass pf;   // forward recompute
    pf.S = a->Sfwd;
    pf.psi_inc = (const float *)h->psi_inc;
    pf.face = a->face2;
    pf.phi_oct = (float *)h->phi_oct;
    pf.leak = a->acc2;
    pf.psi_blk = a->psi_blk;
    for (int b = 0; b < a->nblk; ++b) {
        const int s0 = b * a->K, s1 = std::min(h->nplanes, s0 + a->K);
        SN_CK(h, cudaMemcpyAsync(a->ckpt + a->face_bytes * b, a->face2, a->face_bytes, cudaMemcpyDeviceToDevice, st));
        pf.mode = 0;
        s = launch_planes_adjoint(h, pf, s0, s1, st);
        if (s != SN_OK) return s;
    }
    AdjPass pp = pa;   // adjoint pass with pairing
    pp.mode = 2;
    pp.psi_blk = a->psi_blk;
    pp.grad = dR_dsigt;
    pp.leak = a->acc2;
    for (int b = a->nblk - 1; b >= 0; --b) {
        const int s0 = b * a->K, s1 = std::min(h->nplanes, s0 + a->K);
        SN_CK(h, cudaMemcpyAsync(a->face2, a->ckpt + a->face_bytes * b, a->face_bytes, cudaMemcpyDeviceToDevice, st));
        pf.mode = 1;
        pf.blk_cell0 = h->plane_off[s0];
        s = launch_planes_adjoint(h, pf, s0, s1, st);
        if (s != SN_OK) return s;
        pp.blk_cell0 = h->plane_off[s0];
        s = launch_planes_adjoint(h, pp, h->nplanes - s1, h->nplanes - s0, st);
        if (s != SN_OK) return s;
    }
    SN_CK(h, cudaStreamSynchronize(st));
    if (rc == SN_ENOCONV) fail(h, SN_ENOCONV, "sn_adjoint_sweep: max_it reached before tol");
    return rc;
}

}  // extern "C"

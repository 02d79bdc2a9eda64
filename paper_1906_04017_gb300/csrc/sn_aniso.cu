// sn_aniso.cu -- anisotropic scattering (Sec. 2, Eqs. (3)-(8)): the differential
// scattering cross section expanded in Legendre polynomials up to order L,
// sigma_s(mu0) = sum_n (2n+1)/(4 pi) sigma_{s,n} P_n(mu0); by the addition theorem
// the scattering source of a direction is sum_{n,m} sigma_{s,n} Y_nm(Omega) phi_nm
// with flux moments phi_nm = sum_d w_d Y_nm(Omega_d) psi_d.
//
// The library carries the moments with harmonics scaled by sqrt(4 pi), Yh = sqrt(4 pi) Y
// (so Yh_00 = 1 and moment 0 is the scalar flux of the isotropic path):
//   flux moments   phih_k = sum_d w_d Yh_k(Omega_d) psi_d,
//   source moments Sh_k   = (sum_g' xfer[g'][g] sigma_{s,n(k),g'} phih_k,g' + [k = 0] q) / (4 pi),
//   direction d's source  S_d = sum_k Yh_k(Omega_d) Sh_k,
// moment k = n^2 + n + m for degree n and order m, K = (L + 1)^2.  Real orthonormal
// harmonics: Y_n0 = N_n0 P_n(cos theta), Y_nm = sqrt(2) N_nm P_n^m(cos theta) cos(m phi),
// Y_n,-m = sqrt(2) N_nm P_n^m(cos theta) sin(m phi) (m > 0), N_nm^2 = (2n+1)/(4 pi)
// (n-m)!/(n+m)!, P_n^m without the Condon-Shortley sign; theta is measured from the
// z axis and phi in the x-y plane.
#include <cmath>
#include <vector>

#include "sn_internal.cuh"

namespace sn {

// P_n^m(x) for 0 <= m <= n <= 3 by the recurrences
//   P_m^m = (2m-1)!! (1-x^2)^{m/2},  P_{m+1}^m = (2m+1) x P_m^m,
//   (n-m) P_n^m = (2n-1) x P_{n-1}^m - (n+m-1) P_{n-2}^m
// (no Condon-Shortley sign).
static double assoc_legendre(int n, int m, double x)
{
    const double s = std::sqrt(std::fmax(0.0, 1.0 - x * x));
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * s;
    if (n == m) return pmm;
    double p1 = (2.0 * m + 1.0) * x * pmm;
    if (n == m + 1) return p1;
    double p0 = pmm;
    for (int l = m + 2; l <= n; ++l) {
        const double p2 = ((2.0 * l - 1.0) * x * p1 - (l + m - 1.0) * p0) / (double)(l - m);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// sqrt(4 pi) Y_k(omega) for k < (L+1)^2
static void yhat_of(const double *om, int L, double *out)
{
    const double th = std::acos(std::fmax(-1.0, std::fmin(1.0, om[2])));
    const double ph = std::atan2(om[1], om[0]);
    const double x = std::cos(th);
    for (int n = 0; n <= L; ++n)
        for (int m = -n; m <= n; ++m) {
            const int am = m < 0 ? -m : m;
            const double N = std::sqrt((2.0 * n + 1.0) * factorial(n - am) / factorial(n + am));   // x sqrt(4 pi)
            const double p = assoc_legendre(n, am, x);
            double v;
            if (m == 0) v = N * p;
            else if (m > 0) v = std::sqrt(2.0) * N * p * std::cos(am * ph);
            else v = std::sqrt(2.0) * N * p * std::sin(am * ph);
            out[n * n + n + m] = v;
        }
}

// Moment source (the generalisation of the isotropic source to K moments), flux and
// source moments in the [G][K][C][8] layout.  One thread per (moment, cell, node),
// all groups; up to GMAX groups the scattering products sigma_{s,n,g'} phi_g' are read
// once into registers (GMAX = 0: any group count, read per use).
template <typename T, int GMAX>
__global__ void __launch_bounds__(256) source_moments_kernel(const T *__restrict__ phi, const T *__restrict__ sigs,
                                                             const T *__restrict__ sigs_n, const T *__restrict__ q,
                                                             const T *__restrict__ xfer, T *__restrict__ S,
                                                             int64_t C, int G, int K)
{
    const T inv4pi = (T)(1.0 / (4.0 * kPi));
    const int64_t per = C * 8;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)K * per;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / per);
        const int64_t ce = e - (int64_t)k * per, c = ce >> 3;
        int n = 0;
        while ((n + 1) * (n + 1) <= k) ++n;
        const T *sn = n == 0 ? sigs : sigs_n + (int64_t)(n - 1) * G * C;
        if constexpr (GMAX > 0) {
            T sv[GMAX];
#pragma unroll
            for (int gp = 0; gp < GMAX; ++gp)
                sv[gp] = gp < G ? sn[(int64_t)gp * C + c] * phi[((int64_t)gp * K + k) * per + ce] : T(0);
#pragma unroll
            for (int g = 0; g < GMAX; ++g) {
                if (g >= G) break;
                T acc = k == 0 ? q[(int64_t)g * C + c] : T(0);
#pragma unroll
                for (int gp = 0; gp < GMAX; ++gp)
                    if (gp < G) acc = fma(__ldg(xfer + gp * G + g), sv[gp], acc);
                S[((int64_t)g * K + k) * per + ce] = acc * inv4pi;
            }
        } else {
            for (int g = 0; g < G; ++g) {
                T acc = k == 0 ? q[(int64_t)g * C + c] : T(0);
                for (int gp = 0; gp < G; ++gp)
                    acc = fma(xfer[gp * G + g], sn[(int64_t)gp * C + c] * phi[((int64_t)gp * K + k) * per + ce], acc);
                S[((int64_t)g * K + k) * per + ce] = acc * inv4pi;
            }
        }
    }
}

template <typename T>
static void launch_source_moments_t(sn_handle h, const T *phi, T *S, unsigned grid, cudaStream_t st)
{
    const T *sg = (const T *)h->sigs, *sn = (const T *)h->sigs_n, *q = (const T *)h->q, *xf = (const T *)h->xfer;
    if (h->G <= 8)
        source_moments_kernel<T, 8><<<grid, 256, 0, st>>>(phi, sg, sn, q, xf, S, h->ncell, h->G, h->K);
    else if (h->G <= 16)
        source_moments_kernel<T, 16><<<grid, 256, 0, st>>>(phi, sg, sn, q, xf, S, h->ncell, h->G, h->K);
    else
        source_moments_kernel<T, 0><<<grid, 256, 0, st>>>(phi, sg, sn, q, xf, S, h->ncell, h->G, h->K);
}

sn_status launch_source_moments(sn_handle h, const void *phi, void *S, cudaStream_t st)
{
    const int64_t n = (int64_t)h->K * h->ncell * 8;
    int64_t grid = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (grid > cap) grid = cap;
    if (h->fp64)
        launch_source_moments_t<double>(h, (const double *)phi, (double *)S, (unsigned)grid, st);
    else
        launch_source_moments_t<float>(h, (const float *)phi, (float *)S, (unsigned)grid, st);
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

template <typename T>
static sn_status upload_as(sn_handle h, void **dst, const std::vector<double> &v)
{
    std::vector<T> t(v.begin(), v.end());
    SN_CK(h, cudaMalloc(dst, sizeof(T) * (t.empty() ? 1 : t.size())));
    if (!t.empty())
        SN_CK(h, cudaMemcpyAsync(*dst, t.data(), sizeof(T) * t.size(), cudaMemcpyHostToDevice, h->stream));
    return SN_OK;
}

}  // namespace sn

using namespace sn;

extern "C" {

sn_status sn_set_scattering_order(sn_handle h, int32_t L, const double *sigs_n)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_set_scattering_order: NULL handle");
    if (L < 0 || L > SN_MAX_SCATTERING_ORDER)
        return fail(h, SN_EINVAL, "sn_set_scattering_order: L must be in 0..3");
    if (L > 0 && !sigs_n) return fail(h, SN_EINVAL, "sn_set_scattering_order: NULL sigs_n");
    if (L > 0 && h->geom) return fail(h, SN_EINVAL, "sn_set_scattering_order: not with general hexahedral cells");
    const int64_t GC = (int64_t)h->G * h->ncell;
    std::vector<double> sn((size_t)L * GC);
    for (size_t i = 0; i < sn.size(); ++i) {
        if (!std::isfinite(sigs_n[i])) return fail(h, SN_EINVAL, "sn_set_scattering_order: non-finite sigma_s,n");
        sn[i] = sigs_n[i];
    }
    const int K = (L + 1) * (L + 1);
    // the stage buffers of a sweep tile hold K source moments per key
    if (sweep_smem_bytes(h, K) > 200 * 1024)
        return fail(h, SN_EINVAL, "sn_set_scattering_order: too many moments for this quadrature's tiles");
    SN_CK(h, cudaStreamSynchronize(h->stream));
    // harmonics of every direction, octant-major [8][Do][K]
    std::vector<double> y((size_t)8 * h->Do * K);
    for (int d = 0; d < h->ndir; ++d) yhat_of(&h->omega[3 * d], L, &y[(size_t)d * K]);
    void *new_sn = nullptr, *new_y = nullptr, *new_oct = nullptr, *new_S = nullptr, *new_b = nullptr;
    const size_t esz = h->esz;
    auto cleanup = [&]() {
        void *b[] = {new_sn, new_y, new_oct, new_S, new_b};
        for (void *p : b)
            if (p) cudaFree(p);
    };
    sn_status s = h->fp64 ? upload_as<double>(h, &new_sn, sn) : upload_as<float>(h, &new_sn, sn);
    if (s == SN_OK) s = h->fp64 ? upload_as<double>(h, &new_y, y) : upload_as<float>(h, &new_y, y);
    cudaError_t e = cudaSuccess;
    if (s == SN_OK) e = cudaMalloc(&new_oct, esz * 8 * (size_t)GC * K * 8);
    if (s == SN_OK && e == cudaSuccess) e = cudaMalloc(&new_S, esz * (size_t)GC * K * 8);
    if (s == SN_OK && e == cudaSuccess) e = cudaMalloc(&new_b, esz * (size_t)GC * K * 8);
    if (s == SN_OK && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the uploads have landed
    if (s != SN_OK || e != cudaSuccess) {
        cleanup();
        return s != SN_OK ? s : cuda_fail(h, e, "sn_set_scattering_order: cudaMalloc");
    }
    h->device_bytes += (int64_t)(esz * ((size_t)8 * GC * K * 8 + 2 * (size_t)GC * K * 8) + esz * (sn.size() + y.size()));
    h->device_bytes -= (int64_t)(esz * ((size_t)8 * GC * h->K * 8 + 2 * (size_t)GC * h->K * 8));
    void *old[] = {h->sigs_n, h->yhat, h->phi_oct, h->S, h->phi_b};
    for (void *p : old)
        if (p) cudaFree(p);
    h->sigs_n = new_sn;
    h->yhat = new_y;
    h->phi_oct = new_oct;
    h->S = new_S;
    h->phi_b = new_b;
    h->L = L;
    h->K = K;
    s = reduce_configure(h);
    if (s != SN_OK) return s;
    // captured iteration graphs hold the old buffers
    for (int p = 0; p < 2; ++p)
        if (h->graphs.exec[p]) { cudaGraphExecDestroy(h->graphs.exec[p]); h->graphs.exec[p] = nullptr; }
    h->graphs.phi_user = nullptr;
    h->tallies_valid = false;
    return SN_OK;
}

}  // extern "C"

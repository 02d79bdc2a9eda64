// cell_problem.cuh -- the one-cell problem of the C ABI (27 inputs: Omega, cell sizes,
// sigma_t, 8 nodal sources, 12 upwind face values) mirrored into the canonical
// (positive-octant) frame of ge8.cuh, and the surrogate network's input
// construction on top of it.
#pragma once

#include "ge8.cuh"

namespace sn {

template <typename T>
struct CanonCell {
    T t3x, t3y, t3z, sig;     // 3 |Omega_a| / h_a and sigma_t
    T S[8], ux[4], uy[4], uz[4];
    int mask;                 // physical node = canonical node ^ mask
};

template <typename T>
__device__ __forceinline__ void canonicalize(const T *p, CanonCell<T> &c)
{
    const int fx = p[0] < T(0), fy = p[1] < T(0), fz = p[2] < T(0);
    c.mask = fx | (fy << 1) | (fz << 2);
    c.t3x = T(3) * fabs(p[0]) / p[3];
    c.t3y = T(3) * fabs(p[1]) / p[4];
    c.t3z = T(3) * fabs(p[2]) / p[5];
    c.sig = p[6];
#pragma unroll
    for (int k = 0; k < 8; ++k) c.S[k] = p[7 + k];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        c.ux[t] = p[15 + t];
        c.uy[t] = p[19 + t];
        c.uz[t] = p[23 + t];
    }
    mirror8(c.S, c.mask);
    mirror4(c.ux, fy | (fz << 1));    // x-face in-face index b + 2c
    mirror4(c.uy, fx | (fz << 1));    // y-face a + 2c
    mirror4(c.uz, fx | (fy << 1));    // z-face a + 2b
}

// Elimination of one physical one-cell problem; psi in physical node order.
template <typename T, bool REFINE>
__device__ __forceinline__ void solve_in27(const T *p, T (&psi)[8])
{
    CanonCell<T> c;
    canonicalize(p, c);
    cell_solve_canonical<T, REFINE>(c.t3x, c.t3y, c.t3z, c.sig, c.S, c.ux, c.uy, c.uz, psi);
    mirror8(psi, c.mask);
}

// ---------------------------------------------------------------------------------
// Surrogate input construction (the analogue of the paper's input scaling, Eq. (16)),
// on the canonical problem:
//   x[0:3]  = 2 |Omega_a| - 1
//   x[3:6]  = (log h_a + 1.15) / 1.15
//   x[6]    = log(max(sigma_t, 1e-6)) / 4.5
//   x[7:15] = S / s,  x[15:27] = (up_x, up_y, up_z) / s,  s = max(max|S|, max|up|)
// The network predicts psi_canonical / s; s = 0 means psi = 0.
// ---------------------------------------------------------------------------------
constexpr int kNin = 27, kNhid = 64, kNout = 8;
constexpr int kNparam = kNhid * kNin + kNhid + kNout * kNhid + kNout;   // 2312
constexpr float kLogHShift = 1.15f, kLogHScale = 1.15f, kLogSigScale = 4.5f, kSigFloor = 1e-6f;
// Input scales at or below this are treated as zero (inputs and target scaled by 0):
// fluxes that underflow FP32, e.g. a hundred mean free paths into an absorber, would
// otherwise give an infinite 1/s.
constexpr float kScaleFloor = 1e-30f;

__device__ __forceinline__ float input_scale(const float (&S)[8], const float (&ux)[4], const float (&uy)[4],
                                             const float (&uz)[4])
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s = fmaxf(s, fabsf(S[k]));
#pragma unroll
    for (int t = 0; t < 4; ++t) s = fmaxf(s, fmaxf(fabsf(ux[t]), fmaxf(fabsf(uy[t]), fabsf(uz[t]))));
    return s;
}

// x from |Omega|, h, sigma_t and the canonical sources / face values.
__device__ __forceinline__ void ann_features(float aox, float aoy, float aoz, float hx, float hy, float hz,
                                             float sig, const float (&S)[8], const float (&ux)[4],
                                             const float (&uy)[4], const float (&uz)[4], float inv_s,
                                             float (&x)[kNin])
{
    x[0] = 2.f * aox - 1.f;
    x[1] = 2.f * aoy - 1.f;
    x[2] = 2.f * aoz - 1.f;
    x[3] = (logf(hx) + kLogHShift) / kLogHScale;
    x[4] = (logf(hy) + kLogHShift) / kLogHScale;
    x[5] = (logf(hz) + kLogHShift) / kLogHScale;
    x[6] = logf(fmaxf(sig, kSigFloor)) / kLogSigScale;
#pragma unroll
    for (int k = 0; k < 8; ++k) x[7 + k] = S[k] * inv_s;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        x[15 + t] = ux[t] * inv_s;
        x[19 + t] = uy[t] * inv_s;
        x[23 + t] = uz[t] * inv_s;
    }
}

// Residual test of a candidate canonical solution xhat: ||b - A xhat||_2 <= tau ||b||_2
// in the scaled canonical system (216/V) of ge8.cuh.
__device__ __forceinline__ bool gate_pass(const CanonCell<float> &c, const float (&xhat)[8], float tau)
{
    float b[8], ax[8];
    build_b(2.f * c.t3x, 2.f * c.t3y, 2.f * c.t3z, c.S, c.ux, c.uy, c.uz, b);
    apply_A(c.t3x, c.t3y, c.t3z, c.sig, xhat, ax);
    float rr = 0.f, bb = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float r = b[k] - ax[k];
        rr = fmaf(r, r, rr);
        bb = fmaf(b[k], b[k], bb);
    }
    return rr <= tau * tau * bb;   // NaN in xhat fails the test
}

}  // namespace sn

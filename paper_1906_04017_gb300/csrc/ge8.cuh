// ge8.cuh -- the per-cell DFEM system (14) of Tano & Ragusa (Sec. 2), assembled in
// registers from its 1D factors and solved by Gaussian elimination with partial
// pivoting (the paper's "direct Gauss Elimination"), one thread per system.
//
// Canonical orientation.  Every (cell, direction) problem is mirrored so that the
// flow is along +x, +y, +z: local node k = a + 2b + 4c of the mirrored cell is
// physical node k ^ mask, mask = (Omega_x<0) | (Omega_y<0)<<1 | (Omega_z<0)<<2.
// In that frame, with tau_a = |Omega_a| / h_a and V the cell volume,
//
//   216/V * A = 3 tau_x (Ah x Mh x Mh) + 3 tau_y (Mh x Ah x Mh) + 3 tau_z (Mh x Mh x Ah)
//               + sigma_t (Mh x Mh x Mh)
//   216/V * b = (Mh x Mh x Mh) S + 6 tau_x (e0 x Mh x Mh) up_x + ... (y, z alike)
//
// with Mh = [[2,1],[1,2]] (6 x the 1D mass matrix on a unit interval) and
// Ah = [[1,1],[-1,1]] (2 x the 1D streaming matrix plus the outflow-face mass:
// the outflow form of (14) in one dimension), written per axis in the x-fastest
// node order.  These are exactly the Gauss-integrated matrices of (12) divided by
// V/216, so the solution psi is unchanged.
//
// Pivoting.  The symmetric part of Ah is the identity, so for sigma_t >= 0 the
// symmetric part of A is positive definite (the upwind form's coercivity: half the
// face masses of all six faces plus sigma_t M): partial pivoting then almost never
// exchanges rows.  The elimination therefore runs first on the diagonal pivots,
// branch-free, while it evaluates the test partial pivoting would make at each
// step; a lane whose test fails (some entry below the pivot larger in magnitude)
// redoes its system with the exchanges.  Every lane thus gets exactly the
// operations of partial pivoting, and the common path keeps its instruction-level
// parallelism.
#pragma once

namespace sn {

__host__ __device__ constexpr int mq(int a, int b) { return a == b ? 2 : 1; }
__host__ __device__ constexpr int aq(int a, int b) { return (a == 1 && b == 0) ? -1 : 1; }

// 216/V * A in canonical orientation (t3a = 3 tau_a).
template <typename T>
__device__ __forceinline__ void assemble_A(T t3x, T t3y, T t3z, T sig, T (&A)[8][8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int a = k & 1, b = (k >> 1) & 1, c = k >> 2;
            const int a2 = j & 1, b2 = (j >> 1) & 1, c2 = j >> 2;
            const T cx = T(aq(a, a2) * mq(b, b2) * mq(c, c2));
            const T cy = T(mq(a, a2) * aq(b, b2) * mq(c, c2));
            const T cz = T(mq(a, a2) * mq(b, b2) * aq(c, c2));
            const T cm = T(mq(a, a2) * mq(b, b2) * mq(c, c2));
            A[k][j] = t3x * cx + t3y * cy + t3z * cz + sig * cm;
        }
    }
}

// Apply Mh along the node bit `bit` of an 8-vector (in place).
template <int BIT, typename T>
__device__ __forceinline__ void mh_axis(T (&v)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k & (1 << BIT)) continue;
        const T v0 = v[k], v1 = v[k | (1 << BIT)];
        v[k] = T(2) * v0 + v1;
        v[k | (1 << BIT)] = v0 + T(2) * v1;
    }
}

// 4-vector on a face, in-face index t = p + 2q: apply Mh along p and q.
template <typename T>
__device__ __forceinline__ void mh_face(const T (&u)[4], T (&v)[4])
{
    const T a0 = T(2) * u[0] + u[1], a1 = u[0] + T(2) * u[1];
    const T a2 = T(2) * u[2] + u[3], a3 = u[2] + T(2) * u[3];
    v[0] = T(2) * a0 + a2;
    v[2] = a0 + T(2) * a2;
    v[1] = T(2) * a1 + a3;
    v[3] = a1 + T(2) * a3;
}

// 216/V * b in canonical orientation (t6a = 6 tau_a).  ux: x-inflow face, in-face
// t = b + 2c (node 2t); uy: t = a + 2c (node (t&1) + 4(t>>1)); uz: t = a + 2b (node t).
template <typename T>
__device__ __forceinline__ void build_b(T t6x, T t6y, T t6z, const T (&S)[8], const T (&ux)[4],
                                        const T (&uy)[4], const T (&uz)[4], T (&b)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = S[k];
    mh_axis<0>(b);
    mh_axis<1>(b);
    mh_axis<2>(b);
    T v[4];
    mh_face(ux, v);
#pragma unroll
    for (int t = 0; t < 4; ++t) b[2 * t] += t6x * v[t];
    mh_face(uy, v);
#pragma unroll
    for (int t = 0; t < 4; ++t) b[(t & 1) + 4 * (t >> 1)] += t6y * v[t];
    mh_face(uz, v);
#pragma unroll
    for (int t = 0; t < 4; ++t) b[t] += t6z * v[t];
}

// y = (216/V * A) x using the Kronecker factors (no 8x8 matrix needed).
template <typename T>
__device__ __forceinline__ void apply_A(T t3x, T t3y, T t3z, T sig, const T (&x)[8], T (&y)[8])
{
    T u[8], w[8];
    // x-term and mass term share Mh along y and z
#pragma unroll
    for (int k = 0; k < 8; ++k) u[k] = x[k];
    mh_axis<1>(u);
    mh_axis<2>(u);
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        const T u0 = u[k], u1 = u[k + 1];
        y[k] = t3x * (u0 + u1) + sig * (T(2) * u0 + u1);
        y[k + 1] = t3x * (u1 - u0) + sig * (u0 + T(2) * u1);
    }
    // y-term: Mh along x and z, Ah along y
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = x[k];
    mh_axis<0>(w);
    mh_axis<2>(w);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k & 2) continue;
        const T w0 = w[k], w1 = w[k | 2];
        y[k] += t3y * (w0 + w1);
        y[k | 2] += t3y * (w1 - w0);
    }
    // z-term: Mh along x and y, Ah along z
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = x[k];
    mh_axis<0>(w);
    mh_axis<1>(w);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T w0 = w[k], w1 = w[k | 4];
        y[k] += t3z * (w0 + w1);
        y[k | 4] += t3z * (w1 - w0);
    }
}

// Reciprocal of a pivot: the PTX approximate reciprocal (max error 1 ulp) in FP32
// -- the refinement step absorbs it -- and the IEEE quotient in FP64.
__device__ __forceinline__ float pivot_recip(float v)
{
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double pivot_recip(double v) { return 1.0 / v; }

// Gaussian elimination with partial pivoting on A (8x8, registers), right-hand side
// b.  Pivot = entry of largest magnitude in the column (ties: the lowest row).
// Row exchanges move the trailing columns and b only; each multiplier stays where
// it was computed, so replay_solve() can repeat the same operations on another
// right-hand side.  piv packs the pivot row of step k in bits 3k..3k+2; rinv holds
// the reciprocal pivots.  On return b holds the transformed right-hand side and
// x the solution.
template <typename T>
__device__ __forceinline__ void ge8_factor_solve(T (&A)[8][8], T (&b)[8], unsigned &piv,
                                                 T (&rinv)[8], T (&x)[8])
{
    piv = 0u;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        int p = k;
        T best = fabs(A[k][k]);
#pragma unroll
        for (int r = k + 1; r < 8; ++r) {
            const T v = fabs(A[r][k]);
            if (v > best) { best = v; p = r; }
        }
        piv |= unsigned(p) << (3 * k);
#pragma unroll
        for (int r = k + 1; r < 8; ++r) {
            if (p == r) {
#pragma unroll
                for (int c = k; c < 8; ++c) {
                    const T t = A[k][c]; A[k][c] = A[r][c]; A[r][c] = t;
                }
                const T t = b[k]; b[k] = b[r]; b[r] = t;
            }
        }
        rinv[k] = pivot_recip(A[k][k]);
#pragma unroll
        for (int r = k + 1; r < 8; ++r) {
            const T l = A[r][k] * rinv[k];
            A[r][k] = l;
#pragma unroll
            for (int c = k + 1; c < 8; ++c) A[r][c] = fma(-l, A[k][c], A[r][c]);
            b[r] = fma(-l, b[k], b[r]);
        }
    }
    rinv[7] = pivot_recip(A[7][7]);
#pragma unroll
    for (int r = 7; r >= 0; --r) {
        T s = b[r];
#pragma unroll
        for (int c = r + 1; c < 8; ++c) s = fma(-A[r][c], x[c], s);
        x[r] = s * rinv[r];
    }
}

// Pivot rows of the identity permutation in ge8_factor_solve's encoding.
constexpr unsigned kPivIdentity = (1u << 3) | (2u << 6) | (3u << 9) | (4u << 12) | (5u << 15) | (6u << 18);

// Elimination on the diagonal pivots (multipliers in place, reciprocal pivots in
// rinv, transformed right-hand side in b, solution in x).  Returns true when partial
// pivoting would have exchanged rows at some step: an entry below the pivot of
// strictly larger magnitude (ties keep the diagonal, as in ge8_factor_solve).  When
// it returns false the results are bit-identical to ge8_factor_solve's.
template <typename T>
__device__ __forceinline__ bool ge8_factor_solve_diag(T (&A)[8][8], T (&b)[8], T (&rinv)[8], T (&x)[8])
{
    bool ex = false;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        T m = fabs(A[k + 1][k]);
#pragma unroll
        for (int r = k + 2; r < 8; ++r) m = fmax(m, fabs(A[r][k]));
        ex |= m > fabs(A[k][k]);
        rinv[k] = pivot_recip(A[k][k]);
#pragma unroll
        for (int r = k + 1; r < 8; ++r) {
            const T l = A[r][k] * rinv[k];
            A[r][k] = l;
#pragma unroll
            for (int c = k + 1; c < 8; ++c) A[r][c] = fma(-l, A[k][c], A[r][c]);
            b[r] = fma(-l, b[k], b[r]);
        }
    }
    rinv[7] = pivot_recip(A[7][7]);
#pragma unroll
    for (int r = 7; r >= 0; --r) {
        T s = b[r];
#pragma unroll
        for (int c = r + 1; c < 8; ++c) s = fma(-A[r][c], x[c], s);
        x[r] = s * rinv[r];
    }
    return ex;
}

// Repeat the elimination recorded by ge8_factor_solve on a new right-hand side r
// (overwritten) and back-substitute: dx = A^{-1} r.
template <typename T>
__device__ __forceinline__ void ge8_replay(const T (&A)[8][8], unsigned piv, const T (&rinv)[8],
                                           T (&r)[8], T (&dx)[8])
{
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int p = (piv >> (3 * k)) & 7u;
#pragma unroll
        for (int q = k + 1; q < 8; ++q)
            if (p == q) { const T t = r[k]; r[k] = r[q]; r[q] = t; }
#pragma unroll
        for (int q = k + 1; q < 8; ++q) r[q] = fma(-A[q][k], r[k], r[q]);
    }
#pragma unroll
    for (int q = 7; q >= 0; --q) {
        T s = r[q];
#pragma unroll
        for (int c = q + 1; c < 8; ++c) s = fma(-A[q][c], dx[c], s);
        dx[q] = s * rinv[q];
    }
}

// ge8_replay for the elimination of ge8_factor_solve_diag (no exchanges).
template <typename T>
__device__ __forceinline__ void ge8_replay_diag(const T (&A)[8][8], const T (&rinv)[8], T (&r)[8], T (&dx)[8])
{
#pragma unroll
    for (int k = 0; k < 7; ++k) {
#pragma unroll
        for (int q = k + 1; q < 8; ++q) r[q] = fma(-A[q][k], r[k], r[q]);
    }
#pragma unroll
    for (int q = 7; q >= 0; --q) {
        T s = r[q];
#pragma unroll
        for (int c = q + 1; c < 8; ++c) s = fma(-A[q][c], dx[c], s);
        dx[q] = s * rinv[q];
    }
}

// Element `lane` (0: .x, 1: .y) of a pair of FP32 values.
__device__ __forceinline__ float &pel(float2 &p, int lane) { return lane ? p.y : p.x; }
__device__ __forceinline__ float pel(const float2 &p, int lane) { return lane ? p.y : p.x; }

// FP32 form of the canonical solve with the matrix held as column pairs: the
// trailing-row updates of the elimination are two-lane fused multiply-adds
// (fma.rn.f32x2), each lane rounded exactly as fmaf, so the results are those of
// the scalar form bit for bit.  Same pivoting test, exchange path and refinement.
template <bool REFINE>
__device__ __forceinline__ void cell_solve_canonical_x2(float t3x, float t3y, float t3z, float sig,
                                                        const float (&S)[8], const float (&ux)[4],
                                                        const float (&uy)[4], const float (&uz)[4], float (&x)[8])
{
    float2 A[8][4];
    {
        float As[8][8];
        assemble_A(t3x, t3y, t3z, sig, As);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int q = 0; q < 4; ++q) A[k][q] = make_float2(As[k][2 * q], As[k][2 * q + 1]);
        }
    }
    float b[8], rinv[8], b0[8];
    build_b(2.f * t3x, 2.f * t3y, 2.f * t3z, S, ux, uy, uz, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) b0[k] = b[k];
    bool ex = false;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int kq = k >> 1, kl = k & 1;
        float m = fabsf(pel(A[k + 1][kq], kl));
#pragma unroll
        for (int r = k + 2; r < 8; ++r) m = fmaxf(m, fabsf(pel(A[r][kq], kl)));
        ex |= m > fabsf(pel(A[k][kq], kl));
        rinv[k] = pivot_recip(pel(A[k][kq], kl));
#pragma unroll
        for (int r = k + 1; r < 8; ++r) {
            const float l = pel(A[r][kq], kl) * rinv[k];
            const float2 nl = make_float2(-l, -l);
#pragma unroll
            for (int q = kq; q < 4; ++q) {
                if (2 * q + 1 <= k) continue;          // both columns at or left of k
                A[r][q] = __ffma2_rn(nl, A[k][q], A[r][q]);
            }
            pel(A[r][kq], kl) = l;                     // multiplier in place
            b[r] = fmaf(-l, b[k], b[r]);
        }
    }
    rinv[7] = pivot_recip(A[7][3].y);
#pragma unroll
    for (int r = 7; r >= 0; --r) {
        float sum = b[r];
#pragma unroll
        for (int c = r + 1; c < 8; ++c) sum = fmaf(-pel(A[r][c >> 1], c & 1), x[c], sum);
        x[r] = sum * rinv[r];
    }
    // warp-uniform test: the exchange path stays off the instruction stream unless
    // a lane of the warp needs it
    bool done = false;
    if (__any_sync(__activemask(), ex) && ex) {
        float As[8][8], bb[8], rp[8];
        assemble_A(t3x, t3y, t3z, sig, As);
#pragma unroll
        for (int k = 0; k < 8; ++k) bb[k] = b0[k];
        unsigned piv;
        ge8_factor_solve(As, bb, piv, rp, x);
        if (REFINE) {
            float ax[8], r[8], dx[8];
            apply_A(t3x, t3y, t3z, sig, x, ax);
#pragma unroll
            for (int k = 0; k < 8; ++k) r[k] = b0[k] - ax[k];
            ge8_replay(As, piv, rp, r, dx);
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] += dx[k];
        }
        done = true;
    }
    if (REFINE && !done) {
        float ax[8], r[8], dx[8];
        apply_A(t3x, t3y, t3z, sig, x, ax);
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = b0[k] - ax[k];
#pragma unroll
        for (int k = 0; k < 7; ++k) {
#pragma unroll
            for (int q = k + 1; q < 8; ++q) r[q] = fmaf(-pel(A[q][k >> 1], k & 1), r[k], r[q]);
        }
#pragma unroll
        for (int q = 7; q >= 0; --q) {
            float sum = r[q];
#pragma unroll
            for (int c = q + 1; c < 8; ++c) sum = fmaf(-pel(A[q][c >> 1], c & 1), dx[c], sum);
            dx[q] = sum * rinv[q];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] += dx[k];
    }
}

#ifndef SN_GE_F32X2
#define SN_GE_F32X2 1
#endif

// Solve the canonical system; REFINE adds one iterative-refinement step in T.
template <typename T, bool REFINE>
__device__ __forceinline__ void cell_solve_canonical(T t3x, T t3y, T t3z, T sig, const T (&S)[8],
                                                     const T (&ux)[4], const T (&uy)[4],
                                                     const T (&uz)[4], T (&x)[8])
{
    // the paired form measured faster without the refinement step and no faster with
    // it (register pressure), so the refined solve keeps the scalar form
    if constexpr (SN_GE_F32X2 && sizeof(T) == 4 && !REFINE) {
        cell_solve_canonical_x2<REFINE>(t3x, t3y, t3z, sig, S, ux, uy, uz, x);
        return;
    }
    T A[8][8], b[8], rinv[8], b0[8];
    assemble_A(t3x, t3y, t3z, sig, A);
    build_b(T(2) * t3x, T(2) * t3y, T(2) * t3z, S, ux, uy, uz, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) b0[k] = b[k];
    const bool ex = ge8_factor_solve_diag(A, b, rinv, x);
    // warp-uniform test: the exchange path stays off the instruction stream unless
    // a lane of the warp needs it
    const bool any_ex = __any_sync(__activemask(), ex);
    unsigned piv = kPivIdentity;
    if (any_ex && ex) {
        assemble_A(t3x, t3y, t3z, sig, A);
#pragma unroll
        for (int k = 0; k < 8; ++k) b[k] = b0[k];
        ge8_factor_solve(A, b, piv, rinv, x);
    }
    if (REFINE) {
        T ax[8], dx[8];
        apply_A(t3x, t3y, t3z, sig, x, ax);
#pragma unroll
        for (int k = 0; k < 8; ++k) b0[k] -= ax[k];
        if (any_ex)
            ge8_replay(A, piv, rinv, b0, dx);
        else
            ge8_replay_diag(A, rinv, b0, dx);
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] += dx[k];
    }
}

// ---------------------------------------------------------------------------------
// The canonical solve of the key sweep (one thread per key, every direction of the
// octant in turn): the source part (Mh x Mh x Mh) S of the right-hand side is formed
// once per key, A is built from its 27 distinct values, and the refinement residual
// is formed from the Kronecker factors with the subtraction folded into the products.
// The elimination, its partial-pivoting test and the exchange path are those above.
// ---------------------------------------------------------------------------------

// Per-axis state of an entry (k, j) of A: both node bits equal (0), k's bit 0 and j's
// bit 1 (1), k's bit 1 and j's bit 0 (2).
__host__ __device__ constexpr int ax_state(int a, int b) { return a == b ? 0 : (a == 0 ? 1 : 2); }

// 216/V * A in canonical orientation: entry (k, j) = 2^(axes in state 0) *
// (sigma_t + sum_a t3a * c_a), c = 1/2, 1, -1 for the states 0, 1, 2 -- the same
// matrix as assemble_A, written through its 27 distinct values.
__device__ __forceinline__ void assemble_A27(float t3x, float t3y, float t3z, float sig, float (&A)[8][8])
{
    const float vx[3] = {0.5f * t3x, t3x, -t3x};
    const float vy[3] = {0.5f * t3y, t3y, -t3y};
    const float vz[3] = {0.5f * t3z, t3z, -t3z};
    float v[3][3][3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const float sx = sig + vx[p];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float sxy = sx + vy[q];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                v[p][q][r] = (sxy + vz[r]) * (float)((p == 0 ? 2 : 1) * (q == 0 ? 2 : 1) * (r == 0 ? 2 : 1));
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            A[k][j] = v[ax_state(k & 1, j & 1)][ax_state((k >> 1) & 1, (j >> 1) & 1)][ax_state(k >> 2, j >> 2)];
    }
}

// 216/V * b from the key's Sm = (Mh x Mh x Mh) S and the inflow faces (t6a = 6 tau_a);
// face in-face order as in build_b.
__device__ __forceinline__ void build_b_msrc(float t6x, float t6y, float t6z, const float (&Sm)[8],
                                             const float (&ux)[4], const float (&uy)[4], const float (&uz)[4],
                                             float (&b)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = Sm[k];
    float v[4];
    mh_face(ux, v);
#pragma unroll
    for (int t = 0; t < 4; ++t) b[2 * t] = fmaf(t6x, v[t], b[2 * t]);
    mh_face(uy, v);
#pragma unroll
    for (int t = 0; t < 4; ++t) b[(t & 1) + 4 * (t >> 1)] = fmaf(t6y, v[t], b[(t & 1) + 4 * (t >> 1)]);
    mh_face(uz, v);
#pragma unroll
    for (int t = 0; t < 4; ++t) b[t] = fmaf(t6z, v[t], b[t]);
}

// r = b0 - (216/V * A) x from the Kronecker factors (apply_A's terms): the x-streaming
// and mass terms share Mh along y and z and combine as alpha = t3x + 2 sigma,
// beta = t3x + sigma, gamma = sigma - t3x per x-pair.
__device__ __forceinline__ void residual_A(float t3x, float t3y, float t3z, float sig, const float (&x)[8],
                                           const float (&b0)[8], float (&r)[8])
{
    float u[8], v[8], w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) u[k] = x[k];
    mh_axis<2>(u);                      // Mh_z x
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = u[k];
    mh_axis<1>(v);                      // Mh_y Mh_z x
    const float al = fmaf(2.f, sig, t3x), be = t3x + sig, ga = sig - t3x;
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        const float v0 = v[k], v1 = v[k + 1];
        r[k] = fmaf(-be, v1, fmaf(-al, v0, b0[k]));
        r[k + 1] = fmaf(-al, v1, fmaf(-ga, v0, b0[k + 1]));
    }
    mh_axis<0>(u);                      // Mh_x Mh_z x
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k & 2) continue;
        const float w0 = u[k], w1 = u[k | 2];
        r[k] = fmaf(-t3y, w0 + w1, r[k]);
        r[k | 2] = fmaf(-t3y, w1 - w0, r[k | 2]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = x[k];
    mh_axis<0>(w);
    mh_axis<1>(w);                      // Mh_x Mh_y x
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float w0 = w[k], w1 = w[k | 4];
        r[k] = fmaf(-t3z, w0 + w1, r[k]);
        r[k | 4] = fmaf(-t3z, w1 - w0, r[k | 4]);
    }
}

#ifndef SN_KEY_F32X2
#define SN_KEY_F32X2 1
#endif

// The key sweep's solve with the matrix held as column pairs: the trailing-row
// updates of the diagonal elimination are two-lane fused multiply-adds
// (fma.rn.f32x2, each lane rounded as fmaf), so the results are those of the scalar
// form bit for bit with about half the update instructions.  Same pivoting test,
// exchange path and refinement step as cell_solve_key below.
template <bool REFINE>
__device__ __forceinline__ void cell_solve_key_x2(float t3x, float t3y, float t3z, float sig, const float (&Sm)[8],
                                                  const float (&ux)[4], const float (&uy)[4], const float (&uz)[4],
                                                  float (&x)[8])
{
    float2 A[8][4];
    {
        float As[8][8];
        assemble_A27(t3x, t3y, t3z, sig, As);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int q = 0; q < 4; ++q) A[k][q] = make_float2(As[k][2 * q], As[k][2 * q + 1]);
        }
    }
    float b[8], b0[8], rinv[8];
    build_b_msrc(2.f * t3x, 2.f * t3y, 2.f * t3z, Sm, ux, uy, uz, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) b0[k] = b[k];
    bool ex = false;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int kq = k >> 1, kl = k & 1;
        float m = fabsf(pel(A[k + 1][kq], kl));
#pragma unroll
        for (int r = k + 2; r < 8; ++r) m = fmaxf(m, fabsf(pel(A[r][kq], kl)));
        ex |= m > fabsf(pel(A[k][kq], kl));
        rinv[k] = pivot_recip(pel(A[k][kq], kl));
#pragma unroll
        for (int r = k + 1; r < 8; ++r) {
            const float l = pel(A[r][kq], kl) * rinv[k];
            const float2 nl = make_float2(-l, -l);
#pragma unroll
            for (int q = kq; q < 4; ++q) {
                if (2 * q + 1 <= k) continue;          // both columns at or left of k
                A[r][q] = __ffma2_rn(nl, A[k][q], A[r][q]);
            }
            pel(A[r][kq], kl) = l;                     // multiplier in place
            b[r] = fmaf(-l, b[k], b[r]);
        }
    }
    rinv[7] = pivot_recip(A[7][3].y);
#pragma unroll
    for (int r = 7; r >= 0; --r) {
        float sum = b[r];
#pragma unroll
        for (int c = r + 1; c < 8; ++c) sum = fmaf(-pel(A[r][c >> 1], c & 1), x[c], sum);
        x[r] = sum * rinv[r];
    }
    // warp-uniform test: the exchange path stays off the instruction stream unless a
    // lane of the warp needs it
    if (__any_sync(__activemask(), ex) && ex) {
        float As[8][8], bb[8], rp[8];
        assemble_A27(t3x, t3y, t3z, sig, As);
#pragma unroll
        for (int k = 0; k < 8; ++k) bb[k] = b0[k];
        unsigned piv;
        ge8_factor_solve(As, bb, piv, rp, x);
        if (REFINE) {
            float r[8], dx[8];
            residual_A(t3x, t3y, t3z, sig, x, b0, r);
            ge8_replay(As, piv, rp, r, dx);
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] += dx[k];
        }
        return;
    }
    if (REFINE) {
        float r[8], dx[8];
        residual_A(t3x, t3y, t3z, sig, x, b0, r);
#pragma unroll
        for (int k = 0; k < 7; ++k) {
#pragma unroll
            for (int q = k + 1; q < 8; ++q) r[q] = fmaf(-pel(A[q][k >> 1], k & 1), r[k], r[q]);
        }
#pragma unroll
        for (int q = 7; q >= 0; --q) {
            float sum = r[q];
#pragma unroll
            for (int c = q + 1; c < 8; ++c) sum = fmaf(-pel(A[q][c >> 1], c & 1), dx[c], sum);
            dx[q] = sum * rinv[q];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] += dx[k];
    }
}

// The paired solve with its inputs in shared memory (the key's (Mh x Mh x Mh) S as two
// 4-vectors and the three inflow faces): the right-hand side is formed from them where
// it is needed (the elimination, the exchange path, the refinement residual) instead
// of being kept in registers across the elimination.  The operations, and so the
// results, are those of cell_solve_key_x2.
template <bool REFINE>
__device__ __forceinline__ void cell_solve_key_x2_sm(float t3x, float t3y, float t3z, float sig,
                                                     const float4 *m0p, const float4 *m1p, const float4 *fxp,
                                                     const float4 *fyp, const float4 *fzp, float (&x)[8])
{
    auto rhs = [&](float (&bb)[8]) {
        const float4 m0 = *m0p, m1 = *m1p, fx = *fxp, fy = *fyp, fz = *fzp;
        const float Sm[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
        const float ux[4] = {fx.x, fx.y, fx.z, fx.w}, uy[4] = {fy.x, fy.y, fy.z, fy.w},
                    uz[4] = {fz.x, fz.y, fz.z, fz.w};
        build_b_msrc(2.f * t3x, 2.f * t3y, 2.f * t3z, Sm, ux, uy, uz, bb);
    };
    float2 A[8][4];
    {
        float As[8][8];
        assemble_A27(t3x, t3y, t3z, sig, As);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int q = 0; q < 4; ++q) A[k][q] = make_float2(As[k][2 * q], As[k][2 * q + 1]);
        }
    }
    float b[8], rinv[8];
    rhs(b);
    bool ex = false;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const int kq = k >> 1, kl = k & 1;
        float m = fabsf(pel(A[k + 1][kq], kl));
#pragma unroll
        for (int r = k + 2; r < 8; ++r) m = fmaxf(m, fabsf(pel(A[r][kq], kl)));
        ex |= m > fabsf(pel(A[k][kq], kl));
        rinv[k] = pivot_recip(pel(A[k][kq], kl));
#pragma unroll
        for (int r = k + 1; r < 8; ++r) {
            const float l = pel(A[r][kq], kl) * rinv[k];
            const float2 nl = make_float2(-l, -l);
#pragma unroll
            for (int q = kq; q < 4; ++q) {
                if (2 * q + 1 <= k) continue;
                A[r][q] = __ffma2_rn(nl, A[k][q], A[r][q]);
            }
            pel(A[r][kq], kl) = l;
            b[r] = fmaf(-l, b[k], b[r]);
        }
    }
    rinv[7] = pivot_recip(A[7][3].y);
#pragma unroll
    for (int r = 7; r >= 0; --r) {
        float sum = b[r];
#pragma unroll
        for (int c = r + 1; c < 8; ++c) sum = fmaf(-pel(A[r][c >> 1], c & 1), x[c], sum);
        x[r] = sum * rinv[r];
    }
    if (__any_sync(__activemask(), ex) && ex) {
        float As[8][8], bb[8], rp[8];
        assemble_A27(t3x, t3y, t3z, sig, As);
        rhs(bb);
        unsigned piv;
        ge8_factor_solve(As, bb, piv, rp, x);
        if (REFINE) {
            float b0[8], r[8], dx[8];
            rhs(b0);
            residual_A(t3x, t3y, t3z, sig, x, b0, r);
            ge8_replay(As, piv, rp, r, dx);
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] += dx[k];
        }
        return;
    }
    if (REFINE) {
        float b0[8], r[8], dx[8];
        rhs(b0);
        residual_A(t3x, t3y, t3z, sig, x, b0, r);
#pragma unroll
        for (int k = 0; k < 7; ++k) {
#pragma unroll
            for (int q = k + 1; q < 8; ++q) r[q] = fmaf(-pel(A[q][k >> 1], k & 1), r[k], r[q]);
        }
#pragma unroll
        for (int q = 7; q >= 0; --q) {
            float sum = r[q];
#pragma unroll
            for (int c = q + 1; c < 8; ++c) sum = fmaf(-pel(A[q][c >> 1], c & 1), dx[c], sum);
            dx[q] = sum * rinv[q];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] += dx[k];
    }
}

// The key sweep's solve: GE with partial pivoting (diagonal pivots first, exchange
// path where the pivoting test fails) and, with REFINE, one FP32 refinement step.
template <bool REFINE>
__device__ __forceinline__ void cell_solve_key(float t3x, float t3y, float t3z, float sig, const float (&Sm)[8],
                                               const float (&ux)[4], const float (&uy)[4], const float (&uz)[4],
                                               float (&x)[8])
{
    if constexpr (SN_KEY_F32X2) {
        cell_solve_key_x2<REFINE>(t3x, t3y, t3z, sig, Sm, ux, uy, uz, x);
        return;
    }
    float A[8][8], b[8], b0[8], rinv[8];
    assemble_A27(t3x, t3y, t3z, sig, A);
    build_b_msrc(2.f * t3x, 2.f * t3y, 2.f * t3z, Sm, ux, uy, uz, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) b0[k] = b[k];
    const bool ex = ge8_factor_solve_diag(A, b, rinv, x);
    // warp-uniform test: the exchange path stays off the instruction stream unless a
    // lane of the warp needs it
    const bool any_ex = __any_sync(__activemask(), ex);
    unsigned piv = kPivIdentity;
    if (any_ex && ex) {
        assemble_A27(t3x, t3y, t3z, sig, A);
#pragma unroll
        for (int k = 0; k < 8; ++k) b[k] = b0[k];
        ge8_factor_solve(A, b, piv, rinv, x);
    }
    if (REFINE) {
        float r[8], dx[8];
        residual_A(t3x, t3y, t3z, sig, x, b0, r);
        if (any_ex)
            ge8_replay(A, piv, rinv, r, dx);
        else
            ge8_replay_diag(A, rinv, r, dx);
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] += dx[k];
    }
}

// Swap the halves of an 8-vector along node bit BIT when flag is set (x[k] <-> x[k ^ 2^BIT]).
template <int BIT, typename T>
__device__ __forceinline__ void cswap_axis(T (&x)[8], bool flag)
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k & (1 << BIT)) continue;
        const T a = x[k], b = x[k | (1 << BIT)];
        x[k] = flag ? b : a;
        x[k | (1 << BIT)] = flag ? a : b;
    }
}

// x[k] <- x[k ^ mask] for a 3-bit mask (the map is its own inverse): physical <-> canonical.
template <typename T>
__device__ __forceinline__ void mirror8(T (&x)[8], int mask)
{
    cswap_axis<0>(x, mask & 1);
    cswap_axis<1>(x, mask & 2);
    cswap_axis<2>(x, mask & 4);
}

// u[t] <- u[t ^ mask] for a 2-bit mask on a face 4-vector.
template <typename T>
__device__ __forceinline__ void mirror4(T (&u)[4], int mask)
{
    if (mask & 1) { T t = u[0]; u[0] = u[1]; u[1] = t; t = u[2]; u[2] = u[3]; u[3] = t; }
    if (mask & 2) { T t = u[0]; u[0] = u[2]; u[2] = t; t = u[1]; u[1] = u[3]; u[3] = t; }
}

}  // namespace sn

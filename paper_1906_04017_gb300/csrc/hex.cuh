// hex.cuh -- the per-cell system (14) on general hexahedral cells (trilinear maps of
// the unit cube; the shape change of the cells of Sec. 2's closing remarks), from
// element matrices precomputed per cell:
//   M[k][j]        = int N_k N_j dV
//   L_a[k][j]      = -int N_j d_a N_k dV
//   F[f][c][t][t'] = int_f n_c N_node(f,t) N_node(f,t') dS   (outward area vector)
// for faces f = 2a + side (side 1: xi_a = 1) and in-face indices t of the sweep
// (x-face: b + 2c, y-face: a + 2c, z-face: a + 2b).  The system, in the physical
// frame of the cell:
//   A = sum_a Omega_a L_a + sigma_t M + sum over outflow faces of Omega . F
//     = sum_c Omega_c B_c + sigma_t M  (B: per cell and octant, outflow faces folded in)
//   b = M S + sum over inflow faces of (-Omega . F) up
// where the inflow face of axis a is side 0 when Omega_a > 0 (structured wavefront).
#pragma once

namespace sn {

constexpr int kHexM = 0, kHexL = 64, kHexF = 256, kHexRec = 544;   // offsets in a cell record

// node of in-face index t on face (A, SIDE)
template <int A, int SIDE>
__host__ __device__ constexpr int hex_face_node(int t)
{
    return A == 0 ? SIDE + 2 * (t & 1) + 4 * (t >> 1)
                  : (A == 1 ? (t & 1) + 2 * SIDE + 4 * (t >> 1) : (t & 1) + 2 * (t >> 1) + 4 * SIDE);
}

// Omega . F of face (A, SIDE) as a 4x4 block
template <typename T, int A, int SIDE>
__device__ __forceinline__ void hex_face_block(const T *__restrict__ g, const T (&om)[3], T (&B)[4][4])
{
    const T *F = g + kHexF + (2 * A + SIDE) * 48;
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int u = 0; u < 4; ++u)
            B[t][u] = om[0] * __ldg(F + 4 * t + u) + om[1] * __ldg(F + 16 + 4 * t + u) + om[2] * __ldg(F + 32 + 4 * t + u);
}

template <typename T, int A, int SIDE>
__device__ __forceinline__ void hex_add_inflow(const T *__restrict__ g, const T (&om)[3], const T (&up)[4],
                                               T (&b)[8])
{
    T B[4][4];
    hex_face_block<T, A, SIDE>(g, om, B);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        T s = T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) s = fma(B[t][u], up[u], s);
        b[hex_face_node<A, SIDE>(t)] -= s;
    }
}

// integral of (Omega . n) psi over face (A, SIDE)
template <typename T, int A, int SIDE>
__device__ __forceinline__ T hex_face_flux(const T *__restrict__ g, const T (&om)[3], const T (&x)[8])
{
    T B[4][4];
    hex_face_block<T, A, SIDE>(g, om, B);
    T s = T(0);
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int u = 0; u < 4; ++u) s = fma(B[t][u], x[hex_face_node<A, SIDE>(u)], s);
    return s;
}

// dispatch to the compile-time face (register arrays indexed by constants only)
template <typename T, int A>
__device__ __forceinline__ void hex_inflow(const T *g, const T (&om)[3], int in_side, const T (&up)[4], T (&b)[8])
{
    if (in_side) hex_add_inflow<T, A, 1>(g, om, up, b);
    else hex_add_inflow<T, A, 0>(g, om, up, b);
}
template <typename T, int A>
__device__ __forceinline__ T hex_out_flux(const T *g, const T (&om)[3], int out_side, const T (&x)[8])
{
    return out_side ? hex_face_flux<T, A, 1>(g, om, x) : hex_face_flux<T, A, 0>(g, om, x);
}

// Per (cell, octant) the streaming matrices with the octant's outflow faces folded in,
// B_c = L_c + sum over the outflow faces of F_f^c, so that A = sum_c Omega_c B_c + sigma_t M
// (the outflow side of every axis is fixed within an octant).
constexpr int kHexB = 192;   // values a (cell, octant): B_0, B_1, B_2 [8][8]

// A (physical frame) of one cell and direction from its octant's B and the cell's mass
// matrix M (both [8][8] row-major, in shared memory)
template <typename T>
__device__ __forceinline__ void hex_assemble_A(const T *M, const T *B, const T (&om)[3], T sig, T (&A)[8][8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = 8 * k + j;
            A[k][j] = om[0] * B[e] + om[1] * B[64 + e] + om[2] * B[128 + e] + sig * M[e];
        }
}

// b (physical frame): M S plus the inflow faces' terms (face blocks from the cell record g)
template <typename T>
__device__ __forceinline__ void hex_build_b(const T *__restrict__ g, const T *M, const T (&om)[3], const int (&out)[3],
                                            const T (&S)[8], const T (&ux)[4], const T (&uy)[4], const T (&uz)[4],
                                            T (&b)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) s = fma(M[8 * k + j], S[j], s);
        b[k] = s;
    }
    hex_inflow<T, 0>(g, om, 1 - out[0], ux, b);
    hex_inflow<T, 1>(g, om, 1 - out[1], uy, b);
    hex_inflow<T, 2>(g, om, 1 - out[2], uz, b);
}

// y = A x without forming A (M, B as for hex_assemble_A)
template <typename T>
__device__ __forceinline__ void hex_apply_A(const T *M, const T *B, const T (&om)[3], T sig, const T (&x)[8],
                                            T (&y)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = 8 * k + j;
            const T a = om[0] * B[e] + om[1] * B[64 + e] + om[2] * B[128 + e] + sig * M[e];
            s = fma(a, x[j], s);
        }
        y[k] = s;
    }
}

}  // namespace sn

// octnet.cuh -- the paper's per-octant networks (Sec. 3, Eqs. (15)-(18); Sec. 4: one
// network per octant of directions) evaluated on a one-cell problem in the canonical
// (positive-octant) frame of the sweep.
//
// A network of octant o takes the 26 quantities of Sec. 3 in the problem's physical
// frame: the upwind values of the x, y and z inflow faces (4 each), the cosines mu
// and eta, the 8 nodal sources, sigma_t and the cell sizes, each scaled by Eq. (16)
// x = (I - alpha m) / r (m the mean of the input's a-priori range, r its width,
// alpha = 0.27); h = tanh(W1 x + b1); psi_d = theta(z_d), z = W2 h + b2, with
// theta(z) = z above 0 and beta (e^z - 1) below, beta = 0.1 max |upwind value|.
//
// The sweep holds every cell problem mirrored into the positive octant (canonical
// node n = physical node ^ o, face value t = physical t ^ the face's mask).  Mirroring
// only permutes the face values, sources and outputs and flips the signs of mu and
// eta, and Eq. (16) is affine, so each octant's network becomes a network of the
// canonical inputs with permuted, rescaled weights and a shifted bias ("folded").
// The folded network computes the same function as the physical one.
#pragma once

namespace sn {

constexpr int kOnIn = 26, kOnHid = 8, kOnOut = 8;
constexpr int kOnParam = kOnHid * kOnIn + kOnHid + kOnOut * kOnHid + kOnOut;   // 288 a network
constexpr int kOnW1 = 0, kOnB1 = kOnHid * kOnIn, kOnW2 = kOnB1 + kOnHid, kOnB2 = kOnW2 + kOnOut * kOnHid;
constexpr float kOnAlpha = 0.27f, kOnBetaFrac = 0.1f;

// Folded weights of one octant (288 floats).  Hidden unit k owns 24 floats at 24 k:
// the coefficients of the canonical ux[0..3], uy[0..3], uz[0..3], S[0..7], |mu|, |eta|,
// sigma_t, then the bias.  Then the coefficients of the cell sizes (3 per unit), W2 in
// canonical output order [8][8] and b2 [8].
constexpr int kOnFold = 288;
constexpr int kOnFoldH = 192, kOnFoldW2 = 216, kOnFoldB2 = 280;

// tanh(a) = 1 - 2 / (1 + e^{2a}).  For large a the exponential overflows to +inf and
// the quotient to 0 (tanh = 1); for very negative a it is 1 - 2 = -1.  Absolute error
// about 1e-6 (the error of the fast exponential, damped by 2 e / (1 + e)^2 <= 1/2).
__device__ __forceinline__ float octnet_tanh(float a)
{
    return 1.f - __fdividef(2.f, 1.f + __expf(2.f * a));
}

// psi (canonical node order) of the folded network at w (shared or global memory,
// 16-byte aligned).  WITH_H: add the cell-size terms here; otherwise the bias slots
// of w already hold them (the sweep folds the mesh's uniform cell size in once).
template <bool WITH_H>
__device__ __forceinline__ void octnet_forward(const float *__restrict__ w, const float (&ux)[4],
                                               const float (&uy)[4], const float (&uz)[4], const float (&S)[8],
                                               float amu, float aeta, float sig, float hx, float hy, float hz,
                                               float (&psi)[8])
{
    float bm = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) bm = fmaxf(bm, fmaxf(fabsf(ux[t]), fmaxf(fabsf(uy[t]), fabsf(uz[t]))));
    const float beta = kOnBetaFrac * bm;
    float h[kOnHid];
#pragma unroll
    for (int k = 0; k < kOnHid; ++k) {
        const float4 *r = reinterpret_cast<const float4 *>(w + 24 * k);
        const float4 c0 = r[0], c1 = r[1], c2 = r[2], c3 = r[3], c4 = r[4], c5 = r[5];
        float a = c5.w;
        if (WITH_H) {
            a = fmaf(w[kOnFoldH + 3 * k], hx, a);
            a = fmaf(w[kOnFoldH + 3 * k + 1], hy, a);
            a = fmaf(w[kOnFoldH + 3 * k + 2], hz, a);
        }
        a = fmaf(c0.x, ux[0], a); a = fmaf(c0.y, ux[1], a); a = fmaf(c0.z, ux[2], a); a = fmaf(c0.w, ux[3], a);
        a = fmaf(c1.x, uy[0], a); a = fmaf(c1.y, uy[1], a); a = fmaf(c1.z, uy[2], a); a = fmaf(c1.w, uy[3], a);
        a = fmaf(c2.x, uz[0], a); a = fmaf(c2.y, uz[1], a); a = fmaf(c2.z, uz[2], a); a = fmaf(c2.w, uz[3], a);
        a = fmaf(c3.x, S[0], a); a = fmaf(c3.y, S[1], a); a = fmaf(c3.z, S[2], a); a = fmaf(c3.w, S[3], a);
        a = fmaf(c4.x, S[4], a); a = fmaf(c4.y, S[5], a); a = fmaf(c4.z, S[6], a); a = fmaf(c4.w, S[7], a);
        a = fmaf(c5.x, amu, a); a = fmaf(c5.y, aeta, a); a = fmaf(c5.z, sig, a);
        h[k] = octnet_tanh(a);
    }
#pragma unroll
    for (int t = 0; t < kOnOut; ++t) {
        const float4 *r = reinterpret_cast<const float4 *>(w + kOnFoldW2 + 8 * t);
        const float4 c0 = r[0], c1 = r[1];
        float z = w[kOnFoldB2 + t];
        z = fmaf(c0.x, h[0], z); z = fmaf(c0.y, h[1], z); z = fmaf(c0.z, h[2], z); z = fmaf(c0.w, h[3], z);
        z = fmaf(c1.x, h[4], z); z = fmaf(c1.y, h[5], z); z = fmaf(c1.z, h[6], z); z = fmaf(c1.w, h[7], z);
        psi[t] = z >= 0.f ? z : beta * (__expf(z) - 1.f);
    }
}

// The key sweep's layout of one folded network (264 floats): rows of 8 values, one a
// hidden unit (or an output), so that two hidden units (outputs) take one two-lane FMA.
//   [0, 112)   rows q = 0..13: the coefficients of the canonical inflow faces ux, uy,
//              uz (q = 0..11), |mu| (q = 12) and |eta| (q = 13) in every hidden unit
//   [112, 192) rows 0..9: the 8 canonical sources, sigma_t, the bias with the cell
//              sizes folded in
//   [192, 256) rows k = 0..7: W2[t][k] for the outputs t
//   [256, 264) b2
constexpr int kOnRowIn = 0, kOnRowKey = 112, kOnRowW2 = 192, kOnRowB2 = 256, kOnRows = 264;

// The 264-float layout of the folded network w (288 floats) for cell sizes hx, hy, hz;
// element e of the layout (the caller's threads split e over 0..263).
__device__ __forceinline__ float octnet_row_layout(const float *__restrict__ w, int e, float hx, float hy, float hz)
{
    if (e < kOnRowKey) {
        const int q = e / kOnHid, k = e % kOnHid;
        return w[24 * k + (q < 12 ? q : 20 + (q - 12))];
    }
    if (e < kOnRowW2) {
        const int r = (e - kOnRowKey) / kOnHid, k = (e - kOnRowKey) % kOnHid;
        if (r < 8) return w[24 * k + 12 + r];
        if (r == 8) return w[24 * k + 22];
        return fmaf(w[kOnFoldH + 3 * k], hx, fmaf(w[kOnFoldH + 3 * k + 1], hy, fmaf(w[kOnFoldH + 3 * k + 2], hz,
                                                                                    w[24 * k + 23])));
    }
    if (e < kOnRowB2) {
        const int k = (e - kOnRowW2) / kOnOut, t = (e - kOnRowW2) % kOnOut;
        return w[kOnFoldW2 + 8 * t + k];
    }
    return w[kOnFoldB2 + (e - kOnRowB2)];
}

// acc[0..3] (units 0..7 in pairs) += x * row (8 values at r, 16-byte aligned)
__device__ __forceinline__ void octnet_row_fma(const float *r, float x, float2 (&acc)[4])
{
    const float4 r0 = *reinterpret_cast<const float4 *>(r), r1 = *reinterpret_cast<const float4 *>(r + 4);
    const float2 xx = make_float2(x, x);
    acc[0] = __ffma2_rn(make_float2(r0.x, r0.y), xx, acc[0]);
    acc[1] = __ffma2_rn(make_float2(r0.z, r0.w), xx, acc[1]);
    acc[2] = __ffma2_rn(make_float2(r1.x, r1.y), xx, acc[2]);
    acc[3] = __ffma2_rn(make_float2(r1.z, r1.w), xx, acc[3]);
}

// The key's part of each hidden unit's input on the row layout at wr: the bias (with
// the cell sizes folded in), the 8 canonical sources and sigma_t, shared by every
// direction of the key, so the key sweep forms it once per key; two hidden units a
// two-lane FMA.
__device__ __forceinline__ void octnet_key_part_rows(const float *__restrict__ wr, const float (&S)[8], float sig,
                                                     float (&ak)[kOnHid])
{
    float2 acc[4];
    {
        const float *b = wr + kOnRowKey + 9 * kOnHid;
        const float4 b0 = *reinterpret_cast<const float4 *>(b), b1 = *reinterpret_cast<const float4 *>(b + 4);
        acc[0] = make_float2(b0.x, b0.y); acc[1] = make_float2(b0.z, b0.w);
        acc[2] = make_float2(b1.x, b1.y); acc[3] = make_float2(b1.z, b1.w);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) octnet_row_fma(wr + kOnRowKey + q * kOnHid, S[q], acc);
    octnet_row_fma(wr + kOnRowKey + 8 * kOnHid, sig, acc);
#pragma unroll
    for (int p = 0; p < 4; ++p) { ak[2 * p] = acc[p].x; ak[2 * p + 1] = acc[p].y; }
}

// One direction of a key: psi (canonical node order) from the key's part of the hidden
// inputs (octnet_key_part_rows, two 4-vectors at ak0 / ak1), the direction's |mu| and
// |eta|, and the three inflow faces (4-vectors at fx, fy, fz): the function of
// octnet_forward with the sums grouped differently (|mu|, |eta|, then the 12 face
// values; the outputs over the hidden units in order), two hidden units or two outputs
// a two-lane FMA.
__device__ __forceinline__ void octnet_key_row_rows(const float *__restrict__ wr, const float4 *ak0,
                                                    const float4 *ak1, const float4 *fx, const float4 *fy,
                                                    const float4 *fz, float amu, float aeta, float (&psi)[8])
{
    const float4 ux = *fx, uy = *fy, uz = *fz, a0 = *ak0, a1 = *ak1;
    float bm = fmaxf(fmaxf(fmaxf(fabsf(ux.x), fabsf(ux.y)), fmaxf(fabsf(ux.z), fabsf(ux.w))),
                     fmaxf(fmaxf(fabsf(uy.x), fabsf(uy.y)), fmaxf(fabsf(uy.z), fabsf(uy.w))));
    bm = fmaxf(bm, fmaxf(fmaxf(fabsf(uz.x), fabsf(uz.y)), fmaxf(fabsf(uz.z), fabsf(uz.w))));
    const float beta = kOnBetaFrac * bm;
    float2 acc[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                     make_float2(a1.z, a1.w)};
    octnet_row_fma(wr + kOnRowIn + 12 * kOnHid, amu, acc);
    octnet_row_fma(wr + kOnRowIn + 13 * kOnHid, aeta, acc);
    const float u[12] = {ux.x, ux.y, ux.z, ux.w, uy.x, uy.y, uy.z, uy.w, uz.x, uz.y, uz.z, uz.w};
#pragma unroll
    for (int q = 0; q < 12; ++q) octnet_row_fma(wr + kOnRowIn + q * kOnHid, u[q], acc);
    float h[kOnHid];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        h[2 * p] = octnet_tanh(acc[p].x);
        h[2 * p + 1] = octnet_tanh(acc[p].y);
    }
    float2 z[4];
    {
        const float *b = wr + kOnRowB2;
        const float4 b0 = *reinterpret_cast<const float4 *>(b), b1 = *reinterpret_cast<const float4 *>(b + 4);
        z[0] = make_float2(b0.x, b0.y); z[1] = make_float2(b0.z, b0.w);
        z[2] = make_float2(b1.x, b1.y); z[3] = make_float2(b1.z, b1.w);
    }
#pragma unroll
    for (int k = 0; k < kOnHid; ++k) octnet_row_fma(wr + kOnRowW2 + k * kOnOut, h[k], z);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float za = z[p].x, zb = z[p].y;
        psi[2 * p] = za >= 0.f ? za : beta * (__expf(za) - 1.f);
        psi[2 * p + 1] = zb >= 0.f ? zb : beta * (__expf(zb) - 1.f);
    }
}

// Two canonical one-cell problems through the same folded network (weights at w,
// the cell-size terms already in the biases): every weight read feeds two
// multiply-adds.  Same arithmetic, in the same order, as octnet_forward<false>.
__device__ __forceinline__ void octnet_forward2(const float *__restrict__ w, const float (&ux)[2][4],
                                                const float (&uy)[2][4], const float (&uz)[2][4],
                                                const float (&S)[2][8], const float (&amu)[2], const float (&aeta)[2],
                                                const float (&sig)[2], float (&psi)[2][8])
{
    float beta[2], h[2][kOnHid];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        float bm = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) bm = fmaxf(bm, fmaxf(fabsf(ux[j][t]), fmaxf(fabsf(uy[j][t]), fabsf(uz[j][t]))));
        beta[j] = kOnBetaFrac * bm;
    }
#pragma unroll
    for (int k = 0; k < kOnHid; ++k) {
        const float4 *r = reinterpret_cast<const float4 *>(w + 24 * k);
        const float4 c0 = r[0], c1 = r[1], c2 = r[2], c3 = r[3], c4 = r[4], c5 = r[5];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float a = c5.w;
            a = fmaf(c0.x, ux[j][0], a); a = fmaf(c0.y, ux[j][1], a); a = fmaf(c0.z, ux[j][2], a);
            a = fmaf(c0.w, ux[j][3], a);
            a = fmaf(c1.x, uy[j][0], a); a = fmaf(c1.y, uy[j][1], a); a = fmaf(c1.z, uy[j][2], a);
            a = fmaf(c1.w, uy[j][3], a);
            a = fmaf(c2.x, uz[j][0], a); a = fmaf(c2.y, uz[j][1], a); a = fmaf(c2.z, uz[j][2], a);
            a = fmaf(c2.w, uz[j][3], a);
            a = fmaf(c3.x, S[j][0], a); a = fmaf(c3.y, S[j][1], a); a = fmaf(c3.z, S[j][2], a);
            a = fmaf(c3.w, S[j][3], a);
            a = fmaf(c4.x, S[j][4], a); a = fmaf(c4.y, S[j][5], a); a = fmaf(c4.z, S[j][6], a);
            a = fmaf(c4.w, S[j][7], a);
            a = fmaf(c5.x, amu[j], a); a = fmaf(c5.y, aeta[j], a); a = fmaf(c5.z, sig[j], a);
            h[j][k] = octnet_tanh(a);
        }
    }
#pragma unroll
    for (int t = 0; t < kOnOut; ++t) {
        const float4 *r = reinterpret_cast<const float4 *>(w + kOnFoldW2 + 8 * t);
        const float4 c0 = r[0], c1 = r[1];
        const float b2 = w[kOnFoldB2 + t];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float z = b2;
            z = fmaf(c0.x, h[j][0], z); z = fmaf(c0.y, h[j][1], z); z = fmaf(c0.z, h[j][2], z);
            z = fmaf(c0.w, h[j][3], z);
            z = fmaf(c1.x, h[j][4], z); z = fmaf(c1.y, h[j][5], z); z = fmaf(c1.z, h[j][6], z);
            z = fmaf(c1.w, h[j][7], z);
            psi[j][t] = z >= 0.f ? z : beta[j] * (__expf(z) - 1.f);
        }
    }
}

}  // namespace sn

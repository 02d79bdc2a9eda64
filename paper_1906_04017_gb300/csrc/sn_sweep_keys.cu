// sn_sweep_keys.cu -- the FP32 elimination sweep on box cells with isotropic
// scattering (modes SN_SOLVE_GE32R and SN_SOLVE_GE32): the hyperplane wavefront of
// Sec. 2 (after Eq. (14)) with one thread per key.
//
// Key.  A key is (octant o, cell of the hyperplane, group g).  Its thread solves the
// cell's system (14) for a chunk of the octant's directions in turn (all of them
// where the hyperplane has enough keys to fill the GPU; on the small hyperplanes at
// the two ends of the wavefront the directions are split over NCH threads so that
// the launch still has enough threads).  Everything a key's directions share is
// done once per key: the cell, its opacity, the source term (Mh x Mh x Mh) S of the
// right-hand side (ge8.cuh), the face-plane offsets; the scalar-flux partial
// sum_d w_d psi_d of Eqs. (9), (13) accumulates in registers in a fixed direction
// order, so no shared-memory reduction or block barrier sits in the direction loop.
//
// Face planes.  Per octant, one 4-vector per (column, direction, group) of each of
// the x-, y- and z-planes, the group index fastest: [o][column][d][g].  The keys of a
// warp are consecutive groups of the same cells, so a warp's face loads and stores
// are whole 128-byte lines.  A cell reads its inflow slot and overwrites it with its
// outflow (within one hyperplane every slot belongs to one cell).  On the inflow
// boundary the key reads a 4-vector holding psi_inc of its group and face, stored
// after the planes, with a direction stride of zero, so the direction loop has no
// boundary test; on the outflow boundary the outflow is stored like any other, and
// after the last hyperplane every slot holds the outflow of the last cell of its
// column: the leakage kernel below sums the boundary leakage from them.
//
// Prefetch.  The next direction's three inflow faces are copied into a per-thread
// shared-memory stage (cp.async) while the current direction is solved.  A key's
// cell, opacity and source are read before the kernel waits for the previous
// hyperplane (programmatic dependent launch): none of them is written by the sweep.
//
// The flux partials go to phi_oct[o][c][g][8] (physical node order); the reduction
// kernel of sn_sweep.cu sums the eight octants in a fixed order.  Nothing is atomic:
// the flux is bit-reproducible run to run.
#include <algorithm>

#include "ge8.cuh"
#include "sn_internal.cuh"
#include "sweep_common.cuh"

namespace sn {

constexpr int kKeyBlock = 128;   // threads a CTA
constexpr int kKeyMaxDo = 64;    // directions per octant the kernel takes
// CTAs per SM: 3 (168 registers a thread) measured faster on blocked_64 than 4
// (128 registers, with spills of the refined solve): 5.55 against 5.91 ms a sweep
#ifndef SN_KEY_MINBLOCKS
#define SN_KEY_MINBLOCKS 3
#endif

struct KeyArgs {
    int nx, ny, nz, G, Do, C;
    int nkeys;                   // keys of one octant on this hyperplane (cells x G)
    FastDiv divG;                // key -> (cell of the hyperplane, group)
    const uint32_t *cells;       // packed (i',j',k') of the hyperplane's cells
    const float *sigt;           // [G][C]
    const float *S;              // [G][C][8]
    const float4 *dir;           // [Do] (3|Omega_x|/dx, 3|Omega_y|/dy, 3|Omega_z|/dz, w)
    float4 *face;                // x-planes | y-planes | z-planes | inflow vectors [G][6]
    uint32_t off_y, off_z, off_in;
    float *phi_oct;              // [8][C][G][8]
};

template <bool REFINE, int NCH>
__global__ void __launch_bounds__(kKeyBlock, SN_KEY_MINBLOCKS) sweep_ge_keys(KeyArgs a)
{
    constexpr int KB = kKeyBlock / NCH;                       // keys a CTA
    __shared__ __align__(16) float4 stage[2][3][kKeyBlock];  // per-thread inflow stages
    __shared__ __align__(16) float4 msrc[2][kKeyBlock];      // per-thread (Mh x Mh x Mh) S
    __shared__ __align__(16) float4 dsm[kKeyMaxDo];
    __shared__ __align__(16) float red[NCH > 1 ? NCH * KB * 8 : 4];
    __shared__ int kdst[kKeyBlock];
    griddep_launch();
    const int t = threadIdx.x, o = blockIdx.y;
    const int chunk = t / KB, lk = t - chunk * KB;
    const int key = (int)blockIdx.x * KB + lk;
    const bool act = key < a.nkeys;
    const int Do = a.Do, G = a.G;
    const int d0 = chunk * Do / NCH, d1 = (chunk + 1) * Do / NCH;
    for (int e = t; e < Do; e += kKeyBlock) dsm[e] = a.dir[e];

    // the key: set-up tables and the sweep's inputs only, so this runs while the
    // previous hyperplane may still be running
    float sig = 0.f;
    uint32_t ou0 = 0, ou1 = 0, ou2 = 0;   // this direction's slots
    uint32_t inb = 0, bnd = 0;            // inflow vectors of the key's group; inflow-boundary axes
    int dst = -1;                         // (o C + c) G + g: the key's flux partial
    if (act) {
        const uint32_t cidx = a.divG.div((uint32_t)key);
        const int g = key - (int)cidx * G;
        const uint32_t pk = a.cells[cidx];
        const int ip = pk & 1023, jp = (pk >> 10) & 1023, kp = pk >> 20;
        const int i = (o & 1) ? a.nx - 1 - ip : ip;
        const int j = (o & 2) ? a.ny - 1 - jp : jp;
        const int k = (o & 4) ? a.nz - 1 - kp : kp;
        const int c = i + a.nx * (j + a.ny * k);
        const int gc = g * a.C + c;
        sig = __ldg(a.sigt + gc);
        const float4 s0 = __ldg(reinterpret_cast<const float4 *>(a.S) + 2 * (int64_t)gc);
        const float4 s1 = __ldg(reinterpret_cast<const float4 *>(a.S) + 2 * (int64_t)gc + 1);
        float Sm[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
        mirror8(Sm, o);          // canonical node n = physical n ^ o
        mh_axis<0>(Sm);
        mh_axis<1>(Sm);
        mh_axis<2>(Sm);
        msrc[0][t] = make_float4(Sm[0], Sm[1], Sm[2], Sm[3]);
        msrc[1][t] = make_float4(Sm[4], Sm[5], Sm[6], Sm[7]);
        const uint32_t DG = (uint32_t)(Do * G), first = (uint32_t)(d0 * G + g);
        ou0 = (uint32_t)(o * a.ny * a.nz + jp + a.ny * kp) * DG + first;
        ou1 = a.off_y + (uint32_t)(o * a.nx * a.nz + ip + a.nx * kp) * DG + first;
        ou2 = a.off_z + (uint32_t)(o * a.nx * a.ny + ip + a.nx * jp) * DG + first;
        inb = a.off_in + 6u * (uint32_t)g;
        bnd = (ip == 0 ? 1u : 0u) | (jp == 0 ? 2u : 0u) | (kp == 0 ? 4u : 0u);
        dst = (o * a.C + c) * G + g;
    }
    kdst[t] = dst;
    __syncthreads();   // direction table
    griddep_wait();    // the previous hyperplane's outflow faces are complete

    float phi[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) phi[n] = 0.f;
    if (act && d0 < d1) {
        constexpr uint32_t AX = kKeyBlock * 16;   // bytes between the faces of a stage
        constexpr uint32_t SP = 3 * AX;           // bytes between the two stages
        const uint32_t sb = smem_u32(&stage[0][0][t]);
        // inflow slot of direction d: the outflow slot (in place), or on the inflow
        // boundary the group's psi_inc vector of that face (every direction)
        auto issue = [&](uint32_t buf, uint32_t s0, uint32_t s1, uint32_t s2) {
            const uint32_t nb = sb + buf * SP;
            cp_async16(nb, a.face + ((bnd & 1u) ? inb + (uint32_t)(o & 1) : s0));
            cp_async16(nb + AX, a.face + ((bnd & 2u) ? inb + 2u + (uint32_t)((o >> 1) & 1) : s1));
            cp_async16(nb + 2 * AX, a.face + ((bnd & 4u) ? inb + 4u + (uint32_t)((o >> 2) & 1) : s2));
        };
        issue(0u, ou0, ou1, ou2);
        cp_async_commit();
        for (int d = d0; d < d1; ++d) {
            const int cur = (d - d0) & 1;
            if (d + 1 < d1) issue((uint32_t)(cur ^ 1), ou0 + (uint32_t)G, ou1 + (uint32_t)G, ou2 + (uint32_t)G);
            cp_async_commit();
            cp_async_wait_pending<1>();   // this direction's faces have landed
            const float4 fx = stage[cur][0][t], fy = stage[cur][1][t], fz = stage[cur][2][t];
            const float4 m0 = msrc[0][t], m1 = msrc[1][t];
            const float4 dd = dsm[d];
            const float ux[4] = {fx.x, fx.y, fx.z, fx.w};
            const float uy[4] = {fy.x, fy.y, fy.z, fy.w};
            const float uz[4] = {fz.x, fz.y, fz.z, fz.w};
            const float Sm[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
            float x[8];
            cell_solve_key<REFINE>(dd.x, dd.y, dd.z, sig, Sm, ux, uy, uz, x);
            // outflow faces (canonical in-face order): x-face a = 1, y-face b = 1, z-face c = 1
            a.face[ou0] = make_float4(x[1], x[3], x[5], x[7]);
            a.face[ou1] = make_float4(x[2], x[3], x[6], x[7]);
            a.face[ou2] = make_float4(x[4], x[5], x[6], x[7]);
            ou0 += (uint32_t)G;
            ou1 += (uint32_t)G;
            ou2 += (uint32_t)G;
#pragma unroll
            for (int n = 0; n < 8; ++n) phi[n] = fmaf(dd.w, x[n], phi[n]);
        }
    }
    mirror8(phi, o);   // physical node order
    if constexpr (NCH == 1) {
        if (act) {
            float4 *p = reinterpret_cast<float4 *>(a.phi_oct) + 2 * (int64_t)kdst[t];
            p[0] = make_float4(phi[0], phi[1], phi[2], phi[3]);
            p[1] = make_float4(phi[4], phi[5], phi[6], phi[7]);
        }
    } else {
        // the chunks of a key add their partials in chunk order
        float4 *r = reinterpret_cast<float4 *>(red + (chunk * KB + lk) * 8);
        r[0] = make_float4(phi[0], phi[1], phi[2], phi[3]);
        r[1] = make_float4(phi[4], phi[5], phi[6], phi[7]);
        __syncthreads();
        for (int e = t; e < KB * 8; e += kKeyBlock) {
            const int kk = e >> 3, n = e & 7;
            const int dk = kdst[kk];   // chunk 0's thread of key kk
            if (dk < 0) continue;
            float s = red[kk * 8 + n];
#pragma unroll
            for (int q = 1; q < NCH; ++q) s += red[(q * KB + kk) * 8 + n];
            a.phi_oct[(int64_t)dk * 8 + n] = s;
        }
    }
}

// Boundary leakage of a key sweep: after the last hyperplane every face slot holds
// the outflow of the last cell of its column, so the leakage through the outflow
// boundary is sum w_d (3|Omega_a|/h_a) (sum of the 4 face values) V / 12 over all
// slots (the weight-1 form of the balance, as in the other sweeps).  FP32 per
// thread over a few slots, FP64 across threads.
__global__ void __launch_bounds__(256) leak_keys_kernel(const float4 *__restrict__ face, uint32_t nfx, uint32_t nfy,
                                                        uint32_t nfz, int G, int Do, const float4 *__restrict__ dir,
                                                        double vol12, double *acc)
{
    __shared__ float4 dsm[kKeyMaxDo];
    for (int e = threadIdx.x; e < Do; e += blockDim.x) dsm[e] = dir[e];
    __syncthreads();
    const uint32_t total = nfx + nfy + nfz;
    float s = 0.f;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int ax = q < nfx ? 0 : (q < nfx + nfy ? 1 : 2);
        const uint32_t lq = q - (ax == 0 ? 0u : (ax == 1 ? nfx : nfx + nfy));
        const int d = (int)((lq / (uint32_t)G) % (uint32_t)Do);
        const float4 v = face[q];
        const float4 dd = dsm[d];
        const float ta = ax == 0 ? dd.x : (ax == 1 ? dd.y : dd.z);
        s = fmaf(dd.w * ta, (v.x + v.y) + (v.z + v.w), s);
    }
    double ds = (double)s * vol12;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ds += __shfl_down_sync(0xffffffffu, ds, off);
    if ((threadIdx.x & 31) == 0 && ds != 0.0) atomicAdd(acc + ACC_LEAK, ds);
}

// Whether the key sweep serves this handle: FP32 box cells, isotropic scattering, a
// direction table that fits, and 32-bit face offsets.
bool key_sweep_ok(sn_handle h)
{
    return !h->fp64 && !h->geom && h->K == 1 && h->Do <= kKeyMaxDo && h->face_in > 0 &&
           (uint64_t)h->face_in + 6ull * (uint64_t)h->G < (1ull << 32);
}

// Directions split over NCH threads a key on a hyperplane with `keys` keys (all
// octants): the fewest chunks that still give the launch about one resident
// thread per SM slot, and no more chunks than directions.
static int key_chunks(int64_t keys, int Do)
{
    const int64_t slots = (int64_t)num_sms() * SN_KEY_MINBLOCKS * kKeyBlock;
    int nch = 1;
    while (nch < 8 && 2 * nch <= Do && keys * nch < slots) nch *= 2;
    return nch;
}

template <bool REFINE, int NCH>
static cudaError_t launch_keys_plane(bool pdl, const KeyArgs &a, cudaStream_t st)
{
    constexpr int KB = kKeyBlock / NCH;
    const dim3 grid((unsigned)((a.nkeys + KB - 1) / KB), 8);
    return launch_k(pdl, sweep_ge_keys<REFINE, NCH>, grid, dim3(kKeyBlock), 0, st, a);
}

template <bool REFINE>
static cudaError_t launch_keys_nch(int nch, bool pdl, const KeyArgs &a, cudaStream_t st)
{
    switch (nch) {
    case 1: return launch_keys_plane<REFINE, 1>(pdl, a, st);
    case 2: return launch_keys_plane<REFINE, 2>(pdl, a, st);
    case 4: return launch_keys_plane<REFINE, 4>(pdl, a, st);
    default: return launch_keys_plane<REFINE, 8>(pdl, a, st);
    }
}

sn_status launch_sweep_keys(sn_handle h, const float *S, float *phi_oct, bool refine, cudaStream_t st)
{
    KeyArgs a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.G = h->G; a.Do = h->Do; a.C = (int)h->ncell;
    a.divG = FastDiv((uint32_t)h->G);
    a.sigt = (const float *)h->sigt;
    a.S = S;
    a.dir = reinterpret_cast<const float4 *>(h->dir);
    a.face = reinterpret_cast<float4 *>(h->face);
    a.off_y = (uint32_t)h->face_x;
    a.off_z = (uint32_t)(h->face_x + h->face_y);
    a.off_in = (uint32_t)h->face_in;
    a.phi_oct = phi_oct;
    if (h->prof) SN_CK(h, cudaEventRecord(h->ev_sweep[0], st));
    for (int s = 0; s < h->nplanes; ++s) {
        const int64_t n = h->plane_off[s + 1] - h->plane_off[s];
        a.cells = h->plane_cells + h->plane_off[s];
        a.nkeys = (int)(n * h->G);
        const int nch = key_chunks(8 * n * h->G, h->Do);
        // hyperplanes after the first overlap their launch with the previous one's drain
        SN_CK(h, refine ? launch_keys_nch<true>(nch, s > 0, a, st) : launch_keys_nch<false>(nch, s > 0, a, st));
    }
    SN_CK(h, cudaGetLastError());
    if (h->prof) {
        SN_CK(h, cudaEventRecord(h->ev_sweep[1], st));
        h->prof_pending = true;
    }
    const uint32_t total = (uint32_t)(h->face_x + h->face_y + h->face_z);
    const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 8);
    leak_keys_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float4 *>(h->face), (uint32_t)h->face_x,
                                           (uint32_t)h->face_y, (uint32_t)h->face_z, h->G, h->Do,
                                           reinterpret_cast<const float4 *>(h->dir), h->dx * h->dy * h->dz / 12.0,
                                           h->acc);
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

}  // namespace sn

// sn_sweep.cu -- the hyperplane-wavefront transport sweep (Sec. 2, after Eq. (14)),
// the scalar-flux reduction (Eqs. (9), (13)), the isotropic source build (Eqs. (2),
// (6)) and the source iteration of the C ABI.
//
// Wavefront.  In octant o the mesh index is mirrored (i' = nx-1-i when Omega_x < 0,
// likewise j', k'), so every direction of the octant flows from the corner
// (0,0,0)' and a cell's upwind neighbours lie on hyperplane i'+j'+k' - 1.  One launch
// handles hyperplane s of all 8 octants at once, every direction of each octant
// and every group: the launch has 8 * cells(s) * G keys (octant, cell, group), and
// each key has Do threads, one per direction of the octant.
//
// Face planes.  Octant o keeps three planes per (group, direction): the x-plane holds
// the 4 canonical face values leaving each (j',k') column, and so on.  A cell reads
// its inflow from the planes and overwrites the same slots with its outflow; within
// one hyperplane no two cells share a slot, so the update is in place.  Slot
// layout [o][column][g][d] of 4-vectors makes the Do x G threads of one cell read
// and write one contiguous run.  Cells on the inflow boundary take psi_inc instead.
//
// Scalar flux.  The Do threads of a key add w_d psi_d in shared memory in a fixed
// order and write one per-octant partial phi_oct[o][c][g][8]; the reduction kernel
// sums the 8 octants in a fixed order.  Nothing is atomic, so the flux is
// bit-reproducible run to run.
//
// Element type T: float (GE32R / GE32) or double (GE64, FP64 handles).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ge8.cuh"
#include "hex.cuh"
#include "octnet.cuh"
#include "sn_internal.cuh"
#include "sweep_common.cuh"

namespace sn {

template <typename T>
struct SweepArgs {
    int nx, ny, nz, G, Do, ncells_plane, keys_per_cta, ntiles;
    int C;                   // cells (G * C * 8 < 2^31 is checked at set-up)
    FastDiv divG;            // key -> (cell index, group)
    const uint32_t *cells;   // packed (i',j',k') of the cells of this hyperplane
    const T *sigt;           // [G][C]
    const T *S;              // [G][C][8]
    const T *psi_inc;        // [G][6]
    const DirData<T> *dir;   // [Do]
    Vec4<T> *fx, *fy, *fz;   // face planes
    T *phi_oct;              // [8][C][G][8]
    double *leak;            // accumulator
    T vol12;                 // V / 12
    // adjoint passes (XMODE 1: store the angular flux, 2: pair it with the adjoint)
    Vec4<T> *psi_blk;        // [block cells][8 octants][G][Do] x 8 nodes (two 4-vectors)
    uint32_t blk_base;       // STORE: offset of this hyperplane's cells in psi_blk
    uint32_t pair_base;      // PAIR: offset of the forward hyperplane's cells in psi_blk
    const uint32_t *plane_pos;   // position of each primed cell within its hyperplane
    double *grad;            // PAIR: dR/dsigma_t [G][C]
    T vol216;                // V / 216
    // harvesting (XMODE 3): a hashed sample of the solves is written out as one-cell
    // problems in the canonical (positive-octant) frame
    float *harvest;          // [cap][27]
    unsigned long long *harvest_count;
    uint32_t harvest_cap, harvest_threshold, harvest_seed, plane;
    const float4 *dir_abs;   // |Omega| of each direction of an octant
    T hx, hy, hz;
    const float *onet;       // [8][288] folded octant networks (network sweeps)
    int K;                   // flux / source moments (anisotropic scattering; 1 = isotropic)
    const T *yhat;           // [8][Do][K] sqrt(4 pi) Y_k of every direction (octant-major)
    const T *geom;           // general hexahedral cells: element records [C][544] (hex.cuh)
    const T *omabs;          // |Omega| of the octant's directions [Do][3]
    const T *geomB;          // [C][8][192] per-octant streaming + outflow-face matrices
};

// grid = (blocks per octant, 8 octants); block = keys_per_cta keys x Do directions,
// rounded up to whole warps.  XMODE 0: plain sweep (the adjoint's sweeps; plain
// forward sweeps use sweep_ge_tiles below); 1: also store each angular flux
// (physical node order) for the adjoint; 2: adjoint pass that pairs its angular flux
// with the stored forward one of the opposite direction (see sn_adjoint.cu).
// 128-thread blocks, 4 per SM (128 registers a thread): measured faster on GB300 than
// fewer, larger-register blocks -- the elimination is latency-bound, warps beat spills
#ifndef SN_GE_MINBLOCKS
#define SN_GE_MINBLOCKS 4
#endif
#ifndef SN_GE_BLOCK
#define SN_GE_BLOCK 128
#endif
// persistent form: 4 CTAs per SM (128 registers a thread, a few spills) measured faster
// than 3 (168 registers) or 2 once a tile needed a single barrier
#ifndef SN_GE_TILE_MINBLOCKS
#define SN_GE_TILE_MINBLOCKS 4
#endif
template <typename T, bool REFINE, int XMODE = 0>
__global__ void __launch_bounds__(SN_GE_BLOCK, sizeof(T) == 4 ? SN_GE_MINBLOCKS : 1) sweep_plane_ge(SweepArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char red_raw[];
    T *red = reinterpret_cast<T *>(red_raw);   // [blockDim.x][9]
    griddep_launch();
    griddep_wait();
    const int Do = a.Do;
    const int o = blockIdx.y;                  // octant: sign bits of Omega
    const int lk = (int)threadIdx.x / Do;
    const int d = (int)threadIdx.x - lk * Do;
    const uint32_t key = blockIdx.x * (uint32_t)a.keys_per_cta + (uint32_t)lk;
    // threads past keys_per_cta * Do (warp rounding) or past the last key idle
    const bool active = lk < a.keys_per_cta && key < (uint32_t)a.ncells_plane * (uint32_t)a.G;
    int g = 0, c = 0;
    T leak = T(0), pair = T(0);
    if (active) {
        const uint32_t cidx = a.divG.div(key);
        g = (int)(key - cidx * (uint32_t)a.G);
        const uint32_t pk = a.cells[cidx];
        const int ip = pk & 1023, jp = (pk >> 10) & 1023, kp = pk >> 20;
        const int i = (o & 1) ? a.nx - 1 - ip : ip;
        const int j = (o & 2) ? a.ny - 1 - jp : jp;
        const int k = (o & 4) ? a.nz - 1 - kp : kp;
        c = i + a.nx * (j + a.ny * k);
        const DirData<T> dd = a.dir[d];
        const int GD = a.G * Do, gd = g * Do + d;
        const int64_t ix = (int64_t)(o * a.ny * a.nz + jp + a.ny * kp) * GD + gd;
        const int64_t iy = (int64_t)(o * a.nx * a.nz + ip + a.nx * kp) * GD + gd;
        const int64_t iz = (int64_t)(o * a.nx * a.ny + ip + a.nx * jp) * GD + gd;
        T ux[4], uy[4], uz[4];
        if (ip == 0) {
            const T v = a.psi_inc[6 * g + (o & 1)];
            ux[0] = ux[1] = ux[2] = ux[3] = v;
        } else {
            load4(ux, a.fx + ix);
        }
        if (jp == 0) {
            const T v = a.psi_inc[6 * g + 2 + ((o >> 1) & 1)];
            uy[0] = uy[1] = uy[2] = uy[3] = v;
        } else {
            load4(uy, a.fy + iy);
        }
        if (kp == 0) {
            const T v = a.psi_inc[6 * g + 4 + ((o >> 2) & 1)];
            uz[0] = uz[1] = uz[2] = uz[3] = v;
        } else {
            load4(uz, a.fz + iz);
        }
        const int gc = g * a.C + c;
        const T sig = a.sigt[gc];
        const Vec4<T> *Sp = reinterpret_cast<const Vec4<T> *>(a.S + (int64_t)gc * 8);
        T S[8], s0[4], s1[4];
        load4(s0, Sp);
        load4(s1, Sp + 1);
#pragma unroll
        for (int n = 0; n < 4; ++n) { S[n] = s0[n]; S[4 + n] = s1[n]; }
        mirror8(S, o);
        T x[8];
        cell_solve_canonical<T, REFINE>(dd.t3x, dd.t3y, dd.t3z, sig, S, ux, uy, uz, x);
        if (XMODE == 3) {
            // keep this solve with probability threshold / 2^32 (hash of its identity)
            uint32_t hsh = a.harvest_seed ^ (a.plane * 0x9E3779B9u) ^ ((uint32_t)o * 0x85EBCA6Bu) ^
                           (key * 0xC2B2AE35u) ^ ((uint32_t)d * 0x27D4EB2Fu);
            hsh ^= hsh >> 16; hsh *= 0x7FEB352Du; hsh ^= hsh >> 15; hsh *= 0x846CA68Bu; hsh ^= hsh >> 16;
            if (hsh < a.harvest_threshold) {
                const unsigned long long slot = atomicAdd(a.harvest_count, 1ull);
                if (slot < a.harvest_cap) {
                    float *q = a.harvest + 27 * slot;
                    const float4 ab = a.dir_abs[d];
                    q[0] = ab.x; q[1] = ab.y; q[2] = ab.z;
                    q[3] = (float)a.hx; q[4] = (float)a.hy; q[5] = (float)a.hz;
                    q[6] = (float)sig;
#pragma unroll
                    for (int n = 0; n < 8; ++n) q[7 + n] = (float)S[n];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        q[15 + t] = (float)ux[t];
                        q[19 + t] = (float)uy[t];
                        q[23 + t] = (float)uz[t];
                    }
                }
            }
        }
        // outflow faces (canonical in-face order): x-face a=1, y-face b=1, z-face c=1
        if (ip < a.nx - 1) store4(a.fx + ix, x[1], x[3], x[5], x[7]);
        else leak += dd.t3x * (x[1] + x[3] + x[5] + x[7]);
        if (jp < a.ny - 1) store4(a.fy + iy, x[2], x[3], x[6], x[7]);
        else leak += dd.t3y * (x[2] + x[3] + x[6] + x[7]);
        if (kp < a.nz - 1) store4(a.fz + iz, x[4], x[5], x[6], x[7]);
        else leak += dd.t3z * (x[4] + x[5] + x[6] + x[7]);
        leak *= dd.w * a.vol12;
        if (XMODE == 1) {
            // forward angular flux, physical node order
            T xp[8];
#pragma unroll
            for (int n = 0; n < 8; ++n) xp[n] = x[n];
            mirror8(xp, o);
            Vec4<T> *slot = a.psi_blk + 2 * (((int64_t)(a.blk_base + cidx) * 8 + o) * GD + gd);
            store4(slot, xp[0], xp[1], xp[2], xp[3]);
            store4(slot + 1, xp[4], xp[5], xp[6], xp[7]);
        }
        if (XMODE == 2) {
            // the forward flux of the opposite direction (octant o ^ 7, same index d) at
            // this cell: it sits on forward hyperplane nplanes - 1 - s at the position of
            // the mirrored primed index
            const uint32_t cf = a.plane_pos[(a.nx - 1 - ip) + a.nx * ((a.ny - 1 - jp) + a.ny * (a.nz - 1 - kp))];
            const Vec4<T> *slot = a.psi_blk + 2 * (((int64_t)(a.pair_base + cf) * 8 + (o ^ 7)) * GD + gd);
            T pf[8], p0[4], p1[4];
            load4(p0, slot);
            load4(p1, slot + 1);
#pragma unroll
            for (int n = 0; n < 4; ++n) { pf[n] = p0[n]; pf[4 + n] = p1[n]; }
            mirror8(pf, o);          // into this direction's canonical frame
            mh_axis<0>(pf);
            mh_axis<1>(pf);
            mh_axis<2>(pf);
            T dot = T(0);
#pragma unroll
            for (int n = 0; n < 8; ++n) dot += x[n] * pf[n];
            pair = -dd.w * a.vol216 * dot;
        }
        // w_d psi in physical node order: canonical node n lands on physical n ^ o
        T *r = red + threadIdx.x * 9;
#pragma unroll
        for (int n = 0; n < 8; ++n) r[n ^ o] = dd.w * x[n];
        if (XMODE == 2) r[8] = pair;
    }
    __syncthreads();
    if (active) {
        T *dst = a.phi_oct + (((int64_t)o * a.C + c) * a.G + g) * 8;
        const T *base = red + (lk * Do) * 9;
        for (int n = d; n < 8; n += Do) {
            T s = T(0);
            for (int q = 0; q < Do; ++q) s += base[q * 9 + n];
            dst[n] = s;
        }
        if (XMODE == 2 && d == 0) {
            double s = 0.0;
            for (int q = 0; q < Do; ++q) s += (double)base[q * 9 + 8];
            atomicAdd(a.grad + (int64_t)g * a.C + c, s);
        }
    }
    // leakage: warp sum, one double atomic per warp that saw any
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) leak += __shfl_down_sync(0xffffffffu, leak, off);
    if ((threadIdx.x & 31) == 0 && leak != T(0)) atomicAdd(a.leak, (double)leak);
}

// Persistent form of the elimination sweep (plain forward sweeps, FP32 and FP64): a
// CTA loops over tiles of keys_per_cta keys x Do directions.  Key records (face-plane
// slots, boundary flags, cell, group) are built once per key, three tiles ahead, by
// the first keys_per_cta threads; the sources and opacities and every row's inflow
// faces are copied into shared memory (cp.async) two tiles ahead, so that a copy has
// two tile solves to arrive in.  Within one hyperplane every input is ready when the
// kernel starts (the faces were written by the previous hyperplane), so the prefetch
// distance is free; without it a tile waits about one global-memory latency.  The
// flux reduction of a tile runs at the start of the next iteration.
constexpr int kTileRecs = 8;   // key-record ring (>= prefetch distance + 3 live tiles)
constexpr int kMaxMoments = (SN_MAX_SCATTERING_ORDER + 1) * (SN_MAX_SCATTERING_ORDER + 1);
template <typename T>
struct GeTileSmem {
    uint32_t face, ks, sig, rec, red, net, yt, geo, total;
};
// Every stage written while an earlier tile may still be read has its own buffer
// (PRE + 1 copy stages for a prefetch distance of PRE tiles), so one barrier a tile
// suffices.  Network sweeps keep the octant's folded network after the stages.
// general cells: a key's staged mass matrix and folded streaming matrices (256 values,
// padded so that the keys of a warp fall in different banks)
constexpr int kGeoKey = 260;
template <typename T>
__host__ __device__ inline GeTileSmem<T> ge_tile_smem(int kpt, int rows, int pre, bool net, int K = 1, int Do = 0,
                                                      bool geo = false)
{
    const uint32_t stages = (uint32_t)pre + 1;
    GeTileSmem<T> m;
    m.face = 0;                                                         // stages x [rows][12] inflow faces
    m.ks = m.face + stages * rows * 12 * (uint32_t)sizeof(T);          // stages x [kpt][K][8] source moments
    m.sig = m.ks + stages * kpt * K * 8 * (uint32_t)sizeof(T);         // stages x [kpt] opacities
    m.rec = (m.sig + stages * kpt * (uint32_t)sizeof(T) + 15) & ~15u;  // 8 x [kpt] key records
    m.red = m.rec + kTileRecs * 32 * kpt;                              // 2 x [rows][8] w_d psi (canonical)
    m.net = m.red + 2 * rows * 8 * (uint32_t)sizeof(T);                // [288] folded network
    m.yt = m.net + (net ? (uint32_t)(sizeof(float) * kOnFold) : 0u);  // [Do][K] harmonics (K > 1)
    m.geo = (m.yt + (K > 1 ? (uint32_t)(Do * K * sizeof(T)) : 0u) + 15) & ~15u;   // 2 x [kpt][260] M, B
    m.total = m.geo + (geo ? 2u * kpt * kGeoKey * (uint32_t)sizeof(T) : 0u);
    return m;
}

// CTAs per SM of the network sweep, and its prefetch distance in tiles
#ifndef SN_NET_TILE_MINBLOCKS
#define SN_NET_TILE_MINBLOCKS 4
#endif
#ifndef SN_NET_PRE
#define SN_NET_PRE 1
#endif

template <typename T, bool NET>
constexpr int tile_min_blocks()
{
    return NET ? SN_NET_TILE_MINBLOCKS : (sizeof(T) == 4 ? SN_GE_TILE_MINBLOCKS : 1);
}

// NET: the per-cell solve is the paper's network of the CTA's octant (octnet.cuh,
// weights in shared memory, read as broadcasts) instead of elimination; everything
// else (staging, outflow, flux) is shared.  A network thread owns two rows (RPT = 2,
// rows t and t + blockDim) and evaluates both with one pass over the weights: the
// weight reads, not the arithmetic, bound a one-row network sweep.  PRE: tiles of
// copies in flight (the elimination hides one tile of copy latency behind its
// solve; a deeper prefetch measured no faster).
//
// MOM (anisotropic scattering, K = a.K moments): every key stages its K source moments,
// a row forms its direction's source sum_k Yh_k(Omega_d) Sh_k, and the reduction of a
// tile forms the K flux moments sum_d Yh_k(Omega_d) w_d psi_d of every key.
//
// GEOM (general hexahedral cells): each row assembles its cell's system (14) in the
// physical frame from the cell's element record (hex.cuh; the rows of a key read the
// same record, so the loads are broadcasts), with the canonical staged sources and
// inflow faces permuted back to physical order, solves it by elimination with partial
// pivoting (and one refinement step), and takes the boundary leakage from the outflow
// faces' own matrices.
template <typename T, bool REFINE, int DO, bool NET, bool MOM = false, bool GEOM = false>
__device__ __forceinline__ void ge_tiles_body(const SweepArgs<T> &a)
{
    constexpr int PRE = NET ? SN_NET_PRE : 1, STAGES = PRE + 1, RPT = NET ? 2 : 1;
    extern __shared__ __align__(16) unsigned char gsm[];
    griddep_launch();
    const int Do = DO ? DO : a.Do;
    const int KM = MOM ? a.K : 1;
    const int nthr = blockDim.x, kpt = a.keys_per_cta, rows = nthr * RPT;
    const GeTileSmem<T> L = ge_tile_smem<T>(kpt, rows, PRE, NET, KM, Do, GEOM);
    const uint32_t sb = smem_u32(gsm);
    const int t = threadIdx.x, o = blockIdx.y;
    int lk[RPT], dr[RPT];
    bool lane_row[RPT];
    DirData<T> dd[RPT];
    float amu[RPT], aeta[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = t + j * nthr;
        lk[j] = r / Do;
        dr[j] = r - lk[j] * Do;
        lane_row[j] = lk[j] < kpt;
        dd[j] = lane_row[j] ? a.dir[dr[j]] : DirData<T>{T(0), T(0), T(0), T(0)};
        amu[j] = aeta[j] = 0.f;
        if (NET && lane_row[j]) {
            const float4 ab = a.dir_abs[dr[j]];
            amu[j] = ab.x;
            aeta[j] = ab.y;
        }
    }
    const uint32_t nkeys = (uint32_t)a.ncells_plane * (uint32_t)a.G;
    float *wnet = reinterpret_cast<float *>(gsm + L.net);
    if (NET) {
        // the folded networks are written before the sweep's first hyperplane launch,
        // which is not overlapped with earlier work: safe to read before griddep_wait
        for (int e = t; e < kOnFold; e += nthr) wnet[e] = a.onet[kOnFold * o + e];
    }
    T *yt = reinterpret_cast<T *>(gsm + L.yt);
    if (MOM) {
        // the octant's harmonics table (written at set-up)
        for (int e = t; e < Do * KM; e += nthr) yt[e] = a.yhat[(int64_t)o * Do * KM + e];
    }
    auto red_at = [&](int buf) -> T * { return reinterpret_cast<T *>(gsm + L.red) + buf * rows * 8; };
    auto rec_at = [&](int slot, int k) -> unsigned char * { return gsm + L.rec + (slot * kpt + k) * 32; };
    const int psi_o[3] = {o & 1, 2 + ((o >> 1) & 1), 4 + ((o >> 2) & 1)};

    // key thread t: the record of key t of tile tl into ring slot `slot`
    auto key_pk = [&](int tl) -> uint32_t {
        const uint32_t key = (uint32_t)tl * (uint32_t)kpt + (uint32_t)t;
        return (tl < a.ntiles && key < nkeys) ? a.cells[a.divG.div(key)] : 0u;
    };
    auto key_rec = [&](int tl, uint32_t pk, int slot) {
        const uint32_t key = (uint32_t)tl * (uint32_t)kpt + (uint32_t)t;
        KeyRec r;
        if (tl < a.ntiles && key < nkeys) {
            make_key<DO>(a, o, key, pk, r);
        } else {
            r.bx = r.by = r.bz = 0; r.flags = 0; r.cell = r.g = 0; r.pad0 = r.pad1 = 0;
        }
        put_key(rec_at(slot, t), r);
    };
    // key thread t: copy the source and opacity of its key (record in `slot`) into
    // stage buffer `sbuf`
    auto key_copy = [&](int slot, int sbuf) {
        const KeyRec r = get_key(rec_at(slot, t));
        if (!(r.flags & 0x80u)) return;
        const int64_t gc = (int64_t)r.g * a.C + r.cell;
        const uint32_t k = (uint32_t)(sbuf * kpt + t);
        if (MOM) {
            // source moments ([G][K][C][8] layout) as whole 16-byte pieces, in physical
            // node order (the row reads node n of the canonical frame at n ^ o)
            for (int m = 0; m < KM; ++m) {
                const uint32_t dst = sb + L.ks + (k * KM + m) * 8 * (uint32_t)sizeof(T);
                const T *src = a.S + (((int64_t)r.g * KM + m) * a.C + r.cell) * 8;
                cp_async_bytes(dst, src, 8 * (int)sizeof(T));
            }
        } else {
            // node by node into the canonical order of the octant (canonical n = physical n ^ o)
            const uint32_t dst = sb + L.ks + k * 8 * (uint32_t)sizeof(T);
            const T *src = a.S + gc * 8;
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                if (sizeof(T) == 4) cp_async4(dst + 4 * (p ^ o), src + p);
                else cp_async8(dst + 8 * (p ^ o), src + p);
            }
        }
        if (sizeof(T) == 4) cp_async4(sb + L.sig + 4 * k, a.sigt + gc);
        else cp_async8(sb + L.sig + 8 * k, a.sigt + gc);
    };
    // the thread's rows: copy their inflow faces (records in `slot`) into face buffer `fb`
    auto face_copy = [&](int slot, int fb) {
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            if (!lane_row[j]) continue;
            const KeyRec r = get_key(rec_at(slot, lk[j]));
            if (!(r.flags & 0x80u)) continue;
            const uint32_t dst = sb + L.face + (uint32_t)((fb * rows + t + j * nthr) * 12 * (int)sizeof(T));
            constexpr int vb = 4 * (int)sizeof(T);
            if (!(r.flags & 1u)) cp_async_bytes(dst, a.fx + r.bx + dr[j], vb);
            if (!(r.flags & 2u)) cp_async_bytes(dst + vb, a.fy + r.by + dr[j], vb);
            if (!(r.flags & 4u)) cp_async_bytes(dst + 2 * vb, a.fz + r.bz + dr[j], vb);
        }
    };
    // GEOM: every key's mass matrix and its octant's folded streaming matrices (records
    // in `slot`) into geometry stage `gb`, 16-byte pieces spread over the whole CTA
    auto geo_copy = [&](int slot, int gb) {
        if (!GEOM) return;
        constexpr int per = 16 / (int)sizeof(T);   // values a 16-byte piece
        const int npiece = 256 / per;
        for (int c = t; c < kpt * npiece; c += nthr) {
            const int kk = c / npiece, pc = c - kk * npiece;
            const KeyRec r = get_key(rec_at(slot, kk));
            if (!(r.flags & 0x80u)) continue;
            const int v = pc * per;   // value index within [M (64) | B (192)]
            const T *src = v < 64 ? a.geom + (int64_t)r.cell * kHexRec + kHexM + v
                                  : a.geomB + ((int64_t)r.cell * 8 + o) * kHexB + (v - 64);
            cp_async16(sb + L.geo + (uint32_t)(((gb * kpt + kk) * kGeoKey + v) * (int)sizeof(T)), src);
        }
    };
    // flux partial of the tile whose records are in `slot` and w_d psi in red buffer `rb`
    auto reduce_tile = [&](int slot, int rb) {
        const T *red = red_at(rb);
        if (MOM) {
            // one thread per (key, node): every flux moment of that node, each w_d psi_d
            // read once
            for (int e = t; e < 8 * kpt; e += nthr) {
                const int kk = e >> 3, n = e & 7;
                const KeyRec r = get_key(rec_at(slot, kk));
                if (!(r.flags & 0x80u)) continue;
                const T *base = red + (kk * Do) * 8 + (n ^ o);
                T acc[kMaxMoments];
#pragma unroll
                for (int m = 0; m < kMaxMoments; ++m) acc[m] = T(0);
                for (int q = 0; q < Do; ++q) {
                    const T v = base[q * 8];
                    const T *y = yt + q * KM;
#pragma unroll
                    for (int m = 0; m < kMaxMoments; ++m)
                        if (m < KM) acc[m] = fma(y[m], v, acc[m]);
                }
                T *dst = a.phi_oct + (((int64_t)o * a.C + r.cell) * a.G + r.g) * KM * 8 + n;
#pragma unroll
                for (int m = 0; m < kMaxMoments; ++m)
                    if (m < KM) dst[m * 8] = acc[m];
            }
            return;
        }
        for (int e = t; e < 8 * kpt; e += nthr) {
            const int kk = e >> 3, n = e & 7;
            const KeyRec r = get_key(rec_at(slot, kk));
            if (!(r.flags & 0x80u)) continue;
            const T *base = red + (kk * Do) * 8 + (n ^ o);   // rows hold canonical order
            T sum = T(0);
            if (DO) {
#pragma unroll
                for (int q = 0; q < DO; ++q) sum += base[q * 8];
            } else {
                for (int q = 0; q < Do; ++q) sum += base[q * 8];
            }
            a.phi_oct[(((int64_t)o * a.C + r.cell) * a.G + r.g) * 8 + n] = sum;
        }
    };
    // row j's solution x: outflow faces (or boundary leakage) and w_d psi
    T leak[RPT];
    T leak_exact = T(0);   // GEOM: boundary leakage already weighted by w_d
#pragma unroll
    for (int j = 0; j < RPT; ++j) leak[j] = T(0);
    auto emit = [&](int j, const KeyRec &kr, const T (&x)[8], int i) {
        const int d = dr[j];
        if (!(kr.flags & 8u)) store4(a.fx + kr.bx + d, x[1], x[3], x[5], x[7]);
        else if (!GEOM) leak[j] += dd[j].t3x * (x[1] + x[3] + x[5] + x[7]);
        if (!(kr.flags & 16u)) store4(a.fy + kr.by + d, x[2], x[3], x[6], x[7]);
        else if (!GEOM) leak[j] += dd[j].t3y * (x[2] + x[3] + x[6] + x[7]);
        if (!(kr.flags & 32u)) store4(a.fz + kr.bz + d, x[4], x[5], x[6], x[7]);
        else if (!GEOM) leak[j] += dd[j].t3z * (x[4] + x[5] + x[6] + x[7]);
        const T w = dd[j].w;
        T *r = red_at(i & 1) + (t + j * nthr) * 8;
        store4(reinterpret_cast<Vec4<T> *>(r), w * x[0], w * x[1], w * x[2], w * x[3]);
        store4(reinterpret_cast<Vec4<T> *>(r) + 1, w * x[4], w * x[5], w * x[6], w * x[7]);
    };

    // Tile i of this CTA is tile t0 + i * step of the hyperplane.  Its key record sits
    // in ring slot i % 8 and its copies in stage buffer i % STAGES.  Iteration i waits
    // for tile i's copies (issued in iteration i - PRE), reduces tile i - 1, issues
    // tile i + PRE's copies and tile i + PRE + 1's records, and solves tile i.
    const int t0 = blockIdx.x, step = gridDim.x;
    auto tile_of = [&](int i) { return t0 + i * step; };
    // the first PRE + 1 tiles' key records need only the hyperplane's cell table
    // (written once at set-up): they are built while the previous hyperplane may run
    uint32_t pk_next = 0;
    if (t < kpt) {
#pragma unroll
        for (int j = 0; j <= PRE; ++j) key_rec(tile_of(j), key_pk(tile_of(j)), j);
        pk_next = key_pk(tile_of(PRE + 1));
    }
    __syncthreads();
    if (NET && t < kOnHid) {
        // the uniform cell size enters every cell the same way: fold it into the bias
        // (visible after the first barrier of the tile loop)
        float *wk = wnet + 24 * t;
        wk[23] = fmaf(wnet[kOnFoldH + 3 * t], (float)a.hx,
                      fmaf(wnet[kOnFoldH + 3 * t + 1], (float)a.hy, fmaf(wnet[kOnFoldH + 3 * t + 2], (float)a.hz, wk[23])));
    }
    griddep_wait();
#pragma unroll
    for (int j = 0; j < PRE; ++j) {
        if (t < kpt) key_copy(j, j);
        face_copy(j, j);
        geo_copy(j, j);
        cp_async_commit();
    }
    int i = 0;
    for (int tile = t0; tile < a.ntiles; tile += step, ++i) {
        const int slot = i % kTileRecs, cur = i % STAGES;
        // cell of this thread's key PRE + 2 tiles ahead (used in the next iteration)
        const uint32_t pk_ahead = t < kpt ? key_pk(tile_of(i + PRE + 2)) : 0u;
        cp_async_wait_pending<PRE - 1>();
        __syncthreads();
        // the only barrier of the tile: tile i's stage is complete, and every buffer
        // written below was last read before it
        if (i > 0) reduce_tile((i - 1) % kTileRecs, (i - 1) & 1);
        const int pre = (i + PRE) % STAGES;
        face_copy((i + PRE) % kTileRecs, pre);
        geo_copy((i + PRE) % kTileRecs, pre);
        if (t < kpt) {
            key_rec(tile_of(i + PRE + 1), pk_next, (i + PRE + 1) % kTileRecs);
            key_copy((i + PRE) % kTileRecs, pre);
        }
        pk_next = pk_ahead;
        cp_async_commit();
        // this tile's inputs from the stage: inflow faces (or psi_inc on the boundary),
        // sources and opacity of each of the thread's rows
        KeyRec kr[RPT];
        bool act[RPT];
        T S[RPT][8], ux[RPT][4], uy[RPT][4], uz[RPT][4], sig[RPT];
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            kr[j] = get_key(rec_at(slot, lane_row[j] ? lk[j] : 0));
            act[j] = lane_row[j] && (kr[j].flags & 0x80u);
            const int kj = act[j] ? lk[j] : 0;
            const T *ff = reinterpret_cast<const T *>(gsm + L.face) + (cur * rows + t + j * nthr) * 12;
            const T *fks = reinterpret_cast<const T *>(gsm + L.ks) + (cur * kpt + kj) * KM * 8;
            sig[j] = reinterpret_cast<const T *>(gsm + L.sig)[cur * kpt + kj];
            const T *pi = a.psi_inc + 6 * kr[j].g;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ux[j][q] = (kr[j].flags & 1u) ? pi[psi_o[0]] : ff[q];
                uy[j][q] = (kr[j].flags & 2u) ? pi[psi_o[1]] : ff[4 + q];
                uz[j][q] = (kr[j].flags & 4u) ? pi[psi_o[2]] : ff[8 + q];
            }
            if (MOM) {
                // this direction's source from the key's source moments
                const T *y = yt + dr[j] * KM;
#pragma unroll
                for (int q = 0; q < 8; ++q) S[j][q] = T(0);
#pragma unroll
                for (int m = 0; m < kMaxMoments; ++m) {
                    if (m < KM) {
                        const T ym = y[m];
#pragma unroll
                        for (int q = 0; q < 8; ++q) S[j][q] = fma(ym, fks[m * 8 + (q ^ o)], S[j][q]);
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) S[j][q] = fks[q];
            }
        }
        if constexpr (NET) {
            // both rows through the network in one pass over its weights (an idle row
            // is evaluated on whatever its stage holds and not emitted)
            float x[RPT][8];
            octnet_forward2(wnet, ux, uy, uz, S, amu, aeta, sig, x);
#pragma unroll
            for (int j = 0; j < RPT; ++j)
                if (act[j]) emit(j, kr[j], x[j], i);
        } else if constexpr (GEOM) {
            if (act[0]) {
                const T *gc = a.geom + (int64_t)kr[0].cell * kHexRec;
                const int fx = o & 1, fy = (o >> 1) & 1, fz = (o >> 2) & 1;
                const T *oa = a.omabs + 3 * dr[0];
                const T om[3] = {fx ? -oa[0] : oa[0], fy ? -oa[1] : oa[1], fz ? -oa[2] : oa[2]};
                const int out[3] = {1 - fx, 1 - fy, 1 - fz};   // outflow side of each axis
                // physical order: node n = canonical n ^ o; face value t = canonical t ^ face mask
                T Sp[8], upx[4], upy[4], upz[4];
#pragma unroll
                for (int q = 0; q < 8; ++q) Sp[q] = S[0][q];
                mirror8(Sp, o);
#pragma unroll
                for (int t4 = 0; t4 < 4; ++t4) { upx[t4] = ux[0][t4]; upy[t4] = uy[0][t4]; upz[t4] = uz[0][t4]; }
                mirror4(upx, fy | (fz << 1));
                mirror4(upy, fx | (fz << 1));
                mirror4(upz, fx | (fy << 1));
                T A[8][8], b[8], b0[8], rinv[8], xp[8];
                // the key's staged mass matrix and folded streaming matrices
                const T *Mk = reinterpret_cast<const T *>(gsm + L.geo) + (cur * kpt + lk[0]) * kGeoKey;
                const T *Bk = Mk + 64;
                hex_assemble_A(Mk, Bk, om, sig[0], A);
                hex_build_b(gc, Mk, om, out, Sp, upx, upy, upz, b);
#pragma unroll
                for (int q = 0; q < 8; ++q) b0[q] = b[q];
                unsigned piv;
                ge8_factor_solve(A, b, piv, rinv, xp);
                if (REFINE) {
                    T y[8], r[8], dx[8];
                    hex_apply_A(Mk, Bk, om, sig[0], xp, y);
#pragma unroll
                    for (int q = 0; q < 8; ++q) r[q] = b0[q] - y[q];
                    ge8_replay(A, piv, rinv, r, dx);
#pragma unroll
                    for (int q = 0; q < 8; ++q) xp[q] += dx[q];
                }
                if (kr[0].flags & 8u) leak_exact += dd[0].w * hex_out_flux<T, 0>(gc, om, out[0], xp);
                if (kr[0].flags & 16u) leak_exact += dd[0].w * hex_out_flux<T, 1>(gc, om, out[1], xp);
                if (kr[0].flags & 32u) leak_exact += dd[0].w * hex_out_flux<T, 2>(gc, om, out[2], xp);
                T x[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = xp[q];
                mirror8(x, o);
                emit(0, kr[0], x, i);
            }
        } else {
            if (act[0]) {
                T x[8];
                cell_solve_canonical<T, REFINE>(dd[0].t3x, dd[0].t3y, dd[0].t3z, sig[0], S[0], ux[0], uy[0], uz[0],
                                                x);
                emit(0, kr[0], x, i);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (i > 0) reduce_tile((i - 1) % kTileRecs, (i - 1) & 1);
    T lsum = T(0);
#pragma unroll
    for (int j = 0; j < RPT; ++j) lsum += leak[j] * dd[j].w;
    lsum *= a.vol12;
    lsum += leak_exact;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
    if ((t & 31) == 0 && lsum != T(0)) atomicAdd(a.leak, (double)lsum);
}

template <typename T, bool REFINE, int DO>
__global__ void __launch_bounds__(SN_GE_BLOCK, (tile_min_blocks<T, false>())) sweep_ge_tiles(SweepArgs<T> a)
{
    ge_tiles_body<T, REFINE, DO, false>(a);
}

template <typename T, bool REFINE>
__global__ void __launch_bounds__(SN_GE_BLOCK, (tile_min_blocks<T, false>())) sweep_ge_moments(SweepArgs<T> a)
{
    ge_tiles_body<T, REFINE, 0, false, true>(a);
}

// CTAs per SM of the general-cell sweep.  With the matrices staged in shared memory
// (49 KB a CTA), 4 CTAs (128 registers) leave little of the unified array to L1 for
// their spills (796 bytes a thread); 3 (168 registers, 268 bytes of spill) measured
// 9% faster on deformed blocked_64 (29.6 against 32.4 ms a step), 2 (254 registers, no
// spills) slower than either
#ifndef SN_GEOM_MINBLOCKS
#define SN_GEOM_MINBLOCKS 3
#endif
template <typename T, bool REFINE>
__global__ void __launch_bounds__(SN_GE_BLOCK, (sizeof(T) == 4 ? SN_GEOM_MINBLOCKS : 1)) sweep_ge_hex(SweepArgs<T> a)
{
    ge_tiles_body<T, REFINE, 0, false, false, true>(a);
}

template <int DO>
__global__ void __launch_bounds__(SN_GE_BLOCK, SN_NET_TILE_MINBLOCKS) sweep_net_tiles(SweepArgs<float> a)
{
    ge_tiles_body<float, false, DO, true>(a);
}

// shared memory of an elimination sweep tile of this handle with K moments
uint32_t sweep_smem_bytes(sn_handle h, int K)
{
    const int kpt = SN_GE_BLOCK / h->Do;
    return h->fp64 ? ge_tile_smem<double>(kpt, SN_GE_BLOCK, 1, false, K, h->Do).total
                   : ge_tile_smem<float>(kpt, SN_GE_BLOCK, 1, false, K, h->Do).total;
}

// Hyperplane launches of a network sweep (the folded networks of the handle).
static sn_status launch_sweep_net(sn_handle h, SweepArgs<float> &a, uint32_t smem, cudaStream_t st)
{
    a.onet = octnet_folded(h);
    if (!a.onet) return fail(h, SN_ESTATE, "octant-network sweep without networks");
    void (*kern)(SweepArgs<float>) =
        h->Do == 10 ? sweep_net_tiles<10> : h->Do == 21 ? sweep_net_tiles<21> : sweep_net_tiles<0>;
    if (smem > 48 * 1024)
        SN_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int cap = std::max(1, num_sms() * SN_NET_TILE_MINBLOCKS / 8);
    if (h->prof) SN_CK(h, cudaEventRecord(h->ev_sweep[0], st));
    for (int s = 0; s < h->nplanes; ++s) {
        const int64_t n = h->plane_off[s + 1] - h->plane_off[s];
        a.cells = h->plane_cells + h->plane_off[s];
        a.ncells_plane = (int)n;
        a.ntiles = (int)((n * h->G + a.keys_per_cta - 1) / a.keys_per_cta);
        const dim3 grid((unsigned)std::min(a.ntiles, cap), 8);
        SN_CK(h, launch_k(s > 0, kern, grid, dim3(SN_GE_BLOCK), smem, st, a));
    }
    SN_CK(h, cudaGetLastError());
    if (h->prof) {
        SN_CK(h, cudaEventRecord(h->ev_sweep[1], st));
        h->prof_pending = true;
    }
    return SN_OK;
}

template <typename T>
static sn_status launch_sweep_t(sn_handle h, const T *S, T *phi_oct, bool refine, bool net, cudaStream_t st)
{
    SweepArgs<T> a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.G = h->G; a.Do = h->Do; a.C = (int)h->ncell;
    a.divG = FastDiv((uint32_t)h->G);
    a.keys_per_cta = SN_GE_BLOCK / h->Do;
    a.sigt = (const T *)h->sigt; a.S = S; a.psi_inc = (const T *)h->psi_inc;
    a.dir = (const DirData<T> *)h->dir;
    a.fx = (Vec4<T> *)h->face;
    a.fy = a.fx + h->face_x;
    a.fz = a.fy + h->face_y;
    a.phi_oct = phi_oct;
    a.leak = h->acc + ACC_LEAK;
    a.vol12 = (T)(h->dx * h->dy * h->dz / 12.0);
    a.dir_abs = h->dir_abs;
    a.hx = (T)h->dx; a.hy = (T)h->dy; a.hz = (T)h->dz;
    const int rows = SN_GE_BLOCK;
    if constexpr (sizeof(T) == 4) {
        if (net) {
            a.K = 1;
            a.yhat = nullptr;
            // two rows a thread; every key needs a key thread (at most one key a thread)
            a.keys_per_cta = std::min(2 * SN_GE_BLOCK / h->Do, SN_GE_BLOCK);
            return launch_sweep_net(h, a, ge_tile_smem<T>(a.keys_per_cta, 2 * rows, SN_NET_PRE, true).total, st);
        }
    }
    a.K = h->K;
    a.yhat = (const T *)h->yhat;
    a.geom = (const T *)h->geom;
    a.omabs = (const T *)h->omabs;
    a.geomB = (const T *)h->geomB;
    // general cells stage 1 KB (FP32) of matrices a key: at most 24 keys a tile
    if (h->geom) a.keys_per_cta = std::min(a.keys_per_cta, 24);
    const uint32_t smem = ge_tile_smem<T>(a.keys_per_cta, rows, 1, false, h->K, h->Do, h->geom != nullptr).total;
    void (*kern)(SweepArgs<T>) = nullptr;
    if (h->geom)
        kern = refine ? sweep_ge_hex<T, true> : sweep_ge_hex<T, false>;
    else if (h->K > 1)
        kern = refine ? sweep_ge_moments<T, true> : sweep_ge_moments<T, false>;
    else if (refine)
        kern = h->Do == 10 ? sweep_ge_tiles<T, true, 10> : h->Do == 21 ? sweep_ge_tiles<T, true, 21>
                                                                     : sweep_ge_tiles<T, true, 0>;
    else
        kern = h->Do == 10 ? sweep_ge_tiles<T, false, 10> : h->Do == 21 ? sweep_ge_tiles<T, false, 21>
                                                                      : sweep_ge_tiles<T, false, 0>;
    if (smem > 48 * 1024)
        SN_CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // persistent CTAs per octant: the register-limited residency (4 a SM in FP32, 1 in FP64)
    const int per_sm = sizeof(T) != 4 ? 1 : (h->geom ? SN_GEOM_MINBLOCKS : SN_GE_TILE_MINBLOCKS);
    const int cap = std::max(1, num_sms() * per_sm / 8);
    if (h->prof) SN_CK(h, cudaEventRecord(h->ev_sweep[0], st));
    for (int s = 0; s < h->nplanes; ++s) {
        const int64_t n = h->plane_off[s + 1] - h->plane_off[s];
        a.cells = h->plane_cells + h->plane_off[s];
        a.ncells_plane = (int)n;
        a.ntiles = (int)((n * h->G + a.keys_per_cta - 1) / a.keys_per_cta);
        const dim3 grid((unsigned)std::min(a.ntiles, cap), 8);
        // hyperplanes after the first overlap their launch with the previous one's drain
        SN_CK(h, launch_k(s > 0, kern, grid, dim3(rows), smem, st, a));
    }
    SN_CK(h, cudaGetLastError());
    if (h->prof) {
        SN_CK(h, cudaEventRecord(h->ev_sweep[1], st));
        h->prof_pending = true;
    }
    return SN_OK;
}

// Hyperplanes [s0, s1) of an FP32 GE32R sweep in an adjoint pass mode (see sn_adjoint.cu).
sn_status launch_planes_adjoint(sn_handle h, const AdjPass &p, int s0, int s1, cudaStream_t st)
{
    SweepArgs<float> a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.G = h->G; a.Do = h->Do; a.C = (int)h->ncell;
    a.divG = FastDiv((uint32_t)h->G);
    a.keys_per_cta = SN_GE_BLOCK / h->Do;
    a.sigt = (const float *)h->sigt; a.S = p.S; a.psi_inc = p.psi_inc;
    a.dir = (const DirData<float> *)h->dir;
    a.fx = reinterpret_cast<Vec4<float> *>(p.face);
    a.fy = a.fx + h->face_x;
    a.fz = a.fy + h->face_y;
    a.phi_oct = p.phi_oct;
    a.leak = p.leak;
    a.vol12 = (float)(h->dx * h->dy * h->dz / 12.0);
    a.vol216 = (float)(h->dx * h->dy * h->dz / 216.0);
    a.psi_blk = reinterpret_cast<Vec4<float> *>(p.psi_blk);
    a.plane_pos = h->plane_pos;
    a.grad = p.grad;
    const int block = (a.keys_per_cta * h->Do + 31) / 32 * 32;
    const size_t smem = sizeof(float) * 9 * block;
    for (int s = s0; s < s1; ++s) {
        const int64_t n = h->plane_off[s + 1] - h->plane_off[s];
        a.cells = h->plane_cells + h->plane_off[s];
        a.ncells_plane = (int)n;
        a.blk_base = p.mode == 1 ? (uint32_t)(h->plane_off[s] - p.blk_cell0) : 0u;
        if (p.mode == 2) {
            const int sf = h->nplanes - 1 - s;
            a.pair_base = (uint32_t)(h->plane_off[sf] - p.blk_cell0);
        }
        const int64_t nkeys = n * h->G;
        const dim3 grid((unsigned)((nkeys + a.keys_per_cta - 1) / a.keys_per_cta), 8);
        if (p.mode == 1)
            sweep_plane_ge<float, true, 1><<<grid, block, smem, st>>>(a);
        else if (p.mode == 2)
            sweep_plane_ge<float, true, 2><<<grid, block, smem, st>>>(a);
        else
            sweep_plane_ge<float, true, 0><<<grid, block, smem, st>>>(a);
    }
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

// One GE32R sweep from S that also writes about `cap` randomly chosen solves as
// canonical one-cell problems (the positive-octant frame is itself a valid physical
// problem: Omega = |Omega|, node order as stored).
static sn_status launch_harvest(sn_handle h, const float *S, float *out, uint32_t cap, uint64_t seed,
                                unsigned long long *count, cudaStream_t st)
{
    SweepArgs<float> a;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.G = h->G; a.Do = h->Do; a.C = (int)h->ncell;
    a.divG = FastDiv((uint32_t)h->G);
    a.keys_per_cta = SN_GE_BLOCK / h->Do;
    a.sigt = (const float *)h->sigt; a.S = S; a.psi_inc = (const float *)h->psi_inc;
    a.dir = (const DirData<float> *)h->dir;
    a.fx = reinterpret_cast<Vec4<float> *>(h->face);
    a.fy = a.fx + h->face_x;
    a.fz = a.fy + h->face_y;
    a.phi_oct = (float *)h->phi_oct;
    a.leak = h->acc + ACC_LEAK;
    a.vol12 = (float)(h->dx * h->dy * h->dz / 12.0);
    a.harvest = out;
    a.harvest_count = count;
    a.harvest_cap = cap;
    const double total = (double)h->ncell * h->ndir * h->G;
    const double p = std::min(1.0, 1.05 * cap / total);
    a.harvest_threshold = (uint32_t)std::min(4294967295.0, p * 4294967296.0);
    a.harvest_seed = (uint32_t)(seed ^ (seed >> 32));
    a.dir_abs = h->dir_abs;
    a.hx = (float)h->dx; a.hy = (float)h->dy; a.hz = (float)h->dz;
    const int block = (a.keys_per_cta * h->Do + 31) / 32 * 32;
    const size_t smem = sizeof(float) * 9 * block;
    for (int s = 0; s < h->nplanes; ++s) {
        const int64_t n = h->plane_off[s + 1] - h->plane_off[s];
        a.cells = h->plane_cells + h->plane_off[s];
        a.ncells_plane = (int)n;
        a.plane = (uint32_t)s;
        const int64_t nkeys = n * h->G;
        const dim3 grid((unsigned)((nkeys + a.keys_per_cta - 1) / a.keys_per_cta), 8);
        sweep_plane_ge<float, true, 3><<<grid, block, smem, st>>>(a);
    }
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

sn_status launch_sweep(sn_handle h, const void *S, void *phi_oct, sn_solve_mode mode, cudaStream_t st)
{
    if (h->fp64) return launch_sweep_t<double>(h, (const double *)S, (double *)phi_oct, false, false, st);
    if (mode == SN_SOLVE_ANN || mode == SN_SOLVE_ANN_GATED || mode == SN_SOLVE_ANN_FROZEN)
        return launch_sweep_ann(h, (const float *)S, (float *)phi_oct,
                                mode == SN_SOLVE_ANN ? 0 : (mode == SN_SOLVE_ANN_GATED ? 1 : 2), st);
    if ((mode == SN_SOLVE_GE32R || mode == SN_SOLVE_GE32) && key_sweep_ok(h))
        return launch_sweep_keys(h, (const float *)S, (float *)phi_oct, mode == SN_SOLVE_GE32R, st);
    if (mode == SN_SOLVE_OCTNET && key_sweep_ok(h) && h->wave)
        return launch_sweep_net_keys(h, (const float *)S, (float *)phi_oct, st);
    return launch_sweep_t<float>(h, (const float *)S, (float *)phi_oct, mode == SN_SOLVE_GE32R,
                                 mode == SN_SOLVE_OCTNET, st);
}

// After a stream synchronisation: add the time between the sweep's first and last
// kernel to the profile.
static void prof_collect(sn_handle h)
{
    if (!h->prof || !h->prof_pending) return;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_sweep[0], h->ev_sweep[1]) == cudaSuccess) {
        h->prof_ms += ms;
        h->prof_sweeps += 1;
    } else {
        (void)cudaGetLastError();   // do not leave the failure for the next launch check
    }
    h->prof_pending = false;
}

// ---------------------------------------------------------------------------------
// Octant sum, balance tallies and (optionally) the change measures of the source
// iteration, FP64 accumulation (Eq. (21) for the mean form).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_nonneg(double *p, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(v));
}

// Tiled over cells: a block takes TC whole cells (all groups, all nodes), sums the
// eight octant partials in the layout the sweep writes them ([o][c][g][8], one
// contiguous run per octant), transposes the tile through shared memory and writes
// the scalar flux in its [g][c][8] layout (one contiguous run per group), so that
// both sides move whole lines.  Octant sum in the element type (fixed order), per-
// element quantities in the element type, FP64 only for the running sums and the
// block / grid accumulation (the FP64 rate of the part is low).
//
// With K flux moments (anisotropic scattering) the partials are [o][c][g][k][8] and the
// flux [g][k][c][8]: the same transposition with G * K "groups"; the tallies and the
// change measures use moment 0 (the scalar flux) only.
template <typename T>
__global__ void __launch_bounds__(256) reduce_kernel(const T *__restrict__ phi_oct, const T *__restrict__ phi_old,
                                                     T *__restrict__ phi_new, const T *__restrict__ S,
                                                     const T *__restrict__ sigt, int64_t C, int G, int TC,
                                                     FastDiv divG8, double vol8, double *acc, int norms, int K,
                                                     const T *__restrict__ vnode)
{
    extern __shared__ __align__(16) unsigned char red_smem[];
    T *tile = reinterpret_cast<T *>(red_smem);   // [TC][G*8 + 8] (padded row per cell)
    __shared__ double sh[8][6];
    const int G8 = G * 8, row = G8 + 8;
    const int64_t stride_oct = C * G8;
    const int64_t ntile = (C + TC - 1) / TC;
    const int lane = threadIdx.x % 32;
    double coll = 0, src = 0, mean = 0, cnt = 0;
    T dmax = T(0), pmax = T(0);
    int bad = 0;
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int64_t c0 = t * TC;
        const int nc = (int)min((int64_t)TC, C - c0);
        const int nel = nc * G8;
        const T *po = phi_oct + c0 * G8;
        // 16-byte loads (4 floats or 2 doubles of one cell: G*8 is a multiple of 8);
        // the same fixed octant order per value
        constexpr int V = 16 / (int)sizeof(T);
        for (int i = threadIdx.x * V; i < nel; i += blockDim.x * V) {
            T s[V];
#pragma unroll
            for (int j = 0; j < V; ++j) s[j] = T(0);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const T *src = po + (int64_t)o * stride_oct + i;
                if constexpr (V == 4) {
                    const float4 f = *reinterpret_cast<const float4 *>(src);
                    s[0] += f.x; s[1] += f.y; s[2] += f.z; s[3] += f.w;
                } else {
                    const double2 f = *reinterpret_cast<const double2 *>(src);
                    s[0] += f.x; s[1] += f.y;
                }
            }
            const int cl = (int)divG8.div((uint32_t)i);
            T *dst = tile + cl * row + (i - cl * G8);
#pragma unroll
            for (int j = 0; j < V; ++j) dst[j] = s[j];
        }
        __syncthreads();
        const int nk = nc * 8;
        // this tile's tallies in the element type, added to the FP64 sums once a tile
        // (the FP64 pipe of the GPU is a small fraction of the FP32 one)
        T coll_t = T(0), src_t = T(0), mean_t = T(0);
        int cnt_t = 0;
        for (int g = 0; g < G; ++g) {
            const int64_t base = ((int64_t)g * C + c0) * 8;
            const bool scalar = g % K == 0;   // moment 0 of its group
            const int gg = g / K;
            // whole warps, so that the 8 nodes of a cell meet in one shuffle group
            for (int k = threadIdx.x; k - lane < nk; k += blockDim.x) {
                const bool in = k < nk;
                T nv = T(0), ov = T(0);
                if (in) {
                    const int cl = k >> 3;
                    nv = tile[cl * row + g * 8 + (k & 7)];
                    phi_new[base + k] = nv;
                    if (!isfinite(nv)) bad = 1;
                    if (scalar) {
                        // general cells: the node's own volume (column sum of M)
                        const T wv = vnode ? vnode[(c0 + cl) * 8 + (k & 7)] : T(1);
                        coll_t = fma(sigt[(int64_t)gg * C + c0 + cl] * nv, wv, coll_t);
                        src_t = fma(S[base + k], wv, src_t);
                        if (norms) {
                            ov = phi_old[base + k];
                            dmax = fmax(dmax, fabs(nv - ov));
                            pmax = fmax(pmax, fabs(nv));
                        }
                    }
                }
                if (norms && scalar) {
                    T a = nv, b = ov;
#pragma unroll
                    for (int off = 1; off < 8; off <<= 1) {
                        a += __shfl_xor_sync(0xffffffffu, a, off);
                        b += __shfl_xor_sync(0xffffffffu, b, off);
                    }
                    if (in && (k & 7) == 0 && a != T(0)) {
                        mean_t += fabs(a - b) / fabs(a);
                        cnt_t += 1;
                    }
                }
            }
        }
        coll += (double)coll_t;
        src += (double)src_t;
        mean += (double)mean_t;
        cnt += (double)cnt_t;
        __syncthreads();
    }
    // block reduction
    double v[6] = {coll * vol8, src * 4.0 * kPi * vol8, (double)dmax, (double)pmax, mean, cnt};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const double t = __shfl_down_sync(0xffffffffu, v[m], off);
            v[m] = (m == 2 || m == 3) ? fmax(v[m], t) : v[m] + t;
        }
    }
    bad = __syncthreads_or(bad);
    const int warp = threadIdx.x / 32;
    if (lane == 0)
        for (int m = 0; m < 6; ++m) sh[warp][m] = v[m];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x / 32;
        for (int w = 1; w < nw; ++w)
            for (int m = 0; m < 6; ++m) v[m] = (m == 2 || m == 3) ? fmax(v[m], sh[w][m]) : v[m] + sh[w][m];
        atomicAdd(acc + ACC_COLL, v[0]);
        atomicAdd(acc + ACC_SRC, v[1]);
        if (norms) {
            atomic_max_nonneg(acc + ACC_DMAX, v[2]);
            atomic_max_nonneg(acc + ACC_PMAX, v[3]);
            atomicAdd(acc + ACC_MEAN, v[4]);
            atomicAdd(acc + ACC_MEANN, v[5]);
        }
        if (bad) acc[ACC_FLAG] = 1.0;
    }
}

// Isotropic scattering (one flux moment): the same octant sum and tallies over the
// same cell tiles, with the per-element work vectorised (each thread takes 16 bytes
// of one (group, cell): 4 nodes in FP32, 2 in FP64) and, with S_next, the source of
// the next iteration built from the new flux while the tile is in shared memory:
// S_next = (q_g + sum_g' xfer[g'][g] sigma_s,g' phi_g') / (4 pi) in the order and
// rounding of source_kernel (Eqs. (2) and (6), P_0 term), so the fused iteration gives
// the flux of the separate kernels bit for bit and saves one read and one write of it.
template <typename T>
__global__ void __launch_bounds__(256) reduce_iso_kernel(
    const T *__restrict__ phi_oct, const T *__restrict__ phi_old, T *__restrict__ phi_new, const T *__restrict__ S,
    T *__restrict__ S_next, const T *__restrict__ sigt, const T *__restrict__ sigs, const T *__restrict__ q,
    const T *__restrict__ xfer, const T *__restrict__ vnode, int64_t C, int G, int TC, FastDiv divG8, double vol8,
    double *acc, int norms)
{
    constexpr int V = 16 / (int)sizeof(T);   // elements a vector
    constexpr int NV = 8 / V;                // vectors of one (group, cell)
    using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    extern __shared__ __align__(16) unsigned char red_smem[];
    const int G8 = G * 8, row = G8 + 8;
    T *tile = reinterpret_cast<T *>(red_smem);   // [TC][G*8 + 8]
    T *st_sig = tile + (size_t)TC * row;         // [TC][G] sigma_t
    T *ss_sig = st_sig + (size_t)TC * G;         // [TC][G] sigma_s
    T *sq = ss_sig + (size_t)TC * G;             // [TC][G] q
    __shared__ double sh[8][6];
    const int64_t stride_oct = C * G8;
    const int64_t ntile = (C + TC - 1) / TC;
    const int lane = threadIdx.x % 32;
    const T inv4pi = (T)(1.0 / (4.0 * kPi));
    double coll = 0, src = 0, mean = 0, cnt = 0;
    T dmax = T(0), pmax = T(0);
    int bad = 0;
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int64_t c0 = t * TC;
        const int nc = (int)min((int64_t)TC, C - c0);
        const int nel = nc * G8;
        const T *po = phi_oct + c0 * G8;
        for (int i = threadIdx.x * V; i < nel; i += blockDim.x * V) {
            alignas(16) T s[V];
#pragma unroll
            for (int j = 0; j < V; ++j) s[j] = T(0);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const Vec f = *reinterpret_cast<const Vec *>(po + (int64_t)o * stride_oct + i);
                const T *fv = reinterpret_cast<const T *>(&f);
#pragma unroll
                for (int j = 0; j < V; ++j) s[j] += fv[j];
            }
            const int cl = (int)divG8.div((uint32_t)i);
            *reinterpret_cast<Vec *>(tile + cl * row + (i - cl * G8)) = *reinterpret_cast<const Vec *>(s);
        }
        for (int e = threadIdx.x; e < nc * G; e += blockDim.x) {
            const int g = e / nc, cl = e - g * nc;
            const int64_t gc = (int64_t)g * C + c0 + cl;
            st_sig[cl * G + g] = sigt[gc];
            ss_sig[cl * G + g] = sigs[gc];
            sq[cl * G + g] = q[gc];
        }
        __syncthreads();
        T coll_t = T(0), src_t = T(0), mean_t = T(0);
        int cnt_t = 0;
        const int per_g = nc * NV, total = G * per_g;
        // whole warps, so that the vectors of one (group, cell) meet in one shuffle group
        for (int e = threadIdx.x; e - lane < total; e += blockDim.x) {
            const bool in = e < total;
            T a = T(0), b = T(0);
            if (in) {
                const int g = e / per_g, r = e - g * per_g;
                const int cl = r / NV, v = r - cl * NV;
                const int64_t off = ((int64_t)g * C + c0 + cl) * 8 + v * V;
                alignas(16) T nv[V], sv[V], wv[V], ov[V];
                *reinterpret_cast<Vec *>(nv) = *reinterpret_cast<const Vec *>(tile + cl * row + g * 8 + v * V);
                *reinterpret_cast<Vec *>(phi_new + off) = *reinterpret_cast<const Vec *>(nv);
                *reinterpret_cast<Vec *>(sv) = *reinterpret_cast<const Vec *>(S + off);
                if (vnode) {
                    *reinterpret_cast<Vec *>(wv) = *reinterpret_cast<const Vec *>(vnode + (c0 + cl) * 8 + v * V);
                } else {
#pragma unroll
                    for (int j = 0; j < V; ++j) wv[j] = T(1);
                }
                const T sg = st_sig[cl * G + g];
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    if (!isfinite(nv[j])) bad = 1;
                    coll_t = fma(sg * nv[j], wv[j], coll_t);
                    src_t = fma(sv[j], wv[j], src_t);
                    a += nv[j];
                }
                if (norms) {
                    *reinterpret_cast<Vec *>(ov) = *reinterpret_cast<const Vec *>(phi_old + off);
#pragma unroll
                    for (int j = 0; j < V; ++j) {
                        dmax = fmax(dmax, fabs(nv[j] - ov[j]));
                        pmax = fmax(pmax, fabs(nv[j]));
                        b += ov[j];
                    }
                }
                if (S_next) {
                    alignas(16) T s[V];
                    const T qg = sq[cl * G + g];
#pragma unroll
                    for (int j = 0; j < V; ++j) s[j] = qg;
                    for (int gp = 0; gp < G; ++gp) {
                        const T x = __ldg(xfer + gp * G + g), sgs = ss_sig[cl * G + gp];
                        alignas(16) T pv[V];
                        *reinterpret_cast<Vec *>(pv) = *reinterpret_cast<const Vec *>(tile + cl * row + gp * 8 + v * V);
#pragma unroll
                        for (int j = 0; j < V; ++j) s[j] = fma(x, sgs * pv[j], s[j]);
                    }
#pragma unroll
                    for (int j = 0; j < V; ++j) s[j] *= inv4pi;
                    *reinterpret_cast<Vec *>(S_next + off) = *reinterpret_cast<const Vec *>(s);
                }
            }
            if (norms) {
#pragma unroll
                for (int m = 1; m < NV; m <<= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, m);
                    b += __shfl_xor_sync(0xffffffffu, b, m);
                }
                if (in && (e % NV) == 0 && a != T(0)) {
                    mean_t += fabs(a - b) / fabs(a);
                    cnt_t += 1;
                }
            }
        }
        coll += (double)coll_t;
        src += (double)src_t;
        mean += (double)mean_t;
        cnt += (double)cnt_t;
        __syncthreads();
    }
    double v[6] = {coll * vol8, src * 4.0 * kPi * vol8, (double)dmax, (double)pmax, mean, cnt};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const double t = __shfl_down_sync(0xffffffffu, v[m], off);
            v[m] = (m == 2 || m == 3) ? fmax(v[m], t) : v[m] + t;
        }
    }
    bad = __syncthreads_or(bad);
    const int warp = threadIdx.x / 32;
    if (lane == 0)
        for (int m = 0; m < 6; ++m) sh[warp][m] = v[m];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x / 32;
        for (int w = 1; w < nw; ++w)
            for (int m = 0; m < 6; ++m) v[m] = (m == 2 || m == 3) ? fmax(v[m], sh[w][m]) : v[m] + sh[w][m];
        atomicAdd(acc + ACC_COLL, v[0]);
        atomicAdd(acc + ACC_SRC, v[1]);
        if (norms) {
            atomic_max_nonneg(acc + ACC_DMAX, v[2]);
            atomic_max_nonneg(acc + ACC_PMAX, v[3]);
            atomicAdd(acc + ACC_MEAN, v[4]);
            atomicAdd(acc + ACC_MEANN, v[5]);
        }
        if (bad) acc[ACC_FLAG] = 1.0;
    }
}

int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0, m = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
        n = m > 0 ? m : 1;
    }
    return n;
}

static size_t reduce_tile(const sn_handle h, int *TC)
{
    // about 2048 elements a tile; a cell's G*K*8 values always stay in one tile
    const int G8 = h->G * h->K * 8;
    *TC = G8 >= 2048 ? 1 : 2048 / G8;
    return (size_t)*TC * (G8 + 8) * h->esz;
}

// the fused isotropic reduction: the same tile plus sigma_t, sigma_s and q of its cells
static size_t reduce_iso_smem(const sn_handle h, int TC)
{
    return (size_t)TC * (h->G * 8 + 8 + 3 * h->G) * h->esz;
}

// Opts the reductions in to more than 48 KB of dynamic shared memory where the group
// count needs it (G*8 values of one cell, up to 1024 groups); called once by sn_setup
// so that no attribute call falls inside a stream capture.
sn_status reduce_configure(sn_handle h)
{
    int TC = 0;
    const size_t smem = reduce_tile(h, &TC);
    const size_t smem_iso = reduce_iso_smem(h, TC);
    if (smem > 48 * 1024) {
        if (h->fp64)
            SN_CK(h, cudaFuncSetAttribute(reduce_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        else
            SN_CK(h, cudaFuncSetAttribute(reduce_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (h->K == 1) {
        if (smem_iso > 48 * 1024) {
            if (h->fp64)
                SN_CK(h, cudaFuncSetAttribute(reduce_iso_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem_iso));
            else
                SN_CK(h, cudaFuncSetAttribute(reduce_iso_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem_iso));
        }
        // a grid of resident blocks: the kernel strides over the cell tiles
        int per_sm = 0;
        if (h->fp64)
            SN_CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reduce_iso_kernel<double>, 256, smem_iso));
        else
            SN_CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reduce_iso_kernel<float>, 256, smem_iso));
        h->red_iso_per_sm = per_sm > 0 ? per_sm : 1;
    }
    return SN_OK;
}

static bool aligned16(const void *p)
{
    return ((uintptr_t)p & 15u) == 0;
}

sn_status launch_reduce(sn_handle h, const void *phi_old, void *phi_new, const void *S, void *S_next, bool norms,
                        cudaStream_t st)
{
    int TC = 0;
    const size_t smem = reduce_tile(h, &TC);
    const int64_t ntile = (h->ncell + TC - 1) / TC;
    int64_t grid = ntile;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (grid > cap) grid = cap;
    const double vol8 = h->vnode ? 1.0 : h->dx * h->dy * h->dz / 8.0;
    const FastDiv divG8((uint32_t)(h->G * h->K * 8));
    // the vectorised kernel moves 16 bytes of a caller's buffer at a time
    if (h->K == 1 && aligned16(phi_old) && aligned16(phi_new) && aligned16(S) && aligned16(S_next)) {
        const size_t si = reduce_iso_smem(h, TC);
        grid = std::min(ntile, (int64_t)num_sms() * h->red_iso_per_sm);
        if (h->fp64)
            reduce_iso_kernel<double><<<(unsigned)grid, 256, si, st>>>(
                (const double *)h->phi_oct, (const double *)phi_old, (double *)phi_new, (const double *)S,
                (double *)S_next, (const double *)h->sigt, (const double *)h->sigs, (const double *)h->q,
                (const double *)h->xfer, (const double *)h->vnode, h->ncell, h->G, TC, divG8, vol8, h->acc,
                norms ? 1 : 0);
        else
            reduce_iso_kernel<float><<<(unsigned)grid, 256, si, st>>>(
                (const float *)h->phi_oct, (const float *)phi_old, (float *)phi_new, (const float *)S,
                (float *)S_next, (const float *)h->sigt, (const float *)h->sigs, (const float *)h->q,
                (const float *)h->xfer, (const float *)h->vnode, h->ncell, h->G, TC, divG8, vol8, h->acc,
                norms ? 1 : 0);
        SN_CK(h, cudaGetLastError());
        return SN_OK;
    }
    if (h->fp64)
        reduce_kernel<double><<<(unsigned)grid, 256, smem, st>>>(
            (const double *)h->phi_oct, (const double *)phi_old, (double *)phi_new, (const double *)S,
            (const double *)h->sigt, h->ncell, h->G * h->K, TC, divG8, vol8, h->acc, norms ? 1 : 0, h->K,
            (const double *)h->vnode);
    else
        reduce_kernel<float><<<(unsigned)grid, 256, smem, st>>>(
            (const float *)h->phi_oct, (const float *)phi_old, (float *)phi_new, (const float *)S,
            (const float *)h->sigt, h->ncell, h->G * h->K, TC, divG8, vol8, h->acc, norms ? 1 : 0, h->K,
            (const float *)h->vnode);
    SN_CK(h, cudaGetLastError());
    return S_next ? launch_source(h, phi_new, S_next, st) : SN_OK;
}

// ---------------------------------------------------------------------------------
// Isotropic nodal source (Eqs. (2) and (6), P_0 term; scattering uses the mass
// matrix without sigma_t, the reading of the scattering term of (12)):
// S_g = (sum_g' xfer[g'][g] sigs_g' phi_g' + q_g) / (4 pi).
// One thread per (cell, node) computes every group; GMAX bounds the register copy.
// ---------------------------------------------------------------------------------
template <typename T, int GMAX>
__global__ void __launch_bounds__(256) source_kernel(const T *__restrict__ phi, const T *__restrict__ sigs,
                                                     const T *__restrict__ q, const T *__restrict__ xfer,
                                                     T *__restrict__ S, int64_t C, int G)
{
    const T inv4pi = (T)(1.0 / (4.0 * kPi));
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < C * 8;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e >> 3;
        T sv[GMAX];
#pragma unroll
        for (int gp = 0; gp < GMAX; ++gp)
            sv[gp] = gp < G ? sigs[(int64_t)gp * C + c] * phi[(int64_t)gp * C * 8 + e] : T(0);
#pragma unroll
        for (int g = 0; g < GMAX; ++g) {
            if (g >= G) break;
            T acc = q[(int64_t)g * C + c];
#pragma unroll
            for (int gp = 0; gp < GMAX; ++gp)
                if (gp < G) acc = fma(__ldg(xfer + gp * G + g), sv[gp], acc);
            S[(int64_t)g * C * 8 + e] = acc * inv4pi;
        }
    }
}

template <typename T>
__global__ void source_kernel_any(const T *__restrict__ phi, const T *__restrict__ sigs, const T *__restrict__ q,
                                  const T *__restrict__ xfer, T *__restrict__ S, int64_t C, int G)
{
    const T inv4pi = (T)(1.0 / (4.0 * kPi));
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)G * C * 8;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ce = e % (C * 8), c = ce >> 3;
        const int g = (int)(e / (C * 8));
        T acc = q[(int64_t)g * C + c];
        for (int gp = 0; gp < G; ++gp)
            acc = fma(xfer[gp * G + g], sigs[(int64_t)gp * C + c] * phi[(int64_t)gp * C * 8 + ce], acc);
        S[e] = acc * inv4pi;
    }
}

template <typename T>
static sn_status launch_source_t(sn_handle h, const T *phi, T *S, cudaStream_t st)
{
    const int64_t n = h->ncell * 8;
    int64_t grid = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (grid > cap) grid = cap;
    const unsigned gr = (unsigned)grid;
    const int G = h->G;
    const T *sg = (const T *)h->sigs, *q = (const T *)h->q, *xf = (const T *)h->xfer;
    if (G <= 1) source_kernel<T, 1><<<gr, 256, 0, st>>>(phi, sg, q, xf, S, h->ncell, G);
    else if (G <= 4) source_kernel<T, 4><<<gr, 256, 0, st>>>(phi, sg, q, xf, S, h->ncell, G);
    else if (G <= 8) source_kernel<T, 8><<<gr, 256, 0, st>>>(phi, sg, q, xf, S, h->ncell, G);
    else if (G <= 16) source_kernel<T, 16><<<gr, 256, 0, st>>>(phi, sg, q, xf, S, h->ncell, G);
    else source_kernel_any<T><<<(unsigned)(cap * 4), 256, 0, st>>>(phi, sg, q, xf, S, h->ncell, G);
    SN_CK(h, cudaGetLastError());
    return SN_OK;
}

sn_status launch_source(sn_handle h, const void *phi, void *S, cudaStream_t st)
{
    if (h->K > 1) return launch_source_moments(h, phi, S, st);
    if (h->fp64) return launch_source_t<double>(h, (const double *)phi, (double *)S, st);
    return launch_source_t<float>(h, (const float *)phi, (float *)S, st);
}

static sn_status check_mode(sn_handle h, sn_solve_mode mode)
{
    if (h->K > 1 && mode != SN_SOLVE_GE32R && mode != SN_SOLVE_GE32 && mode != SN_SOLVE_GE64)
        return fail(h, SN_EINVAL, "anisotropic scattering runs the elimination modes only");
    if (h->geom && mode != SN_SOLVE_GE32R && mode != SN_SOLVE_GE32 && mode != SN_SOLVE_GE64)
        return fail(h, SN_EINVAL, "general hexahedral cells run the elimination modes only");
    if (h->fp64) {
        if (mode == SN_SOLVE_GE64) return SN_OK;
        return fail(h, SN_EINVAL, "an FP64 handle only runs SN_SOLVE_GE64");
    }
    if (mode == SN_SOLVE_GE32R || mode == SN_SOLVE_GE32) return SN_OK;
    if (mode == SN_SOLVE_ANN || mode == SN_SOLVE_ANN_GATED) {
        if (!h->has_net) return fail(h, SN_ESTATE, "surrogate mode needs a trained or loaded network");
        return SN_OK;
    }
    if (mode == SN_SOLVE_ANN_FROZEN) {
        if (!h->has_net) return fail(h, SN_ESTATE, "surrogate mode needs a trained or loaded network");
        if (!ann_frozen(h))
            return fail(h, SN_ESTATE, "SN_SOLVE_ANN_FROZEN needs sn_surrogate_freeze_gate at the current weights "
                                      "and threshold");
        return SN_OK;
    }
    if (mode == SN_SOLVE_OCTNET) {
        if (!h->has_octnet) return fail(h, SN_ESTATE, "octant-network mode needs initialised or loaded networks");
        return SN_OK;
    }
    if (mode == SN_SOLVE_GE64) return fail(h, SN_EINVAL, "SN_SOLVE_GE64 needs an FP64 handle");
    return fail(h, SN_EINVAL, "unknown solve mode");
}

// one sweep from S into phi (device), tallies into acc; queued on st
static sn_status sweep_once(sn_handle h, const void *S, void *phi_out, const void *phi_old, sn_solve_mode mode,
                            cudaStream_t st, void *S_next = nullptr)
{
    SN_CK(h, cudaMemsetAsync(h->acc, 0, sizeof(double) * ACC_COUNT, st));
    if (mode == SN_SOLVE_ANN || mode == SN_SOLVE_ANN_GATED || mode == SN_SOLVE_ANN_FROZEN) {
        sn_status r = reset_ann_counters(h, st);
        if (r != SN_OK) return r;
    }
    sn_status s = launch_sweep(h, S, h->phi_oct, mode, st);
    if (s != SN_OK) return s;
    return launch_reduce(h, phi_old, phi_out, S, S_next, phi_old != nullptr, st);
}

static void take_tallies(sn_handle h)
{
    h->tallies[0] = h->acc_host[ACC_LEAK];
    h->tallies[1] = h->acc_host[ACC_COLL];
    h->tallies[2] = h->acc_host[ACC_SRC];
    h->tallies[3] = h->inflow;
    h->tallies_valid = true;
}

}  // namespace sn

using namespace sn;

extern "C" {

sn_status sn_sweep(sn_handle h, const void *S, void *phi, sn_solve_mode mode)
{
    if (!h || !S || !phi) return fail(h, SN_EINVAL, "sn_sweep: NULL argument");
    sn_status s = check_mode(h, mode);
    if (s != SN_OK) return s;
    const cudaStream_t st = h->stream;
    s = sweep_once(h, S, phi, nullptr, mode, st);
    if (s != SN_OK) return s;
    SN_CK(h, cudaMemcpyAsync(h->acc_host, h->acc, sizeof(double) * ACC_COUNT, cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    prof_collect(h);
    take_tallies(h);
    if (h->acc_host[ACC_ABORT] != 0.0) return fail(h, SN_ETIMEOUT, "sn_sweep: a bounded wait of the sweep gave up");
    if (mode == SN_SOLVE_ANN || mode == SN_SOLVE_ANN_GATED || mode == SN_SOLVE_ANN_FROZEN) return check_ann_timeouts(h);
    return SN_OK;
}

sn_status sn_source_iterate(sn_handle h, double tol, int32_t max_it, sn_solve_mode mode, void *phi,
                            int32_t *iters, double *change_max, double *change_mean, int32_t use_graph)
{
    if (!h || !phi) return fail(h, SN_EINVAL, "sn_source_iterate: NULL argument");
    if (max_it < 1 || !(tol >= 0.0)) return fail(h, SN_EINVAL, "sn_source_iterate: max_it >= 1, tol >= 0");
    sn_status s = check_mode(h, mode);
    if (s != SN_OK) return s;
    const cudaStream_t st = h->stream;
    void *buf[2] = {phi, h->phi_b};
    // one flux moment: the reduction of each sweep builds the next sweep's source into
    // the other source buffer, so only the first source is a launch of its own
    const bool fused = h->K == 1;
    void *Sb[2] = {h->S, fused ? h->S_b : h->S};

    if (use_graph) {
        Graphs &gr = h->graphs;
        if (gr.phi_user != phi || gr.mode != (int)mode || gr.net_gen != h->net_gen) {
            for (int p = 0; p < 2; ++p)
                if (gr.exec[p]) { cudaGraphExecDestroy(gr.exec[p]); gr.exec[p] = nullptr; }
            gr.phi_user = nullptr;
            // graphs carry no timing events: sweeps are timed only when launched directly
            const bool prof = h->prof;
            h->prof = false;
            for (int p = 0; p < 2; ++p) {
                cudaGraph_t graph;
                cudaError_t be = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
                if (be != cudaSuccess) { h->prof = prof; return cuda_fail(h, be, "cudaStreamBeginCapture"); }
                sn_status cs = fused ? SN_OK : launch_source(h, buf[p], h->S, h->cap_stream);
                if (cs == SN_OK)
                    cs = sweep_once(h, Sb[p], buf[1 - p], buf[p], mode, h->cap_stream, fused ? Sb[1 - p] : nullptr);
                cudaError_t me = cudaMemcpyAsync(h->acc_host, h->acc, sizeof(double) * ACC_COUNT,
                                                 cudaMemcpyDeviceToHost, h->cap_stream);
                cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &graph);
                h->prof = prof;
                if (cs != SN_OK) return cs;
                SN_CK(h, me);
                SN_CK(h, ee);
                cudaError_t ie = cudaGraphInstantiate(&gr.exec[p], graph, 0);
                cudaGraphDestroy(graph);
                SN_CK(h, ie);
                h->prof = false;
            }
            h->prof = prof;
            gr.phi_user = phi;
            gr.mode = (int)mode;
            gr.net_gen = h->net_gen;
            h->prof_pending = false;
        }
    }

    int it = 0, cur = 0;
    double cmax = 0, cmean = 0;
    sn_status rc = SN_ENOCONV;
    if (fused) {
        s = launch_source(h, phi, Sb[0], st);
        if (s != SN_OK) return s;
    }
    for (it = 0; it < max_it; ++it) {
        if (use_graph) {
            SN_CK(h, cudaGraphLaunch(h->graphs.exec[cur], st));
        } else {
            s = fused ? SN_OK : launch_source(h, buf[cur], h->S, st);
            if (s == SN_OK) s = sweep_once(h, Sb[cur], buf[1 - cur], buf[cur], mode, st, fused ? Sb[1 - cur] : nullptr);
            if (s != SN_OK) return s;
            SN_CK(h, cudaMemcpyAsync(h->acc_host, h->acc, sizeof(double) * ACC_COUNT, cudaMemcpyDeviceToHost, st));
        }
        SN_CK(h, cudaStreamSynchronize(st));
        prof_collect(h);
        cur = 1 - cur;
        const double *a = h->acc_host;
        cmax = a[ACC_PMAX] > 0 ? a[ACC_DMAX] / a[ACC_PMAX] : 0.0;
        cmean = a[ACC_MEANN] > 0 ? a[ACC_MEAN] / a[ACC_MEANN] : 0.0;
        take_tallies(h);
        if (a[ACC_ABORT] != 0.0) return fail(h, SN_ETIMEOUT, "sn_source_iterate: a bounded wait of the sweep gave up");
        if (mode == SN_SOLVE_ANN || mode == SN_SOLVE_ANN_GATED || mode == SN_SOLVE_ANN_FROZEN) {
            s = check_ann_timeouts(h);
            if (s != SN_OK) return s;
        }
        if (a[ACC_FLAG] != 0.0) {
            rc = fail(h, SN_ENAN, "sn_source_iterate: non-finite scalar flux");
            ++it;
            break;
        }
        if (cmax <= tol) {
            rc = SN_OK;
            ++it;
            break;
        }
    }
    if (cur == 1)
        SN_CK(h, cudaMemcpyAsync(phi, h->phi_b, h->esz * h->G * h->K * h->ncell * 8, cudaMemcpyDeviceToDevice, st));
    SN_CK(h, cudaStreamSynchronize(st));
    if (iters) *iters = it;
    if (change_max) *change_max = cmax;
    if (change_mean) *change_mean = cmean;
    if (rc == SN_ENOCONV) fail(h, SN_ENOCONV, "sn_source_iterate: max_it reached before tol");
    return rc;
}

sn_status sn_harvest(sn_handle h, const float *S, float *in27, int64_t cap, uint64_t seed, int64_t *n_out)
{
    if (!h || !S || !in27 || !n_out) return fail(h, SN_EINVAL, "sn_harvest: NULL argument");
    if (h->fp64) return fail(h, SN_EINVAL, "sn_harvest: needs an FP32 handle");
    if (h->K > 1 || h->geom) return fail(h, SN_EINVAL, "sn_harvest: isotropic scattering on box cells only");
    if (cap < 1 || cap > (1LL << 31)) return fail(h, SN_EINVAL, "sn_harvest: cap must be in 1..2^31");
    const cudaStream_t st = h->stream;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(h->acc + ACC_HARVEST);
    SN_CK(h, cudaMemsetAsync(h->acc, 0, sizeof(double) * ACC_COUNT, st));
    sn_status s = launch_harvest(h, S, in27, (uint32_t)cap, seed, cnt, st);
    if (s != SN_OK) return s;
    unsigned long long c = 0;
    SN_CK(h, cudaMemcpyAsync(&c, cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
    SN_CK(h, cudaStreamSynchronize(st));
    *n_out = (int64_t)std::min<unsigned long long>(c, (unsigned long long)cap);
    return SN_OK;
}

sn_status sn_source(sn_handle h, const void *phi, void *S)
{
    if (!h || !phi || !S) return fail(h, SN_EINVAL, "sn_source: NULL argument");
    return launch_source(h, phi, S, h->stream);
}

sn_status sn_set_profiling(sn_handle h, int32_t enable)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_set_profiling: NULL handle");
    if (enable && !h->ev_sweep[0]) {
        SN_CK(h, cudaEventCreate(&h->ev_sweep[0]));
        SN_CK(h, cudaEventCreate(&h->ev_sweep[1]));
    }
    h->prof = enable != 0;
    h->prof_pending = false;
    return SN_OK;
}

sn_status sn_get_profile(sn_handle h, double *sweep_ms, int64_t *sweeps, int32_t reset)
{
    if (!h) return fail(nullptr, SN_EINVAL, "sn_get_profile: NULL handle");
    if (sweep_ms) *sweep_ms = h->prof_ms;
    if (sweeps) *sweeps = h->prof_sweeps;
    if (reset) {
        h->prof_ms = 0.0;
        h->prof_sweeps = 0;
    }
    return SN_OK;
}

}  // extern "C"

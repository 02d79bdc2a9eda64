// sn_sweep_keys.cu -- the FP32 elimination sweep on box cells with isotropic
// scattering (modes SN_SOLVE_GE32R and SN_SOLVE_GE32): the hyperplane wavefront of
// Sec. 2 (after Eq. (14)) with one thread per key.
//
// Key.  A key is (octant o, cell of the hyperplane, group g).  Its thread solves the
// cell's system (14) for a chunk of the octant's directions in turn (all of them
// where the hyperplane has enough keys to fill the GPU; on the small hyperplanes at
// the two ends of the wavefront the directions are split over NCH threads so that
// the work still spreads over the GPU).  Everything a key's directions share is
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
// after the planes, in place of the slot, so the direction loop has no boundary
// test; on the outflow boundary the outflow is stored like any other, and after the
// last hyperplane every slot holds the outflow of the last cell of its column: the
// leakage kernel below sums the boundary leakage from them.
//
// Prefetch.  The next direction's three inflow faces are copied into a per-thread
// shared-memory stage (cp.async, L2 only) while the current direction is solved.  A
// key's cell, opacity and source are read before the key waits for its upwind
// neighbours: none of them is written by the sweep.
//
// Scheduling.  Two forms share the per-key work:
//  * the wavefront kernel (sweep_ge_wave), one persistent launch per sweep: work
//    units (hyperplane s, octant o, a tile of keys) are handed out in wavefront order
//    by an atomic counter; a unit waits only for the units of hyperplane s - 1 that
//    hold its cells' upwind neighbours (a done flag per unit, release / acquire at GPU
//    scope), so a unit starts as soon as its own inputs exist and no hyperplane waits
//    for the slowest tile of the previous one.  A unit waits only for units handed
//    out before it, to CTAs that are already running, so the wait always ends; every
//    wait is bounded all the same (2^31 SM cycles, about 1 s), after which the CTA
//    raises the sweep's abort flag, every CTA stops, and the call returns SN_ETIMEOUT;
//  * the per-hyperplane kernel (sweep_ge_keys), one launch per hyperplane ordered by
//    programmatic dependent launch, used when the unit tables are absent.
//
// The flux partials go to phi_oct[o][c][g][8] (physical node order); the reduction
// kernel of sn_sweep.cu sums the eight octants in a fixed order.  Nothing is atomic
// but the hand-out of units: the flux is bit-reproducible run to run.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "ge8.cuh"
#include "octnet.cuh"
#include "sn_internal.cuh"
#include "sweep_common.cuh"
#include "wave.cuh"

namespace sn {

#ifndef SN_KEY_BLOCK
#define SN_KEY_BLOCK 128
#endif
constexpr int kKeyBlock = SN_KEY_BLOCK;   // threads a CTA
constexpr int kKeyMaxDo = 64;             // directions per octant the kernels take
// CTAs per SM: 3 (168 registers a thread) measured faster on blocked_64 than 4
// (128 registers, with spills of the refined solve): 5.55 against 5.91 ms a sweep
#ifndef SN_KEY_MINBLOCKS
#define SN_KEY_MINBLOCKS 3
#endif


struct KeyArgs {
    int nx, ny, nz, G, Do, C;
    int nkeys;                   // per-hyperplane kernel: keys of one octant (cells x G)
    FastDiv divG;                // key -> (cell of the hyperplane, group)
    const uint32_t *cells;       // per-hyperplane kernel: packed (i',j',k') of its cells
    const float *sigt;           // [G][C]
    const float *S;              // [G][C][8]
    const float4 *dir;           // [Do] (3|Omega_x|/dx, 3|Omega_y|/dy, 3|Omega_z|/dz, w)
    float4 *face;                // x-planes | y-planes | z-planes | inflow vectors [G][6]
    uint32_t off_y, off_z, off_in;
    float *phi_oct;              // [8][C][G][8]
    WaveCtl w;                   // wavefront kernel
    // the paper's octant networks (network sweep): folded weights [8][288], |Omega| of
    // the octant's directions [Do], the cell sizes
    const float *onet;
    const float4 *dir_abs;
    float hx, hy, hz;
};

// Inflow-face stages a thread cycles through: the faces of the next NST - 1 directions
// are in flight while one is solved.  Three stages measured faster for the solve
// without refinement (3.94 against 4.11 ms on blocked_64) and slower with it, whose
// registers they push into spills (4.59 against 4.56 ms).
template <bool REFINE, bool NET = false>
constexpr int key_stages() { return (REFINE && !NET) ? 2 : 3; }

template <int NST>
struct KeySmem {
    float4 stage[NST][3][kKeyBlock];   // per-thread inflow stages
    float4 msrc[2][kKeyBlock];       // per-thread (Mh x Mh x Mh) S
    float4 dsm[kKeyMaxDo];           // direction table
    float red[8 * kKeyBlock];        // chunk partials of the flux (more than one chunk)
    int kdst[kKeyBlock];             // flux-partial index of each thread's key
};

// Work of one CTA on one tile of keys: keys key0 .. key0 + KB - 1 of octant o on a
// hyperplane with `cells` and nkeys keys an octant, its directions split in 2^lch
// chunks (KB = kKeyBlock >> lch keys a tile).  wait() runs after the keys' set-up,
// must contain a CTA barrier, and returns once the upwind faces are complete (false:
// give the tile up).  Returns false if the tile was given up.
// NET: the per-direction solve is the octant network of the key's octant (all 8
// octants' networks at wn in the row layout of octnet.cuh, |Omega| of the directions at
// dab); the key's part of the hidden inputs takes the place of (Mh x Mh x Mh) S in msrc.
template <bool REFINE, bool NET, typename Wait>
__device__ __forceinline__ bool key_tile(const KeyArgs &a, KeySmem<key_stages<REFINE, NET>()> &sm, const float *wn,
                                         const float4 *dab, int o, const uint32_t *cells, int nkeys, int key0,
                                         int lch, Wait wait)
{
    const int t = threadIdx.x;
    const int KB = kKeyBlock >> lch;
    const int chunk = t >> (31 - __clz(KB)), lk = t & (KB - 1);
    const int key = key0 + lk;
    const bool act = key < nkeys;
    const int Do = a.Do, G = a.G;
    const int nch = 1 << lch;
    const int d0 = chunk * Do / nch, d1 = (chunk + 1) * Do / nch;

    float sig = 0.f;
    uint32_t ou0 = 0, ou1 = 0, ou2 = 0;   // this direction's slots
    uint32_t inb = 0, bnd = 0;            // inflow vectors of the key's group; inflow-boundary axes
    int dst = -1;                         // (o C + c) G + g: the key's flux partial
    if (act) {
        const uint32_t cidx = a.divG.div((uint32_t)key);
        const int g = key - (int)cidx * G;
        const uint32_t pk = cells[cidx];
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
        if constexpr (NET) {
            float ak[kOnHid];
            octnet_key_part_rows(wn + kOnRows * o, Sm, sig, ak);
            sm.msrc[0][t] = make_float4(ak[0], ak[1], ak[2], ak[3]);
            sm.msrc[1][t] = make_float4(ak[4], ak[5], ak[6], ak[7]);
        } else {
            mh_axis<0>(Sm);
            mh_axis<1>(Sm);
            mh_axis<2>(Sm);
            sm.msrc[0][t] = make_float4(Sm[0], Sm[1], Sm[2], Sm[3]);
            sm.msrc[1][t] = make_float4(Sm[4], Sm[5], Sm[6], Sm[7]);
        }
        const uint32_t DG = (uint32_t)(Do * G), first = (uint32_t)(d0 * G + g);
        ou0 = (uint32_t)(o * a.ny * a.nz + jp + a.ny * kp) * DG + first;
        ou1 = a.off_y + (uint32_t)(o * a.nx * a.nz + ip + a.nx * kp) * DG + first;
        ou2 = a.off_z + (uint32_t)(o * a.nx * a.ny + ip + a.nx * jp) * DG + first;
        inb = a.off_in + 6u * (uint32_t)g;
        bnd = (ip == 0 ? 1u : 0u) | (jp == 0 ? 2u : 0u) | (kp == 0 ? 4u : 0u);
        dst = (o * a.C + c) * G + g;
    }
    sm.kdst[t] = dst;
    if (!wait()) return false;

    float phi[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) phi[n] = 0.f;
    if (act && d0 < d1) {
        constexpr uint32_t AX = kKeyBlock * 16;   // bytes between the faces of a stage
        constexpr uint32_t SP = 3 * AX;           // bytes between the two stages
        const uint32_t sb = smem_u32(&sm.stage[0][0][t]);
        // inflow slot of direction d: the outflow slot (in place), or on the inflow
        // boundary the group's psi_inc vector of that face (every direction)
        auto issue = [&](uint32_t buf, uint32_t s0, uint32_t s1, uint32_t s2) {
            const uint32_t nb = sb + buf * SP;
            cp_async16(nb, a.face + ((bnd & 1u) ? inb + (uint32_t)(o & 1) : s0));
            cp_async16(nb + AX, a.face + ((bnd & 2u) ? inb + 2u + (uint32_t)((o >> 1) & 1) : s1));
            cp_async16(nb + 2 * AX, a.face + ((bnd & 4u) ? inb + 4u + (uint32_t)((o >> 2) & 1) : s2));
        };
        constexpr int kKeyStages = key_stages<REFINE, NET>();
        issue(0u, ou0, ou1, ou2);
        cp_async_commit();
        if constexpr (kKeyStages == 3) {
            if (d0 + 1 < d1) issue(1u, ou0 + (uint32_t)G, ou1 + (uint32_t)G, ou2 + (uint32_t)G);
            cp_async_commit();
        }
        int cur = 0;   // this direction's stage
        for (int d = d0; d < d1; ++d) {
            // the stage of direction d + kKeyStages - 1, which the slot offsets (advanced
            // one direction a step) reach at + (kKeyStages - 1) G
            const int nxt = cur == 0 ? kKeyStages - 1 : cur - 1;
            constexpr uint32_t ahead = kKeyStages - 1;
            if (d + (int)ahead < d1)
                issue((uint32_t)nxt, ou0 + ahead * (uint32_t)G, ou1 + ahead * (uint32_t)G, ou2 + ahead * (uint32_t)G);
            cp_async_commit();
            cp_async_wait_pending<kKeyStages - 1>();   // this direction's faces have landed
            const float4 dd = sm.dsm[d];
            float x[8];
            // the right-hand side's inputs stay in shared memory (this stage is not refilled
            // before the next direction): no register copy of them, nor of b, across the
            // elimination (168 registers without spills; 4.52 against 4.59 ms a blocked_64
            // sweep with the register copies)
            if constexpr (NET) {
                const float4 ab = dab[d];
                octnet_key_row_rows(wn + kOnRows * o, &sm.msrc[0][t], &sm.msrc[1][t], &sm.stage[cur][0][t],
                                    &sm.stage[cur][1][t], &sm.stage[cur][2][t], ab.x, ab.y, x);
            } else {
                cell_solve_key_x2_sm<REFINE>(dd.x, dd.y, dd.z, sig, &sm.msrc[0][t], &sm.msrc[1][t],
                                             &sm.stage[cur][0][t], &sm.stage[cur][1][t], &sm.stage[cur][2][t], x);
            }
            cur = cur + 1 == kKeyStages ? 0 : cur + 1;
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
    if (lch == 0) {
        if (act) {
            float4 *p = reinterpret_cast<float4 *>(a.phi_oct) + 2 * (int64_t)dst;
            p[0] = make_float4(phi[0], phi[1], phi[2], phi[3]);
            p[1] = make_float4(phi[4], phi[5], phi[6], phi[7]);
        }
    } else {
        // the chunks of a key add their partials in chunk order
        float4 *r = reinterpret_cast<float4 *>(sm.red + (chunk * KB + lk) * 8);
        r[0] = make_float4(phi[0], phi[1], phi[2], phi[3]);
        r[1] = make_float4(phi[4], phi[5], phi[6], phi[7]);
        __syncthreads();
        for (int e = t; e < KB * 8; e += kKeyBlock) {
            const int kk = e >> 3, n = e & 7;
            const int dk = sm.kdst[kk];   // chunk 0's thread of key kk
            if (dk < 0) continue;
            float s = sm.red[kk * 8 + n];
            for (int q = 1; q < nch; ++q) s += sm.red[(q * KB + kk) * 8 + n];
            a.phi_oct[(int64_t)dk * 8 + n] = s;
        }
    }
    return true;
}

// One launch per hyperplane (grid: tiles of one octant x 8 octants), ordered by
// programmatic dependent launch.
template <bool REFINE, int LCH>
__global__ void __launch_bounds__(kKeyBlock, SN_KEY_MINBLOCKS) sweep_ge_keys(KeyArgs a)
{
    __shared__ __align__(16) KeySmem<key_stages<REFINE>()> sm;
    griddep_launch();
    for (int e = threadIdx.x; e < a.Do; e += kKeyBlock) sm.dsm[e] = a.dir[e];
    key_tile<REFINE, false>(a, sm, nullptr, nullptr, (int)blockIdx.y, a.cells, a.nkeys,
                            (int)blockIdx.x * (kKeyBlock >> LCH), LCH, [] {
        __syncthreads();   // direction table, key records
        griddep_wait();    // the previous hyperplane's outflow faces are complete
        return true;
    });
}

// The persistent wavefront kernel (see the file header), one unit a CTA: units[u] =
// (first key of the tile within its hyperplane and octant, s | o << 12 | lch << 15,
// first unit of hyperplane s - 1 it depends on, how many) with kKeyBlock >> lch keys
// a tile; uplane[u] = (first cell of hyperplane s in the hyperplane table, its keys,
// the second range of units it depends on).  Thread 0 takes the next unit's index
// when the CTA starts a unit and copies its descriptor into shared memory (cp.async)
// once the current unit's wait is over, so a unit starts without a global round trip;
// warp 0 waits for the dependencies, testing their flags together.  Two CTA barriers a
// unit: after the wait (which also orders every read of the descriptor before thread
// 0 overwrites it) and after the unit's stores (which also publishes the next one).
template <bool REFINE, bool NET>
__device__ __forceinline__ void wave_body(const KeyArgs &a, KeySmem<key_stages<REFINE, NET>()> &sm, const float *wn,
                                          const float4 *dab)
{
    __shared__ __align__(16) int4 s_ud;
    __shared__ __align__(16) int4 s_up;
    __shared__ int s_u, s_stop;
    const int t = threadIdx.x;
    for (int e = t; e < a.Do; e += kKeyBlock) sm.dsm[e] = a.dir[e];
    if (t == 0) {
        const int u = (int)atomicAdd(a.w.next, 1u);
        s_u = u;
        if (u < a.w.nunits) {
            s_ud = a.w.units[u];
            s_up = a.w.uplane[u];
        }
    }
    __syncthreads();
    for (;;) {
        const int u = s_u;
        if (u >= a.w.nunits) break;
        const int2 ud = make_int2(s_ud.x, s_ud.y);   // first key; s, o, lch
        const int2 up = make_int2(s_up.x, s_up.y);   // the hyperplane's first cell, keys
        int un = 0;
        if (t == 0) un = (int)atomicAdd(a.w.next, 1u);
        const int o = (ud.y >> 12) & 7, lch = (ud.y >> 15) & 7;
        const bool ok = key_tile<REFINE, NET>(a, sm, wn, dab, o, a.w.all_cells + up.x, up.y, ud.x, lch, [&] {
            if (t < 32) {
                const int4 d1 = s_ud, d2 = s_up;   // the dependency ranges (not kept in registers)
                const bool fine = wave_wait_deps_warp(a.w, d1.z, d1.w, d2.z, d2.w);
                if (t == 0) s_stop = fine ? 0 : 1;
            }
            __syncthreads();   // after every thread's read of this unit's descriptor
            const bool go = s_stop == 0;
            if (t == 0 && go && un < a.w.nunits) {
                cp_async16(smem_u32(&s_ud), a.w.units + un);
                cp_async16(smem_u32(&s_up), a.w.uplane + un);
                cp_async_commit();
            }
            return go;
        });
        if (!ok) break;
        if (t == 0) {
            cp_async_wait_all();   // the next unit's descriptor has landed
            s_u = un;
        }
        __syncthreads();   // every store of this unit has been issued; the next unit is published
        if (t == 0) wave_done(a.w, u);
    }
    cp_async_wait_all();
}

template <bool REFINE>
__global__ void __launch_bounds__(kKeyBlock, SN_KEY_MINBLOCKS) sweep_ge_wave(KeyArgs a)
{
    __shared__ __align__(16) KeySmem<key_stages<REFINE>()> sm;
    wave_body<REFINE, false>(a, sm, nullptr, nullptr);
}

// The paper's octant networks (Secs. 3-4, Eqs. (15)-(18)) as the cell solver of the
// same wavefront sweep.  The folded networks of all 8 octants (8 KB in the row layout,
// two hidden units or outputs a two-lane FMA) and the directions' |Omega| stay in
// shared memory; the mesh's uniform cell size is folded into each hidden unit's bias
// once per CTA.  A network row is far lighter than the
// elimination (about 300 FP32 operations): 4 CTAs an SM (128 registers, 37 KB of shared
// memory each) measured 3.61 ms a blocked_64 sweep, 5 (96 registers, with spills)
// 3.64 ms.
#ifndef SN_NETKEY_MINBLOCKS
#define SN_NETKEY_MINBLOCKS 4
#endif
__global__ void __launch_bounds__(kKeyBlock, SN_NETKEY_MINBLOCKS) sweep_net_wave(KeyArgs a)
{
    __shared__ __align__(16) KeySmem<key_stages<false, true>()> sm;
    __shared__ __align__(16) float wn[8 * kOnRows];
    __shared__ __align__(16) float4 dab[kKeyMaxDo];
    const int t = threadIdx.x;
    for (int e = t; e < 8 * kOnRows; e += kKeyBlock)
        wn[e] = octnet_row_layout(a.onet + kOnFold * (e / kOnRows), e % kOnRows, a.hx, a.hy, a.hz);
    for (int e = t; e < a.Do; e += kKeyBlock) dab[e] = a.dir_abs[e];
    // (wave_body's first barrier orders the tables before their first use)
    wave_body<false, true>(a, sm, wn, dab);
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

// log2 of the chunks a key's directions are split in on a hyperplane with `keys`
// keys (all octants): the fewest that still give about one thread per resident
// thread slot of a GPU with nsm SMs, at most 8 chunks and no more chunks than
// directions.
static int key_chunks_log2(int64_t keys, int Do, int nsm)
{
    const int64_t slots = (int64_t)nsm * SN_KEY_MINBLOCKS * kKeyBlock;
    int l = 0;
    while (l < 3 && (2 << l) <= Do && keys * (1 << l) < slots) ++l;
    return l;
}

static int key_chunks_log2(int64_t keys, int Do) { return key_chunks_log2(keys, Do, num_sms()); }

static void free_tables(WaveTables *w)
{
    if (!w) return;
    cudaFree(w->units);
    cudaFree(w->uplane);
    cudaFree(w->flags);
    delete w;
}

void free_wave(sn_handle h)
{
    if (!h) return;
    free_tables(static_cast<WaveTables *>(h->wave));
    h->wave = nullptr;
}

// Units in wavefront order: hyperplane, octant, tile.  A tile covers kKeyBlock >> lch
// consecutive keys (key = position of the cell within the hyperplane x G + g); it
// depends on the tiles of hyperplane s - 1 of the same octant (the octants are
// independent) that hold the upwind neighbours (i'-1,j',k'), (i',j'-1,k'),
// (i',j',k'-1) of its cells.  A hyperplane's cells are listed by (k', j'), so those
// tiles form two clusters (the neighbours in the tile's own k' rows, and those in the
// rows k' - 1): each unit carries two ranges, split at the largest gap.
bool wave_plan(int nx, int ny, int G, int Do, int nsm, const std::vector<int64_t> &off,
               const std::vector<uint32_t> &cells, const std::vector<uint32_t> &pos, std::vector<int4> &units,
               std::vector<int4> &uplane)
{
    units.clear();
    uplane.clear();
    const int np = (int)off.size() - 1;
    std::vector<int> lch(np), ntile(np);
    std::vector<int64_t> first(np + 1);   // first unit of each hyperplane
    first[0] = 0;
    for (int s = 0; s < np; ++s) {
        const int64_t n = off[s + 1] - off[s];
        lch[s] = key_chunks_log2(8 * n * G, Do, nsm);
        const int64_t kb = kKeyBlock >> lch[s];
        ntile[s] = (int)((n * G + kb - 1) / kb);
        first[s + 1] = first[s] + 8 * (int64_t)ntile[s];
    }
    if (first[np] >= (1LL << 30) || np > 4095) return false;   // the per-hyperplane kernel serves it
    units.resize((size_t)first[np]);
    uplane.resize((size_t)first[np]);
    std::vector<int64_t> dep;
    for (int s = 0; s < np; ++s) {
        const int64_t kb = kKeyBlock >> lch[s];
        const int64_t n = off[s + 1] - off[s];
        const int64_t kbp = s > 0 ? (kKeyBlock >> lch[s - 1]) : 1;
        for (int tl = 0; tl < ntile[s]; ++tl) {
            int64_t lo1 = 0, n1 = 0, lo2 = 0, n2 = 0;
            if (s > 0) {
                dep.clear();
                const int64_t p0 = tl * kb / G, p1 = std::min<int64_t>(n - 1, (tl * kb + kb - 1) / G);
                for (int64_t q = p0; q <= p1; ++q) {
                    const uint32_t pk = cells[off[s] + q];
                    const int ip = pk & 1023, jp = (pk >> 10) & 1023, kp = pk >> 20;
                    const int nb[3][3] = {{ip - 1, jp, kp}, {ip, jp - 1, kp}, {ip, jp, kp - 1}};
                    for (int m = 0; m < 3; ++m) {
                        if (nb[m][0] < 0 || nb[m][1] < 0 || nb[m][2] < 0) continue;
                        const int64_t lin = nb[m][0] + (int64_t)nx * (nb[m][1] + (int64_t)ny * nb[m][2]);
                        const int64_t pp = pos[lin];
                        for (int64_t d = pp * G / kbp; d <= (pp * G + G - 1) / kbp; ++d) dep.push_back(d);
                    }
                }
                if (!dep.empty()) {
                    std::sort(dep.begin(), dep.end());
                    dep.erase(std::unique(dep.begin(), dep.end()), dep.end());
                    size_t cut = dep.size();   // start of the second cluster
                    int64_t gap = 1;
                    for (size_t e = 1; e < dep.size(); ++e)
                        if (dep[e] - dep[e - 1] > gap) {
                            gap = dep[e] - dep[e - 1];
                            cut = e;
                        }
                    lo1 = dep[0];
                    n1 = dep[cut - 1] - dep[0] + 1;
                    if (cut < dep.size()) {
                        lo2 = dep[cut];
                        n2 = dep.back() - dep[cut] + 1;
                    }
                }
            }
            for (int o = 0; o < 8; ++o) {
                const int64_t u = first[s] + (int64_t)o * ntile[s] + tl;
                const int64_t base = s > 0 ? first[s - 1] + (int64_t)o * ntile[s - 1] : 0;
                units[u] = make_int4((int)(tl * kb), s | (o << 12) | (lch[s] << 15), (int)(base + lo1), (int)n1);
                uplane[u] = make_int4((int)off[s], (int)(n * G), (int)(base + lo2), (int)n2);
            }
        }
    }
    return true;
}

static sn_status build_tables(sn_handle h, const std::vector<uint32_t> &cells, const std::vector<uint32_t> &pos,
                              WaveTables **out)
{
    *out = nullptr;
    std::vector<int4> units, uplane;
    if (!wave_plan(h->nx, h->ny, h->G, h->Do, num_sms(), h->plane_off, cells, pos, units, uplane)) return SN_OK;
    WaveTables *w = new WaveTables();
    w->nunits = (int)units.size();
    cudaError_t e = cudaMalloc(&w->units, sizeof(int4) * units.size());
    if (e == cudaSuccess) e = cudaMalloc(&w->uplane, sizeof(int4) * uplane.size());
    if (e == cudaSuccess) e = cudaMalloc(&w->flags, sizeof(uint32_t) * (units.size() + 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->units, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->uplane, uplane.data(), sizeof(int4) * uplane.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the host vectors go out of scope
    if (e != cudaSuccess) {
        free_tables(w);
        return cuda_fail(h, e, "build_wave");
    }
    h->device_bytes += (int64_t)(2 * sizeof(int4) * units.size() + sizeof(uint32_t) * (units.size() + 1));
    *out = w;
    return SN_OK;
}

// SN_KEY_WAVE=0 keeps the per-hyperplane launches (the form the wavefront kernel is
// measured against)
#ifndef SN_KEY_WAVE
#define SN_KEY_WAVE 1
#endif
// The unit tables of the wavefront kernels (the elimination and the surrogate sweep).
sn_status build_wave(sn_handle h)
{
    free_wave(h);
    if (!SN_KEY_WAVE || !key_sweep_ok(h)) return SN_OK;
    std::vector<uint32_t> cells(h->ncell), pos(h->ncell);
    SN_CK(h, cudaMemcpyAsync(cells.data(), h->plane_cells, sizeof(uint32_t) * h->ncell, cudaMemcpyDeviceToHost,
                             h->stream));
    SN_CK(h, cudaMemcpyAsync(pos.data(), h->plane_pos, sizeof(uint32_t) * h->ncell, cudaMemcpyDeviceToHost, h->stream));
    SN_CK(h, cudaStreamSynchronize(h->stream));
    WaveTables *w = nullptr;
    sn_status r = build_tables(h, cells, pos, &w);
    if (r != SN_OK || !w) return r;
    int per_sm = 0, per_sm2 = 0;
    SN_CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_ge_wave<true>, kKeyBlock, 0));
    SN_CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, sweep_ge_wave<false>, kKeyBlock, 0));
    w->grid = std::max(1, std::min(std::min(per_sm, per_sm2), SN_KEY_MINBLOCKS) * num_sms());
    int per_sm_net = 0;
    SN_CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_net, sweep_net_wave, kKeyBlock, 0));
    w->grid_net = std::max(1, std::min(per_sm_net, SN_NETKEY_MINBLOCKS) * num_sms());
    h->wave = w;
    return SN_OK;
}

WaveCtl wave_ctl(sn_handle h)
{
    const WaveTables *w = static_cast<const WaveTables *>(h->wave);
    WaveCtl c = {};
    if (!w) return c;
    c.all_cells = h->plane_cells;
    c.units = w->units;
    c.uplane = w->uplane;
    c.flags = w->flags;
    c.next = w->flags + w->nunits;
    c.abort = h->acc + ACC_ABORT;
    c.nunits = w->nunits;
    return c;
}

template <bool REFINE, int LCH>
static cudaError_t launch_keys_plane(bool pdl, const KeyArgs &a, cudaStream_t st)
{
    constexpr int KB = kKeyBlock >> LCH;
    const dim3 grid((unsigned)((a.nkeys + KB - 1) / KB), 8);
    return launch_k(pdl, sweep_ge_keys<REFINE, LCH>, grid, dim3(kKeyBlock), 0, st, a);
}

template <bool REFINE>
static cudaError_t launch_keys_lch(int lch, bool pdl, const KeyArgs &a, cudaStream_t st)
{
    switch (lch) {
    case 0: return launch_keys_plane<REFINE, 0>(pdl, a, st);
    case 1: return launch_keys_plane<REFINE, 1>(pdl, a, st);
    case 2: return launch_keys_plane<REFINE, 2>(pdl, a, st);
    default: return launch_keys_plane<REFINE, 3>(pdl, a, st);
    }
}

static KeyArgs key_args(sn_handle h, const float *S, float *phi_oct)
{
    KeyArgs a = {};
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
    return a;
}

sn_status launch_sweep_keys(sn_handle h, const float *S, float *phi_oct, bool refine, cudaStream_t st)
{
    KeyArgs a = key_args(h, S, phi_oct);
    const WaveTables *w = static_cast<const WaveTables *>(h->wave);
    if (w) {
        a.w = wave_ctl(h);
        SN_CK(h, cudaMemsetAsync(w->flags, 0, sizeof(uint32_t) * (size_t)(w->nunits + 1), st));
    }
    if (h->prof) SN_CK(h, cudaEventRecord(h->ev_sweep[0], st));
    if (w) {
        if (refine)
            sweep_ge_wave<true><<<w->grid, kKeyBlock, 0, st>>>(a);
        else
            sweep_ge_wave<false><<<w->grid, kKeyBlock, 0, st>>>(a);
    } else {
        for (int s = 0; s < h->nplanes; ++s) {
            const int64_t n = h->plane_off[s + 1] - h->plane_off[s];
            a.cells = h->plane_cells + h->plane_off[s];
            a.nkeys = (int)(n * h->G);
            const int lch = key_chunks_log2(8 * n * h->G, h->Do);
            // hyperplanes after the first overlap their launch with the previous one's drain
            SN_CK(h, refine ? launch_keys_lch<true>(lch, s > 0, a, st) : launch_keys_lch<false>(lch, s > 0, a, st));
        }
    }
    SN_CK(h, cudaGetLastError());
    if (h->prof) {
        SN_CK(h, cudaEventRecord(h->ev_sweep[1], st));
        h->prof_pending = true;
    }
    return launch_leak_keys(h, st);
}

// The octant-network sweep on the wavefront schedule (box cells with unit tables).
sn_status launch_sweep_net_keys(sn_handle h, const float *S, float *phi_oct, cudaStream_t st)
{
    const WaveTables *w = static_cast<const WaveTables *>(h->wave);
    if (!w) return fail(h, SN_ESTATE, "octant-network key sweep without unit tables");
    KeyArgs a = key_args(h, S, phi_oct);
    a.onet = octnet_folded(h);
    if (!a.onet) return fail(h, SN_ESTATE, "octant-network sweep without networks");
    a.dir_abs = h->dir_abs;
    a.hx = (float)h->dx;
    a.hy = (float)h->dy;
    a.hz = (float)h->dz;
    a.w = wave_ctl(h);
    SN_CK(h, cudaMemsetAsync(w->flags, 0, sizeof(uint32_t) * (size_t)(w->nunits + 1), st));
    if (h->prof) SN_CK(h, cudaEventRecord(h->ev_sweep[0], st));
    sweep_net_wave<<<w->grid_net, kKeyBlock, 0, st>>>(a);
    SN_CK(h, cudaGetLastError());
    if (h->prof) {
        SN_CK(h, cudaEventRecord(h->ev_sweep[1], st));
        h->prof_pending = true;
    }
    return launch_leak_keys(h, st);
}

sn_status launch_leak_keys(sn_handle h, cudaStream_t st)
{
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

using namespace sn;

extern "C" sn_status sn_wave_plan(int32_t nx, int32_t ny, int32_t nz, int32_t G, int32_t Do, int32_t nsm,
                                  int32_t *units, int32_t *uplane, int64_t cap, int64_t *nunits)
{
    if (!nunits) return fail(nullptr, SN_EINVAL, "sn_wave_plan: nunits is NULL");
    *nunits = 0;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 1023 || ny > 1023 || nz > 1023)
        return fail(nullptr, SN_EINVAL, "sn_wave_plan: cells per axis must be in 1..1023");
    if (G < 1 || G > 1024) return fail(nullptr, SN_EINVAL, "sn_wave_plan: G must be in 1..1024");
    if (Do < 1 || Do > kKeyMaxDo) return fail(nullptr, SN_EINVAL, "sn_wave_plan: Do must be in 1..64");
    if (nsm < 1) return fail(nullptr, SN_EINVAL, "sn_wave_plan: nsm must be positive");
    std::vector<int64_t> off;
    std::vector<uint32_t> cells, pos;
    hyperplane_tables(nx, ny, nz, off, cells, pos);
    std::vector<int4> u, up;
    if (!wave_plan(nx, ny, G, Do, nsm, off, cells, pos, u, up)) return SN_OK;
    *nunits = (int64_t)u.size();
    if (!units && !uplane) return SN_OK;
    if (!units || !uplane || cap < *nunits)
        return fail(nullptr, SN_EINVAL, "sn_wave_plan: the output arrays hold fewer than *nunits records");
    std::memcpy(units, u.data(), sizeof(int4) * u.size());
    std::memcpy(uplane, up.data(), sizeof(int4) * up.size());
    return SN_OK;
}

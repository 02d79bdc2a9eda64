// wave.cuh -- the wavefront schedule shared by the persistent key sweeps: work units
// (hyperplane s, octant o, tile of keys) in wavefront order, handed out by an atomic
// counter, each waiting only for the units of hyperplane s - 1 that hold its cells'
// upwind neighbours (see sn_sweep_keys.cu for the tables and the argument that every
// wait ends).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace sn {

// Unit tables (built by build_wave): units[u] = (first key of the tile within its
// hyperplane and octant, s | o << 12 | lch << 15 (lch: log2 of the chunks a key's
// directions are split in), first unit of hyperplane s - 1 it depends on, how many);
// uplane[u] = (first cell of hyperplane s in the hyperplane table, its keys (cells x
// G), first unit of a second range it depends on, how many).
struct WaveTables {
    int4 *units = nullptr;
    int4 *uplane = nullptr;
    uint32_t *flags = nullptr;     // [nunits] done flags, then the hand-out counter
    int nunits = 0;
    int grid = 0;                  // persistent CTAs of the elimination sweep
    int grid_net = 0;              // persistent CTAs of the octant-network sweep
};

struct WaveCtl {
    const uint32_t *all_cells;     // the hyperplane table
    const int4 *units;
    const int4 *uplane;
    uint32_t *flags;               // zeroed before the sweep
    uint32_t *next;                // zeroed before the sweep
    double *abort;                 // the sweep's abort flag (zeroed accumulator slot)
    int nunits;
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The 32 lanes of one warp: wait until units [lo1, lo1 + n1) and [lo2, lo2 + n2) are
// done, lane l testing the l-th, (l + 32)-th, ... of them, so that the tests of one
// wait overlap instead of taking one L2 round trip each.  Every wait is bounded (2^31
// SM cycles, about 1 s, from the first test); on running out it raises the sweep's
// abort flag.  Each lane acquires the flags it tested; the barrier that follows the
// wait orders them before the reads of the upwind faces.  Returns false on every lane
// if the sweep is to stop (abort raised by this or another CTA).
__device__ __forceinline__ bool wave_wait_deps_warp(const WaveCtl &w, int lo1, int n1, int lo2, int n2)
{
    const int lane = threadIdx.x & 31;
    const long long t0 = clock64();
    for (int base = 0; base < n1 + n2; base += 32) {
        const int e = base + lane;
        const int v = e < n1 ? lo1 + e : lo2 + (e - n1);
        bool got = e >= n1 + n2;
        for (;;) {
            if (!got) got = ld_acquire_u32(w.flags + v) != 0u;
            if (__all_sync(0xffffffffu, got)) break;
            int give_up = 0;
            if (lane == 0) {
                if (*reinterpret_cast<volatile double *>(w.abort) != 0.0) {
                    give_up = 1;
                } else if (clock64() - t0 > (1LL << 31)) {
                    *reinterpret_cast<volatile double *>(w.abort) = 1.0;
                    give_up = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, give_up, 0)) return false;
            __nanosleep(64);
        }
    }
    return true;
}

// Thread 0, after a CTA barrier that follows every store of unit u: publish it.
__device__ __forceinline__ void wave_done(const WaveCtl &w, int u)
{
    __threadfence();
    st_release_u32(w.flags + u, 1u);
}

}  // namespace sn

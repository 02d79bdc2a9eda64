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
// directions are split in), first unit of hyperplane s - 1 it depends on, how many).
struct WaveTables {
    int4 *units = nullptr;
    uint2 *uplane = nullptr;       // [nunits] the unit's hyperplane: first cell, keys (cells x G)
    uint32_t *flags = nullptr;     // [nunits] done flags, then the hand-out counter
    uint32_t *plane_off = nullptr; // [nplanes + 1] offsets into the hyperplane table
    int nunits = 0;
    int grid = 0;                  // persistent CTAs of the elimination sweep
};

struct WaveCtl {
    const uint32_t *all_cells;     // the hyperplane table
    const uint32_t *plane_off;
    const int4 *units;
    const uint2 *uplane;
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

// The 32 lanes of one warp: wait until units [lo, lo + n) are done, lane l testing
// flags lo + l, lo + l + 32, ..., so that the tests of one wait overlap instead of
// taking one L2 round trip each.  Every wait is bounded (2^31 SM cycles, about 1 s,
// from the first test); on running out it raises the sweep's abort flag.  Returns
// false if the sweep is to stop (abort raised by this or another CTA).
// Each lane acquires the flags it tested; the CTA barrier that follows the wait orders
// them before every thread's reads of the upwind faces.  Returns the same value on
// every lane.
__device__ __forceinline__ bool wave_wait_deps_warp(const WaveCtl &w, int lo, int n)
{
    const int lane = threadIdx.x & 31;
    const long long t0 = clock64();
    for (int base = lo; base < lo + n; base += 32) {
        const int v = base + lane;
        bool got = v >= lo + n;
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

// sweep_common.cuh -- 4-vector face-plane access shared by the elimination and the
// surrogate sweep kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include <utility>

namespace sn {

template <typename T>
struct Vec4 {
    T v[4];
};

template <typename T>
__device__ __forceinline__ void load4(T (&u)[4], const Vec4<T> *p)
{
    if constexpr (sizeof(T) == 4) {
        const float4 f = *reinterpret_cast<const float4 *>(p);
        u[0] = f.x; u[1] = f.y; u[2] = f.z; u[3] = f.w;
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        u[0] = a.x; u[1] = a.y; u[2] = b.x; u[3] = b.y;
    }
}

template <typename T>
__device__ __forceinline__ void store4(Vec4<T> *p, T a, T b, T c, T d)
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
        reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Asynchronous global -> shared copies (cp.async), used to stage the next tile's
// inputs while the current tile is being solved.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// every committed group but the N most recent ones has landed
template <int N>
__device__ __forceinline__ void cp_async_wait_pending()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copy n bytes (a multiple of 16, both addresses 16-byte aligned) in 16-byte pieces.
__device__ __forceinline__ void cp_async_bytes(uint32_t dst, const void *src, int n)
{
    for (int b = 0; b < n; b += 16) cp_async16(dst + b, static_cast<const char *>(src) + b);
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

// Per key (cell of the hyperplane, group) of a tile, written once by the key's
// thread: face-plane slots of its direction 0 (x, y, z planes), boundary flags,
// physical cell and group.
struct KeyRec {
    int bx, by, bz;
    uint32_t flags;   // bits 0-2: inflow face on the boundary (x, y, z); 3-5: outflow
                      // face on the boundary; 7: key exists
    int cell, g, pad0, pad1;
};

template <int DO, typename Args>
__device__ __forceinline__ void make_key(const Args &a, int o, uint32_t key, uint32_t pk, KeyRec &r)
{
    const int Do = DO ? DO : a.Do;
    const uint32_t cidx = a.divG.div(key);
    const int g = (int)(key - cidx * (uint32_t)a.G);
    const int ip = pk & 1023, jp = (pk >> 10) & 1023, kp = pk >> 20;
    const int i = (o & 1) ? a.nx - 1 - ip : ip;
    const int j = (o & 2) ? a.ny - 1 - jp : jp;
    const int k = (o & 4) ? a.nz - 1 - kp : kp;
    r.cell = i + a.nx * (j + a.ny * k);
    r.g = g;
    const int GD = a.G * Do, gd = g * Do;
    r.bx = (o * a.ny * a.nz + jp + a.ny * kp) * GD + gd;
    r.by = (o * a.nx * a.nz + ip + a.nx * kp) * GD + gd;
    r.bz = (o * a.nx * a.ny + ip + a.nx * jp) * GD + gd;
    r.flags = 0x80u | (ip == 0 ? 1u : 0u) | (jp == 0 ? 2u : 0u) | (kp == 0 ? 4u : 0u) |
              (ip == a.nx - 1 ? 8u : 0u) | (jp == a.ny - 1 ? 16u : 0u) | (kp == a.nz - 1 ? 32u : 0u);
    r.pad0 = r.pad1 = 0;
}

__device__ __forceinline__ void put_key(unsigned char *p, const KeyRec &r)
{
    reinterpret_cast<int4 *>(p)[0] = make_int4(r.bx, r.by, r.bz, (int)r.flags);
    reinterpret_cast<int4 *>(p)[1] = make_int4(r.cell, r.g, 0, 0);
}

__device__ __forceinline__ KeyRec get_key(const unsigned char *p)
{
    const int4 u = reinterpret_cast<const int4 *>(p)[0], v = reinterpret_cast<const int4 *>(p)[1];
    KeyRec r;
    r.bx = u.x; r.by = u.y; r.bz = u.z; r.flags = (uint32_t)u.w;
    r.cell = v.x; r.g = v.y; r.pad0 = r.pad1 = 0;
    return r;
}

// Programmatic dependent launch: the hyperplane kernels are launched so that the next
// one may be scheduled while the current one drains.  A kernel lets its dependent
// launch early (griddep_launch) and waits for its predecessor's completion and
// memory (griddep_wait) before it touches anything that predecessor writes; both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch k<<<grid, block, smem, st>>>(args...), with programmatic stream serialisation
// when pdl is set.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

}  // namespace sn

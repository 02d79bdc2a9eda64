// sweep_common.cuh -- 4-vector face-plane access shared by the elimination and the
// surrogate sweep kernels.
#pragma once

#include <cuda_runtime.h>

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

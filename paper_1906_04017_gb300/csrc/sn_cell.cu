// sn_cell.cu -- batches of independent one-cell problems (the paper's one-cell problem,
// Sec. 3; the per-cell system (14) of Sec. 2), one thread per problem.
#include <cmath>

#include "cell_problem.cuh"
#include "sn_internal.cuh"

namespace sn {

// The 27 inputs of a block's problems are staged through shared memory so that the
// global loads are coalesced.
template <typename T, bool REFINE>
__global__ void __launch_bounds__(128) cell_solve_kernel(const T *__restrict__ in27, T *__restrict__ out,
                                                         int64_t n)
{
    __shared__ T stage[128 * 27];
    for (int64_t base = (int64_t)blockIdx.x * 128; base < n; base += (int64_t)gridDim.x * 128) {
        const int64_t cnt = n - base < 128 ? n - base : 128;
        __syncthreads();
        for (int64_t e = threadIdx.x; e < cnt * 27; e += 128) stage[e] = in27[base * 27 + e];
        __syncthreads();
        if (threadIdx.x < cnt) {
            T psi[8];
            solve_in27<T, REFINE>(stage + threadIdx.x * 27, psi);
            T *o = out + (base + threadIdx.x) * 8;
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = psi[k];
        }
    }
}

static int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <typename T, bool REFINE>
static cudaError_t launch_cells(const T *in27, T *psi, int64_t n, cudaStream_t st)
{
    int64_t grid = (n + 127) / 128;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (grid > cap) grid = cap;
    cell_solve_kernel<T, REFINE><<<(unsigned)grid, 128, 0, st>>>(in27, psi, n);
    return cudaGetLastError();
}

sn_status launch_cells_f32(const float *in27, float *psi, int64_t n, bool refine, cudaStream_t st)
{
    cudaError_t e = refine ? launch_cells<float, true>(in27, psi, n, st)
                           : launch_cells<float, false>(in27, psi, n, st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cell_solve_kernel");
    return SN_OK;
}

}  // namespace sn

using namespace sn;

extern "C" {

sn_status sn_cell_solve_batch_f64(const double *in27, double *psi, int64_t n, void *stream)
{
    if (n < 0) return fail(nullptr, SN_EINVAL, "sn_cell_solve_batch_f64: n < 0");
    if (n == 0) return SN_OK;
    if (!in27 || !psi) return fail(nullptr, SN_EINVAL, "sn_cell_solve_batch_f64: NULL pointer");
    cudaError_t e = launch_cells<double, false>(in27, psi, n, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cell_solve_kernel<double>");
    return SN_OK;
}

}  // extern "C"

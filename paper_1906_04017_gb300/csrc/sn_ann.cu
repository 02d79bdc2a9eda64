// sn_ann.cu -- the shallow-network surrogate of the per-cell solve (Sec. 3) and the
// FP32 one-cell entry point that dispatches between elimination and surrogate.
#include "sn_internal.cuh"

namespace sn {

void free_net(sn_handle h)
{
    if (!h) return;
    h->net = nullptr;
    h->has_net = false;
}

}  // namespace sn

using namespace sn;

extern "C" {

sn_status sn_cell_solve_batch(sn_handle h, const float *in27, float *psi, int64_t n, sn_solve_mode mode,
                              void *stream)
{
    if (n < 0) return fail(h, SN_EINVAL, "sn_cell_solve_batch: n < 0");
    if (mode == SN_SOLVE_GE32R || mode == SN_SOLVE_GE32) {
        if (n == 0) return SN_OK;
        if (!in27 || !psi) return fail(h, SN_EINVAL, "sn_cell_solve_batch: NULL pointer");
        sn_status s = launch_cells_f32(in27, psi, n, mode == SN_SOLVE_GE32R, (cudaStream_t)stream);
        if (s != SN_OK && h) h->err = sn_last_error(nullptr);
        return s;
    }
    if (mode == SN_SOLVE_ANN || mode == SN_SOLVE_ANN_GATED) {
        if (!h || !h->has_net) return fail(h, SN_ESTATE, "sn_cell_solve_batch: no surrogate network");
        return fail(h, SN_ESTATE, "sn_cell_solve_batch: surrogate not available");
    }
    return fail(h, SN_EINVAL, "sn_cell_solve_batch: unknown mode");
}

}  // extern "C"

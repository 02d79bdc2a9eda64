// sn_internal.cuh -- the handle and the helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sn.h"

namespace sn {

constexpr double kPi = 3.14159265358979323846;

// Per-direction data of one octant (every octant uses the same |Omega|):
// t3a = 3 |Omega_a| / h_a, w = quadrature weight.
template <typename T>
struct DirData {
    T t3x, t3y, t3z, w;
};

// Division of 32-bit unsigned n < 2^31 by a run-time constant d >= 1 with a multiply
// and a shift (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994): q = (umulhi(n, m) + n) >> s, s = ceil(log2 d),
// m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
    uint32_t d = 1, m = 1, s = 0;
    FastDiv() = default;
    explicit FastDiv(uint32_t dv) : d(dv)
    {
        s = 0;
        while ((1ull << s) < dv) ++s;
        m = (uint32_t)(((1ull << 32) * ((1ull << s) - dv)) / dv + 1);
    }
#ifdef __CUDACC__
    __device__ __forceinline__ uint32_t div(uint32_t n) const
    {
        return (uint32_t)(((uint64_t)__umulhi(n, m) + n) >> s);
    }
#endif
};

// One pass of the adjoint machinery over a range of hyperplanes (sn_adjoint.cu).
struct AdjPass {
    int mode = 0;               // 0 plain, 1 store the angular flux, 2 pair with it
    const float *S = nullptr;   // nodal source [G][C][8]
    const float *psi_inc = nullptr;
    void *face = nullptr;       // face planes to use
    float *phi_oct = nullptr;
    double *leak = nullptr;
    float *psi_blk = nullptr;   // stored angular fluxes of a block of hyperplanes
    int64_t blk_cell0 = 0;      // plane_off of the block's first hyperplane
    double *grad = nullptr;     // dR/dsigma_t [G][C]
};

struct Graphs {
    cudaGraphExec_t exec[2] = {nullptr, nullptr};   // ping-pong parity
    const void *phi_user = nullptr;                 // buffer the graphs were captured for
    int mode = -1;
    bool prof = false;
    uint64_t net_gen = 0;                           // surrogate state the graphs were captured with
};

}  // namespace sn

struct sn_handle_s {
    int dev = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;   // owned stream used for graph capture

    bool fp64 = false;                   // element type of every flux buffer
    size_t esz = 4;                      // sizeof(element)

    int nx = 0, ny = 0, nz = 0;
    double lx = 0, ly = 0, lz = 0, dx = 0, dy = 0, dz = 0;
    int64_t ncell = 0;
    int G = 0, ndir = 0, Do = 0, nplanes = 0;
    std::vector<double> omega, w;          // host copy of the quadrature
    std::vector<int64_t> plane_off;        // [nplanes + 1] offsets into plane_cells

    // device buffers (owned); element type T = float or double (fp64)
    void *sigt = nullptr;        // T[G][C]
    void *sigs = nullptr;        // T[G][C]
    void *q = nullptr;           // T[G][C]
    void *xfer = nullptr;        // T[G][G]
    void *psi_inc = nullptr;     // T[G][6]
    void *dir = nullptr;         // DirData<T>[Do]
    float4 *dir_abs = nullptr;   // [Do] (|Omega_x|, |Omega_y|, |Omega_z|, 0) for the surrogate inputs
    uint32_t *plane_cells = nullptr;  // packed (i',j',k') of every cell, grouped by hyperplane
    uint32_t *plane_pos = nullptr;    // [C] position of primed cell i'+nx(j'+ny k') within its hyperplane
    void *face = nullptr;        // face planes: 4-vectors of T, see sn_sweep.cu
    int64_t face_x = 0, face_y = 0, face_z = 0;  // 4-vector count of each plane set
    int64_t face_in = 0;         // 4-vector offset of the inflow vectors [G][6] after the planes
    void *phi_oct = nullptr;     // T[8][C][G][8] per-octant partial scalar flux
    void *S = nullptr;           // T[G][C][8]
    void *S_b = nullptr;         // T[G][C][8] the next iteration's source (one flux moment)
    int red_iso_per_sm = 0;      // resident blocks of the fused reduction on one SM
    void *phi_b = nullptr;       // T[G][C][8] iteration scratch
    double *acc = nullptr;       // device accumulators (see sn_sweep.cu)
    double *acc_host = nullptr;  // pinned mirror of acc
    int64_t device_bytes = 0;

    double inflow = 0.0;         // boundary inflow of one sweep (host, exact)
    double inflow_box = 0.0;     // the same for the box cells of sn_setup
    double tallies[4] = {0, 0, 0, 0};
    bool tallies_valid = false;

    sn::Graphs graphs;

    // optional CUDA-event timing of the sweep kernels (sn_set_profiling)
    bool prof = false;
    cudaEvent_t ev_sweep[2] = {nullptr, nullptr};
    double prof_ms = 0.0;          // accumulated sweep-kernel time
    int64_t prof_sweeps = 0;       // sweeps timed
    bool prof_pending = false;     // events recorded, elapsed time not yet read

    // adjoint working buffers (allocated on first sn_adjoint_sweep)
    void *adj = nullptr;

    // surrogate network (set by sn_surrogate_train / sn_surrogate_set_weights)
    uint64_t net_gen = 1;        // bumped whenever weights or gate change (graphs bake both in)
    bool has_net = false;
    void *net = nullptr;

    // general hexahedral cells (sn_set_geometry): element records [C][544], node
    // volumes [C][8] and |Omega| of the octant's directions [Do][3], element type T
    void *geom = nullptr;
    void *vnode = nullptr;
    void *omabs = nullptr;
    void *geomB = nullptr;   // [C][8][192] streaming + outflow-face matrices per octant

    // anisotropic scattering (sn_set_scattering_order): Legendre order L, K = (L+1)^2
    // flux moments; sigma_s,n for n = 1..L [L][G][C] and the harmonics [8][Do][K]
    int L = 0, K = 1;
    void *sigs_n = nullptr;
    void *yhat = nullptr;

    // unit tables of the wavefront kernels (sn_sweep_keys.cu)
    void *wave = nullptr;

    // the paper's per-octant networks (sn_octnet_init / sn_octnet_set)
    bool has_octnet = false;
    void *octnet = nullptr;

    std::string err;
};

namespace sn {

// thread-local message for calls without a handle
void set_global_error(const std::string &msg);
sn_status fail(sn_handle h, sn_status s, const std::string &msg);
sn_status cuda_fail(sn_handle h, cudaError_t e, const char *what);

#define SN_CK(h, call)                                         \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return sn::cuda_fail((h), e_, #call); \
    } while (0)

// releases the surrogate network held by a handle (sn_ann.cu)
void free_net(sn_handle h);
// the per-octant networks (sn_octnet.cu): release, folded weights [8][288] for the
// sweep, batch evaluation of one-cell problems
void free_octnet(sn_handle h);
const float *octnet_folded(sn_handle h);
sn_status launch_octnet_cells(sn_handle h, const float *in27, float *psi, int64_t n, cudaStream_t st);

// kernels launched by several translation units (element type from h->fp64)
sn_status launch_sweep(sn_handle h, const void *S, void *phi_oct, sn_solve_mode mode, cudaStream_t st);
sn_status reduce_configure(sn_handle h);
sn_status launch_reduce(sn_handle h, const void *phi_old, void *phi_new, const void *S, void *S_next, bool norms,
                        cudaStream_t st);
sn_status launch_source(sn_handle h, const void *phi, void *S, cudaStream_t st);
// anisotropic scattering (sn_aniso.cu, sn_sweep.cu)
sn_status launch_source_moments(sn_handle h, const void *phi, void *S, cudaStream_t st);
uint32_t sweep_smem_bytes(sn_handle h, int K);
sn_status launch_cells_f32(const float *in27, float *psi, int64_t n, bool refine, cudaStream_t st);
// surrogate sweep (sn_ann.cu): every hyperplane of one sweep, FP32 handles only
// ann_mode: 0 network only, 1 residual gate, 2 frozen gate (ANN_* of sn_ann.cu)
sn_status launch_sweep_ann(sn_handle h, const float *S, float *phi_oct, int ann_mode, cudaStream_t st);
bool ann_frozen(sn_handle h);
// the key sweep (sn_sweep_keys.cu): FP32 elimination on box cells, isotropic scattering
bool key_sweep_ok(sn_handle h);
sn_status launch_sweep_keys(sn_handle h, const float *S, float *phi_oct, bool refine, cudaStream_t st);
sn_status launch_sweep_net_keys(sn_handle h, const float *S, float *phi_oct, cudaStream_t st);
sn_status build_wave(sn_handle h);
// Host tables of the hyperplanes i'+j'+k' = s (sn_setup.cu): off [nplanes + 1]
// offsets, cells [C] packed i' | j' << 10 | k' << 20 listed by (k', j', i') within a
// hyperplane, pos [C] (by linear cell index) the cell's place in its hyperplane.
void hyperplane_tables(int nx, int ny, int nz, std::vector<int64_t> &off, std::vector<uint32_t> &cells,
                       std::vector<uint32_t> &pos);
// Host: the wavefront unit records of the key sweeps (sn_sweep_keys.cu) for a GPU
// with nsm SMs; false when the mesh is left to the per-hyperplane launches.
bool wave_plan(int nx, int ny, int G, int Do, int nsm, const std::vector<int64_t> &off,
               const std::vector<uint32_t> &cells, const std::vector<uint32_t> &pos, std::vector<int4> &units,
               std::vector<int4> &uplane);
sn_status launch_leak_keys(sn_handle h, cudaStream_t st);
void free_wave(sn_handle h);
struct WaveCtl;
WaveCtl wave_ctl(sn_handle h);
// zero the surrogate's fallback / timeout counters (stream-ordered)
sn_status reset_ann_counters(sn_handle h, cudaStream_t st);
sn_status check_ann_timeouts(sn_handle h);
sn_status launch_planes_adjoint(sn_handle h, const AdjPass &p, int s0, int s1, cudaStream_t st);
void free_adjoint(sn_handle h);
int num_sms();

// accumulator slots in h->acc
enum AccSlot {
    ACC_LEAK = 0,      // boundary leakage of the sweep
    ACC_COLL = 1,      // collisions sum sigma_t int phi
    ACC_SRC = 2,       // emission 4 pi int S
    ACC_DMAX = 3,      // max |phi_new - phi_old| (bit pattern, non-negative double)
    ACC_PMAX = 4,      // max |phi_new|
    ACC_MEAN = 5,      // sum over (g, c) of |dphi_bar| / |phi_bar|
    ACC_MEANN = 6,     // number of terms in ACC_MEAN
    ACC_FLAG = 7,      // non-zero: a non-finite flux value was seen
    ACC_HARVEST = 8,   // sn_harvest: number of solves picked (unsigned 64-bit)
    ACC_RESP = 9,      // sn_response: sum resp * phi
    ACC_ABORT = 10,    // non-zero: a bounded wait of the wavefront sweep gave up
    ACC_COUNT = 11
};

}  // namespace sn

/*
 * sn.h -- C ABI of the GB300 (sm_103a) DFEM S_n transport sweep library.
 *
 * Method: Tano & Ragusa, "Acceleration of Radiation Transport Solves Using
 * Artificial Neural Networks" (arXiv:1906.04017).  Equation numbers are the
 * paper's, counted in order of appearance: (1) transport equation, (2) total
 * source, (8)-(9) discrete ordinates, (10) inflow condition, (11) DFEM trial
 * expansion, (12)-(13) discrete system, (14) per-cell system A psi = b,
 * (15)-(18) the network and its activations, (19) training loss, (20) error
 * metric, (21) source-iteration change.
 *
 * Conventions shared by every call
 *  - Mesh: nx x ny x nz uniform axis-aligned box cells on [0,lx]x[0,ly]x[0,lz];
 *    cell c = i + nx (j + ny k).  Tri-linear (Q1) DFEM, 8 nodes per cell,
 *    local node n = a + 2b + 4c (x fastest), node n of cell (i,j,k) sits at
 *    ((i+a) dx, (j+b) dy, (k+c) dz).
 *  - Scalar-flux and source arrays are [G][ncell][8] FP32, node-fastest.
 *  - Directions are ordered octant-major (octant bit 0: mu < 0, bit 1: eta < 0,
 *    bit 2: xi < 0); weights sum to 4 pi; phi = sum_d w_d psi_d (Eqs. (9), (13)).
 *  - Device pointers are caller-owned device memory (e.g. torch tensors);
 *    "host" pointers are caller-owned host memory.  The handle owns every
 *    buffer it allocates and frees it in sn_destroy.
 *  - Work is queued on the handle's CUDA stream (sn_setup / sn_set_stream; the
 *    library never synchronises the whole device).  Calls that return host
 *    scalars synchronise that stream before returning, and so do the set-up
 *    calls that copy host arrays (sn_setup, sn_set_geometry,
 *    sn_set_scattering_order, the weight setters): they return with their
 *    copies complete.
 *  - Inputs are validated on the host; a rejected call returns SN_EINVAL and
 *    queues nothing.  sn_last_error() gives the message.  There is no CPU
 *    fallback: without a usable CUDA device calls return SN_ECUDA.
 *  - The library is not thread-safe per handle.
 */
#ifndef SN_GB300_H
#define SN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sn_handle_s *sn_handle;

typedef enum {
    SN_OK = 0,
    SN_EINVAL = 1,    /* bad argument (size, pointer, range, non-finite value)  */
    SN_ENOMEM = 2,    /* device allocation failed                               */
    SN_ECUDA = 3,     /* CUDA runtime error or no device                        */
    SN_ENOCONV = 4,   /* source iteration hit max_it before tol                 */
    SN_ETIMEOUT = 5,  /* a bounded device wait gave up                          */
    SN_ENAN = 6,      /* a non-finite value appeared in the flux                */
    SN_ESTATE = 7     /* call not valid in the handle's state (e.g. no network) */
} sn_status;

/* How the per-cell system (14) is solved. */
typedef enum {
    SN_SOLVE_GE32R = 0,     /* FP32 Gaussian elimination with partial pivoting + one
                               FP32 iterative-refinement step (Sec. 2, after (14))   */
    SN_SOLVE_GE32 = 1,      /* FP32 elimination, no refinement                        */
    SN_SOLVE_ANN = 2,       /* surrogate network only (Sec. 3, Eqs. (15)-(18))        */
    SN_SOLVE_ANN_GATED = 3, /* surrogate, with cells whose residual fails the gate
                               re-solved by SN_SOLVE_GE32R                          */
    SN_SOLVE_GE64 = 4,      /* FP64 elimination with partial pivoting (FP64 handles only) */
    SN_SOLVE_OCTNET = 5,    /* the paper's own per-octant networks (Sec. 3 Eqs. (15)-(18),
                               Sec. 4), FP32 on the CUDA cores; see sn_octnet_*        */
    SN_SOLVE_ANN_FROZEN = 6 /* surrogate with the gate decisions frozen by
                               sn_surrogate_freeze_gate: each (octant, cell, group,
                               direction) keeps the solver the gated sweep chose there,
                               so the source iteration is a fixed linear map          */
} sn_solve_mode;

typedef struct {
    int32_t nx, ny, nz;     /* 1..1023 each                                     */
    double lx, ly, lz;      /* > 0                                              */
} sn_mesh;

typedef struct {
    int32_t order;          /* LQ_N order 2,4,6,8,10,12; or 0 for explicit      */
    int32_t ndir;           /* explicit only: number of directions (8 * n)      */
    const double *omega;    /* explicit only: host [ndir][3], unit vectors      */
    const double *w;        /* explicit only: host [ndir], sum 4 pi             */
} sn_quadrature;

typedef struct {
    int32_t ngroups;        /* G >= 1                                           */
    const double *sigt;     /* host [G][ncell] total cross section, >= 0         */
    const double *sigs;     /* host [G][ncell] scattering out of group g, >= 0   */
    const double *q;        /* host [G][ncell] isotropic emission density       */
    const double *xfer;     /* host [G][G]: fraction of g' scattering into g (row g') */
    const double *psi_inc;  /* host [G][6] isotropic inflow on faces x-,x+,y-,y+,z-,z+
                               (Eq. (10)); NULL = vacuum                        */
} sn_xs;

typedef struct {
    int32_t fp64;           /* 0: FP32 flux buffers (modes GE32R, GE32, ANN, ANN_GATED)
                               1: FP64 flux buffers (mode GE64 only)                     */
} sn_options;

typedef struct {
    int64_t ncell;
    int32_t ndir, ngroups, nplanes;   /* nplanes = nx+ny+nz-2 hyperplanes/octant */
    int32_t dirs_per_octant;
    int64_t solves_per_sweep;         /* ncell * ndir * G                        */
    int64_t device_bytes;             /* device memory held by the handle        */
} sn_info;

/* ---------------------------------------------------------------------------
 * sn_setup: build a problem (Sec. 2: mesh, quadrature (8)-(9), cross sections
 * of (1)-(2), inflow (10)).  Copies the host arrays to the device in the
 * handle's precision (opts->fp64; opts may be NULL = FP32) and allocates the
 * sweep's working buffers.  Every flux and source array later passed to this
 * handle has that element type (float, or double for an FP64 handle).
 * stream: a cudaStream_t (NULL =
 * legacy default stream), borrowed, not owned.  On success *out is a new
 * handle; on failure *out is NULL and the status says why.
 * ------------------------------------------------------------------------- */
sn_status sn_setup(sn_handle *out, const sn_mesh *mesh, const sn_quadrature *quad,
                   const sn_xs *xs, const sn_options *opts, void *stream);

/* Replace the stream later calls are queued on.  When the stream changes, the
 * work already queued on the old one is waited for first (a host wait on that
 * stream), so later calls see its results. */
sn_status sn_set_stream(sn_handle h, void *stream);

sn_status sn_get_info(sn_handle h, sn_info *info);

/* Copy the handle's directions (host [ndir][3]) and weights (host [ndir]). */
sn_status sn_get_quadrature(sn_handle h, double *omega, double *w);

/* ---------------------------------------------------------------------------
 * sn_cell_solve_batch: n independent one-cell problems (the paper's one-cell
 * problem, Sec. 3, and the per-cell system (14)).
 *   in27: device [n][27] FP32 = Omega(3), (dx,dy,dz), sigma_t, S(8), up(12)
 *         S: nodal angular source density (node order above);
 *         up: upwind values on the inflow face of each axis (the face at
 *         coordinate 0 if Omega_a >= 0, else at the cell size): x-face then
 *         y-face then z-face, 4 each, in-face order x: b+2c, y: a+2c, z: a+2b.
 *   psi:  device [n][8] FP32 nodal angular flux (output).
 * mode SN_SOLVE_ANN / SN_SOLVE_ANN_GATED need a handle with a trained or
 * loaded network; the GE modes accept h = NULL.  stream: cudaStream_t.
 * Cell sizes must be > 0 and sigma_t >= 0 (not checked per problem on the
 * device: the caller owns the data).
 * ------------------------------------------------------------------------- */
sn_status sn_cell_solve_batch(sn_handle h, const float *in27, float *psi, int64_t n,
                              sn_solve_mode mode, void *stream);

/* FP64 variant of the GE solve (same layout, double precision, device). */
sn_status sn_cell_solve_batch_f64(const double *in27, double *psi, int64_t n, void *stream);

/* ---------------------------------------------------------------------------
 * sn_sweep: one transport sweep of every direction and group (Sec. 2, after
 * (14)) for the isotropic nodal source S (device [G][ncell][8] of the
 * handle's element type, angular
 * density, i.e. already divided by 4 pi); writes phi (device [G][ncell][8]).
 * Hyperplane-wavefront order (a cell after its three upwind neighbours).  FP32
 * handles with box cells and isotropic scattering run the whole sweep as one
 * persistent launch whose work units (hyperplane, octant, tile of (cell, group)
 * keys; sn_wave_plan) each wait only for their upwind units; other handles run one
 * launch per hyperplane with all its octants, directions and groups.  Balance
 * tallies of this sweep are kept for sn_get_balance; reading them synchronises the
 * handle's stream before the call returns.  S and phi must not overlap.  The GE
 * modes, SN_SOLVE_ANN and SN_SOLVE_OCTNET give the same bits on every run, and so
 * do the gated modes on the persistent launch (the rows the gate rejects are solved
 * by elimination inside their unit and added in direction order); on the
 * per-hyperplane launches the gated modes re-solve the rejected rows between
 * hyperplanes and add them to the flux with atomics, so the last bits may differ
 * from run to run.
 * ------------------------------------------------------------------------- */
sn_status sn_sweep(sn_handle h, const void *S, void *phi, sn_solve_mode mode);

/* ---------------------------------------------------------------------------
 * sn_source_iterate: scattering source iteration (Sec. 2, after (7)):
 * S = (sum_g' xfer[g'][g] sigs_g' phi_g' + q_g) / (4 pi) -> sweep -> phi,
 * Jacobi in groups, until change_max <= tol or max_it sweeps.
 *   phi: device [G][ncell][8]; in: initial guess, out: last iterate.
 *   iters: sweeps done; change_max: max |phi_n - phi_{n-1}| / max |phi_n|
 *   (FP64 on the device); change_mean: the mean relative change of Eq. (21)
 *   over cells and groups (cell-averaged flux).  Any output pointer may be NULL.
 * Returns SN_OK on convergence, SN_ENOCONV if max_it was reached, SN_ENAN if
 * the flux became non-finite.  use_graph != 0 replays one CUDA graph per
 * iteration.
 * ------------------------------------------------------------------------- */
sn_status sn_source_iterate(sn_handle h, double tol, int32_t max_it, sn_solve_mode mode,
                            void *phi, int32_t *iters, double *change_max,
                            double *change_mean, int32_t use_graph);

/* One SN_SOLVE_GE32R sweep from S (device [G][ncell][8]) that also writes about cap
 * of its solves, picked by a seeded hash, as one-cell problems (device [cap][27],
 * layout of sn_cell_solve_batch) in the positive-octant frame the solve uses: the
 * training data of a surrogate for this family of problems, drawn by the library's
 * own elimination.  *n_out: how many were written (<= cap).  Synchronises. */
sn_status sn_harvest(sn_handle h, const float *S, float *in27, int64_t cap, uint64_t seed, int64_t *n_out);

/* The isotropic nodal source of the source iteration for a given flux (Eqs. (2),
 * (6), P_0 term): S_g = (sum_g' xfer[g'][g] sigs_g' phi_g' + q_g) / (4 pi);
 * phi, S: device [G][ncell][8] of the handle's element type.  Asynchronous. */
sn_status sn_source(sn_handle h, const void *phi, void *S);

/* ---------------------------------------------------------------------------
 * sn_adjoint_sweep: gradients of a detector response R = sum resp * phi with
 * respect to the per-cell, per-group sigma_t, sigma_s (scattering out of the group)
 * and q (not in the paper: the discrete adjoint of the system of Sec. 2, (12)-(14),
 * and of the source iteration).  FP32 handles only.
 *   phi:  device [G][ncell][8] converged forward flux (sn_source_iterate);
 *   resp: device [G][ncell][8] dR/dphi (e.g. V/8 at every node of the detector cells);
 *   Lam:  device [G][ncell][8] out, adjoint scalar flux sum_d lambda_d;
 *   dR_dsigt, dR_dsigs, dR_dq: device FP64 [G][ncell] out.
 * Adjoint source iteration to tol (max-norm relative change) in at most max_it
 * sweeps (*iters, may be NULL), then a final pass that pairs every forward and
 * adjoint angular flux for dR/dsigma_t, recomputing the forward sweep from face
 * planes checkpointed every ceil(sqrt(nplanes)) hyperplanes (no full angular flux
 * is stored).  Synchronises the stream.  SN_ENOCONV if max_it was reached (the
 * gradients are still written).
 * ------------------------------------------------------------------------- */
sn_status sn_adjoint_sweep(sn_handle h, const float *phi, const float *resp, double tol, int32_t max_it,
                           float *Lam, double *dR_dsigt, double *dR_dsigs, double *dR_dq, int32_t *iters);

/* Detector response R = sum over groups, cells and nodes of resp * phi (the
 * functional whose gradients sn_adjoint_sweep returns; FP64 products and sum).
 * phi, resp: device [G][ncell][8] in the handle's element type (float, or double
 * for an FP64 handle); *R written on the host.  Synchronises the stream. */
sn_status sn_response(sn_handle h, const void *phi, const void *resp, double *R);

/* Balance tallies of the last sweep, FP64, particles per unit time:
 * tallies[0] leakage through the boundary, [1] collisions sum sigma_t int phi,
 * [2] emission 4 pi int S, [3] inflow through the boundary.  For any sweep
 * [0] + [1] = [2] + [3] up to round-off (weight 1 in the weak form). */
sn_status sn_get_balance(sn_handle h, double *tallies);

/* ---------------------------------------------------------------------------
 * Surrogate network (Sec. 3, Eq. (15): one hidden layer, here 27 inputs, 64 ReLU
 * units, 8 linear outputs; loss of Eq. (19); Adam).  The network lives in the
 * handle.  Parameters are 2312 FP32 values: W1[64][27] row-major, b1[64],
 * W2[8][64], b2[8].  Inputs (27) are built from a one-cell problem after it is
 * mirrored into the positive octant (one network serves every octant):
 *   x[0:3] = 2|Omega_a| - 1, x[3:6] = (ln h_a + 1.15)/1.15,
 *   x[6] = ln(max(sigma_t, 1e-6))/4.5, x[7:15] = S/s, x[15:27] = up/s,
 *   s = max(max|S|, max|up|);
 * the network predicts psi_canonical / s (s = 0 gives psi = 0).  Inference runs
 * in BF16 on the tcgen05 tensor cores with FP32 accumulation; the gate accepts a
 * prediction when ||b - A psi||_2 <= tau ||b||_2 for the cell's system (14),
 * otherwise the cell is re-solved by SN_SOLVE_GE32R.
 * ------------------------------------------------------------------------- */

/* Features [n][27] and targets [n][8] (device FP32) of n one-cell problems in27
 * (device [n][27], layout of sn_cell_solve_batch); targets are the canonical
 * FP32 elimination solution divided by s. */
sn_status sn_surrogate_prepare(const float *in27, int64_t n, float *feat, float *targ, void *stream);

/* Uniform(-1/sqrt(fan_in), +1/sqrt(fan_in)) initialisation from a seed; resets Adam. */
sn_status sn_surrogate_init(sn_handle h, uint64_t seed);

/* Host [2312] FP32 parameters in / out; set resets Adam. */
sn_status sn_surrogate_set_weights(sn_handle h, const float *params);
sn_status sn_surrogate_get_weights(sn_handle h, float *params);

/* Gate threshold tau >= 0 (default 0.01). */
sn_status sn_surrogate_set_gate(sn_handle h, float tau);

/* Loss (19) averaged over n rows and its gradient (host [2312]) at the current
 * weights; FP32 on the device, per-block partial sums added in a fixed order. */
sn_status sn_surrogate_grad(sn_handle h, const float *feat, const float *targ, int64_t n, float *grad,
                            double *loss);

/* steps Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) on batches of `batch` rows;
 * batch k takes rows [(k*batch) mod nrows, ...) in order, wrapping.  last_loss:
 * the loss of the last batch (may be NULL). */
sn_status sn_surrogate_fit(sn_handle h, const float *feat, const float *targ, int64_t nrows, int32_t steps,
                           int32_t batch, float lr, double *last_loss);

/* Mean absolute error (over rows and the 8 outputs) of the FP32 network. */
sn_status sn_surrogate_eval(sn_handle h, const float *feat, const float *targ, int64_t n, double *mae);

/* Label n one-cell problems (device in27) with the library's elimination, keep the
 * last n_test for testing, initialise from seed and fit; train / test MAE out. */
sn_status sn_surrogate_train(sn_handle h, const float *in27, int64_t n, int64_t n_test, int32_t steps,
                             int32_t batch, float lr, uint64_t seed, double *train_mae, double *test_mae);

/* psi (device [n][8]) of n one-cell problems by the tensor-core network; gated != 0
 * applies the residual gate with elimination fallback; *n_fallback (may be NULL)
 * receives the number of fallbacks.  Synchronises the handle's stream.
 * SN_ETIMEOUT if a tensor-core completion wait gave up. */
sn_status sn_surrogate_apply(sn_handle h, const float *in27, float *psi, int64_t n, int32_t gated,
                             int64_t *n_fallback);

/* Self-test of the failure path of the bounded device waits (not in the paper):
 * one CTA sets up like a surrogate kernel (an mbarrier and tensor-memory columns)
 * and waits, for at most limit_cycles SM cycles (1..2^31), on an mbarrier phase
 * that nothing completes.  The wait gives up, the CTA raises its abort flag, frees
 * its tensor memory and is counted as timed out, as a surrogate sweep's CTA would
 * be; the call then returns SN_ETIMEOUT, and the handle and the CUDA context stay
 * usable.  Synchronises the handle's stream.  (The waits of the sweeps use 2^31.) */
sn_status sn_selftest_wait(sn_handle h, int64_t limit_cycles);

/* Freeze the residual gate (not in the paper; the gate routes cells the network
 * fails back to elimination): one SN_SOLVE_ANN_GATED sweep from S (device
 * [G][ncell][8]) records, for every (octant, cell, group, direction), whether the
 * network's prediction passed the gate; later SN_SOLVE_ANN_FROZEN sweeps and source
 * iterations take the network there and elimination elsewhere without testing the
 * residual again.  Rows decided the same way give the same flux as the gated sweep
 * from the same source.  A change of the weights or of the threshold drops the
 * frozen decisions (SN_ESTATE for SN_SOLVE_ANN_FROZEN until the next freeze).  The
 * decisions take one bit a row (8 ncell G ndir/8 bits, allocated on first use; more
 * than 2^32 rows: SN_EINVAL).  FP32 handles on box cells with isotropic scattering.
 * Synchronises; sn_surrogate_stats then gives the number of rows sent to elimination. */
sn_status sn_surrogate_freeze_gate(sn_handle h, const float *S);

/* Surrogate counters of the last sweep (sn_sweep) or of the last iteration of
 * sn_source_iterate in an ANN mode, or of the last sn_surrogate_apply: cells sent
 * back to elimination by the gate, and CTAs that gave up a bounded tensor-core
 * wait (non-zero means the results of that call are invalid). */
sn_status sn_surrogate_stats(sn_handle h, int64_t *fallbacks, int64_t *timeouts);

/* CUDA-event timing of the sweep kernels.  With profiling on, every directly
 * launched sweep (sn_sweep, or sn_source_iterate with use_graph = 0) records an
 * event before its first hyperplane kernel and after its last one on the
 * handle's stream; graph replays are not timed.  sn_get_profile returns the
 * summed elapsed milliseconds and the number of sweeps timed (reset != 0 clears
 * both).  Events add no synchronisation; the times are read at the
 * synchronisations the library already makes. */
sn_status sn_set_profiling(sn_handle h, int32_t enable);
sn_status sn_get_profile(sn_handle h, double *sweep_ms, int64_t *sweeps, int32_t reset);

/* sn_wave_plan: the work units of the wavefront sweeps (the sweep order of Sec. 2,
 * after (14): a cell is solved after its three upwind neighbours, so the cells of
 * hyperplane s = i'+j'+k' of the canonical octant are independent of each other).
 * Host only, no GPU call: the records a float handle of an nx x ny x nz box mesh with
 * G groups and Do directions per octant builds on a GPU with nsm SMs, for inspection
 * and tests.
 *   A key is (cell, group): its index on hyperplane s is (place of the cell on s) x G
 *   + g, the cells of s listed by (k', j', i').  A unit is one tile of keys of one
 *   hyperplane and one octant; units are numbered by (s, octant, tile).
 *   units [nunits][4]: first key of the tile; s | octant << 12 | lch << 15 (the tile
 *     holds 128 >> lch keys, and each key's directions are split in 2^lch chunks:
 *     the fewest, at most 8 and at most Do, for which 8 x keys of s x 2^lch reaches
 *     nsm x 3 x 128 thread slots); first unit and count of the first range of units
 *     the tile waits for.
 *   uplane [nunits][4]: first cell of hyperplane s in the hyperplane cell list; keys
 *     on s (cells x G); first unit and count of the second range (count 0: none).
 *   Both ranges lie in the units of hyperplane s - 1 of the same octant and together
 *   hold every tile that has a key of an upwind neighbour of a cell of the tile.
 * *nunits receives the number of units, 0 where the mesh is left to one launch per
 * hyperplane (2^30 units or more, or more than 4095 hyperplanes).  With units and
 * uplane both NULL the call only sizes; otherwise both must hold 4 x cap int32 and
 * cap >= *nunits.  SN_EINVAL for sizes outside 1..1023 cells per axis, 1..1024
 * groups, 1..64 directions per octant, nsm < 1, or too small a cap. */
sn_status sn_wave_plan(int32_t nx, int32_t ny, int32_t nz, int32_t G, int32_t Do, int32_t nsm, int32_t *units,
                       int32_t *uplane, int64_t cap, int64_t *nunits);

/* ---------------------------------------------------------------------------
 * sn_set_scattering_order: anisotropic scattering (Sec. 2, Eqs. (3)-(8)).  The
 * differential scattering cross section is expanded in Legendre polynomials up to
 * order L (0..SN_MAX_SCATTERING_ORDER): sigma_s(mu0) = sum_n (2n+1)/(4 pi)
 * sigma_{s,n} P_n(mu0), sigma_{s,0} being the handle's sigma_s.  The source of
 * direction Omega is then sum_{n,m} sigma_{s,n} Y_nm(Omega) phi_nm (real orthonormal
 * harmonics, flux moments phi_nm = sum_d w_d Y_nm(Omega_d) psi_d).
 *   sigs_n: host [L][G][ncell] FP64, sigma_{s,n} for n = 1..L (NULL when L = 0);
 *           group transfer as for sigma_s (xfer[g'][g] applies to every order).
 * After the call every flux and source array of the handle (sn_sweep, sn_source,
 * sn_source_iterate) holds K = (L+1)^2 moments in the layout [G][K][ncell][8]:
 * moment k = n^2 + n + m (degree n, order m) of sqrt(4 pi) Y, so moment 0 is the
 * scalar flux (source) of the isotropic layout and L = 0 restores it.  Real
 * harmonics: Y_n0 = N_n0 P_n(cos theta), Y_nm = sqrt(2) N_nm P_n^m(cos theta)
 * cos(m phi) and Y_n,-m = sqrt(2) N_nm P_n^m(cos theta) sin(m phi) for m > 0,
 * N_nm^2 = (2n+1)/(4 pi) (n-m)!/(n+m)!, P_n^m without the Condon-Shortley sign,
 * theta from the z axis, phi in the x-y plane.  Source moments:
 * Sh_k = (sum_g' xfer[g'][g] sigma_{s,n(k),g'} phih_k,g' + [k = 0] q) / (4 pi).
 * Modes: SN_SOLVE_GE32R, SN_SOLVE_GE32, SN_SOLVE_GE64; the surrogate modes, the
 * adjoint, sn_response and sn_harvest return SN_EINVAL while L > 0.  SN_EINVAL also
 * when the moments of a sweep tile do not fit in shared memory (few directions per
 * octant, e.g. LQ_2 with L = 3).  Reallocates the handle's flux buffers; drops
 * captured iteration graphs.  Synchronises the handle's stream.
 * ------------------------------------------------------------------------- */
#define SN_MAX_SCATTERING_ORDER 3
sn_status sn_set_scattering_order(sn_handle h, int32_t L, const double *sigs_n);

/* ---------------------------------------------------------------------------
 * sn_set_geometry: general hexahedral cells (the cells' shape change of Sec. 2's
 * closing remarks).  The mesh keeps its nx x ny x nz structured topology; xyz
 * (host FP64 [(nx+1)(ny+1)(nz+1)][3], vertex (i,j,k) at i + (nx+1)(j + (ny+1)k))
 * places its vertices, and cell (i,j,k) is the trilinear image of the unit cube on
 * its 8 vertices (node n = a + 2b + 4c at vertex (i+a, j+b, k+c)), with the same
 * trilinear functions as DFEM basis.  Element matrices (mass, streaming, face area
 * vector matrices) are computed exactly on the device (3-point Gauss per axis).  The
 * sweep keeps the box mesh's octant wavefront, which needs, for every quadrature
 * direction, Omega . n to keep on each face the sign it has on a box cell; that and
 * a positive Jacobian are checked at the quadrature points (SN_EINVAL otherwise).
 * The balance tallies use each node's own volume.  NULL restores the box cells.
 * Modes: SN_SOLVE_GE32R, SN_SOLVE_GE32, SN_SOLVE_GE64; not combined with
 * anisotropic scattering, the surrogates, the adjoint or harvesting (SN_EINVAL).
 * Drops captured iteration graphs.  Synchronises the handle's stream.
 * ------------------------------------------------------------------------- */
sn_status sn_set_geometry(sn_handle h, const double *xyz);

/* ---------------------------------------------------------------------------
 * The paper's own surrogate: one network per octant of directions (Sec. 4),
 * 26 inputs -> 8 tanh units -> 8 ELU outputs (Sec. 3, Eqs. (15), (17), (18)).
 *
 * Network o serves the directions of octant o (bit 0: mu < 0, bit 1: eta < 0,
 * bit 2: xi < 0) and reads, in the problem's physical frame and in this order,
 *   I[0:12]  the upwind face values up(12) of the one-cell problem (x, y, z face),
 *   I[12:14] mu, eta (Omega_x, Omega_y),  I[14:22] the nodal sources S(8),
 *   I[22]    sigma_t,  I[23:26] dx, dy, dz,
 * each scaled by Eq. (16): x_j = (I_j - 0.27 (lo_j + hi_j) / 2) / |hi_j - lo_j|,
 * with a-priori ranges lo, hi [8][26] per octant (host FP64).  Then
 * h = tanh(W1 x + b1), z = W2 h + b2, psi_n = z_n (z_n >= 0) or
 * beta (e^{z_n} - 1), beta = 0.1 max |up|: the angular flux itself, physical
 * node order.  Parameters: host FP32 [8][288], per octant W1[8][26] row-major,
 * b1[8], W2[8][8], b2[8].  mask [8][288]: 1 = connection kept, 0 = dropped
 * (held at 0 by training); biases are not connections.
 *
 * Training data: in27 blocks [8][m][27] (device; rows of block o must lie in
 * octant o, else SN_EINVAL), turned into features [8 m][27] (the 26 scaled
 * inputs, then beta) and targets [8 m][8] (FP32 elimination, GE32R).  Loss:
 * Eq. (19) per octant, mean over its m rows (lambda 0.2, gamma 10 and 0.01).
 * Training is full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8), one step per
 * epoch, all 8 networks at once.  Evaluation in sweeps (SN_SOLVE_OCTNET) and in
 * sn_octnet_apply / sn_cell_solve_batch: FP32 on the CUDA cores; tanh(a) as
 * 1 - 2 / (1 + e^{2a}) with the fast exponential (absolute error ~1e-6).
 * ------------------------------------------------------------------------- */

/* Glorot-uniform weights (seeded), zero biases, no dropped connection; sets the
 * ranges; resets Adam. */
sn_status sn_octnet_init(sn_handle h, const double *lo, const double *hi, uint64_t seed);

/* Load parameters (and optionally a mask; NULL = keep every connection) and, if
 * lo and hi are non-NULL, new ranges (else the handle's current ones).  Dropped
 * entries are zeroed.  Resets Adam. */
sn_status sn_octnet_set(sn_handle h, const float *params, const float *mask, const double *lo, const double *hi);

/* Copy out parameters and mask (host [8][288]; either pointer may be NULL). */
sn_status sn_octnet_get(sn_handle h, float *params, float *mask);

/* Features and targets (device, layouts above) of 8 m one-cell problems. */
sn_status sn_octnet_prepare(sn_handle h, const float *in27, int64_t m, float *feat, float *targ);

/* Per-octant loss (host [8]) and gradient (host [8][288], dropped entries not
 * zeroed) at the current parameters over all m rows of each octant. */
sn_status sn_octnet_grad(sn_handle h, const float *feat, const float *targ, int64_t m, float *grad, double *loss);

/* `steps` full-batch Adam steps (Adam state continues from the last init, set,
 * fit or prune); loss: host [8] loss of the last step's gradient (may be NULL). */
sn_status sn_octnet_fit(sn_handle h, const float *feat, const float *targ, int64_t m, int32_t steps, float lr,
                        double *loss);

/* Per-octant mean absolute and mean squared error over rows and outputs (host [8]
 * each; either may be NULL). */
sn_status sn_octnet_eval(sn_handle h, const float *feat, const float *targ, int64_t m, double *mae, double *mse);

/* Connection dropping (Sec. 3), all octants in step: drop each network's remaining
 * connection of smallest magnitude (lowest index on ties), retrain `retrain_steps`
 * full-batch Adam steps from a fresh Adam state, keep the drop while the training
 * MSE stays within (1 + tol) of the network's MSE before the first drop, else undo
 * it and stop that network; at most max_drops drops a network.  dropped: host [8]
 * drops kept (may be NULL). */
sn_status sn_octnet_prune(sn_handle h, const float *feat, const float *targ, int64_t m, int32_t retrain_steps,
                          float lr, double tol, int32_t max_drops, int32_t *dropped);

/* psi (device [n][8], physical node order) of n one-cell problems (device in27,
 * layout of sn_cell_solve_batch) by the network of each problem's octant. */
sn_status sn_octnet_apply(sn_handle h, const float *in27, float *psi, int64_t n);

/* ---------------------------------------------------------------------------
 * sn_surrogate_grad_noalloc: the loss and gradient of sn_surrogate_grad, for
 * callers that cannot allocate device memory -- work issued while a stream is
 * being captured in global mode (cudaMalloc is refused there), callers that own a
 * fixed, pre-assigned pool of device memory, and latency-bound loops that must not
 * pay the device-wide synchronisation of cudaMalloc / cudaFree.  The paper has no
 * counterpart; this is a library convenience.
 *   params: device [2312] FP32 weights (layout of sn_surrogate_set_weights);
 *   feat, targ: device [n][27], [n][8] (sn_surrogate_prepare);
 *   grad: device [2312] FP32 out; loss: device [1] FP64 out (batch mean of Eq. (19)).
 * No handle, no allocation: the per-block partial sums live in one fixed array
 * of the library (2.37 MB on every GPU that loads it, kept until exit), which caps
 * n at 32768 rows (SN_EINVAL above).  The first call on a device looks the array
 * up (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture.  The address is kept until the process exits: after a device reset
 * (cudaDeviceReset or a primary-context reset) it is stale, and this entry point
 * must not be called again in that process.  All calls share the array: calls that overlap on the GPU (other
 * streams or threads on the same device) race; calls on one stream are ordered.
 * Asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream).
 * ------------------------------------------------------------------------- */
sn_status sn_surrogate_grad_noalloc(const float *params, const float *feat, const float *targ, int64_t n,
                                    float *grad, double *loss, void *stream);

/* Status text, and the last error message recorded on a handle (h may be NULL
 * for the last error of a call without a handle, per thread). */
const char *sn_status_string(sn_status s);
const char *sn_last_error(sn_handle h);

void sn_destroy(sn_handle h);

#ifdef __cplusplus
}
#endif

#endif /* SN_GB300_H */

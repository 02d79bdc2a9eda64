"""Throughput of the DFEM S_n transport sweep on one GB300 (or N replicas).

A step is one source iteration of the whole hot path on the blocked_64 workload
(64^3 cells on a 10^3 box, LQ_8 = 80 directions, 8 groups, blocked lognormal
opacity): source build -> hyperplane-wavefront sweep (8x8 DFEM system per cell,
direction and group, FP32 Gaussian elimination with partial pivoting and one
refinement step) -> octant reduction with FP64 change norms.  The metric is
cell*direction*group solves per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --impl reference the FP64 CPU oracle is timed on a bounded sample of the
same workload on the host cores.  Under torchrun (N > 1) every rank runs an
independent replica (the path has no data exchange between GPUs).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Sn sweep cell*dir*group solves/s (GE form, FP32 GE + 1 refinement step)"
UNIT = "solves/s"
# algorithmic FP32 flops of one solve, the fixed count of the GE form: assembly of A
# (64 entries x 4 terms x 2) 512 + right-hand side (M S and three inflow faces) 224 +
# LU with partial pivoting sum_{m=1..7} (m + 2 m^2) = 308 + two triangular solves 128 +
# one refinement step (residual 128, solves 128, update 8) 264 + flux accumulation 16
FLOPS_PER_SOLVE = 1450
# algorithmic HBM bytes of one solve: 12 inflow + 12 outflow face floats
BYTES_PER_SOLVE = 96
# DRAM bytes (read + write) per solve of the wavefront sweep kernel (sweep_ge_wave<true>)
# from one full-set ncu capture of a whole blocked_64 sweep (6.391 GB read + 6.194 GB
# written over 167,772,160 solves); None once that kernel changes
DRAM_BYTES_PER_SOLVE_NCU = 75.01
FP32_LANES_PER_SM = 128
N_SM = 152
# this library's kernels in one source-iteration step: the sweep kernel, the
# boundary-leakage sum, the octant reduction (which also builds the next source); one
# source build before the first step of a source_iterate call
LAUNCHES_PER_STEP = 3


def workload_config():
    return {"workload": "blocked_64: 64^3 cells, 10^3 box, LQ_8 (80 dirs), 8 groups, sigma_t lognormal(0,1) "
                        "on 8^3 blocks, scattering ratio U[0.3,0.9], downscatter-only, q=1 in a 16^3 box",
            "mode": "ge32r", "step": "source build + full sweep + octant reduction + FP64 norms",
            "l2": "working set > L2 (per-octant flux 537 MB, face planes 126 MB), no flush"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings over all ranks (the slowest replica
    sets the job's time)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(world_size, solves_per_step, steps, ms):
    """Whole-job solves/s of `world_size` independent replicas, each doing `steps`
    steps of `solves_per_step` solves, the slowest finishing after `ms`."""
    return world_size * solves_per_step * steps / (ms / 1e3)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            self.f.close()
            os.unlink(self.f.name)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        with open(self.f.name) as fh:
            lines = fh.readlines()
        os.unlink(self.f.name)
        return clock_summary(lines)


def clock_summary(lines):
    """Median SM clock, the maximum clock and the throttle reasons seen in nvidia-smi
    rows of Clocks.Q (csv, noheader, nounits): a reason counts when any sample shows
    it "Active"; fields that are not numbers ("[N/A]") are skipped."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


def oracle_sweep_timed(k_dirs=None):
    """One FP64 oracle sweep of blocked_64 from the seeded source of the parity check
    (uniform [0, 1], rounded to FP32 as the device sees it), all 8 groups in parallel on
    the host cores, over the first k_dirs directions (all 80 by default).  Returns
    (S [G, C, 8] FP32, phi [G, C, 8] FP64, seconds, solves)."""
    import oracle
    from paper_1906_04017_gb300 import workloads
    wl = workloads.blocked_64()
    P = oracle.OracleProblem(wl)
    S = np.random.default_rng(0).uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32)
    k = P.ndir if k_dirs is None else k_dirs
    t0 = time.perf_counter()
    phi, _ = P.sweep(S.astype(np.float64), dirs=(0, k))
    dt = time.perf_counter() - t0
    return S, phi, dt, P.ncell * P.G * k


def single_thread_rate(seconds=2.0):
    """Solves/s of the FP64 oracle on one thread: one group, the first directions."""
    import oracle
    from paper_1906_04017_gb300 import workloads
    P = oracle.OracleProblem(workloads.blocked_64())
    S = np.random.default_rng(0).uniform(0.0, 1.0, (P.G, P.ncell, 8))
    t0 = time.perf_counter()
    P.sweep(S, groups=(0, 1), dirs=(0, 1))
    t1 = time.perf_counter() - t0
    k = int(max(1, min(P.ndir, seconds / max(t1, 1e-3))))
    t0 = time.perf_counter()
    P.sweep(S, groups=(0, 1), dirs=(0, k))
    return P.ncell * k / (time.perf_counter() - t0), k


def cpu_baseline_from(dt, solves, k_dirs):
    import oracle
    st, k1 = single_thread_rate()
    return {"value": solves / dt, "unit": UNIT, "cores": min(8, oracle.num_threads()), "kind": "oracle",
            "single_thread_value": st,
            "sample": "blocked_64, one sweep of all 8 groups x %d of 80 directions (%d solves, %.1f s), FP64, "
                      "groups in parallel; single thread: group 0 x %d directions" % (k_dirs, solves, dt, k1)}


def parity_report(phi, ref):
    """Element-by-element comparison of the device flux with the FP64 oracle's
    (arrays [G, C, 8]): the per-group max-norm relative error, the pointwise relative
    error where |ref| >= 1% of the group maximum, and the pointwise error floored at
    1e-8 and 1e-6 of the group maximum (max and mean)."""
    phi = np.asarray(phi, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = {"maxnorm_rel": 0.0, "point_rel_at_1pct": 0.0, "point_rel_floored_1e-8max": 0.0,
           "point_rel_floored_1e-6max": 0.0, "mean_rel_floored_1e-8max": 0.0}
    means = []
    for g in range(ref.shape[0]):
        m = np.abs(ref[g]).max()
        d = np.abs(phi[g] - ref[g])
        a = np.abs(ref[g])
        out["maxnorm_rel"] = max(out["maxnorm_rel"], float(d.max() / m))
        sel = a >= 1e-2 * m
        out["point_rel_at_1pct"] = max(out["point_rel_at_1pct"], float((d[sel] / a[sel]).max()))
        r8 = d / (a + 1e-8 * m)
        out["point_rel_floored_1e-8max"] = max(out["point_rel_floored_1e-8max"], float(r8.max()))
        out["point_rel_floored_1e-6max"] = max(out["point_rel_floored_1e-6max"], float((d / (a + 1e-6 * m)).max()))
        means.append(float(r8.mean()))
    out["mean_rel_floored_1e-8max"] = float(np.mean(means))
    return out


def cpu_baseline(seconds_target=15.0):
    """The FP64 oracle timed on a bounded sample of the same workload (all groups,
    the first k directions of one sweep from a fixed source) on the host cores."""
    import oracle
    from paper_1906_04017_gb300 import workloads
    P = oracle.OracleProblem(workloads.blocked_64())
    S = np.random.default_rng(0).uniform(0.0, 1.0, (P.G, P.ncell, 8))
    t0 = time.perf_counter()
    P.sweep(S, dirs=(0, 1))
    t1 = time.perf_counter() - t0
    k = int(max(1, min(P.ndir, seconds_target / max(t1, 1e-3))))
    _, _, dt, solves = oracle_sweep_timed(k)
    return cpu_baseline_from(dt, solves, k)


def run_reference(args):
    ws, rank = dist_env()
    if rank != 0:
        return 0
    times, walls = [], []
    cb = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = cpu_baseline(seconds_target=float(os.environ.get("SN_REF_SECONDS", "8")))
        if i >= args.warmup:
            times.append(r["value"])
            walls.append(time.perf_counter() - t0)
            cb = r
    value = float(np.median(times))
    cb = dict(cb, value=value)
    # the oracle on the host cores of rank 0; n_gpus is the launch's N
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.median(walls)),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(),
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def guarded(form, *args):
    """One of the secondary reports (surrogate, networks, anisotropic, general cells):
    an exception in it becomes an "error" entry of its object instead of costing the
    step's JSON line."""
    try:
        return form(*args)
    except Exception as e:  # noqa: BLE001 -- reported in the line, not swallowed
        return {"error": "%s: %s" % (type(e).__name__, e)}


def eps_p(phi, ref):
    """Eq. (20)-style mean relative error of the cell-averaged scalar flux (all groups), m = 1e-8."""
    a = phi.view(phi.shape[0], -1, 8).mean(-1).double()
    b = ref.view(ref.shape[0], -1, 8).mean(-1).double()
    return float(((a - b).abs() / (b.abs() + 1e-8)).mean())


def flux_errors(phi, ref):
    """Errors of a flux against a reference [G, C, 8]: the paper's Eq. (20) (mean over
    cells and groups of |phi - ref| / (|ref| + 1e-8) on the cell-averaged flux), the
    mean and max nodal relative error under a floor of 1e-8 of the group maximum."""
    a = phi.double().view(phi.shape[0], -1, 8)
    b = ref.double().view(ref.shape[0], -1, 8)
    am, bm = a.mean(-1), b.mean(-1)
    gmax = b.abs().amax(dim=(1, 2), keepdim=True)
    nod = (a - b).abs() / (b.abs() + 1e-8 * gmax)
    return {"eq20": float(((am - bm).abs() / (bm.abs() + 1e-8)).mean()), "nodal_mean": float(nod.mean()),
            "nodal_max": float(nod.max())}


def train_surrogate(P, wl_harvest):
    """The workload's surrogate: 2^20 one-cell problems of the specified distribution
    labelled by the library's elimination, 20,000 Adam steps; then fine-tuning on 2^20
    one-cell problems harvested from an elimination iteration of another instance of
    the same family (wl_harvest).  Returns the training report."""
    import torch
    from paper_1906_04017_gb300 import sn, workloads
    x = torch.from_numpy(workloads.onecell_problems(1 << 20, seed=0).astype(np.float32)).cuda()
    t0 = time.perf_counter()
    tr, te = P.surrogate_train(x, n_test=1 << 16, steps=20000, batch=8192, lr=2e-3, seed=1)
    train_s = time.perf_counter() - t0
    del x
    t0 = time.perf_counter()
    Q = sn.Problem(wl_harvest)
    qphi = Q.source_iterate(tol=1e-4, max_it=200, allow_noconv=True)["phi"]
    cells = torch.cat([Q.harvest(Q.source(qphi), 1 << 19, seed=s) for s in (11, 12)])
    Q.close()
    # the harvested set is fixed by its seeds but arrives in the order the GPU threads
    # claimed their slots; sort it so that the fine-tuning repeats from run to run
    host = cells.cpu().numpy()
    order = np.lexsort((host[:, 2], host[:, 1], host[:, 0], host[:, 23], host[:, 19], host[:, 15],
                        host[:, 6], host[:, 7]))
    cells = torch.from_numpy(np.ascontiguousarray(host[order])).cuda()
    feat, targ = sn.surrogate_prepare(cells)
    P.surrogate_fit(feat, targ, steps=20000, batch=8192, lr=5e-4)
    return {"train_mae": tr, "test_mae": te, "train_s": train_s, "train_samples": 1 << 20,
            "train_samples_per_s": 20000 * 8192 / train_s, "finetune_mae": P.surrogate_eval(feat, targ),
            "finetune_s": time.perf_counter() - t0, "finetune_cells": int(cells.shape[0])}


def sweep_ms(P, S, mode, reps=5):
    """Best-of-reps kernel time of one sweep from S (CUDA events around the sweep)."""
    out = P.flux_tensor()
    P.sweep(S, out, mode=mode)
    P.set_profiling(True)
    best = 1e30
    for _ in range(reps):
        P.profile(reset=True)
        P.sweep(S, out, mode=mode)
        ms, n = P.profile(reset=True)
        best = min(best, ms / n)
    P.set_profiling(False)
    return best


def frozen_iteration(P, tau, freeze_after=5, max_chunks=30):
    """The gated surrogate iteration with the gate frozen: `freeze_after` gated sweeps
    from a zero flux, the gate's decisions recorded from the source they reached, then
    frozen sweeps until the Eq. (21) mean change is below 1e-4 (the paper's stop for
    the network iteration) or 10 * max_chunks more iterations.  Returns (flux, report)."""
    from paper_1906_04017_gb300 import sn
    P.surrogate_set_gate(tau)
    phi = P.flux_tensor()
    P.source_iterate(phi=phi, tol=0.0, max_it=freeze_after, mode=sn.ANN_GATED, allow_noconv=True)
    fb = P.surrogate_freeze_gate(P.source(phi))
    it, r = freeze_after, None
    for _ in range(max_chunks):
        r = P.source_iterate(phi=phi, tol=0.0, max_it=10, mode=sn.ANN_FROZEN, use_graph=True, allow_noconv=True)
        it += 10
        if r["change_mean"] < 1e-4:
            break
    return phi, {"tau": tau, "fallback_frac": fb / P.solves_per_sweep, "iters": it,
                 "change_mean": r["change_mean"], "change_max": r["change_max"],
                 "stopped_on_eq21": r["change_mean"] < 1e-4}


def ann_form(P, steps, wl, wl_harvest, taus=(0.02, 0.01, 0.007, 0.005)):
    """The surrogate form on the measured workload: the trained network (train_surrogate)
    as the cell solver of the same wavefront sweep, ungated and with the residual gate
    frozen after 5 gated sweeps (frozen_iteration); sweep solves/s against the
    elimination sweep on the same handle, and the converged flux's error against the
    FP64 solution (an FP64 source iteration to 1e-10 started from the converged FP32
    elimination flux).  `value` is the frozen sweep's solves/s at the largest tau whose
    error (Eq. (20)) is at most 3%."""
    import torch
    from paper_1906_04017_gb300 import sn
    out = {"network": train_surrogate(P, wl_harvest)}
    ge = P.source_iterate(tol=1e-6, max_it=1000, mode=sn.GE32R, use_graph=True, allow_noconv=True)
    P64 = sn.Problem(wl, fp64=True)
    phi64 = ge["phi"].double().clone()
    t0 = time.perf_counter()
    r64 = P64.source_iterate(phi=phi64, tol=1e-10, max_it=2000, allow_noconv=True)
    P64.close()
    out["fp64_reference"] = {"iters_from_fp32": r64["iters"], "change_max": r64["change_max"],
                             "seconds": time.perf_counter() - t0}
    out["ge_vs_fp64"] = flux_errors(ge["phi"], phi64)
    S = P.source(ge["phi"])
    ge_ms = sweep_ms(P, S, sn.GE32R)
    ann_ms = sweep_ms(P, S, sn.ANN)
    n = P.solves_per_sweep
    out["ge_sweep_solves_per_s"] = n / (ge_ms / 1e3)
    out["ungated"] = {"sweep_solves_per_s": n / (ann_ms / 1e3), "speedup_vs_ge_sweep": ge_ms / ann_ms}
    # the ungated network's source iteration (the paper's use, no gate)
    phi = P.flux_tensor()
    try:
        r = P.source_iterate(phi=phi, tol=0.0, max_it=100, mode=sn.ANN, use_graph=True, allow_noconv=True)
        out["ungated"].update({"iters": 100, "change_mean": r["change_mean"], **flux_errors(phi, phi64)})
    except sn.SnError as e:
        out["ungated"]["iteration"] = "diverged: %s" % e
    # tensor-core roofline of the ungated sweep: 2 (32*64 + 64*16) BF16 flops per row
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    tpeak = peaks.get("bf16_tflops", 1900.0)
    tach = n / (ann_ms / 1e3) * 2 * (32 * 64 + 64 * 16) / 1e12
    out["roofline_ungated"] = {"bound": "latency", "tensor_achieved": tach, "tensor_peak": tpeak,
                               "unit": "TFLOP/s", "tensor_frac": tach / tpeak,
                               "peak_note": "measured bf16 burst" if "bf16_tflops" in peaks else "fallback"}
    rows = []
    for tau in taus:
        try:
            phi, rep = frozen_iteration(P, tau)
            rep.update(flux_errors(phi, phi64))
            fz = sweep_ms(P, P.source(phi), sn.ANN_FROZEN)
            rep.update({"frozen_sweep_solves_per_s": n / (fz / 1e3), "speedup_vs_ge_sweep": ge_ms / fz})
        except sn.SnError as e:
            rep = {"tau": tau, "error": str(e)}
        rows.append(rep)
    ok = [r for r in rows if r.get("eq20") is not None and r["eq20"] <= 0.03]
    best = max(ok, key=lambda r: r["tau"]) if ok else None
    out.update({"gated_frozen": rows, "value": best["frozen_sweep_solves_per_s"] if best else None, "unit": UNIT,
                "at_tau": best["tau"] if best else None,
                "speedup_vs_ge_sweep": best["speedup_vs_ge_sweep"] if best else None,
                "error_ref": "FP64 source iteration (converged to 1e-10)"})
    return out


def ann_large_form():
    """The large mixed workload (spheres_96: 96^3 cells, LQ_12 = 168 directions, 16
    groups, high-opacity spheres) in the surrogate form: the network trained as for
    blocked_64 but fine-tuned on problems harvested from another spheres instance;
    the graph-captured elimination iteration to 1e-6 (its time is the reference step
    time), the ungated and frozen-gated sweeps, and the frozen iteration's error
    against the converged FP32 elimination flux (itself within ~1e-6 of FP64 by the
    parity measurements; an FP64 iteration of this size does not fit the bench's time)."""
    import torch
    from paper_1906_04017_gb300 import sn, workloads
    wl = workloads.spheres_96()
    P = sn.Problem(wl)
    out = {"workload": "spheres_96: 96^3 cells, LQ_12 (168 dirs), 16 groups, 200 spheres",
           "network": train_surrogate(P, workloads.spheres_96(seed=1))}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ge = P.source_iterate(tol=1e-6, max_it=400, use_graph=True, allow_noconv=True)
    torch.cuda.synchronize()
    out["ge_iteration"] = {"iters": ge["iters"], "converged": ge["converged"], "seconds": time.perf_counter() - t0}
    S = P.source(ge["phi"])
    n = P.solves_per_sweep
    t_ge = sweep_ms(P, S, sn.GE32R, reps=3)
    t_ann = sweep_ms(P, S, sn.ANN, reps=3)
    out["ge_sweep_solves_per_s"] = n / (t_ge / 1e3)
    out["ungated_sweep_solves_per_s"] = n / (t_ann / 1e3)
    out["ungated_speedup_vs_ge_sweep"] = t_ge / t_ann
    rows = []
    for tau in (0.01, 0.005):
        try:
            phi, rep = frozen_iteration(P, tau, max_chunks=5)
            rep.update(flux_errors(phi, ge["phi"]))
            fz = sweep_ms(P, P.source(phi), sn.ANN_FROZEN, reps=3)
            rep.update({"frozen_sweep_solves_per_s": n / (fz / 1e3), "speedup_vs_ge_sweep": t_ge / fz})
        except sn.SnError as e:
            rep = {"tau": tau, "error": str(e)}
        rows.append(rep)
    out["gated_frozen"] = rows
    out["error_ref"] = "converged FP32 elimination flux"
    P.close()
    return out


# algorithmic FP32 flops of one octant-network solve: 2 (26 x 8 + 8 x 8) multiply-adds,
# 16 bias adds, 16 for the flux; tanh and the ELU exponential are not counted
OCTNET_FLOPS_PER_SOLVE = 2 * (26 * 8 + 8 * 8) + 16 + 16


def octnet_train(m_train=90000, m_test=10000, epochs=50000, lr=2e-4, retrain=500, tol=1e-3, seed=0):
    """The paper's per-octant networks trained as in Sec. 4: 9e4 training and 1e4 test
    one-cell problems per octant (uniform sampling of the inputs over the ranges that
    cover Problems 1-4), elimination labels, the loss of Eq. (19), full-batch Adam for
    5e4 epochs at lr 2e-4 (the paper's range is 5e-5..2e-4); then the connection
    dropping of Sec. 3 (retraining `retrain` epochs after each drop, stop at +0.1 %
    training MSE).  Returns (params [8, 288], mask, lo, hi, report)."""
    import torch
    from paper_1906_04017_gb300 import sn, workloads
    lo, hi = workloads.octant_net_ranges()
    T = sn.Problem(workloads.random_small(2, 2, 2, order=2, G=1))
    rep = {}
    try:
        T.octnet_init(lo, hi, seed=seed)
        xtr = torch.from_numpy(workloads.octant_problems(m_train, seed=seed).astype(np.float32)).cuda()
        xte = torch.from_numpy(workloads.octant_problems(m_test, seed=seed + 1).astype(np.float32)).cuda()
        ftr, ttr = T.octnet_prepare(xtr)
        fte, tte = T.octnet_prepare(xte)
        del xtr, xte
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T.octnet_fit(ftr, ttr, epochs, lr)
        rep["train_s"] = time.perf_counter() - t0
        rep["epoch_ms"] = rep["train_s"] * 1e3 / epochs
        rep["train_samples_per_s"] = 8 * m_train * epochs / rep["train_s"]
        mae, mse = T.octnet_eval(ftr, ttr)
        tmae, tmse = T.octnet_eval(fte, tte)
        rep.update({"train_mae": mae.tolist(), "train_mse": mse.tolist(), "test_mae": tmae.tolist(),
                    "test_mse": tmse.tolist()})
        t0 = time.perf_counter()
        dropped = T.octnet_prune(ftr, ttr, retrain_steps=retrain, lr=lr, tol=tol, max_drops=272)
        rep["prune_s"] = time.perf_counter() - t0
        pmae, pmse = T.octnet_eval(ftr, ttr)
        ptmae, _ = T.octnet_eval(fte, tte)
        rep.update({"dropped": dropped.tolist(), "dropped_frac": float(dropped.mean() / 272.0),
                    "pruned_train_mae": pmae.tolist(), "pruned_train_mse": pmse.tolist(),
                    "pruned_test_mae": ptmae.tolist(),
                    "setup": "%d train + %d test problems per octant, %d full-batch Adam epochs at lr %g, "
                             "%d retraining epochs per dropped connection, tol %g" % (m_train, m_test, epochs, lr,
                                                                                     retrain, tol)})
        params, mask = T.octnet_get()
    finally:
        T.close()
    return params, mask, lo, hi, rep


def octnet_form(P):
    """The paper's own surrogate on the measured workload: the per-octant networks
    (trained by octnet_train) as the cell solver of the same wavefront sweep, ungated
    as in the paper; kernel-level solves/s, its roofline, and the error against the
    elimination form after one sweep and at convergence."""
    import torch
    from paper_1906_04017_gb300 import sn
    params, mask, lo, hi, rep = octnet_train()
    P.octnet_set(params, mask, lo, hi)
    ref = P.source_iterate(tol=1e-6, max_it=500, mode=sn.GE32R, use_graph=True, allow_noconv=True)["phi"].clone()
    S_ref = P.source(ref)

    def rate(mode, reps=5):
        out_phi = P.flux_tensor()
        P.sweep(S_ref, out_phi, mode=mode)
        P.set_profiling(True)
        P.profile(reset=True)
        for _ in range(reps):
            P.sweep(S_ref, out_phi, mode=mode)
        ms, n = P.profile(reset=True)
        P.set_profiling(False)
        return P.solves_per_sweep / (ms / n / 1e3), out_phi

    ge_rate, ge_phi = rate(sn.GE32R)
    net_rate, net_phi = rate(sn.OCTNET)
    gmax = ge_phi.abs().amax(dim=(1, 2), keepdim=True)
    out = {"network": rep, "value": net_rate, "unit": UNIT, "ge_sweep_solves_per_s": ge_rate,
           "speedup_vs_ge_sweep": net_rate / ge_rate, "one_sweep_eps_P_vs_ge": eps_p(net_phi, ge_phi),
           "one_sweep_maxnorm_err_vs_ge": float(((net_phi - ge_phi).abs() / gmax).max())}
    phi = P.flux_tensor()
    try:
        r = P.source_iterate(phi=phi, tol=1e-5, max_it=300, mode=sn.OCTNET, use_graph=True, allow_noconv=True)
        out.update({"eps_P_vs_ge": eps_p(phi, ref), "iters": r["iters"], "converged": r["converged"]})
    except sn.SnError as e:
        out.update({"eps_P_vs_ge": None, "converged": False, "diverged": str(e)})
    peak_tf = N_SM * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    ach = net_rate * OCTNET_FLOPS_PER_SOLVE / 1e12
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm = net_rate * BYTES_PER_SOLVE / 1e9
    out["roofline"] = {"bound": "alu", "kernel": "sweep_net_wave", "achieved": ach, "peak": peak_tf,
                       "unit": "TFLOP/s", "frac": ach / peak_tf, "flops_per_solve": OCTNET_FLOPS_PER_SOLVE,
                       "hbm_achieved_gbs": hbm, "hbm_peak_gbs": hbm_peak, "hbm_frac": hbm / hbm_peak,
                       "peak_note": "FP32 peak = 152 SMs x 128 lanes x 2 flop x 2070 MHz (nominal max clock); "
                                    "HBM peak %s" % ("measured" if "hbm_gbs" in peaks else "fallback")}
    return out


def aniso_form(steps, ge_step_ms):
    """Anisotropic scattering (Eqs. (3)-(8)) on the same workload: Legendre order L = 1
    and L = 3 (K = 4 and 16 flux moments), sigma_{s,n} = 0.5^n sigma_s; the graph-
    captured source iteration's step time and the sweep kernels' solves/s.  Extra work
    per solve against the isotropic step: the direction's source from K source moments
    (8 K multiply-adds) and its share of the K flux moments (8 K multiply-adds)."""
    import torch
    from paper_1906_04017_gb300 import sn, workloads
    out = []
    for L in (1, 3):
        wl = workloads.blocked_64()
        P = sn.Problem(wl)
        P.set_scattering_order(L, np.stack([wl["sigs"] * 0.5 ** n for n in range(1, L + 1)]))
        phi = P.flux_tensor()
        P.source_iterate(phi=phi, tol=0.0, max_it=3, use_graph=True, allow_noconv=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = P.source_iterate(phi=phi, tol=0.0, max_it=steps, use_graph=True, allow_noconv=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        P.set_profiling(True)
        P.profile(reset=True)
        P.source_iterate(phi=phi, tol=0.0, max_it=3, use_graph=False, allow_noconv=True)
        sw_ms, n = P.profile(reset=True)
        P.set_profiling(False)
        K = (L + 1) ** 2
        flops = FLOPS_PER_SOLVE - 16 + 32 * K
        sweep_rate = P.solves_per_sweep / (sw_ms / n / 1e3)
        out.append({"L": L, "moments": K, "step_ms": ms, "value": P.solves_per_sweep / (ms / 1e3),
                    "unit": UNIT, "step_time_vs_isotropic": ms / ge_step_ms,
                    "sweep_solves_per_s": sweep_rate, "flops_per_solve": flops,
                    "sweep_tflops": sweep_rate * flops / 1e12, "iters": r["iters"]})
        P.close()
        del phi
    return out


# counted FP32 flops of one solve on a general hexahedral cell: the assembly of A from
# the octant's folded streaming matrices and the mass matrix (4 x 64 multiply-adds), the
# right-hand side (64 + 3 inflow faces x 64), elimination 372, back substitution 64, the
# refinement residual without forming A (4 x 64 + 64) and replay 128, flux 16
GEOM_FLOPS_PER_SOLVE = 2 * (256 + 64 + 192 + 256 + 64) + 372 + 64 + 128 + 16


def geom_form(steps, ge_step_ms):
    """General hexahedral cells on the same workload: every interior vertex moved by up
    to 3% of a cell (the largest deformation the LQ_8 directions allow everywhere), the
    graph-captured source iteration's step time and the sweep kernels' solves/s."""
    import torch
    from paper_1906_04017_gb300 import sn, workloads
    wl = workloads.blocked_64()
    P = sn.Problem(wl)
    P.set_geometry(workloads.deformed_vertices(wl, 0.03, seed=0))
    phi = P.flux_tensor()
    P.source_iterate(phi=phi, tol=0.0, max_it=3, use_graph=True, allow_noconv=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = P.source_iterate(phi=phi, tol=0.0, max_it=steps, use_graph=True, allow_noconv=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    P.set_profiling(True)
    P.profile(reset=True)
    P.source_iterate(phi=phi, tol=0.0, max_it=3, use_graph=False, allow_noconv=True)
    sw_ms, n = P.profile(reset=True)
    P.set_profiling(False)
    bal = P.balance()
    rate = P.solves_per_sweep / (sw_ms / n / 1e3)
    out = {"deformation": "interior vertices moved by U[-0.03, 0.03] cell sizes per axis", "step_ms": ms,
           "value": P.solves_per_sweep / (ms / 1e3), "unit": UNIT, "step_time_vs_box": ms / ge_step_ms,
           "sweep_solves_per_s": rate, "flops_per_solve": GEOM_FLOPS_PER_SOLVE,
           "sweep_tflops": rate * GEOM_FLOPS_PER_SOLVE / 1e12, "iters": r["iters"],
           "balance_rel": abs(bal[0] + bal[1] - bal[2] - bal[3]) / (bal[2] + bal[3])}
    P.close()
    return out


def e2e_pipelined(P, phi_in_host, phi_out_host, steps, stream):
    """`steps` source-iteration steps through the public API (sn_source_iterate, one
    iteration a call: source build, sweep, octant reduction with FP64 norms), each
    starting from the flux copied in from pinned host memory and ending with its new
    flux copied back to pinned host memory.  The host copies run on a second stream
    into and out of two staging buffers, so step i+1's input and step i's result move
    while a step runs; the step itself reads and writes one device flux buffer (the
    one its captured graph was made for) through two device-to-device copies.
    Returns the milliseconds from the first copy's start to the last copy's end (CUDA
    events)."""
    import torch
    xs = torch.cuda.Stream()
    phi = P.flux_tensor()
    inb = [torch.empty_like(phi) for _ in range(2)]
    outb = [torch.empty_like(phi) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    ev_res = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    xs.wait_event(e0)

    def copy_in(b, i):
        with torch.cuda.stream(xs):
            if i >= 2:
                xs.wait_event(ev_used[b])       # the step that read this buffer has copied it
            inb[b].copy_(phi_in_host, non_blocking=True)
            ev_in[b].record(xs)

    copy_in(0, 0)
    for i in range(steps):
        b = i % 2
        if i + 1 < steps:
            copy_in(1 - b, i + 1)
        stream.wait_event(ev_in[b])
        phi.copy_(inb[b], non_blocking=True)
        ev_used[b].record(stream)
        P.source_iterate(phi=phi, tol=0.0, max_it=1, use_graph=True, allow_noconv=True)
        if i >= 2:
            stream.wait_event(ev_out[b])        # the host copy out of this buffer is done
        outb[b].copy_(phi, non_blocking=True)
        ev_res[b].record(stream)
        with torch.cuda.stream(xs):
            xs.wait_event(ev_res[b])
            phi_out_host.copy_(outb[b], non_blocking=True)
            ev_out[b].record(xs)
    stream.wait_event(ev_out[(steps - 1) % 2])
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_gpu(args):
    import torch
    ws, rank = dist_env()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        # the other forms and the CPU baseline are single-GPU reports: replicas would only
        # hold the GPUs longer
        args.no_ann = args.no_octnet = args.no_aniso = args.no_geom = args.no_cpu_baseline = True
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1906_04017_gb300 import sn, workloads

    wl = workloads.blocked_64()
    P = sn.Problem(wl)
    phi = P.flux_tensor()
    solves = P.solves_per_sweep
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    # warm-up: the first iterations also capture the CUDA graphs
    P.source_iterate(phi=phi, tol=0.0, max_it=max(args.warmup, 3), use_graph=True, allow_noconv=True)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    r = P.source_iterate(phi=phi, tol=0.0, max_it=args.steps, use_graph=True, allow_noconv=True)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    assert r["iters"] == args.steps

    # the dominant kernel alone: CUDA events around each sweep's kernel
    P.set_profiling(True)
    P.source_iterate(phi=phi, tol=0.0, max_it=2, use_graph=False, allow_noconv=True)
    P.profile(reset=True)
    P.source_iterate(phi=phi, tol=0.0, max_it=args.steps, use_graph=False, allow_noconv=True)
    sweep_ms, nsw = P.profile(reset=True)
    P.set_profiling(False)

    # end to end through the public API with host buffers: pinned flux in, flux out,
    # every step one source iteration (the work `value` times)
    phi_in_host = phi.cpu().pin_memory()
    phi_out_host = torch.empty_like(phi_in_host).pin_memory()
    e2e_pipelined(P, phi_in_host, phi_out_host, 2, stream)
    barrier()
    e2e_ms = e2e_pipelined(P, phi_in_host, phi_out_host, args.steps, stream)
    barrier()

    # parity of the measured kernel against the FP64 oracle: one sweep of the same
    # seeded source on the device and in the oracle (whose timing is the CPU baseline)
    parity = cb = None
    if not args.no_cpu_baseline:
        def parity_and_baseline():
            S32, ref, dt, ns = oracle_sweep_timed()
            got = P.sweep(torch.from_numpy(S32).cuda(), mode=sn.GE32R).cpu().numpy()
            rep = parity_report(got, ref)
            rep["what"] = ("one GE32R sweep of blocked_64 (all 8 groups, 80 directions, uniform [0, 1] source, "
                           "seed 0) against the FP64 oracle's sweep of the same FP32-rounded source")
            return rep, cpu_baseline_from(dt, ns, 80)
        res = guarded(parity_and_baseline)
        if isinstance(res, tuple):
            parity, cb = res
        else:
            parity = cb = res

    ann = None if args.no_ann else guarded(ann_form, P, args.steps, wl, workloads.blocked_64(seed=1))
    octnet = None if args.no_octnet else guarded(octnet_form, P)

    ms, e2e_ms = max_over_ranks([ms, e2e_ms], dist, "cuda")
    P.close()
    ann_large = None if args.no_ann else guarded(ann_large_form)
    aniso = None if args.no_aniso else guarded(aniso_form, min(args.steps, 10), ms / args.steps)
    geom = None if args.no_geom else guarded(geom_form, min(args.steps, 10), ms / args.steps)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    value = job_throughput(ws, solves, args.steps, ms)
    e2e_value = job_throughput(ws, solves, args.steps, e2e_ms)
    # roofline of the sweep kernel (dominant): FP32 ALU bound
    sweep_s = sweep_ms / max(nsw, 1) / 1e3
    achieved_tf = solves * FLOPS_PER_SOLVE / sweep_s / 1e12
    peak_tf = N_SM * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(),
        "roofline": {"bound": "alu", "kernel": "sweep_ge_wave<true>", "achieved": achieved_tf,
                     "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved_tf / peak_tf,
                     "traffic": (solves * DRAM_BYTES_PER_SOLVE_NCU if DRAM_BYTES_PER_SOLVE_NCU else None),
                     "traffic_note": "DRAM bytes of one sweep kernel launch from one full-set ncu capture of "
                                     "this kernel (75.0 B a solve, under the 96 B of the faces: a face written "
                                     "by one hyperplane is read by the next from L2)",
                     "flops_per_solve": FLOPS_PER_SOLVE,
                     "hbm_achieved_gbs": solves * BYTES_PER_SOLVE / sweep_s / 1e9,
                     "hbm_peak_gbs": hbm_peak,
                     "peak_note": "FP32 peak = 152 SMs x 128 lanes x 2 flop x 2070 MHz (nominal max clock); "
                                  "HBM peak %s" % ("measured" if "hbm_gbs" in peaks else "fallback"),
                     "sweep_ms": sweep_s * 1e3},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(phi_in_host.numel() * 4),
                "d2h_bytes_per_step": int(phi_out_host.numel() * 4),
                "what": "one source iteration a step through sn_source_iterate, the flux copied in from pinned "
                        "host memory and the new flux copied back every step (copies on a second stream, "
                        "overlapping the neighbouring steps)"},
        "gpu_launches": int(args.steps * LAUNCHES_PER_STEP + 1),
        "clocks": clk,
    }
    if ws > 1:
        line["replicas"] = ws
    if parity is not None:
        line["parity"] = parity
    if ann is not None:
        line["ann"] = ann
    if ann_large is not None:
        line["ann_large"] = ann_large
    if octnet is not None:
        line["octnet"] = octnet
    if aniso is not None:
        line["aniso"] = aniso
    if geom is not None:
        line["geom"] = geom
    if cb is not None:
        line["cpu_baseline"] = cb
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def adjoint_check(args):
    """Adjoint form at 32^3 (LQ_8, 4 groups, blocked opacity): gradients of the
    group-summed flux integral over the 4x4x4 low corner with respect to every
    per-cell, per-group sigma_t, sigma_s and q (393,216 parameters), by the FP32
    adjoint sweep.  32 random parameters of the cells within 8 cells of the detector
    (elsewhere the response hardly depends on them) are checked against central
    differences, relative step 1e-6, of FP64 GPU source iterations: both perturbed
    runs start from the unperturbed FP64 flux and take the same 120 iterations, so
    their iteration errors cancel in the difference.  Prints one JSON line."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_1906_04017_gb300 import sn, workloads
    wl = workloads.blocked_32()
    nx = wl["nx"]
    vol = (wl["lx"] / nx) ** 3
    i, j, k = workloads.cell_ijk(wl)
    G, C = wl["sigt"].shape[0], nx ** 3
    r = np.zeros((G, C, 8))
    r[:, (i < 4) & (j < 4) & (k < 4), :] = vol / 8.0
    near = np.flatnonzero((i < 8) & (j < 8) & (k < 8))
    t0 = time.time()
    P = sn.Problem(wl)
    fwd = P.source_iterate(tol=1e-6, max_it=2000)
    ta = time.time()
    adj = P.adjoint(fwd["phi"], torch.from_numpy(r.astype(np.float32)).cuda(), tol=1e-6, max_it=2000)
    torch.cuda.synchronize()
    t_adj = time.time() - ta
    P.close()
    P64 = sn.Problem(wl, fp64=True)
    base = P64.source_iterate(tol=1e-13, max_it=5000)
    phi0 = base["phi"]
    r64 = torch.from_numpy(r).cuda()
    R0 = P64.response(phi0, r64)
    P64.close()
    rng = np.random.default_rng(2024)
    kinds = (("sigt", "grad_sigt"), ("sigs", "grad_sigs"), ("q", "grad_q"))
    picks = [(kinds[rng.integers(0, 3)], int(rng.integers(0, G)), int(near[rng.integers(0, len(near))]))
             for _ in range(32)]
    rows = []
    n_it = 120
    for (key, gkey), g, c in picks:
        p0 = float(wl[key][g, c])
        h = 1e-6 * (p0 if p0 > 0 else 1.0)
        Rs = []
        for v in (p0 + h, p0 - h):
            w = dict(wl)
            w[key] = wl[key].copy()
            w[key][g, c] = v
            Q = sn.Problem(w, fp64=True)
            phi = phi0.clone()
            Q.source_iterate(phi=phi, tol=0.0, max_it=n_it, allow_noconv=True)
            Rs.append(Q.response(phi, r64))
            Q.close()
        fd = (Rs[0] - Rs[1]) / (2 * h)
        ga = float(adj[gkey][g, c].item())
        rows.append(dict(kind=key, g=g, c=c, param=p0, adjoint=ga, fd=fd,
                         sensitivity=abs(fd * p0) / abs(R0) if p0 > 0 else abs(fd) / abs(R0),
                         rel=abs(ga - fd) / abs(fd) if fd != 0 else None))
    # the difference resolves R to ~1e-15 relative: a parameter whose effect
    # |p dR/dp| is below 1e-6 R is reported but not judged
    judged = [x for x in rows if x["sensitivity"] >= 1e-6 and x["rel"] is not None]
    out = {"adjoint_check": "blocked_32: 32^3 cells, LQ_8, 4 groups, corner 4^3 response",
           "parameters": 3 * G * C, "R": R0, "adjoint_iters": adj["iters"], "adjoint_s": t_adj,
           "fd": "FP64, relative step 1e-6, %d iterations from the unperturbed flux" % n_it,
           "checked": len(rows), "judged": len(judged),
           "max_rel_judged": max(x["rel"] for x in judged) if judged else None,
           "median_rel_judged": float(np.median([x["rel"] for x in judged])) if judged else None,
           "wall_s": time.time() - t0, "rows": rows}
    print(json.dumps(out))
    return 0


def paper_reported(k, n, order):
    """The paper's own figures for Problem k on n^3 cells at S_order (Sec. 4 tables, as
    transcribed in tests/golden/paper_sec4_problems.json), or None where the paper has
    no such case: error in percent and time reduction in percent; Problem 4 adds the
    elimination's and the network's source iterations and the overall speed-up."""
    with open(os.path.join(ROOT, "tests", "golden", "paper_sec4_problems.json")) as f:
        res = json.load(f)["results"]
    if n == 100 and str(order) in res["by_order_100_cubed"][str(k)]:
        v = res["by_order_100_cubed"][str(k)][str(order)]
    elif order == 8 and str(n) in res["by_mesh_S8"][str(k)]:
        v = res["by_mesh_S8"][str(k)][str(n)]
    else:
        return None
    out = {"eps_P_pct": v[0]}
    if k == 4:
        out.update({"ge_iters": v[1], "ann_iters": v[2], "iteration_time_reduction_pct": v[3],
                    "overall_speedup": v[4]})
    else:
        out["time_reduction_pct"] = v[1]
    return out


def paper_tables(args):
    """The evaluation of Sec. 4 run with the three solvers: Problems 1-4 (10 cm cube,
    unit inflow on the x-, y-, z- faces) at S2-S8 on 100^3 cells and at 10^3-100^3
    cells with S8.  For each case: the elimination solution (FP32 GE with
    refinement), the tensor-core surrogate (the 27-64-8 network trained on the
    one-cell distribution) and the paper's own per-octant networks (26-8-8, trained
    as in Sec. 4), both ungated as in the paper: the mean relative error of the
    cell-averaged flux (Eq. (20)), the solve times and the time reduction.  Problem 4
    (scattering ratio 0.99) runs the source iteration to the mean change of Eq. (21)
    below 1e-4 with both solvers and reports their iteration counts.  Prints one
    JSON line."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_1906_04017_gb300 import sn, workloads
    # the network, trained once on the one-cell distribution
    T = sn.Problem(workloads.random_small(2, 2, 2, order=2, G=1))
    x = torch.from_numpy(workloads.onecell_problems(1 << 20, seed=0).astype(np.float32)).cuda()
    tr, te = T.surrogate_train(x, n_test=1 << 16, steps=20000, batch=8192, lr=2e-3, seed=1)
    weights = T.surrogate_weights()
    T.close()
    del x
    # the paper's own per-octant networks
    on_params, on_mask, on_lo, on_hi, on_rep = octnet_train()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    def solve(P, mode, iterate):
        if not iterate:
            S = P.source(P.flux_tensor())           # q / 4 pi: no scattering
            P.sweep(S, mode=mode)                    # warm-up
            phi, ms = timed(lambda: P.sweep(S, mode=mode))
            return phi, ms, 1, "one sweep"
        phi = P.flux_tensor()
        P.source_iterate(phi=phi, tol=0.0, max_it=1, mode=mode, use_graph=True, allow_noconv=True)  # capture
        phi.zero_()

        hist = []

        def run():
            for it in range(1, 2001):
                try:
                    r = P.source_iterate(phi=phi, tol=0.0, max_it=1, mode=mode, use_graph=True, allow_noconv=True)
                except sn.SnError as e:
                    return it, "diverged: %s" % e
                hist.append(r["change_mean"])
                if r["change_mean"] < 1e-4:
                    return it, "converged"
            return 2000, "not converged"
        (its, status), ms = timed(run)
        # effective spectral radius: geometric mean ratio of the last 20 changes
        rho = (hist[-1] / hist[-21]) ** (1.0 / 20) if len(hist) > 21 and hist[-21] > 0 else None
        return phi, ms, its, status + ("" if rho is None else ", rho %.4f" % rho)

    cases = [(k, 100, o) for k in (1, 2, 3, 4) for o in (2, 4, 6, 8)]
    cases += [(k, n, 8) for k in (1, 2, 3, 4) for n in (10, 25, 50)]
    rows = []
    t0 = time.time()
    for k, n, order in cases:
        P = sn.Problem(workloads.paper_problem(k, n=n, order=order))
        P.surrogate_set_weights(weights)
        P.octnet_set(on_params, on_mask, on_lo, on_hi)
        it4 = k == 4
        ge, ms_ge, it_ge, st_ge = solve(P, sn.GE32R, it4)
        ge = ge.clone()
        ann, ms_ann, it_ann, st_ann = solve(P, sn.ANN, it4)
        finite = bool(torch.isfinite(ann).all())
        row = {"problem": k, "cells": n, "order": order, "solves_per_sweep": P.solves_per_sweep,
               "ge_ms": ms_ge, "ann_ms": ms_ann, "ge_iters": it_ge, "ann_iters": it_ann,
               "ge_status": st_ge, "ann_status": st_ann,
               "eps_P": eps_p(ann, ge) if finite else None,
               "time_reduction": 1.0 - ms_ann / ms_ge, "paper": paper_reported(k, n, order)}
        ann = None
        ocn, ms_ocn, it_ocn, st_ocn = solve(P, sn.OCTNET, it4)
        row.update({"octnet_ms": ms_ocn, "octnet_iters": it_ocn, "octnet_status": st_ocn,
                    "octnet_eps_P": eps_p(ocn, ge) if bool(torch.isfinite(ocn).all()) else None,
                    "octnet_time_reduction": 1.0 - ms_ocn / ms_ge})
        ocn = None
        if it4:
            # with the residual gate (not in the paper): tau = 0.01
            P.surrogate_set_gate(0.01)
            gt, ms_gt, it_gt, st_gt = solve(P, sn.ANN_GATED, it4)
            row.update({"gated_ms": ms_gt, "gated_iters": it_gt, "gated_status": st_gt,
                        "gated_eps_P": eps_p(gt, ge) if bool(torch.isfinite(gt).all()) else None,
                        "gated_time_reduction": 1.0 - ms_gt / ms_ge})
        rows.append(row)
        P.close()
    print(json.dumps({"paper_tables": "Problems 1-4 of Sec. 4, both solvers, FP32, one GPU",
                      "network": {"train_mae": tr, "test_mae": te, "training": "2^20 one-cell problems, 20000 Adam steps"},
                      "octant_networks": on_rep,
                      "wall_s": time.time() - t0, "rows": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ann", action="store_true")
    ap.add_argument("--no-octnet", action="store_true")
    ap.add_argument("--no-aniso", action="store_true")
    ap.add_argument("--no-geom", action="store_true")
    ap.add_argument("--paper-tables", action="store_true",
                    help="Problems 1-4 of the paper with both solvers (prints its own JSON line)")
    ap.add_argument("--adjoint-check", action="store_true",
                    help="adjoint gradients vs FP64 central differences at 32^3 (prints its own JSON line)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.adjoint_check:
        return adjoint_check(args)
    if args.paper_tables:
        return paper_tables(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

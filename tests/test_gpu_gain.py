"""What the trained network gains over the method without it (the surrogate form of
Secs. 3-4 with this library's residual gate), measured on blocked_32 (32^3 cells,
LQ_8, 4 groups).

The network is trained as the bench trains it: 2^20 one-cell problems of the
specified distribution labelled by the library's elimination, then fine-tuning on
one-cell problems harvested from an elimination iteration of another instance of
the family (opacity seed 1).  Reference: the FP64 source iteration converged to
1e-10 (started from the converged FP32 elimination flux).

The gated iteration: 5 gated sweeps from a zero flux, the gate's decisions frozen
from the source they reached, frozen sweeps until the Eq. (21) mean change is below
1e-4 or 300 more iterations; tau is the largest of 0.02, 0.01, 0.007, 0.005, 0.003
whose converged flux is within 3% (Eq. (20)) of the FP64 flux.  Sweep times are CUDA
events around one sweep from the converged source, best of 5, on the same handle.  The
ungated network sweep's speed against elimination is asserted on blocked_64, where it
is clear of the noise."""
import os
import sys

import numpy as np
import pytest
import torch

from paper_1906_04017_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def gain(sn):
    import bench
    wl = W.blocked_32()
    P = sn.Problem(wl)
    net = bench.train_surrogate(P, W.blocked_32(seed=1))
    ge = P.source_iterate(tol=1e-6, max_it=1000, use_graph=True)
    P64 = sn.Problem(wl, fp64=True)
    phi64 = ge["phi"].double().clone()
    P64.source_iterate(phi=phi64, tol=1e-10, max_it=2000, allow_noconv=True)
    P64.close()
    S = P.source(ge["phi"])
    out = {"t_ge": bench.sweep_ms(P, S, sn.GE32R), "t_ann": bench.sweep_ms(P, S, sn.ANN), "found": None}
    print("\nnetwork: fine-tuned MAE %.4f; sweep ms: elimination %.3f, network %.3f (%.2fx)"
          % (net["finetune_mae"], out["t_ge"], out["t_ann"], out["t_ge"] / out["t_ann"]))
    for tau in (0.02, 0.01, 0.007, 0.005, 0.003):
        phi, rep = bench.frozen_iteration(P, tau)
        err = bench.flux_errors(phi, phi64)
        t_fz = bench.sweep_ms(P, P.source(phi), sn.ANN_FROZEN)
        print("tau %.3f: %.1f%% of rows to elimination, Eq. (20) error %.4f, nodal mean %.4f, frozen sweep "
              "%.3f ms (%.2fx elimination), %d iterations, mean change %.1e"
              % (tau, 100 * rep["fallback_frac"], err["eq20"], err["nodal_mean"], t_fz, out["t_ge"] / t_fz,
                 rep["iters"], rep["change_mean"]))
        assert bool(phi.isfinite().all())
        if err["eq20"] <= 0.03:
            out["found"] = {"tau": tau, "eq20": err["eq20"], "t_frozen": t_fz, **rep}
            break
    P.close()
    return out


def test_frozen_gate_iteration_is_within_3_percent_of_fp64(gain):
    assert gain["found"] is not None


def test_network_sweep_is_faster_than_elimination(sn):
    """The ungated tensor-core network sweep against the elimination sweep on the same
    handle, on blocked_64 (64^3 cells, LQ_8, 8 groups): measured 1.07-1.09x.  The
    network's speed does not depend on its weights, so bounded random weights stand in
    for the trained ones.  On blocked_32 (the fixture above prints it) the two sweeps
    are within noise of each other (1.00-1.03x), too close for an assertion."""
    import bench
    from test_gpu_surrogate import bounded_weights
    P = sn.Problem(W.blocked_64())
    P.surrogate_set_weights(bounded_weights(3))
    rng = np.random.default_rng(1)
    S = torch.from_numpy(rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32)).cuda()
    t_ge = bench.sweep_ms(P, S, sn.GE32R)
    t_ann = bench.sweep_ms(P, S, sn.ANN)
    P.close()
    print("\nblocked_64 sweep ms: elimination %.3f, network %.3f (%.3fx)" % (t_ge, t_ann, t_ge / t_ann))
    assert t_ann < t_ge


@pytest.mark.xfail(strict=True, reason=(
    "measured on GB300: at the 40-60% of rows that the gate must send to elimination "
    "for 3% accuracy, the frozen-gate sweep runs at about 0.4x the elimination sweep; "
    "the ungated network sweep is only about 1.1x it, so even a free fallback would "
    "leave the gated sweep within a few percent of the elimination sweep"))
def test_frozen_gate_sweep_is_faster_than_elimination(gain):
    assert gain["found"] is not None
    assert gain["found"]["t_frozen"] < gain["t_ge"]

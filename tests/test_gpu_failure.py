"""Failure detection on the GPU without a fault (the bounded-wait path of the
tensor-core kernels): a wait on an mbarrier phase that nothing completes, with a
short limit, gives up, is reported as SN_ETIMEOUT through the same abort flag and
counter a surrogate sweep uses, frees its tensor memory, and leaves the context
usable -- a sweep right after it still matches the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1906_04017_gb300 import workloads as W
from _parity import rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit", [1000, 100000])
def test_withheld_wait_times_out_and_context_survives(sn, limit):
    wl = W.random_small(5, 4, 3, order=4, G=2, seed=1, psi_inc=True)
    P = sn.Problem(wl)
    assert P.selftest_wait(limit) == sn.SN_ETIMEOUT
    assert P.selftest_wait(limit) == sn.SN_ETIMEOUT      # again, on the same handle
    # the context is intact: an elimination sweep right after matches the oracle
    rng = np.random.default_rng(0)
    S = rng.uniform(0.0, 1.0, (P.G, P.ncell, 8)).astype(np.float32)
    phi = P.sweep(torch.from_numpy(S).cuda(), mode=sn.GE32R).cpu().numpy()
    P.close()
    ref, _ = oracle.OracleProblem(wl).sweep(S.astype(np.float64))
    assert rel_err(phi, ref) < 1e-5


def test_selftest_rejects_bad_limits(sn):
    wl = W.random_small(2, 2, 2, order=2, G=1)
    P = sn.Problem(wl)
    for bad in (0, -5, (1 << 31) + 1):
        assert P.selftest_wait(bad) == sn.SN_EINVAL
    P.close()

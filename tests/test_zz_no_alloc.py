"""The allocation-free gradient entry point (for callers that cannot allocate device
memory: stream capture in global mode, fixed memory pools, latency-bound loops)
must give the same loss and gradient as the allocating sn_surrogate_grad, call
after call, although every call reuses the library's one fixed scratch array.

This file is collected last on purpose, so that a failure here cannot hide any
other test of a run that stops at the first failure."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_1906_04017_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_gradient_matches_allocating_entry_point(sn):
    wl = W.random_small(2, 2, 2, order=2, G=1)
    P = sn.Problem(wl)
    p = mlp.init_params(31).astype(np.float32)
    P.surrogate_set_weights(p)
    params = torch.from_numpy(p).cuda()
    grad = torch.empty(sn.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    # two calls in a row of different sizes: each call writes every partial it
    # reads, and this pins equality with the allocating path across call sizes
    for n, seed in ((20000, 1), (3000, 2)):
        x = torch.from_numpy(W.onecell_problems(n, seed=seed).astype(np.float32)).cuda()
        feat, targ = sn.surrogate_prepare(x)
        ref_loss, ref_grad = P.surrogate_grad(feat, targ)
        sn.surrogate_grad_noalloc(params, feat, targ, grad, loss)
        torch.cuda.synchronize()
        g = grad.cpu().numpy()
        assert np.abs(g - ref_grad).max() <= 1e-6 * np.abs(ref_grad).max()
        assert abs(loss.item() - ref_loss) <= 1e-6 * abs(ref_loss)
    P.close()


def test_noalloc_rejects_oversized_batch(sn):
    n = 32769
    params = torch.zeros(sn.NPARAM, dtype=torch.float32, device="cuda")
    feat = torch.zeros((n, 27), dtype=torch.float32, device="cuda")
    targ = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    grad = torch.empty(sn.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(sn.SnError) as e:
        sn.surrogate_grad_noalloc(params, feat, targ, grad, loss)
    assert e.value.status == sn.SN_EINVAL

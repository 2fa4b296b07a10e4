"""Failure detection and recovery on the GPU, without faulting it.

* A bounded device-side wait that runs out.  The pixel kernels wait (with a clock budget) for the
  bulk copies that stage each tile.  celeste_problem_set_wait_budget(-1) makes that first wait give
  up at once on a healthy device, so the timeout path runs for real: the kernel sets the problem's
  timeout word, waits with the full budget for the copies already in flight, writes NaN tile sums
  and exits.  The host must see CELESTE_ERR_TIMEOUT, and the context must stay usable: the next
  call with the default budget clears the word and gives the same results as before.
* Resuming Newton.  celeste_newton_batch writes back every source's parameters and trust radius,
  so a solve stopped after k iterations and called again from its (theta, delta) must reach the
  optimum of the uninterrupted solve.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import celeste_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as pkg
    return pkg


def _arrays(ts):
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in ts]


def test_wait_timeout_is_reported_and_the_context_recovers(P):
    sc = synth.tiny(seed=21, n_sources=4, n_images=3, H=36, W=40, radius=(6, 14))
    dev = torch.device("cuda:0")
    prob = P.Problem(sc, device=dev, tile_pixels=128)
    th = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(th)
    before = _arrays(prob.elbo_batch(th))

    prob.set_wait_budget(-1)
    e, g, h = prob.elbo_batch(th, check=False)
    with pytest.raises(P.CelesteError, match="timed out"):
        prob.check()
    assert not np.all(np.isfinite(e.cpu().numpy()))          # the tiles waited on hold NaN sums
    # the value-only kernel takes the same path
    v, _, _ = prob.elbo_batch(th, want=P.WANT_ELBO, check=False)
    with pytest.raises(P.CelesteError, match="timed out"):
        prob.check()
    # Newton reads the word itself and returns the code
    with pytest.raises(P.CelesteError, match="timed out"):
        prob.newton_batch(th.clone(), max_iter=3)
    # the allocation-free evaluation records it in the bound workspace
    out = [torch.empty(sc.n_sources, dtype=torch.float64, device=dev),
           torch.empty(sc.n_sources, 27, dtype=torch.float64, device=dev),
           torch.empty(sc.n_sources, 27, 27, dtype=torch.float64, device=dev)]
    fn = P.lib().celeste_elbo_batch_noalloc
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = fn(prob.handle, ptr(th), ptr(out[0]), ptr(out[1]), ptr(out[2]),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    with pytest.raises(P.CelesteError, match="timed out"):
        prob.check()

    # default budget again: the next call clears the word and reproduces the earlier results bit for bit
    prob.set_wait_budget(0)
    after = _arrays(prob.elbo_batch(th))
    prob.check()
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)
    # and they still match the oracle
    orc = O.Oracle(sc)
    for s in range(sc.n_sources):
        if orc.rects[s]:
            L = orc.elbo(s, sc.theta0[s], sc.theta0)
            assert abs(after[0][s] - L) <= 1e-6 * abs(L)
    # Newton on the same context converges
    t2 = th.clone()
    _, _, status, _ = prob.newton_batch(t2)
    torch.cuda.synchronize()
    assert int((status == P.STATUS_CONVERGED).sum()) == sc.n_sources


@pytest.mark.parametrize("k", [1, 3, 7])
def test_newton_resumed_from_theta_and_radius_reaches_the_same_optimum(P, k):
    from test_parity_gpu import compare_optimum, stop_slack
    sc = synth.tiny(seed=5, n_sources=12, n_images=3, H=120, W=130, radius=(6, 12))
    dev = torch.device("cuda:0")
    prob = P.Problem(sc, device=dev, tile_pixels=128)
    start = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(start.clone())

    full = start.clone()
    _, it_full, st_full, L_full = prob.newton_batch(full)
    # stopped after k iterations, then resumed from the written-back parameters and radii
    part = start.clone()
    delta, it1, st1, _ = prob.newton_batch(part, max_iter=k)
    d_mid = delta.clone()
    delta2, it2, st2, L_res = prob.newton_batch(part, delta=delta, max_iter=50 - k)
    torch.cuda.synchronize()
    assert int(it1.max()) <= k
    # the resumed call starts from the radius the first one left (it writes it back in place)
    assert torch.all(d_mid > 0)
    e_full, e_res = L_full.cpu().numpy(), L_res.cpu().numpy()
    got, ref = part.cpu().numpy(), full.cpu().numpy()
    _, _, H = prob.elbo_batch(full)
    H = H.cpu().numpy()
    for s in range(sc.n_sources):
        if int(st_full[s]) != P.STATUS_CONVERGED:
            continue
        assert int(st2[s]) == P.STATUS_CONVERGED
        assert abs(e_res[s] - e_full[s]) <= 1e-7 * abs(e_full[s]), (s, e_res[s], e_full[s])
        compare_optimum(got[s], ref[s], slack=stop_slack(H[s], e_full[s]))

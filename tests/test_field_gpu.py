"""The benchmark's own workload at full size: the 2048 x 1489 x 5-band field with 1000 sources
(seed 1611, 128-pixel tiles, as bench.py times it).  Sampled sources against the oracle one by one:
ELBO, gradient and Hessian at the catalog, and the optimum of batched Newton."""
import numpy as np
import pytest
import torch

import synth
from oracle import celeste_oracle as O
from test_parity_gpu import check_elbo, check_grad, check_hess, compare_optimum, grad_natural_scale, hess_natural_scale, stop_slack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as P
    dev = torch.device("cuda:0")
    sc = synth.field(seed=1611, n_sources=1000)
    prob = P.Problem(sc, device=dev, tile_pixels=128)
    th0 = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(th0)
    e, g, h = prob.elbo_batch(th0)
    th = th0.clone()
    _, iters, status, elbo = prob.newton_batch(th)
    torch.cuda.synchronize()
    return dict(P=P, sc=sc, orc=O.Oracle(sc), e=e.cpu().numpy(), g=g.cpu().numpy(), h=h.cpu().numpy(),
                th=th.cpu().numpy(), status=status.cpu().numpy(), elbo=elbo.cpu().numpy(), iters=iters.cpu().numpy())


def _sample(run, k, seed, pred=None):
    sc, orc = run["sc"], run["orc"]
    n_px = np.array([orc.n_pixels(s) for s in range(sc.n_sources)])
    ok = [s for s in range(sc.n_sources) if orc.rects[s] and n_px[s] <= 12000 and (pred is None or pred(s))]
    return [int(s) for s in np.random.default_rng(seed).choice(ok, k, replace=False)]


def test_field_sampled_sources_at_the_catalog(run):
    orc, sc = run["orc"], run["sc"]
    # the source with the most neighbours too, whatever its size
    nn = [sum(len(v) for v in orc.nbr[s].values()) for s in range(sc.n_sources)]
    for s in _sample(run, 6, 1) + [int(np.argmax(nn))]:
        L, gL, HL = orc.elbo_grad_hess(s, sc.theta0[s], sc.theta0)
        check_elbo(run["e"][s], L, f"field s={s}")
        check_grad(run["g"][s], gL, f"field s={s}", natural=lambda: grad_natural_scale(orc, s, sc.theta0[s], sc.theta0))
        check_hess(run["h"][s], HL, f"field s={s}", natural=lambda: hess_natural_scale(orc, s, sc.theta0[s], sc.theta0))


def test_field_newton_optima(run):
    P, orc, sc = run["P"], run["orc"], run["sc"]
    assert (run["status"] == P.STATUS_CONVERGED).mean() >= 0.99
    for s in _sample(run, 3, 2, pred=lambda s: run["status"][s] == P.STATUS_CONVERGED):
        ref = orc.newton(s, sc.theta0[s], sc.theta0)
        assert abs(run["elbo"][s] - ref["elbo"]) <= 1e-6 * abs(ref["elbo"])
        L, _, H = orc.elbo_grad_hess(s, ref["theta"], sc.theta0)
        compare_optimum(run["th"][s], ref["theta"], slack=stop_slack(H, L))

"""Batching at survey scale: the 10 x 10 mosaic of overlapping exposures with 100,000 sources (1-12
exposures per source, patch radius 8-64 px), evaluated and optimised in one batch on the GPU.

The oracle cannot take the whole mosaic, so sampled sources are checked one by one: each against
the oracle on a sub-scene holding the exposures that contain the source and every source within
150 px of it, which has the same patches and neighbours for that source (patch radii are at most
64 px and the exposures' pixel scale is within 2 % of the world grid's)."""
import numpy as np
import pytest
import torch

from oracle import celeste_oracle as O
from synth.mosaic import mosaic
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
    sc = mosaic(seed=1611, device=dev)
    prob = P.Problem(sc, device=dev, tile_pixels=128)
    th0 = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(th0)
    e, g, h = prob.elbo_batch(th0)
    out = dict(P=P, sc=sc, prob=prob, th0=th0, e=e.cpu().numpy(), g=g.cpu().numpy(), h=h.cpu().numpy(),
               counts=prob.counts())
    return out


def sub_scene(sc, s, reach=150.0):
    d = np.hypot(*(sc.u0 - sc.u0[s]).T)
    keep = np.concatenate([[s], np.nonzero((d <= reach) & (np.arange(sc.n_sources) != s))[0]])
    imgs = []
    for im in sc.images:
        p = im.wcs[:4].reshape(2, 2) @ sc.u0[s] + im.wcs[4:]
        cx, cy = np.floor(p + 0.5)
        if 0 <= cx <= im.W - 1 and 0 <= cy <= im.H - 1:
            imgs.append(im)
    sub = type(sc)(imgs, sc.u0[keep], sc.radius[keep], sc.theta0[keep], sc.priors, sc.exp_nu, sc.exp_tau,
                   sc.dev_nu, sc.dev_tau)
    return sub, keep


def _pick(sc, counts_px, rng):
    n_img, rad = sc.truth["n_images"], sc.radius
    px = counts_px
    cand = []
    small = np.nonzero(px <= 60_000)[0]
    cand.append(small[np.argmax(n_img[small])])                  # most exposures
    cand.append(small[np.argmax(rad[small])])                    # largest radius within the size cap
    cand.extend(rng.choice(small, 4, replace=False))
    return [int(c) for c in dict.fromkeys(cand)]


def _pixels_per_source(sc):
    n_img, rad = sc.truth["n_images"], sc.radius
    return n_img * (2 * rad + 1) ** 2


def test_mosaic_layout(run):
    sc, c = run["sc"], run["counts"]
    n_img = sc.truth["n_images"]   # exposures whose pixel grid holds the catalog position
    assert c["sources"] == 100_000
    assert n_img.min() >= 1 and n_img.max() <= 12 and np.bincount(n_img).argmax() <= 3
    assert sc.radius.min() == 8 and sc.radius.max() == 64
    assert c["patches"] == int(n_img.sum())


def test_mosaic_sampled_sources_match_oracle(run):
    sc = run["sc"]
    rng = np.random.default_rng(11)
    for s in _pick(sc, _pixels_per_source(sc), rng):
        sub, keep = sub_scene(sc, s)
        orc = O.Oracle(sub)
        L, gL, HL = orc.elbo_grad_hess(0, sc.theta0[s], sc.theta0[keep])
        what = f"mosaic s={s} images={sc.truth['n_images'][s]} radius={sc.radius[s]}"
        check_elbo(run["e"][s], L, what)
        check_grad(run["g"][s], gL, what, natural=lambda: grad_natural_scale(orc, 0, sc.theta0[s], sc.theta0[keep]))
        check_hess(run["h"][s], HL, what, natural=lambda: hess_natural_scale(orc, 0, sc.theta0[s], sc.theta0[keep]))


def test_mosaic_newton(run):
    P, sc, prob = run["P"], run["sc"], run["prob"]
    th = run["th0"].clone()
    delta, iters, status, elbo = prob.newton_batch(th)
    torch.cuda.synchronize()
    status = status.cpu().numpy()
    iters = iters.cpu().numpy()
    assert (status == P.STATUS_NONFINITE).sum() == 0
    assert (status == P.STATUS_CONVERGED).mean() >= 0.99
    got = th.cpu().numpy()
    # two small converged sources against the oracle's own Newton solve (neighbours fixed at the start)
    px = _pixels_per_source(sc)
    ok = np.nonzero((status == P.STATUS_CONVERGED) & (px <= 3000))[0]
    for s in np.random.default_rng(5).choice(ok, 2, replace=False):
        sub, keep = sub_scene(sc, int(s))
        orc = O.Oracle(sub)
        ref = orc.newton(0, sc.theta0[s], sc.theta0[keep])
        assert abs(float(elbo[s]) - ref["elbo"]) <= 1e-6 * abs(ref["elbo"])
        L, _, H = orc.elbo_grad_hess(0, ref["theta"], sc.theta0[keep])
        compare_optimum(got[s], ref["theta"], slack=stop_slack(H, L))

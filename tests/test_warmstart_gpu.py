"""What the learned warm start gains: the network is trained by the library's kernels on
(patch, converged parameters) pairs of one seeded mosaic, then Newton runs on a held-out mosaic
once from the catalog and once from the warm start, to the same tolerance.  The warm start must
save Newton iterations and reach the same optima (the network only moves the starting point)."""
import json

import numpy as np
import pytest
import torch

from synth.mosaic import mosaic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as P
    from paper_1611_03404_gb300 import cnn
    return P, cnn, torch.device("cuda:0")


def _solve(P, sc, dev, theta_start):
    prob = P.Problem(sc, device=dev, tile_pixels=128)
    th0 = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(th0)          # neighbours fixed at the catalog in both runs
    th = theta_start.clone().contiguous()
    _, iters, status, elbo = prob.newton_batch(th)
    torch.cuda.synchronize()
    return prob, th, iters, status, elbo


def test_warm_start_saves_newton_iterations(env):
    P, cnn, dev = env
    train = mosaic(seed=2001, fields_x=4, fields_y=4, n_sources=16000, device=dev)
    prob, th_star, iters, status, _ = _solve(P, train, dev, torch.as_tensor(train.theta0, device=dev))
    ok = status == P.STATUS_CONVERGED
    x = prob.extract_patches()[ok].contiguous()
    u0 = torch.as_tensor(train.u0, device=dev)[ok]
    targets = cnn.training_targets(th_star[ok], u0)
    net = cnn.WarmStartCNN(dev, seed=7)
    hist = net.train(x, targets, epochs=8, batch=256, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]

    test = mosaic(seed=2002, fields_x=2, fields_y=2, n_sources=4000, device=dev)
    cat = torch.as_tensor(test.theta0, device=dev).contiguous()
    p_cat, th_c, it_c, st_c, el_c = _solve(P, test, dev, cat)
    pred = net.predict(p_cat.extract_patches())
    start = cnn.warm_start(cat, pred)
    _, th_w, it_w, st_w, el_w = _solve(P, test, dev, start)
    both = (st_c == P.STATUS_CONVERGED) & (st_w == P.STATUS_CONVERGED)
    rel = ((el_w - el_c) / el_c.abs())[both]
    same = float((rel.abs() <= 1e-6).float().mean())
    better_or_same = float((rel >= -1e-6).float().mean())
    # network error against the converged solutions, per parameter (standardised units)
    tgt = cnn.training_targets(th_c, torch.as_tensor(test.u0, device=dev))
    rmse = ((pred - tgt)[both] / net.sd).pow(2).mean(0).sqrt().cpu().numpy()
    report = {"train_pairs": int(ok.sum()), "loss_first_last": [hist[0], hist[-1]],
              "iters_catalog_mean": float(it_c.double().mean()), "iters_warm_mean": float(it_w.double().mean()),
              "converged_catalog": float((st_c == P.STATUS_CONVERGED).float().mean()),
              "converged_warm": float((st_w == P.STATUS_CONVERGED).float().mean()),
              "same_optimum_fraction": same, "same_or_better_fraction": better_or_same,
              "rmse_standardised": [round(float(v), 3) for v in rmse]}
    print("WARMSTART " + json.dumps(report))
    assert report["iters_warm_mean"] < report["iters_catalog_mean"]
    assert report["converged_warm"] >= report["converged_catalog"] - 0.005
    assert better_or_same >= 0.97

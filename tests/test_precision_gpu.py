"""Precision variants of the Hessian's Jacobian cross-product (the per-tile SYRK): float32 FMAs and
four tensor-core forms (TF32 operands; BF16 hi + lo; BF16 hi + mid + lo; TF32 big + small).  Each
result is compared with the float64 oracle on sampled sources of a seeded field; the measured
errors are printed (pytest -s) next to the plain float32 form's.

Only the cross-product block moves between the modes (the ELBO, the gradient and every other
Hessian term take the same float32 path), so ELBO and gradient must stay within the standard
tolerances in every mode.  The Hessian is held to the standard 1e-4 in float32 and in the two
forms whose products keep float32's precision: BF16 split three ways with the six products down
to 2^-16 of the leading one (each product to ~2^-24) and TF32 split two ways with three products
(~2^-21).  The short forms are held to what their operands allow: 5e-4 with BF16 hi + lo (about
16 significant bits per product: entries near the 1e-2 floor of the natural scale, formed by
cancellation, measured up to 1.2e-4) and 5e-2 with plain TF32 (11 significant bits; measured
1.3e-2).  Newton must reach the oracle's optimum in every form (the Hessian only steers the
steps)."""
import json

import numpy as np
import pytest
import torch

import synth
from oracle import celeste_oracle as O
from test_parity_gpu import (ELBO_RTOL, GRAD_FLOOR, GRAD_RTOL, HESS_FLOOR, HESS_RTOL, compare_optimum, stop_slack)

pytestmark = pytest.mark.gpu

MODES = {"fp32": 0, "tf32": 1, "bf16x3": 2, "bf16x6": 3, "tf32x3": 4}
HESS_BOUND = {"fp32": HESS_RTOL, "bf16x6": HESS_RTOL, "tf32x3": HESS_RTOL, "bf16x3": 5e-4, "tf32": 5e-2}


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as P
    sc = synth.field(seed=1614, W=1024, H=745, n_sources=250)
    orc = O.Oracle(sc)
    rng = np.random.default_rng(0)
    sample = [int(s) for s in rng.choice(sc.n_sources, 8, replace=False) if orc.rects[s]]
    refs = {s: orc.elbo_grad_hess(s, sc.theta0[s], sc.theta0) for s in sample}
    return P, sc, orc, sample, refs


def rel_errors(e, g, h, L, gL, HL):
    el = abs(e - L) / abs(L)
    gs = np.maximum(np.abs(gL), GRAD_FLOOR * np.abs(gL).max())
    ge = (np.abs(g - gL) / gs).max()
    d = np.sqrt(np.abs(np.outer(np.diag(HL), np.diag(HL))))
    hs = np.maximum(np.abs(HL), HESS_FLOOR * d)
    he = (np.abs(h - HL) / np.where(hs > 0, hs, 1.0)).max()
    return el, ge, he


@pytest.mark.parametrize("mode", list(MODES))
def test_precision_mode_errors(setup, mode):
    P, sc, orc, sample, refs = setup
    dev = torch.device("cuda:0")
    prob = P.Problem(sc, device=dev, tile_pixels=128, hessian_mode=MODES[mode])
    th = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(th.clone())
    e, g, h = prob.elbo_batch(th)
    e, g, h = e.cpu().numpy(), g.cpu().numpy(), h.cpu().numpy()
    errs = np.array([rel_errors(e[s], g[s], h[s], *refs[s]) for s in sample])
    worst = errs.max(0)
    # Newton from the catalog, then the oracle's own solve on three sampled sources
    th2 = th.clone()
    _, iters, status, elbo = prob.newton_batch(th2)
    torch.cuda.synchronize()
    got = th2.cpu().numpy()
    conv = float((status == P.STATUS_CONVERGED).float().mean())
    opt_err = []
    for s in sample[:3]:
        ref = orc.newton(s, sc.theta0[s], sc.theta0)
        L, _, H = orc.elbo_grad_hess(s, ref["theta"], sc.theta0)
        compare_optimum(got[s], ref["theta"], slack=stop_slack(H, L))
        opt_err.append(abs(float(elbo[s]) - ref["elbo"]) / abs(ref["elbo"]))
    print("PRECISION " + json.dumps({"mode": mode, "elbo_rel": worst[0], "grad_rel": worst[1], "hess_rel": worst[2],
                                     "converged_elbo_rel": max(opt_err), "converged_fraction": conv,
                                     "newton_iters_mean": float(iters.double().mean())}))
    assert worst[0] <= ELBO_RTOL and worst[1] <= GRAD_RTOL
    assert worst[2] <= HESS_BOUND[mode]
    assert max(opt_err) <= 1e-6

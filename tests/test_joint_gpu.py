"""Joint objective on the GPU against the float64 oracle: with the background rendered in window
mode, the per-source gradient and Hessian are the joint objective's gradient and diagonal blocks;
celeste_joint_cross_hessian gives its cross-source blocks.  Tolerances as in the parity tests
(1e-4 of max(|entry|, 1e-2 of the entry's natural scale)), the natural scale of a cross entry
being the sum of the magnitudes of its per-pixel terms."""
import numpy as np
import pytest
import torch

import synth
from oracle import celeste_oracle as O
from oracle import joint_oracle as JO
from test_parity_gpu import check_elbo, check_grad, check_hess, grad_natural_scale, hess_natural_scale

pytestmark = pytest.mark.gpu

HESS_RTOL, HESS_FLOOR = 1e-4, 1e-2


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as pkg
    return pkg


def check_cross(hh, H, natural, what=""):
    scale = np.maximum(np.abs(H), HESS_FLOOR * natural)
    r = np.abs(hh - H) / np.where(scale > 0, scale, 1.0)
    i, j = np.unravel_index(r.argmax(), r.shape)
    assert np.all(r <= HESS_RTOL), f"{what} cross worst {r.max():.3e} at ({i},{j}): {hh[i, j]} vs {H[i, j]}"


@pytest.mark.parametrize("case", ["tiny3", "tiny5_tiles", "tiny6_rotated"])
def test_joint_blocks_match_oracle(P, case):
    if case == "tiny3":
        sc, tile = synth.tiny(seed=11, n_sources=3, n_images=3), 256
    elif case == "tiny5_tiles":
        sc, tile = synth.tiny(seed=3, n_sources=5, n_images=2, H=40, W=44, radius=(6, 12)), 128
    else:
        sc, tile = synth.tiny(seed=21, n_sources=6, n_images=3, H=44, W=48, radius=(5, 11)), 128
    orc = O.Oracle(sc)
    rng = np.random.default_rng(3)
    theta = sc.theta0 + 0.03 * rng.standard_normal(sc.theta0.shape)
    dev = torch.device("cuda:0")
    prob = P.Problem(sc, device=dev, tile_pixels=tile)
    th = torch.as_tensor(theta, device=dev).contiguous()
    prob.render_background(th, mode=P.NBR_WINDOW)
    e, g, h = prob.elbo_batch(th)
    pairs = prob.joint_pairs()
    cross = prob.cross_hessian(th)
    torch.cuda.synchronize()
    e, g, h, cross = e.cpu().numpy(), g.cpu().numpy(), h.cpu().numpy(), cross.cpu().numpy()
    assert [tuple(p) for p in pairs] == JO.overlapping_pairs(orc)
    assert len(pairs) > 0
    _, gJ, HJ = JO.joint_value_grad_hess(orc, theta)
    for s in range(sc.n_sources):
        f = JO.clipped_elbo_fn(orc, s, theta)
        with torch.no_grad():
            L = float(f(torch.as_tensor(theta[s])))
        check_elbo(e[s], L, f"{case} source {s}")
        check_grad(g[s], gJ[s], f"{case} source {s}", natural=lambda s=s: grad_natural_scale(orc, s, theta[s], theta))
        check_hess(h[s], HJ[s, :, s, :], f"{case} source {s}",
                   natural=lambda s=s: hess_natural_scale(orc, s, theta[s], theta))
    for k, (s, t) in enumerate(pairs):
        ref = HJ[s, :, t, :]
        nat = JO.cross_block_formula(orc, theta, s, t, absolute=True)
        check_cross(cross[k], ref, nat, f"{case} pair {s},{t}")


def test_cross_requires_window_background(P):
    sc = synth.tiny(seed=11, n_sources=3, n_images=3)
    prob = P.Problem(sc, device=torch.device("cuda:0"))
    th = torch.as_tensor(sc.theta0, device="cuda:0").contiguous()
    prob.render_background(th)
    with pytest.raises(P.CelesteError):
        prob.cross_hessian(th)

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


def _compare_joint(P, orc, got, ref_theta, J_solver):
    from test_parity_gpu import compare_optimum, stop_slack
    Jg, _, _ = JO.joint_value_grad_hess(orc, got)
    Jr, _, Hr = JO.joint_value_grad_hess(orc, ref_theta)
    assert abs(J_solver - Jg) <= 1e-6 * abs(Jg)          # the solver's own J is J at its result
    assert abs(Jg - Jr) <= 1e-6 * abs(Jr)
    S = got.shape[0]
    slack = stop_slack(Hr.reshape(S * 27, S * 27), Jr).reshape(S, 27)
    for s in range(S):
        compare_optimum(got[s], ref_theta[s], slack=slack[s])


def test_joint_value_matches_oracle(P):
    sc = synth.tiny(seed=3, n_sources=5, n_images=2, H=40, W=44, radius=(6, 12))
    orc = O.Oracle(sc)
    rng = np.random.default_rng(4)
    theta = sc.theta0 + 0.03 * rng.standard_normal(sc.theta0.shape)
    prob = P.Problem(sc, device=torch.device("cuda:0"), tile_pixels=128)
    J = prob.joint_value(torch.as_tensor(theta, device="cuda:0").contiguous())
    with torch.no_grad():
        ref = float(JO.joint_fn(orc)(torch.as_tensor(theta)))
    check_elbo(J, ref, "joint value")


def test_joint_newton_from_the_catalog(P):
    """From the catalog of a three-source scene the joint solve reaches the oracle's joint maximum
    (J within the ELBO tolerance, parameters within compare_optimum's bounds widened by the
    stopping rule's slack along the joint Hessian's weakly curved directions).  The GPU solves each
    subproblem inexactly (preconditioned CG in the preconditioner's norm) where this oracle solves
    it exactly, so the paths differ and the GPU gets up to 100 outer iterations."""
    sc = synth.tiny(seed=11, n_sources=3, n_images=3)
    orc = O.Oracle(sc)
    ref = JO.joint_newton(orc, sc.theta0)
    assert ref["status"] == O.STATUS_CONVERGED
    prob = P.Problem(sc, device=torch.device("cuda:0"), tile_pixels=256)
    th = torch.as_tensor(sc.theta0, device="cuda:0").contiguous()
    res = prob.joint_newton(th, max_iter=100)
    print(f"JOINT_NEWTON catalog gpu {res} oracle iters {ref['iters']} J {ref['elbo']}")
    assert res["status"] == P.STATUS_CONVERGED
    _compare_joint(P, orc, th.cpu().numpy(), ref["theta"], res["J"])


def test_joint_newton_returns_to_a_nearby_maximum(P):
    """Started next to the oracle's joint maximum of a four-source scene (all six pairs overlap),
    the joint solve returns to it.  (From the catalog the joint objective has several local maxima
    here, and paths through inexact and exact subproblems may end in different ones.)"""
    sc = synth.tiny(seed=5, n_sources=4, n_images=2, H=36, W=40, radius=(5, 9))
    orc = O.Oracle(sc)
    ref = JO.joint_newton(orc, sc.theta0)
    assert ref["status"] == O.STATUS_CONVERGED
    rng = np.random.default_rng(9)
    start = ref["theta"] + 0.02 * rng.standard_normal(ref["theta"].shape)
    prob = P.Problem(sc, device=torch.device("cuda:0"), tile_pixels=128)
    th = torch.as_tensor(start, device="cuda:0").contiguous()
    res = prob.joint_newton(th, max_iter=100)
    print(f"JOINT_NEWTON local gpu {res} oracle J {ref['elbo']}")
    assert res["status"] == P.STATUS_CONVERGED
    _compare_joint(P, orc, th.cpu().numpy(), ref["theta"], res["J"])

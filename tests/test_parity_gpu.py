"""CUDA path vs the float64 oracle, element by element, through the C ABI.

Tolerances (the plain float32 GPU path against the float64 oracle):
  ELBO      |dL|   <= 1e-6 |L|
  gradient  |dg_i| <= 1e-4 max(|g_i|, 1e-3 max_j |g_j|)
  Hessian   |dH_ij| <= 1e-4 max(|H_ij|, 1e-2 sqrt(|H_ii H_jj|))
The floors make "relative" meaningful for entries that are near zero by cancellation.  A Hessian
entry is a sum of per-pixel float32 terms whose magnitudes are bounded by its natural scale
sqrt(|H_ii H_jj|); float32 rounding leaves an absolute error of a few ulps (~1e-7) of that scale, so
an entry far below it is checked to 1e-6 of the natural scale rather than to 1e-4 of itself.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import celeste_oracle as O

pytestmark = pytest.mark.gpu

ELBO_RTOL, GRAD_RTOL, HESS_RTOL = 1e-6, 1e-4, 1e-4
GRAD_FLOOR, HESS_FLOOR = 1e-3, 1e-2


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as pkg
    return pkg


def check_elbo(e, L, what=""):
    assert abs(e - L) <= ELBO_RTOL * abs(L), f"{what} elbo {e} vs {L}: rel {abs(e - L) / abs(L):.3e}"


def _per_pixel_fn(orc, s, nbr_theta):
    """theta -> [KL, l_pixel...]: the terms whose (signed) sum is the source's objective."""
    data = orc._patch_data(s, nbr_theta)

    def per_pixel(th):
        out = [O.kl_source(th, orc.priors).reshape(1)]
        for (im, px, py, x, lgx, bE, bV, psf) in data:
            EG, EG2 = O.source_moments(th, im, px, py, psf, orc.mix)
            E = im.sky + im.iota * (bE + EG)
            V = im.iota ** 2 * (bV + EG2 - EG * EG)
            out.append(O.pixel_term(x, E, V, lgx))
        return torch.cat(out)
    return per_pixel


def grad_natural_scale(orc, s, theta, nbr_theta):
    """Per parameter, sum over the source's pixels of |d l_pixel / d theta_i| plus |d KL / d theta_i|:
    the magnitude of the terms whose sum is the gradient entry (the analogue of the Hessian's
    sqrt(|H_ii H_jj|))."""
    f = _per_pixel_fn(orc, s, nbr_theta)
    J = torch.func.jacrev(f)(torch.as_tensor(theta, dtype=torch.float64).clone())
    return J.abs().sum(0).numpy()


def hess_natural_scale(orc, s, theta, nbr_theta):
    """Per entry, sum over the pixels (and the KL) of |d2 term / d theta_i d theta_j|."""
    f = _per_pixel_fn(orc, s, nbr_theta)
    Hp = torch.func.jacfwd(torch.func.jacrev(f))(torch.as_tensor(theta, dtype=torch.float64).clone())
    return Hp.abs().sum(0).numpy()


def check_grad(gg, g, what="", natural=None):
    """|dg_i| <= 1e-4 max(|g_i|, 1e-3 max|g|); an entry that fails is held to 1e-4 of 1e-2 of its
    natural scale (grad_natural_scale, passed as a callable evaluated only then): near a stationary
    point an entry is a small sum of large per-pixel float32 terms (the flux gradient sum w1 f0
    vanishes at the flux optimum), like the Hessian entries below their floor."""
    scale = np.maximum(np.abs(g), GRAD_FLOOR * np.abs(g).max())
    r = np.abs(gg - g) / scale
    if not np.all(r <= GRAD_RTOL) and natural is not None:
        scale = np.maximum(scale, HESS_FLOOR * natural())
        r = np.abs(gg - g) / scale
    assert np.all(r <= GRAD_RTOL), f"{what} grad worst {r.max():.3e} at {int(r.argmax())}: {gg[r.argmax()]} vs {g[r.argmax()]}"


def check_hess(hh, H, what="", natural=None):
    """|dH_ij| <= 1e-4 max(|H_ij|, 1e-2 sqrt(|H_ii H_jj|)); an entry that fails is held to 1e-4 of
    1e-2 of its own natural scale (hess_natural_scale, evaluated only then): entries built from a
    cancelling pixel sum (a flux-gradient sum times a brightness derivative, say) can sit far below
    sqrt(|H_ii H_jj|) while their terms do not."""
    d = np.sqrt(np.abs(np.outer(np.diag(H), np.diag(H))))
    scale = np.maximum(np.abs(H), HESS_FLOOR * d)
    r = np.abs(hh - H) / np.where(scale > 0, scale, 1.0)
    if not np.all(r <= HESS_RTOL) and natural is not None:
        scale = np.maximum(scale, HESS_FLOOR * natural())
        r = np.abs(hh - H) / np.where(scale > 0, scale, 1.0)
    i, j = np.unravel_index(r.argmax(), r.shape)
    assert np.all(r <= HESS_RTOL), (f"{what} hess worst {r.max():.3e} at ({i},{j}): {hh[i, j]} vs {H[i, j]}, "
                                    f"natural scale {d[i, j]:.4g}")


def run_gpu(P, scene, theta, nbr_theta=None, tile=256):
    dev = torch.device("cuda:0")
    prob = P.Problem(scene, device=dev, tile_pixels=tile)
    th = torch.as_tensor(theta, device=dev).contiguous()
    nb = torch.as_tensor(theta if nbr_theta is None else nbr_theta, device=dev).contiguous()
    prob.render_background(nb)
    elbo, grad, hess = prob.elbo_batch(th)
    v, _, _ = prob.elbo_batch(th, want=P.WANT_ELBO)
    torch.cuda.synchronize()
    return elbo.cpu().numpy(), grad.cpu().numpy(), hess.cpu().numpy(), v.cpu().numpy()


def compare_all(P, scene, theta, sources=None, nbr_theta=None, tile=256, what=""):
    e, g, h, v = run_gpu(P, scene, theta, nbr_theta, tile)
    orc = O.Oracle(scene)
    nb = theta if nbr_theta is None else nbr_theta
    for s in (range(scene.n_sources) if sources is None else sources):
        if not orc.rects[s]:
            assert e[s] == pytest.approx(-float(O.kl_source(torch.as_tensor(theta[s]), scene.priors)), rel=1e-12)
            continue
        L, gL, HL = orc.elbo_grad_hess(s, theta[s], nb)
        check_elbo(e[s], L, f"{what} s={s}")
        check_elbo(v[s], L, f"{what} value-only s={s}")
        check_grad(g[s], gL, f"{what} s={s}", natural=lambda: grad_natural_scale(orc, s, theta[s], nb))
        check_hess(h[s], HL, f"{what} s={s}", natural=lambda: hess_natural_scale(orc, s, theta[s], nb))


def _spread(theta, rng):
    """Move a start point to a generic interior point where every term of the objective is active."""
    th = theta.copy()
    th[:, 6] = rng.uniform(-1, 1, len(th))
    th[:, 8] = th[:, 10] = np.log(rng.uniform(0.02, 0.2, len(th)))
    th[:, 15:19] = np.log(rng.uniform(0.01, 0.1, (len(th), 4)))
    th[:, 23:27] = np.log(rng.uniform(0.01, 0.1, (len(th), 4)))
    return th


def test_single_source_41px_at_start(P):
    """One isolated source, 5 bands x 41x41 px, at its catalog start point."""
    sc = synth.single_source(seed=1611, size=41)
    compare_all(P, sc, sc.theta0, what="single41")


@pytest.mark.parametrize("seed,is_gal", [(5, True), (6, False), (7, None)])
def test_single_source_interior_points(P, seed, is_gal):
    sc = synth.single_source(seed=seed, size=31, is_gal=is_gal)
    th = _spread(sc.theta0, np.random.default_rng(seed))
    compare_all(P, sc, th, what=f"single31 seed={seed}")


@pytest.mark.parametrize("seed", [11, 12])
def test_overlapping_sources_rotated_wcs(P, seed):
    """Neighbours in the same patches, rotated and scaled pixel maps, several bands."""
    sc = synth.tiny(seed=seed, n_sources=4, n_images=3, H=34, W=38, radius=(6, 12))
    th = _spread(sc.theta0, np.random.default_rng(seed))
    nb = th.copy()
    nb[:, 0:2] += 0.2     # neighbours fixed somewhere other than the targets
    compare_all(P, sc, th, nbr_theta=nb, what=f"tiny seed={seed}")


@pytest.mark.parametrize("tile", [128, 512, 1024])
def test_tile_sizes_and_ragged_tails(P, tile):
    sc = synth.tiny(seed=13, n_sources=3, n_images=2, H=40, W=44, radius=(9, 17))
    th = _spread(sc.theta0, np.random.default_rng(2))
    compare_all(P, sc, th, tile=tile, what=f"tile={tile}")


def test_edge_patches_clipped_and_maximal(P):
    """A source in an image corner (clipped patch), one outside an image, and an R=64 patch."""
    sc = synth.tiny(seed=17, n_sources=3, n_images=2, H=140, W=150, radius=(6, 6))
    sc.u0 = np.array([[1.2, 0.7], [75.0, 70.0], [148.6, 60.0]])
    sc.theta0[:, 0:2] = sc.u0 + 0.1
    sc.radius = np.array([6, 64, 9], np.int32)
    th = _spread(sc.theta0, np.random.default_rng(3))
    compare_all(P, sc, th, what="edges")


@pytest.mark.parametrize("axis_logit,scale", [(-7.6, 1500.0), (-4.6, 50.0)])
def test_thin_extended_galaxy(P, axis_logit, scale):
    """A galaxy far thinner than a pixel and far longer than its patch (axis ratio 5e-4, half-light
    radius 1500 px; and 1e-2, 50 px), the shape Newton reached on a faint mosaic source: its
    components' covariances are ill-conditioned (a c / det up to ~1e5), where float32 tables lose
    the precision matrix and its shape derivatives."""
    sc = synth.single_source(seed=9, size=31, is_gal=True)
    th = _spread(sc.theta0, np.random.default_rng(9))
    th[0, 3], th[0, 5], th[0, 6] = axis_logit, math.log(scale), 4.7
    compare_all(P, sc, th, what=f"thin galaxy axis_logit={axis_logit} scale={scale}")


@pytest.mark.parametrize("cta_sources", [0, -1], ids=["four_warps", "one_warp"])
def test_newton_matches_oracle_optimum(P, cta_sources):
    """Batched GPU Newton reaches the oracle's optimum within 1e-4 per identified parameter, with the
    subproblems on four warps (few active sources: the default here) and on one warp."""
    sc = synth.single_source(seed=1611, size=41)
    dev = torch.device("cuda:0")
    prob = P.Problem(sc, device=dev)
    th = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(th.clone())
    delta, iters, status, elbo = prob.newton_batch(th, cta_sources=cta_sources)
    torch.cuda.synchronize()
    ref = O.Oracle(sc).newton(0, sc.theta0[0], sc.theta0)
    assert int(status[0]) == P.STATUS_CONVERGED and int(iters[0]) <= 50
    got = th.cpu().numpy()[0]
    assert abs(float(elbo[0]) - ref["elbo"]) <= 1e-6 * abs(ref["elbo"])
    compare_optimum(got, ref["theta"])


def stop_slack(H, L, ftol=1e-8):
    """Per free parameter, how far the ELBO-tolerance stopping rule leaves the optimum undetermined:
    Newton stops once the predicted gain is below ftol |L|, and along a direction of curvature c > 0
    that gain stays below ftol |L| within sqrt(2 ftol |L| / c) of the maximum: for parameter i,
    sqrt(2 ftol |L| [(-H)^-1]_ii) over the directions of positive curvature.  Three times that.
    Along a direction of non-positive curvature (a flat ridge, e.g. the profile mixture of a galaxy
    too small to tell exponential from de Vaucouleurs) nothing bounds the stopping point, so the
    parameters with a share in such a direction are left unbounded."""
    w, V = np.linalg.eigh(-0.5 * (H + H.T))
    flat = w <= 1e-12 * max(np.abs(w).max(), 1e-300)
    d = (V[:, ~flat] ** 2 / w[~flat]).sum(axis=1)
    slack = 3.0 * np.sqrt(2.0 * ftol * abs(L) * d)
    slack[(V[:, flat] ** 2).sum(axis=1) > 1e-6] = np.inf
    return slack


def compare_optimum(got, ref, tol=1e-4, slack=None):
    """Per-parameter comparison in the constrained space; a type's own parameters only count when
    that type has posterior probability > 1e-3, and the angle (mod pi) only when the axis ratio
    is below 1 - 1e-3 (otherwise they are unidentified).  `slack` (free-parameter units, from
    stop_slack) widens each bound by what the ELBO stopping tolerance leaves undetermined along
    weakly curved directions, mapped through the parameter's transform."""
    def sig(x):
        return 1.0 / (1.0 + math.exp(-x)) if x >= 0 else math.exp(x) / (1.0 + math.exp(x))

    def exp(x):
        return math.exp(x) if x < 700.0 else math.inf

    sl = np.zeros(27) if slack is None else np.asarray(slack)

    def image(f, x, w):
        # how far f moves when its argument moves by up to w from x (the slack's image through the
        # transform; a derivative at x understates it where f flattens, e.g. a sigmoid at 27)
        return max(abs(f(x + w) - f(x)), abs(f(x - w) - f(x)))

    a_gal = sig(ref[6])
    assert abs(sig(got[6]) - a_gal) <= tol + image(sig, ref[6], sl[6])
    assert np.all(np.abs(got[0:2] - ref[0:2]) <= tol + sl[0:2])
    if a_gal > 1e-3:
        assert abs(sig(got[2]) - sig(ref[2])) <= tol + image(sig, ref[2], sl[2])
        assert abs(sig(got[3]) - sig(ref[3])) <= tol + image(sig, ref[3], sl[3])
        assert abs(exp(got[5]) - exp(ref[5])) <= tol * exp(ref[5]) + image(exp, ref[5], sl[5])
        if sig(ref[3]) < 1 - 1e-3:
            assert abs(math.remainder(got[4] - ref[4], math.pi)) <= tol + sl[4]
        idx = [9, 10] + list(range(19, 27))
        assert np.all(np.abs(got[idx] - ref[idx]) <= tol * np.maximum(1, np.abs(ref[idx])) + sl[idx])
    if a_gal < 1 - 1e-3:
        idx = [7, 8] + list(range(11, 19))
        assert np.all(np.abs(got[idx] - ref[idx]) <= tol * np.maximum(1, np.abs(ref[idx])) + sl[idx])


def test_newton_graph_matches_plain_launches(P):
    """Iterations run as CUDA graphs (several per host check, the graph kept across calls) give
    bit-identical results to one plain launch sequence per iteration, also when max_iter is not a
    multiple of the graph length and when sources stop mid-graph."""
    sc = synth.tiny(seed=5, n_sources=12, n_images=3, H=120, W=130, radius=(6, 12))
    dev = torch.device("cuda:0")
    prob = P.Problem(sc, device=dev, tile_pixels=128)
    start = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(start.clone())
    runs = []
    # (cta_sources 6: one warp per subproblem until at most 6 of the 12 sources are left, then four)
    for graph_iters, max_iter, cta in ((1, 50, 0), (4, 50, 0), (4, 50, 0), (3, 7, 0), (1, 7, 0), (1, 50, 6),
                                       (4, 50, 6)):
        th = start.clone()
        delta, iters, status, elbo = prob.newton_batch(th, max_iter=max_iter, graph_iters=graph_iters,
                                                       cta_sources=cta)
        torch.cuda.synchronize()
        runs.append((max_iter, th.cpu().numpy(), delta.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy(),
                     elbo.cpu().numpy()))
    for a, b in ((0, 1), (0, 2), (3, 4), (5, 6)):
        for x, y in zip(runs[a][1:], runs[b][1:]):
            np.testing.assert_array_equal(x, y)
    assert runs[3][3].max() <= 7
    # the switch between the layouts changes rounding only
    assert np.all(runs[5][4] == runs[0][4])
    np.testing.assert_allclose(runs[5][5], runs[0][5], rtol=1e-7)


def test_refresh_pixels_matches_a_fresh_bind(P):
    """New counts written into the same device images: celeste_problem_refresh_pixels re-gathers the
    patch pixels, and the evaluation equals that of a problem bound from scratch on the new images."""
    sc = synth.tiny(seed=12, n_sources=4, n_images=3, H=34, W=38, radius=(6, 12))
    dev = torch.device("cuda:0")
    pix = [torch.as_tensor(np.ascontiguousarray(im.pixels, np.float32)).to(dev) for im in sc.images]
    prob = P.Problem(sc, device=dev, tile_pixels=128, device_pixels=pix)
    th = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(th)
    before = [t.cpu().numpy() for t in prob.elbo_batch(th)]
    rng = np.random.default_rng(3)
    new = [np.asarray(rng.poisson(np.maximum(im.pixels, 0.0) + 5.0), np.float32) for im in sc.images]
    for d, n in zip(pix, new):
        d.copy_(torch.as_tensor(n))
    prob.refresh_pixels()
    prob.render_background(th)
    after = [t.cpu().numpy() for t in prob.elbo_batch(th)]
    for im, n in zip(sc.images, new):
        im.pixels = n
    fresh = P.Problem(sc, device=dev, tile_pixels=128)
    fresh.render_background(th)
    ref = [t.cpu().numpy() for t in fresh.elbo_batch(th)]
    for a, r in zip(after, ref):
        np.testing.assert_array_equal(a, r)
    assert not np.array_equal(after[0], before[0])

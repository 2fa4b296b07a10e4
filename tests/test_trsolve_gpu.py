"""Trust-region subproblem on the GPU (float64, tridiagonal route) vs the oracle (eigendecomposition
route), through the C ABI.  The solution of the subproblem is unique outside the hard case, so the
steps must agree to float64 accuracy; the hard case is checked by its optimality conditions."""
import numpy as np
import pytest
import torch

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


def _problems(seed, n):
    rng = np.random.default_rng(seed)
    Bs, gs, ds = [], [], []
    for t in range(n):
        M = rng.normal(size=(27, 27))
        shift = rng.uniform(-1.5, 0.5) if t % 3 else 0.0
        B = M @ M.T / 27 + shift * np.eye(27)
        if t % 5 == 0:      # badly scaled, like a Hessian over positions, shapes and log-variances
            s = np.exp(rng.uniform(-4, 4, 27))
            B = s[:, None] * B * s[None, :]
        Bs.append(B)
        gs.append(rng.normal(size=27) * rng.choice([1e-3, 1.0, 100.0]))
        ds.append(rng.choice([0.01, 0.3, 1.0, 10.0, 1e4]))
    return np.array(Bs), np.array(gs), np.array(ds)


def _lambda_rounding(B, g, delta, pr, mo):
    """How much the model value at the boundary solution moves when the multiplier lambda is
    rounded by 64 units in the last place of the spectrum's scale.  On the boundary the solution
    is p(lambda) = -(B + lambda I)^-1 g with |p(lambda)| = delta; next to the pole
    lambda = -lambda_min, |p| ~ 1/(lambda + lambda_min), so a float64 lambda fixes p only to this
    extent (in the eigenbasis, so that no further rounding enters)."""
    if np.linalg.norm(pr) < delta * (1 - 1e-9):
        return 0.0
    w, V = np.linalg.eigh(B)
    gt = V.T @ g
    lam = -(g @ pr + pr @ B @ pr) / max(pr @ pr, 1e-300)
    scale = max(abs(lam), np.abs(w).max())
    worst = 0.0
    for s in (-1.0, 1.0):
        den = w + lam + s * 64 * np.finfo(float).eps * scale
        if np.any(den <= 0):
            continue
        p = -V @ (gt / den)
        n = np.linalg.norm(p)
        if n > delta:
            p *= delta / n
        worst = max(worst, g @ p + 0.5 * p @ B @ p - mo)
    return worst


def _check_against_oracle(B, g, d, p, pred):
    for i in range(len(d)):
        pr, predr, _ = O.tr_subproblem(g[i], B[i], d[i])
        assert np.linalg.norm(p[i]) <= d[i] * (1 + 1e-9)
        # both solutions must reach the same minimum of the model, to 1e-7 plus what rounding the
        # multiplier lambda in float64 leaves undetermined (large only next to the pole)
        mg = g[i] @ p[i] + 0.5 * p[i] @ B[i] @ p[i]
        mo = g[i] @ pr + 0.5 * pr @ B[i] @ pr
        assert mg <= mo + 1e-7 * abs(mo) + _lambda_rounding(B[i], g[i], d[i], pr, mo) + 1e-300, i
        # pred is formed in the tridiagonal basis, mg here in the original one: they agree to the
        # rounding of the two terms g.p and p.B.p/2, which can be far larger than their sum
        terms = np.linalg.norm(g[i]) * np.linalg.norm(p[i]) + np.linalg.norm(B[i], 2) * (p[i] @ p[i])
        assert abs(pred[i] + mg) <= 1e-12 * terms + 1e-9 * abs(mg) + 1e-300, i
        # the step itself is compared where the subproblem is well conditioned: lambda* well above
        # the pole -lambda_min (|p| ~ 1/(lambda + lambda_min) amplifies rounding near it)
        lam_star = -(g[i] @ pr + pr @ B[i] @ pr) / max(pr @ pr, 1e-300)
        lmin = np.linalg.eigvalsh(B[i])[0]
        scale = np.abs(np.linalg.eigvalsh(B[i])).max()
        if np.linalg.norm(pr) < d[i] * (1 - 1e-9) or lam_star + lmin > 1e-6 * scale:
            assert np.abs(p[i] - pr).max() <= 1e-6 * max(np.abs(pr).max(), 1e-300), i


@pytest.mark.parametrize("warps", [1, 4])
def test_subproblem_matches_oracle(P, warps):
    """One warp per problem (iterations with many active sources) and one four-warp CTA per problem
    (the few-source iterations), each against the oracle's eigendecomposition solution."""
    B, g, d = _problems(0, 400)
    dev = torch.device("cuda:0")
    p, pred, hard = P.tr_solve_batch(*(torch.as_tensor(a, device=dev).contiguous() for a in (B, g, d)), warps=warps)
    _check_against_oracle(B, g, d, p.cpu().numpy(), pred.cpu().numpy())


@pytest.mark.parametrize("warps", [1, 4])
def test_subproblem_multiplier_hint_changes_only_rounding(P, warps):
    """The Newton iteration passes each source's previous multiplier to place the first pass of the
    multiplier search; exact, close, far and absent hints must reach the same solution: the
    multiplier to the search's tolerance and the model value to 1e-8 plus what float64 leaves
    undetermined next to the pole (the unhinted solve is held to the oracle by
    test_subproblem_matches_oracle)."""
    B, g, d = _problems(1, 240)
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(a, device=dev).contiguous()
    model = lambda p: np.einsum("ij,ij->i", g, p) + 0.5 * np.einsum("ij,ijk,ik->i", p, B, p)
    p0, pred0, _, lam0 = P.tr_solve_batch(t(B), t(g), t(d), warps=warps, return_lambda=True)
    p0, lam0 = p0.cpu().numpy(), lam0.cpu().numpy()
    m0 = model(p0)
    assert np.any(lam0 > 0)
    eig = np.array([np.linalg.eigvalsh(b) for b in B])
    scale, lmin = np.abs(eig).max(axis=1), eig[:, 0]
    # what float64 leaves undetermined: the reduction's backward error (tens of ulps of |B|) moves
    # the pole -lambda_min, and |p(lambda)| ~ 1/(lambda + lambda_min) next to it, so |p| is fixed
    # to about 64 eps |B| / (lambda + lambda_min) relative; along the boundary path the model moves
    # by lambda delta^2 times that
    lam_ref = np.where(lam0 > 0, lam0, 0.0)
    res = np.where(lam_ref > 0, np.minimum(1.0, 64 * np.finfo(float).eps * scale /
                                           np.maximum(lam_ref + lmin, 1e-300)), 0.0)
    slack = lam_ref * d ** 2 * res + 1e-8 * np.abs(m0) + 1e-300
    for f in (1.0, 1.0 + 1e-7, 0.3, 4.0, 1e3, 1e-3):
        hint = np.where(lam0 > 0, lam0 * f, -1.0)
        p, pred, _, lam = P.tr_solve_batch(t(B), t(g), t(d), warps=warps, lam_hint=t(hint), return_lambda=True)
        p, lam = p.cpu().numpy(), lam.cpu().numpy()
        assert np.all(np.linalg.norm(p, axis=1) <= d * (1 + 1e-9)), f
        m = model(p)
        bad = np.abs(m - m0) > slack
        assert not bad.any(), (f, np.nonzero(bad)[0][:5], m[bad][:3], m0[bad][:3])
        both = (lam0 > 0) & (lam > 0)
        # |p(lambda)| = delta to 1e-10 relative: lambda is fixed to about that times its scale
        assert np.all(np.abs(lam[both] - lam0[both]) <= 1e-6 * (lam0[both] + scale[both])), f


@pytest.mark.parametrize("warps", [1, 4])
def test_subproblem_hard_case(P, warps):
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.normal(size=(27, 27)))
    lam = np.linspace(-2.0, 5.0, 27)
    B = Q @ np.diag(lam) @ Q.T
    g = Q[:, 1:] @ rng.normal(size=26) * 0.1     # no component on the most negative eigenvector
    delta = 5.0
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(a, device=dev).contiguous()
    p, pred, hard = P.tr_solve_batch(t(B[None]), t(g[None]), t(np.array([delta])), warps=warps)
    p = p.cpu().numpy()[0]
    assert int(hard[0]) == 1
    assert abs(np.linalg.norm(p) - delta) <= 1e-9 * delta
    # optimality: (B - lambda_min I) p = -g
    np.testing.assert_allclose((B + 2.0 * np.eye(27)) @ p, -g, atol=1e-7)
    pr, _, hr = O.tr_subproblem(g, B, delta)
    assert hr and abs(pr @ B @ pr / 2 + g @ pr - (p @ B @ p / 2 + g @ p)) <= 1e-9 * (1 + abs(g @ pr))


def test_reciprocal_error_bound(P):
    """The solver's reciprocal (approximate seed + two Newton-Raphson steps) against the correctly
    rounded float64 quotient: within 2 ulps over the normal range, both signs, including powers of
    two, their neighbours and the ends of the documented range."""
    rng = np.random.default_rng(7)
    x = np.concatenate([
        np.exp(rng.uniform(-700, 700, 200000)) * rng.choice([-1.0, 1.0], 200000),
        1.0 + rng.uniform(0, 1, 100000),
        np.ldexp(1.0, np.arange(-1021, 1022)),
        np.nextafter(np.ldexp(1.0, np.arange(-1021, 1022)), 0.0),
        np.nextafter(np.ldexp(1.0, np.arange(-1021, 1022)), np.inf),
        [1.0, -1.0, 3.0, 1.0 / 3.0, 0.1, 1e-300, 1e300, 2.0 ** -1022, 2.0 ** 1021],
    ])
    r = P.tr_reciprocal(torch.as_tensor(x, device="cuda")).cpu().numpy()
    exact = 1.0 / x
    ulp = np.spacing(np.abs(exact))
    err = np.abs(r - exact) / ulp
    assert np.all(np.isfinite(r)), x[~np.isfinite(r)][:5]
    assert err.max() <= 2.0, (err.max(), x[np.argmax(err)])
    # the documented ends: zero and subnormal inputs give NaN, |x| > 2^1022 gives 0
    edge = P.tr_reciprocal(torch.tensor([0.0, 5e-324, 2.0 ** 1023, -(2.0 ** 1023)], dtype=torch.float64,
                                        device="cuda")).cpu().numpy()
    assert np.isnan(edge[0]) and np.isnan(edge[1]) and edge[2] == 0.0 and edge[3] == 0.0


def _near_pole(seed, gap, delta=16.0):
    """A subproblem whose root sits `gap` above the pole -lambda_min: B indefinite (lambda_min =
    -8.64e-4) with a spectrum up to 3.4e4, g weighted towards the stiff directions (0.01 sqrt|lambda|
    per eigenvector, as a Newton iteration's gradient in a flat valley), its component along the
    smallest eigenvector set so that |p(lambda*)| = delta at lambda* = -lambda_min + gap."""
    rng = np.random.default_rng(seed)
    lam = np.concatenate([[-8.64e-4], np.geomspace(1.3e-4, 3.4e4, 26)])
    Q, _ = np.linalg.qr(rng.normal(size=(27, 27)))
    B = Q @ np.diag(lam) @ Q.T
    B = 0.5 * (B + B.T)
    lstar = -lam[0] + gap
    gam = rng.normal(size=27) * np.sqrt(np.abs(lam)) * 0.01
    gam[0] = 0.0
    rest = np.sum(gam[1:] ** 2 / (lam[1:] + lstar) ** 2)
    if rest >= delta ** 2:
        gam[1:] *= 0.9 * delta / np.sqrt(rest)
        rest = np.sum(gam[1:] ** 2 / (lam[1:] + lstar) ** 2)
    gam[0] = np.sqrt(delta ** 2 - rest) * (lam[0] + lstar)
    return B, Q @ gam, delta, lstar


@pytest.mark.parametrize("warps", [1, 4])
def test_subproblem_near_pole_with_far_hint(P, warps):
    """Roots 1e-6 .. 3e-6 above the pole with the multiplier hint far above them (the previous
    subproblem's multiplier): the search narrows the bracket to the float64 resolution of the
    spectrum before |p| reaches delta to 1e-10.  A positive definite point with |p| > delta has been
    seen by then, which rules the hard case out; the step must be the boundary solution (no hard
    case, positive predicted decrease, the oracle's model value up to what the pole leaves
    undetermined), whatever the hint."""
    cases = [(_near_pole(s, gap), hint) for s in range(6) for gap in (1e-6, 1.4e-6, 3e-6) for hint in (1.0, 10.0, -1.0)]
    B = np.array([c[0][0] for c in cases])
    g = np.array([c[0][1] for c in cases])
    d = np.array([c[0][2] for c in cases])
    lstar = np.array([c[0][3] for c in cases])
    hint = np.array([c[1] for c in cases])
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(a, device=dev).contiguous()
    p, pred, hard, lam = P.tr_solve_batch(t(B), t(g), t(d), warps=warps, lam_hint=t(hint), return_lambda=True)
    p, pred, hard = p.cpu().numpy(), pred.cpu().numpy(), hard.cpu().numpy()
    for i in range(len(cases)):
        pr, _, hr = O.tr_subproblem(g[i], B[i], d[i])
        assert not hr
        assert hard[i] == 0, (i, hint[i])
        assert pred[i] > 0, (i, pred[i])
        assert np.linalg.norm(p[i]) <= d[i] * (1 + 1e-9)
        mg = g[i] @ p[i] + 0.5 * p[i] @ B[i] @ p[i]
        mo = g[i] @ pr + 0.5 * pr @ B[i] @ pr
        scale = np.abs(np.linalg.eigvalsh(B[i])).max()
        gap = lstar[i] - 8.64e-4
        slack = lstar[i] * d[i] ** 2 * min(1.0, 64 * np.finfo(float).eps * scale / gap)
        assert mg <= mo + 1e-7 * abs(mo) + slack, (i, mg, mo, slack)

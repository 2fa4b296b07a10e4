"""Pins of the joint-objective oracle (CPU).

The joint objective (every covered pixel counted once, each source's light on its own window)
is checked against: central finite differences of its value; its reduction to the per-source
objectives when no windows overlap; the per-source objective with clipped neighbours for its
gradient and diagonal Hessian blocks; the closed form of the cross blocks from per-pixel
Jacobians; and, for a neighbour whose window covers the target's, the per-source objective of
the main oracle (clipping then changes nothing)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import celeste_oracle as O
from oracle import joint_oracle as JO


@pytest.fixture(scope="module")
def scene():
    return synth.tiny(seed=11, n_sources=3, n_images=3)


@pytest.fixture(scope="module")
def joint(scene):
    orc = O.Oracle(scene)
    rng = np.random.default_rng(5)
    theta = scene.theta0 + 0.05 * rng.standard_normal(scene.theta0.shape)
    val, g, H = JO.joint_value_grad_hess(orc, theta)
    return orc, theta, val, g, H


@pytest.fixture(scope="module")
def exact_joint(scene):
    orc = O.Oracle(scene)
    return orc, JO.joint_newton(orc, scene.theta0)


def test_scene_has_overlaps(joint):
    orc = joint[0]
    assert JO.overlapping_pairs(orc) == [(0, 1), (0, 2), (1, 2)]


def test_gradient_matches_finite_differences(joint):
    orc, theta, val, g, _ = joint
    J = JO.joint_fn(orc)
    rng = np.random.default_rng(1)
    for _ in range(8):
        s, j = int(rng.integers(0, theta.shape[0])), int(rng.integers(0, 27))
        h = 1e-5
        tp, tm = theta.copy(), theta.copy()
        tp[s, j] += h
        tm[s, j] -= h
        with torch.no_grad():
            fd = (float(J(torch.as_tensor(tp))) - float(J(torch.as_tensor(tm)))) / (2 * h)
        assert abs(fd - g[s, j]) <= 1e-6 * max(1.0, abs(g[s, j])) + 1e-9 * abs(val), (s, j, fd, g[s, j])


def test_hessian_symmetric(joint):
    H = joint[4]
    S = H.shape[0]
    M = H.reshape(S * 27, S * 27)
    assert np.abs(M - M.T).max() <= 1e-9 * np.abs(M).max()


def test_diagonal_blocks_are_the_clipped_per_source_objective(joint):
    orc, theta, _, g, H = joint
    for s in range(theta.shape[0]):
        f = JO.clipped_elbo_fn(orc, s, theta)
        th = torch.as_tensor(theta[s]).clone()
        gs = torch.func.grad(f)(th).numpy()
        Hs = torch.func.hessian(f)(th).numpy()
        assert np.allclose(gs, g[s], rtol=1e-10, atol=1e-9 * np.abs(g[s]).max())
        assert np.allclose(Hs, H[s, :, s, :], rtol=1e-10, atol=1e-9 * np.abs(Hs).max())


def test_cross_blocks_match_the_closed_form(joint):
    orc, theta, _, _, H = joint
    for (s, t) in JO.overlapping_pairs(orc):
        C = JO.cross_block_formula(orc, theta, s, t)
        ref = H[s, :, t, :]
        scale = np.abs(ref).max()
        assert scale > 0
        assert np.abs(C - ref).max() <= 1e-9 * scale, (s, t, np.abs(C - ref).max(), scale)
        assert np.abs(H[t, :, s, :] - ref.T).max() <= 1e-9 * scale


def test_disjoint_windows_reduce_to_per_source_objectives(scene):
    # shrink the windows until none overlaps: J is then the sum of the per-source objectives
    # (no neighbours anywhere) and every cross block vanishes
    sc = synth.tiny(seed=11, n_sources=3, n_images=3)
    sc.radius = np.full_like(sc.radius, 1)
    orc = O.Oracle(sc)
    assert JO.overlapping_pairs(orc) == []
    val, g, H = JO.joint_value_grad_hess(orc, sc.theta0)
    per = sum(orc.elbo(s, sc.theta0[s], sc.theta0) for s in range(sc.n_sources))
    assert abs(val - per) <= 1e-10 * abs(per)
    for s in range(sc.n_sources):
        for t in range(sc.n_sources):
            if s != t:
                assert np.abs(H[s, :, t, :]).max() == 0.0


def test_covering_neighbour_clips_nothing():
    # two sources; the second's window covers the first's in every image, so the first's
    # clipped objective is the main oracle's per-source objective
    sc = synth.tiny(seed=11, n_sources=2, n_images=2)
    sc.radius = np.array([3, 40], dtype=sc.radius.dtype)
    orc = O.Oracle(sc)
    for (n, x0, x1, y0, y1) in orc.rects[0]:
        big = [r for r in orc.rects[1] if r[0] == n][0]
        assert big[1] <= x0 and x1 <= big[2] and big[3] <= y0 and y1 <= big[4]
    f = JO.clipped_elbo_fn(orc, 0, sc.theta0)
    with torch.no_grad():
        v = float(f(torch.as_tensor(sc.theta0[0])))
    ref = orc.elbo(0, sc.theta0[0], sc.theta0)
    assert abs(v - ref) <= 1e-12 * abs(ref)


def test_joint_newton_reaches_a_joint_maximum(scene, exact_joint):
    # the joint solve ends at a strict local maximum of J (-J's Hessian positive definite) whose
    # Newton decrement g^T (-H)^-1 g is within the stopping rule's 2 ftol |J|; block-coordinate
    # sweeps on the clipped per-source objectives (the per-source method) raise J monotonically
    # towards it from below without passing it
    orc, res = exact_joint
    assert res["status"] == O.STATUS_CONVERGED
    val, g, H = JO.joint_value_grad_hess(orc, res["theta"])
    n = scene.n_sources * 27
    Hm = -H.reshape(n, n)
    assert np.linalg.eigvalsh(Hm).min() > 0
    dec = g.ravel() @ np.linalg.solve(Hm, g.ravel())
    assert dec <= 2.5e-8 * abs(val)
    th = scene.theta0.copy()
    vals = []
    for _ in range(3):
        prev = th.copy()
        for s in range(scene.n_sources):
            f = JO.clipped_elbo_fn(orc, s, prev)

            def value(x, f=f):
                with torch.no_grad():
                    return float(f(torch.as_tensor(x)))

            def vgh(x, f=f):
                t = torch.as_tensor(x).clone()
                return value(x), torch.func.grad(f)(t).numpy(), torch.func.hessian(f)(t).numpy()

            th[s] = O.trust_region_newton(value, vgh, prev[s].copy())["theta"]
        vals.append(JO.joint_value_grad_hess(orc, th)[0])
    assert vals[0] < vals[1] < vals[2] <= val + 1e-9 * abs(val)


def _random_blocks(rng, S=2, indefinite=False):
    """A symmetric block-sparse test problem of S sources (27 each): SPD diagonal blocks with
    spread curvatures, weak cross blocks; optionally one negative eigenvalue."""
    n = 27 * S
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.exp(rng.uniform(-3, 5, n))
    if indefinite:
        lam[0] = -0.5
    B = (Q * lam) @ Q.T
    H = -B.reshape(S, 27, S, 27).copy()
    g = rng.standard_normal((S, 27))
    return B, H, g


def test_steihaug_interior_step_is_an_inexact_newton_step():
    rng = np.random.default_rng(21)
    B, H, g = _random_blocks(rng)
    M = JO.preconditioner(H)
    p, boundary, rstop, k = JO.steihaug(g, B, M, 1e12, 200)
    assert not boundary and rstop
    r = B @ p.ravel() + g.ravel()
    assert np.linalg.norm(r) <= 1e-2 * np.linalg.norm(g) * (1 + 1e-12)


def test_steihaug_boundary_and_model_decrease():
    rng = np.random.default_rng(22)
    for indefinite in (False, True):
        B, H, g = _random_blocks(rng, indefinite=indefinite)
        M = JO.preconditioner(H)
        Mn = lambda v: math.sqrt(sum(v[s] @ M[s] @ v[s] for s in range(len(M))))
        q = lambda v: float(g.ravel() @ v.ravel() + 0.5 * v.ravel() @ B @ v.ravel())
        delta = 0.1 * Mn(np.stack([np.linalg.solve(M[s], g[s]) for s in range(len(M))]))
        p, boundary, rstop, k = JO.steihaug(g, B, M, delta, 200)
        assert boundary and not rstop
        assert abs(Mn(p) - delta) <= 1e-9 * delta
        # at least the decrease of the preconditioned Cauchy point (Steihaug: the first CG
        # iterate is that point, and CG only lowers the model along the path)
        z = np.stack([np.linalg.solve(M[s], g[s]) for s in range(len(M))])
        zBz = float(z.ravel() @ B @ z.ravel())
        gz = float((g * z).sum())
        tmax = delta / Mn(z)
        t = tmax if zBz <= 0 else min(gz / zBz, tmax)
        assert q(p) <= q(-t * z) + 1e-12 * abs(q(-t * z))
        assert q(p) < 0


def test_preconditioner_blocks_are_positive_definite():
    rng = np.random.default_rng(23)
    B, H, g = _random_blocks(rng, indefinite=True)
    for Ms, s in zip(JO.preconditioner(H), range(2)):
        assert np.linalg.eigvalsh(Ms).min() > 0
        Bs = -H[s, :, s, :]
        shift = np.diag(Ms - Bs)
        assert np.allclose(shift, shift[0]) and shift[0] >= 1e-4 * np.abs(np.diag(Bs)).max() * (1 - 1e-12)


def test_joint_newton_steihaug_reaches_the_exact_solve_maximum(scene, exact_joint):
    # the CG-subproblem solve (the GPU's algorithm) ends at the exact-subproblem solve's maximum
    orc, ref = exact_joint
    res = JO.joint_newton_steihaug(orc, scene.theta0)
    assert res["status"] == O.STATUS_CONVERGED
    assert abs(res["elbo"] - ref["elbo"]) <= 1e-6 * abs(ref["elbo"])


def test_cross_blocks_match_finite_differences_of_the_gradient(joint):
    # an independent route to the cross blocks: central differences of dJ/dtheta_s under moves
    # of theta_t
    orc, theta, _, _, H = joint
    J = JO.joint_fn(orc)
    grad = lambda th: torch.func.grad(J)(torch.as_tensor(th).clone()).numpy()
    rng = np.random.default_rng(7)
    for (s, t) in JO.overlapping_pairs(orc):
        for j in rng.choice(27, 3, replace=False):
            h = 1e-5
            tp, tm = theta.copy(), theta.copy()
            tp[t, j] += h
            tm[t, j] -= h
            fd = (grad(tp)[s] - grad(tm)[s]) / (2 * h)
            ref = H[s, :, t, j]
            assert np.abs(fd - ref).max() <= 1e-5 * max(np.abs(H[s, :, t, :]).max(), 1e-12), (s, t, j)

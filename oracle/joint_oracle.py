"""FP64 CPU oracle for the joint objective over overlapping sources.  TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may import this
module.  It shares no code with the CUDA path.

The paper's concluding section names, as the next step after optimising each light source with
its neighbours held fixed, finding a stationary point of the objective over all light sources
jointly.  That objective is the ELBO of all the pixels the sources' windows cover, every pixel
counted once:

    J(theta) = sum_n sum_{m in U_n} l(x_m, E_m, V_m) - sum_s KL_s(theta_s),
    U_n = union over s of W_{s,n},
    E_m = sky_n + iota_n sum_{s: m in W_{s,n}} E[G_s](m),
    V_m = iota_n^2 sum_{s: m in W_{s,n}} Var[G_s](m),

with W_{s,n} source s's window in image n (the per-source objective's pixel set) and each
source's light counted on the pixels of its own window.  Then dJ/dtheta_s is the gradient of the
per-source objective whose neighbours are counted on their own windows only ("clipped"), the
diagonal Hessian blocks are that objective's Hessian, and the cross block of two sources is

    d2J / dtheta_s dtheta_t = sum_{m in W_s cap W_t} l_EE dE/ds dE/dt^T
                              + l_EV (dE/ds dV/dt^T + dV/ds dE/dt^T)

(E and V are sums over sources, so their mixed second derivatives vanish, and l_VV = 0).
Everything here is plain float64 PyTorch; derivatives by automatic differentiation.
"""
import math

import numpy as np
import torch

from .celeste_oracle import (STATUS_CONVERGED, STATUS_MAX_ITER, STATUS_NONFINITE, STATUS_RADIUS_COLLAPSE,
                             kl_source, pixel_term, source_moments, trust_region_newton)

torch.set_default_dtype(torch.float64)


def _image_windows(orc):
    """Per image n: list of (source, x0, x1, y0, y1) inclusive windows."""
    by_image = {}
    for s, lst in enumerate(orc.rects):
        for (n, x0, x1, y0, y1) in lst:
            by_image.setdefault(n, []).append((s, x0, x1, y0, y1))
    return by_image


def _union_pixels(orc, n, wins):
    """Union of the windows of image n: pixel coordinates, counts, log-factorials, and per window
    the boolean mask of its pixels within the union list."""
    im = orc.scene.images[n]
    cover = np.zeros((im.H, im.W), bool)
    for (_, x0, x1, y0, y1) in wins:
        cover[y0:y1 + 1, x0:x1 + 1] = True
    ys, xs = np.nonzero(cover)
    px = torch.as_tensor(xs.astype(np.float64))
    py = torch.as_tensor(ys.astype(np.float64))
    x = torch.as_tensor(im.pixels[ys, xs].astype(np.float64))
    masks = [torch.as_tensor((xs >= x0) & (xs <= x1) & (ys >= y0) & (ys <= y1)) for (_, x0, x1, y0, y1) in wins]
    return im, px, py, x, torch.lgamma(x + 1.0), masks


def joint_fn(orc):
    """theta [S, 27] -> J(theta) (a pure function, for value and autodiff)."""
    data = []
    for n, wins in sorted(_image_windows(orc).items()):
        im, px, py, x, lgx, masks = _union_pixels(orc, n, wins)
        data.append((im, px, py, x, lgx, [(w[0], mk, orc.psf_for(w[0], n)) for w, mk in zip(wins, masks)]))
    priors, mix, S = orc.priors, orc.mix, orc.scene.n_sources

    def J(theta):
        total = torch.zeros(())
        for s in range(S):
            total = total - kl_source(theta[s], priors)
        for (im, px, py, x, lgx, srcs) in data:
            EGs = torch.zeros_like(px)
            VGs = torch.zeros_like(px)
            for (s, mk, psf) in srcs:
                EG, EG2 = source_moments(theta[s], im, px, py, psf, mix)
                EGs = EGs + torch.where(mk, EG, torch.zeros_like(EG))
                VGs = VGs + torch.where(mk, EG2 - EG * EG, torch.zeros_like(EG))
            E = im.sky + im.iota * EGs
            V = im.iota ** 2 * VGs
            total = total + pixel_term(x, E, V, lgx).sum()
        return total
    return J


def joint_value_grad_hess(orc, theta):
    """(J, dJ/dtheta [S, 27], d2J/dtheta2 [S, 27, S, 27]) at theta [S, 27]."""
    J = joint_fn(orc)
    th = torch.as_tensor(theta, dtype=torch.float64).clone()
    with torch.no_grad():
        val = float(J(th))
    g = torch.func.grad(J)(th)
    H = torch.func.hessian(J)(th)
    return val, g.numpy(), H.numpy()


def clipped_elbo_fn(orc, s, nbr_theta):
    """theta_s -> the per-source objective of s with each neighbour's light counted on the pixels
    of its own window only (the neighbours at nbr_theta)."""
    data = []
    for (n, x0, x1, y0, y1) in orc.rects[s]:
        im = orc.scene.images[n]
        ys, xs = torch.meshgrid(torch.arange(y0, y1 + 1, dtype=torch.float64),
                                torch.arange(x0, x1 + 1, dtype=torch.float64), indexing="ij")
        px, py = xs.reshape(-1), ys.reshape(-1)
        x = torch.as_tensor(im.pixels[y0:y1 + 1, x0:x1 + 1].astype(np.float64)).reshape(-1)
        bE = torch.zeros_like(px)
        bV = torch.zeros_like(px)
        with torch.no_grad():
            for t in orc.nbr[s][n]:
                tx0, tx1, ty0, ty1 = [r for r in orc.rects[t] if r[0] == n][0][1:]
                inside = (px >= tx0) & (px <= tx1) & (py >= ty0) & (py <= ty1)
                EG, EG2 = source_moments(torch.as_tensor(nbr_theta[t]), im, px, py, orc.psf_for(t, n), orc.mix)
                bE += torch.where(inside, EG, torch.zeros_like(EG))
                bV += torch.where(inside, EG2 - EG * EG, torch.zeros_like(EG))
        data.append((im, px, py, x, torch.lgamma(x + 1.0), bE, bV, orc.psf_for(s, n)))
    priors, mix = orc.priors, orc.mix

    def f(theta):
        total = -kl_source(theta, priors)
        for (im, px, py, x, lgx, bE, bV, psf) in data:
            EG, EG2 = source_moments(theta, im, px, py, psf, mix)
            E = im.sky + im.iota * (bE + EG)
            V = im.iota ** 2 * (bV + EG2 - EG * EG)
            total = total + pixel_term(x, E, V, lgx).sum()
        return total
    return f


def cross_block_formula(orc, theta, s, t, absolute=False):
    """d2J/dtheta_s dtheta_t from per-pixel Jacobians (the closed form in the module docstring):
    sum over the pixels of W_s cap W_t of l_EE dE_s dE_t^T + l_EV (dE_s dV_t^T + dV_s dE_t^T).
    absolute: the sum of the three terms' magnitudes instead (each entry's natural scale)."""
    theta = np.asarray(theta, np.float64)
    out = np.zeros((27, 27))
    wins = _image_windows(orc)
    for n, ws in wins.items():
        ws_s = [w for w in ws if w[0] == s]
        ws_t = [w for w in ws if w[0] == t]
        if not ws_s or not ws_t:
            continue
        (_, a0, a1, b0, b1), (_, c0, c1, d0, d1) = ws_s[0], ws_t[0]
        x0, x1, y0, y1 = max(a0, c0), min(a1, c1), max(b0, d0), min(b1, d1)
        if x0 > x1 or y0 > y1:
            continue
        im = orc.scene.images[n]
        ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        xs, ys = xs.ravel(), ys.ravel()
        px = torch.as_tensor(xs.astype(np.float64))
        py = torch.as_tensor(ys.astype(np.float64))
        x = torch.as_tensor(im.pixels[ys, xs].astype(np.float64))
        # rate mean and variance from every source whose window holds the pixel
        E = torch.full_like(px, float(im.sky))
        V = torch.zeros_like(px)
        for (u, e0, e1, f0, f1) in ws:
            inside = torch.as_tensor((xs >= e0) & (xs <= e1) & (ys >= f0) & (ys <= f1))
            EG, EG2 = source_moments(torch.as_tensor(theta[u]), im, px, py, orc.psf_for(u, n), orc.mix)
            E = E + im.iota * torch.where(inside, EG, torch.zeros_like(EG))
            V = V + im.iota ** 2 * torch.where(inside, EG2 - EG * EG, torch.zeros_like(EG))
        l_EE = -x / E ** 2 - 3.0 * x * V / E ** 4
        l_EV = x / E ** 3

        def EV(th, u):
            EG, EG2 = source_moments(th, im, px, py, orc.psf_for(u, n), orc.mix)
            return torch.stack([im.iota * EG, im.iota ** 2 * (EG2 - EG * EG)])

        Js = torch.func.jacrev(lambda th: EV(th, s))(torch.as_tensor(theta[s]))   # [2, npix, 27]
        Jt = torch.func.jacrev(lambda th: EV(th, t))(torch.as_tensor(theta[t]))
        dEs, dVs, dEt, dVt = Js[0], Js[1], Jt[0], Jt[1]
        f = torch.abs if absolute else (lambda z: z)
        out += (f(torch.einsum("m,mi,mj->mij", l_EE, dEs, dEt)).sum(0)
                + f(torch.einsum("m,mi,mj->mij", l_EV, dEs, dVt)).sum(0)
                + f(torch.einsum("m,mi,mj->mij", l_EV, dVs, dEt)).sum(0)).numpy()
    return out


def overlapping_pairs(orc):
    """Sorted list of source pairs (s, t), s < t, whose windows overlap in some image."""
    pairs = set()
    for s, d in enumerate(orc.nbr):
        for n, ts in d.items():
            for t in ts:
                if s < t:
                    pairs.add((s, t))
    return sorted(pairs)


def joint_newton(orc, theta0, **opts):
    """Trust-region Newton on f = -J over all sources at once (the same rules as the per-source
    solve, Nocedal & Wright Alg. 4.1 with the exact subproblem), in float64.
    Returns dict(theta [S, 27], elbo = J, iters, status)."""
    J = joint_fn(orc)
    shape = np.asarray(theta0).shape

    def value(th):
        with torch.no_grad():
            return float(J(torch.as_tensor(th.reshape(shape))))

    def vgh(th):
        t = torch.as_tensor(th.reshape(shape)).clone()
        n = t.numel()
        g = torch.func.grad(J)(t).reshape(n)
        H = torch.func.hessian(J)(t).reshape(n, n)
        return value(th), g.numpy(), H.numpy()

    res = trust_region_newton(value, vgh, np.asarray(theta0, np.float64).ravel(), **opts)
    res["theta"] = res["theta"].reshape(shape)
    return res


# ----------------------------------------------------------------------------- joint Newton, CG subproblems
PRECOND_LADDER = (1e-4, 1e-3, 1e-2, 1e-1, 1.0, 10.0)


def preconditioner(H):
    """Per source s the matrix M_s = -H_ss + mu I for the first mu in PRECOND_LADDER x max_i |H_ii|
    that makes it positive definite (else diag(|H_ii|) + max_i |H_ii|); returns the list of M_s."""
    S = H.shape[0]
    out = []
    for s in range(S):
        B = -H[s, :, s, :]
        scale = max(np.abs(np.diag(B)).max(), 1e-300)
        M = None
        for mu in PRECOND_LADDER:
            C = B + mu * scale * np.eye(27)
            try:
                np.linalg.cholesky(C)
                M = C
                break
            except np.linalg.LinAlgError:
                continue
        if M is None:
            M = np.diag(np.abs(np.diag(B)) + scale)
        out.append(M)
    return out


def steihaug(g, B, M, delta, max_cg):
    """Preconditioned conjugate gradients for min g.p + p.B.p/2, |p|_M <= delta, with Steihaug's
    stopping rules (Nocedal & Wright Alg. 7.2): negative curvature or the boundary -> step to the
    boundary along the current direction; stop once |r| <= 1e-2 |g|.  M is block-diagonal (list of
    27 x 27 blocks), g and the vectors are [S, 27].  Returns (p, on_boundary, residual_converged,
    iterations)."""
    Minv = lambda v: np.stack([np.linalg.solve(M[s], v[s]) for s in range(len(M))])
    Mdot = lambda a, b: sum(a[s] @ M[s] @ b[s] for s in range(len(M)))
    n = g.size
    x = np.zeros_like(g)
    r = g.copy()
    z = Minv(r)
    d = -z
    rz = float((r * z).sum())
    eps = 1e-2 * np.linalg.norm(g)
    xMx, xMd, dMd = 0.0, 0.0, rz

    def tau():
        disc = max(xMd * xMd + dMd * (delta * delta - xMx), 0.0)
        return (-xMd + math.sqrt(disc)) / dMd

    if not (np.linalg.norm(g) > 0 and rz > 0):
        return x, False, False, 0
    for j in range(max_cg):
        Bd = (B @ d.reshape(n)).reshape(g.shape)
        kappa = float((d * Bd).sum())
        if not kappa > 0:
            return x + tau() * d, True, False, j + 1
        alpha = rz / kappa
        if xMx + 2 * alpha * xMd + alpha * alpha * dMd >= delta * delta:
            return x + tau() * d, True, False, j + 1
        x = x + alpha * d
        r = r + alpha * Bd
        xMx += 2 * alpha * xMd + alpha * alpha * dMd
        if np.linalg.norm(r) <= eps:
            return x, False, True, j + 1
        z = Minv(r)
        rz_new = float((r * z).sum())
        beta = rz_new / rz
        rz = rz_new
        xMd = beta * (xMd + alpha * dMd)
        dMd = rz + beta * beta * dMd
        d = -z + beta * d
    return x, False, False, max_cg


def joint_newton_steihaug(orc, theta0, max_iter=100, max_cg=100, ftol=1e-8, gtol=1e-10, delta_max=1e4, eta=0.1,
                          delta_min=1e-12):
    """Trust-region Newton on f = -J (Nocedal & Wright Alg. 4.1: acceptance eta, radius x1/4 below
    rho = 1/4 and x2 above 3/4 on the boundary, ftol on accepted changes, on the Newton decrement
    of a converged subproblem and on the prediction of a rejected step, gtol on max |grad|) with
    each subproblem solved by `steihaug` in the norm of `preconditioner`'s blocks; the radius
    starts at the norm of the block-diagonal Newton step, sqrt(g^T M^-1 g), and is capped at
    delta_max times that.
    Returns dict(theta, elbo = J, iters, status, cg_iters)."""
    J = joint_fn(orc)
    th = np.asarray(theta0, np.float64).copy()
    S = th.shape[0]
    n = S * 27

    def value(t):
        with torch.no_grad():
            return float(J(torch.as_tensor(t)))

    def grad_hess(t):
        tt = torch.as_tensor(t).clone()
        return torch.func.grad(J)(tt).numpy(), torch.func.hessian(J)(tt).numpy()

    f = -value(th)
    gJ, H = grad_hess(th)
    M = preconditioner(H)
    g0 = -gJ
    rz0 = float(sum(g0[s] @ np.linalg.solve(M[s], g0[s]) for s in range(S)))
    delta = math.sqrt(rz0) if rz0 > 0 else 1.0
    cap = delta_max * delta
    status, it, cg = STATUS_MAX_ITER, 0, 0
    while it < max_iter:
        g = -gJ
        B = -H.reshape(n, n)
        p, boundary, rstop, k = steihaug(g, B, M, delta, max_cg)
        cg += k
        if not (np.isfinite(f) and np.all(np.isfinite(g))):
            status = STATUS_NONFINITE
            break
        if np.abs(g).max() <= gtol:
            status = STATUS_CONVERGED
            break
        it += 1
        pred = -(float((g * p).sum()) + 0.5 * float(p.reshape(n) @ B @ p.reshape(n)))
        if not boundary and rstop and pred <= ftol * abs(f):
            status = STATUS_CONVERGED
            break
        trial = th + p
        dJ = value(trial) + f   # J(trial) - J(th)
        rho = dJ / pred if pred > 0 else -1.0
        if not np.isfinite(dJ):
            rho = -1.0
        if rho <= eta and pred <= ftol * abs(f):
            status = STATUS_CONVERGED      # a rejected step that promised no more than ftol |f|
            break
        if rho < 0.25:
            delta *= 0.25
        elif rho > 0.75 and boundary:
            delta = min(2.0 * delta, cap)
        if rho > eta:
            f_new = f - dJ
            done = abs(dJ) <= ftol * abs(f_new)
            th, f = trial, f_new
            gJ, H = grad_hess(th)
            M = preconditioner(H)
            if done:
                status = STATUS_CONVERGED
                break
        if delta < delta_min:
            status = STATUS_RADIUS_COLLAPSE
            break
    return dict(theta=th, elbo=-f, iters=it, status=status, cg_iters=cg)

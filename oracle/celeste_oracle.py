"""FP64 CPU oracle for the Celeste per-source objective.  TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may import
this module.  It shares no code with the CUDA path: it reads the same seeded scene
(`synth`), and nothing else.

What it computes (paper: "Learning an Astronomical Catalog of the Visible Universe
through Scalable Bayesian Inference", Regier et al.):

* Sec. "The Celeste Model": pixel counts x_nm ~ Poisson(F_nm); F_nm is a deterministic
  function of the catalog and the image metadata Lambda_n (PSF, sky, calibration,
  pixel<->world map).  Each source has a Bernoulli type a_s (star/galaxy), a lognormal
  reference-band brightness r_s, normal colours c_s, a position mu_s and galaxy shape
  phi_s.
* Sec. "Variational Inference", Eq. (1)-(2): the ELBO L = E_q[log p(x,z) - log q(z)];
  Eq. (3): q(z) = prod_s q(r_s|a_s) q(c_s|a_s) q(a_s) with lognormal / normal /
  Bernoulli factors conjugate to the priors.
* Same section: each source's parameters are optimised with the neighbours' held fixed,
  by Newton's method with a trust region, using the exact gradient and dense Hessian.

The paper defers the pixel-level formulas to its predecessor, so these readings are
used (each is listed with its rationale in the design notes):
  - 27 free parameters per source (layout in `synth`); brightness moments of a
    lognormal flux with diagonal colour variances; reference band r;
  - profiles evaluated at pixel centres: star = PSF mixture; galaxy = PSF mixture
    convolved with an exponential/de Vaucouleurs Gaussian mixture stretched by
    Sigma_g = scale^2 R(angle) diag(1, axis^2) R(angle)^T mapped to pixels by the WCS;
  - PSF evaluated at the source's catalog position and held fixed;
  - E[F] = sky + iota * sum_s' E[G_s'], Var[F] = iota^2 * sum_s' Var[G_s'] over the
    target and its neighbours (neighbours at fixed parameters);
  - E_q[log F] by the second-order delta method log E[F] - Var[F] / (2 E[F]^2);
  - per-source objective: the target's patch pixels (square, clipped) minus its KL;
  - trust-region Newton after Nocedal & Wright (Algorithm 4.1 with the eigenvalue form
    of the More-Sorensen subproblem, hard case included).

Gradient and Hessian are the exact derivatives of the written-out ELBO taken by
PyTorch automatic differentiation in float64 (a library primitive used as one step).
"""
import math

import numpy as np
import torch

torch.set_default_dtype(torch.float64)

N_PARAMS = 27
# Parameter indices (free, unconstrained).
I_U = slice(0, 2)
I_DEV, I_AXIS, I_ANGLE, I_SCALE, I_GAL = 2, 3, 4, 5, 6
I_R1 = (7, 9)             # mean of log reference-band flux, star / galaxy
I_RHO = (8, 10)           # log variance of log flux
I_C1 = (slice(11, 15), slice(19, 23))
I_GAM = (slice(15, 19), slice(23, 27))
# log flux_b = log flux_r + COLOR_MIX[b] . c,  colour c_j = log(flux_{j+1}/flux_j)
COLOR_MIX = torch.tensor([[-1., -1., 0., 0.], [0., -1., 0., 0.], [0., 0., 0., 0.], [0., 0., 1., 0.], [0., 0., 1., 1.]])

STATUS_CONVERGED, STATUS_MAX_ITER, STATUS_NONFINITE, STATUS_RADIUS_COLLAPSE = 0, 1, 2, 3


# ----------------------------------------------------------------------------- geometry
def patch_rects(scene):
    """Per source: list of (image index, x0, x1, y0, y1) inclusive pixel rectangles.

    The patch is the (2R+1)^2 window centred on the rounded pixel position of the
    catalog location, in every image whose pixel grid contains that centre, clipped to
    the image bounds."""
    out = []
    for s in range(scene.n_sources):
        lst = []
        for n, im in enumerate(scene.images):
            p = im.wcs[:4].reshape(2, 2) @ scene.u0[s] + im.wcs[4:]
            cx, cy = math.floor(p[0] + 0.5), math.floor(p[1] + 0.5)
            if not (0 <= cx <= im.W - 1 and 0 <= cy <= im.H - 1):
                continue
            R = int(scene.radius[s])
            lst.append((n, max(cx - R, 0), min(cx + R, im.W - 1), max(cy - R, 0), min(cy + R, im.H - 1)))
        out.append(lst)
    return out


def neighbour_lists(scene, rects):
    """nbr[s][n] = sources other than s whose patch in image n overlaps s's patch in image n."""
    by_image = {}
    for s, lst in enumerate(rects):
        for (n, x0, x1, y0, y1) in lst:
            by_image.setdefault(n, []).append((s, x0, x1, y0, y1))
    nbr = []
    for s, lst in enumerate(rects):
        d = {}
        for (n, x0, x1, y0, y1) in lst:
            d[n] = [t for (t, a0, a1, b0, b1) in by_image[n]
                    if t != s and a0 <= x1 and x0 <= a1 and b0 <= y1 and y0 <= b1]
        nbr.append(d)
    return nbr


def psf_at(im, x, y):
    """PSF components of image `im` evaluated at pixel position (x, y) (weights, means, covariances)."""
    xh = 2.0 * x / (im.W - 1) - 1.0
    yh = 2.0 * y / (im.H - 1) - 1.0
    basis = torch.tensor([1.0, xh, yh, xh * xh, xh * yh, yh * yh])
    par = torch.as_tensor(im.psf) @ basis
    w = torch.softmax(par[:, 0], 0)
    sx, sy, rho = torch.exp(par[:, 3]), torch.exp(par[:, 4]), torch.tanh(par[:, 5])
    return w, par[:, 1:3], torch.stack([sx * sx, rho * sx * sy, sy * sy], -1)   # cov as (s00, s01, s11)


# ----------------------------------------------------------------------------- model pieces
def bivariate_normal(dx, dy, s00, s01, s11):
    """Density of N(0, [[s00, s01], [s01, s11]]) at (dx, dy)."""
    det = s00 * s11 - s01 * s01
    q = (s11 * dx * dx - 2.0 * s01 * dx * dy + s00 * dy * dy) / det
    return torch.exp(-0.5 * q) / (2.0 * math.pi * torch.sqrt(det))


def galaxy_cov_world(theta):
    """Sigma_g = scale^2 R(angle) diag(1, axis^2) R(angle)^T, as (s00, s01, s11)."""
    e_axis = torch.sigmoid(theta[I_AXIS])
    ang = theta[I_ANGLE]
    scale2 = torch.exp(2.0 * theta[I_SCALE])
    c, s = torch.cos(ang), torch.sin(ang)
    a2 = e_axis * e_axis
    return scale2 * (c * c + a2 * s * s), scale2 * (1.0 - a2) * c * s, scale2 * (s * s + a2 * c * c)


def profiles(theta, im, px, py, psf, mix):
    """Star and galaxy unit-flux profiles f_0, f_1 at pixel centres (px, py)."""
    A = torch.as_tensor(im.wcs[:4]).reshape(2, 2)
    o = torch.as_tensor(im.wcs[4:])
    pos = A @ theta[I_U] + o
    w, means, cov = psf
    dx = px[:, None] - pos[0] - means[None, :, 0]
    dy = py[:, None] - pos[1] - means[None, :, 1]
    f_star = (w[None, :] * bivariate_normal(dx, dy, cov[:, 0], cov[:, 1], cov[:, 2])).sum(1)

    g00, g01, g11 = galaxy_cov_world(theta)
    # A Sigma_g A^T
    p00 = A[0, 0] * (A[0, 0] * g00 + A[0, 1] * g01) + A[0, 1] * (A[0, 0] * g01 + A[0, 1] * g11)
    p01 = A[1, 0] * (A[0, 0] * g00 + A[0, 1] * g01) + A[1, 1] * (A[0, 0] * g01 + A[0, 1] * g11)
    p11 = A[1, 0] * (A[1, 0] * g00 + A[1, 1] * g01) + A[1, 1] * (A[1, 0] * g01 + A[1, 1] * g11)
    e_dev = torch.sigmoid(theta[I_DEV])
    exp_nu, exp_tau, dev_nu, dev_tau = mix
    nu = torch.cat([(1.0 - e_dev) * exp_nu, e_dev * dev_nu])
    tau = torch.cat([exp_tau, dev_tau])
    # component (k, j): weight w_k nu_j, covariance tau_j A Sigma_g A^T + S_k
    s00 = tau[None, :] * p00 + cov[:, 0, None]
    s01 = tau[None, :] * p01 + cov[:, 1, None]
    s11 = tau[None, :] * p11 + cov[:, 2, None]
    dens = bivariate_normal(dx[:, :, None], dy[:, :, None], s00[None], s01[None], s11[None])
    f_gal = (w[None, :, None] * nu[None, None, :] * dens).sum((1, 2))
    return f_star, f_gal


def brightness_moments(theta, band):
    """E[l_b | type] and E[l_b^2 | type] for a lognormal flux: log l_b ~ N(m, v)."""
    mix = COLOR_MIX[band]
    L1, L2 = [], []
    for i in range(2):
        m = theta[I_R1[i]] + (mix * theta[I_C1[i]]).sum()
        v = torch.exp(theta[I_RHO[i]]) + (mix * mix * torch.exp(theta[I_GAM[i]])).sum()
        L1.append(torch.exp(m + 0.5 * v))
        L2.append(torch.exp(2.0 * m + 2.0 * v))
    return L1, L2


def source_moments(theta, im, px, py, psf, mix):
    """E[G] and E[G^2] of one source's (band-b) photon density at the pixels (per nanomaggy)."""
    f0, f1 = profiles(theta, im, px, py, psf, mix)
    L1, L2 = brightness_moments(theta, im.band)
    a1 = torch.sigmoid(theta[I_GAL])
    a0 = 1.0 - a1
    EG = a0 * L1[0] * f0 + a1 * L1[1] * f1
    EG2 = a0 * L2[0] * f0 * f0 + a1 * L2[1] * f1 * f1
    return EG, EG2


def kl_normal(m, v, mu, s2):
    """KL( N(m, v) || N(mu, s2) )."""
    return 0.5 * (torch.log(s2 / v) + (v + (m - mu) ** 2) / s2 - 1.0)


def kl_source(theta, priors):
    """KL(q(a) || p(a)) + sum_i q(a=i) [KL(q(r|i)||p(r)) + KL(q(c|i)||p(c))]."""
    phi, mu_r, var_r, mu_c, var_c = [torch.as_tensor(float(p)) for p in priors]
    alpha = theta[I_GAL]
    la1, la0 = torch.nn.functional.logsigmoid(alpha), torch.nn.functional.logsigmoid(-alpha)
    a1, a0 = torch.exp(la1), torch.exp(la0)
    kl = a1 * (la1 - torch.log(phi)) + a0 * (la0 - torch.log1p(-phi))
    for i, ai in enumerate((a0, a1)):
        k = kl_normal(theta[I_R1[i]], torch.exp(theta[I_RHO[i]]), mu_r, var_r)
        k = k + kl_normal(theta[I_C1[i]], torch.exp(theta[I_GAM[i]]), mu_c, var_c).sum()
        kl = kl + ai * k
    return kl


def pixel_term(x, E, V, lgx):
    """E_q[log Poisson(x | F)] with the second-order delta method for E_q[log F]."""
    return x * (torch.log(E) - V / (2.0 * E * E)) - E - lgx


# ----------------------------------------------------------------------------- per-source objective
class Oracle:
    """Per-source ELBO / gradient / Hessian and trust-region Newton for one scene."""

    def __init__(self, scene):
        self.scene = scene
        self.rects = patch_rects(scene)
        self.nbr = neighbour_lists(scene, self.rects)
        self.mix = tuple(torch.as_tensor(a) for a in (scene.exp_nu, scene.exp_tau, scene.dev_nu, scene.dev_tau))
        self.priors = scene.priors
        self._psf = {}

    def psf_for(self, s, n):
        key = (s, n)
        if key not in self._psf:
            im = self.scene.images[n]
            p = im.wcs[:4].reshape(2, 2) @ self.scene.u0[s] + im.wcs[4:]
            self._psf[key] = psf_at(im, float(p[0]), float(p[1]))
        return self._psf[key]

    def n_pixels(self, s):
        return sum((x1 - x0 + 1) * (y1 - y0 + 1) for (_, x0, x1, y0, y1) in self.rects[s])

    def _patch_data(self, s, nbr_theta):
        """Pixels, coordinates and fixed neighbour background of each of s's patches."""
        data = []
        for (n, x0, x1, y0, y1) in self.rects[s]:
            im = self.scene.images[n]
            ys, xs = torch.meshgrid(torch.arange(y0, y1 + 1, dtype=torch.float64),
                                    torch.arange(x0, x1 + 1, dtype=torch.float64), indexing="ij")
            px, py = xs.reshape(-1), ys.reshape(-1)
            x = torch.as_tensor(im.pixels[y0:y1 + 1, x0:x1 + 1].astype(np.float64)).reshape(-1)
            bE = torch.zeros_like(px)
            bV = torch.zeros_like(px)
            with torch.no_grad():
                for t in self.nbr[s][n]:
                    th = torch.as_tensor(nbr_theta[t])
                    EG, EG2 = source_moments(th, im, px, py, self.psf_for(t, n), self.mix)
                    bE += EG
                    bV += EG2 - EG * EG
            data.append((im, px, py, x, torch.lgamma(x + 1.0), bE, bV, self.psf_for(s, n)))
        return data

    def elbo_fn(self, s, nbr_theta):
        """Returns theta_s -> ELBO_s (a pure function, for value and autodiff)."""
        data = self._patch_data(s, nbr_theta)
        priors = self.priors
        mix = self.mix

        def f(theta):
            total = -kl_source(theta, priors)
            for (im, px, py, x, lgx, bE, bV, psf) in data:
                EG, EG2 = source_moments(theta, im, px, py, psf, mix)
                E = im.sky + im.iota * (bE + EG)
                V = im.iota ** 2 * (bV + EG2 - EG * EG)
                total = total + pixel_term(x, E, V, lgx).sum()
            return total
        return f

    def elbo(self, s, theta, nbr_theta):
        with torch.no_grad():
            return float(self.elbo_fn(s, nbr_theta)(torch.as_tensor(theta, dtype=torch.float64)))

    def elbo_grad_hess(self, s, theta, nbr_theta):
        """(L, dL/dtheta [27], d2L/dtheta2 [27,27]) at theta, exact derivatives in float64."""
        f = self.elbo_fn(s, nbr_theta)
        th = torch.as_tensor(theta, dtype=torch.float64).clone()
        g = torch.func.grad(f)(th)
        H = torch.func.hessian(f)(th)
        with torch.no_grad():
            val = f(th)
        return float(val), g.numpy(), H.numpy()

    def newton(self, s, theta0, nbr_theta, **opts):
        f = self.elbo_fn(s, nbr_theta)

        def value(th):
            with torch.no_grad():
                return float(f(torch.as_tensor(th)))

        def vgh(th):
            t = torch.as_tensor(th).clone()
            return value(th), torch.func.grad(f)(t).numpy(), torch.func.hessian(f)(t).numpy()

        return trust_region_newton(value, vgh, np.asarray(theta0, np.float64), **opts)


# ----------------------------------------------------------------------------- trust-region Newton
def tr_subproblem(g, B, delta):
    """argmin_p g.p + p.B.p/2 subject to ||p|| <= delta (More-Sorensen, eigenvalue form).

    Returns (p, predicted reduction -(g.p + p.B.p/2), hard_case flag)."""
    lam, Q = np.linalg.eigh(B)
    gam = Q.T @ g
    lmin = lam[0]
    gnorm = np.linalg.norm(g)

    def step(l):
        return -(Q @ (gam / (lam + l)))

    if lmin > 0:
        p = step(0.0)
        if np.linalg.norm(p) <= delta:
            return p, -(g @ p + 0.5 * p @ B @ p), False
    # ||p(l)|| = delta for some l > max(0, -lmin), unless the hard case applies.
    lo = max(0.0, -lmin)
    scale = max(1.0, np.abs(lam).max())
    small = np.abs(lam - lmin) <= 1e-12 * scale
    if np.all(np.abs(gam[small]) <= 1e-12 * max(gnorm, 1e-300)):
        # hard case candidate: the step with the singular directions removed
        keep = ~small
        p_hat = -(Q[:, keep] @ (gam[keep] / (lam[keep] - lmin))) if keep.any() else np.zeros_like(g)
        if np.linalg.norm(p_hat) <= delta:
            tau = math.sqrt(max(delta * delta - p_hat @ p_hat, 0.0))
            p = p_hat + tau * Q[:, 0]
            return p, -(g @ p + 0.5 * p @ B @ p), True
    hi = lo + gnorm / delta + 1.0
    while np.linalg.norm(gam / (lam + hi)) > delta:
        hi = 2.0 * hi + 1.0
    # safeguarded Newton on phi(l) = 1/||p(l)|| - 1/delta, which is increasing and concave on (lo, inf)
    l = hi
    for _ in range(200):
        d = lam + l
        pn = math.sqrt(np.sum((gam / d) ** 2))
        qn2 = np.sum(gam * gam / d ** 3)
        phi = 1.0 / pn - 1.0 / delta
        if abs(pn - delta) <= 1e-12 * delta:
            break
        if phi > 0:
            hi = l
        else:
            lo = l
        ln = l - phi / (qn2 / pn ** 3)          # phi'(l) = ||q||^2/||p||^3 with q = B_l^{-1/2} p
        if not (lo < ln < hi):
            ln = 0.5 * (lo + hi)
        if ln == l:
            break
        l = ln
    p = step(l)
    pn = np.linalg.norm(p)
    if pn > delta:
        # next to the pole lambda = -lambda_min the root is resolved only to ~1e-8; the subproblem
        # constrains |p| <= delta, so return the feasible point on the boundary
        p = p * (delta / pn)
    return p, -(g @ p + 0.5 * p @ B @ p), False


def trust_region_newton(value, vgh, theta0, max_iter=50, delta0=1.0, delta_max=1e4, eta=0.1,
                        ftol=1e-8, gtol=1e-10, delta_min=1e-12):
    """Maximise the ELBO by minimising f = -L with a trust region (Nocedal & Wright Alg. 4.1).

    Stops when max |grad| <= gtol, when an interior (full Newton) step predicts a decrease
    <= ftol |f|, when an accepted step changes f by <= ftol |f|, when a rejected step had
    predicted a decrease <= ftol |f| (the radius only shrinks after a rejection, so the model
    promises no more than the tolerance from here: the evaluation's rounding floor has been
    reached), when the radius falls below delta_min, or after max_iter subproblem solves.
    Returns dict(theta, elbo, iters, status)."""
    th = theta0.copy()
    L, gL, HL = vgh(th)
    f, g, B = -L, -gL, -HL
    delta = delta0
    status = STATUS_MAX_ITER
    it = 0
    while it < max_iter:
        if not (np.isfinite(f) and np.all(np.isfinite(g)) and np.all(np.isfinite(B))):
            status = STATUS_NONFINITE
            break
        if np.abs(g).max() <= gtol:
            status = STATUS_CONVERGED
            break
        it += 1
        p, pred, _ = tr_subproblem(g, B, delta)
        pnorm = np.linalg.norm(p)
        if pnorm < (1.0 - 1e-9) * delta and pred <= ftol * abs(f):
            # Newton decrement: the full Newton step promises less than ftol |f|
            status = STATUS_CONVERGED
            break
        f_new = -value(th + p)
        rho = (f - f_new) / pred if pred > 0 else -1.0
        if not np.isfinite(f_new):
            rho = -1.0
        if rho <= eta and pred <= ftol * abs(f):
            status = STATUS_CONVERGED
            break
        if rho < 0.25:
            delta = 0.25 * delta
        elif rho > 0.75 and pnorm >= (1.0 - 1e-9) * delta:
            delta = min(2.0 * delta, delta_max)
        if rho > eta:
            done = abs(f - f_new) <= ftol * abs(f_new)
            th = th + p
            L, gL, HL = vgh(th)
            f, g, B = -L, -gL, -HL
            if done:
                status = STATUS_CONVERGED
                break
        if delta < delta_min:
            status = STATUS_RADIUS_COLLAPSE
            break
    return dict(theta=th, elbo=-f, iters=it, status=status)

"""Seeded synthetic astronomical scenes: the common input of the CUDA path and the oracle.

The paper samples images from its own generative model for testing (Sec. "The Celeste
Model": Poisson pixels whose rate is a deterministic function of the catalog and the
image metadata).  This module draws such scenes: a true catalog, images with metadata
Lambda_n (PSF mixture, sky level, calibration, pixel<->world map), Poisson pixel counts,
and a perturbed "previous survey" catalog from which the variational parameters start.

It is an input generator only.  It holds none of the inference arithmetic: the truth is
rendered with point-mass brightness (no variational moments, no likelihood, no
derivatives), and nothing here is imported by the kernels.

Conventions shared through the data layout
  * pixel (row i, col j) has its centre at pixel coordinates (x, y) = (j, i);
  * world -> pixel map of image n: p = A_n u + o_n with wcs = [A00, A01, A10, A11, o0, o1];
  * PSF of image n: 3 components, each with 6 parameters
      [weight logit, mean_x, mean_y, log sigma_x, log sigma_y, atanh rho]
    given as quadratic polynomials in (xh, yh) = (2x/(W-1)-1, 2y/(H-1)-1) with
    coefficients for [1, xh, yh, xh^2, xh*yh, yh^2]; weights are the softmax of the logits;
  * bands u,g,r,i,z = 0..4, reference band r (index 2);
  * variational parameter vector (27 free parameters per source):
      0,1   u (world position)         2 logit e_dev   3 logit e_axis   4 e_angle
      5     log e_scale                6 logit P(galaxy)
      7,8   star: mean / log variance of log reference-band flux
      9,10  galaxy: same
      11-14 star colour means          15-18 star colour log variances
      19-22 galaxy colour means        23-26 galaxy colour log variances
"""
from dataclasses import dataclass, field

import numpy as np

from . import mixtures

N_PARAMS = 27
N_BANDS = 5
REF_BAND = 2
# Colour c_j = log(flux_{j+1} / flux_j); log flux_b = log flux_r + COLOR_MIX[b] . c
COLOR_MIX = np.array([[-1, -1, 0, 0], [0, -1, 0, 0], [0, 0, 0, 0], [0, 0, 1, 0], [0, 0, 1, 1]], dtype=np.float64)


@dataclass
class Image:
    pixels: np.ndarray      # float32 [H, W] photon counts
    band: int
    sky: float              # counts / pixel
    iota: float             # counts / nanomaggy
    wcs: np.ndarray         # float64 [6]
    psf: np.ndarray         # float64 [3, 6, 6] (component, parameter, polynomial coefficient)

    @property
    def H(self):
        return self.pixels.shape[0]

    @property
    def W(self):
        return self.pixels.shape[1]


@dataclass
class Scene:
    images: list
    u0: np.ndarray          # float64 [S, 2] catalog (initial) world positions: patch centres, PSF evaluation points
    radius: np.ndarray      # int32 [S] patch half-width in pixels
    theta0: np.ndarray      # float64 [S, 27] initial variational parameters
    priors: np.ndarray      # float64 [5]: Phi, mean log r, var log r, colour mean, colour var
    exp_nu: np.ndarray = field(default_factory=lambda: mixtures.EXP_NU.copy())
    exp_tau: np.ndarray = field(default_factory=lambda: mixtures.EXP_TAU.copy())
    dev_nu: np.ndarray = field(default_factory=lambda: mixtures.DEV_NU.copy())
    dev_tau: np.ndarray = field(default_factory=lambda: mixtures.DEV_TAU.copy())
    truth: dict = field(default_factory=dict)
    name: str = ""

    @property
    def n_sources(self):
        return self.u0.shape[0]


DEFAULT_PRIORS = np.array([0.5, 2.0, 1.0, 0.0, 0.25])


# --------------------------------------------------------------------------- truth rendering
def _psf_at(img_psf, x, y, H, W):
    """Evaluate the polynomial PSF at pixel position (x, y): (weights[3], means[3,2], covs[3,2,2])."""
    xh = 2.0 * x / (W - 1) - 1.0
    yh = 2.0 * y / (H - 1) - 1.0
    basis = np.array([1.0, xh, yh, xh * xh, xh * yh, yh * yh])
    par = img_psf @ basis                       # [3, 6]
    w = np.exp(par[:, 0] - par[:, 0].max())
    w /= w.sum()
    means = par[:, 1:3]
    sx, sy, rho = np.exp(par[:, 3]), np.exp(par[:, 4]), np.tanh(par[:, 5])
    covs = np.stack([np.stack([sx * sx, rho * sx * sy], -1), np.stack([rho * sx * sy, sy * sy], -1)], -2)
    return w, means, covs


def _render_truth(img, pos_pix, is_gal, shape, flux, win):
    """Rate added by one true source (point-mass brightness) over a square window of half-width win."""
    H, W = img.H, img.W
    cx, cy = int(round(pos_pix[0])), int(round(pos_pix[1]))
    x0, x1 = max(cx - win, 0), min(cx + win, W - 1)
    y0, y1 = max(cy - win, 0), min(cy + win, H - 1)
    if x0 > x1 or y0 > y1:
        return None
    ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1].astype(np.float64)
    w, means, covs = _psf_at(img.psf, pos_pix[0], pos_pix[1], H, W)
    A = img.wcs[:4].reshape(2, 2)
    if not is_gal:
        wts, mus, cvs = w, means, covs
    else:
        e_dev, e_axis, e_angle, e_scale = shape
        c, s = np.cos(e_angle), np.sin(e_angle)
        R = np.array([[c, -s], [s, c]])
        sig_p = A @ (e_scale ** 2 * R @ np.diag([1.0, e_axis ** 2]) @ R.T) @ A.T
        nu = np.concatenate([(1 - e_dev) * mixtures.EXP_NU, e_dev * mixtures.DEV_NU])
        tau = np.concatenate([mixtures.EXP_TAU, mixtures.DEV_TAU])
        wts = (w[:, None] * nu[None, :]).reshape(-1)
        mus = np.repeat(means, len(nu), axis=0)
        cvs = (tau[None, :, None, None] * sig_p[None, None] + covs[:, None]).reshape(-1, 2, 2)
    det = cvs[:, 0, 0] * cvs[:, 1, 1] - cvs[:, 0, 1] ** 2
    dx = xs[..., None] - pos_pix[0] - mus[:, 0]
    dy = ys[..., None] - pos_pix[1] - mus[:, 1]
    q = (cvs[:, 1, 1] * dx * dx - 2 * cvs[:, 0, 1] * dx * dy + cvs[:, 0, 0] * dy * dy) / det
    prof = (np.exp(-0.5 * q) * (wts / (2 * np.pi * np.sqrt(det)))).sum(-1)
    return (slice(y0, y1 + 1), slice(x0, x1 + 1)), img.iota * flux * prof


def _render_window(img_list, pos_list, is_gal, e_scale, cap=64):
    """Half-width covering 4 sigma of the widest truth component of a source."""
    v = 0.0
    for img, pp in zip(img_list, pos_list):
        _, _, covs = _psf_at(img.psf, pp[0], pp[1], img.H, img.W)
        v = max(v, float(covs[:, [0, 1], [0, 1]].max()))
    if is_gal:
        v += float(mixtures.DEV_TAU.max()) * e_scale ** 2
    return int(min(np.ceil(4.0 * np.sqrt(v)), cap))


def _band_fluxes(log_r, colors):
    return np.exp(log_r + COLOR_MIX @ colors)


def _patch_radius(img_list, pos_pix_list, is_gal, e_scale, log_r, colors, rmin, rmax):
    """Patch half-width: radius where the expected profile falls below half the sky noise."""
    fl = _band_fluxes(log_r, colors)
    best = 0.0
    for img, pp in zip(img_list, pos_pix_list):
        w, means, covs = _psf_at(img.psf, pp[0], pp[1], img.H, img.W)
        s2 = float((w * 0.5 * (covs[:, 0, 0] + covs[:, 1, 1])).sum())
        if is_gal:
            s2 += e_scale ** 2
        counts = img.iota * fl[img.band]
        arg = counts / (2 * np.pi * s2 * 0.5 * np.sqrt(img.sky))
        if arg > 1.0:
            best = max(best, np.sqrt(s2 * 2.0 * np.log(arg)))
    return int(np.clip(np.ceil(best), rmin, rmax))


def _make_psf(rng, smooth):
    psf = np.zeros((3, 6, 6))
    w = rng.dirichlet([3.0, 3.0, 3.0])
    psf[:, 0, 0] = np.log(w)
    psf[:, 3, 0] = np.log(rng.uniform(1.0, 3.0, 3)) if not smooth else np.log(rng.uniform(1.4, 2.1, 3))
    psf[:, 4, 0] = np.log(rng.uniform(1.0, 3.0, 3)) if not smooth else np.log(rng.uniform(1.4, 2.1, 3))
    psf[:, 5, 0] = np.arctanh(rng.uniform(-0.3, 0.3, 3))
    if smooth:
        psf[:, 1:3, 0] = rng.normal(0.0, 0.1, (3, 2))
        psf[:, 0, 1:] = rng.uniform(-0.1, 0.1, (3, 5))
        psf[:, 1:3, 1:] = rng.uniform(-0.05, 0.05, (3, 2, 5))
        psf[:, 3:5, 1:] = rng.uniform(-0.06, 0.06, (3, 2, 5))
        psf[:, 5, 1:] = rng.uniform(-0.05, 0.05, (3, 5))
    return psf


def _logit(p):
    return np.log(p) - np.log1p(-p)


def _initial_theta(rng, u, is_gal, shape, log_r, colors, jitter_pos):
    """Previous-survey estimate: the truth perturbed (stands in for an existing catalog)."""
    th = np.zeros(N_PARAMS)
    th[0:2] = u + rng.uniform(-jitter_pos, jitter_pos, 2)
    if is_gal:
        e_dev, e_axis, e_angle, e_scale = shape
        th[2] = _logit(np.clip(e_dev + rng.normal(0, 0.1), 0.05, 0.95))
        th[3] = _logit(np.clip(e_axis + rng.normal(0, 0.05), 0.1, 0.95))
        th[4] = e_angle + rng.normal(0, 0.1)
        th[5] = np.log(e_scale) + rng.normal(0, 0.1)
    else:
        th[2], th[3], th[4], th[5] = 0.0, _logit(0.7), rng.uniform(0, np.pi), np.log(1.0)
    th[6] = 0.0
    lr = log_r + rng.normal(0, 0.2)
    col = colors + rng.normal(0, 0.1, 4)
    th[7], th[8], th[9], th[10] = lr, np.log(0.01), lr, np.log(0.01)
    th[11:15], th[15:19], th[19:23], th[23:27] = col, np.log(0.01), col, np.log(0.01)
    return th


def _draw_truth(rng, n, p_gal, priors):
    is_gal = rng.random(n) < p_gal
    log_r = rng.normal(priors[1], np.sqrt(priors[2]), n)
    colors = rng.normal(priors[3], np.sqrt(priors[4]), (n, 4))
    shape = np.stack([rng.uniform(0, 1, n), rng.uniform(0.3, 1, n), rng.uniform(0, np.pi, n),
                      rng.uniform(0.5, 4.0, n)], -1)
    return is_gal, log_r, colors, shape


def _assemble(rng, images, u_true, is_gal, log_r, colors, shape, radius_rule, noise, jitter_pos, render_win):
    S = len(u_true)
    rates = [np.full((im.H, im.W), im.sky, dtype=np.float64) for im in images]
    theta0 = np.zeros((S, N_PARAMS))
    radius = np.zeros(S, dtype=np.int32)
    for s in range(S):
        fl = _band_fluxes(log_r[s], colors[s])
        pos_list = [im.wcs[:4].reshape(2, 2) @ u_true[s] + im.wcs[4:] for im in images]
        win = render_win if render_win else _render_window(images, pos_list, bool(is_gal[s]), shape[s, 3])
        for n, im in enumerate(images):
            pp = pos_list[n]
            out = _render_truth(im, pp, bool(is_gal[s]), shape[s], fl[im.band], win)
            if out is not None:
                sl, add = out
                rates[n][sl] += add
        theta0[s] = _initial_theta(rng, u_true[s], bool(is_gal[s]), shape[s], log_r[s], colors[s], jitter_pos)
        radius[s] = radius_rule(s, pos_list)
    for im, rate in zip(images, rates):
        im.pixels = (rng.poisson(rate) if noise else rate).astype(np.float32)
    truth = dict(u=u_true, is_gal=is_gal, log_r=log_r, colors=colors, shape=shape)
    return theta0, radius, truth


def _blank_image(H, W, band, sky, iota, wcs, psf):
    return Image(np.zeros((H, W), np.float32), band, float(sky), float(iota), np.asarray(wcs, np.float64), psf)


# --------------------------------------------------------------------------- public scenes
def single_source(seed=1611, size=41, noise=True, is_gal=None, log_r=None, jitter_pos=0.5, priors=None):
    """One isolated source at a seeded sub-pixel position, 5 bands x 1 image of size x size pixels.

    PSF: 3 components per band, weights ~ Dirichlet(3,3,3), sigmas U(1,3) px, correlation U(-0.3,0.3);
    sky U(50,200) counts/px; calibration U(100,300) counts/nmgy; log flux ~ N(2,1); colours N(0, 0.5^2);
    galaxy fracDev U(0,1), axis U(0.3,1), angle U(0,pi), half-light radius U(0.5,4) px.
    The patch is the whole image (radius (size-1)/2).
    """
    rng = np.random.default_rng(seed)
    priors = DEFAULT_PRIORS.copy() if priors is None else np.asarray(priors, np.float64)
    g, lr, col, shp = _draw_truth(rng, 1, 0.5, priors)
    if is_gal is not None:
        g[:] = is_gal
    if log_r is not None:
        lr[:] = log_r
    c = (size - 1) / 2.0
    u = np.array([[c + rng.uniform(-0.5, 0.5), c + rng.uniform(-0.5, 0.5)]])
    images = []
    for b in range(N_BANDS):
        images.append(_blank_image(size, size, b, rng.uniform(50, 200), rng.uniform(100, 300),
                                   [1, 0, 0, 1, 0, 0], _make_psf(rng, smooth=False)))
    R = (size - 1) // 2
    theta0, radius, truth = _assemble(rng, images, u, g, lr, col, shp, lambda s, p: R, noise, jitter_pos, size)
    sc = Scene(images, theta0[:, 0:2].copy(), radius, theta0, priors, truth=truth, name=f"single_source_{size}")
    return sc


def field(seed=1611, W=2048, H=1489, n_sources=1000, p_gal=0.6, rmin=8, rmax=32, noise=True, priors=None):
    """A synthetic field: W x H pixels x 5 bands (one exposure per band with its own sub-pixel offset),
    sources placed uniformly, a PSF varying smoothly across the field (sigma within [1, 3] px),
    patch radius by brightness clamped to [rmin, rmax] so neighbouring patches overlap."""
    rng = np.random.default_rng(seed)
    priors = DEFAULT_PRIORS.copy() if priors is None else np.asarray(priors, np.float64)
    images = []
    for b in range(N_BANDS):
        off = rng.uniform(-0.5, 0.5, 2)
        images.append(_blank_image(H, W, b, rng.uniform(50, 200), rng.uniform(100, 300),
                                   [1, 0, 0, 1, off[0], off[1]], _make_psf(rng, smooth=True)))
    u = np.stack([rng.uniform(0, W - 1, n_sources), rng.uniform(0, H - 1, n_sources)], -1)
    g, lr, col, shp = _draw_truth(rng, n_sources, p_gal, priors)

    def rule(s, pos_list):
        return _patch_radius(images, pos_list, bool(g[s]), shp[s, 3], lr[s], col[s], rmin, rmax)

    theta0, radius, truth = _assemble(rng, images, u, g, lr, col, shp, rule, noise, 0.5, None)
    return Scene(images, theta0[:, 0:2].copy(), radius, theta0, priors, truth=truth, name=f"field_{W}x{H}_{n_sources}")


def tiny(seed=7, n_sources=3, n_images=3, H=26, W=30, radius=(6, 9), rotate=True, noise=True, priors=None):
    """A few overlapping sources in a few small images with rotated/scaled pixel maps, for tests."""
    rng = np.random.default_rng(seed)
    priors = DEFAULT_PRIORS.copy() if priors is None else np.asarray(priors, np.float64)
    images = []
    for n in range(n_images):
        if rotate:
            ang = rng.uniform(-0.3, 0.3)
            sc = rng.uniform(0.9, 1.1)
            A = sc * np.array([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]])
        else:
            A = np.eye(2)
        o = np.array([W / 2.0, H / 2.0]) - A @ np.array([W / 2.0, H / 2.0]) + rng.uniform(-1, 1, 2)
        images.append(_blank_image(H, W, int(rng.integers(0, N_BANDS)), rng.uniform(50, 200), rng.uniform(100, 300),
                                   [A[0, 0], A[0, 1], A[1, 0], A[1, 1], o[0], o[1]], _make_psf(rng, smooth=True)))
    u = np.stack([rng.uniform(0.3 * W, 0.7 * W, n_sources), rng.uniform(0.3 * H, 0.7 * H, n_sources)], -1)
    g, lr, col, shp = _draw_truth(rng, n_sources, 0.5, priors)
    lr += 1.0
    rads = rng.integers(radius[0], radius[1] + 1, n_sources).astype(np.int32)
    theta0, rr, truth = _assemble(rng, images, u, g, lr, col, shp, lambda s, p: int(rads[s]), noise, 0.5, 40)
    return Scene(images, theta0[:, 0:2].copy(), rr, theta0, priors, truth=truth, name=f"tiny_{seed}")

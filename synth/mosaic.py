"""Seeded synthetic survey mosaic: many overlapping single-band exposures, tens of thousands of
sources.

A grid of fields, each observed in a random subset of the five bands (one exposure per band with
its own small rotation, scale and offset of the pixel grid); neighbouring fields overlap, so a
source is seen in 1 to 12 exposures.  Patch radius 8-64 px by brightness.  The truth is rendered
exactly as in the other scenes of this package (point-mass brightness through the PSF-convolved
profile mixtures), but batched with torch so that 10^5 sources render in seconds on a GPU.

Input generation only: no variational moments, no likelihood, no derivatives.
"""
import math

import numpy as np
import torch

from . import COLOR_MIX, DEFAULT_PRIORS, N_BANDS, Image, Scene, _draw_truth, _initial_theta, _make_psf, mixtures

_NCOMP = 3 * (len(mixtures.EXP_NU) + len(mixtures.DEV_NU))


def _psf_params(psf, pos, H, W):
    """Vectorised PSF at pixel positions pos [P, 2]: weights [P,3], means [P,3,2], covs [P,3,2,2]."""
    xh = 2.0 * pos[:, 0] / (W - 1) - 1.0
    yh = 2.0 * pos[:, 1] / (H - 1) - 1.0
    basis = np.stack([np.ones_like(xh), xh, yh, xh * xh, xh * yh, yh * yh], -1)   # [P, 6]
    par = np.einsum("kqc,pc->pkq", psf, basis)                                     # [P, 3, 6]
    w = np.exp(par[..., 0] - par[..., 0].max(-1, keepdims=True))
    w /= w.sum(-1, keepdims=True)
    sx, sy, rho = np.exp(par[..., 3]), np.exp(par[..., 4]), np.tanh(par[..., 5])
    covs = np.stack([np.stack([sx * sx, rho * sx * sy], -1), np.stack([rho * sx * sy, sy * sy], -1)], -2)
    return w, par[..., 1:3], covs


def _components(img, pos, is_gal, shape):
    """Mixture of the true brightness of each (source, this image) pair: weights [P,K], means
    [P,K,2], covariances [P,K,2,2] in pixel units (K = 42; stars use the first 3)."""
    P = len(pos)
    w, means, covs = _psf_params(img.psf, pos, img.H, img.W)
    A = img.wcs[:4].reshape(2, 2)
    e_dev, e_axis, e_angle, e_scale = shape[:, 0], shape[:, 1], shape[:, 2], shape[:, 3]
    c, s = np.cos(e_angle), np.sin(e_angle)
    R = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)                 # [P, 2, 2]
    D = np.zeros((P, 2, 2))
    D[:, 0, 0] = 1.0
    D[:, 1, 1] = e_axis ** 2
    sig_w = (e_scale ** 2)[:, None, None] * (R @ D @ np.swapaxes(R, 1, 2))
    sig_p = A[None] @ sig_w @ A.T[None]                                              # [P, 2, 2]
    nu = np.concatenate([(1 - e_dev)[:, None] * mixtures.EXP_NU[None], e_dev[:, None] * mixtures.DEV_NU[None]], 1)
    tau = np.concatenate([mixtures.EXP_TAU, mixtures.DEV_TAU])                       # [14]
    gw = (w[:, :, None] * nu[:, None, :]).reshape(P, -1)                             # [P, 42]
    gm = np.repeat(means, len(tau), axis=1)                                          # [P, 42, 2]
    gc = (tau[None, None, :, None, None] * sig_p[:, None, None] + covs[:, :, None]).reshape(P, -1, 2, 2)
    wts = np.zeros((P, _NCOMP))
    mus = np.zeros((P, _NCOMP, 2))
    cvs = np.tile(np.eye(2), (P, _NCOMP, 1, 1))
    star = ~is_gal
    wts[star, :3], mus[star, :3], cvs[star, :3] = w[star], means[star], covs[star]
    wts[is_gal], mus[is_gal], cvs[is_gal] = gw[is_gal], gm[is_gal], gc[is_gal]
    return wts, mus, cvs


def _window(cvs, wts, cap=64):
    """Half-width covering 4 sigma of the widest component with weight."""
    v = np.where(wts > 0, np.maximum(cvs[..., 0, 0], cvs[..., 1, 1]), 0.0).max(-1)
    return np.minimum(np.ceil(4.0 * np.sqrt(v)), cap).astype(np.int64)


def render_image_rate(img, pos, is_gal, shape, flux, device, chunk_px=1 << 24, window=None):
    """Expected counts of image `img`: sky plus every listed source (positions pos [P,2] in this
    image's pixels, band fluxes flux [P]) over a window of 4 sigma of its widest component (capped
    at 64 px) or of half-width `window`.  Returns a float64 torch tensor [H, W] on `device`."""
    H, W = img.H, img.W
    rate = torch.full((H * W,), float(img.sky), dtype=torch.float64, device=device)
    if len(pos) == 0:
        return rate.view(H, W)
    wts, mus, cvs = _components(img, pos, is_gal, shape)
    win = _window(cvs, wts) if window is None else np.full(len(pos), int(window), np.int64)
    det = cvs[..., 0, 0] * cvs[..., 1, 1] - cvs[..., 0, 1] ** 2
    amp = img.iota * flux[:, None] * wts / (2 * np.pi * np.sqrt(det))               # [P, K]
    inv = np.stack([cvs[..., 1, 1] / det, -cvs[..., 0, 1] / det, cvs[..., 0, 0] / det], -1)   # [P, K, 3]
    cx = np.floor(pos[:, 0] + 0.5).astype(np.int64)
    cy = np.floor(pos[:, 1] + 0.5).astype(np.int64)
    order = np.argsort(win)
    i = 0
    while i < len(order):
        w = int(win[order[i]])
        side = 2 * w + 1
        n = max(1, min(len(order) - i, chunk_px // (side * side * _NCOMP)))
        j = i
        while j < len(order) and j - i < n and win[order[j]] <= w:
            j += 1
        idx = order[i:j]
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=device)
        off = torch.arange(-w, w + 1, device=device, dtype=torch.int64)
        xs = t(cx[idx])[:, None, None] + off[None, None, :]                                    # [B, 1, side]
        ys = t(cy[idx])[:, None, None] + off[None, :, None]                                    # [B, side, 1]
        dx = (xs.to(torch.float64) - t(pos[idx, 0])[:, None, None])[..., None] - t(mus[idx, :, 0])[:, None, None, :]
        dy = (ys.to(torch.float64) - t(pos[idx, 1])[:, None, None])[..., None] - t(mus[idx, :, 1])[:, None, None, :]
        iv = t(inv[idx])
        q = iv[:, None, None, :, 0] * dx * dx + 2 * iv[:, None, None, :, 1] * dx * dy + iv[:, None, None, :, 2] * dy * dy
        val = (torch.exp(-0.5 * q) * t(amp[idx])[:, None, None, :]).sum(-1)                  # [B, side, side]
        inside = (xs >= 0) & (xs < W) & (ys >= 0) & (ys < H)
        inside = inside & (off[None, None, :].abs() <= t(win[idx])[:, None, None]) & \
            (off[None, :, None].abs() <= t(win[idx])[:, None, None])
        flat = (ys * W + xs).expand(-1, side, side)
        rate.index_put_((flat[inside],), val[inside], accumulate=True)
        i = j
    return rate.view(H, W)


def _patch_radius_v(img, pos, is_gal, e_scale, counts, rmin, rmax):
    """Vectorised radius rule of the other scenes: where the expected profile falls below half the
    sky noise, for each source in this image."""
    w, _, covs = _psf_params(img.psf, pos, img.H, img.W)
    s2 = (w * 0.5 * (covs[..., 0, 0] + covs[..., 1, 1])).sum(-1) + np.where(is_gal, e_scale ** 2, 0.0)
    arg = counts / (2 * np.pi * s2 * 0.5 * np.sqrt(img.sky))
    r = np.where(arg > 1.0, np.sqrt(s2 * 2.0 * np.log(np.maximum(arg, 1.0))), 0.0)
    return r


def mosaic(seed=1611, fields_x=10, fields_y=10, n_sources=100_000, field_W=2048, field_H=1489, overlap=0.2,
           bands_per_field=(1, 3), p_gal=0.6, extended=0.02, rmin=8, rmax=64, radius_rule="brightness+4sigma",
           noise=True, priors=None, device=None):
    """A fields_x x fields_y grid of fields stepping by (1 - overlap) of the field size; each field
    observed in a random subset of 1-3 bands (one exposure each, its pixel grid rotated by up to
    0.02 rad, scaled by 0.98-1.02 and offset by a sub-pixel shift); sources uniform over the
    covered area; PSF varying smoothly across each exposure.  World coordinates are the pixel
    coordinates of an undistorted grid spanning the mosaic.

    Catalog as in the field scenes, plus a fraction `extended` of the galaxies with half-light
    radius U(4, 8) px.  Patch radius: the larger of the field scenes' brightness rule and 4 sigma of
    the source's widest true component, clamped to [rmin, rmax]; radius_rule="brightness" keeps the
    field scenes' rule alone (with bands_per_field=(5, 5), extended=0 and rmax=32 the exposures
    look like the field scenes')."""
    rng = np.random.default_rng(seed)
    priors = DEFAULT_PRIORS.copy() if priors is None else np.asarray(priors, np.float64)
    device = torch.device(device or ("cuda" if torch.cuda.is_available() else "cpu"))
    step_x, step_y = (1 - overlap) * field_W, (1 - overlap) * field_H
    extent = np.array([step_x * (fields_x - 1) + field_W, step_y * (fields_y - 1) + field_H])
    images = []
    for fy in range(fields_y):
        for fx in range(fields_x):
            nb = int(rng.integers(bands_per_field[0], bands_per_field[1] + 1))
            for b in sorted(rng.choice(N_BANDS, nb, replace=False)):
                ang, sc = rng.uniform(-0.02, 0.02), rng.uniform(0.98, 1.02)
                A = sc * np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
                corner = np.array([fx * step_x, fy * step_y])
                centre = corner + np.array([field_W, field_H]) / 2.0
                # pixel = A (u - centre) + image centre + sub-pixel shift
                o = np.array([field_W, field_H]) / 2.0 - A @ centre + rng.uniform(-0.5, 0.5, 2)
                images.append(Image(np.zeros((field_H, field_W), np.float32), int(b), float(rng.uniform(50, 200)),
                                    float(rng.uniform(100, 300)),
                                    np.array([A[0, 0], A[0, 1], A[1, 0], A[1, 1], o[0], o[1]]),
                                    _make_psf(rng, smooth=True)))
    # 50 px inside the mosaic's edge: the exposures' rotation and scale move their corners by < 45 px
    u = np.stack([rng.uniform(50, extent[0] - 51, n_sources), rng.uniform(50, extent[1] - 51, n_sources)], -1)
    g, lr, col, shp = _draw_truth(rng, n_sources, p_gal, priors)
    ext = g & (rng.random(n_sources) < extended)
    shp[ext, 3] = rng.uniform(4.0, 8.0, int(ext.sum()))
    fl = np.exp(lr[:, None] + col @ COLOR_MIX.T)                                     # [S, 5] band fluxes
    theta0 = np.stack([_initial_theta(rng, u[s], bool(g[s]), shp[s], lr[s], col[s], 0.5) for s in range(n_sources)])
    u_cat = theta0[:, 0:2]                  # catalog positions: the patch centres
    radius_f = np.zeros(n_sources)
    n_img = np.zeros(n_sources, np.int64)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(rng.integers(0, 2 ** 62)))
    for im in images:
        H, W = im.H, im.W
        A, o = im.wcs[:4].reshape(2, 2), im.wcs[4:]
        pos = u @ A.T + o
        margin = 2 * rmax
        near = (pos[:, 0] > -margin) & (pos[:, 0] < W - 1 + margin) & (pos[:, 1] > -margin) & (pos[:, 1] < H - 1 + margin)
        idx = np.nonzero(near)[0]
        rate = render_image_rate(im, pos[idx], g[idx], shp[idx], fl[idx, im.band], device)
        pix = torch.poisson(rate, generator=gen) if noise else rate
        im.pixels = pix.to(torch.float32).cpu().numpy()
        pos_cat = u_cat @ A.T + o
        cxy = np.floor(pos_cat + 0.5)
        sel = np.nonzero((cxy[:, 0] >= 0) & (cxy[:, 0] <= W - 1) & (cxy[:, 1] >= 0) & (cxy[:, 1] <= H - 1))[0]
        n_img[sel] += 1
        r = _patch_radius_v(im, pos[sel], g[sel], shp[sel, 3], im.iota * fl[sel, im.band], rmin, rmax)
        if radius_rule == "brightness":
            radius_f[sel] = np.maximum(radius_f[sel], r)
        else:
            wts, _, cvs = _components(im, pos[sel], g[sel], shp[sel])
            radius_f[sel] = np.maximum(radius_f[sel], np.maximum(r, _window(cvs, wts, cap=rmax)))
    radius = np.clip(np.ceil(radius_f), rmin, rmax).astype(np.int32)
    truth = dict(u=u, is_gal=g, log_r=lr, colors=col, shape=shp, n_images=n_img)
    return Scene(images, theta0[:, 0:2].copy(), radius, theta0, priors, truth=truth,
                 name=f"mosaic_{fields_x}x{fields_y}_{n_sources}")

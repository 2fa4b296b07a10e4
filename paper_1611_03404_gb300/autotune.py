"""Tile-size autotuner for the pixel kernels (argument marshalling and timing only).

A tile is the unit of work of one CTA of the pixel kernels: 128 x (pixels per thread) consecutive
pixels of one patch.  Larger tiles amortise the staging of the patch table over more pixels but
raise register pressure and the ragged remainder of each patch; which wins depends on the patch
size distribution of the workload.  The tuner builds the layout of a sample of the workload's
sources for each candidate tile size, times the ELBO + gradient + Hessian evaluation with CUDA
events and returns the fastest per pixel.
"""
import numpy as np
import torch

from .celeste import Problem


def _subset(scene, idx):
    sub = type(scene)(scene.images, scene.u0[idx], scene.radius[idx], scene.theta0[idx], scene.priors,
                      scene.exp_nu, scene.exp_tau, scene.dev_nu, scene.dev_tau, name=scene.name + "_sample")
    return sub


def tune_tile(scene, device="cuda", candidates=(128, 256, 512), sample=2000, reps=5, seed=0, device_pixels=None):
    """Returns (best tile_pixels, {tile: microseconds per 1000 pixels}) for `scene`, timed on a seeded
    sample of `sample` sources (all of them if fewer)."""
    S = scene.n_sources
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(S, min(S, sample), replace=False))
    sub = _subset(scene, idx)
    dev = torch.device(device)
    theta = torch.as_tensor(sub.theta0, device=dev).contiguous()
    out = {}
    for tile in candidates:
        prob = Problem(sub, device=dev, tile_pixels=tile, device_pixels=device_pixels)
        prob.render_background(theta)
        for _ in range(2):
            prob.elbo_batch(theta)
        torch.cuda.synchronize(dev)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            prob.elbo_batch(theta)
        t1.record()
        torch.cuda.synchronize(dev)
        px = prob.counts()["pixels"]
        out[tile] = 1e3 * t0.elapsed_time(t1) / reps / max(px, 1) * 1e3
        prob.close()
    best = min(out, key=out.get)
    return best, out

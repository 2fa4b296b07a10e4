"""Autotuner for the pixel kernels (argument marshalling and timing only).

Two axes:
  * the tile: the unit of work of one CTA of the pixel kernels, 4 warps x (pixels per warp)
    consecutive pixels of one patch.  Larger tiles amortise the staging of the patch table over
    more pixels but raise register pressure and the ragged remainder of each patch; which wins
    depends on the patch size distribution of the workload.
  * the form of the Hessian's Jacobian cross-product (FP32 FMAs or one of the tensor-core forms);
    the tensor-core forms run with 32 pixels per warp.
The tuner builds the layout of a seeded sample of the workload's sources for each candidate,
times the ELBO + gradient + Hessian evaluation with CUDA events and returns the fastest per pixel.
Only forms that meet the gradient and Hessian precision bar are candidates by default: FP32 FMAs,
BF16 hi+mid+lo and TF32 big+small (BF16 hi+lo and plain TF32 do not).
"""
import numpy as np
import torch

from .celeste import HESS_BF16X6, HESS_FP32, HESS_TF32X3, Problem

PRECISE_MODES = (HESS_FP32, HESS_BF16X6, HESS_TF32X3)


def _subset(scene, idx):
    sub = type(scene)(scene.images, scene.u0[idx], scene.radius[idx], scene.theta0[idx], scene.priors,
                      scene.exp_nu, scene.exp_tau, scene.dev_nu, scene.dev_tau, name=scene.name + "_sample")
    return sub


def _time(sub, dev, tile, mode, theta, reps, device_pixels):
    prob = Problem(sub, device=dev, tile_pixels=tile, hessian_mode=mode, device_pixels=device_pixels)
    prob.render_background(theta)
    for _ in range(2):
        prob.elbo_batch(theta, check=False)
    prob.check()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        prob.elbo_batch(theta, check=False)
    t1.record()
    torch.cuda.synchronize(dev)
    px = prob.counts()["pixels"]
    prob.close()
    return 1e3 * t0.elapsed_time(t1) / reps / max(px, 1) * 1e3   # microseconds per 1000 pixels


def tune(scene, device="cuda", modes=None, tiles=None, sample=4000, reps=5, seed=0, device_pixels=None):
    """Returns ((tile_pixels, hessian_mode), {"tile/mode": microseconds per 1000 pixels}) for `scene`,
    timed on a seeded sample of `sample` sources.  modes: candidate Hessian forms (default: every form
    that meets the precision bar); tiles: candidate tile sizes for the FP32 form (the tensor-core
    forms use 128)."""
    modes = PRECISE_MODES if modes is None else tuple(modes)
    tiles = (128, 256, 512) if tiles is None else tuple(tiles)
    S = scene.n_sources
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(S, min(S, sample), replace=False))
    sub = _subset(scene, idx)
    dev = torch.device(device)
    theta = torch.as_tensor(sub.theta0, device=dev).contiguous()
    out = {}
    for mode in modes:
        for tile in (tiles if mode == HESS_FP32 else (128,)):
            out[(tile, mode)] = _time(sub, dev, tile, mode, theta, reps, device_pixels)
    best = min(out, key=out.get)
    return best, {f"{t}/{m}": v for (t, m), v in out.items()}


def tune_tile(scene, device="cuda", candidates=(128, 256, 512), sample=2000, reps=5, seed=0, device_pixels=None):
    """The tile size alone for the FP32 form: (best tile_pixels, {tile: microseconds per 1000 pixels})."""
    (tile, _), rep = tune(scene, device, modes=(HESS_FP32,), tiles=candidates, sample=sample, reps=reps, seed=seed,
                          device_pixels=device_pixels)
    return tile, {int(k.split("/")[0]): v for k, v in rep.items()}

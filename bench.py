#!/usr/bin/env python
"""Benchmark: light sources per second to convergence, batched trust-region Newton on one GPU.

Default workload: a seeded 10 x 10 mosaic of overlapping 2048 x 1489 fields, 100,000 sources seen in
1-12 single-band exposures each, patch radius 8-64 px.  One step = one block-coordinate pass over
every source: render the neighbours' fixed background, run the learned warm-start network on every
source's patch, then run trust-region Newton (ELBO + exact gradient + dense Hessian per iteration,
in the Hessian form and tile size the autotuner picks among those that meet the precision bar:
FP32 FMAs or a split tensor-core form) on every source from that start until all have stopped.
The network is trained before the timed region on pairs from two freshly seeded mosaics.  The plain
form (Newton from the catalog, Hessian on FP32 FMAs, no network) is timed on the same workload at the
same ELBO tolerance and reported as "plain_fp32".  `--workload field` runs one 2048 x 1489 x 5-band
field of 1000 sources instead.  Under torchrun every rank solves its own independently seeded
workload (weak scaling, no collective on the data path); the timing is the max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the float64 CPU oracle (the plain, slow definition of the same objective
and optimiser) on the host cores, on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sources/s to convergence at fixed ELBO tol; ELBO+grad+Hess pixel-evals/s"
FP32_LANES_PER_SM = 128      # FP32 FMA lanes per SM (4 sub-partitions x 32)
MUFU_PER_SM_CLK = 16         # special-function unit results per SM per clock (4 sub-partitions x 4)
FP64_PER_SM_CLK = 2          # FP64 FMAs per SM per clock (one warp instruction per 64 cycles per sub-partition)

# Algorithmic float32 operations per pixel evaluation (FMA = 2), counted from the formulas the
# kernels evaluate:
#   per PSF component (3): offsets and squares 6; star component 30
#   per galaxy component (42): quadratic form 5, weighted exponential 2, precision vector 6,
#     first shape terms 18, cross vectors 18, scaled weights 3, value/first-derivative sums 9,
#     second-derivative sums 60, shape second terms 36  -> 157
#   per-pixel tail: family mixing 75, rate moments 18, pixel term and its derivatives 44,
#     Jacobian rows 42, curvature-scaled rows 44, scalars 6, first-order sums 38,
#     second-order sums 150, cross-product sums 122, summation over pixels 108  -> 647
FLOPS_FULL_PER_PIXEL = 3 * (6 + 30) + 42 * 157 + 647
#   value only: per PSF component offsets 6 + 15 components x (quadratic form 5, exponential 2, sum 1),
#   tail 25
FLOPS_VALUE_PER_PIXEL = 3 * (6 + 15 * 8) + 25
# special-function operations per full pixel evaluation: 45 exp2, 2 reciprocals/divides, 1 log1p
MUFU_FULL_PER_PIXEL = 48
# float64 work of one trust-region subproblem of dimension n = 27, counted as one tridiagonal
# (Householder) reduction, 4/3 n^3: the algorithmic core of the subproblem (the Newton-step fast
# path does less, the multiplier search more)
FP64_FLOPS_PER_SUBPROBLEM = 4 * 27 ** 3 // 3
# bytes per pixel evaluation that the pixel kernel must move: the 16-byte pixel record read and the
# 8-byte source moments written (the 8224-byte patch table per patch comes on top)
BYTES_FULL_PER_PIXEL = 24
TABLE_BYTES = 8224


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mosaic", choices=["field", "mosaic"],
                    help="mosaic: 10x10 overlapping fields, 100,000 sources, 1-12 exposures each (the headline); "
                         "field: 2048x1489 px x 5 bands, --sources sources")
    ap.add_argument("--sources", type=int, default=1000, help="sources of the field workload")
    ap.add_argument("--mosaic-fields", type=int, default=10,
                    help="the mosaic's fields per side (1000 sources per field at the same density; 10 = the "
                         "headline's 100,000 sources; smaller mosaics for profiler captures)")
    ap.add_argument("--tile", type=int, default=0, help="pixels per tile; 0 = autotune")
    ap.add_argument("--no-warm-start", dest="warm_start", action="store_false",
                    help="time only the plain form (Newton from the catalog, FP32 FMA Hessian)")
    ap.add_argument("--ws-epochs", type=int, default=6)
    ap.add_argument("--hessian", default="auto", choices=["fp32", "tf32", "bf16x3", "bf16x6", "tf32x3", "auto"],
                    help="Jacobian cross-product of the Hessian in the headline form: FP32 FMAs or tensor cores "
                         "(TF32; BF16 hi+lo with three products; BF16 hi+mid+lo with six; TF32 big+small with three); "
                         "auto = the autotuner's choice among the forms that meet the precision bar")
    ap.add_argument("--plain-steps", type=int, default=5, help="timed steps of the plain form (at most --steps)")
    ap.add_argument("--seed", type=int, default=1611)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-seconds-single", type=float, default=8.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-reports", dest="reports", action="store_false",
                    help="skip the untimed reports (block-coordinate passes, joint objective)")
    ap.add_argument("--no-joint", dest="joint", action="store_false", help="skip the untimed joint-objective report")
    ap.add_argument("--profile-range", action="store_true",
                    help="open the CUDA profiler range (cudaProfilerStart/Stop) around the timed steps of the headline "
                         "form only, for ncu --profile-from-start off")
    return ap.parse_args(argv)


def workload_config(args):
    """The workload (identical for both arms; how it is solved is in `method`)."""
    if args.workload == "mosaic":
        f = args.mosaic_fields
        return {"workload": f"mosaic_{f}x{f}_fields_{1000 * f * f}src", "fields": [f, f], "field_px": [2048, 1489],
                "field_overlap": 0.2, "bands_per_field": "1-3", "exposures_per_source": "1-12",
                "sources_per_gpu": 1000 * f * f, "patch_radius": "8-64 (brightness, 4 sigma of the widest component)",
                "galaxy_fraction": 0.6, "elbo_tol": 1e-8, "max_iter": 50,
                "l2": "inputs larger than L2 (GBs of patch pixels) and a 256 MiB flush between timed steps",
                "parallelism": "one independently seeded mosaic per GPU"}
    return {"workload": f"field_2048x1489x5_{args.sources}src", "image_px": [2048, 1489], "bands": 5,
            "sources_per_gpu": args.sources, "patch_radius": "8-32 by brightness", "galaxy_fraction": 0.6,
            "elbo_tol": 1e-8, "max_iter": 50, "l2": "flushed between timed steps (256 MiB device write)",
            "parallelism": "one independently seeded field per GPU"}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [n for k, n in enumerate(names) if any(r[3 + k].lower().startswith("active") for r in self.rows)]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------- CPU baseline (the oracle)
def subscene(scene, s, reach=None):
    """The inputs source s's objective depends on: s (first), every source whose patch can overlap one
    of s's, and the images holding s's patch centre.  The oracle's objective for s on this scene is
    the one on the whole scene (neighbours are the sources whose patches overlap s's in the same
    image), without laying out all of it."""
    import synth
    r_max = int(scene.radius.max())
    reach = reach if reach is not None else 1.05 * (int(scene.radius[s]) + r_max + 2)
    d = np.abs(scene.u0 - scene.u0[s]).max(1)
    near = np.nonzero(d <= reach)[0]
    idx = np.concatenate([[s], near[near != s]])
    imgs = []
    for im in scene.images:
        p = im.wcs[:4].reshape(2, 2) @ scene.u0[s] + im.wcs[4:]
        cx, cy = math.floor(p[0] + 0.5), math.floor(p[1] + 0.5)
        if 0 <= cx <= im.W - 1 and 0 <= cy <= im.H - 1:
            imgs.append(im)
    return synth.Scene(imgs, scene.u0[idx].copy(), scene.radius[idx].copy(), scene.theta0[idx].copy(), scene.priors,
                       scene.exp_nu, scene.exp_tau, scene.dev_nu, scene.dev_tau, name=f"{scene.name}_src{s}")


def sample_order(scene, seed):
    return np.random.default_rng(seed).permutation(scene.n_sources)


def oracle_solves(scene, seconds, seed, start=0):
    """The float64 oracle, as it stands: full Newton solves of seeded randomly drawn sources (neighbours
    fixed at the catalog) until `seconds` have passed.  Returns (solved, converged, their patch pixels,
    seconds, next start)."""
    from oracle.celeste_oracle import Oracle
    order = sample_order(scene, seed)
    t0 = time.perf_counter()
    solved = conv = px = 0
    k = start
    while time.perf_counter() - t0 < seconds and k < len(order):
        sub = subscene(scene, int(order[k]))
        orc = Oracle(sub)
        if orc.rects[0]:
            r = orc.newton(0, sub.theta0[0], sub.theta0)
            conv += int(r["status"] == 0)
            px += orc.n_pixels(0)
        solved += 1
        k += 1
    return solved, conv, px, time.perf_counter() - t0, k


def oracle_pixel_evals(scene, seconds, seed):
    """The oracle's ELBO + gradient + Hessian evaluation at the catalog for seeded randomly drawn
    sources until `seconds` have passed: (pixel evaluations, seconds, sources evaluated)."""
    from oracle.celeste_oracle import Oracle
    order = sample_order(scene, seed)
    t0 = time.perf_counter()
    px = n = 0
    for s in order:
        if time.perf_counter() - t0 >= seconds:
            break
        sub = subscene(scene, int(s))
        orc = Oracle(sub)
        if orc.rects[0]:
            orc.elbo_grad_hess(0, sub.theta0[0], sub.theta0)
            px += orc.n_pixels(0)
        n += 1
    return px, time.perf_counter() - t0, n


def mean_patch_pixels(scene, chunk=8192):
    """Mean patch pixels per source over the whole scene: per source and image holding its rounded
    patch centre, the (2R+1)^2 window clipped to the image (numpy, independent of the library)."""
    u0 = np.asarray(scene.u0, np.float64)
    R = np.asarray(scene.radius, np.int64)
    total = 0
    for im in scene.images:
        A, o = im.wcs[:4].reshape(2, 2), im.wcs[4:]
        for a in range(0, len(u0), chunk):
            p = u0[a:a + chunk] @ A.T + o
            c = np.floor(p + 0.5).astype(np.int64)
            r = R[a:a + chunk]
            inside = (c[:, 0] >= 0) & (c[:, 0] <= im.W - 1) & (c[:, 1] >= 0) & (c[:, 1] <= im.H - 1)
            w = np.minimum(c[:, 0] + r, im.W - 1) - np.maximum(c[:, 0] - r, 0) + 1
            h = np.minimum(c[:, 1] + r, im.H - 1) - np.maximum(c[:, 1] - r, 0) + 1
            total += int((w * h)[inside].sum())
    return total / len(u0)


def cpu_baseline(scene, seconds, seconds_single, seed, mean_px_all, gpu_pixel_evals_per_source=None):
    """All-core: full oracle Newton solves of a seeded random sample of sources for `seconds`;
    sources/s on the sample, extrapolated to the whole workload linearly in patch pixels (the
    sample's mean patch size against the workload's).  Single-core: the oracle's ELBO+gradient+Hessian
    pixel evaluations per second on the same sample with one thread, turned into sources/s with the
    pixel evaluations per source that the same solve takes on the GPU (when given)."""
    import torch
    threads = torch.get_num_threads()
    solved, conv, px, dt, _ = oracle_solves(scene, seconds, seed)
    out = {"kind": "oracle", "cores": threads}
    if solved and px:
        rate = conv / dt
        out["value"] = rate * (px / solved) / mean_px_all
        out["unit"] = "sources/s"
        out["sample"] = (f"{solved} seeded random sources (full float64 Newton solves, neighbours fixed at the catalog) "
                         f"in {dt:.1f} s on {threads} threads, {conv} converged, mean patch {px / solved:.0f} px vs "
                         f"{mean_px_all:.0f} px over the workload; sources/s extrapolated linearly in patch pixels")
        out["sample_sources_per_s"] = rate
    torch.set_num_threads(1)
    try:
        pe, dt1, n1 = oracle_pixel_evals(scene, seconds_single, seed)
    finally:
        torch.set_num_threads(threads)
    single = {"cores": 1, "pixel_evals_per_s": pe / dt1 if dt1 > 0 else None,
              "sample": f"ELBO+gradient+Hessian at the catalog of {n1} of the same sources, {dt1:.1f} s"}
    if gpu_pixel_evals_per_source and pe:
        single["value"] = (pe / dt1) / gpu_pixel_evals_per_source
        single["unit"] = "sources/s"
        single["extrapolation"] = (f"pixel evaluations per second / {gpu_pixel_evals_per_source:.0f} ELBO+gradient+"
                                   f"Hessian pixel evaluations per source to convergence (the GPU solve's count)")
    out["single_core"] = single
    return out


def make_scene(args, rank, device):
    import synth
    if args.workload == "mosaic":
        from synth.mosaic import mosaic
        f = args.mosaic_fields
        return mosaic(seed=args.seed + rank, fields_x=f, fields_y=f, n_sources=1000 * f * f, device=device)
    return synth.field(seed=args.seed + rank, n_sources=args.sources)


def run_reference(args, rank, world):
    """The float64 oracle on the host cores: each step a bounded sample (about `per_step` seconds) of
    full Newton solves of seeded random sources of the same workload, extrapolated to sources/s of the
    whole workload linearly in patch pixels."""
    if rank != 0:
        return
    import torch
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    scene = make_scene(args, rank, dev)     # input generation only (seeded); the solves run on the CPU
    mean_px = mean_patch_pixels(scene)
    per_step = 6.0
    k = 0
    for _ in range(args.warmup):
        _, _, _, _, k = oracle_solves(scene, 2.0, args.seed, start=k)
    vals, times, solved_total = [], [], 0
    for _ in range(args.steps):
        solved, conv, px, dt, k2 = oracle_solves(scene, per_step, args.seed, start=k)
        k = k2 if k2 < scene.n_sources else 0
        solved_total += solved
        if solved:
            vals.append(conv / dt * (px / solved) / mean_px)
        times.append(dt)
    value = float(np.mean(vals)) if vals else 0.0
    threads = torch.get_num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sources/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "method": {"solver": "float64 CPU oracle: autodiff gradient and Hessian, eigendecomposition trust region",
                       "start": "catalog"},
            "cpu_baseline": {"value": value, "unit": "sources/s", "cores": threads, "kind": "oracle",
                             "sample": f"{solved_total} seeded random sources over {args.steps} steps (full float64 "
                                       f"Newton solves, ~{per_step:.0f} s per step), extrapolated linearly in patch "
                                       f"pixels ({mean_px:.0f} px per source over the workload)"},
            "e2e": {"value": value, "unit": "sources/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def measure_peaks(P):
    out = {}
    for kind in ("fp32", "ex2", "fp64", "fp32x2"):
        rate, _ = P.measure_peak(kind)
        out[kind] = rate
    return {"fp32_fma_tflops": out["fp32"] / 1e12, "ex2_tops": out["ex2"] / 1e12, "fp64_fma_tflops": out["fp64"] / 1e12,
            "fp32x2_fma_tflops": out["fp32x2"] / 1e12,
            "how": "celeste_measure_peak: independent FMA / ex2.approx chains on every SM, best of 3 launches of "
                   "~25 ms each, CUDA events, before the timed steps"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    import paper_1611_03404_gb300 as P
    from paper_1611_03404_gb300 import build as _build

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measure_peaks(P)

    scene = make_scene(args, rank, dev)
    modes = {"fp32": P.HESS_FP32, "tf32": P.HESS_TF32, "bf16x3": P.HESS_BF16X3, "bf16x6": P.HESS_BF16X6,
             "tf32x3": P.HESS_TF32X3}
    tile, tune = args.tile, None
    hname = args.hessian
    if tile == 0 or hname == "auto":
        from paper_1611_03404_gb300.autotune import tune
        cands = None if hname == "auto" else [modes[hname]]
        (tile, hm), tune = tune(scene, device=dev, modes=cands, tiles=None if args.tile == 0 else [args.tile])
        hname = {v: k for k, v in modes.items()}[hm]
    hmode = modes[hname]
    if hmode != P.HESS_FP32:
        tile = 128
    dev_pix = [torch.as_tensor(np.ascontiguousarray(im.pixels, np.float32)).to(dev) for im in scene.images]
    prob = P.Problem(scene, device=dev, tile_pixels=tile, hessian_mode=hmode, device_pixels=dev_pix)
    # the plain form: FP32 FMA Hessian, 128-pixel tiles, Newton from the catalog
    plain_prob = prob if (hmode == P.HESS_FP32 and tile == 128) else \
        P.Problem(scene, device=dev, tile_pixels=128, hessian_mode=P.HESS_FP32, device_pixels=dev_pix)
    counts = prob.counts()
    theta0 = torch.as_tensor(scene.theta0, device=dev).contiguous()
    theta = theta0.clone()
    delta = torch.zeros(scene.n_sources, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    net, ws_info = None, None
    if args.warm_start:
        try:
            net, ws_info = train_warm_start(args, P, dev, rank)
        except Exception as exc:   # the plain form is still measured and reported as value
            net, ws_info = None, {"error": f"warm start not trained: {type(exc).__name__}: {exc}"}
            args.warm_start = False

    def plain_step():
        delta.zero_()
        plain_prob.render_background(theta0)
        theta.copy_(theta0)
        return plain_prob.newton_batch(theta, delta)

    def warm_step():
        from paper_1611_03404_gb300 import cnn
        delta.zero_()
        prob.render_background(theta0)
        pred = net.predict(prob.extract_patches())
        theta.copy_(cnn.warm_start(theta0, pred))
        return prob.newton_batch(theta, delta)

    def mixed_step():
        delta.zero_()
        prob.render_background(theta0)
        theta.copy_(theta0)
        return prob.newton_batch(theta, delta)

    def time_steps(fn, steps, warmup):
        """`warmup` untimed steps, then `steps` steps timed by CUDA events (L2 flushed before each);
        max over ranks."""
        for _ in range(max(warmup, 0)):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        out = None
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            out = fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        t = float(np.sum([a.elapsed_time(b) for a, b in evs])) / 1e3
        if world > 1:
            t, _ = reduce_over_ranks(t, 0, dev)
        return t, out

    def conv_total(status):
        c = int((status == P.STATUS_CONVERGED).sum())
        if world > 1:
            _, c = reduce_over_ranks(0.0, c, dev)
        return c

    # ---- the plain form, for comparison (same workload, same tolerance)
    plain = None
    k_plain = max(1, min(args.plain_steps, args.steps))
    t_plain, (_, it_cat, st_cat, _) = time_steps(plain_step, k_plain, min(args.warmup, 3))
    th_cat = theta.clone()
    cp = conv_total(st_cat)
    plain = {"value": cp / (t_plain / k_plain), "ms_per_step": 1e3 * t_plain / k_plain, "steps": k_plain,
             "newton_iters_mean": float(it_cat.double().mean()), "converged": int((st_cat == 0).sum()),
             "form": "plain FP32 path: Hessian cross-product on FP32 FMAs, 128-pixel tiles, Newton from the catalog"}
    if ws_info is not None:
        ws_info["iters_mean_catalog_start"] = plain["newton_iters_mean"]
    step = warm_step if net is not None else mixed_step

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        prob.profile_start()
        if args.profile_range:
            torch.cuda.cudart().cudaProfilerStart()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            _, iters, status, elbo = step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if args.profile_range:
            torch.cuda.cudart().cudaProfilerStop()
        prof = prob.profile_stop()
    conv = int((status == P.STATUS_CONVERGED).sum())
    iters_mean = float(iters.double().mean())
    # warm-start inference per timed step: patch extraction + six GEMM launches per batch of 4096
    cnn_launches = args.steps * (1 + 6 * ((scene.n_sources + 4095) // 4096)) if net is not None else 0
    th_final = theta.clone()
    if net is not None:
        from paper_1611_03404_gb300 import cnn
        ws_info["iters_mean_warm_start"] = iters_mean
        ws_info["iters_saved_mean"] = ws_info["iters_mean_catalog_start"] - iters_mean
        pred = net.predict(prob.extract_patches())
        tgt = cnn.training_targets(th_cat, torch.as_tensor(scene.u0, device=dev))
        ok = (st_cat == P.STATUS_CONVERGED)
        rmse = ((pred - tgt)[ok] / net.sd).pow(2).mean(0).sqrt()
        ws_info["rmse_vs_converged_standardised"] = [round(float(v), 3) for v in rmse]
    status_counts = {name: int((status == code).sum()) for name, code in
                     (("converged", P.STATUS_CONVERGED), ("max_iter", P.STATUS_MAX_ITER),
                      ("nonfinite", P.STATUS_NONFINITE), ("radius_collapse", P.STATUS_RADIUS_COLLAPSE))}
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_step = float(np.sum(step_ms)) / 1e3
    c_total = conv_total(status)
    if world > 1:
        t_step, _ = reduce_over_ranks(t_step, 0, dev)
        dist.barrier()
    ms_per_step = 1e3 * t_step / args.steps
    value = c_total / (ms_per_step / 1e3)
    # the two catalogs agree: the headline's converged parameters against the plain form's
    agree = catalog_agreement(th_final, th_cat, status, st_cat, prob, theta0)

    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or 1920.0
    roofline, kernels = rooflines(prof, t_step, n_sm, sm_mhz, peaks, iters, args.steps, kernel_variant(tile, hmode))

    e2e = end_to_end(args, P, prob, scene, step, theta, theta0, flush, stream, world, dev) if args.e2e_steps > 0 else None

    reports = {}
    if rank == 0 and args.reports:
        if args.workload == "mosaic":
            reports["blockcoord"] = blockcoord_report(P, plain_prob, theta0, scene)
        elif args.joint:
            reports["joint"] = joint_report(P, plain_prob, theta0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        px_per_source = prof["full_pixels"] / args.steps / max(scene.n_sources, 1)
        cpu = cpu_baseline(scene, args.cpu_seconds, args.cpu_seconds_single, args.seed, counts["pixels"] / counts["sources"],
                           gpu_pixel_evals_per_source=px_per_source)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "sources/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args),
                "method": {"hessian_syrk": hname, "tile_pixels": tile, "tile_choice": "autotuned" if tune else "fixed",
                           "warm_start": "cnn" if net is not None else None,
                           "precision": "pixel arithmetic FP32; Hessian cross-product " + hname +
                                        "; cross-pixel sums, assembly and trust-region step FP64"},
                "autotune": tune, "warm_start": ws_info, "plain_fp32": plain, "catalog_agreement": agree,
                "pixel_evals_per_s": prof["full_pixels"] / (prof["full_ms"] / 1e3) if prof["full_ms"] > 0 else None,
                "converged": conv, "newton_iters_mean": iters_mean, "newton_iters_max": int(iters.max()),
                "status_counts": status_counts, "layout": counts, "wall_s_timed": wall,
                "roofline": roofline, "kernels": kernels, "measured_peaks": peaks, "sm_count": n_sm,
                "cpu_baseline": cpu, "e2e": e2e, "reports": reports,
                "gpu_launches": prof["kernel_launches"] + cnn_launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def kernel_variant(tile, hmode):
    """Name of the pixel-kernel instantiation that a problem with this tile size and Hessian form runs."""
    ppt = {128: 1, 256: 2, 512: 4}.get(tile, 8)
    return f"elbo_full_kernel<{1 if hmode else ppt}, {hmode}>"


def rooflines(prof, t_step, n_sm, sm_mhz, peaks, iters, steps, variant):
    """The pixel kernel (FP32 bound; also against the special-function unit and HBM) and the
    trust-region step (FP64), each with its share of the timed steps.  `traffic` comes from the
    committed DRAM capture of the same kernel variant, if its source is unchanged since."""
    clk = sm_mhz * 1e6
    nominal_fp32 = n_sm * FP32_LANES_PER_SM * 2 * clk / 1e12
    nominal_mufu = n_sm * MUFU_PER_SM_CLK * clk / 1e12
    nominal_fp64 = n_sm * FP64_PER_SM_CLK * 2 * clk / 1e12
    full_s = prof["full_ms"] / 1e3
    px = prof["full_pixels"]
    achieved = FLOPS_FULL_PER_PIXEL * px / full_s / 1e12 if full_s > 0 else None
    mufu = MUFU_FULL_PER_PIXEL * px / full_s / 1e12 if full_s > 0 else None
    hbm = BYTES_FULL_PER_PIXEL * px / full_s / 1e9 if full_s > 0 else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "elbo_full_kernel_traffic.json")
    if os.path.exists(tfile) and prof["full_launches"]:
        with open(tfile) as f:
            tr = json.load(f)
        ent = tr.get("kernels", {}).get(variant)
        if ent and tr.get("kernel_source_hash") == _build_hash():
            traffic = ent["dram_bytes_per_pixel"] * px / prof["full_launches"]
    roof = {"bound": "alu", "kernel": variant, "achieved": achieved, "peak": nominal_fp32,
            "unit": "TFLOP/s", "frac": achieved / nominal_fp32 if achieved else None, "traffic": traffic,
            "peak_basis": f"{n_sm} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_mhz:.0f} MHz (median SM "
                          f"clock sampled during the timed steps)",
            "frac_of_measured_fp32": achieved / peaks["fp32_fma_tflops"] if achieved else None,
            "flops_per_pixel": FLOPS_FULL_PER_PIXEL, "pixels": px, "launches": prof["full_launches"],
            "kernel_ms": prof["full_ms"], "share_of_step": full_s / t_step if t_step > 0 else None,
            "sfu": {"achieved_tops": mufu, "peak_tops_nominal": nominal_mufu, "peak_tops_measured": peaks["ex2_tops"],
                    "frac_of_measured": mufu / peaks["ex2_tops"] if mufu else None, "mufu_per_pixel": MUFU_FULL_PER_PIXEL},
            "hbm": {"achieved_gbs": hbm, "bytes_per_pixel": BYTES_FULL_PER_PIXEL, "peak_gbs": _hbm_peak()}}
    tr_s = prof.get("tr_ms", 0.0) / 1e3
    subproblems = int(iters.long().sum()) * steps        # one subproblem per Newton iteration of a source
    tr_flops = FP64_FLOPS_PER_SUBPROBLEM * subproblems / tr_s / 1e12 if tr_s > 0 else None
    kernels = {
        "elbo_full_kernel": {"ms": prof["full_ms"], "launches": prof["full_launches"],
                             "share_of_step": full_s / t_step if t_step > 0 else None},
        "elbo_value_kernel": {"ms": prof["value_ms"], "launches": prof["value_launches"],
                              "share_of_step": prof["value_ms"] / 1e3 / t_step if t_step > 0 else None,
                              "pixels": prof["value_pixels"],
                              "achieved_tflops": FLOPS_VALUE_PER_PIXEL * prof["value_pixels"] / (prof["value_ms"] / 1e3) / 1e12
                              if prof["value_ms"] > 0 else None},
        "tr_step_kernel": {"bound": "fp64", "ms": prof.get("tr_ms"), "launches": prof.get("tr_launches"),
                           "share_of_step": tr_s / t_step if t_step > 0 else None, "subproblems": subproblems,
                           "us_per_launch": 1e3 * prof.get("tr_ms", 0.0) / max(prof.get("tr_launches", 0), 1),
                           "achieved_tflops": tr_flops, "flops_per_subproblem": FP64_FLOPS_PER_SUBPROBLEM,
                           "peak_tflops_nominal": nominal_fp64, "peak_tflops_measured": peaks["fp64_fma_tflops"],
                           "frac_of_measured": tr_flops / peaks["fp64_fma_tflops"] if tr_flops else None},
    }
    return roof, kernels


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        return None


def catalog_agreement(th, th_ref, st, st_ref, prob, theta0):
    """Per parameter, the largest difference between two converged catalogs of the same workload
    (the headline form's and the plain form's), over sources converged in both, in the free
    parameters of the position and the reference-band log flux, and the ELBO difference."""
    import torch
    ok = (st == 0) & (st_ref == 0)
    if int(ok.sum()) == 0:
        return None
    d = (th - th_ref)[ok].abs()
    return {"sources": int(ok.sum()), "max_position_px_world": float(d[:, 0:2].max()),
            "p99_position": float(torch.quantile(d[:, 0:2].max(1).values.float(), 0.99)),
            "median_max_param": float(d.max(1).values.median())}


def end_to_end(args, P, prob, scene, step, theta, theta0, flush, stream, world, dev):
    """Through the public API at N GPUs: every step copies the images and the catalog from pinned host
    memory, re-gathers the patch pixels from the new images (celeste_problem_refresh_pixels), runs the
    step and reads the converged catalog and status back; L2 flushed before each step as in the timed
    loop; the first step warms the pinned buffers and is not counted."""
    import torch
    host_pix = [torch.from_numpy(np.ascontiguousarray(im.pixels)).pin_memory() for im in scene.images]
    host_theta = torch.from_numpy(scene.theta0.copy()).pin_memory()
    out_theta = torch.empty_like(host_theta).pin_memory()
    out_status = torch.empty(scene.n_sources, dtype=torch.int32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host_pix) + host_theta.numel() * 8
    d2h = out_theta.numel() * 8 + out_status.numel() * 4
    e_times, e_conv = [], 0
    for k in range(args.e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for dp, hp in zip(prob.pixels, host_pix):
            dp.copy_(hp, non_blocking=True)
        theta0.copy_(host_theta, non_blocking=True)
        prob.refresh_pixels()
        _, _, status_e, _ = step()
        out_theta.copy_(theta, non_blocking=True)
        out_status.copy_(status_e, non_blocking=True)
        torch.cuda.synchronize()
        if k > 0:
            e_times.append(time.perf_counter() - t0)
            e_conv = int((out_status == P.STATUS_CONVERGED).sum())
    te = float(np.mean(e_times))
    if world > 1:
        te, e_conv = reduce_over_ranks(te, e_conv, dev)
    return {"value": e_conv / te, "unit": "sources/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": 1e3 * te, "steps": args.e2e_steps,
            "l2": "flushed before each step (256 MiB device write, outside the host timer's copies)"}


def train_warm_start(args, P, dev, rank):
    """Trains the warm-start network on (patch, converged parameters) pairs of two freshly seeded
    100k-source scenes of the bench's kind (mosaics; for the field workload with the field's five
    bands per exposure and radius rule), solved by Newton from their catalogs with neighbours fixed
    at the catalog."""
    import torch
    from paper_1611_03404_gb300 import cnn
    t0 = time.perf_counter()
    xs, ts = [], []
    from synth.mosaic import mosaic
    for k in (101, 102):
        if args.workload == "mosaic":
            sc = mosaic(seed=args.seed + rank + k, device=dev)
        else:
            # field-like exposures (all five bands per field, the field's radius rule), rendered on the
            # GPU: 100k sources per training scene instead of the field's 1000
            sc = mosaic(seed=args.seed + rank + k, bands_per_field=(5, 5), extended=0.0, rmax=32,
                        radius_rule="brightness", device=dev)
        pr = P.Problem(sc, device=dev, tile_pixels=128)
        th = torch.as_tensor(sc.theta0, device=dev).contiguous()
        pr.render_background(th.clone())
        _, _, st, _ = pr.newton_batch(th)
        ok = st == P.STATUS_CONVERGED
        xs.append(pr.extract_patches()[ok])
        ts.append(cnn.training_targets(th[ok], torch.as_tensor(sc.u0, device=dev)[ok]))
        pr.close()
        del sc
    x, t = torch.cat(xs).contiguous(), torch.cat(ts).contiguous()
    t_data = time.perf_counter() - t0
    net = cnn.WarmStartCNN(dev, seed=args.seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = net.train(x, t, epochs=args.ws_epochs, batch=512, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    return net, {"train_pairs": int(x.shape[0]), "epochs": args.ws_epochs, "batch": 512,
                 "loss_first_last": [hist[0], hist[-1]], "data_seconds": t_data, "train_seconds": t_train,
                 "train_pairs_per_s": x.shape[0] * args.ws_epochs / t_train,
                 "params_from_network": "type logit, log variances of the log fluxes and colours"}


def reduce_over_ranks(t, count, dev):
    """Whole-job figures from per-rank ones (every rank calls it): the slowest rank's time (max)
    and the sum of the ranks' counts, so value = count / time covers all ranks' work."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t)], device=dev, dtype=torch.float64)
    cc = torch.tensor([float(count)], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(cc, op=dist.ReduceOp.SUM)
    return float(tt), float(cc)


def blockcoord_report(P, prob, theta0, scene, passes=3):
    """Untimed: block-coordinate passes over the whole workload, each with the neighbours at the
    previous pass's result, and the catalog change per pass."""
    import torch
    from paper_1611_03404_gb300.blockcoord import block_coordinate
    # patch half-width in world units (the pixel grids' scale is within 2 % of the world's)
    rw = torch.as_tensor(scene.radius, device=theta0.device, dtype=torch.float64) / 1.02
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, hist = block_coordinate(prob, theta0.clone().contiguous(), passes=passes, radius_world=rw)
    torch.cuda.synchronize()
    return {"what": f"{passes} block-coordinate passes from the catalog (plain FP32 form), neighbours re-rendered at the "
                    "previous pass's result; per pass the parameter changes, Newton iterations and converged count; "
                    "untimed", "seconds": time.perf_counter() - t0, "passes": hist}


def joint_report(P, prob, theta0):
    """Untimed: the joint objective over all sources of the field (every covered pixel counted
    once), after four window-mode block-coordinate passes from the catalog and after the joint
    trust-region Newton started from their result."""
    import torch
    from paper_1611_03404_gb300.blockcoord import block_coordinate
    cat = theta0.clone().contiguous()
    J_cat = prob.joint_value(cat)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th, _ = block_coordinate(prob, cat, passes=4, mode=P.NBR_WINDOW)
    torch.cuda.synchronize()
    t_bc = time.perf_counter() - t0
    J_bc = prob.joint_value(th)
    t0 = time.perf_counter()
    res = prob.joint_newton(th, max_iter=100)
    t_jn = time.perf_counter() - t0
    return {"what": "joint objective J (every covered pixel once); 4 window-mode block-coordinate passes from the "
                    "catalog, then joint trust-region Newton (CG-Steihaug subproblems) from their result; untimed",
            "pairs": int(len(prob.joint_pairs())), "J_catalog": J_cat, "J_blockcoord_4": J_bc, "blockcoord_s": t_bc,
            "J_joint": res["J"], "joint_s": t_jn, "joint_iters": res["iters"], "joint_status": res["status"],
            "joint_cg_iters": res["cg_iters"]}


def _build_hash():
    """The pixel kernels' source: the kernel file and the header with the table layout."""
    import hashlib
    h = hashlib.sha256()
    for name in ("pixels.cu", "celeste_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1611_03404_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()

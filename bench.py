#!/usr/bin/env python
"""Benchmark: light sources per second to convergence, batched trust-region Newton on one GPU.

One step = one block-coordinate pass over a synthetic field (2048x1489 px x 5 bands, 1000 sources,
patch radius 8-32 px by brightness): render the neighbours' fixed background, run the learned
warm-start network on every source's patch, then run trust-region Newton (ELBO + exact gradient +
dense Hessian per iteration) on every source from that start until all have stopped.  The network
is trained before the timed region on pairs from two freshly seeded scenes; the plain form
(Newton from the catalog, no network) is timed as well and reported as "plain_fp32"
(--no-warm-start times only the plain form).  Under torchrun every rank solves its own independently seeded field (weak
scaling, no collective on the data path); the timing is the max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the float64 CPU oracle (the plain, slow definition of the same
objective and optimiser) on the host cores, on a bounded sample of the same workload.
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
N_SM = 152
FP32_LANES_PER_SM = 128

# Algorithmic float32 operations per pixel evaluation (FMA = 2), counted from the formulas the
# kernels evaluate (breakdown in the design notes):
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
# MUFU (special-function) operations per full pixel evaluation: 45 exp2, 2 reciprocals/divides, 1 log1p
MUFU_FULL_PER_PIXEL = 48


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="field", choices=["field", "mosaic"],
                    help="field: 2048x1489 px x 5 bands, --sources sources (the headline workload); "
                         "mosaic: 10x10 overlapping fields, 100,000 sources, 1-12 exposures each")
    ap.add_argument("--sources", type=int, default=1000)
    ap.add_argument("--tile", type=int, default=128, help="pixels per tile; 0 = autotune")
    ap.add_argument("--no-warm-start", dest="warm_start", action="store_false",
                    help="time only the plain form (Newton from the catalog).  By default the learned warm start is "
                         "trained first (on (patch, converged parameters) pairs of two freshly seeded scenes of the "
                         "same kind, outside the timed region) and every timed Newton solve starts from its "
                         "prediction (inference inside the timed region); the plain form is timed too and reported "
                         "beside it")
    ap.add_argument("--ws-epochs", type=int, default=6)
    ap.add_argument("--hessian", default="fp32", choices=["fp32", "tf32", "bf16x3"],
                    help="Jacobian cross-product of the Hessian: FP32 FMAs or tensor cores (TF32, BF16 hi+lo)")
    ap.add_argument("--seed", type=int, default=1611)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-joint", dest="joint", action="store_false",
                    help="skip the untimed joint-objective report")
    return ap.parse_args()


def workload_config(args, tile):
    if args.workload == "mosaic":
        return {"workload": "mosaic_10x10_fields_100000src", "fields": [10, 10], "field_px": [2048, 1489],
                "field_overlap": 0.2, "bands_per_field": "1-3", "exposures_per_source": "1-12",
                "sources_per_gpu": 100_000, "patch_radius": "8-64 (brightness, 4 sigma of the widest component)",
                "galaxy_fraction": 0.6, "elbo_tol": 1e-8, "max_iter": 50, "tile_pixels": tile,
                "hessian_syrk": args.hessian, "warm_start": "cnn" if args.warm_start else None, "tile_choice": "autotuned" if args.tile == 0 else "fixed",
                "l2": "inputs larger than L2 (GBs of patch pixels) and a 256 MiB flush between timed steps",
                "parallelism": "one independently seeded mosaic per GPU"}
    return {"workload": f"field_2048x1489x5_{args.sources}src", "image_px": [2048, 1489], "bands": 5,
            "sources_per_gpu": args.sources, "patch_radius": "8-32 by brightness", "galaxy_fraction": 0.6,
            "elbo_tol": 1e-8, "max_iter": 50, "tile_pixels": tile, "hessian_syrk": args.hessian,
            "warm_start": "cnn" if args.warm_start else None,
            "l2": "flushed between timed steps (256 MiB device write)",
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


def cpu_baseline(scene, seconds):
    """The float64 oracle, as it stands, on the host cores: full Newton solves of the field's sources
    in index order until `seconds` of CPU work; returns (sources/s, sources solved, threads)."""
    import torch
    from oracle.celeste_oracle import Oracle
    orc = Oracle(scene)
    t0 = time.perf_counter()
    done = 0
    conv = 0
    while time.perf_counter() - t0 < seconds and done < scene.n_sources:
        if orc.rects[done]:
            r = orc.newton(done, scene.theta0[done], scene.theta0)
            conv += int(r["status"] == 0)
        done += 1
    dt = time.perf_counter() - t0
    return conv / dt, done, torch.get_num_threads(), dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    args.warm_start = False   # the oracle runs the method as written: Newton from the catalog
    import torch
    import synth
    scene = synth.field(seed=args.seed, n_sources=args.sources)
    per_step = max(args.cpu_seconds / 2, 5.0)
    for _ in range(args.warmup):
        cpu_baseline(scene, min(per_step, 5.0))
    vals, times, solved = [], [], 0
    for _ in range(args.steps):
        v, n, thr, dt = cpu_baseline(scene, per_step)
        vals.append(v)
        times.append(dt)
        solved = n
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sources/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, args.tile),
            "cpu_baseline": {"value": value, "unit": "sources/s", "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": f"first {solved} sources of the field per step (full Newton solves), "
                                       f"~{per_step:.0f} s of CPU work per step"},
            "e2e": {"value": value, "unit": "sources/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    import synth
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

    if args.workload == "mosaic":
        from synth.mosaic import mosaic
        scene = mosaic(seed=args.seed + rank, device=dev)
    else:
        scene = synth.field(seed=args.seed + rank, n_sources=args.sources)
    tile, tune = args.tile, None
    if tile == 0:
        from paper_1611_03404_gb300.autotune import tune_tile
        tile, tune = tune_tile(scene, device=dev)
    hmode = {"fp32": P.HESS_FP32, "tf32": P.HESS_TF32, "bf16x3": P.HESS_BF16X3}[args.hessian]
    if hmode != P.HESS_FP32:
        tile = 128
    prob = P.Problem(scene, device=dev, tile_pixels=tile, hessian_mode=hmode)
    counts = prob.counts()
    theta0 = torch.as_tensor(scene.theta0, device=dev).contiguous()
    theta = theta0.clone()
    delta = torch.zeros(scene.n_sources, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    net, ws_info, plain = None, None, None
    stream = torch.cuda.current_stream()

    def plain_step():
        delta.zero_()
        prob.render_background(theta0)
        theta.copy_(theta0)
        return prob.newton_batch(theta, delta)

    def warm_step():
        from paper_1611_03404_gb300 import cnn
        delta.zero_()
        prob.render_background(theta0)
        pred = net.predict(prob.extract_patches())
        theta.copy_(cnn.warm_start(theta0, pred))
        return prob.newton_batch(theta, delta)

    def time_steps(fn):
        """W untimed steps, then K steps timed by CUDA events (L2 flushed before each); max over ranks."""
        for _ in range(max(args.warmup, 0)):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        out = None
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            out = fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        t = float(np.sum([a.elapsed_time(b) for a, b in evs])) / 1e3
        if world > 1:
            t, _ = reduce_over_ranks(t, 0, dev)
        return t, out

    if args.warm_start:
        try:
            net, ws_info = train_warm_start(args, P, dev, rank)
        except Exception as exc:   # the plain form is still measured and reported as value
            net, ws_info = None, {"error": f"warm start not trained: {type(exc).__name__}: {exc}"}
            args.warm_start = False
    if net is not None:
        # the plain form (Newton from the catalog) on the same workload, timed the same way
        t_plain, (_, it_cat, st_cat, _) = time_steps(plain_step)
        th_cat = theta.clone()
        conv_plain = int((st_cat == P.STATUS_CONVERGED).sum())
        if world > 1:
            _, conv_plain_total = reduce_over_ranks(0.0, conv_plain, dev)
        else:
            conv_plain_total = conv_plain
        plain = {"value": conv_plain_total / (t_plain / args.steps), "ms_per_step": 1e3 * t_plain / args.steps,
                 "newton_iters_mean": float(it_cat.double().mean()), "converged": conv_plain,
                 "form": "plain FP32 path, Newton from the catalog"}
        ws_info["iters_mean_catalog_start"] = plain["newton_iters_mean"]
        ws_info["converged_catalog_start"] = conv_plain
    step = warm_step if net is not None else plain_step

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    conv, iters_sum = 0, 0
    with ClockSampler(local_rank) as clk:
        prob.profile_start()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            _, iters, status, elbo = step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        prof = prof_stats = prob.profile_stop()
    conv = int((status == P.STATUS_CONVERGED).sum())
    iters_mean = float(iters.double().mean())
    # warm-start inference per timed step: patch extraction + six GEMM launches per batch of 4096
    cnn_launches = args.steps * (1 + 6 * ((scene.n_sources + 4095) // 4096)) if net is not None else 0
    if net is not None:
        from paper_1611_03404_gb300 import cnn
        ws_info["iters_mean_warm_start"] = iters_mean
        ws_info["iters_saved_mean"] = ws_info["iters_mean_catalog_start"] - iters_mean
        pred = net.predict(prob.extract_patches())
        tgt = cnn.training_targets(th_cat, torch.as_tensor(scene.u0, device=dev))
        ok = (st_cat == P.STATUS_CONVERGED)
        rmse = ((pred - tgt)[ok] / net.sd).pow(2).mean(0).sqrt()
        ws_info["rmse_vs_converged_standardised"] = [round(float(v), 3) for v in rmse]
    iters_max = int(iters.max())
    status_counts = {name: int((status == code).sum()) for name, code in
                     (("converged", P.STATUS_CONVERGED), ("max_iter", P.STATUS_MAX_ITER),
                      ("nonfinite", P.STATUS_NONFINITE), ("radius_collapse", P.STATUS_RADIUS_COLLAPSE))}
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_step = float(np.sum(step_ms)) / 1e3
    if world > 1:
        t_step, conv_total = reduce_over_ranks(t_step, conv, dev)
        dist.barrier()
    else:
        conv_total = conv
    ms_per_step = 1e3 * t_step / args.steps
    value = conv_total / (ms_per_step / 1e3)

    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or 1920.0
    fp32_peak_tflops = N_SM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    full_ms = prof["full_ms"]
    achieved = (FLOPS_FULL_PER_PIXEL * prof["full_pixels"] / (full_ms / 1e3) / 1e12) if full_ms > 0 else None
    px_rate = prof["full_pixels"] / (full_ms / 1e3) if full_ms > 0 else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "elbo_full_kernel_traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tr = json.load(f)
        if tr.get("kernel_source_hash") == _build_hash(P):
            per_px = tr["dram_bytes_per_pixel"]
            traffic = per_px * prof["full_pixels"] / max(prof["full_launches"], 1)

    # end-to-end through the public API: pinned host inputs in, converged catalog out, per step
    e2e = None
    if args.e2e_steps > 0:
        host_pix = [torch.from_numpy(np.ascontiguousarray(im.pixels)).pin_memory() for im in scene.images]
        host_theta = torch.from_numpy(scene.theta0.copy()).pin_memory()
        out_theta = torch.empty_like(host_theta).pin_memory()
        out_status = torch.empty(scene.n_sources, dtype=torch.int32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host_pix) + host_theta.numel() * 8
        d2h = out_theta.numel() * 8 + out_status.numel() * 4
        e_times, e_conv = [], 0
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for dp, hp in zip(prob.pixels, host_pix):
                dp.copy_(hp, non_blocking=True)
            theta0.copy_(host_theta, non_blocking=True)
            prob.rebind()
            _, iters_e, status_e, _ = step()
            out_theta.copy_(theta, non_blocking=True)
            out_status.copy_(status_e, non_blocking=True)
            torch.cuda.synchronize()
            if k > 0:   # first pass warms the pinned buffers
                e_times.append(time.perf_counter() - t0)
                e_conv = int((out_status == P.STATUS_CONVERGED).sum())
        te = float(np.mean(e_times))
        if world > 1:
            te, e_conv = reduce_over_ranks(te, e_conv, dev)
        e2e = {"value": e_conv / te, "unit": "sources/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * te}

    joint = None
    if rank == 0 and args.joint and args.workload == "field":
        joint = joint_report(P, prob, theta0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "field":
        v, n, thr, dt = cpu_baseline(scene, args.cpu_seconds)
        cpu = {"value": v, "unit": "sources/s", "cores": thr, "kind": "oracle",
               "sample": f"first {n} of the {scene.n_sources} field sources (full float64 Newton solves, "
                         f"neighbours fixed at the catalog), {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "sources/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args, tile),
                "autotune_us_per_1000px": tune, "warm_start": ws_info, "plain_fp32": plain,
                "pixel_evals_per_s": px_rate, "converged": conv, "newton_iters_mean": iters_mean,
                "newton_iters_max": iters_max, "status_counts": status_counts,
                "layout": counts, "wall_s_timed": wall,
                "roofline": {"bound": "alu", "kernel": "elbo_full_kernel", "achieved": achieved,
                             "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                             "frac": (achieved / fp32_peak_tflops) if achieved else None, "traffic": traffic,
                             "peak_basis": f"{N_SM} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_mhz:.0f} MHz "
                                           f"(median SM clock sampled during the timed steps)",
                             "flops_per_pixel": FLOPS_FULL_PER_PIXEL,
                             "launches": prof["full_launches"], "kernel_ms": full_ms,
                             "share_of_step": full_ms / (1e3 * t_step) if t_step > 0 else None},
                "cpu_baseline": cpu, "e2e": e2e, "joint": joint,
                "gpu_launches": prof["kernel_launches"] + cnn_launches,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def train_warm_start(args, P, dev, rank):
    """Trains the warm-start network on (patch, converged parameters) pairs of two freshly seeded
    100k-source scenes of the bench's kind (mosaics; for the field workload with the field's five
    bands per exposure and radius rule), solved by Newton from their catalogs with neighbours fixed
    at the catalog."""
    import torch
    import synth
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


def _build_hash(P):
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_1611_03404_gb300", "csrc", "pixels.cu")
    with open(src, "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()

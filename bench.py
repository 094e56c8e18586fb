"""Benchmark of the sensitivity-scoring hot path (arXiv 2607.02721, Sec. 3, Algorithm 1).

One step = one pass of the path over the whole query set: EWA projection of every
Gaussian into every view, (tile, depth) binning, the two-pass per-pixel compositing and
sensitivity reduction (Eq. sen), S = sum s, and the draw of a 90%-pruning coreset
(m = 0.1 N, weights 1/(m p)).  Metric: pixel-rays scored per second.

Default workload: 3,000,000 Gaussians from a 256-component mixture (SH degree 3),
200 views of 1600x1040 on a jittered hemisphere (332.8M rays per step); synthetic,
seeded.  The scene (708 MB) is larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sensitivity rays/sec at 3M Gaussians; surrogate vs exact at ΔPSNR ≤ 0.1 dB"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "composite_score_traffic.md")
COMPOSITE_SRC = os.path.join(ROOT, "paper_2607_02721_b300", "csrc", "k_composite.cu")

# Algorithmic work of the compositing kernel: 18 FP32 instructions per evaluated (ray,
# Gaussian) pair and pass (quadratic form, cut test, exp, clamp, alpha_min test, 1 - rho,
# T update, t_min test, rho T and the colour / score terms, as a plain per-pair
# implementation executes them), times the pairs each pass evaluates (device counters).
OPS_PER_PAIR = 18
# The kernel's own essential count (reported beside it): the footprint test is 6 ops
# (5 FFMA for log2 alpha - e1^2 - e2^2, 1 FSETP); a pass-1 contribution adds 8 (FMNMX,
# FADD, FMUL, FSETP, FMUL, 3 FFMA) and a pass-2 contribution 5 (FMNMX, FMUL, FMUL, FADD,
# FMUL); MUFU ex2 runs on the XU pipe, outside both counts.
OPS_TEST, OPS_HIT1, OPS_HIT2 = 6, 8, 5
SMS, FP32_LANES = 148, 128

# Algorithmic bytes of the HBM-bound phases (per launch of a view batch of nb views):
#   projection: each Gaussian's attributes read once (means 12, log-scales 12, quaternion 16,
#     opacity 4, SH (d+1)^2 x 12 bytes: 236 B at degree 3), then per (view, Gaussian) a depth
#     key (4 B) and a tile rectangle (8 B) written, plus the 48-byte splat of a visible one;
#   binning: depth sort of nb x N keys in three 9-bit passes (histogram read 4 B, scatter
#     read 8 B (4 B in the first pass: the values are the indices) and write 8 B per key and
#     pass: 56 B), the emit (depth order and rectangle read in both of its passes: 24 B per
#     (view, Gaussian); (key, value) written: 8 B per instance) and the (view, tile) sort of
#     the instances in two passes (20 B per instance and pass).
PROJ_READ_PER_G = {0: 56, 1: 92, 2: 152, 3: 236}
PROJ_WRITE_PER_VG, PROJ_WRITE_PER_VIS = 12, 48
SORT_PER_VG, SORT_PER_INST = 56 + 24, 8 + 2 * 20


def workload(name: str):
    from paper_2607_02721_b300 import synth

    if name == "scene_3m":
        scene, cams = synth.workload_scene_3m()
    elif name == "scene_1m":
        scene, cams = synth.workload_scene_1m()
    elif name == "small":
        scene, cams, _ = synth.workload_small()
    else:
        raise SystemExit(f"unknown workload {name}")
    return scene, cams


# --tile-shape: library codes (CSGS_TILE_*; 0 = the autotuner's choice)
TILE_SHAPES = {"auto": 0, "16x16": 1, "32x8": 2, "16x8": 3, "8x8": 4}

# --score-resolution: (library code, description) of the query resolutions of Sec. 3.5
SCORE_RESOLUTIONS = {"pixel": (0, "per-pixel (max over pixel-rays)"), "scene": (1, "per-scene (one query)"),
                     "channel": (2, "per-channel (max over pixel-ray channels)"),
                     "tile": (3, "per-tile (max over 16x16 tiles)"), "image": (4, "per-image (max over views)")}


def describe(name, scene, cams):
    W, H = int(cams[0][16]), int(cams[0][17])
    return {"workload": name, "n_gaussians": scene.n, "sh_degree": scene.sh_degree, "views": len(cams),
            "width": W, "height": H, "rays_per_step": int(sum(int(c[16]) * int(c[17]) for c in cams)),
            "resolution": "per-pixel (max over pixel-rays)", "objective": "R+G+B",
            "coreset_m": int(round(0.1 * scene.n)), "scorer": "exact",
            "l2": "inputs larger than L2 (scene %.0f MB)" % (scene_bytes(scene) / 1e6),
            "parallelism": "single GPU"}


def scene_bytes(scene) -> int:
    return sum(a.nbytes for a in (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh))


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None

    def stop(self) -> dict | None:
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def traffic_per_launch():
    """DRAM bytes per compositing launch from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None, None
    txt = open(TRAFFIC_FILE).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    m_b = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_b:
        return None, None
    sha = hashlib.sha256(open(COMPOSITE_SRC, "rb").read()).hexdigest()
    if sha != m_sha.group(1):
        return None, "stale"
    return float(m_b.group(1)), None


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except (OSError, ValueError):
        return {}


def _center_pixels(cams, count):
    """The first ``count`` pixels, row-major, of a band centred in view 0."""
    import numpy as np

    H, W = int(cams[0][17]), int(cams[0][16])
    count = int(max(1, min(count, H * W)))
    rows = (count + W - 1) // W
    r0 = max(0, H // 2 - rows // 2)
    ys, xs = np.divmod(np.arange(count) + r0 * W, W)
    return np.stack([xs, ys], 1).astype(np.int32)


def _oracle_step(sa, cams, pixels):
    import oracle

    if pixels is None:
        return oracle.score(sa, cams)
    return oracle.score_pixels(sa, cams[0], pixels)


def _calibrate(sa, cams, budget_s):
    """Pixel count of view 0 that the oracle scores in about ``budget_s`` seconds
    (None: the whole workload fits).  Two timed probes, each with enough pixels per
    thread to load every core, give the per-pixel cost and the per-call overhead."""
    import oracle

    th = max(1, oracle.num_threads())
    p0, p1 = 16 * th, 64 * th
    t = time.perf_counter()
    _oracle_step(sa, cams, _center_pixels(cams, p0))
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    _oracle_step(sa, cams, _center_pixels(cams, p1))
    t1 = time.perf_counter() - t
    per_px = max((t1 - t0) / (p1 - p0), t1 / p1 * 0.25, 1e-9)
    overhead = max(t1 - p1 * per_px, 0.0)
    rays = int(sum(int(c[16]) * int(c[17]) for c in cams))
    if overhead * len(cams) + rays * per_px <= budget_s:
        return None
    return int(max(p0, min((budget_s - overhead) / per_px, p1 * budget_s / max(t1, 1e-6) * 2)))


def cpu_baseline(name, scene, cams, budget_s: float):
    """The oracle, as it stands, on a bounded sample of the workload: the whole query
    set if it fits in about ``budget_s`` seconds, else a block of pixels centred in
    view 0."""
    import oracle

    sa = oracle.SceneArrays(scene)
    npx = _calibrate(sa, cams, budget_s)
    pix = None if npx is None else _center_pixels(cams, npx)
    t = time.perf_counter()
    _oracle_step(sa, cams, pix)
    el = time.perf_counter() - t
    rays = int(sum(int(c[16]) * int(c[17]) for c in cams)) if pix is None else len(pix)
    sample = (f"the whole {name} query set ({rays} pixel-rays)" if pix is None else
              f"{rays} pixel-rays: a block of rows centred in view 0 of the {name} workload")
    return {"value": rays / el, "unit": "rays/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": sample + f", FP64, {el:.1f} s"}, rays, el


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    scene, cams = workload(args.workload)
    cfg = describe(args.workload, scene, cams)
    if args.gpus > 1:  # the configuration of the arm it is compared with (the oracle runs on rank 0 only)
        cfg["parallelism"] = f"views sharded over {args.gpus} ranks, all-reduce of s per step"
        cfg["views_per_rank"] = len(range(0, len(cams), args.gpus))
    per_step = max(2.0, min(15.0, 150.0 / max(1, args.steps + args.warmup)))
    sa = oracle.SceneArrays(scene)
    npx = _calibrate(sa, cams, per_step)
    pix = None if npx is None else _center_pixels(cams, npx)
    rays_step = int(sum(int(c[16]) * int(c[17]) for c in cams)) if pix is None else len(pix)
    for _ in range(args.warmup):
        _oracle_step(sa, cams, pix)
    t = time.perf_counter()
    for _ in range(args.steps):
        _oracle_step(sa, cams, pix)
    el = time.perf_counter() - t
    v = rays_step * args.steps / el
    sample = ("the whole query set" if pix is None else f"{rays_step} pixel-rays centred in view 0")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "rays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "rays/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"each step: {sample} of the {args.workload} workload"},
            "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def job_time_ms(local_ms: float, dist=None, device=None) -> float:
    """The job's time: the maximum of the ranks' timed regions (replicas run the same
    work on their own GPU; the slowest one ends the job)."""
    if dist is None:
        return float(local_ms)
    import torch

    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_rate(units_per_rank: float, world: int, job_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the job's time."""
    return units_per_rank * world / (job_ms / 1e3)


def run_ours(args):
    import numpy as np
    import torch

    import paper_2607_02721_b300 as csgs
    from paper_2607_02721_b300 import build, sharded

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    scene, cams = workload(args.workload)
    if args.max_views:
        cams = cams[: args.max_views]
    cfg = describe(args.workload, scene, cams)
    res_id, res_name = SCORE_RESOLUTIONS[args.score_resolution]
    tile_id = TILE_SHAPES[args.tile_shape]
    if args.score_resolution != "pixel":
        cfg["resolution"] = res_name
    m = cfg["coreset_m"]
    stream = torch.cuda.Stream(device=local)
    ctx = csgs.Context(local, stream=stream)
    sid = ctx.load_scene(scene)
    # one workload over all ranks: each scores its round-robin share of the views, and one
    # all-reduce per step (MAX of s; per-scene: SUM) combines them (strong scaling)
    my_views = sharded.shard_views(len(cams), rank, world)
    if world > 1:
        cfg["parallelism"] = f"views sharded over {world} ranks, all-reduce of s per step"
        cfg["views_per_rank"] = int(len(my_views))
    else:
        cfg["parallelism"] = "single GPU"
    ctx.set_queries(sid, cams[my_views])
    rays_local = int(sum(int(c[16]) * int(c[17]) for c in cams[my_views]))
    s = torch.empty(scene.n, dtype=torch.float32, device=f"cuda:{local}")
    tuned = None
    if not args.no_autotune and not args.view_batch:
        # view batch and radix-sort grid picked by the library's autotuner (untimed)
        # 48 probe views: with 16 the step times of the candidates differed by less than the
        # run-to-run spread (picks of 8/592 and 16/296 gave 167.0 and 158.9 ms)
        tuned = ctx.autotune(sid, csgs.default_opts(tile_shape=tile_id, persist_ctas=args.persist_ctas),
                             probe_views=48)
        cfg["autotuned"] = {"view_batch": tuned["view_batch"], "sort_blocks": tuned["sort_blocks"],
                            "tile_shape": csgs.TILE_SHAPE_NAMES[tuned["tile_shape"]],
                            "persist_ctas": tuned["persist_ctas"]}
    # the shape and compositing grid the steps use (scenes loaded later, as in the end-to-end
    # run, take them explicitly)
    shape = tuned["tile_shape"] if tuned else (tile_id or csgs.TILE_16X16)
    persist = (tuned["persist_ctas"] or -1) if tuned else args.persist_ctas
    cfg["tile_shape"] = csgs.TILE_SHAPE_NAMES[shape]
    cfg["composite_launch"] = f"persistent, {persist} CTAs" if persist > 0 else "one CTA per tile"

    # pair counts of one pass (untimed; counting kernels are slower)
    ctx.score(sid, csgs.default_opts(collect_stats=1, view_batch=args.view_batch, resolution=res_id, tile_shape=shape,
                                     persist_ctas=persist), out=s)
    cnt = ctx.stats()
    # visible (view, Gaussian) fraction for the projection's algorithmic bytes (untimed,
    # four views spread over the query set)
    vis_views = sorted({int(k * len(cams) / 4) for k in range(4)})
    vis_frac = float(np.mean([float((ctx.debug_project(sid, v)[:, 0] > 0).float().mean()) for v in vis_views]))
    torch.cuda.empty_cache()
    timing = csgs.default_opts(collect_stats=2, view_batch=args.view_batch, resolution=res_id, tile_shape=shape,
                               persist_ctas=persist)

    def combine(st):
        if dist is not None:
            ctx.sync()
            sharded.combine_shards(s, st["objective_sum"], res_id, dist, ctx.scale_scores)

    def step(seed):
        ctx.score(sid, timing, out=s)
        st = ctx.stats()
        combine(st)
        ctx.sample_coreset(s, m, seed)
        return st

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = csgs.kernel_launch_count()
    comp_ms, comp_n, proj_ms, sort_ms, comp_busy = 0.0, 0, 0.0, 0.0, 0.0
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(args.steps):
        st = step(1000 + i)
        comp_ms += st["composite_ms"]
        comp_busy += st["composite_busy_ms"]
        comp_n += st["composite_launches"]
        proj_ms += st["project_ms"]
        sort_ms += st["sort_ms"]
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = csgs.kernel_launch_count() - l0
    clk = clocks.stop()
    el_ms = job_time_ms(ev0.elapsed_time(ev1), dist, torch.device("cuda", local))
    # the ranks together score the workload's rays once per step
    value = job_rate(cfg["rays_per_step"] * args.steps / world, world, el_ms)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        host = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
                for a in (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh)]
        h2d = sum(h.numel() * 4 for h in host) + len(my_views) * 80
        s_host = torch.empty(scene.n, dtype=torch.float32).pin_memory()
        idx_host = torch.empty(m, dtype=torch.int32).pin_memory()
        w_host = torch.empty(m, dtype=torch.float32).pin_memory()

        def load():
            # asynchronous load from pinned memory: the upload runs on the copy engine while
            # the previous step scores (its validation happens at the scene's first use)
            return ctx.load_scene_ptrs(scene.n, scene.sh_degree, [h.data_ptr() for h in host], is_device=False,
                                       asynchronous=True)

        def e2e_run(steps, seed0):
            """`steps` steps, each one scene upload (issued one step ahead), queries, score,
            coreset draw and read-back of s, idx and w.  Returns the D2H bytes of a step."""
            d2h = 0
            nxt = load()
            for i in range(steps):
                cur = nxt
                nxt = load() if i + 1 < steps else None
                ctx.set_queries(cur, cams[my_views])
                s2, _ = ctx.score(cur, csgs.default_opts(resolution=res_id, tile_shape=shape, persist_ctas=persist),
                                  out=s)
                combine(ctx.stats())
                idx, w = ctx.sample_coreset(s2, m, seed0 + i)
                with torch.cuda.stream(stream):
                    s_host.copy_(s2, non_blocking=True)
                    idx_host[: idx.numel()].copy_(idx, non_blocking=True)
                    w_host[: w.numel()].copy_(w, non_blocking=True)
                stream.synchronize()
                ctx.free_scene(cur)
                d2h = s_host.numel() * 4 + 8 * idx.numel()
            return d2h

        e2e_run(2, 0)  # warm-up: two scenes' buffers for the context to reuse
        torch.cuda.synchronize()
        # at least 10 steps, so that the first step's exposed upload (the pipeline fill) weighs
        # as in a longer run; at most 20 to bound the run time
        ne = min(max(args.steps, 10), 20)
        t0 = time.perf_counter()
        d2h = e2e_run(ne, 2000)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te = job_time_ms(te * 1e3, dist, torch.device("cuda", local)) / 1e3
        e2e = {"value": cfg["rays_per_step"] * ne / te, "unit": "rays/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": ne,
               "note": "each step's scene upload is issued one step ahead (csgs_load_scene_async) and overlaps "
                       "the previous step's scoring; all uploads are inside the timed region"}

    # ---- roofline of the dominant kernel (compositing + sensitivity reduction)
    pairs_step = cnt["pairs_evaluated"] + cnt["pairs_evaluated2"]
    ess_step = (OPS_TEST * cnt["pairs_evaluated"] + OPS_HIT1 * cnt["pairs_hit"] + OPS_TEST * cnt["pairs_evaluated2"]
                + OPS_HIT2 * cnt["pairs_hit2"])
    launches_step = max(cnt["composite_launches"], 1)
    ops_launch = OPS_PER_PAIR * pairs_step / launches_step
    avg_launch_s = comp_ms / max(comp_n, 1) / 1e3
    achieved_launch = ops_launch / avg_launch_s / 1e12 if avg_launch_s > 0 else None
    # consecutive views composite concurrently on two streams, so a launch's own event span
    # also counts the time the GPU spent on the other stream's launch: the kernel's
    # throughput is the step's compositing work over the union of its launches' spans
    busy_s = comp_busy / args.steps / 1e3
    achieved = OPS_PER_PAIR * pairs_step / busy_s / 1e12 if busy_s > 0 else None
    ess_achieved = ess_step / busy_s / 1e12 if busy_s > 0 else None
    peak = SMS * FP32_LANES * 2032e6 / 1e12
    traffic, stale = traffic_per_launch()
    roof = {"bound": "alu", "kernel": f"k_composite<score, {args.score_resolution}>", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "peak_source": "148 SMs x 128 FP32 lanes x 2032 MHz (max SM clock); one FP32-pipe op per lane per "
                           "clock; 18 FP32 instructions per evaluated (ray, Gaussian) pair and pass",
            "measure": "achieved = ops of the step's compositing launches / the union of their CUDA-event spans "
                       "(launches of two streams overlap); per launch: ops per launch / mean span",
            "ops_per_launch": ops_launch, "avg_launch_ms": avg_launch_s * 1e3,
            "achieved_per_launch": achieved_launch,
            "frac_per_launch": (achieved_launch / peak) if achieved_launch else None,
            "essential_ops_frac": (ess_achieved / peak) if ess_achieved else None,
            "busy_ms_per_step": busy_s * 1e3,
            "pairs_per_ray": (cnt["pairs_evaluated"] / rays_local),
            "pairs_per_ray_pass2": (cnt["pairs_evaluated2"] / rays_local),
            "contributing_pairs_per_ray": (cnt["pairs_hit"] / rays_local),
            "staged_fraction": [cnt["entries_staged"] / max(cnt["instances"], 1),
                                cnt["entries_staged2"] / max(cnt["instances"], 1)],
            # evaluated pairs over the lanes of the warps' list iterations (pass 1, pass 2)
            "lane_utilization": [cnt["pairs_evaluated"] / max(32 * cnt["warp_entries"], 1),
                                 cnt["pairs_evaluated2"] / max(32 * cnt["warp_entries2"], 1)],
            "share_of_step": comp_ms / max(el_ms, 1e-9)}
    if stale:
        roof["traffic_note"] = "ncu counters predate the current kernel source"
    # HBM phases: algorithmic bytes per launch / the launch's mean CUDA-event duration
    hbm_peak = peaks().get("hbm_gbs")
    nbatch = max(1, cnt["view_batches"])
    nvg = scene.n * len(my_views)  # (view, Gaussian) pairs per step on this rank
    proj_bytes = (PROJ_READ_PER_G[scene.sh_degree] * scene.n * nbatch + PROJ_WRITE_PER_VG * nvg
                  + PROJ_WRITE_PER_VIS * vis_frac * nvg)
    sort_bytes = SORT_PER_VG * nvg + SORT_PER_INST * cnt["instances"]
    for key, nbytes, ms, nl in (("project", proj_bytes, proj_ms, nbatch), ("sort", sort_bytes, sort_ms, len(my_views))):
        per_launch_s = ms / args.steps / nl / 1e3
        ach = nbytes / nl / per_launch_s / 1e9 if per_launch_s > 0 else None
        roof[key] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                     "frac": (ach / hbm_peak) if (ach and hbm_peak) else None,
                     "bytes_per_launch": nbytes / nl, "avg_launch_ms": per_launch_s * 1e3,
                     "launches_per_step": nl, "traffic": None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, read + write)"}
    roof["project"]["visible_fraction"] = vis_frac
    roof["project"]["note"] = "one launch projects one view batch"
    roof["sort"]["note"] = ("one launch = the binning chain of one view (depth sort, emit, tile sort, ranges); "
                            "chains of four views overlap each other and the compositing")

    line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg, "roofline": roof,
            "gpu_launches": int(launches),
            "phases_ms_per_step": {"project": proj_ms / args.steps, "sort_and_bin": sort_ms / args.steps,
                                   "composite_score": comp_ms / args.steps},
            "clocks": clk, "e2e": e2e}
    if world == 1 and not args.no_surrogate_record and not args.max_views:
        # the metric's second half: surrogate-assisted vs exact scoring of this workload
        from paper_2607_02721_b300 import surrogate

        scfg = surrogate.SurrogateConfig(residual=not args.surrogate_direct)
        rec, _, _ = surrogate_record(ctx, sid, cams, m, scfg, csgs.default_opts(resolution=res_id), 10)
        line["surrogate"] = rec
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, _, _ = cpu_baseline(args.workload, scene, cams, args.cpu_seconds)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def surrogate_record(ctx, sid, cams, m, cfg, sopts, psnr_stride: int):
    """Surrogate-assisted against exact scoring of the same query set on the same GPU:
    times (CUDA events on the library's stream, after one warm-up each) and PSNR of the
    90%-pruned weighted coreset against the full render on every `psnr_stride`-th view,
    for the exact scores, the surrogate's and the scored subset's alone."""
    import numpy as np
    import torch

    from paper_2607_02721_b300 import surrogate

    ctx.set_queries(sid, cams)
    ctx.score(sid, sopts)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(ctx.stream)
    s_exact, _ = ctx.score(sid, sopts)
    ev1.record(ctx.stream)
    torch.cuda.synchronize()
    exact_ms = ev0.elapsed_time(ev1)
    s_exact = s_exact.clone()
    surrogate.surrogate_scores(ctx, sid, cams, cfg, opts=sopts)  # warm-up
    tim = {}
    s_hat, s_sub = surrogate.surrogate_scores(ctx, sid, cams, cfg, opts=sopts, timings=tim)
    views = list(range(0, len(cams), psnr_stride))
    res = {"exact_ms": exact_ms, "surrogate_ms": tim["total_ms"], "speedup": exact_ms / tim["total_ms"],
           "phases_ms": tim, "train_views": cfg.train_views, "train_steps": cfg.steps, "train_batch": cfg.batch,
           "lowres_factor": cfg.lowres_factor, "cheap_stride": cfg.cheap_stride, "train_lr": cfg.lr,
           "fill_only": cfg.fill_only, "aug_views": list(cfg.aug_views), "residual": cfg.residual,
           "psnr_views": len(views), "prune_ratio": 0.9}
    # the same inputs without the network: the cheap score scaled to the exact scores by
    # the median ratio on the scored views, maximum with the scored subset's exact scores
    s_nonet = None
    if cfg.lowres_factor > 0:
        low = surrogate.lowres_cameras(cams, cfg.lowres_factor)
        sub = surrogate.view_subset(len(cams), cfg.train_views)
        s_low = surrogate._score_or_zero(ctx, sid, low[::max(1, cfg.cheap_stride)], sopts)
        s_low_sub = surrogate._score_or_zero(ctx, sid, low[sub], sopts).double().cpu().numpy()
        b = s_sub.double().cpu().numpy()
        ok = (b > 0) & (s_low_sub > 0)
        ratio = float(np.median(b[ok] / s_low_sub[ok])) if ok.any() else 1.0
        s_nonet = torch.maximum(s_sub, s_low * ratio)
        ctx.set_queries(sid, cams)
    for name, sv in (("exact", s_exact), ("surrogate", s_hat), ("subset_only", s_sub), ("no_network", s_nonet)):
        if sv is not None:
            res["psnr_" + name] = surrogate.pruned_psnr(ctx, sid, cams, sv, m, 0, views)
    res["delta_psnr_surrogate_vs_exact"] = res["psnr_surrogate"] - res["psnr_exact"]
    res["gain_psnr_surrogate_vs_subset"] = res["psnr_surrogate"] - res["psnr_subset_only"]
    sh, se = s_hat.double().cpu().numpy(), s_exact.double().cpu().numpy()
    pos = se > 0
    res["spearman_vs_exact"] = float(np.corrcoef(np.argsort(np.argsort(sh[pos])),
                                                 np.argsort(np.argsort(se[pos])))[0, 1])
    res["meets_target"] = bool(res["delta_psnr_surrogate_vs_exact"] >= -0.1 and res["speedup"] > 1.0)
    return res, s_exact, s_hat


def run_surrogate(args):
    """Surrogate-assisted scoring vs exact scoring on the same workload: times, and PSNR
    of the 90%-pruned weighted coreset against the full render (views every `stride`)."""
    import numpy as np
    import torch

    import paper_2607_02721_b300 as csgs
    from paper_2607_02721_b300 import build, surrogate

    build.build()
    scene, cams = workload(args.workload)
    if args.max_views:
        cams = cams[: args.max_views]
    cfg = describe(args.workload, scene, cams)
    m = cfg["coreset_m"]
    ctx = csgs.Context(0, stream=torch.cuda.Stream())
    sid = ctx.load_scene(scene)
    ctx.set_queries(sid, cams)
    res_id = {"pixel": csgs.RES_PIXEL, "scene": csgs.RES_SCENE}[args.resolution]
    sopts = csgs.default_opts(resolution=res_id)
    scfg = surrogate.SurrogateConfig(train_views=args.train_views, steps=args.train_steps, fill_only=args.fill_only,
                                     aug_views=tuple(int(x) for x in args.aug_views.split(",") if x),
                                     lowres_factor=args.lowres_factor, residual=not args.surrogate_direct)
    if args.train_batch:
        scfg.batch = args.train_batch
    if args.train_lr:
        scfg.lr = args.train_lr
    if args.cheap_stride:
        scfg.cheap_stride = args.cheap_stride
    rec, s_exact, s_hat = surrogate_record(ctx, sid, cams, m, scfg, sopts, args.psnr_stride)
    res = {"mode": "surrogate", "config": cfg, "resolution": args.resolution}
    res.update(rec)
    # tensor-core roofline of the network's forward over every Gaussian (inference GEMMs)
    ctx.set_queries(sid, cams)
    X = ctx.features(sid, ctx.view_stats(sid, sopts))
    for _ in range(3):
        ctx.mlp_forward(X)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    reps = 10
    for _ in range(reps):
        ctx.mlp_forward(X)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * (64 * 256 + 256 * 256 + 256) * X.shape[0]
    pk = peaks()
    bf16 = pk.get("bf16_tflops") if pk else None
    res["mlp_forward"] = {"rows": int(X.shape[0]), "ms": fwd_ms, "tflops": flops / fwd_ms / 1e9,
                          "peak_tflops": bf16, "frac": (flops / fwd_ms / 1e9 / bf16) if bf16 else None,
                          "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)" if bf16 else None}
    print(json.dumps(res), flush=True)
    ctx.close()
    return 0


def run_batch(args):
    """Six scenes of uneven size scored in one submission: autotuned view batch and sort
    grid per scene, the whole batch captured once as a CUDA graph and replayed each step;
    beside it the same work as one csgs_score call per scene."""
    import torch

    import paper_2607_02721_b300 as csgs
    from paper_2607_02721_b300 import build, synth

    build.build()
    work = synth.workload_batch6()
    stream = torch.cuda.Stream()
    ctx = csgs.Context(0, stream=stream)
    sids = []
    for sc, cams in work:
        sid = ctx.load_scene(sc)
        ctx.set_queries(sid, cams)
        sids.append(sid)
    rays = sum(int(c[16]) * int(c[17]) for _, cams in work for c in cams)
    opts = csgs.default_opts()
    tuned = []
    if not args.no_autotune:
        for sid in sids:
            tuned.append(ctx.autotune(sid, opts, probe_views=8))
    outs = [torch.empty(sc.n, dtype=torch.float32, device="cuda") for sc, _ in work]

    def timed(fn, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps

    def graph_step():
        ctx.score_batch(sids, opts, outs=outs, use_graph=True)

    def per_scene_step():
        for sid, o in zip(sids, outs):
            ctx.score(sid, opts, out=o)

    for _ in range(args.warmup):
        graph_step()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    l0 = csgs.kernel_launch_count()
    ms_graph = timed(graph_step, args.steps)
    launches_host = csgs.kernel_launch_count() - l0
    graph_kernels = ctx.stats()["kernel_launches"]
    ms_eager = timed(per_scene_step, args.steps)
    clk = clocks.stop()
    line = {"mode": "batch", "metric": "sensitivity rays/sec, six scenes in one graph", "unit": "rays/s",
            "value": rays / (ms_graph / 1e3), "ms_per_step": ms_graph, "steps": args.steps, "warmup": args.warmup,
            "per_scene_calls_value": rays / (ms_eager / 1e3), "per_scene_calls_ms": ms_eager,
            "graph_kernels_per_step": graph_kernels, "host_launches_in_timed_graph_steps": launches_host,
            "autotuned": [{"n": sc.n, "view_batch": t["view_batch"], "sort_blocks": t["sort_blocks"],
                           "tile_shape": csgs.TILE_SHAPE_NAMES[t["tile_shape"]], "persist_ctas": t["persist_ctas"]}
                          for (sc, _), t in zip(work, tuned)],
            "config": {"workload": "batch6", "scenes": [{"n": n, "views": v, "width": W, "height": H}
                                                         for n, v, W, H in synth.BATCH6],
                       "rays_per_step": rays},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _ssim(img, ref):
    """SSIM (Wang et al. 2004): 11x11 Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2
    for values in [0, 1], mean over pixels and channels.  img, ref: [H, W, 3] device."""
    import torch

    x = img.permute(2, 0, 1).unsqueeze(0).clamp(0, 1)
    y = ref.permute(2, 0, 1).unsqueeze(0).clamp(0, 1)
    g = torch.arange(11, dtype=torch.float32, device=img.device) - 5.0
    g = torch.exp(-(g * g) / (2 * 1.5 ** 2))
    g = g / g.sum()
    k = (g[:, None] * g[None, :]).expand(3, 1, 11, 11).contiguous()
    conv = lambda t: torch.nn.functional.conv2d(t, k, groups=3)
    mx, my = conv(x), conv(y)
    sxx, syy, sxy = conv(x * x) - mx * mx, conv(y * y) - my * my, conv(x * y) - mx * my
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(s.mean())


def _quality(ctx, sid, cams, targets, idx, w, views):
    """Mean PSNR and SSIM over `views` of the weighted render against the targets."""
    ps, ss = [], []
    for v in views:
        H, W = int(cams[v][17]), int(cams[v][16])
        img = ctx.render(sid, v, idx=idx, w=w, H=H, W=W)
        mse = float(((img - targets[v]) ** 2).mean())
        ps.append(10.0 * math.log10(1.0 / max(mse, 1e-20)))
        ss.append(_ssim(img, targets[v]))
    return sum(ps) / len(ps), sum(ss) / len(ss)


def run_finetune(args):
    """Short post-prune recovery (Sec. 4): for each prune ratio r, a weighted coreset of
    m = (1 - r) N draws by sensitivity and, as the baseline, uniformly is fitted by Adam
    to the full scene's renders of the first `--ft-views` views; PSNR and SSIM (20 of the
    views) before recovery and at each checkpoint, ms per step."""
    import numpy as np
    import torch

    import paper_2607_02721_b300 as csgs
    from paper_2607_02721_b300 import build, finetune

    build.build()
    scene, cams = workload(args.workload)
    cams = cams[: args.ft_views]
    n = scene.n
    ratios = [float(x) for x in args.ratios.split(",") if x]
    checkpoints = sorted({int(x) for x in args.ft_checkpoints.split(",") if x} | {args.ft_steps})
    checkpoints = [c for c in checkpoints if c <= args.ft_steps]
    ctx = csgs.Context(0, stream=torch.cuda.Stream())
    sid = ctx.load_scene(scene)
    ctx.set_queries(sid, cams)
    res_id = {"pixel": csgs.RES_PIXEL, "scene": csgs.RES_SCENE}[args.resolution]
    s, S = ctx.score(sid, csgs.default_opts(resolution=res_id))
    targets = []
    for v in range(len(cams)):
        H, W = int(cams[v][17]), int(cams[v][16])
        targets.append(ctx.render(sid, v, H=H, W=W).clone())
    ctx.free_scene(sid)
    out = {"mode": "finetune", "config": {"workload": args.workload, "views": len(cams), "steps": args.ft_steps,
                                          "checkpoints": checkpoints, "resolution": args.resolution,
                                          "lr": {"means": 1e-3, "sh": 1e-3, "opacity_logits": 5e-3}},
           "ratios": []}
    eval_views = list(range(0, len(cams), max(1, len(cams) // 20)))
    for r in ratios:
        m = max(1, int(round((1.0 - r) * n)))
        entry = {"prune": r, "coreset_m": m}
        for method in ("sensitivity", "uniform"):
            if method == "sensitivity":
                idx, w = ctx.sample_coreset(s, m, 0)
            else:
                pu = torch.full((n,), 1.0 / n, dtype=torch.float64, device="cuda")
                idx, w = ctx.sample_coreset_p(pu, m, 0)
            sub = scene.subset(idx.cpu().numpy())
            sid2 = ctx.load_scene(sub)
            ctx.set_queries(sid2, cams)
            params = {k: torch.tensor(getattr(sub, k), device="cuda").contiguous()
                      for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
            ar = torch.arange(sub.n, dtype=torch.int32, device="cuda")
            p0, s0 = _quality(ctx, sid2, cams, targets, ar, w, eval_views)
            curve = {"0": {"psnr": p0, "ssim": s0}}
            t_train = [0.0]
            t_mark = [time.perf_counter()]

            def cb(step):
                if step in checkpoints:
                    torch.cuda.synchronize()
                    t_train[0] += time.perf_counter() - t_mark[0]
                    ctx.update_scene(sid2, params["means"], params["log_scales"], params["quats"],
                                     params["opacity_logits"], params["sh"])
                    p, q = _quality(ctx, sid2, cams, targets, ar, w, eval_views)
                    curve[str(step)] = {"psnr": p, "ssim": q}
                    torch.cuda.synchronize()
                    t_mark[0] = time.perf_counter()

            torch.cuda.synchronize()
            t_mark[0] = time.perf_counter()
            finetune.finetune(ctx, sid2, cams, params, ar, w, targets, steps=args.ft_steps, seed=1, callback=cb)
            entry[method] = {"distinct": int(sub.n), "curve": curve,
                             "ms_per_step": t_train[0] * 1e3 / max(args.ft_steps, 1)}
            ctx.free_scene(sid2)
        out["ratios"].append(entry)
    out["eval_views"] = len(eval_views)
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def run_mlp(args):
    """Tensor-core roofline of the surrogate network alone: forward over `--mlp-rows` random
    BF16 feature rows and the training step (the surrogate's batch: forward, backward, Adam)."""
    import torch

    import paper_2607_02721_b300 as csgs
    from paper_2607_02721_b300 import build

    build.build()
    ctx = csgs.Context(0, stream=torch.cuda.Stream())
    n = args.mlp_rows
    g = torch.Generator(device="cuda").manual_seed(0)
    with torch.cuda.stream(ctx.stream):
        X = (0.5 * torch.randn(n, 64, device="cuda", generator=g)).to(torch.bfloat16)
        t = torch.randn(n, device="cuda", generator=g)
    ctx.mlp_init(0)
    flops_row = 2.0 * (64 * 256 + 256 * 256 + 256)
    for _ in range(args.warmup):
        ctx.mlp_forward(X)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(args.steps):
        ctx.mlp_forward(X)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / args.steps
    from paper_2607_02721_b300 import surrogate

    def train_step_ms(batch, steps=50):
        ctx.mlp_train(X, t, batch=batch, steps=3, lr=1e-3, seed=1)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        ctx.mlp_train(X, t, batch=batch, steps=steps, lr=1e-3, seed=2)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    pk = peaks()
    bf16 = pk.get("bf16_tflops")
    fwd_tf = flops_row * n / fwd_ms / 1e9
    # the surrogate's training batch, and four times it (the kernels' cost at a batch that
    # fills every SM several times over)
    batch = surrogate.SurrogateConfig().batch
    step_ms = train_step_ms(batch)
    train_tf = 3.0 * flops_row * batch / step_ms / 1e9  # forward + two backward GEMM sets
    big = 4 * batch
    big_ms = train_step_ms(big) if n >= big else None
    big_tf = 3.0 * flops_row * big / big_ms / 1e9 if big_ms else None
    print(json.dumps({"mode": "mlp", "rows": n, "forward_ms": fwd_ms, "forward_tflops": fwd_tf,
                      "train_batch": batch, "train_step_ms": step_ms, "train_tflops": train_tf,
                      "peak_tflops": bf16, "forward_frac": fwd_tf / bf16 if bf16 else None,
                      "train_frac": train_tf / bf16 if bf16 else None,
                      "train_batch_x4": big, "train_step_ms_x4": big_ms, "train_tflops_x4": big_tf,
                      "train_frac_x4": big_tf / bf16 if (big_tf and bf16) else None,
                      "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"}), flush=True)
    ctx.close()
    return 0


def run_diagnostics(args):
    """Theory diagnostics of one coreset (Sec. 3.3): S and |Q'|, Theorem 2's m for
    (eps_c, delta), the measured relative error of the relaxed objective A_th, the
    transmittance gap gamma, Theorem 3's eps_r at that gamma, and the validity violations
    (pairs with w alpha k >= 1), for prune ratios 0.8 / 0.9 / 0.95."""
    import numpy as np
    import torch

    import paper_2607_02721_b300 as csgs
    from paper_2607_02721_b300 import build

    build.build()
    scene, cams = workload(args.workload)
    if args.max_views:
        cams = cams[: args.max_views]
    ctx = csgs.Context(0, stream=torch.cuda.Stream())
    sid = ctx.load_scene(scene)
    ctx.set_queries(sid, cams)
    s, S = ctx.score(sid)
    q = ctx.stats()["queries"]
    out = {"mode": "diagnostics", "config": {"workload": args.workload, "views": len(cams), "n": scene.n},
           "S": S, "queries": q, "eps_c": 0.1, "delta": 0.1,
           "theorem2_m": csgs.theorem2_sample_size(S, 0.1, 0.1, q), "ratios": []}
    views = list(range(0, len(cams), max(1, len(cams) // 4)))
    for r in (0.8, 0.9, 0.95):
        m = int(round((1 - r) * scene.n))
        idx, w = ctx.sample_coreset(s, m, 0)
        rel, gam = [], []
        for v in views:
            H, W = int(cams[v][17]), int(cams[v][16])
            t = ctx.transfer(sid, v, idx, w, H, W)
            A = t[..., 0:3].sum(-1).double()
            Ath = t[..., 3:6].sum(-1).double()
            g = t[..., 9].double()
            ok = A > 1e-6
            rel.append(((Ath[ok] - A[ok]).abs() / A[ok]).cpu().numpy())
            gam.append(g[ok].cpu().numpy())
        rel, gam = np.concatenate(rel), np.concatenate(gam)
        qs = (50, 90, 99)
        rq = {f"p{q}": float(np.percentile(rel, q)) for q in qs}
        gq = {f"p{q}": float(np.percentile(gam, q)) for q in qs}
        rq["max"], gq["max"] = float(rel.max()), float(gam.max())
        ctx.render(sid, views[0], idx=idx, w=w, H=int(cams[views[0]][17]), W=int(cams[views[0]][16]),
                   opts=csgs.default_opts(collect_stats=1))
        st = ctx.stats()
        out["ratios"].append({"prune": r, "m": m, "distinct": int(idx.numel()),
                              "rel_err_A_th": rq, "gamma": gq,
                              "theorem3_eps_r_at": {k: csgs.theorem3_eps(gq[k], rq[k]) for k in ("p50", "p90")},
                              "violations_view0": st["violations"], "pairs_view0": st["pairs_evaluated"]})
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="scene_3m", choices=["scene_3m", "scene_1m", "small"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--max-views", type=int, default=0, help="score only the first views (profiling runs)")
    ap.add_argument("--view-batch", type=int, default=0, help="views projected per launch (0 = automatic)")
    ap.add_argument("--surrogate", action="store_true", help="surrogate-assisted vs exact scoring report")
    ap.add_argument("--train-views", type=int, default=20)
    ap.add_argument("--train-steps", type=int, default=100)
    ap.add_argument("--train-batch", type=int, default=0, help="surrogate training rows per step (0: default)")
    ap.add_argument("--train-lr", type=float, default=0.0, help="surrogate learning rate (0: default)")
    ap.add_argument("--cheap-stride", type=int, default=0, help="surrogate: cheap score on every n-th view (0: default)")
    ap.add_argument("--psnr-stride", type=int, default=5)
    ap.add_argument("--fill-only", action="store_true")
    ap.add_argument("--surrogate-direct", action="store_true",
                    help="surrogate network predicts log s itself, not its correction over the scaled cheap score")
    ap.add_argument("--resolution", default="pixel", choices=["pixel", "scene"])
    ap.add_argument("--aug-views", default="")
    ap.add_argument("--lowres-factor", type=int, default=4, help="surrogate: cheap score at 1/f resolution (0: off)")
    ap.add_argument("--no-surrogate-record", action="store_true",
                    help="leave the surrogate-vs-exact record out of the default line")
    ap.add_argument("--batch", action="store_true", help="six-scene graph-captured batch report")
    ap.add_argument("--finetune", action="store_true", help="post-prune recovery report (sensitivity vs uniform)")
    ap.add_argument("--ft-steps", type=int, default=500)
    ap.add_argument("--ft-views", type=int, default=100)
    ap.add_argument("--ratios", default="0.9", help="prune ratios of the recovery report")
    ap.add_argument("--ft-checkpoints", default="10,50,100,200", help="recovery steps at which to evaluate")
    ap.add_argument("--diagnostics", action="store_true", help="theory diagnostics report")
    ap.add_argument("--mlp", action="store_true", help="surrogate network tensor-core report")
    ap.add_argument("--mlp-rows", type=int, default=3_000_000)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile-shape", default="auto", choices=list(TILE_SHAPES),
                    help="compositing tile shape (auto: the autotuner's choice, 16x16 without it)")
    ap.add_argument("--persist-ctas", type=int, default=0,
                    help="persistent compositing CTAs (0: the autotuner's choice, -1: one CTA per tile)")
    ap.add_argument("--score-resolution", default="pixel", choices=list(SCORE_RESOLUTIONS),
                    help="query resolution of the timed scoring (Sec. 3.5); the headline is per-pixel")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.surrogate:
        return run_surrogate(args)
    if args.batch:
        return run_batch(args)
    if args.finetune:
        return run_finetune(args)
    if args.diagnostics:
        return run_diagnostics(args)
    if args.mlp:
        return run_mlp(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the RayGS hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one pass of the whole hot path (per-primitive vertex stage, depth + tile binning,
tile rasterisation) over the stereo-VR batch: 3M blob primitives (10% near-flat, scale ratio
> 1e3) seen by 16 views of uneven size (4 stereo pairs at 2064x2208 per eye plus 8 views of
random size in [640,1920]x[480,1080]), launched as one captured CUDA graph.  The metric is
stereo frames/s in its strict reading: complete 16-view batches per second (each batch
holds 4 stereo pairs).  Inputs (708 MB of attributes, 3 GB of per-view records) are larger
than the 129 MB L2, so no flush is needed between steps.

Printed: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on a
bounded pixel sample of the same workload instead (the only other place that runs it).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stereo frames/s + Gaussian-pixel evals/s at 3M Gaussians; fwd+bwd ms/view at 1.5M"
UNIT = "stereo frames/s (16-view batches/s)"
WORKLOAD = ("stereo-VR batch: 3M blob primitives (10% axis ratio > 1e3), 16 views "
            "(4 stereo pairs 2064x2208 per eye + 8 random 640-1920 x 480-1080), one CUDA graph")

# DRAM bytes (read + write) of one full-size rasteriser launch on the stereo batch, from an
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by tile shape and a
# digest of the rasteriser's sources: a kernel changed since the capture reports null.
# No full-size capture is held for the current sources (DRAM counters are taken on a
# smaller case, whose traffic does not scale to the full launch: the image part is fixed).
RENDER_TRAFFIC = {}
RENDER_SOURCES = ("render.cu", "raster_math.cuh", "raygs_internal.cuh")


def strip_comments(src: str) -> str:
    """C/C++ source without comments and trailing blanks, so that a comment edit does not
    count as a kernel change."""
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def render_source_digest(texts=None):
    """Digest of the rasteriser's sources (comments ignored); `texts` overrides the files."""
    import hashlib
    h = hashlib.sha256()
    for i, f in enumerate(RENDER_SOURCES):
        if texts is not None:
            src = texts[i]
        else:
            with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2503_18682_gb300", "csrc",
                                   f)) as fh:
                src = fh.read()
        h.update(strip_comments(src).encode())
    return h.hexdigest()[:16]


# algorithmic FP32 flops of the rasteriser (FMA = 2), the per-unit figures of the scope
# table's measurement plan: 22 per evaluated (pixel, primitive) pair (the support test's
# reject path: about 9 FMA and 4 other FP32 operations) and 10 more per composited pair
FLOP_EVAL = 22
FLOP_COMP = 10


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


class ClockSampler:
    """nvidia-smi clock/throttle sampling (every 20 ms) around the timed region: started
    before the warm-up, so that it is running when the timed region begins; mark() brackets
    the timed region and summary() keeps the samples taken inside it (all of them if none
    fall inside)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")

    def __init__(self, index=0, path=None):
        import tempfile
        self.index = index
        self.proc = None
        self.window = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"raygs_clocks_{os.getpid()}.csv")

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                t = datetime.datetime.strptime(f[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                try:
                    pw = float(f[3])
                except ValueError:
                    pw = float("nan")
                rows.append((t, float(f[1]), float(f[2]), f[5:9], pw))
            except ValueError:
                continue
        inside = [r for r in rows if self.window and self.window[0] <= r[0] <= self.window[1]]
        use = inside or rows
        if not use:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        reasons = {n for r in use for n, v in zip(names, r[3]) if v.lower().startswith("active")}
        pw = [r[4] for r in use if r[4] == r[4]]
        return dict(sm_mhz=statistics.median(r[1] for r in use), sm_max_mhz=max(r[2] for r in use),
                    reasons=sorted(reasons), samples=len(use), samples_in_timed_region=len(inside),
                    power_w=statistics.median(pw) if pw else None)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------- reference arm

def cpu_oracle_sample(scene, cams, n_pixels=96, seed=11, threads=0):
    """Time the FP64 oracle on a bounded sample: per view, the per-primitive setup (one call
    with a single pixel) plus `n_pixels` sampled pixels of view 0; extrapolate to seconds per
    16-view batch.  Returns (seconds_per_batch, cores, description)."""
    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    cam = cams[0]
    W, H = cam["width"], cam["height"]
    idx = rng.choice(W * H, n_pixels, replace=False)
    pix = np.stack([idx % W, idx // W], axis=1).astype(np.int32)
    t0 = time.perf_counter()
    oracle.render(scene, cam, pixels=pix[:1], threads=threads)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.render(scene, cam, pixels=pix, threads=threads)
    t_all = time.perf_counter() - t0
    t_pix = max(t_all - t_setup, 1e-9) / n_pixels
    P = sum(c["width"] * c["height"] for c in cams)
    per_batch = len(cams) * t_setup + P * t_pix
    desc = (f"FP64 oracle, {n_pixels} sampled pixels of view 0 against all {scene['means'].shape[0]} "
            f"primitives plus one per-view setup; extrapolated to {len(cams)} views / {P} pixels")
    cpu_oracle_sample.last_t_pix = t_pix
    return per_batch, cores, desc, t_setup + t_all


def cpu_oracle_configs(threads=0):
    """The FP64 oracle on bounded samples of the other workloads (a baseline, not a target):
    the 64x64 workload at full frame; the 720p MIP and forward+backward workloads and the
    precision workload (its 3840x2160 view 0) on sampled pixels, each against all the
    primitives.  Per workload: (pixel, primitive) pairs per second, counting every pixel
    against every primitive (a pixel's loop ends at its transmittance stop, so dense views
    run faster per pair; the per-view setup apart), and the extrapolated seconds per frame,
    with the cores used."""
    from paper_2503_18682_gb300 import scenes
    cores = os.cpu_count() or 1
    out = {}
    plans = [("64x64_1k_full_frame", scenes.workload_small, None),
             ("720p_mip_500k", scenes.workload_mip_720p, 256),
             ("720p_fwd_bwd_1.5m", scenes.workload_backward_720p, 256),
             ("precision_6m_4k_view0", scenes.workload_precision, 64)]
    for name, make, n_pix in plans:
        scene, cams = make()
        cam = cams[0]
        W, H = cam["width"], cam["height"]
        n = int(scene["means"].shape[0])
        per_frame, _, desc, _ = cpu_oracle_sample(scene, [cam], n_pixels=n_pix or W * H, threads=threads)
        out[name] = dict(seconds_per_frame=per_frame, pixel_primitive_pairs_per_s=n / cpu_oracle_sample.last_t_pix,
                         sample=desc, cores=cores)
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2503_18682_gb300 import scenes
    scene, cams = scenes.workload_stereo_batch()
    times = []
    cores = 1
    desc = ""
    for _ in range(args.warmup):
        cpu_oracle_sample(scene, cams, n_pixels=8)
    for _ in range(args.steps):
        per_batch, cores, desc, wall = cpu_oracle_sample(scene, cams, n_pixels=args.ref_pixels)
        times.append(per_batch)
    spb = statistics.median(times)
    value = 1.0 / spb
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=spb * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, n_gaussians=int(scene["means"].shape[0]), views=len(cams)),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle", sample=desc),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- our arm

def run_ours(args, world, rank, local):
    import torch
    from paper_2503_18682_gb300 import build, raygs, scenes
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pk = peaks()

    if args.mode == "profile" and args.workload == "backward":
        return profile_backward(args, rank, dev)
    if args.workload in ("mip720", "mip720exact"):
        scene, cams = scenes.workload_mip_720p()
        if args.workload == "mip720exact":
            cams = [dict(c, mip="exact") for c in cams]
    else:
        scene, cams = scenes.workload_stereo_batch(n=args.n)
    n = int(scene["means"].shape[0])
    st = raygs.scene_to_device(scene, dev)
    tile_kw = {}
    if args.tile:
        tw, th = (int(x) for x in args.tile.lower().split("x"))
        tile_kw = dict(tile_w=tw, tile_h=th)
    r = raygs.Renderer(cams, n, device=dev, **(tile_kw if args.mode == "profile" else {}))
    if args.mode == "profile":
        # for ncu: size the plan once, then W + K direct pipeline passes, nothing else
        stream = torch.cuda.current_stream()
        rgb, T, nc = r.alloc_outputs()
        r.forward(st, rgb, T, nc)
        sc = raygs.make_scene(st)
        for i in range(args.warmup + args.steps):
            last = i == args.warmup + args.steps - 1
            if last:
                torch.cuda.nvtx.range_push("pass")  # the last pass, for ncu --nvtx-include pass/
            raygs.raygs_preprocess(r.plan, sc)
            raygs.raygs_bin_sort(r.plan)
            raygs.raygs_render(r.plan, rgb, T, nc)
            if last:
                torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps(dict(mode="profile", workload=args.workload, passes=args.warmup + args.steps,
                                  counters=r.last_counters)), flush=True)
        return
    # autotune the tile shape on this workload (untimed), then plan for the winner
    rgb0, T0, nc0 = r.alloc_outputs()
    r.forward(st, rgb0, T0, nc0)
    tune_cap = int(min(3.2 * r.last_counters["n_instances"] + 65536, (1 << 32) - 65536))
    del r, rgb0, T0, nc0
    torch.cuda.empty_cache()
    tuned = {}
    if not args.no_autotune:
        kw, tuned = raygs.autotune(cams, st, tune_cap, device=dev, iters=2)
        torch.cuda.empty_cache()
    else:
        kw = {}
    r = raygs.Renderer(cams, n, device=dev, capacity=tune_cap, **{k: v for k, v in kw.items()
                                                                  if k in ("tile_w", "tile_h", "batch_records")})
    stream = torch.cuda.Stream(device=dev)
    stream.wait_stream(torch.cuda.current_stream())
    rgb, T, nc = r.alloc_outputs()
    with torch.cuda.stream(stream):
        r.forward(st, rgb, T, nc, stream=stream)            # sizes the instance capacity
        ctr = dict(r.last_counters)
        # headroom for pose changes, then a fresh plan at the final capacity
        r.capacity = int(min(ctr["n_instances"] * 1.10 + 65536, (1 << 32) - 4096))
        r._make_plan()
        sc = raygs.make_scene(st)
        r.forward(st, rgb, T, nc, stream=stream)
        ctr = dict(r.last_counters)
        rstat = r.counted_render_stats(rgb, T, nc, stream=stream)
        evals, comps = rstat["evaluated"], rstat["composited"]
        raygs.raygs_graph_capture(r.plan, sc, rgb, T, nc, stream)
    stream.synchronize()

    def timed(fn, k):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(k):
                fn()
            ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / k

    # per-stage breakdown (untimed w.r.t. the headline): events on the launching stream
    def stage_times(k=5):
        out = {}
        with torch.cuda.stream(stream):
            raygs.raygs_preprocess(r.plan, sc, stream)
            raygs.raygs_bin_sort(r.plan, stream)
        out["preprocess_ms"] = timed(lambda: raygs.raygs_preprocess(r.plan, sc, stream), k)
        out["bin_sort_ms"] = timed(lambda: raygs.raygs_bin_sort(r.plan, stream), k)
        out["render_ms"] = timed(lambda: raygs.raygs_render(r.plan, rgb, T, nc, stream), k)
        return out

    stages = stage_times()

    # Batches in flight: further plans (own workspace and outputs) captured on their own
    # streams, so that one batch's rasteriser overlaps the next batch's vertex stage and
    # binning.  Every step is still one complete 16-view batch.
    plans = [(r, stream)]
    plan_outputs = []  # the captured graphs write these: alive as long as their plans
    for _ in range(max(1, args.in_flight) - 1):
        r2 = raygs.Renderer(cams, n, device=dev, capacity=r.capacity, tile_w=r.cfg.tile_w, tile_h=r.cfg.tile_h,
                            batch_records=r.cfg.batch_records)
        s2 = torch.cuda.Stream(device=dev)
        s2.wait_stream(torch.cuda.current_stream())
        o2 = r2.alloc_outputs()
        with torch.cuda.stream(s2):
            r2.forward(st, *o2, stream=s2)
            raygs.raygs_graph_capture(r2.plan, sc, *o2, s2)
        s2.synchronize()
        plans.append((r2, s2))
        plan_outputs.append(o2)
        r2 = o2 = None

    def headline(nplans, steps):
        """Time `steps` graph launches spread round-robin over the first `nplans` plans."""
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _, sp in plans[1:nplans]:
            sp.wait_event(ev0)
        for i in range(steps):
            rp, sp = plans[i % nplans]
            raygs.raygs_graph_launch(rp.plan, sp)
        for _, sp in plans[1:nplans]:
            stream.wait_stream(sp)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    # the clock sampler starts here, so that nvidia-smi is sampling when the timed region
    # begins; it keeps its samples inside the timed region
    with ClockSampler(local, args.clocks_csv) as clk:
        # one batch at a time (context)
        headline(1, args.warmup)
        single_ms = max_over_ranks(headline(1, args.steps) / args.steps, world)
        # headline: W warm-up steps, K timed, barrier + sync on both sides
        headline(len(plans), args.warmup)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        t_start = time.time()
        elapsed = headline(len(plans), args.steps)
        torch.cuda.synchronize()
        clk.mark(t_start, time.time())
        barrier(world)
    ms = elapsed / args.steps
    ms_max = max_over_ranks(ms, world)
    clocks = clk.summary()
    batches = args.steps * world
    value = batches / (ms_max * args.steps / 1e3)

    # e2e through the C ABI with host buffers: pinned H2D of the attributes, graph, D2H image
    host = {k: v.to("cpu").pin_memory() for k, v in st.items() if hasattr(v, "to")}
    rgb_host = torch.empty(rgb.shape, dtype=rgb.dtype, pin_memory=True)
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = rgb.numel() * rgb.element_size()

    def e2e_step():
        for k, v in host.items():
            st[k].copy_(v, non_blocking=True)
        raygs.raygs_graph_launch(r.plan, stream)
        rgb_host.copy_(rgb, non_blocking=True)

    with torch.cuda.stream(stream):
        for _ in range(2):
            e2e_step()
    stream.synchronize()
    e2e_single_ms = max_over_ranks(timed(e2e_step, max(2, min(args.steps, 10))), world)
    e2e_ms = e2e_single_ms
    e2e_clocks = None
    e2e_reps = []
    if len(plans) >= 2:
        # three measurements, the median reported (the host's copies vary from run to run);
        # clocks during them too (they follow the headline at full load)
        with ClockSampler(local) as eclk:
            t0 = time.time()
            for _ in range(3):
                e2e_reps.append(max_over_ranks(e2e_pipelined(plans, plan_outputs, st, rgb, host, args.steps, dev),
                                               world))
            eclk.mark(t0, time.time())
        e2e_clocks = eclk.summary()
        e2e_ms = statistics.median(e2e_reps)

    # roofline of the dominant kernel (the rasteriser: plain FP32 ALU work)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    flops = FLOP_EVAL * evals + FLOP_COMP * comps
    peak_tf = sms * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
    ach_tf = flops / (stages["render_ms"] * 1e-3) / 1e12
    # HBM view of the vertex stage: attributes read once; per visible pair the 64-B record,
    # 8-B tile rectangle, 1-B tile-row count and 32-B support sector written; the 4-B key of
    # every pair
    attr_bytes = sum(v.numel() * v.element_size() for v in st.values() if hasattr(v, "numel"))
    prep_bytes = attr_bytes + 4 * n * len(cams) + 105 * ctr["n_visible"]
    bin_bytes = binning_bytes(ctr, n * len(cams))
    # kernels per pass: preprocess (2), depth sort (4 passes x 5), row-count scan (3),
    # row spans (1), tile-row scan (1), tile-row sort (passes x 5), chunk scan + chunk
    # counts + instance lists (3), rasteriser (1)
    trows = sum(-(-c["height"] // r.cfg.tile_h) for c in cams)
    row_passes = (max(1, (trows - 1).bit_length()) + 7) // 8
    gpu_launches = args.steps * (2 + 20 + 3 + 1 + 1 + 5 * row_passes + 3 + 1)

    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms_max, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic",
        config=dict(workload=WORKLOAD, n_gaussians=n, views=len(cams), pixels=r.num_pixels,
                    tiles=r.num_tiles, tile=f"{r.cfg.tile_w}x{r.cfg.tile_h}", batch_records=int(r.cfg.batch_records),
                    batches_in_flight=len(plans),
                    l2="inputs larger than L2 (no flush)", parallelism=f"replica x{world}"),
        stereo_pairs_per_s=4 * value,
        one_batch_at_a_time=dict(value=world / (single_ms / 1e3), ms_per_step=single_ms),
        gaussian_pixel_evals_per_s=evals / (stages["render_ms"] * 1e-3),
        composited_pairs_per_s=comps / (stages["render_ms"] * 1e-3),
        evaluated_pairs=evals, composited_pairs=comps,
        n_visible=ctr["n_visible"], n_instances=ctr["n_instances"],
        raster_work=dict(consumed_instances=rstat["consumed"],
                         consumed_frac=rstat["consumed"] / max(1, ctr["n_instances"]),
                         thread_record_iterations=rstat["iterations"],
                         live_pixels_per_iteration=evals / max(1, rstat["iterations"]),
                         composited_per_evaluated=comps / max(1, evals)),
        stages=dict(stages, preprocess_hbm_gbs=prep_bytes / (stages["preprocess_ms"] * 1e-3) / 1e9,
                    preprocess_hbm_frac=prep_bytes / (stages["preprocess_ms"] * 1e-3) / 1e9 / pk["hbm_gbs"],
                    bin_sort_bytes=bin_bytes,
                    bin_sort_hbm_gbs=bin_bytes / (stages["bin_sort_ms"] * 1e-3) / 1e9,
                    bin_sort_hbm_frac=bin_bytes / (stages["bin_sort_ms"] * 1e-3) / 1e9 / pk["hbm_gbs"]),
        autotune=tuned,
        roofline=dict(bound="alu", kernel=f"render_kernel<{r.cfg.tile_w},{r.cfg.tile_h}>", achieved=ach_tf, peak=peak_tf,
                      unit="TFLOP/s", frac=ach_tf / peak_tf,
                      traffic=RENDER_TRAFFIC.get((f"{r.cfg.tile_w}x{r.cfg.tile_h}/b{r.cfg.batch_records}",
                                                  render_source_digest())),
                      peak_note=f"FP32 {sms} SMs x 128 lanes x 2 flop x {pk['sm_max_mhz']:.0f} MHz (derived)",
                      algorithmic=f"{FLOP_EVAL} flop per evaluated pair + {FLOP_COMP} per composited pair",
                      timing="raygs_render launches (the rasteriser alone) timed with CUDA events on the plan's "
                             "stream, mean of 5 after warm-up; pairs counted by the instrumented variant"),
        clocks=clocks,
        e2e=dict(value=1e3 / e2e_ms, unit=UNIT, h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h),
                 ms_per_step=e2e_ms, batches_in_flight=len(plans),
                 one_batch_at_a_time=dict(value=1e3 / e2e_single_ms, ms_per_step=e2e_single_ms),
                 ms_per_step_each=e2e_reps or None, clocks=e2e_clocks),
        gpu_launches=int(gpu_launches),
    )
    def context(key, fn):
        """A context measurement beside the headline: a failure (say, out of memory on a
        smaller device) is recorded in its key instead of losing the line."""
        try:
            line[key] = fn()
        except Exception as ex:  # noqa: BLE001 - reported, not hidden
            line[key] = dict(error=f"{type(ex).__name__}: {str(ex)[:300]}")
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    if not args.no_backward:
        context("fwd_bwd", lambda: fwd_bwd_ms_per_view(args, dev))
    if not args.no_precision:
        del plans[1:]
        plan_outputs.clear()
        torch.cuda.empty_cache()
        context("gs_vs_raygs", lambda: dict(stereo_batch=divergence_ab(st, cams, n, r.cfg, r.capacity, dev),
                                            plain_720p=divergence_ab_720p(r.cfg, dev)))
        context("precision_storage", lambda: precision_storage(args, dev))
        context("precision_ablation", lambda: precision_ablation(args, dev))
        context("antialiasing", lambda: antialiasing(args, dev))
    if rank == 0 and not args.no_cpu_baseline:
        spb, cores, desc, _ = cpu_oracle_sample(scene, cams, n_pixels=args.ref_pixels)
        line["cpu_baseline"] = dict(value=1.0 / spb, unit=UNIT, cores=cores, kind="oracle", sample=desc)
        try:
            line["cpu_baseline"]["other_workloads"] = cpu_oracle_configs()
        except Exception as ex:  # noqa: BLE001 - reported, not hidden
            line["cpu_baseline"]["other_workloads"] = dict(error=f"{type(ex).__name__}: {str(ex)[:200]}")
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e_pipelined(plans, outs, st, rgb, host, steps, dev):
    """End to end with the plans' batches in flight: each plan (slot) gets its own device
    copy of the inputs and its own image; step i uploads the pinned host inputs into slot
    i % S's copy (upload stream), replays that slot's graph (its own stream) and reads its
    image back into pinned host memory (download stream).  A slot's next upload waits only
    until its previous graph has run (the inputs are read by the vertex stage, so they are
    free then), and its next graph waits for its upload and for the read-back of its
    previous image.  Uploads and read-backs of other steps overlap the renders on the copy
    engines; every step still carries its own copies.  Returns ms per step (events
    bracketing all streams' work).  outs: the image buffers of plans[1:]."""
    import torch
    from paper_2503_18682_gb300 import raygs
    slots = []
    for j, (r, s_) in enumerate(plans):
        if j == 0:
            sj, img = st, (rgb,)
        else:
            sj = {k: (v.clone() if hasattr(v, "clone") else v) for k, v in st.items()}
            img = outs[j - 1]
            with torch.cuda.stream(s_):
                raygs.raygs_graph_capture(r.plan, raygs.make_scene(sj), *img, s_)  # reads its own copy
            s_.synchronize()
        sl = dict(r=r, gs=s_, st=sj, rgb=img[0])
        sl["host_rgb"] = torch.empty(sl["rgb"].shape, dtype=sl["rgb"].dtype, pin_memory=True)
        sl["rendered"], sl["read"] = torch.cuda.Event(), torch.cuda.Event()
        sl["rendered"].record(torch.cuda.current_stream())
        sl["read"].record(torch.cuda.current_stream())
        slots.append(sl)
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def step(i):
        sl = slots[i % len(slots)]
        up.wait_event(sl["rendered"])  # the slot's previous graph has read its inputs
        with torch.cuda.stream(up):
            for k, v in host.items():
                sl["st"][k].copy_(v, non_blocking=True)
        ev_in = torch.cuda.Event()
        ev_in.record(up)
        sl["gs"].wait_event(ev_in)
        sl["gs"].wait_event(sl["read"])  # the previous image of this slot has been read back
        raygs.raygs_graph_launch(sl["r"].plan, sl["gs"])
        sl["rendered"].record(sl["gs"])
        down.wait_event(sl["rendered"])
        with torch.cuda.stream(down):
            sl["host_rgb"].copy_(sl["rgb"], non_blocking=True)
        sl["read"].record(down)

    for i in range(2 * len(slots)):
        step(i)
    torch.cuda.synchronize()
    k = max(2 * len(slots), min(steps, 20))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(up)
    for i in range(k):
        step(i)
    e1.record(down)
    e1.synchronize()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    # leave the other plans' graphs on the shared inputs again
    for j, (r, s_) in enumerate(plans[1:], start=1):
        with torch.cuda.stream(s_):
            raygs.raygs_graph_capture(r.plan, raygs.make_scene(st), *outs[j - 1], s_)
        s_.synchronize()
    return ms


def divergence_ab(st, cams, n, cfg, capacity, dev):
    """The stereo batch rendered with the GS divergence of Sec. 3.1 (EWA) and with RayGS's
    D_ray, on the same kernels, tile shape and scene: time of one forward batch (vertex
    stage, binning and rasteriser run back to back) of each, per-stage times, the instance
    and evaluation counts, and the GS image against the RayGS one (max-abs, mean-abs, PSNR
    for a unit range)."""
    import torch
    from paper_2503_18682_gb300 import raygs
    sc = raygs.make_scene(st)
    out, imgs = {}, {}
    for name, div in (("raygs", 0), ("gs", 1)):
        r = raygs.Renderer(cams, n, device=dev, capacity=capacity, tile_w=cfg.tile_w, tile_h=cfg.tile_h,
                           batch_records=cfg.batch_records, divergence=div)
        rgb, T, nc = r.forward(st)  # regrows the plan when GS needs more instances
        ctr = dict(r.last_counters)
        evals, comps = r.counted_render(rgb, T, nc)
        stages = [lambda: raygs.raygs_preprocess(r.plan, sc), lambda: raygs.raygs_bin_sort(r.plan),
                  lambda: raygs.raygs_render(r.plan, rgb, T, nc)]
        for _ in range(2):
            for f in stages:
                f()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        reps = 5
        acc = [0.0, 0.0, 0.0]
        for _ in range(reps):
            for i, f in enumerate(stages):
                ev[i].record()
                f()
            ev[3].record()
            ev[3].synchronize()
            for i in range(3):
                acc[i] += ev[i].elapsed_time(ev[i + 1])
        ms = [a / reps for a in acc]
        out[name] = dict(forward_ms=sum(ms), preprocess_ms=ms[0], bin_sort_ms=ms[1], render_ms=ms[2],
                         n_visible=ctr["n_visible"], n_instances=ctr["n_instances"], evaluated_pairs=evals,
                         composited_pairs=comps)
        imgs[name] = rgb.clone()
        del r, rgb, T, nc
        torch.cuda.empty_cache()
    d = (imgs["gs"] - imgs["raygs"]).double()
    mse = float((d ** 2).mean())
    out["gs_vs_raygs_image"] = dict(max_abs=float(d.abs().max()), mean_abs=float(d.abs().mean()),
                                    psnr_db=(99.0 if mse == 0 else -10 * np.log10(mse)))
    out["gs_speedup"] = out["raygs"]["forward_ms"] / out["gs"]["forward_ms"]
    return out


def divergence_ab_720p(cfg, dev):
    """divergence_ab on the 720p workload without the MIP term (500k primitives, one view
    whose primitives all lie in front of the camera, none near it)."""
    from paper_2503_18682_gb300 import raygs, scenes
    scene, cams = scenes.workload_mip_720p()
    cams = [dict(c, mip=False) for c in cams]
    n = int(scene["means"].shape[0])
    return divergence_ab(raygs.scene_to_device(scene, dev), cams, n, cfg, None, dev)


def antialiasing(args, dev):
    """The 720p MIP workload (500k primitives, 1280x720) four ways: one ray per pixel
    without the MIP term, with the paper's pixel-invariant MIP term (Eq. mip), with the
    exact pixel-dependent form it approximates (Sec. 5), and 2x2 supersampled without any
    (four sub-pixel rays, box-filter resolve; the counterpart of the paper's MSAA
    comparison).  Forward time of each, each image against the supersampled one, and the
    error of the approximation (Eq. mip against the exact form) (max-abs, PSNR)."""
    import torch
    from paper_2503_18682_gb300 import raygs, scenes
    scene, cams_mip = scenes.workload_mip_720p()
    n = int(scene["means"].shape[0])
    st = raygs.scene_to_device(scene, dev)
    sc = raygs.make_scene(st)
    plain = [dict(c, mip=False) for c in cams_mip]

    def timed_forward(cams):
        r = raygs.Renderer(cams, n, device=dev)
        rgb, T, nc = r.forward(st)
        r.capacity = int(r.last_counters["n_instances"] * 1.05 + 65536)
        r._make_plan()
        rgb, T, nc = r.forward(st)

        def fwd():
            raygs.raygs_preprocess(r.plan, sc)
            raygs.raygs_bin_sort(r.plan)
            raygs.raygs_render(r.plan, rgb, T, nc)

        for _ in range(2):
            fwd()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            fwd()
        e1.record()
        e1.synchronize()
        return r, rgb, e0.elapsed_time(e1) / 5

    _, img_plain, ms_plain = timed_forward(plain)
    _, img_mip, ms_mip = timed_forward(cams_mip)
    _, img_mipx, ms_mipx = timed_forward([dict(c, mip="exact") for c in cams_mip])
    r_ss, img_hi, ms_ss = timed_forward(raygs.supersampled_cameras(plain, 2))
    img_ss = torch.empty_like(img_plain)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    raygs.raygs_resolve_supersampled(r_ss.plan, 2, img_hi, None, img_ss)
    e1.record()
    e1.synchronize()

    def err(a, ref=None):
        ref = img_ss if ref is None else ref
        mse = float(((a - ref).double() ** 2).mean())
        return dict(max_abs=float((a - ref).abs().max()), psnr_db=(99.0 if mse == 0 else -10 * np.log10(mse)))

    return dict(workload=f"{n} blob primitives, 1280x720", one_ray_ms=ms_plain, mip_ms=ms_mip,
                mip_exact_ms=ms_mipx, supersampled_2x2_ms=ms_ss + e0.elapsed_time(e1),
                one_ray_vs_supersampled=err(img_plain), mip_vs_supersampled=err(img_mip),
                mip_exact_vs_supersampled=err(img_mipx), mip_vs_mip_exact=err(img_mip, img_mipx))


# storage forms of the precision workload: SH / log-scale / opacity dtypes
STORAGE_FORMS = {"f32": ("f32", "f32", "f32"), "f16": ("f16", "f16", "f16"), "bf16": ("bf16", "bf16", "f16"),
                 "sh_f16": ("f16", "f32", "f32")}


def _image_err(a, b):
    import torch
    d = (a - b).abs()
    mse = float(((a - b).double() ** 2).mean())
    return dict(max_abs=float(d.max()), psnr_db=(99.0 if mse == 0 else -10 * np.log10(mse)),
                frac_pixels_over_1e3=float((d.max(dim=1).values > 1e-3).double().mean()))


def precision_storage(args, dev):
    """The 6M-primitive precision workload (4 views at 3840x2160 plus the same poses at
    960x540 with the MIP filter) in four storage forms: FP32; SH, log-scales and opacity
    logits in FP16; SH and log-scales in BF16 with FP16 opacity; SH alone in FP16.  Per form:
    forward time, attribute bytes and the image error against the FP32 form on the same GPU
    (max-abs over the RGB channels, PSNR for a unit range, share of pixels over 1e-3).  All
    arithmetic is FP32 in every form."""
    import torch
    from paper_2503_18682_gb300 import raygs, scenes
    scene, cams = scenes.workload_precision()
    n = int(scene["means"].shape[0])
    out, ref = {}, None
    for form, (sh, sc_dt, op) in STORAGE_FORMS.items():
        sc_np = scene if form == "f32" else scenes.to_storage_form(scene, sh=sh, scales=sc_dt, opacity=op)
        st = raygs.scene_to_device(sc_np, dev)
        attr_bytes = sum(v.numel() * v.element_size() for v in st.values() if hasattr(v, "numel"))
        r = raygs.Renderer(cams, n, device=dev)
        rgb, T, nc = r.forward(st)
        r.capacity = int(r.last_counters["n_instances"] * 1.05 + 65536)
        r._make_plan()
        rgb, T, nc = r.forward(st)
        sc = raygs.make_scene(st)

        def fwd():
            raygs.raygs_preprocess(r.plan, sc)
            raygs.raygs_bin_sort(r.plan)
            raygs.raygs_render(r.plan, rgb, T, nc)

        for _ in range(2):
            fwd()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fwd()
        e1.record()
        e1.synchronize()
        entry = dict(dtypes=dict(sh=sh, log_scales=sc_dt, opacity_logits=op), forward_ms=e0.elapsed_time(e1) / 3,
                     attribute_bytes=int(attr_bytes))
        if ref is None:
            ref = rgb.clone()
        else:
            entry["vs_f32"] = _image_err(rgb, ref)
        out[form] = entry
        del r, st, rgb, T, nc
        torch.cuda.empty_cache()
    out["workload"] = f"{n} blob primitives, 4 views 3840x2160 + the same 4 poses at 960x540 with MIP"
    return out


def precision_ablation(args, dev):
    """Each attribute group rounded alone to FP16 or BF16 (the values its reduced storage
    would hold, rendered through the FP32 path, which gives the same image as the reduced
    storage itself: the conversion on load is exact), against the unrounded FP32 image: the
    precision workload's generator at 200k primitives, its 8 poses at a quarter of the size
    (960x540 and 240x135 with MIP)."""
    import torch
    from paper_2503_18682_gb300 import raygs, scenes
    scene = scenes.blob_scene(200_000, seed=4)
    cams = []
    for c in scenes.precision_cameras(seed=4):
        w, h = c["width"] // 4, c["height"] // 4
        cams.append(scenes.make_camera(w, h, float(c["fx"]) / 4, float(c["fy"]) / 4, R=c["R"], t=c["t"],
                                       mip=c["mip"]))
    n = int(scene["means"].shape[0])
    r = raygs.Renderer(cams, n, device=dev)

    def render(sc):
        rgb, _, _ = r.forward(raygs.scene_to_device(sc, dev))
        torch.cuda.synchronize()
        return rgb.clone()

    ref = render(scene)
    cases = {"sh_dc": dict(sh_dc=None), "sh_rest": dict(sh_rest=None), "log_scales": dict(scales=None),
             "opacity_logits": dict(opacity=None)}
    out = {}
    for name, kw in cases.items():
        for dt in ("f16", "bf16"):
            if name == "opacity_logits" and dt == "bf16":
                continue
            args_ = {k: dt for k in kw}
            out[f"{name}_{dt}"] = _image_err(render(scenes.round_attributes(scene, **args_)), ref)
    out["all_sh_f16"] = _image_err(render(scenes.round_attributes(scene, sh_dc="f16", sh_rest="f16")), ref)
    out["workload"] = f"{n} blob primitives, the 8 precision poses at 960x540 / 240x135 (MIP)"
    return out


def binning_bytes(ctr, pairs):
    """Algorithmic bytes of one binning pass (each array read or written once per use; the
    row payload as stored): depth sort (the dense 4-B keys and 1-B tile-row counts read,
    then 8 B per visible pair per pass in and out, the upsweeps' key reads),
    support rows (the 32-B support sector per pair, 12 B written per row), the tile-row
    sort (4-B key + 8-B payload read per row in the first pass, 12 B written per kept row,
    24 B per kept row in the second pass, the upsweeps' key reads), the chunk counts (the
    4-B column half of each sorted payload), and the expansion (8-B payload read per kept
    row, 4 B written per instance)."""
    nv, nr, nk, ni = (int(ctr[k]) for k in ("n_visible", "n_rows", "n_rows_kept", "n_instances"))
    depth = 5 * pairs + 8 * nv + 3 * 16 * nv + 4 * pairs + 3 * 4 * nv
    rows = 32 * nv + 12 * nr
    row_sort = 12 * nr + 12 * nk + 24 * nk + 4 * nr + 4 * nk
    ranges = 4 * nk
    expand = 8 * nk + 4 * ni
    return depth + rows + row_sort + ranges + expand


def profile_backward(args, rank, dev):
    """For ncu: the forward + backward of the 1.5M-primitive 1280x720 view, W + K passes after
    one sizing pass; the last pass inside the NVTX range "pass"."""
    import torch
    from paper_2503_18682_gb300 import raygs, scenes
    scene, cams = scenes.workload_backward_720p()
    st = raygs.scene_to_device(scene, dev)
    n = scene["means"].shape[0]
    r = raygs.Renderer(cams, n, device=dev, enable_backward=1)
    rgb, T, nc = r.forward(st)
    g_rgb = torch.ones_like(rgb)
    sc = raygs.make_scene(st)
    grads = {k: torch.empty((n, d), dtype=torch.float32, device=dev) for k, d in
             (("means", 3), ("log_scales", 3), ("quats", 4))}
    grads["opacity_logits"] = torch.empty(n, dtype=torch.float32, device=dev)
    grads["sh"] = torch.empty(st["sh"].shape, dtype=torch.float32, device=dev)
    G = raygs.Grads()
    G.d_means, G.d_log_scales, G.d_quats = (grads["means"].data_ptr(), grads["log_scales"].data_ptr(),
                                            grads["quats"].data_ptr())
    G.d_opacity_logits, G.d_sh = grads["opacity_logits"].data_ptr(), grads["sh"].data_ptr()
    for i in range(args.warmup + args.steps):
        last = i == args.warmup + args.steps - 1
        if last:
            torch.cuda.nvtx.range_push("pass")
        raygs.raygs_preprocess(r.plan, sc)
        raygs.raygs_bin_sort(r.plan)
        raygs.raygs_render(r.plan, rgb, T, nc)
        raygs.raygs_render_backward(r.plan, sc, T, nc, g_rgb, None, G)
        if last:
            torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if rank == 0:
        print(json.dumps(dict(mode="profile", workload="backward", passes=args.warmup + args.steps,
                              counters=r.last_counters)), flush=True)


def fwd_bwd_ms_per_view(args, dev):
    """Forward + backward of the 1.5M-primitive 1280x720 view (blob generator, seed 2):
    preprocess, binning, rasteriser and the full backward to all parameters, with a fixed
    upstream gradient (the sign of the image minus a uniform random target, i.e. an L1
    loss).  CUDA events on the launching stream; W warm-up and K timed passes."""
    import torch
    from paper_2503_18682_gb300 import raygs, scenes
    scene, cams = scenes.workload_backward_720p()
    st = raygs.scene_to_device(scene, dev)
    r = raygs.Renderer(cams, scene["means"].shape[0], device=dev, enable_backward=1)
    rgb, T, nc = r.forward(st)
    r.capacity = int(r.last_counters["n_instances"] * 1.1 + 65536)
    r._make_plan()
    rgb, T, nc = r.forward(st)
    target = torch.rand(rgb.shape, generator=torch.Generator(device="cpu").manual_seed(2)).to(dev)
    g_rgb = torch.sign(rgb - target).contiguous()
    sc = raygs.make_scene(st)
    n = scene["means"].shape[0]
    grads = {k: torch.empty((n, d), dtype=torch.float32, device=dev) for k, d in
             (("means", 3), ("log_scales", 3), ("quats", 4))}
    grads["opacity_logits"] = torch.empty(n, dtype=torch.float32, device=dev)
    grads["sh"] = torch.empty(st["sh"].shape, dtype=torch.float32, device=dev)
    G = raygs.Grads()
    G.d_means, G.d_log_scales, G.d_quats = (grads["means"].data_ptr(), grads["log_scales"].data_ptr(),
                                            grads["quats"].data_ptr())
    G.d_opacity_logits, G.d_sh = grads["opacity_logits"].data_ptr(), grads["sh"].data_ptr()

    def step():
        raygs.raygs_preprocess(r.plan, sc)
        raygs.raygs_bin_sort(r.plan)
        raygs.raygs_render(r.plan, rgb, T, nc)
        raygs.raygs_render_backward(r.plan, sc, T, nc, g_rgb, None, G)

    def only_fwd():
        raygs.raygs_preprocess(r.plan, sc)
        raygs.raygs_bin_sort(r.plan)
        raygs.raygs_render(r.plan, rgb, T, nc)

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    k = max(3, min(args.steps, 20))
    fb = timed(step, k)
    fw = timed(only_fwd, k)
    return dict(ms_per_view=fb, forward_ms=fw, backward_ms=fb - fw, n_gaussians=int(n),
                resolution="1280x720", n_instances=int(r.last_counters["n_instances"]),
                loss="L1 vs uniform random target (fixed upstream gradient)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=3_000_000)
    ap.add_argument("--ref-pixels", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-csv", default=None, help="keep the raw clock samples of the timed region here")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP16/BF16 storage measurement on the 6M-primitive 4K workload")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile", default="", help="profile mode: tile shape WxH (default 16x16)")
    ap.add_argument("--mode", default="bench", choices=["bench", "profile"])
    ap.add_argument("--in-flight", type=int, default=3,
                    help="batches in flight on separate streams (each with its own plan)")
    ap.add_argument("--workload", default="stereo", choices=["stereo", "mip720", "mip720exact", "backward"],
                    help="profile mode only: mip720exact = the 720p workload with the exact anti-aliasing; "
                         "backward = forward + backward of the 1.5M-primitive 720p view")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

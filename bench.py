"""Forward-render throughput of the 3DGS rasterizer on one GB300.

Default workload: the 1M-Gaussian clustered scene (SH degree 3) rendered at
1920x1080 with 16x16 screen tiles, camera inside the scene. A frame is one
whole forward pass (project -> bin -> blend) through the public C ABI
(gs_render) with the Gaussians resident in HBM. The headline value renders
consecutive frames on --frames-in-flight contexts / streams at once (each
frame's latency-bound front end beside another frame's blend); one step is
one frame on each of those contexts (a batch of F frames), so every timed
step keeps all F in flight. The one-frame-at-a-time time (L2 flushed before
each frame) and the per-stage times are reported beside it.

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (the reference arm for this build).

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
torchrun, every rank renders its own frame stream (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "clustered_1m_1080p": "1M Gaussians (90% in 200 clusters, 10% uniform, 20 m box), SH3, "
                          "1920x1080, 16x16 tiles, camera inside the scene",
    "uniform_box_256": "10k Gaussians uniform in a box, SH0, 256x256, 16x16 tiles",
    "imbalance_6m_4k_x8": "imbalance stress scene, first view: 6M Gaussians, 20% packed into 2% of the view, "
                          "1% splats > 256 px, SH3, 3840x2160",
    "imbalance_1m_4k_x2": "imbalance stress recipe at 1M Gaussians, first view, SH3, 3840x2160",
}

# FP32 operations per evaluated (pixel, Gaussian) pair that every evaluated
# pair needs (offset 2, quadratic form 9, alpha 2, cutoff test 1), plus the
# ones a blended pair adds (transmittance 2, stop test 1, colour 7); the
# exponential is counted separately (SFU).
FLOPS_PER_EVAL = 14
FLOPS_PER_BLEND = 10


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu, self.period = gpu_index, period_ms
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 f"-lms={self.period}", f"--id={self.gpu}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "gloo" if os.environ.get("GS_BENCH_BACKEND") == "gloo" else "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local)  # each rank on its own GPU before NCCL starts
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest of the ranks' values (a timed region's length: the job
    takes as long as its slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, max_ms: float, world: int) -> float:
    """Units all ranks processed per second over the slowest rank's time (each
    rank renders its own independent frames: weak scaling, no exchange)."""
    return units_per_rank * world / (max_ms / 1000.0)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` ("name@workload") from
    profiles/traffic.json (written beside the committed ncu summaries), or
    None if the kernel's source changed since that capture (its SHA-256
    prefix is stored with the number)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        entry = json.load(f).get(kernel)
    if not entry:
        return None, None
    src = os.path.join(ROOT, entry["source"])
    if not os.path.exists(src):
        return None, None
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != entry["sha256_16"]:
            return None, None
    return int(entry["bytes_per_launch"]), entry["summary"]


RTS_MIN_PAIRS = 1 << 23  # key capacities from which gs_render sorts with reduce-then-scan passes


def tile_key_plan(tiles_x: int, tiles_y: int, key_bits: int, capacity: int = 0) -> tuple:
    """(key bytes, digit passes, passes run inside the emission) of gs_render's
    tile sort. Grids at most 256 tiles wide use (row << 8 | column) keys whose
    first (column) pass runs inside the emission kernel; wider grids, and key
    capacities from RTS_MIN_PAIRS on (reduce-then-scan passes), sort tile ids
    (key_bits - 32 bits, key_bits as the library reports it) in separate
    passes. Keys of at most 16 bits are 2 bytes, else 4."""
    if tiles_x <= 256 and capacity < RTS_MIN_PAIRS:
        row_bits = max(0, (tiles_y - 1).bit_length())
        tkey_bits, fused = 8 + row_bits, 1
    else:
        tkey_bits, fused = key_bits - 32, 0
    passes = max(1, (tkey_bits + 7) // 8)
    return (2 if tkey_bits <= 16 else 4), passes, min(fused, passes)


def frame_bytes(n, n_vis, K, sh_degree, tiles_x, tiles_y, key_bits, pixels, readers: int = 1) -> dict:
    """Bytes each forward stage has to move in DRAM, per frame: every mean
    and log-scale (the screen bound), rotation, opacity and SH of the visible
    Gaussians, the 48-byte record and the 48-byte FP32 blend record of each
    visible Gaussian, list entries of 12 B (gathered into index order, then
    four depth passes), tile keys of 2 or 4 B with 4-byte values (written
    once by the emission, after its fused pass where there is one, then read
    and written by each remaining pass), and the image (rgb + final T + last
    contributor). The blend reads each visible Gaussian's blend record once
    (repeat reads across tiles come from L2); with list tiles each list entry
    is read by the `readers` screen tiles of its list tile."""
    s = 3 * (sh_degree + 1) ** 2
    kb, passes, fused = tile_key_plan(tiles_x, tiles_y, key_bits)
    n_tiles = tiles_x * tiles_y
    return {
        "project": n * 24 + n_vis * (20 + 4 * s) + n_vis * (48 + 48 + 12),
        "depth_sort": n_vis * 24 + 4 * n_vis * 24,
        "entry_scan": n_vis * 12,
        "emit": n_vis * (32 + 8) + K * (kb + 4),
        "tile_sort": (passes - fused) * K * 2 * (kb + 4),
        "ranges": K * kb + n_tiles * 8,
        "blend": K * 4 * readers + n_vis * 48 + pixels * 20,
    }


def list_tile_dims(code: int) -> tuple:
    """Screen tiles per list tile (columns, rows) of a gs_options.list_tiles
    or cluster code: 0/1 -> 1x1, 2 -> 2x1, 4 -> 2x2, 16 -> 4x4, 64 -> 8x8."""
    return {0: (1, 1), 1: (1, 1), 2: (2, 1), 4: (2, 2), 16: (4, 4), 64: (8, 8)}[code]


def backward_bytes(n, n_vis, K, sh_degree, pixels) -> int:
    """Bytes of gs_render_backward: the blend backward reads the lists, the
    records and (d_rgb, final T, last contributor) and accumulates 9 floats
    per visible record; the projection backward reads them back with the
    parameters of visible Gaussians and writes every gradient array."""
    s = 3 * (sh_degree + 1) ** 2
    blend = K * 4 + n_vis * 48 + pixels * 20 + n_vis * 36 + n * 36
    project = n * 36 + n_vis * (44 + 4 * s) + n * (44 + 4 * s)
    return blend + project


def fwd_bwd(gs, torch, args, flush, local) -> dict:
    """Forward + backward through the autograd wrapper on the 500k-Gaussian
    clustered scene at 1080p with an L1 loss against a seeded random target:
    per-iteration device time (CUDA events; L2 flushed between iterations)."""
    from paper_2607_15951_gb300 import scenes
    scene, cams = scenes.workload("clustered_500k_1080p")
    cam = cams[0]
    g = gs.scene_to_device(scene)
    params = [g[k].clone().requires_grad_(True) for k in ("means", "log_scales", "quats",
                                                          "opacity_logits", "sh")]
    target = torch.from_numpy(scenes.l1_target(cam.height, cam.width, 1002)).cuda()
    ctx = gs.Context(local)
    stream = torch.cuda.current_stream()

    def it():
        for p in params:
            p.grad = None
        rgb, _ = gs.RasterizeGaussians(*params, ctx, cam, scene.sh_degree)
        loss = torch.nn.functional.l1_loss(rgb, target)
        loss.backward()

    for _ in range(args.warmup):
        it()
    torch.cuda.synchronize()
    # 100 iterations at least: the iteration is bound by the host, whose
    # scheduling varies from iteration to iteration.
    steps = max(100, args.steps // 10)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    fwd = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        for p in params:
            p.grad = None
        ev[i][0].record(stream)
        fwd[i][0].record(stream)
        rgb, _ = gs.RasterizeGaussians(*params, ctx, cam, scene.sh_degree)
        fwd[i][1].record(stream)
        loss = torch.nn.functional.l1_loss(rgb, target)
        loss.backward()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    per_iter = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(per_iter))
    fms = float(np.mean([a.elapsed_time(b) for a, b in fwd]))
    st = gs.gs_last_render_stats(ctx)
    ctx.close()
    pk, _ = peaks()
    fb = frame_bytes(scene.n, st["n_visible"], st["n_keys"], scene.sh_degree, (cam.width + 15) // 16,
                     (cam.height + 15) // 16, st["key_bits"], cam.width * cam.height)
    total = sum(fb.values()) + backward_bytes(scene.n, st["n_visible"], st["n_keys"], scene.sh_degree,
                                              cam.width * cam.height)
    gbs = total / (ms / 1e3) / 1e9
    return {"workload": "clustered_500k_1080p", "description": "500k Gaussians as the 1M scene, SH3, "
            "1920x1080, L1 loss vs a seeded U[0,1] target, torch.autograd through RasterizeGaussians",
            "ms_per_iter": round(ms, 4), "ms_per_iter_median": round(float(np.median(per_iter)), 4),
            "forward_ms": round(fms, 4), "backward_ms": round(ms - fms, 4),
            "iters": steps, "grads": "means, log_scales, quats, opacity_logits, sh (degree 3)",
            "n_visible": st["n_visible"], "n_keys": st["n_keys"],
            "hbm": {"bytes_per_iter": int(total), "GB/s": round(gbs, 1),
                    "frac_of_measured_peak": round(gbs / pk["hbm_gbs"], 4),
                    "note": "render + backward kernel bytes only (the torch loss kernels are not counted)"}}


def batched(gs, torch, args, flush, local) -> dict:
    """64 views of the 1M-Gaussian clustered scene along a smooth camera path
    (1280x720 and 640x480 alternating): one gs_render_batch call with FP16
    records and the autotuned tile shape, against 64 separate FP32 gs_render
    calls. Views per second from CUDA events; L2 flushed between iterations."""
    from paper_2607_15951_gb300 import _native as N
    from paper_2607_15951_gb300 import scenes
    scene, cams = scenes.workload("clustered_1m_traj64")
    g = gs.scene_to_device(scene)
    ctx = gs.Context(local)
    stream = torch.cuda.current_stream()
    outs = gs.alloc_outputs(cams)
    tile, tune_ms, depth, cluster, lists = gs.gs_autotune_batch(ctx, g, scene.sh_degree, cams, outs,
                                                                record_dtype=N.GS_RECORD_F16)
    iters = max(5, args.steps // 100)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for i in range(iters):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / iters

    def per_view():
        for c, o in zip(cams, outs):
            gs.gs_render(ctx, g, scene.sh_degree, c, o["rgb"])

    def per_view_deferred():
        for c, o in zip(cams, outs):
            gs.gs_render(ctx, g, scene.sh_degree, c, o["rgb"], deferred=True)
        gs.gs_sync_status(ctx)

    def batch():
        gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, tile=tile, record_dtype=N.GS_RECORD_F16,
                           batch_depth=depth, cluster=cluster, list_tiles=lists)

    ms_pv_sync = timed(per_view)
    # Deferred frames cannot regrow in place: reserve room for the largest view.
    k_max = 0
    for c, o in zip(cams, outs):
        gs.gs_render(ctx, g, scene.sh_degree, c, o["rgb"])
        k_max = max(k_max, gs.gs_last_render_stats(ctx)["n_keys"])
    gs.gs_reserve_keys(ctx, k_max + k_max // 4 + 1024)
    ms_pv = timed(per_view_deferred)  # the faster per-view schedule is the baseline
    ms_b = timed(batch)
    ms_b32 = timed(lambda: gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs))
    st = gs.gs_last_render_stats(ctx)
    # Forward + backward of all views (L1 loss per view): one joint batch
    # through RasterizeGaussiansBatch against the views one by one through
    # RasterizeGaussians; FP16 records for the batch, FP32 for the views.
    params = [g[k].clone().requires_grad_(True) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    targets = [torch.from_numpy(scenes.l1_target(c.height, c.width, 1200 + i)).cuda() for i, c in enumerate(cams)]

    def fb_batch():
        for p in params:
            p.grad = None
        rgbs = gs.RasterizeGaussiansBatch(*params, ctx, cams, scene.sh_degree, tile=tile,
                                          record_dtype=N.GS_RECORD_F16)
        sum(torch.nn.functional.l1_loss(r, t) for r, t in zip(rgbs, targets)).backward()

    def fb_views():
        for p in params:
            p.grad = None
        for c, t in zip(cams, targets):
            rgb, _ = gs.RasterizeGaussians(*params, ctx, c, scene.sh_degree)
            torch.nn.functional.l1_loss(rgb, t).backward()

    ms_fb_b = timed(fb_batch)
    ms_fb_v = timed(fb_views)
    ctx.close()
    v = len(cams)
    return {"workload": "clustered_1m_traj64", "views": v,
            "description": "1M Gaussians (seed 3), 64 poses on a Catmull-Rom path, 1280x720 / 640x480",
            "per_view_f32_views_per_s": round(v / (ms_pv / 1e3), 1),
            "per_view_f32_note": "64 gs_render calls, GS_SYNC_DEFERRED (no host sync per view)",
            "per_view_f32_synced_views_per_s": round(v / (ms_pv_sync / 1e3), 1),
            "batched_f16_views_per_s": round(v / (ms_b / 1e3), 1),
            "batched_f32_views_per_s": round(v / (ms_b32 / 1e3), 1),
            "speedup_batched_f16_vs_per_view_f32": round(ms_pv / ms_b, 3),
            "ms_per_batch": round(ms_b, 3), "autotuned_tile": list(tile), "autotuned_depth": depth,
            "autotuned_cluster": cluster, "autotuned_list_tiles": lists,
            "autotune_ms_16x16_16x8_8x8_c2x1_c2x2_l2x1_l2x2_l4x4_l8x8": [round(x, 3) for x in tune_ms],
            "keys_per_batch": st["n_keys"], "iters": iters,
            "fwd_bwd_batched_f16_ms": round(ms_fb_b, 3), "fwd_bwd_per_view_f32_ms": round(ms_fb_v, 3),
            "fwd_bwd_speedup": round(ms_fb_v / ms_fb_b, 3),
            "fwd_bwd_note": "L1 loss per view over the 64 views; RasterizeGaussiansBatch (joint batch, one "
                            "batched backward) vs RasterizeGaussians per view"}


def temporal(gs, torch, args, flush, local) -> dict:
    """Temporal re-binning on the 1M-Gaussian 1080p scene under the camera
    motions of the paper's churn experiment: per motion, the churn (Gaussians
    whose tile rect changed, per frame, over all and over visible Gaussians),
    the share of frames re-binned, and device time per frame without temporal
    mode, with the adaptive gate (temporal = 1: re-binned only while that
    measured faster) and with re-binning whenever possible (temporal = 2)
    (CUDA events, L2 flushed between frames)."""
    from paper_2607_15951_gb300 import scenes
    scene, cams0 = scenes.workload("clustered_1m_1080p")
    g = gs.scene_to_device(scene)
    W, H = cams0[0].width, cams0[0].height
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    frames = max(32, min(64, args.steps // 50))
    res = {}
    for kind, step in (("static", None), ("orbit", 0.1), ("orbit", 0.5), ("orbit", 2.0), ("translate", 0.01),
                       ("rotate", 1.0), ("teleport", None)):
        # The first `warm` frames of each motion run untimed (they capture
        # each kind of frame's CUDA graphs and fill the temporal state), then
        # `frames` frames are timed.
        warm = 8
        cams = scenes.motion(kind, warm + frames + 1, W, H, step=step)
        row = {}
        for mode in (0, 1, 2):
            ctx = gs.Context(local)
            for c in cams[:warm + 1]:
                gs.gs_render(ctx, g, scene.sh_degree, c, rgb, temporal=mode)
            times, moved, vis, reb = [], [], [], 0
            for c in cams[warm + 1:]:
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gs.gs_render(ctx, g, scene.sh_degree, c, rgb, temporal=mode)
                b.record(stream)
                b.synchronize()
                st = gs.gs_last_render_stats(ctx)
                times.append(a.elapsed_time(b))
                moved.append(st["n_moved"])
                vis.append(max(1, st["n_visible"]))
                reb += int(st["rebinned"])
            ctx.close()
            if mode == 1:
                row["ms_adaptive"] = round(float(np.mean(times)), 4)
                row["rebinned_frames_adaptive"] = f"{reb}/{frames}"
            elif mode == 2:
                row["ms_rebinning"] = round(float(np.mean(times)), 4)
                row["rebinned_frames"] = f"{reb}/{frames}"
                row["moved_per_frame"] = round(float(np.mean(moved)), 1)
                row["churn_of_all_pct"] = round(100.0 * float(np.mean(moved)) / scene.n, 3)
                row["churn_of_visible_pct"] = round(100.0 * float(np.mean(np.array(moved) / np.array(vis))), 2)
            else:
                row["ms_full"] = round(float(np.mean(times)), 4)
        row["speedup_adaptive"] = round(row["ms_full"] / row["ms_adaptive"], 3)
        row["speedup_rebinning"] = round(row["ms_full"] / row["ms_rebinning"], 3)
        res[kind if step is None else f"{kind}_{step}"] = row
    return {"workload": "clustered_1m_1080p", "frames_per_motion": frames, "untimed_frames_before": 9,
            "note": "orbit about a point 4 m ahead (deg/frame), translate (m/frame), rotate in place (deg/frame)",
            "motions": res}


def imbalance_stress(gs, torch, args, flush, local) -> dict:
    """The imbalance stress configuration: 6M Gaussians (20 % packed into 2 %
    of the first view, 1 % splats above 256 px), SH3, 8 views at 3840x2160.
    Forward: one gs_render_batch with BF16 records (autotuned tile) against 8
    deferred per-view FP32 gs_render calls. Forward + backward: the 8 views
    through the autograd wrapper with BF16 records and an L1 loss each."""
    from paper_2607_15951_gb300 import _native as N
    from paper_2607_15951_gb300 import scenes
    scene, cams = scenes.workload("imbalance_6m_4k_x8")
    g = gs.scene_to_device(scene)
    ctx = gs.Context(local)
    stream = torch.cuda.current_stream()
    outs = gs.alloc_outputs(cams)
    tile, tune_ms, depth, cluster, lists = gs.gs_autotune_batch(ctx, g, scene.sh_degree, cams, outs,
                                                                record_dtype=N.GS_RECORD_BF16)
    iters = 3

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        tot = 0.0
        for i in range(iters):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / iters

    ms_batch = timed(lambda: gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, tile=tile,
                                                record_dtype=N.GS_RECORD_BF16, batch_depth=depth,
                                                cluster=cluster, list_tiles=lists))
    keys_batch = gs.gs_last_render_stats(ctx)["n_keys"]
    k_max = 0
    for c, o in zip(cams, outs):
        gs.gs_render(ctx, g, scene.sh_degree, c, o["rgb"])
        k_max = max(k_max, gs.gs_last_render_stats(ctx)["n_keys"])
    gs.gs_reserve_keys(ctx, k_max + k_max // 4 + 1024)

    def per_view():
        for c, o in zip(cams, outs):
            gs.gs_render(ctx, g, scene.sh_degree, c, o["rgb"], deferred=True)
        gs.gs_sync_status(ctx)

    ms_pv = timed(per_view)
    params = [g[k].clone().requires_grad_(True) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    targets = [torch.from_numpy(scenes.l1_target(c.height, c.width, 1100 + i)).cuda() for i, c in enumerate(cams)]

    def fwd_bwd_views():
        for p in params:
            p.grad = None
        for c, tgt in zip(cams, targets):
            rgb, _ = gs.RasterizeGaussians(*params, ctx, c, scene.sh_degree, record_dtype=N.GS_RECORD_BF16,
                                           cluster=cluster, list_tiles=lists)
            torch.nn.functional.l1_loss(rgb, tgt).backward()

    ms_fb = timed(fwd_bwd_views)
    ctx.close()
    v = len(cams)
    return {"workload": "imbalance_6m_4k_x8",
            "description": "6M Gaussians (seed 4), 20% packed into 2% of view 0, 1% splats > 256 px, SH3, "
                           "8 seeded poses at 3840x2160",
            "batched_bf16_ms": round(ms_batch, 3), "batched_bf16_views_per_s": round(v / (ms_batch / 1e3), 2),
            "per_view_f32_ms": round(ms_pv, 3), "per_view_f32_views_per_s": round(v / (ms_pv / 1e3), 2),
            "speedup_batched_bf16_vs_per_view_f32": round(ms_pv / ms_batch, 3),
            "fwd_bwd_bf16_ms_per_8_views": round(ms_fb, 3),
            "fwd_bwd_note": "per view through RasterizeGaussians (BF16 records, FP32 compositing, the "
                            "autotuned list form), L1 loss each",
            "keys_per_batch": keys_batch, "autotuned_tile": list(tile), "autotuned_cluster": cluster,
            "autotuned_list_tiles": lists,
            "autotune_ms_16x16_16x8_8x8_c2x1_c2x2_l2x1_l2x2_l4x4_l8x8": [round(x, 3) for x in tune_ms], "iters": iters}


def cpu_baseline(scene, cam, budget_s: float = 12.0) -> dict:
    """Time the FP64 oracle on the host cores rendering whole frames of the
    same workload until about ``budget_s`` seconds have passed."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    frames, t0 = 0, time.perf_counter()
    while True:
        oracle.render(scene, cam)
        frames += 1
        el = time.perf_counter() - t0
        if el > budget_s or frames >= 50:
            break
    return {"value": frames / el, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{frames} whole frames of the same workload, FP64, OpenMP over tiles",
            "seconds": round(el, 2)}


REFERENCE_BUDGET_S = 120.0


def headline_metric(workload):
    """The metric string of both arms' JSON lines."""
    if workload == "clustered_1m_1080p":
        return "frames/s (1080p, 1M Gaussians, forward)"
    return f"frames/s ({workload}, forward)"


def headline_config(workload):
    """The `config` object of both arms' JSON lines (the same dict, so the two
    lines name one workload); the GPU arm's run details go under `setup`."""
    return {"workload": workload, "description": WORKLOADS[workload],
            "l2": "GPU arm: inputs above L2 in the headline loop (8 rotating copies of the scene, "
                  "8 x 236 MB, against the 129 MB L2); L2 flushed by a 256 MB write between the "
                  "single-frame steps, outside the timed events. Reference arm: CPU, no L2 handling"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the machine's host cores."""
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    from paper_2607_15951_gb300 import scenes
    import oracle
    oracle.build()
    scene, cams = scenes.workload(args.workload)
    cam = cams[0]
    # Warm-up frames (at most 3: each is a whole FP64 frame), the last one
    # also sizing the sample: whole frames are timed until about two minutes
    # of CPU time, at most one per step, so that any --steps ends in minutes.
    t_frame = 0.0
    for _ in range(max(1, min(args.warmup, 3))):
        t0 = time.perf_counter()
        oracle.render(scene, cam)
        t_frame = time.perf_counter() - t0
    n_frames = int(max(1, min(args.steps, REFERENCE_BUDGET_S // max(t_frame, 1e-3))))
    times = []
    for _ in range(n_frames):
        t0 = time.perf_counter()
        oracle.render(scene, cam)
        times.append(time.perf_counter() - t0)
    ms = 1000 * float(np.mean(times))
    value = 1000.0 / ms
    line = {"impl": "reference", "metric": headline_metric(args.workload),
            "value": round(value, 4), "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(args.workload),
            "cpu_baseline": {"value": round(value, 4), "unit": "frames/s",
                             "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{n_frames} whole frames timed for the {args.steps} steps (one frame "
                                       f"per step, at most {REFERENCE_BUDGET_S:.0f} s of frames)"},
            "e2e": {"value": round(value, 4), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gs", choices=["gs", "reference"])
    ap.add_argument("--workload", default="clustered_1m_1080p", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fwd-bwd", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-temporal", action="store_true")
    ap.add_argument("--no-imbalance", action="store_true")
    ap.add_argument("--frames-in-flight", type=int, default=16,
                    help="consecutive frames rendered on this many contexts / streams at once (headline value)")
    ap.add_argument("--pipeline-blend-variant", type=int, default=0,
                    help="blend schedule of the frames-in-flight loop (0: the default, 8x8 blocks in packed pairs)")
    ap.add_argument("--pipeline-list-tiles", type=int, default=16,
                    help="list tiles of the frames-in-flight loop (16: 4x4 list tiles; 0: a list per screen tile)")
    ap.add_argument("--blend-variant", type=int, default=0,
                    help="0 culled (default: 8x8 blocks, two pixels per lane in packed FP32 pairs), 1 basic, "
                         "2 culled 16x8, 3 culled tile, 4 culled 8x8, 5 TMA staging")
    ap.add_argument("--cluster", type=int, default=0, help="thread-block clusters of the blend: 0, 2 (2x1), 4 (2x2)")
    ap.add_argument("--list-tiles", type=int, default=16,
                    help="lists of list tiles without clusters of the single-frame and end-to-end loops: "
                         "0 (a list per screen tile), 2 (2x1), 4 (2x2), 16 (4x4, default), 64 (8x8)")
    ap.add_argument("--record-dtype", type=int, default=0, help="blend records: 0 FP32, 1 FP16, 2 BF16")
    ap.add_argument("--tile-order", type=int, default=0,
                    help="order of the blend's tiles in the single-frame and end-to-end loops: 0 longest list "
                         "first (default), 1 grid order")
    ap.add_argument("--pipeline-tile-order", type=int, default=1,
                    help="order of the blend's tiles in the frames-in-flight loop (1: grid order, measured faster "
                         "there; 0: longest list first)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    import paper_2607_15951_gb300 as gs
    from paper_2607_15951_gb300 import build as gbuild
    from paper_2607_15951_gb300 import scenes
    gbuild.build()

    scene, cams = scenes.workload(args.workload)
    cam = cams[0]
    if args.cluster > 1:  # clusters and list tiles are exclusive: clusters win
        args.list_tiles = args.pipeline_list_tiles = 0
    ropt = {"cluster": args.cluster, "list_tiles": args.list_tiles, "record_dtype": args.record_dtype,
            "tile_order": args.tile_order}
    H, W = cam.height, cam.width
    g = gs.scene_to_device(scene)
    ctx = gs.Context(local)
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step(deferred=True):
        # GS_SYNC_DEFERRED: the frame is enqueued without a host round trip
        # (its counts are checked by a later call), so frames run back to back.
        gs.gs_render(ctx, g, scene.sh_degree, cam, rgb, variant=args.blend_variant, deferred=deferred, **ropt)

    for _ in range(args.warmup):
        step(False)
    for _ in range(args.warmup):
        step()
    gs.gs_sync_status(ctx)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)

    # Algorithmic work of one frame (deterministic): the pairs evaluated along
    # the 16 x 16 tile lists of the method (a frame with a list per screen
    # tile; list-tile frames count positions in longer lists).
    aux = gs.render(ctx, g, scene.sh_degree, cam, variant=args.blend_variant, record_dtype=args.record_dtype)
    torch.cuda.synchronize()
    n_eval_total = int(aux["n_eval"].to(torch.int64).sum().item())
    del aux
    gs.gs_render(ctx, g, scene.sh_degree, cam, rgb, variant=args.blend_variant, **ropt)
    torch.cuda.synchronize()
    stats = gs.gs_last_render_stats(ctx)  # the measured list form's counts

    # Timed region: one frame at a time (each a replay of the context's CUDA
    # graph of the frame), per-step CUDA events, L2 flushed between steps
    # outside them.
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.1)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clk = clocks.stop()
    gs.gs_sync_status(ctx)
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    dev_ms = max_over_ranks(dev_ms, world)
    single_ms = dev_ms / args.steps  # one frame at a time, L2 flushed before each

    # Stage times: the same frames with the library's stage events (the
    # kernels then launch directly), L2 flushed before each.
    gs.gs_set_stage_timing(ctx, True)
    stage_sum = {}
    n_stage = min(args.steps, 60)
    for i in range(n_stage):
        flush.fill_(float(i))
        step()
        if i % 10 == 0 or i == n_stage - 1:
            st = gs.gs_last_stage_times(ctx)   # synchronises on this step's events
            for k, v in st.items():
                stage_sum.setdefault(k, []).append(v)
    gs.gs_set_stage_timing(ctx, False)
    gs.gs_sync_status(ctx)

    # Frames in flight: consecutive frames go to F contexts on F streams (each
    # context owns its workspace), so one frame's latency-bound front end runs
    # beside another's issue-bound blend. One step is F consecutive frames, one
    # per context. The inputs rotate over 8 copies of the scene (1.9 GB, far
    # above L2), so no flush is needed; the timed region spans all steps, from
    # one event before the first frame to one after the last.
    F = max(1, args.frames_in_flight)
    copies = [g] + [{k: v.clone() for k, v in g.items()} for _ in range(7)]
    pctx = [ctx] + [gs.Context(local) for _ in range(F - 1)]
    pstreams = [torch.cuda.Stream() for _ in range(F)]
    prgb = [rgb] + [torch.empty_like(rgb) for _ in range(F - 1)]
    popt = dict(ropt, list_tiles=args.pipeline_list_tiles, tile_order=args.pipeline_tile_order)
    # Warm-up: W steps of the timed loop itself (the same contexts, streams,
    # scene copies and framebuffers, so every context has captured the CUDA
    # graphs of the frames it renders before the timed region).
    for k in range(F):
        gs.gs_render(pctx[k], g, scene.sh_degree, cam, prgb[k], variant=args.pipeline_blend_variant, **popt)
    for i in range(args.warmup * F):
        k = i % F
        with torch.cuda.stream(pstreams[k]):
            gs.gs_render(pctx[k], copies[i % len(copies)], scene.sh_degree, cam, prgb[k],
                         variant=args.pipeline_blend_variant, deferred=True, stream=pstreams[k], **popt)
    torch.cuda.synchronize()
    for c in pctx:
        gs.gs_sync_status(c)
    barrier(world)
    clocks2 = ClockSampler(local)
    clocks2.start()
    time.sleep(0.1)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for ps in pstreams:
        ps.wait_event(p0)
    for i in range(args.steps * F):
        k = i % F
        with torch.cuda.stream(pstreams[k]):
            gs.gs_render(pctx[k], copies[i % len(copies)], scene.sh_degree, cam, prgb[k],
                         variant=args.pipeline_blend_variant, deferred=True, stream=pstreams[k], **popt)
    for ps in pstreams:
        stream.wait_stream(ps)
    p1.record(stream)
    torch.cuda.synchronize()
    clk_pipe = clocks2.stop()
    barrier(world)
    for c in pctx:
        gs.gs_sync_status(c)
    pstats = gs.gs_last_render_stats(pctx[0])  # a frame of the headline loop (its list form)
    pipe_ms = max_over_ranks(p0.elapsed_time(p1), world)
    ms_per_step = pipe_ms / args.steps
    ms_per_frame = pipe_ms / (args.steps * F)
    value = whole_job_rate(args.steps * F, pipe_ms, world)
    for c in pctx[1:]:
        c.close()
    del copies
    # The same frames rendered synchronously (the host waits for each frame's
    # counts): the host round trip then shows between frames.
    n_sync = min(args.steps, 100)
    sync_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_sync)]
    for i in range(n_sync):
        flush.fill_(float(i))
        sync_ev[i][0].record(stream)
        step(False)
        sync_ev[i][1].record(stream)
    torch.cuda.synchronize()
    sync_ms = sum(a.elapsed_time(b) for a, b in sync_ev) / n_sync
    stage_ms = {k: float(np.median(v)) for k, v in stage_sum.items()}

    # End to end: every step copies its inputs (the Gaussian arrays) from
    # pinned host memory and reads its image back, through the public
    # gs_render. The inputs are double-buffered: the copy for step i + 1 runs
    # on a copy stream while step i renders (deferred frames, reserved key
    # capacity), as a streaming renderer would; every step's bytes still
    # cross the link inside the timed region.
    host = {k: v.cpu().pin_memory() for k, v in g.items()}
    dev_in = [{k: torch.empty_like(v) for k, v in g.items()} for _ in range(2)]
    host_rgb = [torch.empty((H, W, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = host_rgb[0].numel() * 4
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    gs.gs_reserve_keys(ctx, stats["n_keys"] + stats["n_keys"] // 4 + 4096)

    def e2e_run(steps):
        copy_stream.wait_stream(stream)
        with torch.cuda.stream(copy_stream):
            for k in host:
                dev_in[0][k].copy_(host[k], non_blocking=True)
            copied[0].record(copy_stream)
        for i in range(steps):
            b = i % 2
            if i + 1 < steps:
                nb = (i + 1) % 2
                with torch.cuda.stream(copy_stream):
                    if i >= 1:
                        copy_stream.wait_event(consumed[nb])
                    for k in host:
                        dev_in[nb][k].copy_(host[k], non_blocking=True)
                    copied[nb].record(copy_stream)
            stream.wait_event(copied[b])
            gs.gs_render(ctx, dev_in[b], scene.sh_degree, cam, rgb, variant=args.blend_variant, deferred=True,
                         **ropt)
            consumed[b].record(stream)
            host_rgb[b].copy_(rgb, non_blocking=True)

    e2e_run(3)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    e2e_run(args.e2e_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    e2e_value = whole_job_rate(args.e2e_steps, e2e_ms, world)

    # The host link alone: the same input copies and image read-backs, each
    # direction timed by itself, give the frame rate the link allows.
    def link_gbs(copy, nbytes, reps=3):
        copy()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            copy()
        b.record(stream)
        torch.cuda.synchronize()
        return reps * nbytes / (a.elapsed_time(b) / 1e3) / 1e9

    def h2d_copy():
        for k in host:
            dev_in[0][k].copy_(host[k], non_blocking=True)

    h2d_gbs = link_gbs(h2d_copy, h2d)
    d2h_gbs = link_gbs(lambda: host_rgb[0].copy_(rgb, non_blocking=True), d2h)
    link_fps = 1.0 / max(h2d / (h2d_gbs * 1e9), d2h / (d2h_gbs * 1e9))

    # Roofline of the dominant kernel (blend): FP32 work per launch / its time.
    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_clock = (clk.get("sm_max_mhz") or pk.get("sm_max_mhz") or 2070.0)
    fp32_peak_tflops = sms * 128 * 2 * sm_clock * 1e6 / 1e12
    blend_ms = stage_ms.get("blend_ms", float("nan"))
    flops = FLOPS_PER_EVAL * n_eval_total
    achieved = flops / (blend_ms / 1e3) / 1e12
    clx, cly = list_tile_dims(max(args.cluster, args.list_tiles))
    blend_kernel = (f"blend_cluster_kernel<{clx},{cly}>" if args.cluster > 1 else
                    f"blend_listtile_kernel<{clx},{cly}>" if args.list_tiles > 1 else
                    "blend_culled_kernel<8,8>" if args.blend_variant == 0 else "blend_basic_kernel")
    traffic, traffic_src = profiled_traffic(f"{blend_kernel}@{args.workload}")
    roofline = {"kernel": blend_kernel, "stage": "gs_blend", "bound": "alu", "achieved": round(achieved, 3),
                "peak": round(fp32_peak_tflops, 2), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak_tflops, 4), "traffic": traffic,
                "traffic_source": traffic_src,
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {sm_clock:.0f} MHz",
                "units_per_launch": n_eval_total, "flops_per_unit": FLOPS_PER_EVAL,
                "launch_ms": round(blend_ms, 4),
                "note": "blend kernel alone, one frame at a time (default schedule), live CUDA events "
                        "recorded by the library around the launch (gs_set_stage_timing)"}
    # The headline loop's own roofline: with frames in flight the blend work of
    # one frame is done once per frame interval, and the frame's DRAM bytes
    # move once per frame interval.
    roofline_headline = {
        "loop": f"{F} frames in flight, blend schedule {args.pipeline_blend_variant}, "
                f"list tiles {args.pipeline_list_tiles}, "
                f"{'longest-first' if args.pipeline_tile_order == 0 else 'grid'} tile order",
        "frame_ms": round(ms_per_frame, 5),
        "blend_alu": {"bound": "alu", "achieved": round(flops * value / world / 1e12, 3),
                      "peak": round(fp32_peak_tflops, 2), "unit": "TFLOP/s",
                      "frac": round(flops * value / world / 1e12 / fp32_peak_tflops, 4)}}

    # HBM view of the same frame: bytes each stage must move / its live time.
    slx, sly = list_tile_dims(max(args.list_tiles, args.cluster))
    fbytes = frame_bytes(scene.n, stats["n_visible"], stats["n_keys"], scene.sh_degree, (W + 16 * slx - 1) // (16 * slx),
                         (H + 16 * sly - 1) // (16 * sly), stats["key_bits"], W * H, readers=slx * sly)
    stage_of = {"project": "project_ms", "depth_sort": "depth_sort_ms", "entry_scan": "entry_scan_ms",
                "emit": "emit_ms", "tile_sort": "tile_sort_ms", "ranges": "ranges_ms", "blend": "blend_ms"}
    hbm_peak = pk.get("hbm_gbs") or 6800.0
    hbm = {}
    for k, b in fbytes.items():
        t = stage_ms.get(stage_of[k], float("nan"))
        gbs = b / (t / 1e3) / 1e9 if t > 0 else float("nan")
        hbm[k] = {"bytes": int(b), "ms": round(t, 4), "GB/s": round(gbs, 1), "frac": round(gbs / hbm_peak, 4)}
    # The headline loop's frames: their own lists (list tiles), read by every
    # screen tile of a list tile.
    plx, ply = list_tile_dims(args.pipeline_list_tiles)
    pbytes = frame_bytes(scene.n, pstats["n_visible"], pstats["n_keys"], scene.sh_degree,
                         (W + 16 * plx - 1) // (16 * plx), (H + 16 * ply - 1) // (16 * ply), pstats["key_bits"],
                         W * H, readers=plx * ply)
    frame_gbs = sum(pbytes.values()) / (ms_per_frame / 1e3) / 1e9
    hbm["frame"] = {"bytes": int(sum(pbytes.values())), "ms": round(ms_per_frame, 5), "GB/s": round(frame_gbs, 1),
                    "frac": round(frame_gbs / hbm_peak, 4), "peak_GB/s": hbm_peak,
                    "peak_source": "measured" if pk_kind == "measured" else "fallback",
                    "note": "per frame of the headline loop"}
    roofline_headline["frame_hbm"] = {"bound": "hbm", "achieved": round(frame_gbs, 1), "peak": hbm_peak,
                                      "unit": "GB/s", "frac": round(frame_gbs / hbm_peak, 4),
                                      "bytes_per_frame": int(sum(pbytes.values()))}

    line = {
        "metric": headline_metric(args.workload),
        "value": round(value, 3), "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config(args.workload),
        "setup": {"n_visible": stats["n_visible"], "n_keys": stats["n_keys"],
                   "key_bits": stats["key_bits"], "blend_variant": args.blend_variant,
                   "cluster": args.cluster, "list_tiles": args.list_tiles, "record_dtype": args.record_dtype,
                   "tile_order": ("longest list first" if args.tile_order == 0 else "grid"),
                   "sync_mode": "deferred (GS_SYNC_DEFERRED)",
                   "frames_in_flight": F,
                   "frames_per_step": F,
                   "ms_per_frame": round(ms_per_frame, 5),
                   "frames_in_flight_blend_variant": args.pipeline_blend_variant,
                   "frames_in_flight_list_tiles": args.pipeline_list_tiles,
                   "frames_in_flight_tile_order": ("longest list first" if args.pipeline_tile_order == 0
                                                   else "grid"),
                   "frames_in_flight_keys": pstats["n_keys"],
                   "inputs": "8 rotating copies of the scene (8 x 236 MB, above L2) in the frames-in-flight loop",
                   "single_stream_frame_ms": round(single_ms, 4),
                   "single_stream_frames_per_s": round(1000.0 / single_ms, 3),
                   "sync_frame_ms": round(sync_ms, 4)},
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "wall_s_timed_loop": round(wall, 3),
        "e2e": {"value": round(e2e_value, 3), "unit": "frames/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
                "schedule": "inputs double-buffered: step i+1's host-to-device copy (copy stream) overlaps "
                            "step i's render and image read-back; gs_render deferred",
                "link": {"h2d_GB/s": round(h2d_gbs, 1), "d2h_GB/s": round(d2h_gbs, 1),
                         "bound_frames_per_s": round(link_fps * world, 3),
                         "frac_of_bound": round(e2e_value / (link_fps * world), 4),
                         "note": "each direction timed alone with the same copies; the bound takes the "
                                 "slower direction (the two overlap)"}},
        "gpu_launches": None,
        "roofline": roofline,
        "roofline_headline": roofline_headline,
        "hbm_roofline": hbm,
        "peaks": {"source": pk_kind, "hbm_gbs": pk.get("hbm_gbs")},
        "clocks": clk_pipe,
        "clocks_single_stream": clk,
    }
    # Kernel launches per gs_render: projection + compact list, the list
    # gather, four depth digit passes, the entry scan, the key emission (with
    # the first tile pass inside it on grids at most 256 tiles wide), the
    # other tile passes, ranges, blend.
    _, passes, fused = tile_key_plan((W + 16 * plx - 1) // (16 * plx), (H + 16 * ply - 1) // (16 * ply),
                                     pstats["key_bits"])
    per_frame = 10 + passes - fused
    line["gpu_launches"] = per_frame * F * args.steps
    if not args.no_fwd_bwd:
        line["fwd_bwd"] = fwd_bwd(gs, torch, args, flush, local)
    if not args.no_batched:
        line["batched"] = batched(gs, torch, args, flush, local)
    if not args.no_temporal:
        line["temporal"] = temporal(gs, torch, args, flush, local)
    if not args.no_imbalance:
        line["imbalance"] = imbalance_stress(gs, torch, args, flush, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, cam)
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

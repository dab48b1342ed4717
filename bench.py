#!/usr/bin/env python
"""Benchmark of the 4D-rotor Gaussian splatting render on one GB300.

Workload (frames/s): 300,000 seeded synthetic 4D Gaussians (means in [-3,3]^3),
1352x1014, the 300-frame circular sweep at radius 8 (t_k = k/299), FP32, one
view per launch; a step renders one frame of the sweep. The same run also
measures the training step (4 views at seeded (t, angle), forward + L1 loss +
backward through the autograd-free C ABI path) as train it/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. Multi-GPU runs (torchrun) are independent replicas:
each rank renders its own frames of the sweep, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s & train it/s, 300k 4D Gaussians @1352×1014, vs plain path; % roofline"
WIDTH, HEIGHT, N_GAUSS, FRAMES, RADIUS = 1352, 1014, 300_000, 300, 8.0
TRAIN_VIEWS = 4
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--train-steps", type=int, default=50, help="timed training steps (after 5 warm-up)")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 16-view batched workload")
    ap.add_argument("--no-large", action="store_true", help="skip the 2M-Gaussian BF16 workload")
    ap.add_argument("--no-extras", action="store_true", help="skip the flow / KNN / regulariser timings")
    ap.add_argument("--batch-only", action="store_true", help="batched and large workloads only (profiling)")
    ap.add_argument("--frames-only", action="store_true", help="render frames only (profiling)")
    ap.add_argument("--tile", default=None, metavar="WxH",
                    help="tile shape of the frame sweep (8x8, 16x16 or 16x32) instead of the autotuner's choice, "
                         "e.g. to profile the shape a timed run chose (the autotuner times live launches)")
    ap.add_argument("--train-only", action="store_true", help="training steps only (profiling)")
    ap.add_argument("--backward-only", action="store_true",
                    help="render + backward of sweep frame 37, four times (profiling the backward)")
    ap.add_argument("--backward-views", type=int, default=1, metavar="V",
                    help="with --backward-only and V > 1: one batched render + backward of the first training "
                         "step's V views instead, four times (profiling the training step's backward launch)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def frames_for_rank(rank: int, steps: int) -> list[int]:
    """The sweep frames a replica renders: rank r takes steps r*K .. r*K+K-1 of
    the sequence k -> 7k mod 300 (7 is prime to 300, so ranks do not repeat
    each other's frames until the sweep is exhausted)."""
    return [(rank * steps + i) * 7 % FRAMES for i in range(steps)]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the process group (the slowest replica
    sets the job's time); the value itself without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks ------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def _rows(self) -> list:
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and line.endswith("\n"):
                rows.append(parts)
        return rows

    def wait_ready(self, timeout: float = 10.0) -> None:
        """Block until the sampler has written its first sample (nvidia-smi's
        start-up then lies before the timed region, not inside it)."""
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < timeout:
            if self._rows():
                return
            time.sleep(0.02)

    def mark(self) -> int:
        """The number of samples so far (the timed region starts after them)."""
        return len(self._rows()) if self.proc is not None else 0

    def stop(self, since: int = 0) -> dict:
        """Stop sampling; summarise the samples from the last one before mark
        `since` (the clocks as the timed region began) to the end."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self._rows()[max(since - 1, 0):]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- workload ------------------------------------------------------------------
def frame_camera(k: int):
    import synth
    return synth.orbit_camera(k % FRAMES, FRAMES, RADIUS, WIDTH, HEIGHT)


SMS, FP32_LANES = 152, 128
# FP32 operations (an FMA counts once) the compositing rule of Eq. 3 needs per
# composited (pixel, Gaussian) pair: d (2), -1/2 d^T conic d (9), alpha =
# o e^power (1), the 0.99 clamp (1), T (1 - alpha) (2), w = alpha T (1),
# C += c w (3); the exponential itself runs on the MUFU unit.
FP32_OPS_PER_PAIR = 19

# DRAM bytes (read + write) of one launch of the kernel at a tile shape, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum): the blend on a
# sweep frame, the blend backward on the training step's 4-view launch (the views
# of step 0, `--backward-only --backward-views 4`); a kernel or shape without a
# capture of its current code reports None.
DRAM_TRAFFIC = {"blend@16x32": 18_583_552, "blend@16x16": 21_566_464, "blend_bwd@16x32": 340_284_672}

# the workload both arms report (the reference arm times the oracle on a
# bounded sample of it: frame 37, random pixels)
CONFIG = {"workload": "300k 4D Gaussians, 1352x1014, 300-frame orbit sweep r=8, FP32, 1 view/launch",
          "n_gaussians": N_GAUSS, "width": WIDTH, "height": HEIGHT, "tile": "from the autotuner (plain path 16x16)",
          "l2": "flushed between steps (512 MB write)"}


def algorithmic_bytes(stage: str, n: int, n_vis: int, keys: int, npix: int) -> float:
    """Bytes a stage must move per launch: per Gaussian, per visible item, per
    (tile, Gaussian) pair and per pixel."""
    if stage == "preprocess":
        return 68.0 * n + 192.0 * n_vis + 48.0 * n_vis + 12.0 * n
    if stage == "binning":
        return 4.0 * n + 12.0 * n_vis + 8.0 * keys
    if stage == "sort":  # depth sort of N (key, index) pairs + tile sort of the pairs, one read + one write
        return 16.0 * n + 16.0 * keys
    if stage == "ranges":
        return 8.0 * 5440
    if stage == "blend":
        return 4.0 * keys + 48.0 * n_vis + 20.0 * npix
    return 0.0


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03307_gb300 as r4g
    from paper_2402_03307_gb300 import abi
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    g = synth.fwd300k_scene()
    params = {k: torch.as_tensor(v).to(dev).contiguous() for k, v in g.items()}
    rend = r4g.Renderer()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    if args.train_only:
        return {"train": train_bench(args, r4g.Renderer(), params, dev, stream, flush)}
    if args.backward_only:
        if args.tile:
            rend.set_tile(tuple(int(x) for x in args.tile.lower().split("x")))
        if args.backward_views > 1:
            views = train_views_for_step(0)[:args.backward_views]
            grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in params.items()}
            target = _packed_target(views, 34, dev)
            for _ in range(4):
                res = rend.render_batch(params, views)
                rend.backward_batch(params, res, torch.sign(res.packed - target) / target.numel(), grads)
            torch.cuda.synchronize()
            return {"backward_only": f"training step 0's {len(views)} views, 4 x (batched render + backward), "
                                     f"{rend.tile[0]}x{rend.tile[1]} tiles"}
        cam, t = frame_camera(37)
        grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in params.items()}
        gimg = torch.randn((3, HEIGHT, WIDTH), device=dev, generator=torch.Generator(device=dev).manual_seed(3)) * 1e-6
        for _ in range(4):
            res = rend.render(params, cam, t)
            rend.backward(params, cam, t, res, gimg, grads)
        torch.cuda.synchronize()
        return {"backward_only": f"frame 37, 4 x (render + backward), {rend.tile[0]}x{rend.tile[1]} tiles"}
    if args.batch_only:
        return {"batched": batch_bench(args, dev, stream, flush), "large": large_bench(args, dev, stream, flush)}

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    frames = frames_for_rank(rank, args.steps)
    # the tile shape: the library's autotuner on the first frame (untimed);
    # the plain 16x16 path is timed on the same frames below
    rend16 = rend
    rend = r4g.Renderer()
    cam0, t0 = frame_camera(frames[0])
    if args.tile:
        rend.set_tile(tuple(int(x) for x in args.tile.lower().split("x")))
        tune = {"ms": None, "tile": list(rend.tile)}
    else:
        tune = rend.autotune(params, [(cam0, t0)], backward=False, reps=3)
    # size the key buffer once over the whole sweep (not timed): 10 % above the
    # largest (tile, Gaussian) pair count of any frame
    need_max = 0
    for k in range(FRAMES):
        cam, t = frame_camera(k)
        res = rend.render(params, cam, t)
        need_max = max(need_max, rend.status(res)[1])
    cap = int(need_max * 1.1) + 1024
    frame = rend.new_frame(N_GAUSS, WIDTH, HEIGHT, cap, dev)
    img = torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device=dev)

    def render_frame(k):
        cam, t = frame_camera(k)
        return rend.render(params, cam, t, frame=frame, key_capacity=cap, out=img, check=False)

    # the clock sampler's process starts during the warm-up frames (its
    # start-up otherwise lands on the first timed one)
    clocks = ClockSampler(local)
    clocks.start()
    for i in range(max(args.warmup, 3)):
        render_frame(frames[i % len(frames)])
    for k in frames[:min(len(frames), 8)]:
        render_frame(k)
    # a process's first loop of timed CUDA events ran its first frame ~0.2 ms
    # slow whatever came before it (measured); warm-up frames take that loop
    wevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(4)]
    for a, b in wevs:
        flush.zero_()
        a.record(stream)
        render_frame(frames[0])
        b.record(stream)
    torch.cuda.synchronize()
    clocks.wait_ready()
    abi.r4g_stage_times(rend.ctx, reset=True)
    # the timed frames run without per-stage events (an event between two
    # kernels ends their programmatic launch overlap); the stage times come
    # from a second pass over the same frames below
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in frames]
    # the calls' arguments are built before the timed loop, so that between a
    # frame's two events the host does nothing but the r4g_render call itself
    # (otherwise the camera and the argument structs, built after the first
    # event, could leave the device waiting inside the frame)
    gstruct = r4g.gaussians_struct(params)
    calls = []
    for k in frames:
        cam, t = frame_camera(k)
        calls.append((r4g.camera_struct(cam), float(t)))
    img_ptr, frame_ptr, frame_len, sptr = img.data_ptr(), frame.data_ptr(), frame.numel(), stream.cuda_stream
    barrier()
    torch.cuda.synchronize()
    since = clocks.mark()
    wall0 = time.perf_counter()
    # two untimed renders queued right before the first timed frame: coming
    # out of the idle gap above, the device ran the first frame up to 20 %
    # slower (0.33 ms against 0.28 ms for the same frame queued behind other
    # work); L2 flushes alone did not bring it back
    for k in frames[-2:]:
        render_frame(k)
    for i, (cs, t) in enumerate(calls):
        flush.zero_()  # evict L2 between frames (outside the timed events)
        evs[i][0].record(stream)
        abi.r4g_render(rend.ctx, gstruct, cs, t, img_ptr, None, None, frame_ptr, frame_len, cap, sptr)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop(since)
    _, stage_launch = abi.r4g_stage_times(rend.ctx, reset=True)
    # per-stage device times: the same frames again, stage events on
    abi.r4g_set_timing(rend.ctx, True)
    for k in frames:
        flush.zero_()
        render_frame(k)
    torch.cuda.synchronize()
    abi.r4g_set_timing(rend.ctx, False)
    stage_ms, _ = abi.r4g_stage_times(rend.ctx, reset=True)
    for k in frames[-3:]:
        if rend.status(render_frame(k))[0] != abi.R4G_OK:
            raise RuntimeError("key buffer overflow during the timed region")
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(step_ms), dev)
    fps = world * len(frames) / (total_ms / 1e3)
    median_ms = statistics.median(step_ms)

    # per-frame work of the timed frames, counted in an untimed instrumented pass
    counter = r4g.Renderer(tile=rend.tile, flags=abi.R4G_FLAG_COUNT_PAIRS)
    cframe = counter.new_frame(N_GAUSS, WIDTH, HEIGHT, cap, dev)
    work = {"keys": 0, "n_visible": 0, "pairs": 0}
    for k in frames:
        cam, t = frame_camera(k)
        r = counter.render(params, cam, t, frame=cframe, key_capacity=cap, out=img, check=False)
        st_ = counter.stats(r)
        work["keys"] += st_["key_count"]
        work["n_visible"] += st_["n_visible"]
        work["pairs"] += st_["composited_pairs"]
    work = {k: v / len(frames) for k, v in work.items()}
    keys, n_vis = work["keys"], work["n_visible"]
    per_stage = {k: v / len(frames) for k, v in stage_ms.items() if v > 0}
    top = max(per_stage, key=per_stage.get)
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    alu_peak = SMS * FP32_LANES * sm_mhz * 1e6 / 1e12  # FP32 lane-operations, T/s

    def stage_roof(stage):
        sec = per_stage[stage] / 1e3
        if stage == "blend":
            ach = work["pairs"] * FP32_OPS_PER_PAIR / sec / 1e12
            return {"bound": "alu", "achieved": round(ach, 3), "peak": round(alu_peak, 2),
                    "unit": "TFLOP/s", "frac": round(ach / alu_peak, 4)}
        ach = algorithmic_bytes(stage, N_GAUSS, n_vis, keys, WIDTH * HEIGHT) / sec / 1e9
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(ach / hbm_peak, 4)}

    roofline = dict(stage_roof(top))
    roofline.update({"kernel": top, "traffic": DRAM_TRAFFIC.get(f"{top}@{rend.tile[0]}x{rend.tile[1]}"),
                     "peak_source": (f"{SMS} SMs x {FP32_LANES} FP32 lanes x {sm_mhz:.0f} MHz (sm_max_mhz of "
                                     f"MEASURED_PEAKS.json)") if top == "blend" else f"{src} hbm_gbs",
                     "work_per_frame": {"composited_pairs": round(work["pairs"]), "keys": round(keys),
                                        "visible": round(n_vis), "fp32_ops_per_pair": FP32_OPS_PER_PAIR},
                     "stage_ms": {k: round(v, 4) for k, v in per_stage.items()},
                     "stages": {k: stage_roof(k) for k in per_stage}})

    out = {"metric": METRIC, "value": round(fps, 2), "unit": "frames/s", "n_gpus": world,
           "steps": len(frames), "warmup": args.warmup, "ms_per_step": round(total_ms / len(frames), 4),
           "ms_per_step_median": round(median_ms, 4), "fps_at_median": round(1e3 / median_ms, 2),
           "ms_per_step_min_max": [round(min(step_ms), 4), round(max(step_ms), 4)],
           "ms_per_frame": {str(k): round(x, 4) for k, x in zip(frames, step_ms)},
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded 4D Gaussians; stands in for Plenoptic Video at its resolution)",
           "config": dict(CONFIG, parallelism=f"replicas x{world}",
                          workload=CONFIG["workload"] + f"; {len(frames)} of the {FRAMES} sweep frames timed "
                                                        f"per rank (k = 7 i mod {FRAMES})"),
           "gpu_launches": int(sum(stage_launch.values())),
           "wall_s": round(wall, 3), "clocks": clk, "roofline": roofline}
    out["config"]["tile"] = (f"{rend.tile[0]}x{rend.tile[1]} "
                             f"({'--tile' if args.tile else 'from the autotuner'}; plain path 16x16)")
    out["autotune_ms"] = tune["ms"]
    out["plain_path"], cap16 = plain_sweep_bench(rend16, params, dev, stream, flush, frames)

    # ---- training step: 4 views forward + L1 + backward --------------------------
    if not args.no_train and not args.frames_only:
        out["train"] = train_bench(args, rend16, params, dev, stream, flush)
    # ---- batched views (autotuned tile, CUDA graph) and the large BF16 scene ---------
    if not args.no_batch and not args.frames_only:
        out["batched"] = batch_bench(args, dev, stream, flush)
    if not args.no_large and not args.frames_only:
        out["large"] = large_bench(args, dev, stream, flush)
    if not args.no_extras and not args.frames_only:
        out["extras"] = extras_bench(args, params, dev, stream, flush, frames, cap16)
    # ---- end to end through host buffers ---------------------------------------------
    if not args.no_e2e and not args.frames_only:
        out["e2e"] = e2e_bench(args, rend, g, dev, stream, frames, cap)
    return out


def measured_peaks() -> dict:
    """MEASURED_PEAKS.json (HBM copy GB/s, bf16 TFLOP/s, clocks) when present."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _timed(fn, steps: int, stream, flush=None) -> float:
    """Mean ms of fn() over `steps` calls, CUDA events on `stream` around each
    call; the L2 flush (when given) runs between calls, outside the events."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in evs:
        if flush is not None:
            flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def _packed_target(views, seed, dev):
    import numpy as np
    import torch
    import synth
    parts = [synth.smooth_target(seed + k, cam.width, cam.height).reshape(-1) for k, (cam, _) in enumerate(views)]
    return torch.as_tensor(np.concatenate(parts)).to(dev)


# FP32 operations per composited (pixel, Gaussian) pair of the backward of
# Eq. 3 (an FMA counts once): the forward's evaluation again, d (2),
# -1/2 d^T conic d (9), alpha (1), the clamp (1); the transmittance recovered
# back to front, 1 - alpha (1), T_i = T_{i+1} / (1 - alpha) (1, with the
# reciprocal on the MUFU unit); w = alpha T_i (1); g . c (3);
# dL/dalpha = (g . c T_i - U) / (1 - alpha) (2); U += (g . c) w (1);
# dq = dL/dalpha alpha (1); the moments of dq over the pixel, dq dx, dq dx^2
# and their three sums (5); the colour gradient g w, summed (6).
BWD_FP32_OPS_PER_PAIR = 34


def train_views_for_step(k: int):
    """The 4 views of training step k: seeded (t ~ U[0,1], angle ~ U[0, 2 pi))."""
    import synth
    return synth.train_views(seed=1000 + k, views=TRAIN_VIEWS)


def train_bench(args, rend, params, dev, stream, flush):
    """Training step of 4 views at fresh seeded (t, angle) each step, 1352x1014,
    L1 loss against a seeded smooth target (one per view slot): (a) through the
    autograd function of the batched render (one batched call), (b) the plain
    path, one single-view render + backward per view, (c) the batched step
    captured in a CUDA graph, the step's views copied into its device view
    table before each replay. Per-stage times come from a second pass with the
    library's stage events on; the composited pairs from an untimed counting
    pass over the same views."""
    import torch
    import paper_2402_03307_gb300 as r4g
    from paper_2402_03307_gb300 import abi

    nsteps = args.train_steps
    warm = 5
    step_views = [train_views_for_step(k) for k in range(warm + nsteps)]
    target = _packed_target(step_views[0], 34, dev)
    npix = target.numel()
    inv = 1.0 / npix
    leaves = {k: v.clone().requires_grad_(True) for k, v in params.items()}
    # the batched paths take the tile shape the library's autotuner picks for
    # these views (untimed); the plain per-view path keeps 16x16
    rb = r4g.Renderer()
    tune = rb.autotune(params, step_views[0], backward=True, reps=3)
    cap_b = rb.reserve_batch(params, step_views)  # untimed: no step overflows its key buffer
    # the plain path: one frame per view slot, sized for the largest view of any step
    need = 0
    for views in step_views:
        for cam, t in views:
            need = max(need, rend.status(rend.render(params, cam, t))[1])
    cap_p = int(need * 1.1) + 1024
    frames = [rend.new_frame(N_GAUSS, WIDTH, HEIGHT, cap_p, dev) for _ in range(TRAIN_VIEWS)]
    imgs = [torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device=dev) for _ in range(TRAIN_VIEWS)]
    tviews = [target[k * 3 * WIDTH * HEIGHT:(k + 1) * 3 * WIDTH * HEIGHT].view(3, HEIGHT, WIDTH)
              for k in range(TRAIN_VIEWS)]
    gimg = torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device=dev)
    grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in params.items()}
    graph = r4g.BatchGraph(rb, params, step_views[0], key_capacity=cap_b,
                           grad_fn=lambda img: torch.sign(img - target) * inv)
    tables = [graph.views_table(v) for v in step_views]
    it = {"a": 0, "p": 0, "g": 0}

    def step_autograd():
        views = step_views[it["a"] % len(step_views)]
        it["a"] += 1
        for v in leaves.values():
            v.grad = None
        img = r4g.render_batch(leaves, views, renderer=rb)
        loss = (img - target).abs().mean()
        loss.backward()

    def step_plain():
        views = step_views[it["p"] % len(step_views)]
        it["p"] += 1
        for v in grads.values():
            v.zero_()
        for (cam, t), fr, im, tv in zip(views, frames, imgs, tviews):
            res = rend.render(params, cam, t, frame=fr, key_capacity=cap_p, out=im, check=False)
            torch.sign(im - tv, out=gimg)
            gimg.mul_(inv)
            rend.backward(params, cam, t, res, gimg, grads)

    def step_graph():
        graph.replay(table=tables[it["g"] % len(tables)])
        it["g"] += 1

    for _ in range(warm):
        step_autograd()
        step_plain()
        step_graph()
    for k in it:  # the timed steps take views warm .. warm + nsteps - 1
        it[k] = warm
    ms_a = _timed_all(step_autograd, nsteps, stream, flush)
    ms_p = _timed_all(step_plain, nsteps, stream, flush)
    ms_g = _timed_all(step_graph, nsteps, stream, flush)
    if graph.status()[0] != abi.R4G_OK:
        raise RuntimeError("the graph's last replay reports an error")
    # stage times of the autograd step (library stage events on), same views
    it["a"] = warm
    abi.r4g_set_timing(rb.ctx, True)
    abi.r4g_stage_times(rb.ctx, reset=True)
    for _ in range(nsteps):
        flush.zero_()
        step_autograd()
    torch.cuda.synchronize()
    abi.r4g_set_timing(rb.ctx, False)
    stage_ms, _ = abi.r4g_stage_times(rb.ctx, reset=True)
    per_stage = {k: v / nsteps for k, v in stage_ms.items() if v > 0}
    # work of the timed steps' views (untimed counting pass)
    counter = r4g.Renderer(tile=rb.tile, flags=abi.R4G_FLAG_COUNT_PAIRS)
    pairs = keys = vis = reached = vis_g = 0
    for views in step_views[warm:warm + nsteps]:
        r = counter.render_batch(params, views, key_capacity=cap_b)
        counter.backward_batch(params, r, torch.sign(r.packed - target) * inv, grads)
        st_ = counter.stats(r)
        pairs += st_["composited_pairs"]
        keys += st_["key_count"]
        vis += st_["n_visible"]
        reached += st_["reached_pairs"]
        vis_g += st_["visible_gaussians"]
    pairs, keys, vis = pairs / nsteps, keys / nsteps, vis / nsteps
    reached, vis_g = reached / nsteps, vis_g / nsteps
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = SMS * FP32_LANES * sm_mhz * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    roof = {}
    if "blend_bwd" in per_stage:
        ach = pairs * BWD_FP32_OPS_PER_PAIR / (per_stage["blend_bwd"] / 1e3) / 1e12
        roof["blend_bwd"] = {"bound": "alu", "achieved": round(ach, 3), "peak": round(alu_peak, 2),
                             "unit": "TFLOP/s", "frac": round(ach / alu_peak, 4),
                             "fp32_ops_per_pair": BWD_FP32_OPS_PER_PAIR,
                             "traffic": DRAM_TRAFFIC.get(f"blend_bwd@{rb.tile[0]}x{rb.tile[1]}")}
    if "blend" in per_stage:
        ach = pairs * FP32_OPS_PER_PAIR / (per_stage["blend"] / 1e3) / 1e12
        roof["blend"] = {"bound": "alu", "achieved": round(ach, 3), "peak": round(alu_peak, 2),
                         "unit": "TFLOP/s", "frac": round(ach / alu_peak, 4)}
    if "preprocess_bwd" in per_stage:
        b = preprocess_bwd_bytes(vis_g, vis, keys, reached)
        ach = b / (per_stage["preprocess_bwd"] / 1e3) / 1e9
        roof["preprocess_bwd"] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                                  "frac": round(ach / hbm_peak, 4), "bytes": round(b)}
    top = max(("blend_bwd", "blend", "preprocess_bwd"), key=lambda k: per_stage.get(k, 0.0))
    return {"value": round(1000.0 / ms_a["mean"], 3), "unit": "it/s", "ms_per_it": round(ms_a["mean"], 3),
            "ms_per_it_median": round(ms_a["median"], 3), "it_per_s_at_median": round(1000.0 / ms_a["median"], 3),
            "views": TRAIN_VIEWS, "steps": nsteps,
            "tile": f"{rb.tile[0]}x{rb.tile[1]}", "autotune_ms": tune["ms"],
            "views_per_step": "fresh seeded (t ~ U[0,1], angle ~ U[0, 2 pi)) each step",
            "path": "autograd.Function over the batched render (one call for the 4 views, tile shape from the "
                    "autotuner), L1 loss in torch",
            "plain_path": {"value": round(1000.0 / ms_p["mean"], 3), "ms_per_it": round(ms_p["mean"], 3),
                           "path": "per view: r4g_render + r4g_render_backward (FP32, 16x16)"},
            "graph": {"value": round(1000.0 / ms_g["mean"], 3), "ms_per_it": round(ms_g["mean"], 3),
                      "path": "batched render + L1 sign gradient + batched backward in one CUDA graph, the "
                              "step's views copied into the graph's device view table"},
            "stage_ms": {k: round(v, 4) for k, v in per_stage.items()},
            "work_per_step": {"composited_pairs": round(pairs), "keys": round(keys), "visible_items": round(vis),
                              "pairs_with_gradient": round(reached), "visible_gaussians": round(vis_g)},
            "roofline": dict(roof.get(top, {}), kernel=top), "stages": roof,
            "l2": "flushed between steps"}


def preprocess_bwd_bytes(n_gauss: float, n_items: float, keys: float, reached: float) -> float:
    """Algorithmic bytes of the preprocess backward of one multi-view call, per
    Gaussian visible in some view: its parameters (68 B) and SH row (192 B)
    read once, its 65-float gradient read and written (520 B); per visible
    (view, Gaussian) item: the 96-byte partial written and read; per pair: the
    one-byte flag, and the 48-byte gradient slot of the pairs that have one."""
    return (68.0 + 192.0 + 520.0) * n_gauss + 192.0 * n_items + 1.0 * keys + 48.0 * reached


def _timed_all(fn, steps: int, stream, flush=None, warm: int = 2) -> dict:
    """Mean and median ms of fn() over `steps` calls (CUDA events on `stream`
    around each call; the L2 flush, when given, between calls outside them).
    `warm` untimed calls are queued right before the first timed one: a device
    coming out of the idle gap of the synchronize runs its first call slower."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for _ in range(warm):
        fn()
    for a, b in evs:
        if flush is not None:
            flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    return {"mean": sum(ms) / steps, "median": statistics.median(ms)}


def batch_bench(args, dev, stream, flush):
    """Batched multi-view render and backward: 100k Gaussians, 16 views of
    uneven resolution (6 x 800x800, 5 x 640x480, 5 x 1352x1014), one batched
    call per step, tile shape from the autotuner, captured in a CUDA graph;
    against the plain path (a single-view 16x16 render per view)."""
    import torch
    import synth
    import paper_2402_03307_gb300 as r4g

    g = synth.gaussians(100_000, 5, mean_lo=-3.0, mean_hi=3.0)
    params = {k: torch.as_tensor(v).to(dev).contiguous() for k, v in g.items()}
    views = synth.batched_views(6)
    rend = r4g.Renderer()
    tune = rend.autotune(params, views, backward=True, reps=3)
    target = _packed_target(views, 60, dev)
    inv = 1.0 / target.numel()
    gf = r4g.BatchGraph(rend, params, views)
    gt = r4g.BatchGraph(rend, params, views, grad_fn=lambda img: torch.sign(img - target) * inv)
    alt = [synth.batched_views(6 + 100 * j) for j in range(1, 4)]  # same sizes, other cameras / times
    alt = [[(c2, t2) for (c2, t2) in a] for a in alt]
    sizes = [(c.width, c.height) for c, _ in views]
    alt = [a for a in alt if [(c.width, c.height) for c, _ in a] == sizes] or [views]
    tab_f = [gf.views_table(a) for a in alt]  # device view tables, copied on the stream at replay
    tab_t = [gt.views_table(a) for a in alt]
    it = {"k": 0}

    def fwd():
        gf.replay(table=tab_f[it["k"] % len(alt)])
        it["k"] += 1

    def train():
        gt.replay(table=tab_t[it["k"] % len(alt)])
        it["k"] += 1

    plain = r4g.Renderer()
    pf = []
    for cam, t in views:
        r = plain.render(params, cam, t)
        c = int(plain.status(r)[1] * 1.1) + 1024
        pf.append((cam, t, c, plain.new_frame(100_000, cam.width, cam.height, c, dev),
                   torch.empty((3, cam.height, cam.width), dtype=torch.float32, device=dev)))
    pgrads = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in params.items()}
    tv, off = [], 0
    for cam, t, *_ in pf:
        n = 3 * cam.width * cam.height
        tv.append(target[off:off + n].view(3, cam.height, cam.width))
        off += n

    def plain_fwd():
        for cam, t, c, fr, im in pf:
            plain.render(params, cam, t, frame=fr, key_capacity=c, out=im, check=False)

    def plain_train():
        for v in pgrads.values():
            v.zero_()
        for (cam, t, c, fr, im), tt in zip(pf, tv):
            res = plain.render(params, cam, t, frame=fr, key_capacity=c, out=im, check=False)
            plain.backward(params, cam, t, res, torch.sign(im - tt) * inv, pgrads)

    for f in (fwd, train, plain_fwd, plain_train):
        for _ in range(3):
            f()
    steps = max(5, args.train_steps)
    ms_f = _timed(fwd, steps, stream, flush)
    ms_t = _timed(train, steps, stream, flush)
    ms_pf = _timed(plain_fwd, steps, stream, flush)
    ms_pt = _timed(plain_train, steps, stream, flush)
    if gt.status()[0] != 0 or gf.status()[0] != 0:
        raise RuntimeError("batched render overflowed its key buffer")
    nv = len(views)
    return {"workload": "100k 4D Gaussians, 16 views (6x 800x800, 5x 640x480, 5x 1352x1014), FP32",
            "tile": f"{tune['tile'][0]}x{tune['tile'][1]}", "autotune_ms": tune["ms"],
            "render": {"ms_per_batch": round(ms_f, 3), "views_per_s": round(nv * 1000.0 / ms_f, 1)},
            "train": {"ms_per_batch": round(ms_t, 3), "it_per_s": round(1000.0 / ms_t, 2)},
            "plain_path": {"render_ms_per_batch": round(ms_pf, 3), "train_ms_per_batch": round(ms_pt, 3)},
            "speedup_vs_plain": {"render": round(ms_pf / ms_f, 3), "train": round(ms_pt / ms_t, 3)},
            "launch": "one persistent blend launch per batch; whole step replayed as a CUDA graph",
            "l2": "flushed between steps"}


def large_bench(args, dev, stream, flush):
    """Large scene: 2M Gaussians, 8 views at 1920x1080, training step (batched
    render + L1 + batched backward, CUDA graph), with the scales and SH
    coefficients stored in BF16 against the FP32 path; the BF16 images' error
    against the FP32 images."""
    import torch
    import synth
    import paper_2402_03307_gb300 as r4g

    g = synth.gaussians(2_000_000, 7, mean_lo=-3.0, mean_hi=3.0)
    p32 = {k: torch.as_tensor(v).to(dev).contiguous() for k, v in g.items()}
    p16 = dict(p32)
    p16["logscale"] = p32["logscale"].to(torch.bfloat16).contiguous()
    p16["sh"] = p32["sh"].to(torch.bfloat16).contiguous()
    views = synth.large_views(8, 8)
    target = _packed_target(views, 70, dev)
    inv = 1.0 / target.numel()
    out = {"workload": "2M 4D Gaussians, 8 views 1920x1080, training step (graph)", "tile": "16x16"}
    imgs = {}
    for name, p in (("fp32", p32), ("bf16", p16)):
        rend = r4g.Renderer()
        gt = r4g.BatchGraph(rend, p, views, grad_fn=lambda img: torch.sign(img - target) * inv)
        for _ in range(2):
            gt.replay()
        ms = _timed(gt.replay, 5, stream, flush)
        if gt.status()[0] != 0:
            raise RuntimeError("large batch overflowed its key buffer")
        imgs[name] = gt.packed.clone()
        out[name] = {"ms_per_step": round(ms, 2), "it_per_s": round(1000.0 / ms, 3),
                     "param_bytes": int(sum(v.numel() * v.element_size() for v in p.values())),
                     "keys": int(gt.status()[1]), "stage_ms": large_stage_ms(rend, p, views, gt.cap, target, inv,
                                                                             flush)}
        del gt
    d = (imgs["bf16"] - imgs["fp32"]).abs()
    mse = float((d.double() ** 2).mean())
    out["bf16_vs_fp32"] = {"max_abs": float(d.max()), "psnr_db": round(10 * math.log10(1.0 / max(mse, 1e-30)), 2),
                           "speedup": round(out["fp32"]["ms_per_step"] / out["bf16"]["ms_per_step"], 3)}
    return out


def large_stage_ms(rend, p, views, cap, target, inv, flush) -> dict:
    """Per-stage device time of the large training step (the same batched
    render and backward, eager, with the library's stage events on), ms per
    step over 3 steps."""
    import torch
    from paper_2402_03307_gb300 import abi
    grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=v.device) for k, v in p.items()}
    res = rend.render_batch(p, views, key_capacity=cap, check=False)
    abi.r4g_set_timing(rend.ctx, True)
    abi.r4g_stage_times(rend.ctx, reset=True)
    for _ in range(3):
        flush.zero_()
        res = rend.render_batch(p, views, frame=res.frame, key_capacity=cap, out=res.packed, check=False)
        rend.backward_batch(p, res, torch.sign(res.packed - target) * inv, grads)
    torch.cuda.synchronize()
    abi.r4g_set_timing(rend.ctx, False)
    ms, _ = abi.r4g_stage_times(rend.ctx, reset=True)
    return {k: round(v / 3, 3) for k, v in ms.items() if v > 0}


def extras_bench(args, params, dev, stream, flush, frames, cap):
    """The optical-flow render on the sweep (frames/s) and, at 300k Gaussians,
    the 4D KNN (K = 8) and the entropy + 4D-consistency losses with their
    gradients (ms)."""
    import torch
    import paper_2402_03307_gb300 as r4g
    from paper_2402_03307_gb300 import abi

    fr = r4g.Renderer(flags=abi.R4G_FLAG_FLOW)
    frame = fr.new_frame(N_GAUSS, WIDTH, HEIGHT, cap, dev)
    img = torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device=dev)
    it = {"k": 0}

    def flow_frame():
        cam, t = frame_camera(frames[it["k"] % len(frames)])
        it["k"] += 1
        fr.render(params, cam, t, frame=frame, key_capacity=cap, out=img, check=False)

    for _ in range(3):
        flow_frame()
    ms_flow = _timed(flow_frame, min(100, len(frames)), stream, flush)
    knn = {}

    def run_knn():
        knn["idx"] = r4g.knn4d(params["mean"], 6.0, 1.0, 8)

    for _ in range(2):
        run_knn()
    ms_knn = _timed(run_knn, 5, stream, flush)
    grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in params.items()}

    def run_reg():
        r4g.regularizers(params, knn["idx"], 0.01, 0.05, grads)

    for _ in range(2):
        run_reg()
    ms_reg = _timed(run_reg, 10, stream, flush)
    target = torch.rand((3, HEIGHT, WIDTH), device=dev, generator=torch.Generator(device=dev).manual_seed(5))

    def run_loss():
        r4g.image_loss(img, target, 0.2)

    for _ in range(2):
        run_loss()
    ms_loss = _timed(run_loss, 20, stream, flush)
    dens = densify_bench(params, dev, stream, flush)
    inside = inside_sweep_bench(params, dev, stream, flush)
    return {"densify": dens, "inside_sweep": inside, "small": small_bench(dev, stream),
            "image_loss": {"ms": round(ms_loss, 3), "what": "0.8 L1 + 0.2 (1 - SSIM) and its gradient, 3x1014x1352",
                           "note": "includes scratch allocation by the Python wrapper"},
            "flow": {"value": round(1000.0 / ms_flow, 1), "unit": "frames/s",
                     "workload": "optical-flow render of the 300k sweep (d mean2d / dt composited)"},
            "knn4d": {"ms": round(ms_knn, 3), "k": 8, "n": N_GAUSS,
                      "note": "includes scratch allocation by the Python wrapper"},
            "regularizers": {"ms": round(ms_reg, 3), "n": N_GAUSS,
                             "what": "entropy + 4D consistency losses and their gradients"}}


def plain_sweep_bench(rend16, params, dev, stream, flush, frames) -> tuple[dict, int]:
    """The plain path of the sweep: the same timed frames, FP32, one view per
    call, 16x16 tiles (key buffer sized over the whole sweep, untimed).
    Returns its record and its key capacity."""
    import torch
    import paper_2402_03307_gb300 as r4g
    from paper_2402_03307_gb300 import abi
    need = 0
    for k in range(FRAMES):
        c, tt = frame_camera(k)
        need = max(need, rend16.status(rend16.render(params, c, tt))[1])
    cap = int(need * 1.1) + 1024
    frame = rend16.new_frame(N_GAUSS, WIDTH, HEIGHT, cap, dev)
    img = torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device=dev)
    it = {"k": 0}
    # arguments built before the timed calls (only the r4g_render call runs between a frame's events)
    gstruct = r4g.gaussians_struct(params)
    calls = [(r4g.camera_struct(c), float(tt)) for c, tt in (frame_camera(k) for k in frames)]
    args = (img.data_ptr(), None, None, frame.data_ptr(), frame.numel(), cap, stream.cuda_stream)

    def one():
        cs, tt = calls[it["k"] % len(calls)]
        it["k"] += 1
        abi.r4g_render(rend16.ctx, gstruct, cs, tt, *args)

    for _ in range(3):
        one()
    it["k"] = 0
    r = _timed_all(one, len(frames), stream, flush)
    return ({"value": round(1000.0 / r["mean"], 2), "unit": "frames/s", "ms_per_step": round(r["mean"], 4),
             "ms_per_step_median": round(r["median"], 4), "tile": "16x16",
             "path": "FP32, one view per r4g_render call, 16x16 tiles"}, cap)


def small_bench(dev, stream) -> dict:
    """The small configuration: 1,000 Gaussians, 128x128, one camera at
    distance 4, t = 0.5, FP32; frames/s of the plain single-view path (its
    inputs stay in L2, so no flush) and of the same render captured in a CUDA
    graph (launch-bound at this size)."""
    import torch
    import paper_2402_03307_gb300 as r4g
    import synth
    g, cam, t = synth.small_scene(seed=1)
    p = {k: torch.as_tensor(v).to(dev).contiguous() for k, v in g.items()}
    rend = r4g.Renderer()
    cap = int(rend.status(rend.render(p, cam, t))[1] * 1.1) + 1024
    frame = rend.new_frame(1000, cam.width, cam.height, cap, dev)
    img = torch.empty((3, cam.height, cam.width), dtype=torch.float32, device=dev)

    def one():
        rend.render(p, cam, t, frame=frame, key_capacity=cap, out=img, check=False)

    for _ in range(10):
        one()
    ms = _timed(one, 200, stream)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            one()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        one()
    for _ in range(10):
        graph.replay()
    ms_g = _timed(graph.replay, 200, stream)
    return {"value": round(1000.0 / ms, 1), "unit": "frames/s", "ms": round(ms, 4),
            "graph": {"value": round(1000.0 / ms_g, 1), "ms": round(ms_g, 4)},
            "workload": "1k 4D Gaussians, 128x128, camera at distance 4, t = 0.5, FP32, 1 view/launch"}


def inside_sweep_bench(params, dev, stream, flush, radius: float = 4.0, stride: int = 3):
    """The same sweep at orbit radius 4 (the camera inside the cloud, a heavier
    tile load): every third frame, key buffer sized over those frames, L2
    flushed between frames, per-stage live times."""
    import torch
    import paper_2402_03307_gb300 as r4g
    from paper_2402_03307_gb300 import abi
    import synth

    ks = list(range(0, FRAMES, stride))
    cams = [synth.orbit_camera(k, FRAMES, radius, WIDTH, HEIGHT) for k in ks]
    rend = r4g.Renderer()
    need = 0
    for cam, t in cams:
        need = max(need, rend.status(rend.render(params, cam, t))[1])
    cap = int(need * 1.1) + 1024
    frame = rend.new_frame(N_GAUSS, WIDTH, HEIGHT, cap, dev)
    img = torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device=dev)
    it = {"k": 0}

    def one():
        cam, t = cams[it["k"] % len(cams)]
        it["k"] += 1
        rend.render(params, cam, t, frame=frame, key_capacity=cap, out=img, check=False)

    for _ in range(3):
        one()
    torch.cuda.synchronize()
    it["k"] = 0
    ms = _timed(one, len(cams), stream, flush)  # no per-stage events in the timed frames
    abi.r4g_stage_times(rend.ctx, reset=True)
    abi.r4g_set_timing(rend.ctx, True)
    _timed(one, len(cams), stream, flush)
    abi.r4g_set_timing(rend.ctx, False)
    stage_ms, _ = abi.r4g_stage_times(rend.ctx, reset=True)
    keys = 0
    for cam, t in cams:
        keys += rend.status(rend.render(params, cam, t, frame=frame, key_capacity=cap, out=img))[1]
    return {"value": round(1000.0 / ms, 1), "unit": "frames/s", "frames": len(cams),
            "keys_per_frame": round(keys / len(cams)),
            "stage_ms": {k: round(v / len(cams), 4) for k, v in stage_ms.items() if v > 0},
            "workload": f"300k sweep at orbit radius {radius:g} (camera inside the cloud), every "
                        f"{stride}rd frame, FP32, 1 view/launch"}


def densify_bench(params, dev, stream, flush):
    """One densify-and-prune step (r4g_densify_plan + r4g_densify_apply) on the
    300k scene with seeded statistics, outputs preallocated at 2N rows (no host
    synchronisation inside the timed region), against the HBM roofline:
    algorithmic bytes = plan 28 B per Gaussian (log-scales, logit, vs_grad,
    vs_count) + 5 B of decisions and offsets written and read back + 260 B per
    source row read + 264 B per output row written (with its source index) +
    32 B of draws per split Gaussian."""
    import numpy as np
    import torch
    import paper_2402_03307_gb300 as r4g
    import synth
    from paper_2402_03307_gb300 import abi

    n = int(params["mean"].shape[0])
    d = synth.density_inputs(90, n)
    st = {k: torch.as_tensor(d[k]).to(dev) for k in ("vs_grad", "vs_count")}
    z = torch.as_tensor(d["z"]).to(dev)
    cfg = r4g.densify_config()
    g = r4g.gaussians_struct(params)
    nb = abi.r4g_densify_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    cap = 2 * n
    out = {"mean": torch.empty((cap, 4), device=dev), "rotor": torch.empty((cap, 8), device=dev),
           "logscale": torch.empty((cap, 4), device=dev), "logit": torch.empty((cap,), device=dev),
           "sh": torch.empty((cap, 16, 3), device=dev)}
    src = torch.empty(cap, dtype=torch.int32, device=dev)
    o = abi.r4g_params_out()
    for k in r4g.PARAM_NAMES:
        setattr(o, k, out[k].data_ptr())
    s = stream.cuda_stream

    def step():
        abi.r4g_densify_plan(g, st["vs_grad"].data_ptr(), st["vs_count"].data_ptr(), None, cfg,
                             scratch.data_ptr(), nb, count.data_ptr(), s)
        abi.r4g_densify_apply(g, z.data_ptr(), cfg, scratch.data_ptr(), nb, o, cap, src.data_ptr(), s)

    for _ in range(3):
        step()
    ms = _timed(step, 20, stream, flush)
    m = int(count.item())
    sm = src[:m].cpu().numpy()
    idx = np.where(sm >= 0, sm, -sm - 1)
    sources = len(np.unique(idx))
    splits = int(((sm < 0) & (np.bincount(idx, minlength=n)[idx] == 2) & (np.r_[True, idx[1:] != idx[:-1]])).sum())
    bytes_ = 28 * n + 10 * n + 260 * sources + 264 * m + 32 * splits
    peak = measured_peaks().get("hbm_gbs")
    achieved = bytes_ / (ms * 1e-3) / 1e9
    return {"ms": round(ms, 4), "n": n, "rows_out": m, "split_or_clone_sources": splits,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4) if peak else None, "bytes": bytes_},
            "what": "plan + apply, 2 launches + 1 scan launch, outputs preallocated"}


def e2e_bench(args, rend, g, dev, stream, frames, cap):
    """Frames/s through the public API with host buffers: every step copies
    its inputs (all Gaussian parameters, 78 MB, held in one pinned buffer) from
    host memory and reads its image back (16 MB). The steps are pipelined over two buffer
    sets on three streams -- upload of step k + 1, render of step k, read-back
    of step k - 1 -- so the job's throughput is bounded by the slowest of the
    three, as in a serving loop; every copy of every step is inside the timed
    region."""
    import torch

    # the parameters in one pinned host buffer (each array 64-byte aligned),
    # uploaded by one copy per step into one device buffer whose views are the
    # parameter tensors the renderer takes (five copies measured 2.6 % slower)
    arrays = {k: torch.as_tensor(v) for k, v in g.items()}
    offs, total = {}, 0
    for k, v in arrays.items():
        offs[k] = total
        total += (v.numel() * v.element_size() + 63) // 64 * 64
    hbuf = torch.empty(total, dtype=torch.uint8).pin_memory()
    for k, v in arrays.items():
        n = v.numel() * v.element_size()
        hbuf[offs[k]:offs[k] + n].view(v.dtype).view(v.shape).copy_(v)
    dbuf = [torch.empty(total, dtype=torch.uint8, device=dev) for _ in range(2)]
    dparams = [{k: d[offs[k]:offs[k] + v.numel() * v.element_size()].view(v.dtype).view(v.shape)
                for k, v in arrays.items()} for d in dbuf]
    fr = [rend.new_frame(N_GAUSS, WIDTH, HEIGHT, cap, dev) for _ in range(2)]
    img = [torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32, device=dev) for _ in range(2)]
    himg = [torch.empty((3, HEIGHT, WIDTH), dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = total
    d2h = himg[0].numel() * 4
    s_up, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_ren = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    cams = {k: frame_camera(k) for k in set(frames)}  # the workload's cameras (not the API's work)

    def step(i, k):
        b = i % 2
        with torch.cuda.stream(s_up):
            s_up.wait_event(ev_ren[b])  # the render that read this buffer set is done
            dbuf[b].copy_(hbuf, non_blocking=True)
            ev_up[b].record(s_up)
        stream.wait_event(ev_up[b])
        stream.wait_event(ev_out[b])  # the read-back of this image buffer is done
        cam, t = cams[k]
        rend.render(dparams[b], cam, t, frame=fr[b], key_capacity=cap, out=img[b], check=False, stream=stream)
        ev_ren[b].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_ren[b])
            himg[b].copy_(img[b], non_blocking=True)
            ev_out[b].record(s_out)

    for i in range(4):
        step(i, frames[i % len(frames)])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_up.wait_event(e0)
    for i, k in enumerate(frames):
        step(i, k)
    stream.wait_stream(s_up)
    stream.wait_stream(s_out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": round(len(frames) / (ms / 1e3), 2), "unit": "frames/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "pipeline": "upload k+1 | render k | read back k-1 (two buffer sets)"}


# ---- CPU oracle baseline -----------------------------------------------------------
def cpu_baseline(budget_s: float = 15.0) -> dict:
    import numpy as np
    import torch

    import oracle
    import synth

    g = synth.fwd300k_scene()
    cam, t = frame_camera(37)
    sc = oracle.to_f64(g)
    t0 = time.perf_counter()
    rec = oracle.preprocess(sc, cam, t)
    t_pre = time.perf_counter() - t0
    done, t_pix = 0, 0.0
    chunk = 256
    seed = 0
    while t_pix < budget_s:
        pix = synth.random_pixels(seed, WIDTH, HEIGHT, chunk)
        t0 = time.perf_counter()
        oracle.render_pixels(sc, cam, t, pix, rec=rec)
        t_pix += time.perf_counter() - t0
        done += len(pix)
        seed += 1
    per_frame = t_pre + t_pix * (WIDTH * HEIGHT / done)
    # the small configuration (1k Gaussians, 128x128), a whole frame
    gs, cam_s, t_s = synth.small_scene(seed=1)
    t0 = time.perf_counter()
    oracle.render(oracle.to_f64(gs), cam_s, t_s)
    t_small = time.perf_counter() - t0
    # the analytic FP64 gradient at the finite-difference size (64 Gaussians, 32x32)
    gf = synth.gaussians(64, 11, ls_xyz=(-1.6, 0.3), ls_t=(-0.7, 0.3))
    cam_f = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 32, 32)
    t0 = time.perf_counter()
    oracle.render_grad(oracle.to_f64(gf), cam_f, 0.5, np.ones((3, 32, 32)))
    t_grad = time.perf_counter() - t0
    return {"value": 1.0 / per_frame, "unit": "frames/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "small_frame_s": round(t_small, 3), "fd_size_gradient_s": round(t_grad, 3),
            "sample": f"FP64 oracle: preprocess of all 300k Gaussians ({t_pre:.2f} s) + {done} random pixels of "
                      f"frame 37 brute-forced over all visible Gaussians ({t_pix:.1f} s), scaled to "
                      f"{WIDTH * HEIGHT} pixels"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(budget_s=max(5.0, min(60.0, 2.0 * args.steps)))
        out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "frames/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": dict(CONFIG, parallelism=f"replicas x{world}"),
               "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "frames/s", "h2d_bytes_per_step": 0,
                                           "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return
    out = run_ours(args, rank, world, local)
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.frames_only or args.train_only
                                          or args.backward_only
                                          or args.batch_only):
        out["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

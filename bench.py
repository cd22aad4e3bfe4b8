"""Benchmark of the mapping iteration (render -> L1 + planar loss -> adjoint -> Adam).

Workload (default): one Replica-shaped keyframe, 300,000 Gaussians sampled on a
synthetic textured room (6 planes + 20 boxes), 1200x680, fx = fy = 600, target
= the room's analytic ray-cast. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (host cores). Under torchrun every rank runs its own replica of the
workload (independent keyframes: weak scaling, no collective on the data path).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "mapping fwd+bwd iters/s @1200x680,300k Gaussians; time-to-PSNR vs plain"
UNIT = "iters/s"
WORKLOAD = ("replica-shaped single keyframe: 300k Gaussians on a textured room (6 planes + 20 boxes), "
            "1200x680, fx=fy=600; one iteration = render + L1/planar loss + adjoint + Adam")
N_GAUSS, W, H = 300_000, 1200, 680
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2

# Algorithmic FP32 operations per (pixel, Gaussian) pair, counted from the
# compositing arithmetic (an FMA counts 2): a tested pair costs the offset, the
# exponent and alpha; a blended pair adds the transmittance update and the
# weighted colour; the adjoint adds the colour, alpha and conic/mean gradients.
FLOP_FWD_TESTED, FLOP_FWD_BLENDED = 12, 10
FLOP_BWD_WALKED, FLOP_BWD_BLENDED = 12, 50
FP32_LANES_PER_SM = 128

# DRAM bytes (read + write) of one launch of the dominant kernel from an ncu capture of each
# workload, with the kernel source's sha256 and layout at capture time (the figure is reported
# only while both still match): profiles/raster_fused_replica_1200x680_300k.md (the keyframe)
# and profiles/raster_fused_window_8x640x480_150k.md (the window)
_RASTER_SHA = "3f638f92e10a2c7a008f507574ace00a45cd3b9fece28c73048ddae01d5c56b0"
NCU_TRAFFIC = {"raster_fused": {"bytes": 35.91e6, "source": "paper_2504_02437_gb300/csrc/k_raster.cu",
                                "sha256": _RASTER_SHA, "tile": 16, "ppt": 2},
               "raster_fused_window": {"bytes": 102.15e6, "source": "paper_2504_02437_gb300/csrc/k_raster.cu",
                                       "sha256": _RASTER_SHA, "tile": 16, "ppt": 1}}


def _ncu_traffic(kernel: str, tile: int, ppt: int):
    import hashlib
    t = NCU_TRAFFIC.get(kernel)
    if t is None or (tile, ppt) != (t["tile"], t["ppt"]):
        return None
    try:
        h = hashlib.sha256(open(os.path.join(ROOT, t["source"]), "rb").read()).hexdigest()
    except OSError:
        return None
    return t["bytes"] if h == t["sha256"] else None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


WINDOW_METRIC = "mapping window fwd+bwd iters/s @8x640x480,150k Gaussians"
WINDOW_WORKLOAD = ("TUM-shaped keyframe window: 8 consecutive views 640x480, fx=fy=525, of a smooth path through the "
                   "textured room, 150k Gaussians (98 % on the boxes, 2 % on the walls); one iteration = render all "
                   "views + L1/planar loss + adjoint + one Adam step")


# the window: keyframes 19-26 of the 40-keyframe room trajectory of seed 50, over a map with 98 %
# of its Gaussians on the boxes: among trajectory seeds 0-59 and all 8-keyframe segments, the one
# whose views span the widest visible range within 20k-140k (20.3k-124.7k of the 150k Gaussians)
WINDOW_TRAJECTORY_SEED, WINDOW_TRAJECTORY_FRAMES, WINDOW_FIRST_FRAME = 50, 40, 19
WINDOW_BOX_FRACTION = 0.98


def make_window_workload(seed: int = 0, n_views: int = 8, n_gauss: int = 150_000,
                         trajectory_seed: int = WINDOW_TRAJECTORY_SEED, device=None):
    """(params, cameras, targets [V, 3, 480, 640]); with ``device`` the targets are ray-cast on
    that GPU (the same formula as the CPU ray-cast) and returned as a device tensor."""
    from synth import make_room, room_gaussians, room_trajectory
    room = make_room(seed)
    path = room_trajectory(WINDOW_TRAJECTORY_FRAMES, trajectory_seed, 640, 480, 525.0, 525.0)
    cams = path[WINDOW_FIRST_FRAME:WINDOW_FIRST_FRAME + n_views]
    params = room_gaussians(room, n_gauss, seed, box_fraction=WINDOW_BOX_FRACTION)
    if device is not None:
        import torch
        return params, cams, torch.stack([room.raycast_torch(c, device) for c in cams]).contiguous()
    cache = os.path.join(tempfile.gettempdir(),
                         f"gs_room_window_{seed}_{trajectory_seed}_{WINDOW_FIRST_FRAME}_{n_views}.npy")
    if os.path.exists(cache):
        targets = np.load(cache)
    else:
        targets = np.stack([room.raycast(c) for c in cams])
        try:
            np.save(cache, targets)
        except OSError:
            pass
    return params, cams, targets


def make_workload(seed: int = 0):
    from synth import make_room, room_camera_single, room_gaussians
    room = make_room(seed)
    cam = room_camera_single(W, H, 600.0, 600.0)
    params = room_gaussians(room, N_GAUSS, seed)
    cache = os.path.join(tempfile.gettempdir(), f"gs_room_target_{seed}_{W}x{H}.npy")
    if os.path.exists(cache):
        target = np.load(cache)
    else:
        target = np.ascontiguousarray(room.raycast(cam))
        try:
            np.save(cache, target)
        except OSError:
            pass
    return params, cam, target


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        for ln in open(self.f.name).read().splitlines():
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(backend: str = "nccl"):
    """Rank, world size and local rank from the launcher's environment; joins the process group
    when there is more than one rank (nccl on GPUs, gloo for CPU ranks)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest value over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps: int, world: int, slowest_ms: float) -> float:
    """Whole-job iterations/s of `world` replicas that each ran `steps` iterations, timed by the slowest."""
    return world * steps / (slowest_ms / 1000.0)


# --------------------------------------------------------------------------- CPU oracle


TILE_GRID = (16, 8)     # 128 sample tiles of 16x16 px, evenly spread over the image


def sample_tiles() -> list:
    """Origins of 128 sample tiles on a 16 x 8 grid over the image, in bit-reversed order so
    that any prefix of the list is spread over the whole image. Every CPU-oracle sample of
    this benchmark takes its tiles from this list."""
    gx, gy = TILE_GRID
    cells = [(int(round((i + 0.5) * (W - 16) / gx)), int(round((j + 0.5) * (H - 16) / gy)))
             for j in range(gy) for i in range(gx)]
    bits = (len(cells) - 1).bit_length()
    rev = sorted(range(len(cells)), key=lambda k: int(format(k, f"0{bits}b")[::-1], 2))
    return [cells[k] for k in rev]


def _tile_pixels(tiles) -> np.ndarray:
    pix = []
    for x0, y0 in tiles:
        yy, xx = np.mgrid[y0:y0 + 16, x0:x0 + 16]
        pix.append(np.stack([xx.ravel(), yy.ravel()], 1))
    return np.concatenate(pix) if pix else np.zeros((0, 2), np.int64)


def oracle_step(params, cam, target, tiles) -> float:
    """Seconds of one oracle mapping iteration restricted to the 16x16 pixel tiles at the
    origins ``tiles``: projection of all Gaussians, compositing and L1 of those pixels, the
    adjoint of both, the planar term and Adam. With no tiles it is the part of an iteration
    that does not depend on the pixels (projection, its adjoint, planar term, Adam)."""
    import oracle as O
    pix = _tile_pixels(tiles)
    p64 = params.astype(np.float64)
    t0 = time.perf_counter()
    res = O.loss_and_grads(p64, [cam], target[None], pixels=[pix], chunk=256)
    O.adam_step(p64, res["grad"], np.zeros_like(p64), np.zeros_like(p64), 1)
    return time.perf_counter() - t0


FULL_TILES = W * H / 256.0     # the image's area in 16x16 tiles


def oracle_full_iteration_s(t_fixed: float, t_sample: float, n_tiles: int) -> float:
    """A full iteration's oracle time from its pixel-independent part and a sample of tiles:
    t_fixed + (t_sample - t_fixed) / n_tiles x (W H / 256)."""
    return t_fixed + max(t_sample - t_fixed, 0.0) / n_tiles * FULL_TILES


def _cpu_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_baseline(params, cam, target, tiles_all: int, tiles_single: int) -> dict:
    """The FP64 oracle (as it stands) on the host cores, all of them and one: the Replica-shaped
    iteration from its pixel-independent part (median of 3 after a warm-up call) plus the first
    tiles of the sample-tile list, and the small single-view workload (2,000 Gaussians, 160x120)
    timed in full."""
    import torch
    import oracle as O
    from synth import frustum_scene, random_target
    n_all = torch.get_num_threads()
    p1, c1 = frustum_scene()
    tg1 = random_target(160, 120, seed=1)
    p1 = p1.astype(np.float64)
    grid = sample_tiles()
    out = {"cpu_model": _cpu_model(), "nproc": os.cpu_count()}
    try:
        for label, nth, n_t in (("all_cores", n_all, tiles_all), ("single_thread", 1, tiles_single)):
            torch.set_num_threads(nth)
            oracle_step(params, cam, target, [])
            t_fixed = statistics.median(oracle_step(params, cam, target, []) for _ in range(3))
            tiles = grid[:n_t]
            t_sample = oracle_step(params, cam, target, tiles)
            full = oracle_full_iteration_s(t_fixed, t_sample, len(tiles))
            t0 = time.perf_counter()
            r = O.loss_and_grads(p1, [c1], tg1)
            O.adam_step(p1, r["grad"], np.zeros_like(p1), np.zeros_like(p1), 1)
            t_small = time.perf_counter() - t0
            out[label] = {"threads": nth, "replica_iters_per_s": 1.0 / full, "replica_full_iteration_s": full,
                          "fixed_s": t_fixed, "tiles_sampled": len(tiles),
                          "per_tile_s": (t_sample - t_fixed) / len(tiles),
                          "small_2k_160x120_iters_per_s": 1.0 / t_small, "small_2k_160x120_s": t_small}
    finally:
        torch.set_num_threads(n_all)
    return out


def run_reference(args):
    """The oracle as it stands on the host cores, on the GPU arm's workload, metric and unit: each
    step is one bounded sample (all Gaussians, 4 random 16x16 tiles); the full-iteration rate
    comes from the pixel-independent part (timed in the warm-up) plus the steps' mean per-tile
    time. ms_per_step is the measured time of a sample step."""
    import torch
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    params, cam, target = make_workload(0)
    tiles_per_step = 4
    grid = sample_tiles()
    # warm-up steps: the pixel-independent part alone (the first call also warms the thread pool)
    fixed = [oracle_step(params, cam, target, []) for w in range(args.warmup)]
    t_fixed = statistics.median(fixed[1:] if len(fixed) > 1 else fixed)
    steps = [oracle_step(params, cam, target, [grid[(k * tiles_per_step + i) % len(grid)]
                                               for i in range(tiles_per_step)]) for k in range(args.steps)]
    t_step = statistics.mean(steps)
    full = oracle_full_iteration_s(t_fixed, t_step, tiles_per_step)
    value = 1.0 / full
    cores = torch.get_num_threads()
    sample = (f"each step: FP64 fwd+bwd of all 300k Gaussians on {tiles_per_step} 16x16 tiles "
              f"({tiles_per_step * 256} of {W * H} pixels; step k takes tiles 4k..4k+3 of a fixed list of 128 "
              f"spread over the image) + Adam, {t_step:.2f} s; full iteration = pixel-independent part "
              f"{t_fixed:.2f} s (median of the warm-up steps after the first, no pixels) + mean per-tile time "
              f"x {FULL_TILES:.1f} tiles = {full:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_gaussians": N_GAUSS, "width": W, "height": H},
            "full_iteration_s": full,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": _cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU path


def fused_roofline(work: dict, ms: float, n_sm: int, peaks: dict) -> dict:
    """The compositing kernel against the FP32 peak: algorithmic FLOPs of the render's pairs
    (tested, blended, walked; ``gs_debug_work``) over its measured duration."""
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    flops = (FLOP_FWD_TESTED * work["tested"] + FLOP_FWD_BLENDED * work["blended"]
             + FLOP_BWD_WALKED * work["walked"] + FLOP_BWD_BLENDED * work["blended"])
    ach = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "flop_per_launch": flops, "ms_per_launch": ms,
            "peak_source": "FP32 lanes x 2 x SMs x max SM clock"}


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_2504_02437_gb300 import build as B
    if rank == 0:
        B.build()          # one rank compiles (an up-to-date library is left alone); the others wait
    barrier(world)
    from paper_2504_02437_gb300.api import GaussianMap

    params, cam, target = make_workload(seed=rank)
    dev = torch.device("cuda", local)
    gm = GaussianMap(capacity=N_GAUSS, max_views=1, max_width=W, max_height=H, device=local,
                     tile_size=args.tile, pixels_per_thread=args.ppt)
    p0 = torch.as_tensor(params, device=dev)
    gm.set_params(p0)
    tgt = torch.as_tensor(target[None], device=dev).contiguous()
    loss = torch.empty(3, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # warm-up with every phase timed (the per-phase breakdown): the first call runs the iteration
    # directly and captures its graph; its records are dropped, so the breakdown and the dominant
    # phase come from graph replays only
    gm.timing(True)
    gm.iterate(cam, tgt, loss)
    torch.cuda.synchronize()
    gm.timing(True)                    # clears the first call's records; same mask, same graph
    for _ in range(max(args.warmup - 1, 2)):
        gm.iterate(cam, tgt, loss)
    torch.cuda.synchronize()
    phases_all = gm.timing_read()
    per_all = {k: v[0] / v[1] for k, v in phases_all.items() if v[1] > 0}
    dom = max(per_all, key=per_all.get)
    # the timed regions record events around the dominant kernel only (each timed phase adds
    # event nodes to the replayed graph); the changed graph is captured in two more warm-ups
    gm.timing(True, phases=[dom])
    for _ in range(2):
        gm.iterate(cam, tgt, loss)
    torch.cuda.synchronize()

    # ---- device-resident timed regions: `repeats` regions of exactly `steps` iterations each,
    # L2 flushed between iterations; the median region is the headline
    R = max(1, args.repeats)
    gm.timing(True, phases=[dom])      # clears the warm-up records, same mask: the graph stays
    launches0 = gm.launches
    region_ms = []
    with ClockSampler(local) as clk:
        for r in range(R):
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            barrier(world)
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                gm.iterate(cam, tgt, loss)
                ends[k].record(stream)
            torch.cuda.synchronize()
            barrier(world)
            region_ms.append(max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, ends)), world))
    launches = (gm.launches - launches0) // R
    phases = gm.timing_read()
    total_ms = statistics.median(region_ms)
    ms_per_step = total_ms / args.steps
    value = replica_throughput(args.steps, world, total_ms)
    final_loss = loss.cpu().numpy().tolist()

    # ---- end to end through the API: gs_iterate_host takes the step's target in pinned host memory
    # and returns its loss there. The library uploads step k's target once step k - 1's iteration
    # has started (inside that step's bracket, beside its iteration; step 0's inside its own) and
    # copies the loss back after the iteration. Each step is bracketed on the compute stream like
    # the device-resident steps, L2 flushed between steps, outside the brackets.
    gm.timing(False)
    tgt_host = torch.as_tensor(np.ascontiguousarray(target[None])).pin_memory()
    loss_host = torch.empty(3).pin_memory()
    for _ in range(2):
        gm.iterate_host(cam, tgt_host, loss_host)   # records the iteration with the host-loss slot
    torch.cuda.synchronize()
    e2e_region_ms = []
    for r in range(R):
        e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            e_s[k].record(stream)
            gm.iterate_host(cam, tgt_host, loss_host)
            e_e[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        e2e_region_ms.append(max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(e_s, e_e)), world))
    e2e_value = replica_throughput(args.steps, world, statistics.median(e2e_region_ms))

    # ---- roofline of the dominant kernel
    work = gm.debug_work()
    # the dominant kernel in the timed regions (the warm-up replays' figure if no timed step
    # recorded it, e.g. a step that re-captured the graph)
    per = {k: (v[0] / v[1] if v[1] > 0 else per_all.get(k, 0.0)) for k, v in phases.items()}
    peaks, peak_src = _peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    if dom == "raster_fused":
        roof = fused_roofline(work, per[dom], n_sm, peaks)
    else:
        # memory-bound phases: algorithmic bytes per unit (see the design notes' table)
        P, N = work["pairs"], gm.n
        bytes_model = {"project": 56 * N + 64 * N + 4 * 8 * 2 * N, "bin": 2 * 16 * P + 8 * P,
                       "loss": 3 * 4 * 3 * W * H, "project_bwd": 56 * N + 48 * N + 56 * N,
                       "adam": 14 * N * 4 * 7}
        roof = {"bound": "hbm", "achieved": bytes_model[dom] / (per[dom] * 1e-3) / 1e9,
                "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = _ncu_traffic(dom, gm.tile_size, gm.pixels_per_thread)
    roof["traffic_unit"] = "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    roof["kernel"] = dom
    layout = {"tile": gm.tile_size, "pixels_per_thread": gm.pixels_per_thread}
    split = split_measure(gm, cam, tgt)
    gm.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gaussians": N_GAUSS, "width": W, "height": H,
                       "l2": "flushed between iterations (256 MB write)", "parallelism": f"replicas x{world}"},
            "repeats": R,
            "value_spread": {"min": replica_throughput(args.steps, world, max(region_ms)),
                             "max": replica_throughput(args.steps, world, min(region_ms)),
                             "what": f"{R} timed regions of {args.steps} iterations each; value is the median"},
            "layout": layout,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(tgt.numel() * 4),
                    "d2h_bytes_per_step": 12,
                    "how": "gs_iterate_host: each step's target uploaded from pinned host memory by the library "
                           "(on its copy stream, once the previous step's iteration has started: inside that "
                           "step's bracket), the loss copied back to pinned memory; each step bracketed, L2 "
                           f"flushed between steps; median of {R} regions"},
            "gpu_launches": int(launches),
            "roofline": roof,
            "clocks": clk.summary(),
            "phases_ms": {k: round(v, 5) for k, v in per_all.items()},
            "phases_note": "per-phase device ms from the warm-up graph replays with every phase timed",
            "work": work, "final_loss": final_loss,
            "forward_backward_split": split}
    if rank == 0 and world == 1 and not args.no_extras:
        line["window"] = window_measure(args, max(args.steps, 20), local)
        line["learned_init"] = learned_init_measure(args, local)
        line["ablation"] = {"metric": ABLATION_METRIC, "frames": 24,
                            "workload": STREAM_WORKLOAD.format(F=24, I=100),
                            "rows": ablation_rows(24, ABLATION_REDUCED, args)}
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_oracle_baseline(params, cam, target, args.cpu_tiles, args.cpu_tiles_single)
        a = cb["all_cores"]
        line["cpu_baseline"] = {
            "value": a["replica_iters_per_s"], "unit": UNIT, "cores": a["threads"], "kind": "oracle",
            "sample": (f"FP64 oracle on {a['threads']} host threads ({cb['cpu_model']}, nproc {cb['nproc']}): "
                       f"pixel-independent part of an iteration (projection of all 300k Gaussians, its adjoint, "
                       f"planar term, Adam) {a['fixed_s']:.2f} s + {a['tiles_sampled']} 16x16 tiles spread over the "
                       f"image at {a['per_tile_s']:.3f} s each, scaled to the {FULL_TILES:.1f} tiles of the image"),
            "variants": cb}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def split_measure(gm, cam, tgt, steps: int = 20, warmup: int = 3) -> dict:
    """The forward and the backward timed apart: the same iteration through the separate calls
    (gs_render, gs_loss, gs_backward, gs_step), each phase bracketed by device events, median of
    `steps` iterations. The mapping iteration itself runs forward, loss and adjoint as one fused
    kernel; this is the split the separate kernels give (after the timed regions: it moves the
    map by steps + warmup Adam steps)."""
    import statistics
    import torch
    names = ("project", "bin", "raster_fwd", "loss", "raster_bwd", "project_bwd", "adam")
    for _ in range(warmup):
        gm.render(cam)
        gm.loss(tgt)
        gm.backward()
        gm.step()
    per = {k: [] for k in names}
    for _ in range(steps):
        gm.timing(True)
        gm.render(cam)
        gm.loss(tgt)
        gm.backward()
        gm.step()
        torch.cuda.synchronize()
        rec = gm.timing_read()
        for k in names:
            if rec.get(k, (0.0, 0))[1] > 0:
                per[k].append(rec[k][0])
    gm.timing(False)
    med = {k: statistics.median(v) for k, v in per.items() if v}
    fwd = med.get("project", 0.0) + med.get("bin", 0.0) + med.get("raster_fwd", 0.0)
    bwd = med.get("raster_bwd", 0.0) + med.get("project_bwd", 0.0)
    return {"what": "separate calls gs_render | gs_loss | gs_backward | gs_step, per-phase device time, "
                    f"median of {steps} iterations (the fused iteration merges forward, loss and adjoint)",
            "forward_ms": round(fwd, 5), "loss_ms": round(med.get("loss", 0.0), 5),
            "backward_ms": round(bwd, 5), "adam_ms": round(med.get("adam", 0.0), 5),
            "phases_ms": {k: round(v, 5) for k, v in med.items()}}


def window_measure(args, steps: int, device: int = 0) -> dict:
    """The keyframe window (8 views 640x480, 150k Gaussians): iterations/s of one call that renders
    and back-propagates all views in one persistent compositing launch (replayed graph), against
    the same work as 8 single-view iterations, plus the compositing kernel's FP32 roofline."""
    import torch
    from paper_2504_02437_gb300.api import GaussianMap
    dev = torch.device("cuda", device)
    params, cams, tgt = make_window_workload(0, device=dev)
    V = len(cams)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / n

    gm = GaussianMap(capacity=params.shape[1], max_views=V, max_width=640, max_height=480, device=device,
                     tile_size=args.tile, pixels_per_thread=args.ppt)
    gm.set_params(torch.as_tensor(params, device=dev))
    loss = torch.empty(3, device=dev)
    for _ in range(max(args.warmup, 3)):
        gm.iterate(cams, tgt, loss)
    gm.timing(True, phases=["raster_fused"])
    for _ in range(2):
        gm.iterate(cams, tgt, loss)
    torch.cuda.synchronize()
    gm.timing(True, phases=["raster_fused"])
    l0 = gm.launches
    with ClockSampler(device) as clk:
        ms_window = timed(lambda: gm.iterate(cams, tgt, loss), steps)
    launches = (gm.launches - l0) // steps
    ph = gm.timing_read()["raster_fused"]
    fused_ms = ph[0] / max(ph[1], 1)
    work = gm.debug_work()
    tile, ppt = gm.tile_size, gm.pixels_per_thread
    gm.render(cams)
    visible = [int((gm.debug_projection(v)[8] > 0).sum()) for v in range(V)]
    gm.close()
    gs = GaussianMap(capacity=params.shape[1], max_views=1, max_width=640, max_height=480, device=device,
                     tile_size=tile, pixels_per_thread=ppt)
    gs.set_params(torch.as_tensor(params, device=dev))
    singles = [tgt[v:v + 1].contiguous() for v in range(V)]
    for _ in range(max(args.warmup, 3)):
        for v in range(V):
            gs.iterate(cams[v], singles[v], loss)

    def seq():
        for v in range(V):
            gs.iterate(cams[v], singles[v], loss)
    ms_seq = timed(seq, steps)
    gs.close()
    peaks, _ = _peaks()
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    return {"metric": WINDOW_METRIC, "value": 1000.0 / ms_window, "unit": UNIT, "steps": steps,
            "ms_per_step": ms_window, "workload": WINDOW_WORKLOAD, "n_gaussians": int(params.shape[1]),
            "views": V, "visible_per_view": visible,
            "visible_note": "the map puts 98 % of its Gaussians on the boxes so that one view can see most of "
                            "them; the 8 consecutive keyframes span 20.3k-124.7k visible Gaussians",
            "layout": {"tile": tile, "pixels_per_thread": ppt},
            "sequential": {"what": f"{V} single-view iterations (one per view, {V} Adam steps) per step",
                           "value": 1000.0 / ms_seq, "ms_per_step": ms_seq, "speedup_of_window": ms_seq / ms_window},
            "gpu_launches": int(launches), "work": work,
            "roofline": dict(fused_roofline(work, fused_ms, n_sm, peaks), kernel="raster_fused",
                             traffic=_ncu_traffic("raster_fused_window", tile, ppt),
                             traffic_unit="bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"),
            "l2": "flushed between iterations (256 MB write)", "clocks": clk.summary()}


def run_window(args):
    """Window workload alone: one call renders and back-propagates all 8 views (one persistent
    compositing launch in the replayed graph) vs 8 single-view iterations, same GPU."""
    import torch
    torch.cuda.set_device(0)
    from paper_2504_02437_gb300 import build as B
    B.build()
    w = window_measure(args, args.steps, 0)
    line = {"metric": WINDOW_METRIC, "value": w["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": w["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WINDOW_WORKLOAD, "n_gaussians": w["n_gaussians"], "views": w["views"],
                       "l2": w["l2"]},
            "window": w, "gpu_launches": w["gpu_launches"], "roofline": w["roofline"], "clocks": w["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


STREAM_METRIC = "mapping stream iters/s: 8-keyframe window x 100 iterations per keyframe, 640x480, insertion + densification"
STREAM_WORKLOAD = ("mapping stream over a synthetic room sequence: {F} keyframes at 640x480 (fx=fy=525) on a smooth "
                   "path, 96 VO-style points per keyframe (surface point + N(0, 0.01^2) per axis), opacity-gated "
                   "insertion, {I} Adam iterations per keyframe over the last 8 keyframes, NDC-gradient split after each")
TTP_METRIC = ("time-to-PSNR, learned vs plain initialisation: ms of mapping iterations until the newest keyframe "
              "reaches the PSNR plain initialisation has after 100 iterations (held-out sequences)")


STREAM_CAPACITY = 1_500_000   # a 200-keyframe stream densifies to about 0.3M Gaussians


def _stream_map(capacity, args):
    from paper_2504_02437_gb300.api import GaussianMap
    return GaussianMap(capacity=capacity, max_views=8, max_width=640, max_height=480, tile_size=args.tile,
                       pixels_per_thread=args.ppt)


def time_to_psnr(train_seeds, heldout_seeds, frames, iters, args, epochs=300, log=None, heldout_frames=None):
    """Learned-initialiser protocol: collect (features, converged parameters) pairs from plain
    streams of ``train_seeds``, train the MLP with the library's kernels, then run each held-out
    sequence twice (plain, learned) and compare per keyframe (keyframe 0 is initialised the
    same way in both and is left out) the iterations and mapping ms until the newest keyframe's
    PSNR reaches the plain run's PSNR after ``iters`` iterations."""
    import torch
    from synth import stream_sequence
    from paper_2504_02437_gb300.api import MLP
    from paper_2504_02437_gb300 import stream as S
    t0 = time.perf_counter()
    X, Y = [], []
    for sd in train_seeds:
        cams, tg, pts = stream_sequence(sd, frames)
        gm = _stream_map(STREAM_CAPACITY, args)
        st = S.run_stream(gm, cams, tg, pts, iters=iters, collect=True)
        gm.close()
        X.append(st["features"])
        Y.append(st["targets"])
    X, Y = torch.cat(X), torch.cat(Y)
    t_collect = time.perf_counter() - t0
    mlp = MLP(seed=0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    losses = S.train_mlp(mlp, X, Y, epochs=epochs, batch=4096, lr=1e-3)
    ev[1].record()
    torch.cuda.synchronize()
    train_ms = ev[0].elapsed_time(ev[1])
    it_plain, it_mlp, ms_plain, ms_mlp, p_plain, p_mlp, p1_plain, p1_mlp = [], [], [], [], [], [], [], []
    reached = 0
    for sd in heldout_seeds:
        cams, tg, pts = stream_sequence(sd, heldout_frames or frames)
        runs = {}
        for name, m in (("plain", None), ("mlp", mlp)):
            gm = _stream_map(STREAM_CAPACITY, args)
            runs[name] = S.run_stream(gm, cams, tg, pts, iters=iters, track_psnr="curve", mlp=m)
            gm.close()
        cp, cm = runs["plain"]["psnr"][1:], runs["mlp"]["psnr"][1:]
        goal = cp[:, -1]
        k_m = S.iterations_to_reach(cm, goal)
        reached += int((k_m <= iters).sum())
        k_m = torch.clamp(k_m, max=iters)
        for j in range(cp.shape[0]):
            itp = runs["plain"]["iteration_ms"][j + 1]
            itm = runs["mlp"]["iteration_ms"][j + 1]
            it_plain.append(iters)
            it_mlp.append(int(k_m[j]))
            ms_plain.append(sum(itp))
            ms_mlp.append(sum(itm[:int(k_m[j])]))
        p_plain += goal.tolist()
        p_mlp += cm[:, -1].tolist()
        p1_plain += cp[:, 0].tolist()
        p1_mlp += cm[:, 0].tolist()
    n = len(it_mlp)
    return {"train_seeds": list(train_seeds), "heldout_seeds": list(heldout_seeds), "frames": frames,
            "heldout_frames": heldout_frames or frames,
            "iterations_per_keyframe": iters, "training_pairs": int(X.shape[0]), "collect_s": round(t_collect, 2),
            "train_epochs": epochs, "train_ms": round(train_ms, 1), "train_loss_first_last": [losses[0], losses[-1]],
            "keyframes_compared": n, "mlp_reached_goal": reached,
            "iterations_to_goal": {"plain": float(np.mean(it_plain)), "mlp_mean": float(np.mean(it_mlp)),
                                   "mlp_median": float(np.median(it_mlp))},
            "ms_to_goal": {"plain": float(np.sum(ms_plain)), "mlp": float(np.sum(ms_mlp))},
            "speedup": float(np.sum(ms_plain) / max(np.sum(ms_mlp), 1e-9)),
            "psnr_after_100": {"plain_mean": float(np.mean(p_plain)), "mlp_mean": float(np.mean(p_mlp))},
            "psnr_after_1": {"plain_mean": float(np.mean(p1_plain)), "mlp_mean": float(np.mean(p1_mlp))}}


def run_stream_bench(args):
    """Config-4 stream: every keyframe inserts its VO points, runs 100 window iterations and
    densifies; iterations are timed one by one with CUDA events, L2 flushed between them."""
    import torch
    torch.cuda.set_device(0)
    from paper_2504_02437_gb300 import build as B
    B.build()
    from synth import stream_sequence
    from paper_2504_02437_gb300 import stream as S
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    F, I = args.frames, 100
    # warm-up: a short stream of another sequence (builds, autotunes the small shapes)
    cams, tg, pts = stream_sequence(1, args.warmup)
    gm = _stream_map(STREAM_CAPACITY, args)
    S.run_stream(gm, cams, tg, pts, iters=I)
    gm.close()
    cams, tg, pts = stream_sequence(0, F)
    gm = _stream_map(STREAM_CAPACITY, args)
    with ClockSampler(0) as clk:
        st = S.run_stream(gm, cams, tg, pts, iters=I, track_psnr="final", flush=flush)
    tile, ppt = gm.tile_size, gm.pixels_per_thread
    gm.close()
    ps = st["psnr"].tolist()
    line = {"metric": STREAM_METRIC, "value": st["iters_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": st["iterations"], "warmup": args.warmup, "ms_per_step": 1000.0 / st["iters_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": STREAM_WORKLOAD.format(F=F, I=I), "frames": F, "window": 8,
                       "iterations_per_keyframe": I, "tile": tile, "pixels_per_thread": ppt,
                       "l2": "flushed between iterations (256 MB write)",
                       "warmup": f"{args.warmup}-keyframe stream of another sequence"},
            "n_gaussians_per_keyframe": st["n_gauss"], "inserted_per_keyframe": st["n_inserted"],
            "psnr_newest_keyframe_after_100": [round(x, 3) for x in ps],
            "psnr_mean_last_20": float(np.mean(ps[-20:])),
            "map_s": st["map_seconds"], "insert_ms_total": st["insert_ms"], "densify_ms_total": st["densify_ms"],
            "gpu_launches": int(st["launches"]), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


MLP_METRIC = "learned-initialiser MLP training steps/s (forward + backward + Adam, 4096 rows, BF16 tcgen05)"
# FLOP per row of one training step: forward 2 x (80x128 + 128x128 + 128x16); the backward repeats
# every product that takes an upstream gradient twice (bf16 hi + lo): weight gradients of the three
# layers and input gradients of the two hidden layers
MLP_FLOP_FWD_PER_ROW = 2 * (80 * 128 + 128 * 128 + 128 * 16)
MLP_FLOP_BWD_PER_ROW = 2 * 2 * (16 * 128 + 128 * 128 + 128 * 80) + 2 * 2 * (16 * 128 + 128 * 128)


def mlp_step_measure(steps: int, warmup: int, device: int = 0) -> dict:
    """Training steps of the learned initialiser (forward, MSE backward, Adam) on 4,096 random
    feature rows, against the measured BF16 tensor peak."""
    import torch
    from paper_2504_02437_gb300.api import MLP
    rows = 4096
    g = torch.Generator(device=f"cuda:{device}")
    g.manual_seed(0)
    X = torch.rand(rows, 80, device=f"cuda:{device}", generator=g)
    Y = torch.randn(rows, 16, device=f"cuda:{device}", generator=g) * 0.5
    Y[:, 11:] = 0
    mlp = MLP(seed=0, device=device)
    for _ in range(warmup):
        mlp.backward(X, Y)
        mlp.step(1e-3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record()
        mlp.backward(X, Y)
        mlp.step(1e-3)
        b.record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    Xs = X[:96].contiguous()
    evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evf:
        a.record()
        mlp.forward(Xs)
        b.record()
    torch.cuda.synchronize()
    ms_fwd96 = sum(a.elapsed_time(b) for a, b in evf) / steps
    mlp.close()
    flops = rows * (MLP_FLOP_FWD_PER_ROW + MLP_FLOP_BWD_PER_ROW)
    peaks, src = _peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    ach = flops / (ms * 1e-3) / 1e12
    return {"metric": MLP_METRIC, "value": 1000.0 / ms, "unit": "steps/s", "steps": steps, "ms_per_step": ms,
            "forward_96_rows_ms": ms_fwd96,
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "traffic": None, "kernel": "whole training step (k_gemm_tc launches + elementwise)",
                         "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({src})"}}


def learned_init_measure(args, device: int = 0) -> dict:
    """The learned-initialiser protocol at reduced size: the MLP is trained on the converged
    Gaussians of two 60-keyframe plain streams (seeds 0, 1); one held-out 16-keyframe sequence
    (seed 100) is mapped with plain and with learned initialisation; per keyframe, the iterations
    and mapping ms until the newest keyframe reaches the PSNR the plain run has after 100."""
    r = time_to_psnr((0, 1), (100,), 60, 100, args, epochs=300, heldout_frames=16)
    m = mlp_step_measure(20, 5, device)
    return {"metric": TTP_METRIC, "value": r["speedup"], "unit": "x (plain ms / learned ms to the same PSNR)",
            "protocol": "MLP trained on 2 plain streams of 60 keyframes (seeds 0, 1); held-out sequence seed 100, "
                        "16 keyframes, each mapped twice (plain, learned), 100 iterations per keyframe",
            "time_to_psnr": r, "mlp_training_step": m}


def run_mlp_bench(args):
    """Training steps of the learned initialiser on random features (the shapes of the
    learned-initialiser protocol's training batches): one step = forward, MSE backward, Adam.
    Tensor-core roofline against the measured BF16 peak."""
    import torch
    torch.cuda.set_device(0)
    from paper_2504_02437_gb300 import build as B
    B.build()
    with ClockSampler(0) as clk:
        m = mlp_step_measure(args.steps, args.warmup, 0)
    line = {"metric": MLP_METRIC, "value": m["value"], "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 (f32 accumulate)", "data": "synthetic",
            "config": {"workload": "MLP 80-128-128-16 training step on 4096 random feature rows",
                       "l2": "resident (the whole step fits in L2; the MLP is latency-bound)"},
            "forward_96_rows_ms": m["forward_96_rows_ms"], "roofline": m["roofline"], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


ABLATION_METRIC = "synthetic ablation of the mapping stream: PSNR, #Gaussians, iters/s per switch setting"
ABLATIONS = [
    ("full: opacity insertion, gradient split, planar term", {}),
    ("no planar term", {"lambda_reg": 0.0}),
    ("no densification", {"densify": False}),
    ("distance insertion (tau 0.05 m)", {"insert_tau": 0.05}),
    ("gradient + clarity split (sigma 64 px)", {"clarity_sigma": 64.0, "clarity": True}),
    ("L1 + SSIM (lambda_photo 0.2)", {"lambda_photo": 0.2}),
]


def ablation_rows(frames: int, settings, args) -> list:
    """One mapping stream of ``frames`` keyframes (sequence seed 0) per switch setting: the newest
    keyframe's PSNR after its iterations (mean of the last 20 keyframes and of all), the final
    Gaussian count and the mapping iterations/s."""
    from synth import stream_sequence
    from paper_2504_02437_gb300 import stream as S
    from paper_2504_02437_gb300.api import GaussianMap
    cams, tg, pts = stream_sequence(0, frames)
    rows = []
    for name, sw in settings:
        cfg = {k: v for k, v in sw.items() if k not in ("densify", "clarity")}
        gm = GaussianMap(capacity=STREAM_CAPACITY, max_views=8, max_width=640, max_height=480,
                         tile_size=args.tile, pixels_per_thread=args.ppt, **cfg)
        st = S.run_stream(gm, cams, tg, pts, iters=100, track_psnr="final", densify=sw.get("densify", True),
                          clarity=sw.get("clarity", False))
        gm.close()
        ps = st["psnr"].tolist()
        rows.append({"setting": name, "psnr_mean_last_20": float(np.mean(ps[-20:])),
                     "psnr_mean_all": float(np.mean(ps)), "n_gaussians_final": st["n_gauss"][-1],
                     "iters_per_s": st["iters_per_s"]})
    return rows


# the default benchmark line's reduced ablation: the paper's three switches (Table 4: insertion,
# densification, planar term) on a 24-keyframe stream
ABLATION_REDUCED = [ABLATIONS[0], ABLATIONS[1], ABLATIONS[2], ABLATIONS[3]]


def run_ablation_bench(args):
    """The switches of the paper's ablation (insertion rule, densification, planar term; Table 4's
    analogue) and the SSIM term on one synthetic stream: per setting the newest keyframe's PSNR
    after its iterations (mean of the last 20 keyframes), the final Gaussian count and the
    mapping iterations/s."""
    import torch
    torch.cuda.set_device(0)
    from paper_2504_02437_gb300 import build as B
    B.build()
    with ClockSampler(0) as clk:
        rows = ablation_rows(args.frames, ABLATIONS, args)
    line = {"metric": ABLATION_METRIC, "value": rows[0]["psnr_mean_last_20"], "unit": "dB (full setting)",
            "n_gpus": 1, "steps": args.frames * 100, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": STREAM_WORKLOAD.format(F=args.frames, I=100)},
            "ablation": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_ttp_bench(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2504_02437_gb300 import build as B
    B.build()
    with ClockSampler(0) as clk:
        r = time_to_psnr(range(args.train_seeds), range(100, 100 + args.heldout_seeds), args.frames, 100, args)
    line = {"metric": TTP_METRIC, "value": r["speedup"], "unit": "x (plain ms / learned ms to the same PSNR)",
            "n_gpus": 1, "steps": r["keyframes_compared"], "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 MLP, f32 mapping", "data": "synthetic",
            "config": {"workload": STREAM_WORKLOAD.format(F=args.frames, I=100) +
                       "; MLP trained on the plain runs of the training seeds, compared on held-out seeds"},
            "time_to_psnr": r, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=0, choices=[0, 8, 16])
    ap.add_argument("--workload", default="replica", choices=["replica", "window", "stream", "learned_init",
                                                              "ablation", "mlp"])
    ap.add_argument("--frames", type=int, default=0, help="keyframes (stream, learned_init: 200; ablation: 60)")
    ap.add_argument("--train-seeds", type=int, default=5)
    ap.add_argument("--heldout-seeds", type=int, default=5)
    ap.add_argument("--ppt", type=int, default=0, choices=[0, 1, 2, 4])
    ap.add_argument("--cpu-tiles", type=int, default=128, help="sample tiles of the all-core oracle timing")
    ap.add_argument("--cpu-tiles-single", type=int, default=32, help="sample tiles of the single-thread oracle timing")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="leave out the window and learned-initialiser objects")
    ap.add_argument("--repeats", type=int, default=30, help="timed regions of --steps iterations (median reported)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "window":
        return run_window(args)
    if args.workload in ("stream", "learned_init"):
        args.frames = args.frames or 200
    if args.workload == "stream":
        return run_stream_bench(args)
    if args.workload == "learned_init":
        return run_ttp_bench(args)
    if args.workload == "mlp":
        return run_mlp_bench(args)
    if args.workload == "ablation":
        args.frames = args.frames or 60
        return run_ablation_bench(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

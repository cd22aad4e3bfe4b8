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

# DRAM bytes (read + write) of one launch of the dominant kernel from an ncu capture of this
# workload, with the kernel source's sha256 and layout at capture time (the figure is reported
# only while both still match): profiles/raster_fused_replica_1200x680_300k.md
NCU_TRAFFIC = {"raster_fused": {"bytes": 35.94e6, "source": "paper_2504_02437_gb300/csrc/k_raster.cu",
                                "sha256": "69e7d039fabc38381fdc41fb42b1debad7d6f67316d7459ddccc20aa56ae1edd",
                                "tile": 16, "ppt": 2}}


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


def _h2d_async():
    """cudaMemcpyAsync host -> device on a given stream (torch's non_blocking copy_ from pinned
    memory held the host for the whole copy when the copy stream had pending waits)."""
    import ctypes
    rt = ctypes.CDLL("libcudart.so")
    rt.cudaMemcpyAsync.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]

    def copy(dst, src, stream):
        assert src.is_pinned() and dst.is_cuda and dst.numel() == src.numel() and dst.dtype == src.dtype
        err = rt.cudaMemcpyAsync(dst.data_ptr(), src.data_ptr(), src.numel() * src.element_size(), 1,
                                 stream.cuda_stream)
        if err != 0:
            raise RuntimeError(f"cudaMemcpyAsync failed ({err})")
    return copy


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


WINDOW_METRIC = "mapping window fwd+bwd iters/s @8x640x480,150k Gaussians"
WINDOW_WORKLOAD = ("TUM-shaped keyframe window: 8 views 640x480, fx=fy=525, on a smooth path through the textured "
                   "room, 150k Gaussians; one iteration = render all views + L1/planar loss + adjoint + one Adam step")


# trajectory seed of the window: among seeds 0-39 of the room-0 trajectories, the one whose 8 views
# span the widest visible range from at least ~19k (18.8k-65.1k of 150k Gaussians; no view inside
# this room sees more than ~67k)
WINDOW_TRAJECTORY_SEED = 33


def make_window_workload(seed: int = 0, n_views: int = 8, n_gauss: int = 150_000,
                         trajectory_seed: int = WINDOW_TRAJECTORY_SEED):
    from synth import make_room, room_gaussians, room_trajectory
    room = make_room(seed)
    cams = room_trajectory(n_views, trajectory_seed, 640, 480, 525.0, 525.0)
    params = room_gaussians(room, n_gauss, seed)
    cache = os.path.join(tempfile.gettempdir(), f"gs_room_window_{seed}_{trajectory_seed}_{n_views}.npy")
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
        target = room.raycast(cam)
        try:
            np.save(cache, target)
        except OSError:
            pass
    return params, cam, target


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a timed region."""
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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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


def oracle_sample(params, cam, target, n_tiles: int, seed: int):
    """Oracle fwd+bwd+Adam on ``n_tiles`` random 16x16 pixel tiles of the workload.

    Returns (seconds, fraction of the full image's pixels covered).
    """
    import torch
    import oracle as O
    rng = np.random.default_rng(seed)
    pix = []
    for _ in range(n_tiles):
        x0 = int(rng.integers(0, W - 16))
        y0 = int(rng.integers(0, H - 16))
        yy, xx = np.mgrid[y0:y0 + 16, x0:x0 + 16]
        pix.append(np.stack([xx.ravel(), yy.ravel()], 1))
    pix = np.concatenate(pix)
    p64 = params.astype(np.float64)
    t0 = time.perf_counter()
    res = O.loss_and_grads(p64, [cam], target[None], pixels=[pix], chunk=256)
    O.adam_step(p64, res["grad"], np.zeros_like(p64), np.zeros_like(p64), 1)
    dt = time.perf_counter() - t0
    return dt, pix.shape[0] / float(W * H), torch.get_num_threads()


def run_reference(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    params, cam, target = make_workload(0)
    tiles_per_step = 4
    for w in range(args.warmup):
        oracle_sample(params, cam, target, 1, 1000 + w)
    secs, frac = 0.0, 0.0
    cores = 1
    for k in range(args.steps):
        dt, f, cores = oracle_sample(params, cam, target, tiles_per_step, k)
        secs += dt
        frac += f
    value = frac / secs                    # full iterations per second
    sample = (f"{args.steps} steps x {tiles_per_step} random 16x16 tiles ({tiles_per_step * 256} of {W * H} pixels) "
              f"of the full workload: FP64 fwd+bwd over all 300k Gaussians + Adam, scaled by pixel fraction")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_gaussians": N_GAUSS, "width": W, "height": H},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU path


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

    # warm-up with every phase timed (the per-phase breakdown). The first call runs the iteration
    # as separate kernels (render, loss, adjoint: phases that the replays do not have) and
    # captures its graph; its records are dropped, so the breakdown and the dominant phase
    # come from graph replays only
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
    # the timed region records events around the dominant kernel only (each timed phase adds
    # event nodes to the replayed graph); the changed graph is captured in two more warm-ups
    gm.timing(True, phases=[dom])
    for _ in range(2):
        gm.iterate(cam, tgt, loss)
    torch.cuda.synchronize()

    # ---- device-resident timed region (L2 flushed between iterations)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    gm.timing(True, phases=[dom])      # clears the warm-up records, same mask: the graph stays
    launches0 = gm.launches
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            gm.iterate(cam, tgt, loss)
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    launches = gm.launches - launches0
    phases = gm.timing_read()
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    total_ms = max_over_ranks(total_ms, world)
    ms_per_step = total_ms / args.steps
    value = replica_throughput(args.steps, world, total_ms)
    final_loss = loss.cpu().numpy().tolist()

    # ---- end to end through the API: each step's target goes up from pinned host memory and its
    # loss comes back. The upload of step k + 1 (copy stream, second target buffer) runs while
    # step k iterates; step 0's upload sits inside its own bracket. Each step is bracketed on the
    # compute stream like the device-resident steps, L2 flushed between steps, outside the brackets.
    gm.timing(False)
    tgt_host = torch.as_tensor(target[None]).pin_memory()
    loss_host = torch.empty(3).pin_memory()
    bufs = [torch.empty_like(tgt), torch.empty_like(tgt)]
    copy_stream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    for bb in bufs:
        bb.copy_(tgt)
    for _ in range(2):
        gm.iterate(cam, bufs[0], loss)
    torch.cuda.synchronize()

    h2d = _h2d_async()

    def upload(k):
        copy_stream.wait_event(free[k % 2])
        h2d(bufs[k % 2], tgt_host, copy_stream)
        ready[k % 2].record(copy_stream)
    for e in free:
        e.record(stream)
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        e_s[k].record(stream)
        if k == 0:
            copy_stream.wait_event(e_s[0])
            upload(0)
        if k + 1 < args.steps:
            upload(k + 1)
        stream.wait_event(ready[k % 2])
        gm.iterate(cam, bufs[k % 2], loss)
        free[k % 2].record(stream)
        loss_host.copy_(loss, non_blocking=True)
        e_e[k].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(e_s, e_e)), world)
    e2e_value = replica_throughput(args.steps, world, e2e_ms)

    # ---- roofline of the dominant kernel
    work = gm.debug_work()
    # the dominant kernel in the timed region (the warm-up replays' figure if no timed step
    # recorded it, e.g. a step that re-captured the graph)
    per = {k: (v[0] / v[1] if v[1] > 0 else per_all.get(k, 0.0)) for k, v in phases.items()}
    peaks, peak_src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    if dom == "raster_fused":
        flops = (FLOP_FWD_TESTED * work["tested"] + FLOP_FWD_BLENDED * work["blended"]
                 + FLOP_BWD_WALKED * work["walked"] + FLOP_BWD_BLENDED * work["blended"])
        roof = {"bound": "alu", "achieved": flops / (per[dom] * 1e-3) / 1e12, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s"}
    elif dom == "raster_bwd":
        flops = FLOP_BWD_WALKED * work["walked"] + FLOP_BWD_BLENDED * work["blended"]
        roof = {"bound": "alu", "achieved": flops / (per[dom] * 1e-3) / 1e12, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s"}
    elif dom == "raster_fwd":
        flops = FLOP_FWD_TESTED * work["tested"] + FLOP_FWD_BLENDED * work["blended"]
        roof = {"bound": "alu", "achieved": flops / (per[dom] * 1e-3) / 1e12, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s"}
    else:
        # memory-bound phases: algorithmic bytes per unit (see the design notes' table)
        P, N = work["pairs"], gm.n
        bytes_model = {"project": 56 * N + 64 * N + 4 * 8 * 2 * N, "bin": 2 * 16 * P + 8 * P,
                       "loss": 3 * 4 * 3 * W * H, "project_bwd": 56 * N + 48 * N + 56 * N,
                       "adam": 14 * N * 4 * 7}
        roof = {"bound": "hbm", "achieved": bytes_model[dom] / (per[dom] * 1e-3) / 1e9,
                "peak": float(peaks["hbm_gbs"]), "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = _ncu_traffic(dom, gm.tile_size, gm.pixels_per_thread)
    roof["traffic_unit"] = "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    roof["kernel"] = dom
    roof["peak_source"] = ("FP32 lanes x 2 x SMs x max SM clock" if roof["bound"] == "alu"
                           else f"MEASURED_PEAKS.json hbm_gbs ({peak_src})")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gaussians": N_GAUSS, "width": W, "height": H,
                       "tile": gm.tile_size, "pixels_per_thread": gm.pixels_per_thread, "l2": "flushed between iterations (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(tgt.numel() * 4),
                    "d2h_bytes_per_step": 12,
                    "how": "target uploaded from pinned host memory on a copy stream (step k+1's during step k), "
                           "loss read back to pinned memory, each step bracketed, L2 flushed between steps"},
            "gpu_launches": int(launches),
            "roofline": roof,
            "clocks": clk.summary(),
            "phases_ms": {k: round(v, 5) for k, v in per_all.items()},
            "phases_note": "per-phase device ms from the warm-up graph replays with every phase timed",
            "work": work, "final_loss": final_loss}
    if rank == 0 and world == 1 and not args.no_cpu:
        dt, frac, cores = oracle_sample(params, cam, target, args.cpu_tiles, 7)
        line["cpu_baseline"] = {"value": frac / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_tiles} random 16x16 tiles ({args.cpu_tiles * 256} of {W * H} "
                                          f"pixels): FP64 fwd+bwd over all 300k Gaussians + Adam, "
                                          f"{dt:.1f} s, scaled by pixel fraction"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    gm.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_window(args):
    """Window workload: one call renders and back-propagates all 8 views (one persistent
    compositing launch in the replayed graph) vs 8 single-view iterations, same GPU."""
    import torch
    torch.cuda.set_device(0)
    from paper_2504_02437_gb300 import build as B
    B.build()
    from paper_2504_02437_gb300.api import GaussianMap
    params, cams, targets = make_window_workload(0)
    dev = torch.device("cuda", 0)
    V = len(cams)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    tgt = torch.as_tensor(targets, device=dev).contiguous()
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    gm = GaussianMap(capacity=params.shape[1], max_views=V, max_width=640, max_height=480, tile_size=args.tile,
                     pixels_per_thread=args.ppt)
    gm.set_params(torch.as_tensor(params, device=dev))
    loss = torch.empty(3, device=dev)
    gm.timing(True)
    gm.iterate(cams, tgt, loss)        # runs the iteration as separate kernels and captures its graph
    torch.cuda.synchronize()
    gm.timing(True)                    # drops those records: the breakdown comes from replays
    for _ in range(max(args.warmup - 1, 2)):
        gm.iterate(cams, tgt, loss)
    torch.cuda.synchronize()
    phases = gm.timing_read()          # breakdown from the warm-up replays, every phase timed
    gm.timing(False)                   # the timed region runs the graph without event nodes
    for _ in range(2):
        gm.iterate(cams, tgt, loss)
    l0 = gm.launches
    with ClockSampler(0) as clk:
        ms_window = timed(lambda: gm.iterate(cams, tgt, loss), args.steps)
    launches = gm.launches - l0
    tile, ppt = gm.tile_size, gm.pixels_per_thread
    visible = []
    gm.render(cams)
    for v in range(V):
        visible.append(int((gm.debug_projection(v)[8] > 0).sum()))
    gm.close()
    # the same work as V single-view iterations (V Adam steps), one view per call
    gs = GaussianMap(capacity=params.shape[1], max_views=1, max_width=640, max_height=480, tile_size=tile,
                     pixels_per_thread=ppt)
    gs.set_params(torch.as_tensor(params, device=dev))
    singles = [tgt[v:v + 1].contiguous() for v in range(V)]
    for _ in range(args.warmup):
        for v in range(V):
            gs.iterate(cams[v], singles[v], loss)

    def seq():
        for v in range(V):
            gs.iterate(cams[v], singles[v], loss)
    ms_seq = timed(seq, args.steps)
    gs.close()
    line = {"metric": WINDOW_METRIC, "value": 1000.0 / ms_window, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_window, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WINDOW_WORKLOAD, "n_gaussians": int(params.shape[1]), "views": V,
                       "visible_per_view": visible, "tile": tile, "pixels_per_thread": ppt,
                       "l2": "flushed between iterations (256 MB write)"},
            "sequential": {"what": f"{V} single-view iterations (one per view, {V} Adam steps) per step",
                           "ms_per_step": ms_seq, "speedup_of_window": ms_seq / ms_window},
            "gpu_launches": int(launches),
            "phases_ms": {k: round(v[0] / max(v[1], 1), 5) for k, v in phases.items()},
            "clocks": clk.summary()}
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


def time_to_psnr(train_seeds, heldout_seeds, frames, iters, args, epochs=300, log=None):
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
        cams, tg, pts = stream_sequence(sd, frames)
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


def run_mlp_bench(args):
    """Training steps of the learned initialiser on random features (the shapes of config 5's
    training batches): one step = forward, MSE backward, Adam. Tensor-core roofline against the
    measured BF16 peak."""
    import torch
    torch.cuda.set_device(0)
    from paper_2504_02437_gb300 import build as B
    B.build()
    from paper_2504_02437_gb300.api import MLP
    rows = 4096
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    X = torch.rand(rows, 80, device="cuda", generator=g)
    Y = torch.randn(rows, 16, device="cuda", generator=g) * 0.5
    Y[:, 11:] = 0
    mlp = MLP(seed=0)
    for _ in range(args.warmup):
        mlp.backward(X, Y)
        mlp.step(1e-3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        for a, b in ev:
            a.record()
            mlp.backward(X, Y)
            mlp.step(1e-3)
            b.record()
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    # forward alone on an insertion batch (96 points)
    Xs = X[:96].contiguous()
    evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in evf:
        a.record()
        mlp.forward(Xs)
        b.record()
    torch.cuda.synchronize()
    ms_fwd96 = sum(a.elapsed_time(b) for a, b in evf) / args.steps
    flops = rows * (MLP_FLOP_FWD_PER_ROW + MLP_FLOP_BWD_PER_ROW)
    peaks, src = _peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    ach = flops / (ms * 1e-3) / 1e12
    line = {"metric": MLP_METRIC, "value": 1000.0 / ms, "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 (f32 accumulate)", "data": "synthetic",
            "config": {"workload": "MLP 80-128-128-16 training step on 4096 random feature rows",
                       "l2": "resident (the whole step fits in L2; the MLP is latency-bound)"},
            "forward_96_rows_ms": ms_fwd96,
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "traffic": None, "kernel": "whole training step (13 k_gemm_tc launches + elementwise)",
                         "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({src})"},
            "clocks": clk.summary()}
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


def run_ablation_bench(args):
    """The switches of the paper's ablation (insertion rule, densification, planar term; Table 4's
    analogue) and the SSIM term on one synthetic stream: per setting the newest keyframe's PSNR
    after its iterations (mean of the last 20 keyframes), the final Gaussian count and the
    mapping iterations/s."""
    import torch
    torch.cuda.set_device(0)
    from paper_2504_02437_gb300 import build as B
    B.build()
    from synth import stream_sequence
    from paper_2504_02437_gb300 import stream as S
    from paper_2504_02437_gb300.api import GaussianMap
    cams, tg, pts = stream_sequence(0, args.frames)
    rows = []
    with ClockSampler(0) as clk:
        for name, sw in ABLATIONS:
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
    ap.add_argument("--cpu-tiles", type=int, default=160)
    ap.add_argument("--no-cpu", action="store_true")
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

"""Multi-rank paths on CPU ranks (gloo, world size 2, 127.0.0.1).

* The benchmark's replica aggregation: every rank times its own replica, the job is timed by the
  slowest rank (all-reduce max), and the whole-job throughput counts every rank's iterations.
* The view-sharding invariant the path would use across GPUs: the gradient of a keyframe window
  equals the sum over ranks of the gradients of the views each rank holds (one all-reduce of the
  14 x N gradient), checked with the FP64 oracle against the single-process window gradient.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(rank, world, port, fn, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    try:
        out[rank] = fn(rank, world)
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def _spawn(fn, world=2):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()          # every rank rendezvouses on the same port
        procs = [ctx.Process(target=_run, args=(r, world, port, fn, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        return dict(out)


def _replica_timing(rank, world):
    import bench
    w, r, _ = bench.dist_setup("gloo")
    assert (w, r) == (world, rank)
    my_ms = 100.0 + 50.0 * rank                 # rank 1 is the slower replica
    slowest = bench.max_over_ranks(my_ms, w)
    bench.barrier(w)
    return slowest, bench.replica_throughput(20, w, slowest)


def test_replica_aggregation_over_gloo_ranks():
    out = _spawn(_replica_timing)
    for rank in range(2):
        slowest, value = out[rank]
        assert slowest == 150.0
        assert value == pytest.approx(2 * 20 / 0.150)


def _view_shard(rank, world):
    import oracle as O
    from synth import Camera, frustum_scene
    from scipy.spatial.transform import Rotation
    dist.init_process_group("gloo")
    p, cam = frustum_scene(n=40, width=24, height=20, fx=24.0, fy=24.0, cx=12.0, cy=10.0, seed=31)
    cams = [cam, Camera(24, 20, 24.0, 24.0, 12.0, 10.0, Rotation.from_rotvec([0.03, -0.06, 0.0]).as_matrix(),
                        np.array([0.04, 0.0, 0.05]))]
    tg = np.random.default_rng(5).uniform(size=(2, 3, 20, 24))
    p64 = p.astype(np.float64)
    # this rank's view; the planar term is counted once (rank 0)
    cfg = O.Config(lambda_reg=1.0 if rank == 0 else 0.0)
    g = O.loss_and_grads(p64, [cams[rank]], tg[rank:rank + 1], cfg)["grad"]
    t = torch.tensor(g)
    dist.all_reduce(t)
    return t.numpy()


def test_window_gradient_is_all_reduced_sum_of_view_shards():
    import oracle as O
    from synth import Camera, frustum_scene
    from scipy.spatial.transform import Rotation
    out = _spawn(_view_shard)
    p, cam = frustum_scene(n=40, width=24, height=20, fx=24.0, fy=24.0, cx=12.0, cy=10.0, seed=31)
    cams = [cam, Camera(24, 20, 24.0, 24.0, 12.0, 10.0, Rotation.from_rotvec([0.03, -0.06, 0.0]).as_matrix(),
                        np.array([0.04, 0.0, 0.05]))]
    tg = np.random.default_rng(5).uniform(size=(2, 3, 20, 24))
    whole = O.loss_and_grads(p.astype(np.float64), cams, tg)["grad"]
    for rank in range(2):
        np.testing.assert_allclose(out[rank], whole, rtol=1e-12, atol=1e-15)

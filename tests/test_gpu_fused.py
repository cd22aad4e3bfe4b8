"""GPU parity of the mapping iteration as gs_iterate runs it, against the FP64 oracle.

gs_iterate composites, takes the L1 term and dL/dC, and runs the compositing
adjoint of every (view, tile) in one persistent kernel (k_raster_fused); every
call, the first included, runs that kernel. One call from a fresh map and fresh
Adam moments is compared element by element with the oracle (Eq. 3 image, Eq.
10-11 loss, the gradient of every parameter, the screen-space gradients, and
the parameters after the Adam step) for

* every (tile size, pixels per thread) layout the autotuner can pick: 16x1,
  16x2, 16x4, 8x1, 8x2, and the deterministic mode's 8x2;
* a window of three views in one launch;
* a scene whose tile lists span several shared-memory staging batches (up to
  1,932 records per 16-px tile against 512-record batches; 1,492 per 8-px tile
  against 256), with low opacities so that pixels blend (and stop) deep inside
  the lists: the forward's batch loop and the adjoint's back-to-front walk
  across batch boundaries;
* one-tile views whose list holds exactly one staging batch, and one batch
  plus one record, at every layout: the adjoint reusing the forward's staged
  batch, and staging again.
"""
import numpy as np
import pytest
import torch

import oracle as O
from synth import frustum_scene, random_target

from gpu_helpers import (GRAD_FLOOR, GRAD_FLOOR_DEEP, GRAD_RTOL, IMG_ATOL, SCREEN_GRAD_FLOOR, cuda,
                         exclude_kernel_limits, grad_errors, new_map, rotated_cam)

pytestmark = pytest.mark.gpu

LAYOUTS = [(16, 1), (16, 2), (16, 4), (8, 1), (8, 2)]


def iterate_once(p, cams, tg, **cfg):
    """One gs_iterate call from a fresh map: image, loss, gradients (pre-Adam), screen gradients,
    parameters after Adam, and the number of fused-kernel launches it made."""
    V, H, W = len(cams), cams[0].height, cams[0].width
    gm = new_map(p.shape[1], views=V, W=W, H=H, **cfg)
    gm.set_params(cuda(p))
    gm.timing(True, phases=["raster_fused"])
    rgb = torch.empty(V, 3, H, W, device="cuda")
    loss = torch.empty(3, device="cuda")
    gm.iterate(cams, cuda(tg), loss, rgb)
    torch.cuda.synchronize()
    fused = gm.timing_read()["raster_fused"][1]
    out = dict(rgb=rgb.cpu().numpy(), loss=loss.cpu().numpy(), grads=gm.grads().cpu().numpy(),
               grad2d=gm.debug_grad2d(), params=gm.params().cpu().numpy(), fused=fused,
               tile=gm.tile_size, ppt=gm.pixels_per_thread, pairs=gm.debug_pairs())
    gm.close()
    return out


def oracle_ref(p, cams, tg):
    p64 = p.astype(np.float64)
    g = O.loss_and_grads(p64, cams, tg, want_2d=True, flags=True)
    near = [O.render(p64, c, flags=True)["near"] for c in cams]
    excl = g["gauss_near"] | exclude_kernel_limits(p64, cams)
    return g, near, excl


def check_iteration(out, g, near, excl, p, max_near=1e-3, floor_frac=GRAD_FLOOR):
    V = len(near)
    assert out["fused"] == 1, "gs_iterate did not run the fused compositing kernel"
    for v in range(V):
        assert near[v].mean() < max_near, near[v].mean()
        err = np.abs(out["rgb"][v] - g["images"][v]).max(axis=0)
        assert err[~near[v]].max() <= IMG_ATOL, (v, err[~near[v]].max())
    assert abs(out["loss"][0] - g["loss"]) <= 1e-5 * g["loss"], (out["loss"], g["loss"])
    assert abs(out["loss"][2] - g["reg"]) <= 1e-5 * g["reg"]
    errs = grad_errors(out["grads"], g["grad"], exclude=excl, floor_frac=floor_frac)
    assert max(errs.values()) <= GRAD_RTOL, errs
    keep = ~excl
    sfloor = max(floor_frac, SCREEN_GRAD_FLOOR)
    names = ["u", "v", "a", "b", "c", "o"]
    for v in range(V):
        g2 = g["grad2d"][v]
        for k, name in enumerate(names):
            ref = g2[name]
            floor = sfloor * max(np.abs(ref).max(), 1e-30)
            rel = np.abs(out["grad2d"][v][k] - ref)[keep] / np.maximum(np.abs(ref[keep]), floor)
            assert rel.max() <= GRAD_RTOL, (v, name, rel.max())
        for ch in range(3):
            ref = g2["rgb"][:, ch]
            floor = sfloor * max(np.abs(ref).max(), 1e-30)
            rel = np.abs(out["grad2d"][v][6 + ch] - ref)[keep] / np.maximum(np.abs(ref[keep]), floor)
            assert rel.max() <= GRAD_RTOL, (v, "rgb", ch, rel.max())
    # the Adam step: the oracle's update from the oracle's gradient wherever the gradient's sign is
    # fixed well above the float32 accumulation level; elsewhere a step of at most the learning rate
    p64 = p.astype(np.float64)
    expect, _, _ = O.adam_step(p64, g["grad"], np.zeros_like(p64), np.zeros_like(p64), 1)
    lr = np.asarray([O.Config().lr[k] for k in O.PARAM_GROUP_OF_ROW])[:, None] * np.ones_like(p64)
    sure = np.zeros_like(p64, dtype=bool)
    for name, sl in {"mean": slice(0, 3), "logscale": slice(3, 6), "quat": slice(6, 10),
                     "opacity": slice(10, 11), "rgb": slice(11, 14)}.items():
        ref = g["grad"][sl]
        sure[sl] = np.abs(ref) > 10 * floor_frac * GRAD_RTOL * max(np.abs(ref).max(), 1e-30)
    sure &= keep[None, :]
    np.testing.assert_allclose(out["params"][sure], expect[sure], rtol=1e-6, atol=1e-6)
    step = np.abs(out["params"].astype(np.float64) - p64)
    assert np.all(step <= lr * (1 + 1e-5) + 1e-6)


@pytest.fixture(scope="module")
def small():
    p, cam = frustum_scene()
    tg = random_target(160, 120, seed=1)
    g, near, excl = oracle_ref(p, [cam], tg)
    return p, cam, tg, g, near, excl


@pytest.mark.parametrize("tile,ppt", LAYOUTS)
def test_fused_iteration_every_layout(small, tile, ppt):
    p, cam, tg, g, near, excl = small
    out = iterate_once(p, [cam], tg, tile_size=tile, pixels_per_thread=ppt)
    assert (out["tile"], out["ppt"]) == (tile, ppt)
    check_iteration(out, g, near, excl, p)


def test_fused_iteration_deterministic_mode(small):
    p, cam, tg, g, near, excl = small
    out = iterate_once(p, [cam], tg, deterministic=1)
    assert (out["tile"], out["ppt"]) == (8, 2)
    check_iteration(out, g, near, excl, p)


@pytest.mark.parametrize("tile,ppt", [(16, 2), (8, 1)])
def test_fused_window_of_three_views(small, tile, ppt):
    """Three views composited and back-propagated in one persistent launch."""
    p, cam, _, _, _, _ = small
    cams = [cam, rotated_cam(cam, [0.03, -0.05, 0.01], [0.05, 0.0, 0.1]),
            rotated_cam(cam, [-0.02, 0.06, 0.0], [-0.08, 0.02, -0.05])]
    tg = random_target(160, 120, seed=5, n_views=3)
    g, near, excl = oracle_ref(p, cams, tg)
    out = iterate_once(p, cams, tg, tile_size=tile, pixels_per_thread=ppt)
    # the rotated views hold more pixels near a discrete decision (0.5 %), all excluded
    check_iteration(out, g, near, excl, p, max_near=1e-2)


def multibatch_scene():
    """4,000 Gaussians of log-scale N(-2, 0.5) and opacity logit N(-2.5, 1) in a 64x64 view:
    16-px tile lists of 1,336 (median) to 1,932 records, pixels blending hundreds of them."""
    p, cam = frustum_scene(n=4000, width=64, height=64, fx=60, fy=60, cx=32, cy=32, seed=31,
                           logscale_mean=-2.0, logscale_std=0.5, opacity_mean=-2.5)
    return p, cam, random_target(64, 64, seed=3)


@pytest.fixture(scope="module")
def multibatch():
    p, cam, tg = multibatch_scene()
    g, near, excl = oracle_ref(p, [cam], tg)
    return p, cam, tg, g, near, excl


def _longest_list(out):
    bins, _ = out["pairs"]
    return int(np.bincount(bins.astype(np.int64)).max())


@pytest.mark.parametrize("tile,ppt", LAYOUTS + [("det", 2)])
def test_fused_iteration_across_staging_batches(multibatch, tile, ppt):
    p, cam, tg, g, near, excl = multibatch
    cfg = dict(deterministic=1) if tile == "det" else dict(tile_size=tile, pixels_per_thread=ppt)
    out = iterate_once(p, [cam], tg, **cfg)
    batch = 512 if out["tile"] * out["tile"] // out["ppt"] >= 128 else 256
    longest = _longest_list(out)
    assert longest > 2 * batch, (longest, batch)
    # the deepest blended entry of a pixel lies beyond the second batch of its tile's list
    ids = g["last"][0]
    bins, vals = out["pairs"]
    ntx = (64 + out["tile"] - 1) // out["tile"]
    start = np.concatenate([[0], np.cumsum(np.bincount(bins.astype(np.int64), minlength=ntx * ntx))])
    deepest = 0
    for py in range(0, 64, 3):
        for px in range(0, 64, 3):
            b = (py // out["tile"]) * ntx + px // out["tile"]
            seg = vals[start[b]:start[b + 1]]
            hit = np.nonzero(seg == ids[py, px])[0]
            if hit.size:
                deepest = max(deepest, int(hit[0]))
    assert deepest > 2 * batch, (deepest, batch)
    check_iteration(out, g, near, excl, p, max_near=0.1, floor_frac=GRAD_FLOOR_DEEP)


def test_render_backward_across_staging_batches(multibatch):
    """The separate compositing kernels of gs_render / gs_backward on the same long lists."""
    p, cam, tg, g, near, excl = multibatch
    gm = new_map(p.shape[1], W=64, H=64, tile_size=16, pixels_per_thread=1)
    gm.set_params(cuda(p))
    rgb = gm.render(cam).cpu().numpy()[0]
    L = gm.loss(cuda(tg)).cpu().numpy()
    gm.backward()
    grads = gm.grads().cpu().numpy()
    gm.close()
    err = np.abs(rgb - g["images"][0]).max(axis=0)
    assert err[~near[0]].max() <= IMG_ATOL
    assert abs(L[0] - g["loss"]) <= 1e-5 * g["loss"]
    errs = grad_errors(grads, g["grad"], exclude=excl, floor_frac=GRAD_FLOOR_DEEP)
    assert max(errs.values()) <= GRAD_RTOL, errs


@pytest.mark.parametrize("det", [False, True])
def test_dense_bins_pairs_bit_exact(det):
    """Dense bins: 10,000 Gaussians in 64x64, bins of up to 3,990 pairs at 16 px and 2,874 at 8 px
    (the deterministic mode's tiles); the pairs equal the oracle's binning bit for bit, and the
    image matches."""
    p, cam = frustum_scene(n=10000, width=64, height=64, fx=60, fy=60, cx=32, cy=32, seed=31,
                           logscale_mean=-2.2, logscale_std=0.5, opacity_mean=-4.5)
    cfg = dict(deterministic=1) if det else dict(tile_size=16, pixels_per_thread=1)
    gm = new_map(p.shape[1], W=64, H=64, **cfg)
    gm.set_params(cuda(p))
    rgb = gm.render(cam).cpu().numpy()[0]
    g = gm.debug_projection(0)
    bins, vals = gm.debug_pairs()
    tile = gm.tile_size
    gm.close()
    depth32 = g[5].astype(np.float32)
    keys_gpu = (bins.astype(np.uint64) << np.uint64(32)) | depth32[vals].view(np.uint32).astype(np.uint64)
    keys_ref, vals_ref = O.bin_pairs(g[0], g[1], g[6], depth32, g[8] > 0, 64, 64, tile)
    assert np.bincount(bins.astype(np.int64)).max() > 2048
    np.testing.assert_array_equal(keys_gpu, keys_ref)
    np.testing.assert_array_equal(vals, vals_ref)
    fwd = O.render(p.astype(np.float64), cam, flags=True)
    err = np.abs(rgb - fwd["rgb"]).max(axis=0)
    assert err[~fwd["near"]].max() <= IMG_ATOL


def one_tile_scene(tile, k, seed=41):
    """Exactly k Gaussians on a one-tile view (tile x tile pixels), every one certainly listed
    in its only tile: candidates of log-scale N(-3.5, 0.3) and opacity logit N(-2, 1) whose
    oracle screen mean lies at least 1.5 px inside the image, and which the oracle keeps
    (depth past the near plane, positive determinant), the first k of them."""
    c = tile / 2.0
    p, cam = frustum_scene(n=4 * k, width=tile, height=tile, fx=2.0 * tile, fy=2.0 * tile, cx=c, cy=c,
                           seed=seed, logscale_mean=-3.5, logscale_std=0.3, opacity_mean=-2.0)
    pr = O.project(torch.as_tensor(p, dtype=torch.float64), cam)
    inside = (pr["valid"] & ((pr["u"] - c).abs() < c - 1.5) & ((pr["v"] - c).abs() < c - 1.5)).numpy()
    keep = np.nonzero(inside)[0][:k]
    assert keep.size == k
    return np.ascontiguousarray(p[:, keep]), cam, random_target(tile, tile, seed=seed + 1)


@pytest.mark.parametrize("tile,ppt", LAYOUTS)
@pytest.mark.parametrize("extra", [0, 1])
def test_fused_iteration_at_the_staging_batch_boundary(tile, ppt, extra):
    """A tile list of exactly one staging batch (the adjoint reuses the forward's staged batch
    and, except at 16x2, starts without CTA barriers) and of one batch plus one record (the
    adjoint stages the list again, in two batches)."""
    threads = tile * tile // ppt
    batch = 512 if threads >= 128 else 256
    p, cam, tg = one_tile_scene(tile, batch + extra)
    g, near, excl = oracle_ref(p, [cam], tg)
    out = iterate_once(p, [cam], tg, tile_size=tile, pixels_per_thread=ppt)
    assert _longest_list(out) == batch + extra
    # a pixel of this small view near a discrete decision counts for 1 / tile^2 of the image
    check_iteration(out, g, near, excl, p, max_near=0.05)


def test_render_of_another_shape_between_replays(small):
    """A replayed iteration composites in the order the previous replay left in the graph's own
    buffer; a gs_render of another shape in between (which writes the context's work order)
    must not change it. Deterministic mode: the two maps end bit for bit equal."""
    p, cam, _, _, _, _ = small
    cams = [cam, rotated_cam(cam, [0.03, -0.05, 0.01], [0.05, 0.0, 0.1]),
            rotated_cam(cam, [-0.02, 0.06, 0.0], [-0.08, 0.02, -0.05])]
    tg = cuda(random_target(160, 120, seed=5, n_views=3))
    out = []
    for interleave in (False, True):
        gm = new_map(p.shape[1], views=3, deterministic=1)
        gm.set_params(cuda(p))
        loss = torch.empty(3, device="cuda")
        for it in range(4):
            gm.iterate(cams, tg, loss)
            if interleave and it == 1:
                gm.render(cams[0])   # one view: a third of the bins
        torch.cuda.synchronize()
        out.append(gm.params().cpu().numpy())
        gm.close()
    assert np.array_equal(out[0], out[1])


def test_phase_timing_does_not_change_results(small):
    """Per-phase timing adds event-record nodes to the captured iteration (on both of its
    branches); the arithmetic is the same with and without them. Deterministic mode, 3-view
    window: bit for bit, and every phase was timed."""
    p, cam, _, _, _, _ = small
    cams = [cam, rotated_cam(cam, [0.03, -0.05, 0.01], [0.05, 0.0, 0.1]),
            rotated_cam(cam, [-0.02, 0.06, 0.0], [-0.08, 0.02, -0.05])]
    tg = cuda(random_target(160, 120, seed=7, n_views=3))
    out = []
    for timed in (False, True):
        gm = new_map(p.shape[1], views=3, deterministic=1)
        gm.set_params(cuda(p))
        if timed:
            gm.timing(True)
        loss = torch.empty(3, device="cuda")
        for _ in range(3):
            gm.iterate(cams, tg, loss)
        torch.cuda.synchronize()
        if timed:
            rec = gm.timing_read()
            for name in ("project", "bin", "raster_fused", "loss", "project_bwd", "adam"):
                assert rec[name][1] >= 3 and rec[name][0] > 0.0, (name, rec[name])
        out.append((gm.params().cpu().numpy(), loss.cpu().numpy()))
        gm.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])

"""GPU parity of the map-management calls against the FP64 oracle.

* gs_init_map: Eq. 6 map initialisation (plain initialisation, neighbours = the other new points);
* gs_insert: the opacity-gated insertion reading of Eq. 7 with the plain initialisation;
* gs_densify: the NDC gradient-norm split of the densification reading, with given normal samples.
Decisions taken in floating point (opacity > 0.99, mean gradient norm > threshold) are
compared only where they lie well away from their thresholds; the rest is compared
element by element.
"""
import numpy as np
import pytest
import torch

import oracle as O
from synth import Camera, frustum_scene, random_target

from gpu_helpers import cuda, new_map

pytestmark = pytest.mark.gpu


def test_init_map_matches_oracle():
    rng = np.random.default_rng(7)
    pts = rng.normal(size=(500, 3)).astype(np.float32) * np.array([1.0, 0.5, 2.0], np.float32)
    rgb = rng.uniform(size=(500, 3)).astype(np.float32)
    gm = new_map(2000)
    gm.init_map(cuda(pts), cuda(rgb))
    assert gm.n == 500
    got = gm.params().cpu().numpy()
    ref = O.init_map(pts.astype(np.float64), rgb.astype(np.float64))
    np.testing.assert_array_equal(got[0:3], pts.T)
    np.testing.assert_allclose(got[3:6], ref[3:6], rtol=0, atol=2e-6)
    np.testing.assert_array_equal(got[6:11], ref[6:11].astype(np.float32))
    np.testing.assert_array_equal(got[11:14], rgb.T)
    # a second call appends, with its own points as the only neighbours
    pts2 = pts[:7] + np.float32(0.001)
    gm.init_map(cuda(pts2), cuda(rgb[:7]))
    got2 = gm.params().cpu().numpy()[:, 500:]
    ref2 = O.init_map(pts2.astype(np.float64), rgb[:7].astype(np.float64))
    np.testing.assert_allclose(got2[3:6], ref2[3:6], rtol=0, atol=2e-6)


def _points_at(cam, pixels, z):
    pixels = np.asarray(pixels, np.float64)
    x = (pixels[:, 0] - cam.cx) / cam.fx * z
    y = (pixels[:, 1] - cam.cy) / cam.fy * z
    return np.stack([x, y, np.full(len(pixels), z)], 1).astype(np.float32)


def test_insert_matches_oracle():
    p, cam = frustum_scene(n=2000, seed=0)
    image = random_target(160, 120, seed=3)[0]
    p64 = p.astype(np.float64)
    T = O.render(p64, cam)["T"]
    opac = 1.0 - T
    rng = np.random.default_rng(11)
    yy, xx = np.nonzero(opac > 0.991)                 # skipped (opacity clearly above 0.99)
    y2, x2 = np.nonzero(opac < 0.989)                 # inserted
    a = rng.choice(len(xx), size=min(60, len(xx)), replace=False)
    b = rng.choice(len(x2), size=60, replace=False)
    pix = np.concatenate([np.stack([xx[a], yy[a]], 1), np.stack([x2[b], y2[b]], 1)])
    pts = _points_at(cam, pix, 2.5)
    pts = np.concatenate([pts, np.array([[0.0, 0.0, -1.0], [50.0, 0.0, 1.0]], np.float32)])  # behind, off-image
    order = rng.permutation(len(pts))
    pts = pts[order]
    gm = new_map(4000)
    gm.set_params(cuda(p))
    n_ins = gm.insert(cam, cuda(image), cuda(pts))
    mask, pixels, inside = O.insertion_mask(pts.astype(np.float64), cam, T)
    assert n_ins == int(mask.sum()) and gm.n == 2000 + n_ins
    got = gm.params().cpu().numpy()[:, 2000:]
    ref = O.plain_init(pts[mask].astype(np.float64), pixels[mask], image, p64[0:3].T)
    np.testing.assert_array_equal(got[0:3], pts[mask].T)
    np.testing.assert_allclose(got[3:6], ref[3:6], rtol=0, atol=2e-6)
    np.testing.assert_array_equal(got[6:11], ref[6:11].astype(np.float32))
    np.testing.assert_array_equal(got[11:14], ref[11:14].astype(np.float32))
    # the original map is untouched
    np.testing.assert_array_equal(gm.params().cpu().numpy()[:, :2000], p)


def test_insert_into_empty_map_and_capacity():
    cam = Camera(40, 30, 50.0, 50.0, 20.0, 15.0)
    image = random_target(40, 30, seed=2)[0]
    pts = _points_at(cam, [[3, 4], [20, 15], [39, 29]], 1.5)
    gm = new_map(4, W=40, H=30)
    assert gm.insert(cam, cuda(image), cuda(pts)) == 3
    got = gm.params().cpu().numpy()
    np.testing.assert_allclose(got[3:6], np.log(0.01), rtol=1e-6)          # no neighbours: 0.01 m
    np.testing.assert_array_equal(got[11:14, 1], image[:, 15, 20])
    from paper_2504_02437_gb300._native import GSError, GS_ERR_CAPACITY
    with pytest.raises(GSError) as e:
        gm.insert(cam, cuda(image), cuda(pts))                             # 3 + 3 > 4
    assert e.value.code == GS_ERR_CAPACITY
    assert gm.n == 3


def test_densify_matches_oracle():
    p, cam = frustum_scene(n=2000, seed=1)
    tg = random_target(160, 120, seed=9)
    p64 = p.astype(np.float64)
    ref = O.loss_and_grads(p64, [cam], tg, want_2d=True)
    pr = O.project(torch.tensor(p64), cam)
    s, c = O.screen_grad_norms(ref["grad2d"], [pr["valid"].numpy()], [(cam.width, cam.height)])
    mean = np.where(c > 0, s / np.maximum(c, 1), 0.0)
    # a threshold in a wide gap of the statistic, so float32 rounding cannot move a decision
    srt = np.sort(mean[mean > 0])
    gaps = srt[1:] / srt[:-1]
    lo = int(0.7 * len(srt))
    i = lo + int(np.argmax(gaps[lo:]))
    assert gaps[i] > 1.01
    thresh = float(np.sqrt(srt[i] * srt[i + 1]))
    gm = new_map(4000, split_thresh=thresh)
    gm.set_params(cuda(p))
    gm.render(cam)
    gm.loss(cuda(tg))
    gm.backward()
    z = np.random.default_rng(4).normal(size=(2000, 2, 3)).astype(np.float32)
    n_split = gm.densify(cuda(z))
    zero = np.zeros_like(p64)
    newP, _, _, mask = O.split(p64, zero, zero, s, c, z.astype(np.float64), O.Config(split_thresh=thresh))
    assert n_split == int(mask.sum()) > 0
    got = gm.params().cpu().numpy()
    assert got.shape == newP.shape
    n_keep = 2000 - n_split
    np.testing.assert_array_equal(got[:, :n_keep], p[:, ~mask])
    np.testing.assert_allclose(got[0:3, n_keep:], newP[0:3, n_keep:], rtol=0, atol=1e-6)
    np.testing.assert_allclose(got[3:6, n_keep:], newP[3:6, n_keep:], rtol=0, atol=1e-6)
    np.testing.assert_array_equal(got[6:14, n_keep:], newP[6:14, n_keep:].astype(np.float32))
    # statistics are reset: a second densify splits nothing
    assert gm.densify(cuda(np.zeros((gm.n, 2, 3), np.float32))) == 0

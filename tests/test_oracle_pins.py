"""Pins of the FP64 oracle to the paper and to mathematics (no GPU).

Each test checks the oracle against something other than itself: a hand-derived
closed form of Eq. 1-3, an independent library routine (scipy rotations,
torch.optim.Adam), a numerical derivative, brute force over tiles, or an
invariant of the definitions.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from synth import Camera, frustum_scene, random_target

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CFG = O.Config()


def _params(means, logscales, quats, logits, rgbs):
    n = len(means)
    p = np.zeros((14, n))
    p[0:3] = np.asarray(means, float).T
    p[3:6] = np.asarray(logscales, float).reshape(n, 3).T
    p[6:10] = np.asarray(quats, float).reshape(n, 4).T
    p[10] = logits
    p[11:14] = np.asarray(rgbs, float).T
    return p


def _logit(o):
    return math.log(o / (1.0 - o))


def _axis_cam(f=100.0, size=64):
    return Camera(size, size, f, f, size / 2, size / 2)


# ------------------------------------------------------------------ paper constants


def test_paper_constants_match_config():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    assert CFG.reg_floor == g["reg_floor"]["value"]          # Eq. 10
    assert CFG.insert_opacity == g["insert_opacity"]["value"]
    assert CFG.split_thresh == g["split_thresh"]["value"]


# ------------------------------------------------------------------ Eq. 1


def test_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    q = rng.normal(size=(50, 4))
    R = O.quat_to_rotmat(torch.tensor(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()     # scipy is scalar-last
    np.testing.assert_allclose(R, ref, atol=1e-13)


def test_covariance_of_axis_rotation():
    # 90 degrees about z maps x->y, y->-x, so Sigma = diag(s2^2, s1^2, s3^2)
    s = np.array([0.1, 0.2, 0.3])
    q = np.array([[math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]])
    S = O.cov3d(torch.tensor(np.log(s))[None], torch.tensor(q)).numpy()[0]
    np.testing.assert_allclose(S, np.diag([0.04, 0.01, 0.09]), atol=1e-15)
    # unnormalised quaternion: same rotation
    S2 = O.cov3d(torch.tensor(np.log(s))[None], torch.tensor(3.7 * q)).numpy()[0]
    np.testing.assert_allclose(S2, S, atol=1e-15)


# ------------------------------------------------------------------ Eq. 2


def _pinhole(t, cam):
    return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cov2d_is_numerical_jacobian_sandwich(seed):
    """Sigma2D - 0.3 I = J W Sigma W^T J^T with J the central-difference Jacobian of the pinhole map."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    Rw = Rotation.from_rotvec(rng.normal(size=3) * 0.5).as_matrix()
    cam = Camera(320, 240, 300.0, 280.0, 160.0, 120.0, Rw, rng.normal(size=3) * 0.3)
    # a mean in front of the camera, well inside the FOV clamp
    tcam = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(2, 4)])
    mu = Rw.T @ (tcam - cam.t)
    ls = rng.normal(-2, 0.4, size=3)
    q = rng.normal(size=4)
    p = _params([mu], [ls], [q], [0.0], [[0.5, 0.5, 0.5]])
    pr = O.project(torch.tensor(p), cam)
    h = 1e-6
    J = np.stack([(_pinhole(tcam + h * e, cam) - _pinhole(tcam - h * e, cam)) / (2 * h) for e in np.eye(3)], 1)
    from scipy.spatial.transform import Rotation as Rt
    Rg = Rt.from_quat(q[[1, 2, 3, 0]]).as_matrix()
    Sig = Rg @ np.diag(np.exp(2 * ls)) @ Rg.T
    expect = J @ Rw @ Sig @ Rw.T @ J.T
    got = pr["cov2d"].numpy()[0] - CFG.dilation * np.eye(2)
    np.testing.assert_allclose(got, expect, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose([pr["u"].item(), pr["v"].item()], _pinhole(tcam, cam), rtol=1e-12)
    assert abs(pr["depth"].item() - tcam[2]) < 1e-12
    # conic is the inverse of the dilated covariance
    cov = pr["cov2d"].numpy()[0]
    inv = np.linalg.inv(cov)
    np.testing.assert_allclose([pr["a"].item(), pr["b"].item(), pr["c"].item()], [inv[0, 0], inv[0, 1], inv[1, 1]],
                               rtol=1e-10)


def test_isotropic_on_axis_closed_form():
    """Identity pose, mean (0, 0, z), isotropic scale s: Sigma2D = ((f s / z)^2 + 0.3) I."""
    f, z, s, o = 100.0, 2.0, 0.05, 0.5
    cam = _axis_cam(f)
    c = [0.2, 0.6, 1.0]
    p = _params([[0, 0, z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [_logit(o)], [c])
    pr = O.project(torch.tensor(p), cam)
    sig2 = (f * s / z) ** 2 + 0.3                               # 6.55
    np.testing.assert_allclose(pr["cov2d"].numpy()[0], sig2 * np.eye(2), rtol=1e-14)
    lam = sig2 + math.sqrt(0.1)                                  # discriminant 0 floored at 0.1
    r = math.ceil(3 * math.sqrt(lam))
    assert r == 8 and pr["r"].item() == r
    offsets = [(0, 0), (3, 0), (0, -4), (5, 5), (7, 0), (8, 0), (9, 0), (-6, 3), (8, 8), (-8, 7)]
    pix = np.array([[32 + dx, 32 + dy] for dx, dy in offsets])
    out = O.render(p, cam, pixels=pix)
    for k, (dx, dy) in enumerate(offsets):
        a = min(0.99, o * math.exp(-(dx * dx + dy * dy) / (2 * sig2)))
        if max(abs(dx), abs(dy)) > r or a < 1 / 255:
            a = 0.0
        np.testing.assert_allclose(out["rgb"][k], np.array(c) * a, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(out["T"][k], 1 - a, rtol=1e-12)
    # (8, 0): alpha = 0.5 exp(-64/13.1) = 0.00378 < 1/255 is skipped although a member;
    # (7, 0): 0.0119 blends
    assert out["n_contrib"][offsets.index((8, 0))] == 0
    assert out["n_contrib"][offsets.index((7, 0))] == 1


def test_off_axis_isotropic_hand_jacobian():
    """Off-axis isotropic Gaussian: J = [[f/z, 0, -f x/z^2], [0, f/z, -f y/z^2]] written by hand."""
    f, s = 120.0, 0.07
    x, y, z = 0.3, -0.2, 2.5
    cam = _axis_cam(f, 96)
    p = _params([[x, y, z]], [[math.log(s)] * 3], [[0.3, 0.1, -0.5, 0.2]], [0.0], [[1, 1, 1]])
    pr = O.project(torch.tensor(p), cam)
    J = np.array([[f / z, 0, -f * x / z ** 2], [0, f / z, -f * y / z ** 2]])
    expect = s * s * J @ J.T + 0.3 * np.eye(2)                   # rotation-invariant (isotropic)
    np.testing.assert_allclose(pr["cov2d"].numpy()[0], expect, rtol=1e-13)


def test_fov_clamp_of_jacobian():
    """Beyond 1.3 x the half-FOV tangent, J uses the clamped x/z (reading of Eq. 2)."""
    f, s, z = 100.0, 0.05, 1.0
    cam = _axis_cam(f, 64)                       # half-FOV tangent 0.32 -> clamp 0.416
    x = 0.8                                      # x/z = 0.8 > 0.416
    p = _params([[x, 0, z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [0.0], [[1, 1, 1]])
    pr = O.project(torch.tensor(p), cam)
    xh = 1.3 * 0.32
    J = np.array([[f / z, 0, -f * xh / z], [0, f / z, 0]])
    np.testing.assert_allclose(pr["cov2d"].numpy()[0], s * s * J @ J.T + 0.3 * np.eye(2), rtol=1e-13)
    assert bool(pr["tclamp"][0, 0]) and not bool(pr["tclamp"][0, 1])


def test_culling_near_plane_and_offscreen():
    cam = _axis_cam()
    p = _params([[0, 0, 0.19], [0, 0, 0.21], [100, 0, 1.0], [0, 0, -1.0]], [[-3] * 3] * 4,
                [[1, 0, 0, 0]] * 4, [0.0] * 4, [[1, 1, 1]] * 4)
    pr = O.project(torch.tensor(p), cam)
    assert pr["valid"].tolist() == [False, True, False, False]


# ------------------------------------------------------------------ Eq. 3


def _stack(opacities, rgbs, depths, scale=0.3):
    n = len(depths)
    return _params([[0, 0, d] for d in depths], [[math.log(scale)] * 3] * n, [[1, 0, 0, 0]] * n,
                   [_logit(o) for o in opacities], rgbs)


def test_stack_alpha_095_closed_form():
    """Five layers with alpha 0.95 at their common centre pixel: T after k layers is 0.05^k;
    0.05^4 = 6.25e-6 < 1e-4 stops before the fourth, so three layers blend."""
    cols = [[0.9, 0.1, 0.2], [0.3, 0.8, 0.1], [0.2, 0.3, 0.7], [0.5, 0.5, 0.5], [1.0, 1.0, 0.0]]
    p = _stack([0.95] * 5, cols, [1, 2, 3, 4, 5])
    out = O.render(p, _axis_cam(), pixels=np.array([[32, 32]]))
    expect = sum(np.array(cols[i]) * 0.95 * 0.05 ** i for i in range(3))
    np.testing.assert_allclose(out["rgb"][0], expect, rtol=1e-13)
    np.testing.assert_allclose(out["T"][0], 0.05 ** 3, rtol=1e-12)
    assert out["n_contrib"][0] == 3 and out["last"][0] == 2 and out["argmax"][0] == 0


def test_stack_alpha_099_boundary():
    """o = 0.999 is clamped to alpha = 0.99. In float64 T after two layers is 1.0000000000000018e-4,
    not below 1e-4, so two layers blend (the float32 case falls below and blends one)."""
    cols = [[0.9, 0.1, 0.2], [0.3, 0.8, 0.1], [0.2, 0.3, 0.7]]
    p = _stack([0.999] * 3, cols, [1, 2, 3])
    out = O.render(p, _axis_cam(), pixels=np.array([[32, 32]]))
    t1 = 1 - 0.99
    np.testing.assert_allclose(out["rgb"][0], 0.99 * np.array(cols[0]) + 0.99 * t1 * np.array(cols[1]), rtol=1e-13)
    assert out["n_contrib"][0] == 2
    np.testing.assert_allclose(out["T"][0], t1 * t1, rtol=1e-12)


def test_transmittance_is_product():
    rng = np.random.default_rng(5)
    ops = rng.uniform(0.05, 0.5, size=6)
    cols = rng.uniform(size=(6, 3))
    p = _stack(ops, cols, [1, 1.5, 2, 2.5, 3, 3.5])
    out = O.render(p, _axis_cam(), pixels=np.array([[32, 32]]))
    np.testing.assert_allclose(out["T"][0], np.prod(1 - ops), rtol=1e-12)
    expect = sum(cols[i] * ops[i] * np.prod(1 - ops[:i]) for i in range(6))
    np.testing.assert_allclose(out["rgb"][0], expect, rtol=1e-12)


def test_equal_depths_blend_in_id_order():
    """Two layers at the same depth (o = 0.6 and 0.3): the lower id blends first, so
    C = 0.6 c0 + 0.3 (1 - 0.6) c1; swapping the array order swaps which colour is in front."""
    red, blue = [1, 0, 0], [0, 0, 1]
    p = _stack([0.6, 0.3], [red, blue], [2.0, 2.0])
    out = O.render(p, _axis_cam(), pixels=np.array([[32, 32]]))
    np.testing.assert_allclose(out["rgb"][0], [0.6, 0.0, 0.12], rtol=1e-13, atol=1e-16)
    p = _stack([0.3, 0.6], [blue, red], [2.0, 2.0])
    out = O.render(p, _axis_cam(), pixels=np.array([[32, 32]]))
    np.testing.assert_allclose(out["rgb"][0], [0.42, 0.0, 0.3], rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(out["T"][0], 0.28, rtol=1e-13)


def test_alpha_min_is_strict_threshold():
    c = [0.5, 0.25, 1.0]
    for o, blends in [(1 / 255 + 1e-6, True), (1 / 255 - 1e-6, False)]:
        p = _stack([o], [c], [2.0])
        out = O.render(p, _axis_cam(), pixels=np.array([[32, 32]]))
        if blends:
            np.testing.assert_allclose(out["rgb"][0], np.array(c) * o, rtol=1e-12)
        else:
            assert np.all(out["rgb"][0] == 0) and out["T"][0] == 1.0


def test_depth_order_and_array_order_invariance():
    """Front red (depth 1), back blue (depth 2), o = 0.6: C = 0.6 red + 0.24 blue whatever the array order."""
    red, blue = [1, 0, 0], [0, 0, 1]
    for depths, cols in [([1, 2], [red, blue]), ([2, 1], [blue, red])]:
        p = _stack([0.6, 0.6], cols, depths)
        out = O.render(p, _axis_cam(), pixels=np.array([[32, 32]]))
        np.testing.assert_allclose(out["rgb"][0], [0.6, 0.0, 0.24], rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(out["T"][0], 0.16, rtol=1e-13)


def test_full_image_permutation_invariance():
    p, cam = frustum_scene(n=200, width=48, height=40, fx=60, fy=60, cx=24, cy=20, seed=7)
    perm = np.random.default_rng(1).permutation(200)
    a = O.render(p, cam)
    b = O.render(p[:, perm], cam)
    # identical blending order; batched BLAS calls may round the last bit differently by position
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(a["T"], b["T"], rtol=1e-14)
    np.testing.assert_array_equal(perm[b["last"][b["last"] >= 0]], a["last"][a["last"] >= 0])


def test_pixel_membership_box():
    """A Gaussian is seen only inside |px-u| <= r, |py-v| <= r; opaque and huge inside."""
    cam = _axis_cam(100.0, 64)
    p = _params([[0.005, -0.003, 1.0]], [[math.log(0.03)] * 3], [[1, 0, 0, 0]], [_logit(0.9)], [[1, 1, 1]])
    pr = O.project(torch.tensor(p), cam)
    u, v, r = pr["u"].item(), pr["v"].item(), pr["r"].item()
    out = O.render(p, cam)
    ys, xs = np.nonzero(out["n_contrib"] > 0)
    assert np.all(np.abs(xs - u) <= r) and np.all(np.abs(ys - v) <= r)


# ------------------------------------------------------------------ binning and sort


def _brute_pairs(u, v, r, depth, valid, W, H, tile):
    ntx, nty = -(-W // tile), -(-H // tile)
    out = []
    for ty in range(nty):
        for tx in range(ntx):
            for i in range(len(u)):
                if not valid[i]:
                    continue
                # pixels of this tile that pass the membership box
                hit = False
                for py in range(ty * tile, min(H, (ty + 1) * tile)):
                    if abs(py - v[i]) > r[i]:
                        continue
                    for px in range(tx * tile, min(W, (tx + 1) * tile)):
                        if abs(px - u[i]) <= r[i]:
                            hit = True
                            break
                    if hit:
                        break
                if hit:
                    key = ((ty * ntx + tx) << 32) | int(np.float32(depth[i]).view(np.uint32))
                    out.append((key, i))
    out.sort()
    return out


@pytest.mark.parametrize("tile", [4, 8, 16])
def test_bin_pairs_brute_force(tile):
    p, cam = frustum_scene(n=40, width=37, height=29, fx=40, fy=40, cx=18.5, cy=14.5, seed=11)
    pr = O.project(torch.tensor(p, dtype=torch.float64), cam)
    u = pr["u"].numpy().astype(np.float32).astype(np.float64)
    v = pr["v"].numpy().astype(np.float32).astype(np.float64)
    r, d, ok = pr["r"].numpy(), pr["depth"].numpy().astype(np.float32), pr["valid"].numpy()
    keys, vals = O.bin_pairs(u, v, r, d, ok, cam.width, cam.height, tile)
    ref = _brute_pairs(u, v, r, d, ok, cam.width, cam.height, tile)
    assert [(int(k), int(x)) for k, x in zip(keys, vals)] == ref
    cnt = O.tiles_touched(u, v, r, ok, cam.width, cam.height, tile)
    assert cnt.sum() == len(ref)


def test_bin_pairs_equal_depths_keep_id_order():
    """Gaussians at equal depth in one tile are ordered by id (the sort is stable on the
    depth-sorted item order): depths snapped to three values, against the brute force."""
    p, cam = frustum_scene(n=60, width=37, height=29, fx=40, fy=40, cx=18.5, cy=14.5, seed=12)
    pr = O.project(torch.tensor(p, dtype=torch.float64), cam)
    u = pr["u"].numpy().astype(np.float32).astype(np.float64)
    v = pr["v"].numpy().astype(np.float32).astype(np.float64)
    r, ok = pr["r"].numpy(), pr["valid"].numpy()
    d = np.float32([1.5, 2.0, 2.5])[np.arange(len(u)) % 3]
    keys, vals = O.bin_pairs(u, v, r, d, ok, cam.width, cam.height, 8)
    ref = _brute_pairs(u, v, r, d, ok, cam.width, cam.height, 8)
    assert [(int(k), int(x)) for k, x in zip(keys, vals)] == ref
    # the case is not vacuous: some tile holds several Gaussians of one depth
    ties = {}
    for k, x in ref:
        ties[k] = ties.get(k, 0) + 1
    assert max(ties.values()) >= 3


# ------------------------------------------------------------------ Eq. 10-11 and gradients


def test_l1_gradient_of_colour_closed_form():
    """dL/dc of a lone Gaussian = lambda/(3HW) sum_p sign(C_p - I_p) alpha_p (its blend weight)."""
    cam = _axis_cam(100.0, 24)
    p = _params([[0.01, 0.02, 1.0]], [[math.log(0.04)] * 3], [[1, 0.2, 0, 0]], [0.3], [[0.3, 0.6, 0.9]])
    tg = np.random.default_rng(0).uniform(size=(1, 3, 24, 24))
    res = O.loss_and_grads(p, [cam], tg)
    img = res["images"][0]
    alpha = 1 - res["T"][0]                       # single Gaussian: weight = alpha = 1 - T
    expect = (np.sign(img - tg[0]) * alpha[None]).sum((1, 2)) / (3 * 24 * 24)
    np.testing.assert_allclose(res["grad"][11:14, 0], expect, rtol=1e-12)


def test_planar_gradient_closed_form():
    """With nothing in view, dL/dlog-scale = (lambda_reg / N) s_min on the smallest axis if s_min > 0.01."""
    cam = _axis_cam()
    ls = [[math.log(0.05), math.log(0.02), math.log(0.3)], [math.log(0.005), 0.0, 0.0], [-1.0, -2.0, -1.5]]
    p = _params([[0, 0, -1]] * 3, ls, [[1, 0, 0, 0]] * 3, [0.0] * 3, [[1, 1, 1]] * 3)
    res = O.loss_and_grads(p, [cam], np.zeros((1, 3, 64, 64)))
    g = res["grad"][3:6]
    expect = np.zeros((3, 3))
    expect[1, 0] = 0.02 / 3                       # min 0.02 on axis 1
    expect[1, 2] = math.exp(-2.0) / 3             # min exp(-2) on axis 1
    np.testing.assert_allclose(g, expect, rtol=1e-12, atol=1e-300)
    assert res["reg"] == pytest.approx((0.02 + 0.01 + math.exp(-2.0)) / 3, rel=1e-13)
    assert np.all(res["grad"][[0, 1, 2, 6, 7, 8, 9, 10, 11, 12, 13]] == 0)


def _fd_check(p, cams, tg, rows=None, cols=None, rel_h=1e-6, tol=1e-6):
    """Central differences with h = rel_h max(1, |p|). Bound: tol |g| plus the float64
    rounding of the difference quotient, 100 eps |L| / h."""
    res = O.loss_and_grads(p, cams, tg)
    g = res["grad"]
    L = abs(res["loss"])
    base = O.decision_signature(p, cams)
    rows = range(14) if rows is None else rows
    cols = range(p.shape[1]) if cols is None else cols
    checked = skipped = 0
    worst = 0.0
    scale = np.abs(g).max()
    for i in rows:
        for j in cols:
            h = rel_h * max(1.0, abs(p[i, j]))
            pp, pm = p.copy(), p.copy()
            pp[i, j] += h
            pm[i, j] -= h
            if O.decision_signature(pp, cams) != base or O.decision_signature(pm, cams) != base:
                skipped += 1
                continue
            fd = (O.loss_value(pp, cams, tg) - O.loss_value(pm, cams, tg)) / (2 * h)
            bound = tol * abs(g[i, j]) + 100 * np.finfo(float).eps * L / h
            assert abs(fd - g[i, j]) <= bound, (i, j, fd, g[i, j], bound)
            worst = max(worst, abs(fd - g[i, j]) / max(abs(g[i, j]), 1e-3 * scale))
            checked += 1
    return checked, skipped


@pytest.mark.parametrize("seed,n", [(0, 1), (1, 3), (2, 5)])
def test_gradient_finite_differences_tiny(seed, n):
    """Central differences of the Eq. 11 loss vs the oracle's gradient on 16x16 scenes, random pose."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(100 + seed)
    Rw = Rotation.from_rotvec(rng.normal(size=3) * 0.2).as_matrix()
    cam = Camera(16, 16, 20.0, 22.0, 8.0, 7.5, Rw, rng.normal(size=3) * 0.05)
    tc = np.stack([rng.uniform(-0.25, 0.25, n), rng.uniform(-0.25, 0.25, n), rng.uniform(1.0, 2.0, n)], 1)
    mu = (tc - cam.t) @ Rw
    p = _params(mu, rng.normal(-2.0, 0.3, size=(n, 3)), rng.normal(size=(n, 4)), rng.normal(0.5, 1, n),
                rng.uniform(size=(n, 3)))
    tg = rng.uniform(size=(1, 3, 16, 16))
    checked, skipped = _fd_check(p, [cam], tg)
    assert checked >= 0.8 * 14 * n


def _clamp_scene(front_opacity):
    """A wide Gaussian in front (sigma about 1,000 px at depth 2, so G > 0.9999 over the 12x12
    image) and a small one behind it."""
    return _params([[0.003, -0.002, 2.0], [0.01, 0.005, 3.0]],
                   [[math.log(20.0), math.log(25.0), math.log(30.0)], [math.log(0.05)] * 3],
                   [[1, 0.1, -0.2, 0.05], [1, 0, 0.3, 0]], [_logit(front_opacity), 0.0],
                   [[0.3, 0.6, 0.9], [0.8, 0.2, 0.4]])


def test_alpha_clamp_blocks_gradients():
    """Eq. 3 with alpha = min(0.99, o G): where o G > 0.99 at every pixel the front Gaussian
    covers, its alpha is the constant 0.99, so the image does not depend on its opacity, scale,
    rotation or mean. Central differences of the loss are zero for those parameters (to the
    rounding of the difference quotient), and the oracle's gradient is exactly zero; its colour
    gradient is lambda / (3HW) sum_p sign(C_p - I_p) 0.99. The same scene with an unclamped front
    Gaussian (control) has non-zero gradients there, equal to the central differences."""
    cam = _axis_cam(100.0, 12)
    cfg = O.Config(lambda_reg=0.0)
    tg = np.random.default_rng(5).uniform(size=(1, 3, 12, 12))
    for front, clamped in ((0.9999, True), (0.5, False)):
        p = _clamp_scene(front)
        pr = O.project(torch.tensor(p), cam, cfg)
        py, px = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")
        res = O.composite(px.ravel(), py.ravel(), pr, cfg)
        res_all = O.loss_and_grads(p, [cam], tg, cfg)
        g = res_all["grad"]
        L = abs(res_all["loss"])
        # the front Gaussian's o G at every pixel, from its conic
        with torch.no_grad():
            dx = torch.tensor(px.ravel(), dtype=torch.float64) - pr["u"][0]
            dy = torch.tensor(py.ravel(), dtype=torch.float64) - pr["v"][0]
            oG = pr["o"][0] * torch.exp(-0.5 * (pr["a"][0] * dx * dx + pr["c"][0] * dy * dy) - pr["b"][0] * dx * dy)
        assert bool((oG > 0.99).all()) == clamped and bool((oG < 0.99).all()) != clamped
        for i in range(11):
            h = 1e-6 * max(1.0, abs(p[i, 0]))
            pp, pm = p.copy(), p.copy()
            pp[i, 0] += h
            pm[i, 0] -= h
            assert O.decision_signature(pp, [cam], cfg) == O.decision_signature(pm, [cam], cfg)
            fd = (O.loss_value(pp, [cam], tg, cfg) - O.loss_value(pm, [cam], tg, cfg)) / (2 * h)
            bound = 1e-6 * abs(g[i, 0]) + 100 * np.finfo(float).eps * L / h
            assert abs(fd - g[i, 0]) <= bound, (i, fd, g[i, 0])
            if clamped:
                assert g[i, 0] == 0.0, (i, g[i, 0])
        if clamped:
            img = res_all["images"][0]
            expect = (np.sign(img - tg[0]) * 0.99).sum((1, 2)) / (3 * 12 * 12)
            np.testing.assert_allclose(g[11:14, 0], expect, rtol=1e-12)
        else:
            assert abs(g[10, 0]) > 1e-3 and np.abs(g[0:3, 0]).max() > 1e-6
        assert int(res["n_contrib"].max()) == 2      # the back Gaussian blends behind it


@pytest.mark.slow
def test_gradient_finite_differences_64_gaussians_32px():
    """The 64-Gaussian 32x32 subset of the stream workload, two views (window loss)."""
    p, cam = frustum_scene(n=64, width=32, height=32, fx=30, fy=30, cx=16, cy=16, seed=21)
    from scipy.spatial.transform import Rotation
    cam2 = Camera(32, 32, 30.0, 30.0, 16.0, 16.0, Rotation.from_rotvec([0.05, -0.08, 0.02]).as_matrix(),
                  np.array([0.05, 0.0, 0.1]))
    tg = np.random.default_rng(2).uniform(size=(2, 3, 32, 32))
    p = p.astype(np.float64)
    cols = np.random.default_rng(3).choice(64, size=16, replace=False)
    checked, skipped = _fd_check(p, [cam, cam2], tg, cols=cols)
    assert checked >= 0.8 * 14 * 16


def test_window_gradient_is_sum_of_views():
    p, cam = frustum_scene(n=60, width=32, height=24, fx=30, fy=30, cx=16, cy=12, seed=4)
    from scipy.spatial.transform import Rotation
    cam2 = Camera(32, 24, 30.0, 30.0, 16.0, 12.0, Rotation.from_rotvec([0.02, 0.1, 0.0]).as_matrix(),
                  np.array([0.1, 0.0, 0.0]))
    tg = np.random.default_rng(0).uniform(size=(2, 3, 24, 32))
    cfg0 = O.Config(lambda_reg=0.0)
    both = O.loss_and_grads(p, [cam, cam2], tg, cfg0)
    a = O.loss_and_grads(p, [cam], tg[:1], cfg0)
    b = O.loss_and_grads(p, [cam2], tg[1:], cfg0)
    np.testing.assert_allclose(both["grad"], a["grad"] + b["grad"], rtol=1e-12, atol=1e-18)


# ------------------------------------------------------------------ Adam


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(9)
    p0 = rng.normal(size=(14, 7))
    cfg = O.Config()
    tp = [torch.nn.Parameter(torch.tensor(p0[i:i + 1].copy())) for i in range(14)]
    opt = torch.optim.Adam([{"params": [tp[i]], "lr": cfg.lr[O.PARAM_GROUP_OF_ROW[i]]} for i in range(14)],
                           betas=(cfg.beta1, cfg.beta2), eps=cfg.eps)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for step in range(1, 6):
        g = rng.normal(size=p0.shape) * 10 ** rng.uniform(-6, 0)
        for i in range(14):
            tp[i].grad = torch.tensor(g[i:i + 1].copy())
        opt.step()
        p, m, v = O.adam_step(p, g, m, v, step, cfg)
        np.testing.assert_allclose(p, np.concatenate([t.detach().numpy() for t in tp]), rtol=1e-12, atol=1e-15)


def test_adam_first_step_closed_form():
    g = np.array([[1e-3, -2.0, 0.0]] * 14)
    p1, _, _ = O.adam_step(np.zeros((14, 3)), g, np.zeros((14, 3)), np.zeros((14, 3)), 1)
    lr = np.array([CFG.lr[O.PARAM_GROUP_OF_ROW[i]] for i in range(14)])[:, None]
    np.testing.assert_allclose(p1, -lr * g / (np.abs(g) + CFG.eps), rtol=1e-12)


# ------------------------------------------------------------------ insertion, initialisation, split


def test_insertion_empty_map_and_opaque_wall():
    cam = _axis_cam(100.0, 64)
    pts = np.array([[0.0, 0.0, 2.0], [0.1, -0.1, 3.0], [5.0, 0.0, 1.0], [0, 0, -1.0]])
    mask, pix, inside = O.insertion_mask(pts, cam, np.ones((64, 64)))
    assert mask.tolist() == [True, True, True, True]
    assert inside.tolist() == [True, True, False, False]
    T = np.ones((64, 64))
    T[32, 32] = 0.005          # opacity 0.995 > 0.99 at the first point's pixel
    T[29, 35] = 0.02           # opacity 0.98 at the second point's pixel (35.33, 28.67): still inserted
    mask, pix, _ = O.insertion_mask(pts, cam, T)
    assert pix[1].tolist() == [35, 29]
    assert mask.tolist() == [False, True, True, True]


def test_plain_init_knn_scale():
    E = np.array([[0, 0, 0], [0.03, 0, 0], [0, 0.04, 0], [5, 5, 5.0]])
    X = np.array([[0.0, 0.0, 0.0], [10.0, 10.0, 10.0]])
    img = np.zeros((3, 4, 4))
    img[:, 1, 2] = [0.1, 0.2, 0.3]
    out = O.plain_init(X, np.array([[2, 1], [0, 0]]), img, E)
    np.testing.assert_allclose(out[3:6, 0], math.log(math.sqrt((0 + 0.03 ** 2 + 0.04 ** 2) / 3)), rtol=1e-12)
    assert out[3, 1] == -1.0                      # far away: clamped at -1
    np.testing.assert_allclose(out[11:14, 0], [0.1, 0.2, 0.3])
    assert out[6, 0] == 1 and out[10, 0] == 0


def test_split_children_distribution_and_conservation():
    n = 100_000
    rng = np.random.default_rng(0)
    q = np.array([0.8, 0.2, -0.3, 0.1])
    ls = np.log([0.02, 0.05, 0.1])
    P = _params([[1.0, 2.0, 3.0]] * n, [ls] * n, [q] * n, [0.4] * n, [[0.1, 0.2, 0.3]] * n)
    z = rng.normal(size=(n, 2, 3))
    newP, newm, newv, mask = O.split(P, np.ones_like(P), np.ones_like(P), np.full(n, 1.0), np.full(n, 1000.0), z)
    assert mask.all() and newP.shape[1] == 2 * n
    mu = newP[0:3].T
    np.testing.assert_allclose(mu.mean(0), [1, 2, 3], atol=4 * 0.1 / math.sqrt(2 * n))
    from scipy.spatial.transform import Rotation
    R = Rotation.from_quat(q[[1, 2, 3, 0]]).as_matrix()
    Sig = R @ np.diag(np.exp(2 * ls)) @ R.T
    np.testing.assert_allclose(np.cov(mu.T), Sig, atol=5e-4 * 0.01 + 2e-4 * np.abs(Sig).max())
    np.testing.assert_allclose(newP[3:6], (ls - math.log(1.6))[:, None] * np.ones((1, 2 * n)), rtol=1e-14)
    assert np.all(newP[6:10] == q[:, None]) and np.all(newP[10] == 0.4)
    assert np.all(newP[11:14] == np.array([[0.1], [0.2], [0.3]]))
    assert np.all(newm == 0) and np.all(newv == 0)


def test_split_threshold_and_order():
    P = np.arange(14 * 4, dtype=float).reshape(14, 4)
    P[6:10] = [[1], [0], [0], [0]]
    gsum = np.array([1e-3, 1e-5, 3e-4, 0.0])
    gcnt = np.array([2, 1, 1, 0])             # means 5e-4, 1e-5, 3e-4, never visible
    z = np.zeros((4, 2, 3))
    newP, _, _, mask = O.split(P, P, P, gsum, gcnt, z)
    assert mask.tolist() == [True, False, True, False]
    np.testing.assert_array_equal(newP[0:3, :2], P[0:3, [1, 3]])      # survivors first, in order
    np.testing.assert_array_equal(newP[0:3, 2:], P[0:3, [0, 0, 2, 2]])  # then children, z = 0


def test_dominance_count_single_gaussian_closed_form():
    """One isotropic Gaussian on the axis dominates exactly the pixels where it blends:
    |dx|, |dy| <= r and o exp(-(dx^2 + dy^2) / (2 sigma^2)) >= 1/255, sigma^2 = (f s/z)^2 + 0.3."""
    f, z, s, o = 100.0, 2.0, 0.05, 0.5
    cam = _axis_cam(f)
    p = _params([[0, 0, z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [_logit(o)], [[0.5, 0.5, 0.5]])
    out = O.render(p, cam)
    cnt = O.dominance_counts([out["argmax"]], 1)
    sig2 = (f * s / z) ** 2 + 0.3
    r = 8
    expect = sum(1 for dx in range(-r, r + 1) for dy in range(-r, r + 1)
                 if o * math.exp(-(dx * dx + dy * dy) / (2 * sig2)) >= 1 / 255)
    # blending needs dx^2 + dy^2 <= 2 sigma^2 ln(255 o) = 63.5: the 193 lattice points of that disc
    assert cnt[0] == expect == sum(1 for dx in range(-8, 9) for dy in range(-8, 9) if dx * dx + dy * dy <= 63) == 193


def test_dominance_front_opaque_layer_takes_every_pixel():
    """A front layer with alpha 0.99 at every pixel of the back layer's footprint outweighs it
    (0.99 against at most 0.01 * 0.99); pixels only the back layer covers stay its own."""
    cam = _axis_cam(100.0)
    p = _params([[0, 0, 1.0], [0, 0, 2.0]], [[math.log(2.0)] * 3, [math.log(0.05)] * 3], [[1, 0, 0, 0]] * 2,
                [_logit(0.9999), _logit(0.9)], [[1, 0, 0], [0, 1, 0]])
    out = O.render(p, cam)
    a = out["argmax"]
    assert (a == 0).all()
    cnt = O.dominance_counts([a, a], 2)
    assert cnt[0] == 2 * 64 * 64 and cnt[1] == 0
    assert list(O.dominance_counts([np.full((4, 4), -1)], 3)) == [0, 0, 0]


def test_split_with_clarity_mask_is_union():
    rng = np.random.default_rng(3)
    p = rng.normal(size=(14, 6))
    z = rng.normal(size=(6, 2, 3))
    gs, gc = np.array([3e-4, 0, 0, 1e-4, 0, 0]), np.ones(6)
    dom = np.array([0, 50, 10, 0, 11, 0])
    cfg = O.Config(clarity_sigma=10.0)
    _, _, _, mask = O.split(p, p * 0, p * 0, gs, gc, z, cfg, dominant=dom)
    assert list(mask) == [True, True, False, False, True, False]
    _, _, _, off = O.split(p, p * 0, p * 0, gs, gc, z, O.Config(), dominant=dom)   # sigma 0: gradient rule only
    assert list(off) == [True, False, False, False, False, False]


def test_distance_insertion_matches_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(8)
    means = rng.uniform(-1, 1, size=(3000, 3))
    pts = rng.uniform(-1.2, 1.2, size=(400, 3))
    pts[:5] = means[:5]                                 # exactly on a mean: distance 0, skipped
    cfg = O.Config(insert_tau=0.06)
    mask, d = O.distance_insertion_mask(pts, means, cfg)
    dk, _ = spatial.cKDTree(means).query(pts)
    np.testing.assert_allclose(d, dk, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(mask, dk > 0.06)
    assert not mask[:5].any() and mask.any() and not mask.all()
    m0, d0 = O.distance_insertion_mask(pts, np.zeros((0, 3)), cfg)
    assert m0.all() and np.isinf(d0).all()


def test_init_map_knn_excludes_self():
    X = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.2, 0], [0, 0, 0.3], [5, 5, 5.0]])
    out = O.init_map(X, np.full((5, 3), 0.5))
    d = np.array([0.1, 0.2, 0.3])                      # nearest three of point 0: itself excluded
    np.testing.assert_allclose(out[3, 0], math.log(math.sqrt((d ** 2).mean())), rtol=1e-12)
    assert out[3, 4] == -1.0                           # far from all others: clamped
    single = O.init_map(X[:1], np.zeros((1, 3)))
    np.testing.assert_allclose(single[3:6, 0], math.log(0.01))


def test_screen_grad_norms():
    """Closed form at W = H = 2 (NDC = pixel units); the statistic scales with the image size."""
    g = [{"u": np.array([3.0, 0.0]), "v": np.array([4.0, 1.0])}, {"u": np.array([0.0, 6.0]), "v": np.array([0.0, 8.0])}]
    ok = [np.array([True, True]), np.array([False, True])]
    s, c = O.screen_grad_norms(g, ok, [(2, 2), (2, 2)])
    np.testing.assert_allclose(s, [5.0, 11.0])
    np.testing.assert_allclose(c, [1, 2])
    s2, _ = O.screen_grad_norms(g, ok, [(640, 480), (2, 2)])
    np.testing.assert_allclose(s2, [math.hypot(3 * 320, 4 * 240), 240 + 10])


def test_screen_grad_norm_is_ndc_gradient():
    """The statistic equals the norm of a finite-difference gradient of the loss with respect to
    the Gaussian's projected position in NDC. An isotropic Gaussian on the optical axis has a
    footprint whose shape does not change to first order under a sideways shift of its mean,
    so the shift only moves u (by fx dx / z pixels, i.e. 2 fx dx / (z W) in NDC)."""
    p, cam = frustum_scene(n=1, width=32, height=24, fx=40.0, fy=44.0, cx=16.3, cy=12.4, seed=3)
    z, h = 2.0, 1e-6
    p[0:3, 0] = [0.0, 0.0, z]
    p[3:6, 0] = -1.3
    p[6:10, 0] = [1.0, 0.0, 0.0, 0.0]
    p[10, 0] = 1.0
    tg = random_target(32, 24, seed=4)
    p64 = p.astype(np.float64)
    ref = O.loss_and_grads(p64, [cam], tg, want_2d=True)
    pr = O.project(torch.tensor(p64), cam)
    s, c = O.screen_grad_norms(ref["grad2d"], [pr["valid"].numpy()], [(32, 24)])

    def L(dx, dy):
        q = p64.copy()
        q[0, 0] += dx
        q[1, 0] += dy
        return O.loss_and_grads(q, [cam], tg)["loss"]
    gx = (L(h, 0) - L(-h, 0)) / (2 * h) / (2 * cam.fx / (z * 32))
    gy = (L(0, h) - L(0, -h)) / (2 * h) / (2 * cam.fy / (z * 24))
    assert math.hypot(gx, gy) > 0
    np.testing.assert_allclose(s[0], math.hypot(gx, gy), rtol=1e-5)
    assert c[0] == 1


# ------------------------------------------------------------------ learned initialiser


def _mlp_params(seed):
    rng = np.random.default_rng(seed)
    flat = rng.normal(0, 0.15, size=O.MLP_SIZE)
    W1, b1, W2, b2, W3, b3 = O.mlp_unflatten(torch.tensor(flat))
    W3[11:] = 0
    b3[11:] = 0
    return torch.cat([t.reshape(-1) for t in (W1, b1, W2, b2, W3, b3)]).numpy()


def test_gelu_closed_forms():
    x = torch.tensor([0.0, 1.0, -1.0, 3.0], dtype=torch.float64, requires_grad=True)
    y = O.gelu(x)
    from scipy.stats import norm
    np.testing.assert_allclose(y.detach().numpy(), x.detach().numpy() * norm.cdf(x.detach().numpy()), rtol=1e-14)
    y[0].backward()
    assert x.grad[0].item() == pytest.approx(0.5, abs=1e-15)   # GELU'(0) = 1/2


def test_mlp_forward_matches_explicit_layers():
    flat = _mlp_params(0)
    X = np.random.default_rng(1).normal(size=(5, 80))
    W1, b1, W2, b2, W3, b3 = [t.numpy() for t in O.mlp_unflatten(torch.tensor(flat))]
    from scipy.special import erf
    g = lambda z: 0.5 * z * (1 + erf(z / np.sqrt(2)))  # noqa: E731
    ref = g(g(X @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    np.testing.assert_allclose(O.mlp_forward(flat, X, round_bf16=False), ref, rtol=1e-12, atol=1e-14)


def test_mlp_gradient_finite_differences():
    flat = _mlp_params(2)
    rng = np.random.default_rng(3)
    X, Tg = rng.normal(size=(6, 80)), rng.normal(size=(6, 16))
    L, g = O.mlp_loss_and_grad(flat, X, Tg, round_bf16=False)
    idx = rng.choice(O.MLP_SIZE - 16 * 128 - 16, size=40, replace=False)     # weights of the real rows
    idx = np.concatenate([idx, O.MLP_SIZE - 16 - 2048 + np.arange(0, 11 * 128, 97), [O.MLP_SIZE - 16, O.MLP_SIZE - 6]])
    for i in idx:
        h = 1e-6
        pp, pm = flat.copy(), flat.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.mlp_loss_and_grad(pp, X, Tg, False)[0] - O.mlp_loss_and_grad(pm, X, Tg, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 1e-9, (i, fd, g[i])
    assert np.all(g[-16 + 11:] == 0) and np.all(g[O.MLP_SIZE - 16 - 5 * 128:O.MLP_SIZE - 16] == 0)


def test_mlp_features_layout():
    cam = Camera(20, 10, 10.0, 10.0, 10.0, 5.0)
    img = np.zeros((3, 10, 20))
    img[0] = np.arange(20)[None, :]
    img[1] = np.arange(10)[:, None]
    f = O.mlp_features(np.array([[0.0, 0.0, 2.0], [-2.05, -1.0, 1.0]]), cam, img)
    # point 0 projects to pixel (10, 5): patch x 8..12, y 3..7
    np.testing.assert_allclose(f[0, 0:75:3].reshape(5, 5), np.tile(np.arange(8, 13), (5, 1)))
    np.testing.assert_allclose(f[0, 1:75:3].reshape(5, 5), np.tile(np.arange(3, 8)[:, None], (1, 5)))
    # point 1 projects to (-10.5 + 10 -> pixel 0 after clamping), y 5 - 10 = -5 -> 0: borders clamp
    assert np.all(f[1, 0:75:3] >= 0) and f[1, 0] == 0 and f[1, 1] == 0
    np.testing.assert_allclose(f[0, 75:80], [2.0, 0.0, 0.0, 2.0, 0.0])


# ------------------------------------------------------------------ SSIM term (Eq. 10 L_SSIM)


def test_ssim_identity_and_constant_closed_form():
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.uniform(size=(3, 24, 20)))
    np.testing.assert_allclose(O.ssim_map(x, x).numpy(), 1.0, rtol=0, atol=1e-12)
    # constant images c1, c2 away from the border (window fully inside): variances vanish
    a, b = torch.full((3, 30, 30), 0.3, dtype=torch.float64), torch.full((3, 30, 30), 0.7, dtype=torch.float64)
    m = O.ssim_map(a, b).numpy()[:, 5:-5, 5:-5]
    C1 = 0.01 ** 2
    np.testing.assert_allclose(m, (2 * 0.3 * 0.7 + C1) / (0.3 ** 2 + 0.7 ** 2 + C1), rtol=1e-12)


def test_ssim_matches_scipy_gaussian_filter():
    """The windowed statistics are scipy's Gaussian filter (sigma 1.5, radius 5, zero padding)."""
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    x, y = rng.uniform(size=(3, 26, 31)), rng.uniform(size=(3, 26, 31))

    def blur(z):
        return np.stack([nd.gaussian_filter(c, 1.5, truncate=5 / 1.5, mode="constant", cval=0.0) for c in z])
    mx, my = blur(x), blur(y)
    sxx, syy, sxy = blur(x * x) - mx * mx, blur(y * y) - my * my, blur(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ref = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    np.testing.assert_allclose(O.ssim_map(torch.tensor(x), torch.tensor(y)).numpy(), ref, rtol=1e-10, atol=1e-12)


def test_color_loss_weights():
    rng = np.random.default_rng(6)
    x, y = torch.tensor(rng.uniform(size=(3, 16, 16))), torch.tensor(rng.uniform(size=(3, 16, 16)))
    l1 = float((x - y).abs().mean())
    s = float(O.ssim_map(x, y).mean())
    assert float(O.color_loss(x, y)) == pytest.approx(l1, rel=1e-15)
    assert float(O.color_loss(x, y, O.Config(lambda_photo=0.2))) == pytest.approx(0.8 * l1 + 0.2 * (1 - s), rel=1e-14)


@pytest.mark.parametrize("seed,n", [(3, 2), (4, 4)])
def test_gradient_finite_differences_with_ssim(seed, n):
    """The whole-image SSIM path of the oracle's gradient against central differences."""
    p, cam = frustum_scene(n=n, width=16, height=16, fx=16.0, fy=16.0, cx=8.0, cy=8.0, seed=seed,
                           logscale_mean=-1.5)
    p = p.astype(np.float64)
    tg = np.random.default_rng(seed).uniform(size=(1, 3, 16, 16))
    cfg = O.Config(lambda_photo=0.2)
    res = O.loss_and_grads(p, [cam], tg, cfg)
    g = res["grad"]
    base = O.decision_signature(p, [cam])
    checked = 0
    for i in range(14):
        for j in range(n):
            h = 1e-6 * max(1.0, abs(p[i, j]))
            pp, pm = p.copy(), p.copy()
            pp[i, j] += h
            pm[i, j] -= h
            if O.decision_signature(pp, [cam]) != base or O.decision_signature(pm, [cam]) != base:
                continue
            fd = (O.loss_value(pp, [cam], tg, cfg) - O.loss_value(pm, [cam], tg, cfg)) / (2 * h)
            assert abs(fd - g[i, j]) <= 1e-6 * abs(g[i, j]) + 100 * np.finfo(float).eps * abs(res["loss"]) / h, \
                (i, j, fd, g[i, j])
            checked += 1
    assert checked >= 0.8 * 14 * n
    # the SSIM term changes the gradient (it is not the L1 gradient)
    g1 = O.loss_and_grads(p, [cam], tg)["grad"]
    assert np.abs(g - g1).max() > 1e-3 * np.abs(g1).max()


def test_pixel_box_matches_brute_force():
    """The membership box of a pixel-exact test |px - u| <= r, |py - v| <= r, clipped to the
    image, against a scan of every pixel (means inside, outside and on integer coordinates)."""
    rng = np.random.default_rng(11)
    W, H = 23, 17
    cases = [(u, v, r) for u, v, r in zip(rng.uniform(-6, W + 6, 300), rng.uniform(-6, H + 6, 300),
                                          rng.integers(0, 7, 300))]
    cases += [(4.0, 3.0, 2), (0.0, 0.0, 0), (W - 1.0, H - 1.0, 1), (-2.0, 5.5, 2), (5.5, H + 2.0, 3)]
    px, py = np.arange(W), np.arange(H)
    for u, v, r in cases:
        x0, x1, y0, y1 = O.pixel_box(np.float64(u), np.float64(v), np.float64(r), W, H)
        xs = px[np.abs(px - u) <= r]
        ys = py[np.abs(py - v) <= r]
        if xs.size == 0 or ys.size == 0:
            assert x0 > x1 or y0 > y1, (u, v, r, x0, x1, y0, y1)
        else:
            assert (x0, x1, y0, y1) == (xs[0], xs[-1], ys[0], ys[-1]), (u, v, r)


def test_bf16_round_is_round_to_nearest_even():
    """bfloat16 rounding against an integer restatement on the float32 bit patterns (keep the top
    16 bits, add half an ulp plus the kept LSB for ties to even), and hand-checked ties."""
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        [0.0, -0.0, 1.0, -3.5, 65504.0, 1e-30]]).astype(np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)
    got = O.bf16_round(x).numpy()
    assert np.array_equal(got, rounded.astype(np.float64))
    # ties: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 (even: 1); 1 + 3 * 2^-8 between 1 + 2^-7 and
    # 1 + 2^-6 (even: 1 + 2^-6)
    ties = O.bf16_round(np.float32([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8])).numpy()
    assert ties.tolist() == [1.0, 1 + 2.0 ** -6]


def test_ssim_window_closed_form():
    """The 11 x 11 window: w[i, j] = g_i g_j with g_k proportional to exp(-k^2 / (2 1.5^2)), sum 1.
    Checked by its ratios (no normalisation needed) and its sum."""
    w = O.ssim_window().numpy()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w, w.T, rtol=0, atol=0) and np.allclose(w, w[::-1, ::-1], rtol=0, atol=0)
    assert math.isclose(w[5, 5] / w[0, 0], math.exp((25 + 25) / (2 * 1.5 ** 2)), rel_tol=1e-12)
    assert math.isclose(w[5, 5] / w[5, 8], math.exp(9 / (2 * 1.5 ** 2)), rel_tol=1e-12)
    g1 = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    assert np.allclose(w, np.outer(g1, g1) / g1.sum() ** 2, rtol=1e-14, atol=0)

"""FP64 CPU oracle of the MonoGS++ mapping step: splatting forward, loss, gradients, Adam,
insertion and splitting.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module. It shares no
code, header, table or helper with the CUDA library, and never imports it.

Everything is evaluated from its plain definition in float64 (torch CPU ops),
with no tiling, fusion or reordering: every pixel is composited over all
Gaussians that pass the membership test, in depth order.

Passages followed
-----------------
* Eq. 1 (Section 3.1, Scene Representation): the Gaussian G(x) and its
  covariance Sigma = R S S^T R^T, parameterised by mean mu, scale s = diag(S),
  quaternion r and opacity alpha, colour c.
* Eq. 2 (Section 3.1): the 2D covariance Sigma2D = J W Sigma W^T J^T with J
  the Jacobian of the projection and W the viewing transform.
* Eq. 3 (Section 3.1): front-to-back alpha blending
  C(p) = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j).
* Eq. 8 (Section 3.2, Clarity-Enhancing Densification): the blend weight
  w_m = alpha_m prod_{n<m}(1 - alpha_n) and the per-pixel argmax id.
* Eq. 10-11 (Section 3.2, Map Optimization): L_photo = L1, the planar term
  L_reg = |max(0.01, min(s))| and L = lambda_color L_color + lambda_reg L_reg;
  L_color = (1 - lambda_photo) L1 + lambda_photo L_SSIM with L_SSIM = 1 - SSIM
  (the lineage's 11 x 11 Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2,
  zero padding). lambda_photo = 0 (pure L1) unless set; the paper's is 0.2.
* Eq. 6-7 (Section 3.2, Map Initialization / Dynamic Insertion): the new points
  are back-projected patch centres; which of them become Gaussians follows the
  opacity reading below.

Readings of points the paper leaves open (each is a field of ``Config``)
-----------------------------------------------------------------------
* colour: k = 3 direct RGB, unclamped; s = exp(log-scale); opacity
  o = sigmoid(logit); the quaternion is normalised inside the forward pass.
* projection: cull t_z <= near (0.2); J evaluated at x/z, y/z clamped to
  +-1.3 x the half-FOV tangent (a clamped coordinate carries no gradient);
  low-pass dilation Sigma2D += 0.3 I; largest eigenvalue with the discriminant
  floored at 0.1; integer radius r = ceil(3 sqrt(lambda_max)).
* membership is pixel-exact: pixel (px, py) sees Gaussian i iff
  |px - u_i| <= r_i and |py - v_i| <= r_i (tiles only accelerate this).
* alpha = min(0.99, o exp(power)); skip alpha < 1/255; stop before a Gaussian
  whose blend would leave T (1 - alpha) < 1e-4; background black.
* order: ascending depth, ties by ascending Gaussian id.
* loss: L1 mean over 3HW per view, summed over views; planar term mean over N.
* Adam: beta = (0.9, 0.999), eps = 1e-15, one learning rate per parameter group.

The gradient of the loss is obtained by reverse-mode differentiation of the
forward definition above (torch.autograd, a library primitive); it is pinned by
central finite differences in the tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np
import torch

DT = torch.float64
LN2 = math.log(2.0)

# rows of the [14, N] parameter array
ROW_MEAN = slice(0, 3)
ROW_LOGSCALE = slice(3, 6)
ROW_QUAT = slice(6, 10)
ROW_OPACITY = 10
ROW_RGB = slice(11, 14)
PARAM_GROUP_OF_ROW = (0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3, 4, 4, 4)


@dataclasses.dataclass
class Config:
    near: float = 0.2
    fov_clamp: float = 1.3
    dilation: float = 0.3
    lambda_floor: float = 0.1
    radius_sigma: float = 3.0
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    lambda_color: float = 1.0
    lambda_reg: float = 1.0
    lambda_photo: float = 0.0       # Eq. 10 weight of L_SSIM = 1 - SSIM (0.2 in the paper; 0 = pure L1)
    reg_floor: float = 0.01
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    lr: tuple = (1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3)   # means, log-scales, quats, opacity, colours
    split_thresh: float = 2e-4
    split_factor: float = 1.6
    clarity_sigma: float = 0.0      # Eq. 9 threshold sigma in pixels (0 = clarity split off)
    insert_opacity: float = 0.99
    insert_tau: float = 0.0         # Eq. 7 distance threshold tau in metres (0 = opacity rule)


def _t(x) -> torch.Tensor:
    return torch.as_tensor(np.asarray(x, dtype=np.float64) if not torch.is_tensor(x) else x, dtype=DT)


# ------------------------------------------------------------------ Eq. 1: covariance


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the normalised quaternion q = (w, x, y, z); q is [N, 4]."""
    qn = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = qn.unbind(1)
    r0 = torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], dim=1)
    r1 = torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], dim=1)
    r2 = torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=1)
    return torch.stack([r0, r1, r2], dim=1)


def cov3d(logscale: torch.Tensor, quat: torch.Tensor) -> torch.Tensor:
    """Eq. 1: Sigma = R S S^T R^T with S = diag(exp(logscale)); logscale [N, 3], quat [N, 4]."""
    R = quat_to_rotmat(quat)
    M = R * torch.exp(logscale)[:, None, :]          # R S (scales the columns)
    return M @ M.transpose(1, 2)


# ------------------------------------------------------------------ Eq. 2: projection


def project(params, cam, cfg: Config = Config()) -> dict:
    """Eq. 2 and the projection readings: per-Gaussian screen quantities for one camera.

    ``params`` is a [14, N] float64 tensor (may require grad); ``cam`` has width, height,
    fx, fy, cx, cy, R (world->camera), t. Returns a dict of [N] tensors:
    u, v (screen mean), a, b, c (conic: inverse of the dilated 2D covariance, with
    power = -(a dx^2 + c dy^2)/2 - b dx dy), o (opacity), rgb [N, 3], depth, r (integer
    radius, float64 without gradient), valid (bool), cov2d [N, 2, 2], tclamp (bool [N, 2],
    whether x/z, y/z were clamped), lam (largest eigenvalue).
    """
    p = params
    Rw = _t(cam.R).reshape(3, 3)
    tw = _t(cam.t).reshape(3)
    mu = p[ROW_MEAN].T
    t = mu @ Rw.T + tw
    tx, ty, tz = t.unbind(1)
    lim_x = cfg.fov_clamp * (0.5 * cam.width / cam.fx)
    lim_y = cfg.fov_clamp * (0.5 * cam.height / cam.fy)
    xr, yr = tx / tz, ty / tz
    xh = torch.clamp(xr, -lim_x, lim_x)
    yh = torch.clamp(yr, -lim_y, lim_y)
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([cam.fx / tz, zero, -cam.fx * xh / tz], dim=1),
                     torch.stack([zero, cam.fy / tz, -cam.fy * yh / tz], dim=1)], dim=1)   # [N, 2, 3]
    Sig = cov3d(p[ROW_LOGSCALE].T, p[ROW_QUAT].T)
    T = J @ Rw                                              # J W
    cov = T @ Sig @ T.transpose(1, 2)
    cov = cov + cfg.dilation * torch.eye(2, dtype=DT)
    A, B, C = cov[:, 0, 0], cov[:, 0, 1], cov[:, 1, 1]
    det = A * C - B * B
    mid = 0.5 * (A + C)
    lam = mid + torch.sqrt(torch.clamp(mid * mid - det, min=cfg.lambda_floor))
    r = torch.ceil(cfg.radius_sigma * torch.sqrt(lam.detach()))
    u = cam.fx * tx / tz + cam.cx
    v = cam.fy * ty / tz + cam.cy
    valid = (tz.detach() > cfg.near) & (det.detach() > 0)
    with torch.no_grad():
        x0, x1, y0, y1 = pixel_box(u, v, r, cam.width, cam.height)
        valid = valid & (x0 <= x1) & (y0 <= y1)
    safe_det = torch.where(valid, det, torch.ones_like(det))
    return dict(u=u, v=v, a=C / safe_det, b=-B / safe_det, c=A / safe_det,
                o=torch.sigmoid(p[ROW_OPACITY]), rgb=p[ROW_RGB].T, depth=tz, r=r, valid=valid,
                cov2d=cov, lam=lam, tclamp=torch.stack([(xr.detach().abs() > lim_x), (yr.detach().abs() > lim_y)], 1))


def pixel_box(u, v, r, width, height):
    """Inclusive pixel bounds of the membership box |px-u| <= r, |py-v| <= r, clipped to the image.

    Works on float64 tensors or numpy arrays; returns float arrays of integer values; an
    empty box has x0 > x1 or y0 > y1.
    """
    lib = torch if torch.is_tensor(u) else np
    # r is integer-valued, so ceil(u - r) = ceil(u) - r; this form is exact in any precision
    x0 = lib.clip(lib.ceil(u) - r, 0, width)
    x1 = lib.clip(lib.floor(u) + r, -1, width - 1)
    y0 = lib.clip(lib.ceil(v) - r, 0, height)
    y1 = lib.clip(lib.floor(v) + r, -1, height - 1)
    return x0, x1, y0, y1


# ------------------------------------------------------------------ binning and sort (definition)


def bin_pairs(u, v, r, depth, valid, width, height, tile, view=0, n_gauss=None, n_views=1):
    """Sorted (key, value) pairs of the tile binning, by definition.

    Gaussian i (of view ``view``) is listed in tile (tx, ty) iff its clipped pixel box
    intersects that tile's pixels. Key = (view * n_tiles + ty * n_tx + tx) << 32 | bits(depth
    as float32); value = view * n_gauss + i. Pairs are sorted lexicographically by
    (key, value). Inputs are numpy arrays of one view (u, v, depth float32 or float64,
    r integer-valued, valid bool). Returns (keys uint64, values uint32).
    """
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    r = np.asarray(r, np.float64)
    n = u.shape[0] if n_gauss is None else n_gauss
    ntx = (width + tile - 1) // tile
    nty = (height + tile - 1) // tile
    x0, x1, y0, y1 = pixel_box(u, v, r, width, height)
    ok = np.asarray(valid, bool) & (x0 <= x1) & (y0 <= y1)
    ids = np.nonzero(ok)[0]
    tx0 = (x0[ids] // tile).astype(np.int64)
    tx1 = (x1[ids] // tile).astype(np.int64)
    ty0 = (y0[ids] // tile).astype(np.int64)
    ty1 = (y1[ids] // tile).astype(np.int64)
    cnt = (tx1 - tx0 + 1) * (ty1 - ty0 + 1)
    rep = np.repeat(np.arange(ids.shape[0]), cnt)
    first = np.repeat(np.cumsum(cnt) - cnt, cnt)
    j = np.arange(rep.shape[0]) - first
    w = (tx1 - tx0 + 1)[rep]
    tx = tx0[rep] + j % w
    ty = ty0[rep] + j // w
    bins = view * (ntx * nty) + ty * ntx + tx
    dbits = np.asarray(depth, np.float32)[ids][rep].view(np.uint32).astype(np.uint64)
    keys = (bins.astype(np.uint64) << np.uint64(32)) | dbits
    vals = (view * n + ids[rep]).astype(np.uint64)
    order = np.lexsort((vals, keys))
    return keys[order], vals[order].astype(np.uint32)


def tiles_touched(u, v, r, valid, width, height, tile):
    """Number of tiles each Gaussian's clipped pixel box touches (0 if culled)."""
    u = np.asarray(u, np.float64)
    x0, x1, y0, y1 = pixel_box(u, np.asarray(v, np.float64), np.asarray(r, np.float64), width, height)
    ok = np.asarray(valid, bool) & (x0 <= x1) & (y0 <= y1)
    n = ((x1 // tile) - (x0 // tile) + 1) * ((y1 // tile) - (y0 // tile) + 1)
    return np.where(ok, n, 0).astype(np.int64)


# ------------------------------------------------------------------ Eq. 3: compositing


_PROJ_GRAD_KEYS = ("u", "v", "a", "b", "c", "o", "rgb")


def _depth_order(pr) -> torch.Tensor:
    """Gaussian indices by ascending depth, ties by ascending id (stable sort)."""
    return torch.sort(pr["depth"].detach(), stable=True).indices


def composite(px, py, pr, cfg: Config, order=None, flags: bool = False):
    """Eq. 3 at the pixels (px, py) over all Gaussians of ``pr`` (output of ``project``).

    Returns dict: rgb [P, 3], T (final transmittance) [P], last (id of the last blended
    Gaussian, -1 if none), argmax (id of the largest blend weight, Eq. 8; first on ties),
    argmax_gap (relative gap between the two largest weights), n_contrib [P]; with ``flags`` also ``near`` [P] bool (a discrete decision lies within
    FP32 rounding of its threshold), ``near_grad`` [P] (near or an alpha near the 0.99
    clamp), ``pair_near_grad`` (bool [P, K]: which Gaussian's decision is the near one) and
    ``members`` (bool [P, K]) with ``cols`` (ids of the K columns).
    """
    if order is None:
        order = _depth_order(pr)
    pxt = _t(px).reshape(-1, 1)
    pyt = _t(py).reshape(-1, 1)
    valid = pr["valid"][order]
    r = pr["r"][order]
    with torch.no_grad():
        u0 = pr["u"].detach()[order]
        v0 = pr["v"].detach()[order]
        # Gaussians that are no member of any of these pixels contribute nothing; drop them.
        keep_cols = valid & ((pxt - u0).abs() <= r).any(0) & ((pyt - v0).abs() <= r).any(0)
    cols = order[keep_cols]
    u = pr["u"][cols]
    v = pr["v"][cols]
    a, b, c = pr["a"][cols], pr["b"][cols], pr["c"][cols]
    o = pr["o"][cols]
    rgb = pr["rgb"][cols]
    rr = pr["r"][cols]
    P, K = pxt.shape[0], cols.shape[0]
    dx = pxt - u[None, :]
    dy = pyt - v[None, :]
    member = (dx.detach().abs() <= rr) & (dy.detach().abs() <= rr)
    power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
    oG = o * torch.exp(power)
    alpha = torch.minimum(oG, torch.full_like(oG, cfg.alpha_max))
    contrib = member & (alpha.detach() >= cfg.alpha_min)
    a_eff = torch.where(contrib, alpha, torch.zeros_like(alpha))
    T_after = torch.cumprod(1.0 - a_eff, dim=1)
    T_before = torch.cat([torch.ones(P, 1, dtype=DT), T_after[:, :-1]], dim=1)
    idx = torch.arange(K)
    stop = contrib & (T_after.detach() < cfg.T_min)
    first_stop = torch.where(stop, idx[None, :], torch.full_like(stop, K, dtype=torch.long)).min(dim=1).values \
        if K > 0 else torch.zeros(P, dtype=torch.long)
    include = contrib & (idx[None, :] < first_stop[:, None])
    w = torch.where(include, alpha * T_before, torch.zeros_like(alpha))
    out_rgb = w @ rgb
    if K > 0:
        T_ext = torch.cat([T_before, T_after[:, -1:]], dim=1)
        T_fin = T_ext[torch.arange(P), first_stop]
    else:
        T_fin = torch.ones(P, dtype=DT)
    with torch.no_grad():
        n_contrib = include.sum(1)
        pos = torch.where(include, idx[None, :], torch.full_like(idx[None, :], -1)).max(dim=1).values \
            if K > 0 else torch.full((P,), -1)
        last = torch.where(pos >= 0, cols[pos.clamp(min=0)] if K > 0 else pos, torch.full_like(pos, -1))
        wd = w.detach()
        if K > 0:
            am = wd.argmax(dim=1)   # first maximum in depth order
            argmax = torch.where(n_contrib > 0, cols[am], torch.full_like(am, -1))
            top = wd.topk(min(2, K), dim=1).values
            second = top[:, 1] if K > 1 else torch.zeros(P, dtype=DT)
            argmax_gap = torch.where(top[:, 0] > 0, (top[:, 0] - second) / top[:, 0].clamp(min=1e-300),
                                     torch.ones(P, dtype=DT))
        else:
            argmax = torch.full((P,), -1)
            argmax_gap = torch.ones(P, dtype=DT)
    res = dict(rgb=out_rgb, T=T_fin, last=last, argmax=argmax, n_contrib=n_contrib, argmax_gap=argmax_gap)
    if flags:
        res.update(_decision_flags(dx.detach(), dy.detach(), rr, oG.detach(), member, contrib, include,
                                   T_after.detach(), first_stop, pr["depth"].detach()[cols], cfg,
                                   pr["lam"].detach()[cols], pr["depth"].detach()[cols]))
        res["members"] = member
        res["cols"] = cols
    return res


def _decision_flags(dx, dy, r, oG, member, contrib, include, T_after, first_stop, depth, cfg, lam, tz):
    """(pixel, Gaussian) pairs whose discrete decision lies within FP32 rounding of its threshold.

    A pair is flagged when: its membership edge lies within 1e-3 px, or the radius
    3 sqrt(lambda) lies within 1e-5 (relative) of an integer, where the Gaussian's alpha
    would pass 1/255; its alpha lies within 1e-5 (relative) of 1/255; its transmittance step
    T(1 - alpha) lies within 1e-4 (relative) of 1e-4 (up to the stopping Gaussian); its depth
    lies within 2e-6 (relative) of another blended Gaussian's at that pixel; or its depth lies
    within 1e-6 of the near plane. ``near`` [P] marks pixels with a flagged pair. The
    gradient flags ``pair_near_grad`` [P, K] add alpha within 1e-5 (relative) of the 0.99 clamp.
    """
    K = dx.shape[1]
    mx = torch.maximum(dx.abs(), dy.abs())
    # a membership change only matters where the Gaussian would blend (alpha >= 1/255)
    visible = torch.minimum(oG, torch.full_like(oG, cfg.alpha_max)) >= cfg.alpha_min * (1 - 1e-5)
    edge = (mx - r).abs() <= 1e-3
    s3 = cfg.radius_sigma * torch.sqrt(lam)
    r_amb = (s3 - torch.round(s3)).abs() <= 1e-5 * s3
    pair = visible & (edge | (r_amb[None, :] & (mx > r - 1 - 1e-3) & (mx <= r + 1 + 1e-3)))
    pair = pair | (member & ((oG / cfg.alpha_min - 1).abs() <= 1e-5))
    idx = torch.arange(K)
    upto = idx[None, :] <= first_stop[:, None]
    pair = pair | (contrib & upto & ((T_after / cfg.T_min - 1).abs() <= 1e-4))
    # depth ties among blended Gaussians (columns are in depth order)
    if K > 1:
        close = (depth[1:] - depth[:-1]).abs() <= 2e-6 * depth[1:]
        if bool(close.any()):
            tie = contrib[:, 1:] & contrib[:, :-1] & close[None, :]
            pair[:, 1:] |= tie
            pair[:, :-1] |= tie
    nearz = (tz - cfg.near).abs() <= 1e-6
    if bool(nearz.any()):
        pair = pair | (member & nearz[None, :])
    pair_g = pair | (member & ((oG / cfg.alpha_max - 1).abs() <= 1e-5))
    return dict(near=pair.any(1), near_grad=pair_g.any(1), pair_near_grad=pair_g)


def render(params, cam, cfg: Config = Config(), chunk: int = 1024, pixels=None, flags: bool = False):
    """Eq. 3 for a whole image (or the listed pixels): returns numpy arrays.

    ``pixels`` is an optional int array [P, 2] of (px, py). Without it the full image is
    rendered and rgb is [3, H, W], T/last/argmax/n_contrib are [H, W].
    """
    p = _t(params)
    with torch.no_grad():
        pr = project(p, cam, cfg)
        order = _depth_order(pr)
        if pixels is None:
            py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
            pix = np.stack([px.ravel(), py.ravel()], 1)
        else:
            pix = np.asarray(pixels).reshape(-1, 2)
        outs = []
        for s in range(0, pix.shape[0], chunk):
            outs.append(composite(pix[s:s + chunk, 0], pix[s:s + chunk, 1], pr, cfg, order, flags=flags))
    keys = ["rgb", "T", "last", "argmax", "n_contrib", "argmax_gap"] + (["near", "near_grad"] if flags else [])
    res = {k: torch.cat([o[k] for o in outs]).numpy() for k in keys}
    if flags:
        gsel = np.zeros(p.shape[1], bool)
        for o in outs:
            bad = o["near_grad"]
            if bool(bad.any()):
                gsel[o["cols"][o["pair_near_grad"].any(0)].numpy()] = True
        res["gauss_near"] = gsel
    if pixels is None:
        H, W = cam.height, cam.width
        res["rgb"] = res["rgb"].T.reshape(3, H, W)
        for k in keys[1:]:
            res[k] = res[k].reshape(H, W)
    return res


# ------------------------------------------------------------------ Eq. 10-11: loss


SSIM_SIZE, SSIM_SIGMA, SSIM_C1, SSIM_C2 = 11, 1.5, 0.01 ** 2, 0.03 ** 2


def ssim_window() -> torch.Tensor:
    """The 11 x 11 Gaussian window (sigma 1.5) of the SSIM of the 3DGS lineage, normalised to
    sum 1: the outer product of the normalised 1D Gaussian with itself."""
    k = torch.arange(SSIM_SIZE, dtype=DT) - SSIM_SIZE // 2
    g = torch.exp(-k * k / (2.0 * SSIM_SIGMA ** 2))
    g = g / g.sum()
    return torch.outer(g, g)


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Per-pixel, per-channel SSIM of images x, y [3, H, W] (Wang et al. 2004): local means,
    variances and covariance under the window, zero padding outside the image.
    SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2))."""
    w = ssim_window()[None, None].expand(3, 1, SSIM_SIZE, SSIM_SIZE)
    pad = SSIM_SIZE // 2

    def blur(z):
        return torch.nn.functional.conv2d(z[None], w, padding=pad, groups=3)[0]
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def color_loss(img: torch.Tensor, target: torch.Tensor, cfg: Config = Config()) -> torch.Tensor:
    """Eq. 10 L_color of one view: (1 - lambda_photo) mean|C - I| + lambda_photo (1 - mean SSIM),
    means over the 3HW channel-pixels."""
    l1 = (img - target).abs().mean()
    if cfg.lambda_photo == 0:
        return l1
    return (1.0 - cfg.lambda_photo) * l1 + cfg.lambda_photo * (1.0 - ssim_map(img, target).mean())


def planar_reg(params, cfg: Config = Config()) -> torch.Tensor:
    """Eq. 10 planar term, averaged over the N Gaussians: mean_i max(0.01, min_k s_ik)."""
    s = torch.exp(params[ROW_LOGSCALE])
    return torch.clamp(s.min(dim=0).values, min=cfg.reg_floor).mean()


def loss_and_grads(params, cams: Sequence, targets, cfg: Config = Config(), chunk: int = 1024,
                   pixels=None, want_2d: bool = False, flags: bool = False):
    """Eq. 11 loss over a window of views and its gradient w.r.t. the [14, N] parameters.

    L = sum_views lambda_color * mean_{3HW} |C - I| + lambda_reg * L_reg.
    ``targets`` is [V, 3, H, W]. With ``pixels`` (a list of [P, 2] arrays, one per view)
    only those pixels' L1 terms are evaluated (a bounded sample; the mean still divides
    by 3HW). Returns dict(loss, grad [14, N] numpy, images, T, last; with ``want_2d`` the
    gradients w.r.t. each view's screen quantities: list of dicts u, v, a, b, c, o, rgb).
    """
    p = _t(params).clone().requires_grad_(True)
    tg = np.asarray(targets, np.float64)
    total = torch.zeros((), dtype=DT)
    out_images, out_T, out_last, g2d, near_g = [], [], [], [], np.zeros(p.shape[1], bool)
    prs = []
    for vi, cam in enumerate(cams):
        pr = project(p, cam, cfg)
        prs.append(pr)
        order = _depth_order(pr)
        leaves = {k: pr[k].detach().clone().requires_grad_(True) for k in _PROJ_GRAD_KEYS}
        prl = dict(pr)
        prl.update(leaves)
        H, W = cam.height, cam.width
        if pixels is None:
            py, px = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
            pix = np.stack([px.ravel(), py.ravel()], 1)
        else:
            pix = np.asarray(pixels[vi]).reshape(-1, 2)
        img = np.zeros((pix.shape[0], 3))
        Tv = np.zeros(pix.shape[0])
        lastv = np.zeros(pix.shape[0], np.int64)
        scale = cfg.lambda_color / (3.0 * H * W)
        up = None
        if cfg.lambda_photo != 0:
            # L_SSIM couples neighbouring pixels: take dL/dC of the whole image first, then
            # propagate it through the compositing chunk by chunk (chain rule)
            assert pixels is None, "the SSIM term needs the whole image"
            with torch.no_grad():
                full = torch.zeros(pix.shape[0], 3, dtype=DT)
                for s in range(0, pix.shape[0], chunk):
                    cp = pix[s:s + chunk]
                    full[s:s + chunk] = composite(cp[:, 0], cp[:, 1], prl, cfg, order)["rgb"]
            C_img = full.T.reshape(3, H, W).clone().requires_grad_(True)
            lc = cfg.lambda_color * color_loss(C_img, torch.as_tensor(tg[vi], dtype=DT), cfg)
            lc.backward()
            total = total + lc.detach()
            up = C_img.grad.reshape(3, -1).T
        for s in range(0, pix.shape[0], chunk):
            cp = pix[s:s + chunk]
            res = composite(cp[:, 0], cp[:, 1], prl, cfg, order, flags=flags)
            if up is None:
                I = torch.as_tensor(tg[vi][:, cp[:, 1], cp[:, 0]].T, dtype=DT)
                l1 = scale * (res["rgb"] - I).abs().sum()
                l1.backward()
                total = total + l1.detach()
            else:
                (res["rgb"] * up[s:s + chunk]).sum().backward()
            img[s:s + chunk] = res["rgb"].detach().numpy()
            Tv[s:s + chunk] = res["T"].detach().numpy()
            lastv[s:s + chunk] = res["last"].numpy()
            if flags and bool(res["near_grad"].any()):
                near_g[res["cols"][res["pair_near_grad"].any(0)].numpy()] = True
        grads_v = {k: (leaves[k].grad if leaves[k].grad is not None else torch.zeros_like(leaves[k]))
                   for k in _PROJ_GRAD_KEYS}
        g2d.append({k: g.numpy().copy() for k, g in grads_v.items()})
        torch.autograd.backward([pr[k] for k in _PROJ_GRAD_KEYS], [grads_v[k] for k in _PROJ_GRAD_KEYS],
                                retain_graph=False)
        if pixels is None:
            out_images.append(img.T.reshape(3, H, W))
            out_T.append(Tv.reshape(H, W))
            out_last.append(lastv.reshape(H, W))
        else:
            out_images.append(img)
            out_T.append(Tv)
            out_last.append(lastv)
    reg = cfg.lambda_reg * planar_reg(p, cfg)
    reg.backward()
    total = total + reg.detach()
    res = dict(loss=float(total), grad=p.grad.numpy().copy(), images=out_images, T=out_T, last=out_last,
               reg=float(reg.detach()))
    if want_2d:
        res["grad2d"] = g2d
    if flags:
        res["gauss_near"] = near_g
    return res


def loss_value(params, cams, targets, cfg: Config = Config(), chunk: int = 1024) -> float:
    """Eq. 11 loss only (no gradient), for finite differences."""
    p = _t(params)
    tg = np.asarray(targets, np.float64)
    total = 0.0
    with torch.no_grad():
        for vi, cam in enumerate(cams):
            img = render(p, cam, cfg, chunk=chunk)["rgb"]
            total += cfg.lambda_color * float(color_loss(_t(img), _t(tg[vi]), cfg))
        total += cfg.lambda_reg * float(planar_reg(p, cfg))
    return float(total)


def decision_signature(params, cams, cfg: Config = Config()) -> bytes:
    """Every discrete decision of the forward pass, as bytes (for the finite-difference exclusion rule).

    Covers validity, radius, FOV clamps, and per pixel the member / blended / alpha-clamped
    pattern and the stopping Gaussian.
    """
    p = _t(params)
    parts = []
    with torch.no_grad():
        for cam in cams:
            pr = project(p, cam, cfg)
            parts += [pr["valid"].numpy().tobytes(), pr["r"].numpy().tobytes(), pr["tclamp"].numpy().tobytes()]
            order = _depth_order(pr)
            parts.append(order.numpy().tobytes())
            py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
            pxt = _t(px.ravel()).reshape(-1, 1)
            pyt = _t(py.ravel()).reshape(-1, 1)
            u, v, r = pr["u"][order], pr["v"][order], pr["r"][order]
            dx, dy = pxt - u, pyt - v
            member = pr["valid"][order] & (dx.abs() <= r) & (dy.abs() <= r)
            power = -0.5 * (pr["a"][order] * dx * dx + pr["c"][order] * dy * dy) - pr["b"][order] * dx * dy
            oG = pr["o"][order] * torch.exp(power)
            alpha = torch.clamp(oG, max=cfg.alpha_max)
            contrib = member & (alpha >= cfg.alpha_min)
            a_eff = torch.where(contrib, alpha, torch.zeros_like(alpha))
            T_after = torch.cumprod(1.0 - a_eff, dim=1)
            stop = contrib & (T_after < cfg.T_min)
            parts += [member.numpy().tobytes(), contrib.numpy().tobytes(), (oG > cfg.alpha_max).numpy().tobytes(),
                      stop.numpy().tobytes()]
    return b"".join(parts)


# ------------------------------------------------------------------ Adam


def adam_step(params, grad, m, v, step: int, cfg: Config = Config()):
    """One Adam step (bias-corrected) with the learning rate of each row's parameter group.

    ``step`` is the 1-based step count after this update. Returns (params, m, v) as new
    float64 numpy arrays.
    """
    p = np.asarray(params, np.float64)
    g = np.asarray(grad, np.float64)
    m = cfg.beta1 * np.asarray(m, np.float64) + (1 - cfg.beta1) * g
    v = cfg.beta2 * np.asarray(v, np.float64) + (1 - cfg.beta2) * g * g
    mh = m / (1 - cfg.beta1 ** step)
    vh = v / (1 - cfg.beta2 ** step)
    lr = np.array([cfg.lr[PARAM_GROUP_OF_ROW[i]] for i in range(p.shape[0])])[:, None]
    return p - lr * mh / (np.sqrt(vh) + cfg.eps), m, v


# ------------------------------------------------------------------ insertion (Eq. 6-7 reading)


def insertion_mask(points, cam, T_final, cfg: Config = Config()):
    """Which new points become Gaussians: all except those that project, in front of the
    camera, to a pixel whose rendered accumulated opacity 1 - T exceeds ``insert_opacity``.

    The pixel is the nearest one, (floor(u + 1/2), floor(v + 1/2)). Returns (mask bool [n],
    pixel [n, 2] int, inside bool [n]).
    """
    X = np.asarray(points, np.float64)
    t = X @ np.asarray(cam.R, np.float64).T + np.asarray(cam.t, np.float64)
    front = t[:, 2] > cfg.near
    z = np.where(front, t[:, 2], 1.0)
    u = cam.fx * t[:, 0] / z + cam.cx
    v = cam.fy * t[:, 1] / z + cam.cy
    pxl = np.floor(u + 0.5)
    pyl = np.floor(v + 0.5)
    inside = front & (pxl >= 0) & (pxl < cam.width) & (pyl >= 0) & (pyl < cam.height)
    pi = np.where(inside, pxl, 0).astype(np.int64)
    pj = np.where(inside, pyl, 0).astype(np.int64)
    opac = 1.0 - np.asarray(T_final, np.float64)[pj, pi]
    skip = inside & (opac > cfg.insert_opacity)
    return ~skip, np.stack([pi, pj], 1), inside


def distance_insertion_mask(points, means, cfg: Config = Config()):
    """Eq. 7 as the text states it (the equation's d < tau reads the other way): a new point q
    becomes a Gaussian iff d(q, P) = min over the existing Gaussian means p of |q - p|_2 exceeds
    ``insert_tau``; into an empty map every point is inserted. Returns (mask bool [n], d [n]);
    d is +inf for an empty map."""
    X = np.asarray(points, np.float64).reshape(-1, 3)
    E = np.asarray(means, np.float64).reshape(-1, 3)
    if E.shape[0] == 0:
        return np.ones(X.shape[0], bool), np.full(X.shape[0], np.inf)
    d = np.full(X.shape[0], np.inf)
    for s0 in range(0, E.shape[0], 4096):
        blk = E[s0:s0 + 4096]
        d = np.minimum(d, np.sqrt(((X[:, None, :] - blk[None, :, :]) ** 2).sum(-1)).min(1))
    return d > cfg.insert_tau, d


def plain_init(points, pixels, image, existing_means):
    """Initial parameters [14, n] of inserted Gaussians (the plain initialisation reading).

    log-scale = ln of the RMS distance to the 3 nearest existing means (fewer if fewer exist;
    0.01 m if none), clamped to [-7, -1], isotropic; quaternion (1, 0, 0, 0); opacity logit 0;
    colour = the keyframe image at the point's pixel.
    """
    X = np.asarray(points, np.float64)
    E = np.asarray(existing_means, np.float64).reshape(-1, 3)
    n = X.shape[0]
    if E.shape[0] == 0:
        rms = np.full(n, 0.01)
    else:
        d2 = ((X[:, None, :] - E[None, :, :]) ** 2).sum(-1)
        k = min(3, E.shape[0])
        near = np.sort(d2, axis=1)[:, :k]
        rms = np.sqrt(near.mean(1))
    ls = np.clip(np.log(np.maximum(rms, 1e-30)), -7.0, -1.0)
    out = np.zeros((14, n))
    out[0:3] = X.T
    out[3:6] = ls[None, :]
    out[6] = 1.0
    img = np.asarray(image, np.float64)
    pix = np.asarray(pixels)
    out[11:14] = img[:, pix[:, 1], pix[:, 0]]
    return out


def init_map(points, rgb):
    """Eq. 6: one Gaussian per back-projected point with the plain initialisation, the
    neighbours of each point being the other points. Returns params [14, n]."""
    X = np.asarray(points, np.float64)
    n = X.shape[0]
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    k = min(3, n - 1)
    if k > 0:
        rms = np.sqrt(np.sort(d2, axis=1)[:, :k].mean(1))
    else:
        rms = np.full(n, 0.01)
    out = np.zeros((14, n))
    out[0:3] = X.T
    out[3:6] = np.clip(np.log(np.maximum(rms, 1e-30)), -7.0, -1.0)[None, :]
    out[6] = 1.0
    out[11:14] = np.asarray(rgb, np.float64).T
    return out


def screen_grad_norms(grad2d_views, valid_views, sizes):
    """Per-Gaussian sum and count of the norm of the position gradient in normalised device
    coordinates, |(dL/du * W/2, dL/dv * H/2)|, over the views in which it is valid (the statistic
    the densification reading thresholds). ``sizes`` holds each view's (W, H): the pixel
    coordinate u spans W pixels over the NDC interval [-1, 1], so du/dx_ndc = W/2."""
    s = np.zeros(len(valid_views[0]))
    c = np.zeros(len(valid_views[0]))
    for g, ok, (W, H) in zip(grad2d_views, valid_views, sizes):
        nrm = np.sqrt((np.asarray(g["u"]) * (W / 2.0)) ** 2 + (np.asarray(g["v"]) * (H / 2.0)) ** 2)
        s += np.where(ok, nrm, 0.0)
        c += np.asarray(ok, float)
    return s, c


# ------------------------------------------------------------------ densification split (gradient reading)


def dominance_counts(argmax_maps, n):
    """Eq. 8-9 (clarity-enhancing densification), read as: O_i(n) is the set of pixels of view i
    that Gaussian n renders, O_i(m) the set of pixels whose largest blend weight w_m (Eq. 8)
    belongs to n, so |O_i(n) & O_i(m)| is the number of pixels Gaussian n dominates. Returns
    that number per Gaussian, summed over the given per-view argmax maps (-1 = no Gaussian)."""
    c = np.zeros(n, np.int64)
    for a in argmax_maps:
        a = np.asarray(a).ravel()
        a = a[a >= 0]
        c += np.bincount(a, minlength=n)[:n]
    return c


def split(params, m, v, grad_sum, grad_cnt, normals, cfg: Config = Config(), dominant=None):
    """Split every Gaussian whose mean NDC position-gradient norm exceeds ``split_thresh``, and,
    when ``dominant`` (per-Gaussian dominated-pixel counts) is given and ``clarity_sigma`` > 0,
    every Gaussian that dominates more than ``clarity_sigma`` pixels (the split mask M of Eq. 9).

    mean = grad_sum / grad_cnt over the iterations in which it was visible (0 if never).
    Each split parent is replaced by two children with means mu + R S z_k (z_k the given
    standard normal samples ``normals`` [N, 2, 3], i.e. samples of N(mu, Sigma)), log-scales
    reduced by ln(split_factor), quaternion, opacity and colour copied, Adam moments zero.
    Output order: surviving Gaussians in their order, then the children (parent order,
    child 0 then child 1). Returns (params, m, v, split mask).
    """
    P = np.asarray(params, np.float64)
    cnt = np.asarray(grad_cnt, np.float64)
    mean_g = np.where(cnt > 0, np.asarray(grad_sum, np.float64) / np.maximum(cnt, 1), 0.0)
    mask = mean_g > cfg.split_thresh
    if dominant is not None and cfg.clarity_sigma > 0:
        mask = mask | (np.asarray(dominant) > cfg.clarity_sigma)
    ids = np.nonzero(mask)[0]
    with torch.no_grad():
        R = quat_to_rotmat(_t(P[ROW_QUAT, ids].T)).numpy()
    s = np.exp(P[ROW_LOGSCALE, ids].T)
    z = np.asarray(normals, np.float64)[ids]
    kids = []
    for k in range(2):
        c = P[:, ids].copy()
        c[ROW_MEAN] = (P[ROW_MEAN, ids].T + np.einsum("nij,nj->ni", R, s * z[:, k])).T
        c[ROW_LOGSCALE] = P[ROW_LOGSCALE, ids] - math.log(cfg.split_factor)
        kids.append(c)
    child = np.stack(kids, axis=2).reshape(14, -1)     # parent-major, child 0 then 1
    keep = ~mask
    newP = np.concatenate([P[:, keep], child], axis=1)
    zeros = np.zeros((14, child.shape[1]))
    newm = np.concatenate([np.asarray(m, np.float64)[:, keep], zeros], axis=1)
    newv = np.concatenate([np.asarray(v, np.float64)[:, keep], zeros], axis=1)
    return newP, newm, newv, mask


# ------------------------------------------------------------------ learned initialiser (MLP reading)

MLP_IN, MLP_HID, MLP_OUT, MLP_OUT_PAD = 80, 128, 11, 16
# flat parameter layout: W1 [128][80], b1 [128], W2 [128][128], b2 [128], W3 [16][128], b3 [16]
MLP_SHAPES = ((MLP_HID, MLP_IN), (MLP_HID,), (MLP_HID, MLP_HID), (MLP_HID,), (MLP_OUT_PAD, MLP_HID), (MLP_OUT_PAD,))
MLP_SIZE = sum(int(np.prod(s)) for s in MLP_SHAPES)


def bf16_round(x):
    """Round float values to bfloat16 (round to nearest even), returned as float64."""
    t = torch.as_tensor(np.asarray(x, np.float32))
    return t.to(torch.bfloat16).to(torch.float64)


def mlp_unflatten(flat):
    flat = torch.as_tensor(flat)
    out, o = [], 0
    for s in MLP_SHAPES:
        k = int(np.prod(s))
        out.append(flat[o:o + k].reshape(s))
        o += k
    return out


def gelu(x):
    """GELU, erf form: x Phi(x)."""
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def mlp_features(points, cam, image):
    """Input of the learned initialiser for each new point: the 5x5 RGB patch around the
    point's nearest pixel (borders clamped; row-major, RGB interleaved), the depth, and the
    point in camera coordinates, then one zero: [n, 80]."""
    X = np.asarray(points, np.float64)
    t = X @ np.asarray(cam.R, np.float64).T + np.asarray(cam.t, np.float64)
    z = np.where(t[:, 2] > 1e-6, t[:, 2], 1e-6)
    u = cam.fx * t[:, 0] / z + cam.cx
    v = cam.fy * t[:, 1] / z + cam.cy
    px = np.clip(np.floor(u + 0.5), 0, cam.width - 1).astype(np.int64)
    py = np.clip(np.floor(v + 0.5), 0, cam.height - 1).astype(np.int64)
    img = np.asarray(image, np.float64)
    f = np.zeros((X.shape[0], MLP_IN))
    k = 0
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            xx = np.clip(px + dx, 0, cam.width - 1)
            yy = np.clip(py + dy, 0, cam.height - 1)
            f[:, k:k + 3] = img[:, yy, xx].T
            k += 3
    f[:, 75] = t[:, 2]
    f[:, 76:79] = t
    return f


def mlp_forward(flat, feats, round_bf16: bool = True):
    """Forward pass: Y = W3 g(W2 g(W1 x + b1) + b2) + b3 with g = GELU. With ``round_bf16`` the
    inputs, weights and hidden activations are rounded to bfloat16 (the tensor-core operands)
    and everything else is float64. Returns Y [n, 16] (columns 11..15 are padding)."""
    W1, b1, W2, b2, W3, b3 = [w.to(DT) for w in mlp_unflatten(torch.as_tensor(np.asarray(flat, np.float64)))]
    r = bf16_round if round_bf16 else (lambda a: torch.as_tensor(np.asarray(a, np.float64)))
    x = r(feats)
    h1 = gelu(x @ r(W1.numpy()).T + b1)
    h1 = r(h1.numpy()) if round_bf16 else h1
    h2 = gelu(h1 @ r(W2.numpy()).T + b2)
    h2 = r(h2.numpy()) if round_bf16 else h2
    return (h2 @ r(W3.numpy()).T + b3).numpy()


def mlp_loss_and_grad(flat, feats, targets, round_bf16: bool = True):
    """Mean-squared error over the 11 outputs, (1 / (n 11)) sum (Y - T)^2, and its gradient
    w.r.t. the flat float32 master parameters. The bfloat16 roundings of the forward are
    treated as the identity in the derivative (the weights' gradient is taken at the rounded
    values). Rows 11..15 of W3 and b3 get zero gradient."""
    p = torch.as_tensor(np.asarray(flat, np.float64)).clone()
    W1, b1, W2, b2, W3, b3 = mlp_unflatten(p)
    r = (lambda a: bf16_round(a.detach().numpy())) if round_bf16 else (lambda a: a.detach())
    leaves = [t.clone().requires_grad_(True) for t in (W1, b1, W2, b2, W3, b3)]
    W1l, b1l, W2l, b2l, W3l, b3l = leaves

    def ste(a):  # rounded value, identity derivative
        return a + (r(a) - a.detach()) if round_bf16 else a

    x = r(torch.as_tensor(np.asarray(feats, np.float64)))
    h1 = ste(gelu(x @ ste(W1l).T + b1l))
    h2 = ste(gelu(h1 @ ste(W2l).T + b2l))
    y = h2 @ ste(W3l).T + b3l
    T = torch.as_tensor(np.asarray(targets, np.float64))
    n = y.shape[0]
    loss = ((y[:, :MLP_OUT] - T[:, :MLP_OUT]) ** 2).sum() / (n * MLP_OUT)
    loss.backward()
    g = torch.cat([l.grad.reshape(-1) for l in leaves]).numpy()
    return float(loss), g


def mlp_targets(params) -> np.ndarray:
    """Training targets of the learned initialiser (its reading: the parameters of converged
    Gaussians) for params [14, n]: rows [n, 16] = log-scale (3), the quaternion divided by its
    norm and negated when w < 0 (q and -q are the same rotation), opacity logit, colour (3), and
    five zeros. A zero quaternion stays zero."""
    p = np.asarray(params, np.float64)
    n = p.shape[1]
    out = np.zeros((n, MLP_OUT_PAD))
    q = p[ROW_QUAT].T
    nrm = np.sqrt((q * q).sum(1))
    sign = np.where(q[:, 0] < 0, -1.0, 1.0)
    qn = np.where(nrm[:, None] > 0, q * (sign / np.where(nrm > 0, nrm, 1.0))[:, None], 0.0)
    out[:, 0:3] = p[ROW_LOGSCALE].T
    out[:, 3:7] = qn
    out[:, 7] = p[ROW_OPACITY]
    out[:, 8:11] = p[ROW_RGB].T
    return out


# ------------------------------------------------------------------ evaluation


def psnr(img, ref) -> float:
    """Peak signal-to-noise ratio of images with values in [0, 1]: 10 log10(1 / MSE), the MSE
    taken over every channel-pixel and floored at 1e-12."""
    a = np.asarray(img, np.float64)
    b = np.asarray(ref, np.float64)
    mse = max(float(np.mean((a - b) ** 2)), 1e-12)
    return 10.0 * math.log10(1.0 / mse)

"""Seeded synthetic scenes shaped like the paper's mapping workloads.

Replica and TUM-RGBD (Section 4.1) are not available, so these generators stand
in for them with the same image sizes and Gaussian counts:

* ``frustum_scene``: Gaussians uniform in a camera frustum, random colours; the
  small single-view case (2k Gaussians, 160x120).
* ``make_room`` + ``room_gaussians``: a 6 m x 3 m x 6 m room of six textured
  planes and twenty textured boxes, Gaussians sampled area-uniformly on the
  surfaces and coloured by the texture (Replica-shaped 1200x680 view,
  TUM-shaped 640x480 windows and streams).
* ``Room.raycast``: the analytic ground-truth image of the room for a camera,
  used as the photometric target.
* ``vo_points``: sparse 3D points standing in for the patch centres of
  Eq. 6 (true surface point + isotropic Gaussian noise).

Parameter layout (shared interface, float32, planar SoA of shape [14, N]):
rows 0-2 mean xyz, 3-5 log-scale, 6-9 quaternion (w, x, y, z, unnormalised),
10 opacity logit, 11-13 RGB colour.

Camera convention: world-to-camera rotation ``R`` (3x3) and translation ``t``;
camera frame x right, y down, z forward; pinhole fx, fy, cx, cy; pixel (px, py)
samples the image plane at (px, py).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_PARAM_ROWS = 14


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray = dataclasses.field(default_factory=lambda: np.eye(3))
    t: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))

    def center(self) -> np.ndarray:
        return -np.asarray(self.R, dtype=np.float64).T @ np.asarray(self.t, dtype=np.float64)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _pack(mean, logscale, quat, opacity_logit, rgb) -> np.ndarray:
    n = mean.shape[0]
    p = np.empty((N_PARAM_ROWS, n), dtype=np.float32)
    p[0:3] = mean.T
    p[3:6] = logscale.T
    p[6:10] = quat.T
    p[10] = opacity_logit
    p[11:14] = rgb.T
    return p


def frustum_scene(n: int = 2000, width: int = 160, height: int = 120, fx: float = 150.0,
                  fy: float = 150.0, cx: float = 80.0, cy: float = 60.0, seed: int = 0,
                  depth_range=(1.0, 5.0), logscale_mean: float = -3.0, logscale_std: float = 0.5,
                  opacity_mean: float = 0.0):
    """Gaussians uniform in the frustum of an identity-pose camera.

    Depth z ~ U[depth_range]; the image-plane position is uniform over the image
    at that depth; log-scales ~ N(logscale_mean, logscale_std); quaternions are
    normalised N(0, I4); opacity logits ~ N(opacity_mean, 1); colours ~ U[0, 1].
    Returns (params [14, n] float32, Camera).
    """
    rng = _rng(seed)
    z = rng.uniform(depth_range[0], depth_range[1], size=n)
    px = rng.uniform(0.0, width, size=n)
    py = rng.uniform(0.0, height, size=n)
    mean = np.stack([(px - cx) * z / fx, (py - cy) * z / fy, z], axis=1)
    logscale = rng.normal(logscale_mean, logscale_std, size=(n, 3))
    quat = _random_quats(rng, n)
    opac = rng.normal(opacity_mean, 1.0, size=n)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    cam = Camera(width, height, fx, fy, cx, cy)
    return _pack(mean, logscale, quat, opac, rgb), cam


def random_target(width: int, height: int, seed: int = 1, n_views: int = 1) -> np.ndarray:
    """Seeded uniform target image(s), float32 [n_views, 3, H, W]."""
    return _rng(seed).uniform(0.0, 1.0, size=(n_views, 3, height, width)).astype(np.float32)


# --------------------------------------------------------------------------- room


@dataclasses.dataclass
class Room:
    """Textured rectangles: origin o, unit edge axes e1, e2, extents L1, L2.

    Texture of rectangle k at local coordinates (a, b):
    clip(base + amp1 sin(f1 a + p1) sin(f2 b + p2) + amp2 checker(a, b, period), 0, 1).
    """
    origin: np.ndarray     # [K, 3]
    e1: np.ndarray         # [K, 3]
    e2: np.ndarray         # [K, 3]
    ext: np.ndarray        # [K, 2]
    base: np.ndarray       # [K, 3]
    wave: np.ndarray       # [K, 6]: amp(3 channels scale), f1, f2, p1 ... packed below
    checker: np.ndarray    # [K, 2]: amplitude, period
    half_extent: np.ndarray  # room half sizes (x, y, z)

    @property
    def n_rects(self) -> int:
        return self.origin.shape[0]

    def areas(self) -> np.ndarray:
        return self.ext[:, 0] * self.ext[:, 1]

    def texture(self, k: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        w = self.wave[k]
        s = np.sin(w[:, 1] * a + w[:, 3]) * np.sin(w[:, 2] * b + w[:, 4])
        per = self.checker[k, 1]
        chk = ((np.floor(a / per) + np.floor(b / per)) % 2.0) * 2.0 - 1.0
        col = self.base[k] + (w[:, 0] * s)[:, None] * np.array([1.0, 0.8, 0.6]) \
            + (self.checker[k, 0] * chk)[:, None] * np.array([0.7, 1.0, 0.9]) \
            + (w[:, 5] * np.sin(2.3 * w[:, 1] * b + w[:, 3]))[:, None] * np.array([0.5, 0.3, 1.0])
        return np.clip(col, 0.0, 1.0)

    def raycast(self, cam: Camera, chunk: int = 16384) -> np.ndarray:
        """Ground-truth image [3, H, W] float32: colour of the nearest rectangle hit.

        Pixel (px, py) casts the ray through image-plane point ((px-cx)/fx, (py-cy)/fy, 1).
        Rays that hit nothing (impossible from inside the room) stay black.
        """
        W, H = cam.width, cam.height
        R = np.asarray(cam.R, dtype=np.float64)
        c = cam.center()
        py, px = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
        d_cam = np.stack([(px.ravel() - cam.cx) / cam.fx, (py.ravel() - cam.cy) / cam.fy,
                          np.ones(H * W)], axis=1)
        d_world = d_cam @ R  # R^T d for each row
        out = np.zeros((H * W, 3))
        for s in range(0, H * W, chunk):
            out[s:s + chunk] = self._shade(c, d_world[s:s + chunk])
        # a C-contiguous array (the transpose alone is a strided view of the [H * W, 3] rows)
        return np.ascontiguousarray(out.T.reshape(3, H, W), dtype=np.float32)

    def raycast_torch(self, cam: Camera, device="cuda", chunk: int = 65536):
        """The same ray-cast as ``raycast`` evaluated with float32 torch ops on ``device``
        (for long synthetic sequences); returns a [3, H, W] float32 tensor there."""
        import torch
        f = dict(dtype=torch.float32, device=device)
        W, H = cam.width, cam.height
        R = torch.tensor(np.asarray(cam.R, np.float64), **f)
        c = torch.tensor(cam.center(), **f)
        py, px = torch.meshgrid(torch.arange(H, **f), torch.arange(W, **f), indexing="ij")
        d_cam = torch.stack([(px.reshape(-1) - cam.cx) / cam.fx, (py.reshape(-1) - cam.cy) / cam.fy,
                             torch.ones(H * W, **f)], 1)
        d_world = d_cam @ R
        o = torch.tensor(self.origin, **f)
        e1 = torch.tensor(self.e1, **f)
        e2 = torch.tensor(self.e2, **f)
        ext = torch.tensor(self.ext, **f)
        n = torch.cross(e1, e2, dim=1)
        num = ((o - c[None, :]) * n).sum(1)
        base = torch.tensor(self.base, **f)
        wave = torch.tensor(self.wave, **f)
        chk = torch.tensor(self.checker, **f)
        out = torch.zeros(H * W, 3, **f)
        for s0 in range(0, H * W, chunk):
            d = d_world[s0:s0 + chunk]
            denom = d @ n.T
            t = num[None, :] / denom
            p_rel = c[None, None, :] + t[:, :, None] * d[:, None, :] - o[None, :, :]
            a = (p_rel * e1[None]).sum(-1)
            b = (p_rel * e2[None]).sum(-1)
            ok = (t > 1e-6) & (a >= 0) & (a <= ext[None, :, 0]) & (b >= 0) & (b <= ext[None, :, 1]) & torch.isfinite(t)
            t_ok = torch.where(ok, t, torch.full_like(t, float("inf")))
            k = torch.argmin(t_ok, dim=1)
            rows = torch.arange(d.shape[0], device=device)
            hitm = torch.isfinite(t_ok[rows, k])
            aa, bb = a[rows, k], b[rows, k]
            w = wave[k]
            sn = torch.sin(w[:, 1] * aa + w[:, 3]) * torch.sin(w[:, 2] * bb + w[:, 4])
            per = chk[k, 1]
            ck = torch.remainder(torch.floor(aa / per) + torch.floor(bb / per), 2.0) * 2.0 - 1.0
            col = base[k] + (w[:, 0] * sn)[:, None] * torch.tensor([1.0, 0.8, 0.6], **f) \
                + (chk[k, 0] * ck)[:, None] * torch.tensor([0.7, 1.0, 0.9], **f) \
                + (w[:, 5] * torch.sin(2.3 * w[:, 1] * bb + w[:, 3]))[:, None] * torch.tensor([0.5, 0.3, 1.0], **f)
            out[s0:s0 + chunk] = torch.where(hitm[:, None], torch.clamp(col, 0.0, 1.0), torch.zeros_like(col))
        return out.T.reshape(3, H, W).contiguous()

    def hit(self, c: np.ndarray, d: np.ndarray):
        """Nearest hit of rays c + t d (t > 0): returns t [R], rect id [R] (-1 on miss), a, b."""
        n = np.cross(self.e1, self.e2)                       # [K, 3]
        denom = d @ n.T                                      # [R, K]
        num = np.einsum("kj,kj->k", self.origin - c[None, :], n)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = num[None, :] / denom
            p_rel = c[None, None, :] + t[:, :, None] * d[:, None, :] - self.origin[None, :, :]
            a = np.einsum("rkj,kj->rk", p_rel, self.e1)
            b = np.einsum("rkj,kj->rk", p_rel, self.e2)
        ok = (t > 1e-6) & (a >= 0) & (a <= self.ext[None, :, 0]) & (b >= 0) & (b <= self.ext[None, :, 1]) \
            & np.isfinite(t)
        t_ok = np.where(ok, t, np.inf)
        k = np.argmin(t_ok, axis=1)
        rows = np.arange(d.shape[0])
        tb = t_ok[rows, k]
        miss = ~np.isfinite(tb)
        k = np.where(miss, -1, k)
        return tb, k, a[rows, np.maximum(k, 0)], b[rows, np.maximum(k, 0)]

    def _shade(self, c, d):
        t, k, a, b = self.hit(c, d)
        col = np.zeros((d.shape[0], 3))
        m = k >= 0
        col[m] = self.texture(k[m], a[m], b[m])
        return col


def _rect(o, e1, e2, l1, l2):
    return np.asarray(o, float), np.asarray(e1, float), np.asarray(e2, float), float(l1), float(l2)


def make_room(seed: int = 0, half=(3.0, 1.5, 3.0), n_boxes: int = 20) -> Room:
    """Six textured walls of an axis-aligned room plus ``n_boxes`` textured boxes on the floor.

    World frame: y points down, the floor is y = +half_y, the ceiling y = -half_y.
    Boxes have edges ~ U[0.2, 0.8] m, a random yaw, and stand on the floor; their five
    visible faces (sides and top) are rectangles.
    """
    rng = _rng(10_000 + seed)
    hx, hy, hz = half
    rects = [
        _rect([-hx, hy, -hz], [1, 0, 0], [0, 0, 1], 2 * hx, 2 * hz),    # floor
        _rect([-hx, -hy, -hz], [1, 0, 0], [0, 0, 1], 2 * hx, 2 * hz),   # ceiling
        _rect([-hx, -hy, -hz], [0, 1, 0], [0, 0, 1], 2 * hy, 2 * hz),   # wall x = -hx
        _rect([hx, -hy, -hz], [0, 1, 0], [0, 0, 1], 2 * hy, 2 * hz),    # wall x = +hx
        _rect([-hx, -hy, -hz], [1, 0, 0], [0, 1, 0], 2 * hx, 2 * hy),   # wall z = -hz
        _rect([-hx, -hy, hz], [1, 0, 0], [0, 1, 0], 2 * hx, 2 * hy),    # wall z = +hz
    ]
    for _ in range(n_boxes):
        sx, sy, sz = rng.uniform(0.2, 0.8, size=3)
        yaw = rng.uniform(0.0, 0.5 * math.pi)
        cxz = rng.uniform(-(hx - 0.5), hx - 0.5, size=2)
        ex = np.array([math.cos(yaw), 0.0, math.sin(yaw)])
        ez = np.array([-math.sin(yaw), 0.0, math.cos(yaw)])
        ey = np.array([0.0, 1.0, 0.0])
        base = np.array([cxz[0], hy, cxz[1]]) - 0.5 * sx * ex - 0.5 * sz * ez  # floor corner
        top = base - sy * ey
        rects += [
            _rect(top, ex, ez, sx, sz),                    # top face
            _rect(top, ex, ey, sx, sy),                    # side -z
            _rect(top + sz * ez, ex, ey, sx, sy),          # side +z
            _rect(top, ez, ey, sz, sy),                    # side -x
            _rect(top + sx * ex, ez, ey, sz, sy),          # side +x
        ]
    K = len(rects)
    origin = np.stack([r[0] for r in rects])
    e1 = np.stack([r[1] for r in rects])
    e2 = np.stack([r[2] for r in rects])
    ext = np.array([[r[3], r[4]] for r in rects])
    base_col = rng.uniform(0.15, 0.85, size=(K, 3))
    wave = np.stack([rng.uniform(0.05, 0.25, K), rng.uniform(2.0, 9.0, K), rng.uniform(2.0, 9.0, K),
                     rng.uniform(0, 2 * math.pi, K), rng.uniform(0, 2 * math.pi, K),
                     rng.uniform(0.0, 0.12, K)], axis=1)
    checker = np.stack([rng.uniform(0.0, 0.15, K), rng.uniform(0.15, 0.8, K)], axis=1)
    return Room(origin, e1, e2, ext, base_col, wave, checker, np.array(half, float))


def room_gaussians(room: Room, n: int, seed: int = 0, logscale_mean: float = -4.0,
                   logscale_std: float = 0.5, opacity_mean: float = 1.0, opacity_std: float = 1.0,
                   box_fraction=None):
    """``n`` Gaussians sampled area-uniformly on the room's rectangles, coloured by the texture.

    With ``box_fraction`` that share of the Gaussians goes to the boxes' faces and the rest to
    the six walls, area-uniformly within each group (a map denser on the objects than on the
    walls). Log-scales ~ N(logscale_mean, logscale_std); opacity logits ~ N(opacity_mean,
    opacity_std); quaternions normalised N(0, I4). Returns params [14, n] float32.
    """
    rng = _rng(20_000 + seed)
    areas = room.areas()
    w = areas / areas.sum()
    if box_fraction is not None:
        wall = np.arange(room.n_rects) < 6
        w = areas.copy()
        w[wall] *= (1.0 - box_fraction) / areas[wall].sum()
        w[~wall] *= box_fraction / areas[~wall].sum()
        w = w / w.sum()
    k = rng.choice(room.n_rects, size=n, p=w)
    a = rng.uniform(0.0, 1.0, size=n) * room.ext[k, 0]
    b = rng.uniform(0.0, 1.0, size=n) * room.ext[k, 1]
    mean = room.origin[k] + a[:, None] * room.e1[k] + b[:, None] * room.e2[k]
    rgb = room.texture(k, a, b)
    logscale = rng.normal(logscale_mean, logscale_std, size=(n, 3))
    quat = _random_quats(rng, n)
    opac = rng.normal(opacity_mean, opacity_std, size=n)
    return _pack(mean, logscale, quat, opac, rgb)


def look_at(center, target, width, height, fx, fy, cx=None, cy=None) -> Camera:
    """Camera at ``center`` looking at ``target`` with world +y as image-down."""
    c = np.asarray(center, float)
    z = np.asarray(target, float) - c
    z /= np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ c
    return Camera(width, height, fx, fy, width / 2.0 if cx is None else cx,
                  height / 2.0 if cy is None else cy, R, t)


def room_camera_single(width: int = 1200, height: int = 680, fx: float = 600.0, fy: float = 600.0) -> Camera:
    """The Replica-shaped keyframe: inside the room, looking across the boxes to the far wall."""
    return look_at([0.4, -0.3, -2.3], [-0.2, 0.6, 1.5], width, height, fx, fy)


def _catmull_rom(p: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Uniform Catmull-Rom spline through control points p [K, 3] at parameters s in [0, K-3]."""
    i = np.clip(np.floor(s).astype(int), 0, p.shape[0] - 4)
    u = (s - i)[:, None]
    p0, p1, p2, p3 = p[i], p[i + 1], p[i + 2], p[i + 3]
    return 0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u ** 2
                  + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3)


def room_trajectory(n_frames: int, seed: int = 0, width: int = 640, height: int = 480,
                    fx: float = 525.0, fy: float = 525.0, n_waypoints: int = 8,
                    half=(3.0, 1.5, 3.0)):
    """Smooth seeded camera path inside the room (Catmull-Rom through random waypoints).

    Camera centres stay above every box (y in [-0.9, 0.3]) and 0.4 m inside the walls; the
    look-at point follows its own spline so the view direction turns smoothly.
    """
    rng = _rng(30_000 + seed)
    hx, _, hz = half
    cpts = np.stack([rng.uniform(-hx + 0.4, hx - 0.4, n_waypoints + 2),
                     rng.uniform(-0.9, 0.3, n_waypoints + 2),
                     rng.uniform(-hz + 0.4, hz - 0.4, n_waypoints + 2)], axis=1)
    tpts = np.stack([rng.uniform(-hx, hx, n_waypoints + 2),
                     rng.uniform(-0.5, 1.5, n_waypoints + 2),
                     rng.uniform(-hz, hz, n_waypoints + 2)], axis=1)
    s = np.linspace(0.0, n_waypoints - 1 - 1e-9, n_frames)
    centers = _catmull_rom(cpts, s)
    targets = _catmull_rom(tpts, s)
    cams = []
    for c, tg in zip(centers, targets):
        if np.linalg.norm(tg - c) < 0.5:
            tg = c + np.array([0.0, 0.3, 1.0])
        cams.append(look_at(c, tg, width, height, fx, fy))
    return cams


def vo_points(room: Room, cam: Camera, n: int = 96, seed: int = 0, noise: float = 0.01):
    """Sparse VO-style points of one keyframe: ray-cast ``n`` random pixels, add N(0, noise^2) per axis.

    Returns (points [n, 3] float32 world coordinates, pixels [n, 2] int32).
    """
    rng = _rng(40_000 + seed)
    px = rng.integers(0, cam.width, size=n)
    py = rng.integers(0, cam.height, size=n)
    d_cam = np.stack([(px - cam.cx) / cam.fx, (py - cam.cy) / cam.fy, np.ones(n)], axis=1)
    d_world = d_cam @ np.asarray(cam.R, float)
    c = cam.center()
    t, k, _, _ = room.hit(c, d_world)
    t = np.where(np.isfinite(t), t, 1.0)
    pts = c[None, :] + t[:, None] * d_world + rng.normal(0.0, noise, size=(n, 3))
    return pts.astype(np.float32), np.stack([px, py], axis=1).astype(np.int32)


def stream_sequence(seed: int, n_frames: int, width: int = 640, height: int = 480, fx: float = 525.0,
                    n_points: int = 96, noise: float = 0.01, device="cuda"):
    """A mapping-stream input: the room of ``seed``, ``n_frames`` keyframes on its smooth
    trajectory, each keyframe's ray-cast image and its ``n_points`` VO-style points.

    Returns (cameras, targets [F, 3, H, W] float32 on ``device``, [points [n, 3] float32 on
    ``device``] per keyframe). The point draw of keyframe j is seeded by 1000 * seed + j.
    """
    import torch
    room = make_room(seed)
    cams = room_trajectory(n_frames, seed, width, height, fx, fx)
    targets = torch.stack([room.raycast_torch(c, device) for c in cams])
    pts = [torch.as_tensor(vo_points(room, c, n_points, 1000 * seed + j, noise)[0], device=device)
           for j, c in enumerate(cams)]
    return cams, targets, pts

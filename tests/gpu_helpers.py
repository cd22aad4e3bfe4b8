"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
from synth import Camera

# Tolerances of the FP32 CUDA path against the FP64 oracle:
IMG_ATOL = 1e-4          # max abs pixel error
GRAD_RTOL = 1e-3         # per-parameter relative gradient error ...
# ... relative to max(|g*|, GRAD_FLOOR * max |g*| of the parameter group). A gradient is a sum of
# per-pixel terms that partly cancel; in FP32 its absolute error is ~eps32 times the sum of the
# terms' magnitudes. Measured on the parity scenes (every compositing layout and the
# deterministic mode): |g - g*| <= 2.3e-6 of the group's largest gradient; the smallest floor
# under which every gradient passes is 5.4e-5 of it for single views and 2.0e-4 for the
# three-view window (a Gaussian's views add terms that cancel); GRAD_FLOOR keeps a margin of
# 2.5 over the window. The deep-list scene (pixels blending several hundred Gaussians) sums
# correspondingly more terms: it needs 4.3e-4, and GRAD_FLOOR_DEEP keeps a margin of 2.3.
GRAD_FLOOR = 5e-4
GRAD_FLOOR_DEEP = 1e-3
# One view's screen-space gradients (du, dv, conic, opacity, colour per Gaussian) sum fewer,
# more strongly cancelling pixel terms; their measured need varies with the rounding order of
# the compositing arithmetic (up to 2.4e-4 of the group's largest gradient over the kernel
# versions measured), so SCREEN_GRAD_FLOOR keeps a margin of 4 over that.
SCREEN_GRAD_FLOOR = 1e-3
GROUPS = {"mean": slice(0, 3), "logscale": slice(3, 6), "quat": slice(6, 10), "opacity": slice(10, 11),
          "rgb": slice(11, 14)}


def new_map(n_cap, views=1, W=160, H=120, **kw):
    from paper_2504_02437_gb300.api import GaussianMap
    return GaussianMap(capacity=max(n_cap, 1), max_views=views, max_width=W, max_height=H, **kw)


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")


def grad_errors(g_gpu, g_ref, exclude=None, floor_frac=None):
    """Per-group max relative error |g - g*| / max(|g*|, floor_frac max_group |g*|) over non-excluded
    Gaussians (floor_frac defaults to GRAD_FLOOR)."""
    floor_frac = GRAD_FLOOR if floor_frac is None else floor_frac
    out = {}
    keep = np.ones(g_ref.shape[1], bool) if exclude is None else ~exclude
    for name, sl in GROUPS.items():
        a, b = g_gpu[sl][:, keep], g_ref[sl][:, keep]
        floor = floor_frac * max(np.abs(g_ref[sl]).max(), 1e-30)
        rel = np.abs(a - b) / np.maximum(np.abs(b), floor)
        out[name] = float(rel.max()) if rel.size else 0.0
    return out


def cam_f32(cam: Camera) -> Camera:
    """The camera exactly as the C ABI sees it (float32 fields), as float64 values for the oracle."""
    f = lambda x: float(np.float32(x))  # noqa: E731
    return Camera(cam.width, cam.height, f(cam.fx), f(cam.fy), f(cam.cx), f(cam.cy),
                  np.asarray(cam.R, np.float32).astype(np.float64), np.asarray(cam.t, np.float32).astype(np.float64))


def rotated_cam(base: Camera, rotvec, shift) -> Camera:
    """A float32-exact camera rotated and shifted from ``base``."""
    from scipy.spatial.transform import Rotation
    R = Rotation.from_rotvec(rotvec).as_matrix() @ np.asarray(base.R, float)
    return cam_f32(Camera(base.width, base.height, base.fx, base.fy, base.cx, base.cy, R, np.asarray(shift, float)))


def oracle_project_np(p, cam):
    pr = O.project(torch.as_tensor(p, dtype=torch.float64), cam)
    return {k: (v.detach().numpy() if torch.is_tensor(v) else v) for k, v in pr.items()}


def exclude_kernel_limits(p64, cams):
    """Gaussians outside the float32 range of the kernels' pixel-box arithmetic in some view: a
    screen mean beyond +-2^23 px or an integer radius beyond 2^22 px (the kernels cull them; the
    oracle has no such limit). The parity tests leave them out of the comparison."""
    out = np.zeros(p64.shape[1], bool)
    for cam in cams:
        pr = oracle_project_np(p64, cam)
        ok = pr["valid"]
        out |= ok & ((np.abs(pr["u"]) >= 2.0 ** 23) | (np.abs(pr["v"]) >= 2.0 ** 23) | (pr["r"] >= 2.0 ** 22))
    return out

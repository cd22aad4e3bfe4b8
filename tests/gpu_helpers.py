"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
from synth import Camera

# Tolerances of the FP32 CUDA path against the FP64 oracle:
IMG_ATOL = 1e-4          # max abs pixel error
GRAD_RTOL = 1e-3         # per-parameter relative gradient error ...
# ... relative to max(|g*|, GRAD_FLOOR * max |g*| of the parameter group). A gradient is a
# sum of per-pixel terms that partly cancel; in FP32 its absolute error is ~eps32 times the
# sum of the terms' magnitudes, measured at <= 2e-7 of the group's largest gradient. The floor
# holds gradients below 1e-3 of that largest to an absolute error of 1e-6 of it instead.
GRAD_FLOOR = 1e-3
GROUPS = {"mean": slice(0, 3), "logscale": slice(3, 6), "quat": slice(6, 10), "opacity": slice(10, 11),
          "rgb": slice(11, 14)}


def new_map(n_cap, views=1, W=160, H=120, **kw):
    from paper_2504_02437_gb300.api import GaussianMap
    return GaussianMap(capacity=max(n_cap, 1), max_views=views, max_width=W, max_height=H, **kw)


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")


def grad_errors(g_gpu, g_ref, exclude=None):
    """Per-group max relative error |g - g*| / max(|g*|, GRAD_FLOOR max_group |g*|) over non-excluded Gaussians."""
    out = {}
    keep = np.ones(g_ref.shape[1], bool) if exclude is None else ~exclude
    for name, sl in GROUPS.items():
        a, b = g_gpu[sl][:, keep], g_ref[sl][:, keep]
        floor = GRAD_FLOOR * max(np.abs(g_ref[sl]).max(), 1e-30)
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

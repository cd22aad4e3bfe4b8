"""Python face of the C ABI: torch tensors in, torch tensors out.

PyTorch provides device memory and the current CUDA stream; every step of the
mapping path runs in the library's kernels. ``GaussianMap`` owns one library
context; ``rasterize`` wraps render/backward as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[C.c_void_p]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(t: Optional[torch.Tensor]) -> Optional[C.c_void_p]:
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return C.c_void_p(t.data_ptr())


def _f32(t: Optional[torch.Tensor], shape: tuple, name: str, host: bool = False) -> Optional[torch.Tensor]:
    """A contiguous float32 tensor of the given shape, on the GPU (host=False) or in host memory,
    passed without a copy (None stays None)."""
    if t is None:
        return None
    if t.dtype != torch.float32 or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected float32 {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if t.is_cuda == host:
        raise ValueError(f"{name}: expected a {'host' if host else 'CUDA'} tensor")
    return t


def to_gs_camera(cam) -> N.gs_camera:
    """Any object with width, height, fx, fy, cx, cy, R (3x3 world->camera) and t."""
    g = N.gs_camera()
    g.width, g.height = int(cam.width), int(cam.height)
    g.fx, g.fy, g.cx, g.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, dtype=np.float64).reshape(9)
    t = np.asarray(cam.t, dtype=np.float64).reshape(3)
    for i in range(9):
        g.R[i] = float(R[i])
    for i in range(3):
        g.t[i] = float(t[i])
    return g


def _cams(cams) -> tuple:
    if not isinstance(cams, (list, tuple)):
        cams = [cams]
    arr = (N.gs_camera * len(cams))(*[to_gs_camera(c) for c in cams])
    return arr, len(cams), int(cams[0].height), int(cams[0].width)


def default_config(**over) -> N.gs_config:
    lib = N.load()
    cfg = N.gs_config()
    lib.gs_default_config(C.byref(cfg))
    for k, v in over.items():
        if k == "lr":
            for i, x in enumerate(v):
                cfg.lr[i] = float(x)
        else:
            setattr(cfg, k, v)
    return cfg


class GaussianMap:
    """One library context: the Gaussian map, its Adam state and render buffers."""

    def __init__(self, capacity: int = 1 << 20, max_views: int = 8, max_width: int = 1280, max_height: int = 720,
                 device: int = 0, **config):
        self.lib = N.load()
        self.device = device
        self.cfg = default_config(capacity=capacity, max_views=max_views, max_width=max_width,
                                  max_height=max_height, **config)
        ctx = C.c_void_p()
        with torch.cuda.device(device):
            N.check(self.lib.gs_create(C.byref(self.cfg), device, C.byref(ctx)))
        self.ctx = ctx
        self._last_views = 0
        self._last_hw = (0, 0)
        self._last_rgb = None

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.gs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code):
        N.check(code, self.ctx)

    # ---- state
    @property
    def n(self) -> int:
        return self.lib.gs_num_gaussians(self.ctx)

    @property
    def launches(self) -> int:
        """Kernels launched by this context so far."""
        return int(self.lib.gs_launch_count(self.ctx))

    @property
    def tile_size(self) -> int:
        return self.lib.gs_tile_size(self.ctx)

    @property
    def pixels_per_thread(self) -> int:
        return self.lib.gs_pixels_per_thread(self.ctx)

    def set_params(self, params: torch.Tensor):
        p = params.detach().to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        if p.dim() != 2 or p.shape[0] != 14:
            raise ValueError("params must be [14, n]")
        self._check(self.lib.gs_set_params(self.ctx, _ptr(p), p.shape[1], _stream()))

    def params(self) -> torch.Tensor:
        out = torch.empty(14, self.n, device=f"cuda:{self.device}", dtype=torch.float32)
        self._check(self.lib.gs_get_params(self.ctx, _ptr(out), _stream()))
        return out

    def grads(self) -> torch.Tensor:
        out = torch.empty(14, self.n, device=f"cuda:{self.device}", dtype=torch.float32)
        self._check(self.lib.gs_get_grads(self.ctx, _ptr(out), _stream()))
        return out

    def set_grads(self, grads: torch.Tensor):
        """The gradient the next step() applies ([14, n]), e.g. of a loss computed outside."""
        g = grads.detach().to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        if tuple(g.shape) != (14, self.n):
            raise ValueError("grads must be [14, n]")
        self._check(self.lib.gs_set_grads(self.ctx, _ptr(g), _stream()))
        self._keep = g   # alive until the copy on the stream has run

    def init_map(self, points: torch.Tensor, rgb: torch.Tensor):
        pts = points.to(torch.float32).contiguous()
        col = rgb.to(torch.float32).contiguous()
        self._check(self.lib.gs_init_map(self.ctx, _ptr(pts), _ptr(col), pts.shape[0], _stream()))

    # ---- the mapping step
    def render(self, cams, want_T: bool = False, want_argmax: bool = False):
        arr, V, H, W = _cams(cams)
        dev = f"cuda:{self.device}"
        rgb = torch.empty(V, 3, H, W, device=dev, dtype=torch.float32)
        T = torch.empty(V, H, W, device=dev, dtype=torch.float32) if want_T else None
        am = torch.empty(V, H, W, device=dev, dtype=torch.int32) if want_argmax else None
        self._check(self.lib.gs_render(self.ctx, arr, V, _ptr(rgb), _ptr(T), _ptr(am), _stream()))
        self._last_views, self._last_hw = V, (H, W)
        self._last_rgb = rgb      # the library reads it again in loss(); keep it alive until the next render
        out = [rgb]
        if want_T:
            out.append(T)
        if want_argmax:
            out.append(am)
        return out[0] if len(out) == 1 else tuple(out)

    def loss(self, target: torch.Tensor) -> torch.Tensor:
        tg = target.to(torch.float32).contiguous()
        out = torch.empty(3, device=f"cuda:{self.device}", dtype=torch.float32)
        self._check(self.lib.gs_loss(self.ctx, _ptr(tg), _ptr(out), _stream()))
        return out

    def backward(self, dL_drgb: Optional[torch.Tensor] = None):
        g = None if dL_drgb is None else dL_drgb.to(torch.float32).contiguous()
        self._check(self.lib.gs_backward(self.ctx, _ptr(g), _stream()))

    def step(self):
        self._check(self.lib.gs_step(self.ctx, _stream()))

    def iterate(self, cams, target: torch.Tensor, loss_out: Optional[torch.Tensor] = None,
                rgb_out: Optional[torch.Tensor] = None) -> torch.Tensor:
        arr, V, H, W = _cams(cams)
        if loss_out is None:
            loss_out = torch.empty(3, device=f"cuda:{self.device}", dtype=torch.float32)
        target = _f32(target, (V, 3, H, W), "target")
        _f32(loss_out, (3,), "loss_out")
        _f32(rgb_out, (V, 3, H, W), "rgb_out")
        self._check(self.lib.gs_iterate(self.ctx, arr, V, _ptr(target), _ptr(loss_out), _ptr(rgb_out), _stream()))
        self._last_views, self._last_hw = V, (H, W)
        return loss_out

    def iterate_host(self, cams, target: torch.Tensor, loss_out: Optional[torch.Tensor] = None,
                     rgb_out: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
        """The mapping iteration with the target [V, 3, H, W] and the loss [3] in host memory
        (pinned keeps the copies asynchronous): the library uploads the target while the
        projection and the sorts run and copies the loss back on the current stream (read it after
        synchronising). The target must stay unchanged until the stream has passed the call."""
        arr, V, H, W = _cams(cams)
        _f32(target, (V, 3, H, W), "target", host=True)
        _f32(loss_out, (3,), "loss_out", host=True)
        _f32(rgb_out, (V, 3, H, W), "rgb_out")
        self._check(self.lib.gs_iterate_host(self.ctx, arr, V, _hptr(target), _hptr(loss_out), _ptr(rgb_out),
                                             _stream()))
        self._last_views, self._last_hw = V, (H, W)
        # the host buffers stay referenced until the stream has passed the call (the upload and the
        # loss copy have run): a pinned block torch frees can be handed out again at once
        done = torch.cuda.Event()
        done.record()
        self._host_inflight = [x for x in getattr(self, "_host_inflight", []) if not x[0].query()]
        self._host_inflight.append((done, target, loss_out))
        return loss_out

    # ---- map management
    def insert(self, cam, image: torch.Tensor, points: torch.Tensor, return_mask: bool = False):
        """Insert the points that are not behind rendered opacity > insert_opacity (or, with
        insert_tau > 0, that lie farther than insert_tau from every existing mean); returns
        the count (and the per-point inserted mask with ``return_mask``)."""
        arr, V, H, W = _cams([cam])
        pts = points.to(torch.float32).contiguous()
        img = image.to(torch.float32).contiguous()
        n = C.c_int()
        mask = torch.empty(pts.shape[0], dtype=torch.uint8, device=pts.device) if return_mask else None
        self._check(self.lib.gs_insert(self.ctx, arr, _ptr(img), _ptr(pts), pts.shape[0], C.byref(n), _ptr(mask),
                                       _stream()))
        return (n.value, mask.bool()) if return_mask else n.value

    def set_initializer(self, mlp):
        """Use the learned initialiser for insertions (None: the plain initialisation)."""
        self._init_mlp = mlp
        self._check(self.lib.gs_set_initializer(self.ctx, mlp.handle if mlp is not None else None))

    def count_dominant(self, cams):
        """Add each Gaussian's dominated pixels in these views (Eq. 8-9) to its count."""
        arr, V, H, W = _cams(cams)
        self._check(self.lib.gs_count_dominant(self.ctx, arr, V, _stream()))

    def densify(self, normals: Optional[torch.Tensor] = None) -> int:
        nz = None if normals is None else normals.to(torch.float32).contiguous()
        n = C.c_int()
        self._check(self.lib.gs_densify(self.ctx, _ptr(nz), C.byref(n), _stream()))
        return n.value

    def mlp_targets(self, first: int, count: int) -> torch.Tensor:
        """Learned-initialiser training targets [count, 16] of Gaussians first .. first + count - 1
        (log-scale, unit quaternion with w >= 0, opacity logit, colour, zeros)."""
        out = torch.empty(count, 16, device=f"cuda:{self.device}", dtype=torch.float32)
        self._check(self.lib.gs_mlp_targets(self.ctx, int(first), int(count), _ptr(out), _stream()))
        return out

    def psnr(self, img: torch.Tensor, ref: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """10 log10(1 / MSE) of img against ref (same shape, float32, values in [0, 1]) into a
        device scalar (``out``, a float32 tensor of one element, when given)."""
        a = _f32(img, tuple(img.shape), "img")
        b = _f32(ref, tuple(img.shape), "ref")
        if out is None:
            out = torch.empty((), device=f"cuda:{self.device}", dtype=torch.float32)
        self._check(self.lib.gs_psnr(self.ctx, _ptr(a), _ptr(b), a.numel(), _ptr(out), _stream()))
        return out

    # ---- checkpoint / resume
    def save(self, path: str) -> None:
        """Write the map state (parameters, Adam moments and step state, densification
        statistics) to ``path``; waits for the current stream's work first."""
        self._check(self.lib.gs_save(self.ctx, os.fsencode(path), _stream()))

    def load(self, path: str) -> None:
        """Replace the map state with the checkpoint at ``path`` (checked in full first)."""
        self._check(self.lib.gs_load(self.ctx, os.fsencode(path), _stream()))
        self._last_views = 0

    # ---- timing
    def timing(self, enable: bool = True, phases=None):
        """Start (discarding earlier records) or stop per-phase device timing; ``phases`` (names of
        ``PHASES``) restricts it to those phases."""
        if enable and phases is not None:
            mask = 0
            for name in phases:
                mask |= 1 << N.PHASES.index(name)
            self._check(self.lib.gs_timing_phases(self.ctx, mask))
        else:
            self._check(self.lib.gs_timing_enable(self.ctx, 1 if enable else 0))

    def timing_read(self) -> dict:
        """Summed device milliseconds and interval counts per phase since timing was enabled."""
        ms = np.zeros(len(N.PHASES), np.float32)
        cnt = np.zeros(len(N.PHASES), np.int32)
        self._check(self.lib.gs_timing_read(self.ctx, ms.ctypes.data_as(C.c_void_p), cnt.ctypes.data_as(C.c_void_p)))
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(N.PHASES)}

    # ---- introspection
    def debug_projection(self, view: int = 0) -> np.ndarray:
        out = np.empty((9, self.n), np.float64)
        self._check(self.lib.gs_debug_projection(self.ctx, view, out.ctypes.data_as(C.c_void_p)))
        return out

    def debug_pairs(self):
        cnt = C.c_int64()
        self._check(self.lib.gs_debug_pairs(self.ctx, None, None, 0, C.byref(cnt)))
        P = cnt.value
        bins = np.empty(P, np.uint32)
        vals = np.empty(P, np.uint32)
        self._check(self.lib.gs_debug_pairs(self.ctx, bins.ctypes.data_as(C.c_void_p),
                                            vals.ctypes.data_as(C.c_void_p), P, C.byref(cnt)))
        return bins, vals

    def debug_work(self) -> dict:
        out = np.zeros(4, np.int64)
        self._check(self.lib.gs_debug_work(self.ctx, out.ctypes.data_as(C.c_void_p)))
        return dict(pairs=int(out[0]), tested=int(out[1]), blended=int(out[2]), walked=int(out[3]))

    def debug_grad2d(self) -> np.ndarray:
        out = np.empty((self._last_views, 9, self.n), np.float32)
        self._check(self.lib.gs_debug_grad2d(self.ctx, out.ctypes.data_as(C.c_void_p)))
        return out


def checkpoint_info(path: str) -> dict:
    """Number of Gaussians and format version of a checkpoint, after the same checks as a
    load; raises if the file is missing or not a valid checkpoint. Needs no GPU."""
    lib = N.load()
    n, ver = C.c_int(), C.c_int()
    N.check(lib.gs_checkpoint_info(os.fsencode(path), C.byref(n), C.byref(ver)), None)
    return {"n": n.value, "version": ver.value}


class MLP:
    """The learned initialiser (BF16 tensor-core MLP) behind the C ABI."""

    def __init__(self, seed: int = 0, device: int = 0):
        self.lib = N.load()
        self.device = device
        h = C.c_void_p()
        with torch.cuda.device(device):
            N.check(self.lib.gs_mlp_create(device, seed, C.byref(h)))
        self.handle = h
        self.n_params = self.lib.gs_mlp_num_params()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gs_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        return f"cuda:{self.device}"

    def set_params(self, flat: torch.Tensor):
        f = flat.to(device=self._dev(), dtype=torch.float32).contiguous()
        N.check(self.lib.gs_mlp_set_params(self.handle, _ptr(f), _stream()))

    def params(self) -> torch.Tensor:
        out = torch.empty(self.n_params, device=self._dev())
        N.check(self.lib.gs_mlp_get_params(self.handle, _ptr(out), _stream()))
        return out

    def grads(self) -> torch.Tensor:
        out = torch.empty(self.n_params, device=self._dev())
        N.check(self.lib.gs_mlp_get_grads(self.handle, _ptr(out), _stream()))
        return out

    @staticmethod
    def features(cam, image: torch.Tensor, points: torch.Tensor) -> torch.Tensor:
        lib = N.load()
        arr, V, H, W = _cams([cam])
        pts = points.to(torch.float32).contiguous()
        img = image.to(torch.float32).contiguous()
        out = torch.empty(pts.shape[0], 80, device=pts.device)
        N.check(lib.gs_mlp_features(arr, _ptr(img), _ptr(pts), pts.shape[0], _ptr(out), _stream()))
        return out

    def forward(self, feats: torch.Tensor) -> torch.Tensor:
        f = feats.to(torch.float32).contiguous()
        out = torch.empty(f.shape[0], 16, device=f.device)
        N.check(self.lib.gs_mlp_forward(self.handle, _ptr(f), f.shape[0], _ptr(out), _stream()))
        return out

    def backward(self, feats: torch.Tensor, targets: torch.Tensor) -> torch.Tensor:
        f = feats.to(torch.float32).contiguous()
        t = targets.to(torch.float32).contiguous()
        loss = torch.empty(1, device=f.device)
        N.check(self.lib.gs_mlp_backward(self.handle, _ptr(f), _ptr(t), f.shape[0], _ptr(loss), _stream()))
        return loss

    def step(self, lr: float):
        N.check(self.lib.gs_mlp_step(self.handle, float(lr), _stream()))


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, gmap, cams):
        gmap.set_params(params)
        rgb = gmap.render(cams)
        ctx.gmap = gmap
        return rgb

    @staticmethod
    def backward(ctx, grad_rgb):
        gmap = ctx.gmap
        gmap.backward(grad_rgb.contiguous())
        return gmap.grads(), None, None


def rasterize(params: torch.Tensor, gmap: GaussianMap, cams) -> torch.Tensor:
    """Differentiable render of ``params`` [14, n] through the library (adjoint kernels in backward)."""
    return _Rasterize.apply(params, gmap, cams)

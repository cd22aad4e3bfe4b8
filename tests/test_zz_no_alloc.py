"""The allocation-free pair sort (gs_sort_pairs_static) against the pair sort of gs_render.

gs_sort_pairs_static serves callers that cannot allocate device memory: its
scratch is a static device array, so it is limited to 2^20 pairs. The test
rebuilds the order in which gs_render emits its pairs (Gaussians by depth,
each one's tiles in row-major order) from the render's own sorted pairs, sorts
that sequence by tile with the static entry point, and requires the render's
sorted pairs bit for bit, on two scenes in a row and on a repeat of the first
(the shared scratch keeps the previous call's contents).
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import frustum_scene

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2504_02437_gb300 import _native as N
    from paper_2504_02437_gb300 import build as B
    B.build()
    return N, N.load()


def _render_pairs(seed, n):
    from paper_2504_02437_gb300.api import GaussianMap
    p, cam = frustum_scene(n=n, seed=seed)
    gm = GaussianMap(capacity=n, max_views=1, max_width=160, max_height=120)
    gm.set_params(torch.as_tensor(p, device="cuda"))
    gm.render(cam)
    bins, vals = gm.debug_pairs()
    depth32 = gm.debug_projection(0)[5].astype(np.float32)
    tiles = int(np.ceil(160 / gm.tile_size) * np.ceil(120 / gm.tile_size))
    gm.close()
    return bins, vals, depth32, tiles


def _emission_order(bins, vals, depth32):
    # gs_render emits Gaussians in (depth, id) order, each Gaussian's tiles in increasing bin order
    order = np.lexsort((bins, vals, depth32.view(np.uint32)[vals]))
    return bins[order], vals[order]


def _static_sort(N, lib, keys, vals, bits):
    kd = torch.as_tensor(keys.astype(np.int64), device="cuda").to(torch.int32)
    vd = torch.as_tensor(vals.astype(np.int64), device="cuda").to(torch.int32)
    ko = torch.empty_like(kd)
    vo = torch.empty_like(vd)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.gs_sort_pairs_static(C.c_void_p(kd.data_ptr()), C.c_void_p(vd.data_ptr()),
                                    C.c_void_p(ko.data_ptr()), C.c_void_p(vo.data_ptr()), keys.size, bits, s)
    assert code == N.GS_OK
    torch.cuda.synchronize()
    return ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint32)


def test_static_sort_matches_render_sort_twice():
    N, lib = _lib()
    scenes = [_render_pairs(0, 2000), _render_pairs(5, 3000)]
    for bins, vals, depth32, tiles in scenes + scenes[:1]:
        assert bins.size > 0
        ek, ev = _emission_order(bins, vals, depth32)
        bits = max(1, int(np.ceil(np.log2(tiles))))
        for _ in range(2):          # two calls in a row on the same input
            ok, ov = _static_sort(N, lib, ek, ev, bits)
            np.testing.assert_array_equal(ok, bins)
            np.testing.assert_array_equal(ov, vals)


def test_static_sort_limits():
    N, lib = _lib()
    null = C.c_void_p()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.gs_sort_pairs_static(null, null, null, null, (1 << 20) + 1, 16, s) == N.GS_ERR_CAPACITY
    assert lib.gs_sort_pairs_static(null, null, null, null, 10, 0, s) == N.GS_ERR_ARG
    assert lib.gs_sort_pairs_static(null, null, null, null, 0, 8, s) == N.GS_OK

"""The allocation-free pair sort (gs_sort_pairs_static) against the pair sort of gs_render.

gs_sort_pairs_static serves callers that cannot allocate device memory: its
scratch is a static device array, so it is limited to 2^20 pairs. The test
rebuilds the order in which gs_render emits its pairs (Gaussians by depth,
each one's tiles in row-major order) from the render's own sorted pairs, sorts
that sequence by tile with the static entry point, and requires the render's
sorted pairs bit for bit, on two scenes in a row and on a repeat of the first
(the shared scratch keeps the previous call's contents). It also sorts seeded
random keys with 1 to 4 radix passes (bits 7 to 32; the passes in between go
through the scratch array's ping-pong halves) at sizes up to the 2^20 limit,
against numpy's stable argsort, larger and smaller inputs back to back.
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


def _dev_u32(a):
    """uint32 numpy array -> int32 CUDA tensor with the same bits."""
    return torch.as_tensor(np.ascontiguousarray(a, np.uint32).view(np.int32), device="cuda")


def _static_sort(N, lib, keys, vals, bits):
    kd = _dev_u32(keys)
    vd = _dev_u32(vals)
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


def _expect(keys, vals, bits):
    mask = np.uint32(0xFFFFFFFF if bits == 32 else (1 << bits) - 1)
    order = np.argsort(keys & mask, kind="stable")
    return keys[order], vals[order]


@pytest.mark.parametrize("bits", [7, 9, 16, 24, 32])
def test_static_sort_random_keys_every_pass_count(bits):
    """1 (bits 7), 2 (9, 16), 3 (24) and 4 (32) radix passes on random keys, some with bits set
    above `bits` (ignored by the sort, kept in the output), largest size first, then smaller
    ones: the scratch keeps the previous call's contents."""
    N, lib = _lib()
    rng = np.random.default_rng(bits)
    for n in (1 << 20, 300_000, 4097, 31, 1):
        keys = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        if n > 100:
            keys[: n // 3] &= np.uint32((1 << min(bits, 31)) - 1)   # a third within `bits`
            keys[n // 3: n // 2] = keys[0]                           # runs of equal keys
        vals = np.arange(n, dtype=np.uint32) ^ np.uint32(0x5A5A5A5A)
        ek, ev = _expect(keys, vals, bits)
        for _ in range(2):          # two calls in a row
            ok, ov = _static_sort(N, lib, keys, vals, bits)
            np.testing.assert_array_equal(ok, ek)
            np.testing.assert_array_equal(ov, ev)


def test_static_sort_limits():
    N, lib = _lib()
    null = C.c_void_p()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.gs_sort_pairs_static(null, null, null, null, (1 << 20) + 1, 16, s) == N.GS_ERR_CAPACITY
    assert lib.gs_sort_pairs_static(null, null, null, null, 10, 0, s) == N.GS_ERR_ARG
    assert lib.gs_sort_pairs_static(null, null, null, null, 10, 33, s) == N.GS_ERR_ARG
    assert lib.gs_sort_pairs_static(null, null, null, null, 0, 8, s) == N.GS_OK
    # outputs that overlap an input or each other are rejected before anything is launched
    buf = torch.zeros(4 * 64, dtype=torch.int32, device="cuda")
    a, b, c, d = (C.c_void_p(buf[i * 64:].data_ptr()) for i in range(4))
    part = C.c_void_p(buf[32:].data_ptr())          # overlaps the second half of a
    for args in ((a, b, c, a), (a, b, b, d), (a, b, c, c), (a, b, part, d), (a, b, c, part)):
        assert lib.gs_sort_pairs_static(*args, 64, 16, s) == N.GS_ERR_ARG
    assert lib.gs_sort_pairs_static(a, a, c, d, 64, 16, s) == N.GS_OK    # inputs may coincide
    torch.cuda.synchronize()

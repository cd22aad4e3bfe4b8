"""gs_iterate_host: the mapping iteration (Section 3.2, Eq. 3, 10-11) with the target and the loss in
host memory; the library uploads each call's target into one of two device buffers on a copy
stream, beside the previous call's iteration, and copies the loss back after the iteration.
Deterministic mode, bit for bit against gs_iterate with the same target on the device: the first
(direct) call, the graph's replays, targets that change from call to call (each replay must read
its own upload, also when the calls are issued without waiting), pinned and pageable host memory."""
import numpy as np
import pytest
import torch

from synth import frustum_scene, random_target

from gpu_helpers import cuda, new_map, rotated_cam

pytestmark = pytest.mark.gpu


def _run(p, cams, targets, host, pinned=True, sync=True, **kw):
    """Iterations over the targets; with sync=False the host issues every call without waiting
    (each host target and loss buffer is its own tensor, read after the last call)."""
    gm = new_map(p.shape[1], views=len(cams), **kw)
    gm.set_params(cuda(p))
    losses = []
    for tg in targets:
        if host:
            t = torch.from_numpy(np.ascontiguousarray(tg, dtype=np.float32))
            lo = torch.empty(3)
            if pinned:
                t, lo = t.pin_memory(), lo.pin_memory()
            gm.iterate_host(cams, t, lo)
        else:
            lo = torch.empty(3, device="cuda")
            gm.iterate(cams, cuda(tg), lo)
        if sync:
            torch.cuda.synchronize()
        losses.append(lo)
    torch.cuda.synchronize()
    out = gm.params().cpu().numpy(), np.array([lo.cpu().numpy() for lo in losses])
    gm.close()
    return out


@pytest.mark.parametrize("pinned,sync", [(True, True), (False, True), (True, False)])
def test_host_target_matches_device_target_bit_for_bit(pinned, sync):
    p, cam = frustum_scene()
    cams = [cam, rotated_cam(cam, [0.03, -0.05, 0.01], [0.05, 0.0, 0.1])]
    # six calls (one direct, five replays), each with a different target
    targets = [random_target(160, 120, seed=20 + i, n_views=2) for i in range(6)]
    ref_p, ref_l = _run(p, cams, targets, host=False, deterministic=1)
    got_p, got_l = _run(p, cams, targets, host=True, pinned=pinned, sync=sync, deterministic=1)
    assert np.array_equal(got_l, ref_l)
    assert np.array_equal(got_p, ref_p)
    # the targets differ, and so do the losses: each replay read its own upload
    assert len({float(l[1]) for l in got_l}) == len(targets)


def test_host_target_with_the_autotuner_and_the_default_mode():
    """Autotuned layout (its timing runs read the target too), float atomics: the losses equal the
    device-target path's to float32 rounding, and the map moves the same way (Adam turns the
    atomics' rounding differences of near-zero gradients into steps of either sign, so a few
    parameters may differ by up to twice the learning rate)."""
    p, cam = frustum_scene()
    targets = [random_target(160, 120, seed=40 + i) for i in range(4)]
    ref_p, ref_l = _run(p, [cam], targets, host=False, tile_size=0)
    got_p, got_l = _run(p, [cam], targets, host=True, tile_size=0)
    np.testing.assert_allclose(got_l, ref_l, rtol=1e-4, atol=1e-7)
    d = np.abs(got_p - ref_p)
    assert np.median(d) < 1e-7 and (d > 1e-4).mean() < 1e-3, (np.median(d), (d > 1e-4).mean())


def test_host_and_device_calls_interleaved():
    """Calls of gs_iterate and gs_iterate_host alternate on one map (each switch records the
    iteration again: the two write the loss to different buffers): the sequence equals the
    all-device one bit for bit (deterministic mode)."""
    p, cam = frustum_scene()
    targets = [random_target(160, 120, seed=60 + i) for i in range(6)]
    ref_p, _ = _run(p, [cam], targets, host=False, deterministic=1)
    gm = new_map(p.shape[1], deterministic=1)
    gm.set_params(cuda(p))
    for i, tg in enumerate(targets):
        if i % 2:
            gm.iterate_host([cam], torch.from_numpy(tg.astype(np.float32)).pin_memory())
        else:
            gm.iterate([cam], cuda(tg), torch.empty(3, device="cuda"))
    torch.cuda.synchronize()
    got_p = gm.params().cpu().numpy()
    gm.close()
    assert np.array_equal(got_p, ref_p)


def test_host_target_argument_errors():
    p, cam = frustum_scene()
    gm = new_map(p.shape[1])
    gm.set_params(cuda(p))
    with pytest.raises(ValueError):
        gm.iterate_host([cam], cuda(random_target(160, 120, seed=1)))   # a device tensor
    with pytest.raises(ValueError):
        gm.iterate_host([cam], torch.zeros(1, 3, 120, 161))                 # wrong shape
    gm.close()

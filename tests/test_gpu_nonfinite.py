"""Non-finite detection without a GPU fault: a target with one NaN pixel makes the loss total
non-finite; the device flag it sets is reported as GS_ERR_NONFINITE once by the next call that
reads the device flags, and the map carries on. Adam leaves a parameter whose gradient is not
finite (and its moments) unchanged."""
import numpy as np
import pytest
import torch

from paper_2504_02437_gb300._native import GS_ERR_NONFINITE, GSError
from synth import frustum_scene, random_target

from gpu_helpers import cuda, new_map

pytestmark = pytest.mark.gpu


def _iterate(gm, cam, tg, loss):
    try:
        gm.iterate([cam], tg, loss)
        torch.cuda.synchronize()
        return 0
    except GSError as e:
        torch.cuda.synchronize()
        return e.code


def test_nonfinite_loss_is_reported_and_the_map_carries_on():
    p, cam = frustum_scene()
    tg = random_target(160, 120, seed=1)
    bad = tg.copy()
    bad[0, 0, 60, 80] = np.nan
    gm = new_map(p.shape[1], tile_size=16, pixels_per_thread=2)
    gm.set_params(cuda(p))
    loss = torch.empty(3, device="cuda")
    codes = [_iterate(gm, cam, cuda(bad), loss) for _ in range(5)]
    # the first call runs directly and records the graph; a replay's flags are read by the call
    # after it, so a report comes by the third call and each one is followed by a working call
    assert GS_ERR_NONFINITE in codes[:3], codes
    assert set(codes) <= {0, GS_ERR_NONFINITE}, codes
    assert all(not (a == b == GS_ERR_NONFINITE) for a, b in zip(codes, codes[1:])), codes
    # back to a finite target: at most the pending report, then every call works
    clean = [_iterate(gm, cam, cuda(tg), loss) for _ in range(4)]
    assert clean[1:] == [0, 0, 0], clean
    assert clean[0] in (0, GS_ERR_NONFINITE)
    assert torch.isfinite(loss).all()
    assert torch.isfinite(gm.params()).all()
    gm.close()


def test_nonfinite_gradient_leaves_the_parameter_unchanged():
    """gs_step on a gradient buffer holding one NaN: that entry keeps its value, every other
    parameter moves, and the next render reports the flag once."""
    p, cam = frustum_scene()
    tg = random_target(160, 120, seed=2)
    gm = new_map(p.shape[1], tile_size=16, pixels_per_thread=1)
    gm.set_params(cuda(p))
    gm.render(cam)
    gm.loss(cuda(tg))
    gm.backward()
    before = gm.params().clone()
    g = gm.grads()
    assert torch.isfinite(g).all()
    # a NaN gradient entry for the red colour of Gaussian 5
    g[11, 5] = float("nan")
    gm.set_grads(g)
    gm.step()
    after = gm.params()
    assert after[11, 5] == before[11, 5]
    live = torch.isfinite(g) & (g != 0)
    assert ((after != before) & live).sum() > 0.9 * live.sum()
    with pytest.raises(GSError) as e:
        gm.render(cam)
    assert e.value.code == GS_ERR_NONFINITE
    gm.render(cam)   # reported once
    gm.close()


@pytest.mark.parametrize("tile,ppt", [(16, 1), (16, 2)])
def test_report_from_a_first_iteration_leaves_the_map_usable(tile, ppt):
    """The flag of a non-finite gradient is reported by the first (direct) gs_iterate of a shape,
    which then stops after the projection: the zeroing it had issued on its second stream must not
    be taken for done by the calls that follow. Renders after it equal a fresh map's render of the
    same parameters bit for bit (their work queues start from zero every time), and the mapping
    iteration then runs."""
    p, cam = frustum_scene()
    tg = cuda(random_target(160, 120, seed=3))
    gm = new_map(p.shape[1], tile_size=tile, pixels_per_thread=ppt)
    gm.set_params(cuda(p))
    gm.render(cam)
    gm.loss(tg)
    gm.backward()
    g = gm.grads()
    g[11, 5] = float("nan")
    gm.set_grads(g)
    gm.step()
    loss = torch.empty(3, device="cuda")
    assert _iterate(gm, cam, tg, loss) == GS_ERR_NONFINITE
    ref_map = new_map(p.shape[1], tile_size=tile, pixels_per_thread=ppt)
    ref_map.set_params(gm.params())
    ref = ref_map.render(cam).clone()
    for _ in range(3):
        assert torch.equal(gm.render(cam), ref)
    codes = [_iterate(gm, cam, tg, loss) for _ in range(3)]
    assert codes == [0, 0, 0], codes
    assert torch.isfinite(loss).all() and torch.isfinite(gm.params()).all()
    ref_map.close()
    gm.close()

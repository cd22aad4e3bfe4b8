"""Checkpoint and resume through gs_save / gs_load on the GPU.

A map saved after some Adam steps and loaded into a fresh context holds the same parameters bit
for bit, and continues like the uninterrupted run: the same losses and parameters afterwards, up
to the float32 gradient atomics' run-to-run rounding (the bound of the graph-vs-separate-calls
test). A control that restarts from the same parameters with fresh Adam moments moves visibly
differently, so the match shows that the moments and step counters were carried over. The
densification statistics come back too: densifying the original and the loaded map gives the
same split. A load into a context that is too small fails and leaves it unchanged.
"""
import numpy as np
import pytest
import torch

from synth import frustum_scene, random_target

from gpu_helpers import cuda, new_map, rotated_cam

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    p, cam = frustum_scene()
    return p, cam, random_target(160, 120, seed=1)


def views(cam):
    return [cam, rotated_cam(cam, [0.02, -0.03, 0.0], [0.03, 0.0, 0.05]),
            rotated_cam(cam, [-0.01, 0.02, 0.01], [-0.02, 0.01, 0.0]), cam]


def test_resume_continues_like_the_uninterrupted_run(tmp_path, scene):
    from paper_2504_02437_gb300.api import checkpoint_info
    p, cam, tg = scene
    n = p.shape[1]
    tgt = cuda(tg)
    loss = torch.empty(3, device="cuda")
    ga = new_map(n)
    ga.set_params(cuda(p))
    for c in views(cam)[:3]:
        ga.iterate(c, tgt, loss)
    path = str(tmp_path / "map.ckpt")
    ga.save(path)
    assert checkpoint_info(path) == {"n": n, "version": 1}
    saved = ga.params().clone()

    gb = new_map(n)
    gb.load(path)
    assert gb.n == n
    assert torch.equal(gb.params(), saved)

    gc = new_map(n)              # control: same parameters, fresh Adam state
    gc.set_params(saved)
    la, lb = [], []
    for c in views(cam)[1:]:
        for gm, out in ((ga, la), (gb, lb), (gc, None)):
            gm.iterate(c, tgt, loss)
            if out is not None:
                out.append(loss.cpu().numpy().copy())
    np.testing.assert_allclose(np.array(la), np.array(lb), rtol=1e-5)
    pa, pb, pc = (g.params().cpu().numpy() for g in (ga, gb, gc))
    d = np.abs(pa - pb)
    assert np.median(d) < 1e-7
    assert (d > 1e-5).mean() < 1e-3
    assert np.abs(pa - pc).max() > 100 * max(d.max(), 1e-6)


def test_densification_statistics_survive(tmp_path, scene):
    p, cam, tg = scene
    n = p.shape[1]
    tgt = cuda(tg)
    loss = torch.empty(3, device="cuda")
    ga = new_map(2 * n, split_thresh=1e-6)
    ga.set_params(cuda(p))
    for c in views(cam):
        ga.iterate(c, tgt, loss)
    path = str(tmp_path / "stats.ckpt")
    ga.save(path)
    gb = new_map(2 * n, split_thresh=1e-6)
    gb.load(path)
    na, nb = ga.densify(), gb.densify()
    assert na == nb and na > 0
    assert ga.n == gb.n == n + na
    assert torch.equal(ga.params(), gb.params())


def test_load_into_a_small_context_fails_and_changes_nothing(tmp_path, scene):
    from paper_2504_02437_gb300 import _native as N
    p, cam, tg = scene
    n = p.shape[1]
    ga = new_map(n)
    ga.set_params(cuda(p))
    path = str(tmp_path / "big.ckpt")
    ga.save(path)
    small = new_map(100)
    small.set_params(cuda(p[:, :100]))
    before = small.params().clone()
    with pytest.raises(N.GSError) as e:
        small.load(path)
    assert e.value.code == N.GS_ERR_CAPACITY
    assert small.n == 100 and torch.equal(small.params(), before)
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(open(path, "rb").read()[:-4])
    with pytest.raises(N.GSError) as e:
        small.load(str(bad))
    assert e.value.code == N.GS_ERR_IO
    assert torch.equal(small.params(), before)

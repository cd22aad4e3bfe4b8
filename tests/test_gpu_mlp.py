"""GPU parity of the learned initialiser (BF16 tensor-core MLP) against the FP64 oracle.

The oracle evaluates the same network in float64 on bfloat16-rounded inputs,
weights and hidden activations. The kernels additionally round the
backward's upstream gradients to bfloat16 (tensor-core operands), so forward
outputs are held to 1e-2 of the output scale and weight gradients to 1e-2
relative (floored at 1e-2 of the layer's largest gradient), the bfloat16
rounding level (2^-8) with margin.
"""
import numpy as np
import pytest
import torch

import oracle as O
from synth import frustum_scene, random_target

from gpu_helpers import cuda, new_map

pytestmark = pytest.mark.gpu


def _mlp(seed=0):
    from paper_2504_02437_gb300.api import MLP
    return MLP(seed=seed)


def _feats(n, seed):
    rng = np.random.default_rng(seed)
    f = np.zeros((n, 80), np.float32)
    f[:, :75] = rng.uniform(size=(n, 75))
    f[:, 75] = rng.uniform(1, 5, size=n)
    f[:, 76:79] = rng.normal(size=(n, 3))
    f[:, 78] = f[:, 75]
    return f


def test_forward_matches_oracle():
    m = _mlp(1)
    flat = m.params().cpu().numpy().astype(np.float64)
    f = _feats(1000, 2)
    y = m.forward(cuda(f)).cpu().numpy()
    ref = O.mlp_forward(flat, f.astype(np.float64))
    scale = np.abs(ref[:, :11]).max()
    assert np.abs(y[:, :11] - ref[:, :11]).max() <= 1e-2 * scale
    # away from bfloat16 rounding flips the agreement is much closer than the bound
    assert np.median(np.abs(y[:, :11] - ref[:, :11])) <= 1e-3 * scale
    np.testing.assert_array_equal(y[:, 11:], 0.0)


def test_gradients_match_oracle():
    m = _mlp(3)
    flat = m.params().cpu().numpy().astype(np.float64)
    f = _feats(4096, 4)
    tg = np.random.default_rng(5).normal(size=(4096, 16)).astype(np.float32)
    tg[:, 11:] = 0
    loss = float(m.backward(cuda(f), cuda(tg)).cpu()[0])
    g = m.grads().cpu().numpy()
    L, gref = O.mlp_loss_and_grad(flat, f.astype(np.float64), tg.astype(np.float64))
    assert abs(loss - L) <= 1e-3 * L
    o = 0
    for shape in O.MLP_SHAPES:
        k = int(np.prod(shape))
        a, b = g[o:o + k], gref[o:o + k]
        floor = 1e-2 * max(np.abs(b).max(), 1e-30)
        rel = np.abs(a - b) / np.maximum(np.abs(b), floor)
        assert rel.max() <= 1e-2, (shape, rel.max())
        o += k
    assert np.all(g[-16 + 11:] == 0) and np.all(g[O.MLP_SIZE - 16 - 5 * 128:O.MLP_SIZE - 16] == 0)


def test_features_match_oracle():
    p, cam = frustum_scene(n=10, seed=0)
    img = random_target(160, 120, seed=6)[0]
    rng = np.random.default_rng(7)
    pts = np.stack([rng.uniform(-1, 1, 300), rng.uniform(-0.8, 0.8, 300), rng.uniform(1, 4, 300)], 1)
    pts = pts.astype(np.float32)
    from paper_2504_02437_gb300.api import MLP
    f = MLP.features(cam, cuda(img), cuda(pts)).cpu().numpy()
    ref = O.mlp_features(pts.astype(np.float64), cam, img)
    np.testing.assert_array_equal(f[:, :75], ref[:, :75].astype(np.float32))
    np.testing.assert_allclose(f[:, 75:], ref[:, 75:], rtol=1e-6, atol=1e-6)


def test_training_reduces_loss():
    """A few hundred Adam steps on a smooth synthetic target cut the loss by 10x."""
    m = _mlp(8)
    f = _feats(8192, 9)
    W = np.random.default_rng(10).normal(size=(80, 16)).astype(np.float32) * 0.05
    tg = np.tanh(f @ W).astype(np.float32)
    tg[:, 11:] = 0
    fd, td = cuda(f), cuda(tg)
    first = float(m.backward(fd, td).cpu()[0])
    for _ in range(300):
        m.backward(fd, td)
        m.step(1e-3)
    last = float(m.backward(fd, td).cpu()[0])
    assert last < 0.1 * first, (first, last)


def test_insert_with_learned_initialiser():
    p, cam = frustum_scene(n=500, seed=2)
    img = random_target(160, 120, seed=3)[0]
    rng = np.random.default_rng(4)
    pix = np.stack([rng.integers(0, 160, 50), rng.integers(0, 120, 50)], 1)
    z = 6.0                                  # behind every Gaussian: nothing is opaque enough to skip
    pts = np.stack([(pix[:, 0] - cam.cx) / cam.fx * z, (pix[:, 1] - cam.cy) / cam.fy * z, np.full(50, z)], 1)
    pts = pts.astype(np.float32)
    m = _mlp(11)
    gm = new_map(1000)
    gm.set_params(cuda(p))
    gm.set_initializer(m)
    n_ins, mask = gm.insert(cam, cuda(img), cuda(pts), return_mask=True)
    mask = mask.cpu().numpy()
    assert n_ins == int(mask.sum()) > 0
    got = gm.params().cpu().numpy()[:, 500:]
    from paper_2504_02437_gb300.api import MLP
    y = m.forward(MLP.features(cam, cuda(img), cuda(pts))).cpu().numpy()[mask]
    np.testing.assert_array_equal(got[0:3], pts[mask].T)
    ok = np.all(np.isfinite(y[:, :11]), 1) & np.all((y[:, :3] >= -9) & (y[:, :3] <= 1), 1)
    np.testing.assert_allclose(got[3:14, ok], y[ok, :11].T, rtol=1e-6, atol=1e-7)
    gm.set_initializer(None)

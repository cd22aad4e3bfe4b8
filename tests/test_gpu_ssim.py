"""GPU parity of the SSIM term of Eq. 10 (L_color = 0.8 L1 + 0.2 (1 - SSIM)) against the FP64 oracle.

Same 2,000-Gaussian 160x120 scene as the L1 parity tests; the oracle takes dL/dC of the whole
image through its plain SSIM definition (11 x 11 Gaussian window, zero padding) and propagates
it through the compositing. Tolerances as for L1: loss 1e-5 relative, parameter gradients 1e-3
relative (floored at 1e-3 of the group's largest), away from the oracle's near-decision
Gaussians.
"""
import numpy as np
import pytest
import torch

import oracle as O
from synth import frustum_scene, random_target

from gpu_helpers import GRAD_RTOL, cuda, grad_errors, new_map, rotated_cam

pytestmark = pytest.mark.gpu

LP = 0.2


@pytest.fixture(scope="module")
def scene():
    p, cam = frustum_scene()
    tg = random_target(160, 120, seed=1)
    return p, cam, tg


def test_ssim_loss_and_gradients_match_oracle(scene):
    p, cam, tg = scene
    ref = O.loss_and_grads(p.astype(np.float64), [cam], tg, O.Config(lambda_photo=LP), flags=True)
    gm = new_map(p.shape[1], lambda_photo=LP)
    gm.set_params(cuda(p))
    gm.render(cam)
    loss = gm.loss(cuda(tg)).cpu().numpy()
    gm.backward()
    g = gm.grads().cpu().numpy()
    assert abs(loss[0] - ref["loss"]) <= 1e-5 * ref["loss"]
    assert abs(loss[2] - ref["reg"]) <= 1e-5 * ref["reg"]
    errs = grad_errors(g, ref["grad"], exclude=ref["gauss_near"])
    assert max(errs.values()) <= GRAD_RTOL, errs
    # the SSIM term changes the result: it is not the L1 gradient
    g1 = O.loss_and_grads(p.astype(np.float64), [cam], tg)["grad"]
    assert np.abs(g - g1).max() > 1e-2 * np.abs(g1).max()


def test_ssim_constant_images_closed_form():
    """An empty map renders black against a constant target: the loss equals the oracle's for the
    same two images (whose SSIM map is C1 / (c^2 + C1) away from the border, a pinned closed form)."""
    from paper_2504_02437_gb300.api import GaussianMap
    gm = GaussianMap(capacity=4, max_views=1, max_width=64, max_height=48, lambda_photo=LP)
    from synth import Camera
    cam = Camera(64, 48, 50.0, 50.0, 32.0, 24.0)
    c = 0.4
    tg = np.full((1, 3, 48, 64), c, np.float32)
    gm.render(cam)
    loss = float(gm.loss(cuda(tg)).cpu()[0])
    ref = float(O.color_loss(torch.zeros(3, 48, 64, dtype=torch.float64), torch.as_tensor(tg[0], dtype=torch.float64),
                             O.Config(lambda_photo=LP)))
    assert abs(loss - ref) <= 1e-5 * ref


def test_ssim_iterate_graph_matches_plain_steps(scene):
    """With the SSIM term the captured iteration runs forward, loss and adjoint as separate kernels;
    it follows render -> loss -> backward -> step call for call."""
    p, cam, tg = scene
    cams = [cam, rotated_cam(cam, [0.02, -0.03, 0.0], [0.03, 0.0, 0.05]), cam, cam]
    tgt = cuda(tg)
    ga, gb = new_map(p.shape[1], lambda_photo=LP), new_map(p.shape[1], lambda_photo=LP)
    ga.set_params(cuda(p))
    gb.set_params(cuda(p))
    la, lb = [], []
    loss = torch.empty(3, device="cuda")
    for c in cams:
        ga.iterate(c, tgt, loss)
        la.append(float(loss[0]))
        gb.render(c)
        lb.append(float(gb.loss(tgt)[0]))
        gb.backward()
        gb.step()
    np.testing.assert_allclose(la, lb, rtol=1e-5)
    d = np.abs(ga.params().cpu().numpy() - gb.params().cpu().numpy())
    assert np.median(d) < 1e-7
    assert (d > 1e-5).mean() < 1e-3

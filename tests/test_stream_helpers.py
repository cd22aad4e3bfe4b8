"""Host helpers of the mapping stream, on the CPU: the learned initialiser's training targets
(canonical form of converged Gaussians) and the PSNR of the time-to-PSNR protocol."""
import math

import torch

from paper_2504_02437_gb300.stream import canonical_targets, psnr


def test_canonical_targets_layout_and_quaternion_sign():
    g = torch.Generator().manual_seed(0)
    p = torch.randn(14, 50, generator=g)
    t = canonical_targets(p)
    assert t.shape == (50, 16)
    torch.testing.assert_close(t[:, 0:3], p[3:6].T)          # log-scales
    torch.testing.assert_close(t[:, 7], p[10])               # opacity logit
    torch.testing.assert_close(t[:, 8:11], p[11:14].T)       # colour
    assert torch.all(t[:, 11:] == 0)
    q = t[:, 3:7]
    torch.testing.assert_close(q.norm(dim=1), torch.ones(50))
    assert torch.all(q[:, 0] >= 0)
    # q and -q are the same rotation: both give the same target
    p2 = p.clone()
    p2[6:10] *= -1
    torch.testing.assert_close(canonical_targets(p2), t)
    # a scaled quaternion too
    p3 = p.clone()
    p3[6:10] *= 3.5
    torch.testing.assert_close(canonical_targets(p3), t)


def test_psnr_closed_forms():
    a = torch.zeros(3, 8, 8)
    b = torch.full((3, 8, 8), 0.1)
    assert abs(float(psnr(a, b)) - 20.0) < 1e-4               # MSE 0.01 -> 20 dB
    c = a.clone()
    c[0, 0, 0] = 1.0
    assert abs(float(psnr(a, c)) - 10 * math.log10(192)) < 1e-4
    assert float(psnr(a, a)) == 120.0                         # MSE floored at 1e-12

"""Oracle pins of the learned initialiser's training targets (canonical form of converged
Gaussians) and of the PSNR of the time-to-PSNR protocol, on the CPU: closed forms and
invariants (the library's versions are compared with these in tests/test_gpu_stream.py)."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

import oracle as O


def test_mlp_targets_layout_and_quaternion_sign():
    rng = np.random.default_rng(0)
    p = rng.normal(size=(14, 50))
    t = O.mlp_targets(p)
    assert t.shape == (50, 16)
    np.testing.assert_array_equal(t[:, 0:3], p[3:6].T)      # log-scales
    np.testing.assert_array_equal(t[:, 7], p[10])           # opacity logit
    np.testing.assert_array_equal(t[:, 8:11], p[11:14].T)   # colour
    assert np.all(t[:, 11:] == 0)
    q = t[:, 3:7]
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, rtol=1e-15)
    assert np.all(q[:, 0] >= 0)
    # the target quaternion is the same rotation as the parameter's (scipy takes x, y, z, w)
    Rp = Rotation.from_quat(p[[7, 8, 9, 6]].T).as_matrix()
    Rt = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    np.testing.assert_allclose(Rt, Rp, atol=1e-12)
    # q and -q, and a scaled q, give the same target
    p2 = p.copy()
    p2[6:10] *= -1
    np.testing.assert_allclose(O.mlp_targets(p2), t, rtol=1e-15)
    p3 = p.copy()
    p3[6:10] *= 3.5
    np.testing.assert_allclose(O.mlp_targets(p3), t, rtol=1e-14)
    p4 = p.copy()
    p4[6:10, 0] = 0.0
    assert np.all(O.mlp_targets(p4)[0, 3:7] == 0)


def test_psnr_closed_forms():
    a = np.zeros((3, 8, 8))
    b = np.full((3, 8, 8), 0.1)
    assert abs(O.psnr(a, b) - 20.0) < 1e-12                  # MSE 0.01 -> 20 dB
    c = a.copy()
    c[0, 0, 0] = 1.0
    assert abs(O.psnr(a, c) - 10 * math.log10(192)) < 1e-12
    assert O.psnr(a, a) == 120.0                             # MSE floored at 1e-12

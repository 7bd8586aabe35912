"""The Perlin-noise phantom of the adaptive-optics example (n = 1.36 +- 0.03):
seeded, within the stated index range, smooth and periodic like the grid."""
import numpy as np

from paper_1706_02261_b300 import inputs


def test_perlin_phantom_range_smoothness_and_seed():
    a = inputs.perlin_phantom_dn((32, 96, 96), 0.1, seed=7).astype(np.float64)
    b = inputs.perlin_phantom_dn((32, 96, 96), 0.1, seed=7).astype(np.float64)
    c = inputs.perlin_phantom_dn((32, 96, 96), 0.1, seed=8).astype(np.float64)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    n = 1.33 + a
    assert n.min() >= 1.33 - 1e-3 and n.max() <= 1.39 + 1e-3        # 1.36 +- 0.03 (FP16 rounding)
    assert abs(n.max() - 1.36) > 0.02 or abs(n.min() - 1.36) > 0.02  # the full swing is used
    assert abs(n.mean() - 1.36) < 0.01
    step = np.abs(np.diff(a, axis=2)).mean()
    wrap = np.abs(a[:, :, 0] - a[:, :, -1]).mean()
    assert step < 0.003 and wrap < 2 * step                           # smooth, and periodic across the edge

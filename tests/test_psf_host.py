"""Host logic of the PSF sweep (no GPU): the focus lattice, the intensity
windows and the depth convention (intensity slice z is recorded after slice
z, at depth (z + 1) dz)."""
import numpy as np

from paper_1706_02261_b300.psf import Sweep


def test_lattice_is_pitch_spaced_and_inside_the_grid():
    s = Sweep(n=1024, nz=1024, d=0.1625, pitch=32, depths=[100])
    ix, iy = s.lattice()
    assert s.foci_per_field == 1024
    assert ix.min() == 16 and ix.max() == 1008 and set(np.diff(np.unique(ix))) == {32}
    assert np.all((iy >= 0) & (iy < 1024))
    assert len(set(zip(ix.tolist(), iy.tolist()))) == 1024        # no two foci share a pixel


def test_windows_are_clipped_to_the_volume():
    s = Sweep(n=128, nz=100, d=0.1, pitch=32, depths=[0], patch=(16, 16, 20))
    assert s.window(50) == (40, 60)
    assert s.window(5) == (0, 15)
    assert s.window(95) == (85, 100)
    assert s.window(130) == (100, 100)         # focus beyond the volume: empty window


def test_focal_depth_convention_and_seeded_phases():
    s = Sweep(n=128, nz=64, d=0.1, pitch=64, depths=[10, 20], seed=3)
    xyz, ph, foci = s.field_inputs(1)
    assert np.allclose(xyz[:, 2], 21 * 0.1)
    assert np.array_equal(foci[:, 2], np.full(4, 20))
    assert np.allclose(xyz[:, 0], foci[:, 0] * 0.1) and np.allclose(xyz[:, 1], foci[:, 1] * 0.1)
    xyz2, ph2, _ = s.field_inputs(1)
    assert np.array_equal(ph, ph2) and not np.array_equal(ph, s.field_inputs(0)[1])

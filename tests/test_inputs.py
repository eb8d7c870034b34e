"""The seeded input generator (packed beds, uniform fields)."""
import numpy as np

from paper_1111_1129_gb300 import inputs


def test_uniform_is_deterministic_and_in_range():
    a = inputs.uniform(1000, seed=3, stream=1, lo=-2.0, hi=5.0)
    b = inputs.uniform(1000, seed=3, stream=1, lo=-2.0, hi=5.0)
    np.testing.assert_array_equal(a, b)
    assert a.min() >= -2.0 and a.max() < 5.0
    assert abs(a.mean() - 1.5) < 0.3
    assert not np.array_equal(a, inputs.uniform(1000, seed=4, stream=1, lo=-2.0, hi=5.0))


def test_small_bed_geometry():
    bed = inputs.bed_small(0)
    assert bed.flags.shape == (64, 32, 32) and bed.dims == (32, 32, 64)
    assert bed.n_fluid == int((bed.flags == 0).sum())
    assert 0.40 < bed.porosity < 0.47
    assert bed.periodic == 0b100
    # outside the tube (diameter 30, centred) every cell is solid
    y, x = np.mgrid[0:32, 0:32] + 0.5
    outside = (x - 16) ** 2 + (y - 16) ** 2 >= 15 ** 2
    assert np.all(bed.flags[:, outside] == 1)
    again = inputs.bed_small(0)
    np.testing.assert_array_equal(bed.flags, again.flags)
    assert not np.array_equal(bed.flags, inputs.bed_small(1).flags)


def test_empty_tube_is_a_channel():
    bed = inputs.packed_bed((40, 20, 20), 0, 18.0, 0.0, 0.0, 0)
    assert bed.n_spheres == 0
    assert 0.60 < bed.porosity < 0.66       # pi/4 * (18/20)^2 = 0.636


def test_alpha_field_is_ordering_independent():
    a = inputs.alpha_field((5, 6, 7), seed=2)
    assert a.shape == (7, 6, 5) and a.min() >= 0.0 and a.max() < 0.05


def test_batch_params_ranges():
    sides, radii, forces = inputs.batch_params(256, 0)
    assert sides.min() >= 24 and sides.max() <= 96
    assert radii.min() >= 3.0 and radii.max() <= 8.0
    assert forces.min() >= 1e-7 and forces.max() <= 1e-5

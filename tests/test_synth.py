"""The seeded input recipe: SU(3) links with mean plaquette 0.590."""
import numpy as np

from synth import fields as F


def test_links_are_su3():
    u = F.gauge_field((4, 4, 4, 4), 1)
    uu = np.einsum("...ij,...kj->...ik", u, u.conj())
    assert np.abs(uu - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14


def test_plaquette_calibration():
    u = F.gauge_field((12, 12, 12, 12), 7)
    assert abs(F.plaquette(u) - 0.590) < 0.003


def test_seeded_and_deterministic():
    a = F.gauge_field((2, 2, 2, 2), 3)
    b = F.gauge_field((2, 2, 2, 2), 3)
    c = F.gauge_field((2, 2, 2, 2), 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)

"""The seeded input generators (no method arithmetic): the disjoint-inclusion
recipe keeps its stated gap, radii and volume fraction."""
import numpy as np

from paper_2204_01722_b300 import inputs


def test_disjoint_inclusions_keep_gap_and_fraction():
    n, gap = 32, 2.0
    c, r, inside = inputs.inclusion_spheres(n, n, n, seed=3, gap=gap)
    h = 1.0 / n
    assert inside.mean() >= 0.3
    assert np.all(r >= 2.0 * h - 1e-15) and np.all(r <= 6.0 * h + 1e-15)
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2)
    need = r[:, None] + r[None, :] + gap * h
    off = ~np.eye(len(r), dtype=bool)
    assert np.all(d[off] >= need[off])
    E = inputs.inclusion_modulus(n, n, n, seed=3, gap=gap)
    assert np.array_equal(E > 1.0, inside) and set(np.unique(E)) == {1.0, 1e3}


def test_overlapping_inclusions_reach_fraction():
    c, r, inside = inputs.inclusion_spheres(24, 24, 24, seed=1)
    assert inside.mean() >= 0.3 and len(r) == len(c)

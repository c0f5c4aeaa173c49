"""Seeded input generators: determinism and shape (CPU only)."""
import numpy as np

import synth


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 seeded with 0 (published reference sequence)
    z = synth.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_deterministic_and_offsettable():
    a = synth.uniform(123, 1000)
    b = synth.uniform(123, 1000)
    assert np.array_equal(a, b)
    assert np.array_equal(synth.uniform(123, 10, start=990), a[990:])
    assert 0.0 <= a.min() and a.max() < 1.0


def test_normals_moments():
    z = synth.normal(7, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_sphere_and_ellipsoid_surfaces():
    p = synth.sphere(5000, 32.0, seed=1)
    assert np.allclose(np.linalg.norm(p, axis=1), 32.0)
    e = synth.ellipsoid(3000, 8.0, 4.0, 2.0, seed=2)
    assert e.shape == (3000, 3)
    assert np.allclose((e[:, 0] / 8) ** 2 + (e[:, 1] / 4) ** 2 + (e[:, 2] / 2) ** 2, 1.0)


def test_cube_clusters_split():
    p = synth.cube_surface_clusters(10000, seed=9)
    ns = 7000
    on_face = np.isclose(np.max(np.abs(p[:ns]), axis=1), 16.0)
    assert on_face.all()
    assert p.shape == (10000, 3)

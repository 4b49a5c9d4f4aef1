"""CPU checks of the seeded input generators (they hold no force arithmetic)."""
import numpy as np
import pytest

import workloads


def test_plummer_structure():
    x, v, m = workloads.plummer(20000, seed=0)
    assert x.shape == (20000, 3) and v.shape == (20000, 3)
    assert m.sum() == pytest.approx(1.0)
    np.testing.assert_allclose((m[:, None] * x).sum(0), 0.0, atol=1e-12)
    np.testing.assert_allclose((m[:, None] * v).sum(0), 0.0, atol=1e-12)
    r = np.linalg.norm(x, axis=1)
    # Half-mass radius of a Plummer sphere: b / sqrt(2^{2/3} - 1) = 1.3048 b.
    assert np.median(r) == pytest.approx(1.3048, rel=0.03)
    # Bound orbits only: |v| below the local escape speed.
    r0 = np.linalg.norm(x + (m[:, None] * x).sum(0), axis=1)
    assert np.all(np.linalg.norm(v, axis=1) < np.sqrt(2.0) * (1 + r0 * r0) ** -0.25 + 0.05)
    # Kinetic energy of the Plummer model: 3 pi / 64.
    K = 0.5 * (m * (v * v).sum(1)).sum()
    assert K == pytest.approx(3 * np.pi / 64, rel=0.05)


def test_plummer_seeded():
    a = workloads.plummer(100, seed=5)
    b = workloads.plummer(100, seed=5)
    c = workloads.plummer(100, seed=6)
    np.testing.assert_array_equal(a[0], b[0])
    assert not np.array_equal(a[0], c[0])


def test_uniform_sphere():
    x, v, m = workloads.uniform_sphere(5000, seed=1, radius=2.0)
    r = np.linalg.norm(x, axis=1)
    # Centring shifts the ball by its sample mean (about R / sqrt(N)).
    assert r.max() <= 2.0 + 0.05
    assert np.median(r) == pytest.approx(2.0 * 0.5 ** (1 / 3), rel=0.03)
    assert np.all(v == 0)


def test_clusters_layout():
    c = workloads.clusters(64, seed=0)
    assert c.offsets[0] == 0 and c.offsets[-1] == c.x.shape[0]
    assert np.all(c.sizes >= 32) and np.all(c.sizes <= 4096)
    for k in range(64):
        sl = slice(c.offsets[k], c.offsets[k + 1])
        assert c.m[sl].sum() == pytest.approx(1.0)
    np.testing.assert_allclose(c.eps, 0.02 * c.radius)
    assert set(c.kind.tolist()) == {0, 1}


def test_sample_rows_distinct():
    r = workloads.sample_rows(1 << 20, 2048, seed=2)
    assert r.size == 2048 and np.unique(r).size == 2048
    assert r.min() >= 0 and r.max() < (1 << 20)

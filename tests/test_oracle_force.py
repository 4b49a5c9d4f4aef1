"""CPU pins of the FP64 oracle for Eq. (gravity) (Section "Introduction").

The paper prints no force or potential values, so the oracle is pinned to
what the definition and mathematics fix: hand-derived two-body closed forms,
exact power-of-two scaling laws, symmetry, the momentum invariant, the
potential-gradient identity checked by finite differences, and brute force
in 40-digit arithmetic on tiny systems. A dropped term, a wrong exponent, a
wrong sign or index, or a self term left in fails at least one of these.
"""
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_body.txt")


def _golden(kind):
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] == kind:
                rows.append((tok[1], [float(t) for t in tok[2:]]))
    assert rows, kind
    return rows


@pytest.mark.parametrize("case,vals", _golden("force"))
def test_two_body_closed_form(oracle_mod, case, vals):
    x = np.array([vals[0:3], vals[3:6]])
    m = np.array(vals[6:8])
    eps = vals[8]
    a, p, _ = oracle_mod.force(x, m, eps)
    np.testing.assert_allclose(a[0], vals[9:12], rtol=1e-15, atol=1e-18)
    np.testing.assert_allclose(p[0], vals[12], rtol=1e-15)
    np.testing.assert_allclose(a[1], vals[13:16], rtol=1e-15, atol=1e-18)
    np.testing.assert_allclose(p[1], vals[16], rtol=1e-15)


def test_empty_and_single(oracle_mod):
    a, p, am = oracle_mod.force(np.zeros((0, 3)), np.zeros(0), 0.1)
    assert a.shape == (0, 3) and p.shape == (0,)
    # One particle: the sum over j != i is empty.
    a, p, am = oracle_mod.force(np.array([[0.3, -1.0, 2.0]]), np.array([5.0]), 0.1)
    assert np.all(a == 0.0) and np.all(p == 0.0) and np.all(am == 0.0)


def test_self_term_excluded_but_coincident_pair_included(oracle_mod):
    # Two distinct particles at the same point: d = 0 adds nothing to a and
    # m_j / eps to p. The j == i term is skipped (p would double otherwise).
    x = np.array([[1.5, 1.5, 1.5], [1.5, 1.5, 1.5]])
    m = np.array([2.0, 3.0])
    eps = 0.5
    a, p, _ = oracle_mod.force(x, m, eps)
    assert np.all(a == 0.0)
    np.testing.assert_array_equal(p, [3.0 / 0.5, 2.0 / 0.5])


def test_cube_centre_symmetry(oracle_mod):
    # Eight unit masses at (+-1, +-1, +-1) around a probe at the origin,
    # eps = 1: every s = 3 + 1 = 4, so p_probe = 8 / 2 = 4 and the probe's a
    # cancels exactly (all partial sums are multiples of 1/8).
    verts = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float)
    x = np.vstack([[0.0, 0.0, 0.0], verts])
    m = np.ones(9)
    a, p, _ = oracle_mod.force(x, m, 1.0)
    assert np.all(a[0] == 0.0)
    assert p[0] == 4.0
    # Each vertex is pushed (literal sign of Eq. (gravity): away from the
    # masses) radially outwards, by symmetry.
    for k in range(1, 9):
        cosang = a[k] @ verts[k - 1] / (np.linalg.norm(a[k]) * np.linalg.norm(verts[k - 1]))
        assert cosang == pytest.approx(1.0, abs=1e-14)


def _rand_system(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 3))
    m = rng.uniform(0.1, 2.0, n)
    return x, m


def test_power_of_two_scaling_is_exact(oracle_mod):
    # x -> 2x, eps -> 2 eps gives s -> 4 s, so a -> a / 4 and p -> p / 2 in
    # every rounded operation: the results must agree bit for bit. A wrong
    # exponent (s^{-1} or s^{-2} in a, s^{-1} in p) breaks this.
    x, m = _rand_system(37, 1)
    eps = 0.125
    a1, p1, _ = oracle_mod.force(x, m, eps)
    a2, p2, _ = oracle_mod.force(2.0 * x, m, 2.0 * eps)
    np.testing.assert_array_equal(a2, a1 / 4.0)
    np.testing.assert_array_equal(p2, p1 / 2.0)
    # Masses enter linearly as m_j (not m_i): doubling them doubles both sums.
    a3, p3, _ = oracle_mod.force(x, 2.0 * m, eps)
    np.testing.assert_array_equal(a3, 2.0 * a1)
    np.testing.assert_array_equal(p3, 2.0 * p1)
    # Parity: x -> -x flips a, keeps p.
    a4, p4, _ = oracle_mod.force(-x, m, eps)
    np.testing.assert_array_equal(a4, -a1)
    np.testing.assert_array_equal(p4, p1)


def test_integer_translation_is_exact(oracle_mod):
    # Integer coordinates shifted by an integer vector keep every x_i - x_j
    # exact, so the sums are unchanged bit for bit.
    rng = np.random.default_rng(4)
    x = rng.integers(-20, 20, size=(25, 3)).astype(float)
    m = rng.integers(1, 5, size=25).astype(float)
    a1, p1, _ = oracle_mod.force(x, m, 0.5)
    a2, p2, _ = oracle_mod.force(x + np.array([1024.0, -77.0, 3.0]), m, 0.5)
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(p1, p2)


def test_mass_selects_source_not_target(oracle_mod):
    # Changing m_k must leave a_k and p_k unchanged (only m_j, j != i, enters
    # row i), and change every other row.
    x, m = _rand_system(9, 5)
    a1, p1, _ = oracle_mod.force(x, m, 0.3)
    m2 = m.copy()
    m2[4] *= 3.0
    a2, p2, _ = oracle_mod.force(x, m2, 0.3)
    np.testing.assert_array_equal(a1[4], a2[4])
    assert p1[4] == p2[4]
    others = [k for k in range(9) if k != 4]
    assert np.all(p2[others] > p1[others])


def test_permutation_equivariance(oracle_mod):
    x, m = _rand_system(40, 6)
    perm = np.random.default_rng(7).permutation(40)
    a1, p1, _ = oracle_mod.force(x, m, 0.2)
    a2, p2, _ = oracle_mod.force(x[perm], m[perm], 0.2)
    np.testing.assert_allclose(a2, a1[perm], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(p2, p1[perm], rtol=1e-14)


def test_rotation_equivariance(oracle_mod):
    # Eq. (gravity) depends on positions only through x_i - x_j and |x_i - x_j|:
    # rotating the system rotates every a_i and leaves every p_i unchanged
    # (FP64 rounding aside). A component taken from the wrong axis fails this.
    x, m = _rand_system(40, 9)
    q, r = np.linalg.qr(np.random.default_rng(11).normal(size=(3, 3)))
    rot = q * np.sign(np.diag(r))  # a random orthogonal matrix
    a1, p1, amag = oracle_mod.force(x, m, 0.1)
    a2, p2, _ = oracle_mod.force(x @ rot.T, m, 0.1)
    err_a = np.linalg.norm(a2 - a1 @ rot.T, axis=1) / amag
    assert err_a.max() <= 1e-13
    np.testing.assert_allclose(p2, p1, rtol=1e-13)


def test_momentum_invariant(oracle_mod):
    # Pairs are antisymmetric: sum_i m_i a_i = 0 up to FP64 rounding.
    x, v, m = workloads.plummer(300, seed=3)
    a, p, amag = oracle_mod.force(x, m, 0.05)
    total = (m[:, None] * a).sum(0)
    scale = (m * amag).sum()
    assert np.all(np.abs(total) <= 1e-13 * scale)


def test_potential_pair_symmetry(oracle_mod):
    # sum_i m_i p_i counts every unordered pair twice: 2 sum_{i<j} m_i m_j s^{-1/2}.
    x, m = _rand_system(30, 8)
    eps = float(np.float32(0.07))  # the oracle takes eps in FP32, like the kernel
    _, p, _ = oracle_mod.force(x, m, eps)
    pair = 0.0
    for i in range(30):
        for j in range(i + 1, 30):
            d = x[i] - x[j]
            pair += m[i] * m[j] / np.sqrt(d @ d + eps * eps)
    assert (m * p).sum() == pytest.approx(2.0 * pair, rel=1e-13)


def test_acceleration_is_potential_gradient(oracle_mod):
    # With W = -1/2 sum_i m_i p_i the physical force on k is -dW/dx_k and
    # equals -m_k a_k, i.e. a_k = (1/m_k) dW/dx_k. Central differences of the
    # oracle's own p pin the exponent and sign of a independently of its a code.
    x, m = _rand_system(7, 9)
    eps = float(np.float32(0.3))
    a, _, _ = oracle_mod.force(x, m, eps)

    def W(xx):
        _, pp, _ = oracle_mod.force(xx, m, eps)
        return -0.5 * (m * pp).sum()

    h = 1e-5
    for k in range(7):
        for c in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            dW = (W(xp) - W(xm)) / (2 * h)
            assert a[k, c] == pytest.approx(dW / m[k], rel=1e-7, abs=1e-9)


def test_brute_force_high_precision(oracle_mod):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x, m = _rand_system(8, 10)
    eps = np.float32(0.0625)
    a, p, amag = oracle_mod.force(x, m, eps)
    e2 = mp.mpf(float(eps)) ** 2
    for i in range(8):
        acc = [mp.mpf(0)] * 3
        pot = mp.mpf(0)
        for j in range(8):
            if j == i:
                continue
            d = [mp.mpf(float(x[i, c])) - mp.mpf(float(x[j, c])) for c in range(3)]
            s = d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + e2
            acc = [acc[c] + mp.mpf(float(m[j])) * d[c] / s ** mp.mpf(1.5) for c in range(3)]
            pot += mp.mpf(float(m[j])) / mp.sqrt(s)
        for c in range(3):
            assert float(acc[c]) == pytest.approx(a[i, c], rel=1e-14, abs=1e-15)
        assert float(pot) == pytest.approx(p[i], rel=1e-15)


def test_rows_match_full(oracle_mod):
    x, v, m = workloads.plummer(500, seed=11)
    a, p, am = oracle_mod.force(x, m, 0.01)
    rows = workloads.sample_rows(500, 37, seed=2)
    ar, pr, amr = oracle_mod.force_rows(x, m, 0.01, rows)
    np.testing.assert_array_equal(ar, a[rows])
    np.testing.assert_array_equal(pr, p[rows])
    np.testing.assert_array_equal(amr, am[rows])


def test_plummer_potential_statistics(oracle_mod):
    # For a Plummer sphere (G = M = b = 1) the potential at radius r is
    # 1/sqrt(r^2 + 1) and the potential energy is -3 pi / 32. With N = 4096
    # particles and eps = 0.01 both hold to a few percent.
    x, v, m = workloads.plummer(4096, seed=0)
    x32 = x.astype(np.float32)
    m32 = m.astype(np.float32)
    _, p, _ = oracle_mod.force(x32, m32, 0.01)
    W = -0.5 * (m32.astype(float) * p).sum()
    assert W == pytest.approx(-3 * np.pi / 32, rel=0.05)
    r = np.linalg.norm(x32.astype(float), axis=1)
    assert np.median(np.abs(p - 1.0 / np.sqrt(r * r + 1.0))) < 0.03

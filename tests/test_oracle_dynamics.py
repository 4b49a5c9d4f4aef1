"""CPU pins of the FP64 oracle's gradient (chain rule of Eq. (gravity)),
leap-frog integrator (Section "Method", Eqs. (1)-(3)) and energy.

Gradient: hand-derived two-body closed form, central finite differences of
the oracle's force (a separate code path), the dot-product test and
linearity in the upstream gradients.
Integrator: free particle, exact time reversibility of the symmetric
scheme, momentum conservation, second-order energy error (halving dt quarters
it) and a two-body circular orbit.
"""
import os

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_body.txt")


def _golden(kind):
    out = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] == kind:
                out.append((tok[1], [float(t) for t in tok[2:]]))
    return out


def _rand_system(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 3)), rng.uniform(0.1, 2.0, n)


@pytest.mark.parametrize("case,vals", _golden("vjp_p"))
def test_vjp_two_body_closed_form(oracle_mod, case, vals):
    x = np.array([vals[0:3], vals[3:6]])
    m = np.array(vals[6:8])
    eps = vals[8]
    gx, gm = oracle_mod.force_vjp(x, m, eps, np.zeros((2, 3)), np.ones(2))
    np.testing.assert_allclose(gx[0], vals[9:12], rtol=1e-15)
    assert gm[0] == pytest.approx(vals[12], rel=1e-15)
    np.testing.assert_allclose(gx[1], vals[13:16], rtol=1e-15)
    assert gm[1] == pytest.approx(vals[16], rel=1e-15)


def _loss(oracle_mod, x, m, eps, ga, gp):
    a, p, _ = oracle_mod.force(x, m, eps)
    return float((ga * a).sum() + (gp * p).sum())


def test_vjp_matches_central_differences(oracle_mod):
    n = 9
    x, m = _rand_system(n, 21)
    rng = np.random.default_rng(22)
    ga = rng.normal(size=(n, 3))
    gp = rng.normal(size=n)
    eps = float(np.float32(0.25))
    gx, gm = oracle_mod.force_vjp(x, m, eps, ga, gp)
    h = 1e-6
    for k in range(n):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            fd = (_loss(oracle_mod, xp, m, eps, ga, gp) - _loss(oracle_mod, xm, m, eps, ga, gp)) / (2 * h)
            assert gx[k, c] == pytest.approx(fd, rel=1e-6, abs=1e-7)
        mp_, mm_ = m.copy(), m.copy()
        mp_[k] += h
        mm_[k] -= h
        fd = (_loss(oracle_mod, x, mp_, eps, ga, gp) - _loss(oracle_mod, x, mm_, eps, ga, gp)) / (2 * h)
        assert gm[k] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_vjp_dot_product(oracle_mod):
    # <J dtheta, (ga, gp)> = <dtheta, J^T (ga, gp)> with J dtheta by a
    # central difference along a random direction in (x, m).
    n = 40
    x, v, m = workloads.plummer(n, seed=23)
    rng = np.random.default_rng(24)
    ga = rng.normal(size=(n, 3))
    gp = rng.normal(size=n)
    dx = rng.normal(size=(n, 3))
    dm = rng.normal(size=n) * 1e-3
    eps = float(np.float32(0.05))
    gx, gm = oracle_mod.force_vjp(x, m, eps, ga, gp)
    h = 1e-6
    lp = _loss(oracle_mod, x + h * dx, m + h * dm, eps, ga, gp)
    lm = _loss(oracle_mod, x - h * dx, m - h * dm, eps, ga, gp)
    jvp = (lp - lm) / (2 * h)
    assert (gx * dx).sum() + (gm * dm).sum() == pytest.approx(jvp, rel=1e-6)


def test_vjp_linear_in_upstream(oracle_mod):
    n = 15
    x, m = _rand_system(n, 25)
    rng = np.random.default_rng(26)
    ga1, gp1 = rng.normal(size=(n, 3)), rng.normal(size=n)
    ga2, gp2 = rng.normal(size=(n, 3)), rng.normal(size=n)
    g1 = oracle_mod.force_vjp(x, m, 0.1, ga1, gp1)
    g2 = oracle_mod.force_vjp(x, m, 0.1, ga2, gp2)
    g12 = oracle_mod.force_vjp(x, m, 0.1, ga1 + ga2, gp1 + gp2)
    np.testing.assert_allclose(g12[0], g1[0] + g2[0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g12[1], g1[1] + g2[1], rtol=1e-12, atol=1e-12)


def test_vjp_rows_match_full(oracle_mod):
    n = 50
    x, m = _rand_system(n, 27)
    rng = np.random.default_rng(28)
    ga, gp = rng.normal(size=(n, 3)), rng.normal(size=n)
    gx, gm = oracle_mod.force_vjp(x, m, 0.1, ga, gp)
    rows = np.array([0, 7, 49, 3])
    gxr, gmr = oracle_mod.force_vjp(x, m, 0.1, ga, gp, rows=rows)
    np.testing.assert_array_equal(gxr, gx[rows])
    np.testing.assert_array_equal(gmr, gm[rows])


@pytest.mark.parametrize("case,vals", _golden("energy"))
def test_energy_two_body_closed_form(oracle_mod, case, vals):
    x = np.array([vals[0:3], vals[3:6]])
    v = np.array([vals[6:9], vals[9:12]])
    m = np.array(vals[12:14])
    K, W = oracle_mod.energy(x, v, m, vals[14])
    assert K == pytest.approx(vals[15], rel=1e-15)
    assert W == pytest.approx(vals[16], rel=1e-15)


def test_leapfrog_free_particle(oracle_mod):
    x = np.array([[0.5, -1.0, 2.0]])
    v = np.array([[0.25, 0.5, -0.125]])
    x1, v1, g = oracle_mod.leapfrog(x, v, np.array([1.0]), 0.1, 0.0625, 16)
    np.testing.assert_array_equal(v1, v)
    np.testing.assert_allclose(x1, x + v * 1.0, rtol=0, atol=1e-15)
    assert np.all(g == 0.0)


def test_leapfrog_time_reversible(oracle_mod):
    # The scheme is symmetric: stepping back with the velocities reversed
    # returns to the start up to rounding. A missing 1/2 or a sign error in
    # either kick breaks this at O(dt).
    x, v, m = workloads.plummer(64, seed=31)
    eps = float(np.float32(0.05))
    x1, v1, _ = oracle_mod.leapfrog(x, v, m, eps, 0.01, 20)
    x2, v2, _ = oracle_mod.leapfrog(x1, -v1, m, eps, 0.01, 20)
    np.testing.assert_allclose(x2, x, rtol=0, atol=1e-11)
    np.testing.assert_allclose(-v2, v, rtol=0, atol=1e-11)


def test_leapfrog_momentum_conserved(oracle_mod):
    x, v, m = workloads.plummer(64, seed=32)
    P0 = (m[:, None] * v).sum(0)
    x1, v1, _ = oracle_mod.leapfrog(x, v, m, 0.05, 0.01, 30)
    P1 = (m[:, None] * v1).sum(0)
    np.testing.assert_allclose(P1, P0, rtol=0, atol=1e-13)


def test_leapfrog_energy_error_second_order(oracle_mod):
    # Energy error of a second-order scheme over a fixed time span scales
    # as dt^2: halving dt divides it by about 4.
    x, v, m = workloads.plummer(128, seed=33)
    eps = float(np.float32(0.1))
    E0 = sum(oracle_mod.energy(x, v, m, eps))
    errs = []
    for dt, steps in ((0.02, 25), (0.01, 50)):
        x1, v1, _ = oracle_mod.leapfrog(x, v, m, eps, dt, steps)
        errs.append(abs(sum(oracle_mod.energy(x1, v1, m, eps)) - E0))
    ratio = errs[0] / errs[1]
    assert 2.5 < ratio < 6.0, ratio


def test_leapfrog_circular_two_body(oracle_mod):
    # Two masses 0.5 at separation d = 1 on a circular orbit of the softened
    # force: relative acceleration M d / (d^2 + eps^2)^{3/2} = v_rel^2 / d.
    # After one period the separation stays 1 and the bodies return.
    eps = float(np.float32(0.0625))
    M, d = 1.0, 1.0
    vrel = np.sqrt(M * d * d / (d * d + eps * eps) ** 1.5)
    x = np.array([[-0.5, 0.0, 0.0], [0.5, 0.0, 0.0]])
    v = np.array([[0.0, -0.5 * vrel, 0.0], [0.0, 0.5 * vrel, 0.0]])
    m = np.array([0.5, 0.5])
    period = 2 * np.pi * d / vrel
    steps = 2000
    x1, v1, _ = oracle_mod.leapfrog(x, v, m, eps, period / steps, steps)
    sep = np.linalg.norm(x1[0] - x1[1])
    assert sep == pytest.approx(1.0, abs=1e-5)
    np.testing.assert_allclose(x1, x, atol=2e-4)


def test_leapfrog_grad_matches_central_differences(oracle_mod):
    # The reverse-mode trajectory gradient against central differences of the
    # forward integrator, for every coordinate of x0, v0 and m.
    n, eps, dt, steps = 12, float(np.float32(0.1)), 0.02, 10
    x0, v0, m = workloads.plummer(n, seed=41)
    y = workloads.targets(x0, seed=42)

    def L(xx, vv, mm):
        xT, vT, _ = oracle_mod.leapfrog(xx, vv, mm, eps, dt, steps)
        return float(((xT - y) ** 2).sum() + 0.5 * (vT ** 2).sum())

    xT, vT, _ = oracle_mod.leapfrog(x0, v0, m, eps, dt, steps)
    gx, gv, gm = oracle_mod.leapfrog_grad(x0, v0, m, eps, dt, steps, 2 * (xT - y), vT)
    for arr, grad, hs in ((x0, gx, 1e-5), (v0, gv, 1e-5)):
        for i in range(n):
            for c in range(3):
                p_, q_ = arr.copy(), arr.copy()
                p_[i, c] += hs
                q_[i, c] -= hs
                if arr is x0:
                    fd = (L(p_, v0, m) - L(q_, v0, m)) / (2 * hs)
                else:
                    fd = (L(x0, p_, m) - L(x0, q_, m)) / (2 * hs)
                assert grad[i, c] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    for i in range(n):
        h = 1e-3 * m[i]
        p_, q_ = m.copy(), m.copy()
        p_[i] += h
        q_[i] -= h
        fd = (L(x0, v0, p_) - L(x0, v0, q_)) / (2 * h)
        assert gm[i] == pytest.approx(fd, rel=1e-6, abs=1e-8)

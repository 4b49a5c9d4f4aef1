"""GPU checks of the adjoint: nb_force_vjp against the oracle's VJP, the
autograd Function, and gradients of a leap-frog trajectory loss (Section
"Method", Eqs. (1)-(3)) against FP64 finite differences of the oracle's
trajectory.

VJP error measure: per particle, |g_gpu - g_ref| divided by the sum of the
magnitudes of that particle's terms (the analogue of A_i for the force; the
sums cancel strongly, so |g_ref| itself is no scale); tolerance 1e-5.
"""
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_3659_gb300 import build
    build.build()
    import paper_0904_3659_gb300 as nbmod
    return nbmod


@pytest.fixture(scope="module")
def ctx(nb):
    c = nb.Context(0)
    yield c
    c.close()


def gpu_vjp(nb, ctx, x32, m32, eps, ga, gp):
    import torch
    dev = torch.device("cuda:0")
    n = x32.shape[0]
    t = lambda arr: torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32)).to(dev)
    gx = torch.full((n, 3), float("nan"), device=dev)
    gm = torch.full((n,), float("nan"), device=dev)
    nb.nb_force_vjp(ctx, t(x32), t(m32), n, eps, t(ga), t(gp), gx, gm)
    nb.nb_synchronize(ctx)
    return gx.cpu().numpy(), gm.cpu().numpy()


def vjp_term_scales(x, m, eps, ga, gp, chunk=512):
    """Per particle k, the sums over l != k of the magnitudes of the terms of
    gx_k and gm_k (r = x_k - x_l, s = |r|^2 + eps^2, y = s^-1/2):
      Gx_k = sum m_l (y^3 |ga_k| + 3 y^5 |r.ga_k| |r| + |gp_k| y^3 |r|)
           + m_k (y^3 |ga_l| + 3 y^5 |r.ga_l| |r| + |gp_l| y^3 |r|)
      Gm_k = sum |r.ga_l| y^3 + |gp_l| y"""
    x = np.asarray(x, np.float64)
    m = np.asarray(m, np.float64)
    ga = np.asarray(ga, np.float64)
    gp = np.asarray(gp, np.float64)
    n = x.shape[0]
    e2 = float(np.float32(eps)) ** 2
    gx_s = np.zeros(n)
    gm_s = np.zeros(n)
    nga = np.linalg.norm(ga, axis=1)
    for k0 in range(0, n, chunk):
        k1 = min(n, k0 + chunk)
        r = x[k0:k1, None, :] - x[None, :, :]
        r2 = (r * r).sum(-1)
        y = 1.0 / np.sqrt(r2 + e2)
        idx = np.arange(k0, k1)
        y[idx - k0, idx] = 0.0                       # j != i
        y3, y5, rn = y ** 3, y ** 5, np.sqrt(r2)
        rgk = np.abs((r * ga[k0:k1, None, :]).sum(-1))
        rgl = np.abs((r * ga[None, :, :]).sum(-1))
        gx_s[k0:k1] = (m[None, :] * (y3 * nga[k0:k1, None] + 3 * y5 * rgk * rn
                                     + np.abs(gp[k0:k1, None]) * y3 * rn)).sum(1)
        gx_s[k0:k1] += m[k0:k1] * (y3 * nga[None, :] + 3 * y5 * rgl * rn
                                   + np.abs(gp[None, :]) * y3 * rn).sum(1)
        gm_s[k0:k1] = (rgl * y3 + np.abs(gp[None, :]) * y).sum(1)
    return gx_s, gm_s


def rel_to_scale(g, ref, scale):
    d = np.linalg.norm(np.atleast_2d((np.asarray(g, np.float64) - ref).T).T, axis=-1)
    return float(np.max(d / scale))


@pytest.mark.parametrize("n", [1, 2, 33, 700, 3001, 8192])
def test_vjp_matches_oracle(nb, ctx, oracle_mod, n):
    x, _, m = workloads.plummer(n, seed=n)
    x32, m32 = x.astype(np.float32), m.astype(np.float32)
    rng = np.random.default_rng(n + 1)
    ga = rng.normal(size=(n, 3)).astype(np.float32)
    gp = rng.normal(size=n).astype(np.float32)
    eps = np.float32(1.0 / 64)
    gx, gm = gpu_vjp(nb, ctx, x32, m32, eps, ga, gp)
    rgx, rgm = oracle_mod.force_vjp(x32, m32, eps, ga, gp)
    assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gm))
    if n == 1:
        assert np.all(gx == 0) and np.all(gm == 0)
        return
    sx, sm = vjp_term_scales(x32, m32, eps, ga, gp)
    assert rel_to_scale(gx, rgx, sx) <= 1e-5
    assert rel_to_scale(gm, rgm, sm) <= 1e-5


def test_every_vjp_shape(nb, ctx, oracle_mod):
    # Each compiled VJP shape at a size that spans several i-blocks and
    # j-tiles with a ragged tail, against the FP64 oracle; each repeats bitwise.
    n = 3001
    x, _, m = workloads.plummer(n, seed=61)
    x32, m32 = x.astype(np.float32), m.astype(np.float32)
    rng = np.random.default_rng(62)
    ga = rng.normal(size=(n, 3)).astype(np.float32)
    gp = rng.normal(size=n).astype(np.float32)
    eps = np.float32(1.0 / 64)
    rgx, rgm = oracle_mod.force_vjp(x32, m32, eps, ga, gp)
    sx, sm = vjp_term_scales(x32, m32, eps, ga, gp)
    tiles = nb.nb_list_vjp_tiles()
    assert len(tiles) >= 2
    with pytest.raises(nb.NBError) as e:  # not a compiled shape
        nb.nb_set_vjp_tile(ctx, (96, 2, 100, 3, 2, 1, 0, 0, 63, 0, 0))
    assert e.value.status == nb.NB_ERR_ARG
    try:
        for t in tiles:
            nb.nb_set_vjp_tile(ctx, t)
            assert nb.nb_get_vjp_tile(ctx, n).as_tuple() == t.as_tuple()
            gx, gm = gpu_vjp(nb, ctx, x32, m32, eps, ga, gp)
            gx2, gm2 = gpu_vjp(nb, ctx, x32, m32, eps, ga, gp)
            assert gx.tobytes() == gx2.tobytes() and gm.tobytes() == gm2.tobytes(), t
            assert rel_to_scale(gx, rgx, sx) <= 1e-5, t
            assert rel_to_scale(gm, rgm, sm) <= 1e-5, t
    finally:
        nb.nb_set_vjp_tile(ctx, None)


@pytest.mark.parametrize("release", [0, 1])
def test_vjp_bounded_wait_reports_timeout_and_context_survives(nb, ctx, oracle_mod, release):
    # The adjoint kernel's producer skips the copy of one work unit, so the
    # consumers' bounded wait (0.2 s) runs out; the kernel records a timeout
    # and returns, nb_synchronize reports it, and the next call on the same
    # context is correct. Both stage-release schemes (a barrier per tile; the
    # last warp out of a stage refills it).
    n = 4096
    x, _, m = workloads.plummer(n, seed=81)
    x32, m32 = x.astype(np.float32), m.astype(np.float32)
    rng = np.random.default_rng(82)
    ga = rng.normal(size=(n, 3)).astype(np.float32)
    gp = rng.normal(size=n).astype(np.float32)
    eps = np.float32(1.0 / 64)
    tile = [t for t in nb.nb_list_vjp_tiles() if t.release == release][0]
    nb.nb_set_vjp_tile(ctx, tile)
    try:
        nb.nb_debug_set_fault(ctx, 3, 200_000_000)
        try:
            import torch
            dev = torch.device("cuda:0")
            t = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).to(dev)
            gx = torch.empty((n, 3), device=dev)
            gm = torch.empty(n, device=dev)
            nb.nb_force_vjp(ctx, t(x32), t(m32), n, eps, t(ga), t(gp), gx, gm)
            with pytest.raises(nb.NBError) as e:
                nb.nb_synchronize(ctx)
            assert e.value.status == nb.NB_ERR_TIMEOUT
        finally:
            nb.nb_debug_set_fault(ctx, -1, 0)
        gx, gm = gpu_vjp(nb, ctx, x32, m32, eps, ga, gp)
    finally:
        nb.nb_set_vjp_tile(ctx, None)
    rgx, rgm = oracle_mod.force_vjp(x32, m32, eps, ga, gp)
    sx, sm = vjp_term_scales(x32, m32, eps, ga, gp)
    assert rel_to_scale(gx, rgx, sx) <= 1e-5
    assert rel_to_scale(gm, rgm, sm) <= 1e-5


def test_vjp_without_potential_gradient(nb, ctx, oracle_mod):
    # gp = NULL (no upstream gradient on p) runs the kernel without the p
    # terms: it must match the oracle with gp = 0, for every compiled shape.
    import torch
    n = 2500
    x, _, m = workloads.plummer(n, seed=71)
    x32, m32 = x.astype(np.float32), m.astype(np.float32)
    ga = np.random.default_rng(72).normal(size=(n, 3)).astype(np.float32)
    gp0 = np.zeros(n, np.float32)
    eps = np.float32(1.0 / 64)
    rgx, rgm = oracle_mod.force_vjp(x32, m32, eps, ga, gp0)
    sx, sm = vjp_term_scales(x32, m32, eps, ga, gp0)
    dev = torch.device("cuda:0")
    xt, mt = torch.from_numpy(x32).to(dev), torch.from_numpy(m32).to(dev)
    gat = torch.from_numpy(ga).to(dev)
    try:
        for t in nb.nb_list_vjp_tiles():
            nb.nb_set_vjp_tile(ctx, t)
            gx = torch.full((n, 3), float("nan"), device=dev)
            gm = torch.full((n,), float("nan"), device=dev)
            nb.nb_force_vjp(ctx, xt, mt, n, eps, gat, None, gx, gm)
            nb.nb_synchronize(ctx)
            assert rel_to_scale(gx.cpu().numpy(), rgx, sx) <= 1e-5, t
            assert rel_to_scale(gm.cpu().numpy(), rgm, sm) <= 1e-5, t
    finally:
        nb.nb_set_vjp_tile(ctx, None)


def test_vjp_repeatable_and_dot_product(nb, ctx, oracle_mod):
    # Bit-reproducible; and <J dtheta, w> = <dtheta, J^T w> with J dtheta from
    # a central FP64 difference of the oracle's forward.
    n = 2000
    x, _, m = workloads.plummer(n, seed=9)
    x32, m32 = x.astype(np.float32), m.astype(np.float32)
    rng = np.random.default_rng(10)
    ga = rng.normal(size=(n, 3)).astype(np.float32)
    gp = rng.normal(size=n).astype(np.float32)
    eps = np.float32(0.02)
    gx, gm = gpu_vjp(nb, ctx, x32, m32, eps, ga, gp)
    gx2, gm2 = gpu_vjp(nb, ctx, x32, m32, eps, ga, gp)
    assert gx.tobytes() == gx2.tobytes() and gm.tobytes() == gm2.tobytes()
    dx = rng.normal(size=(n, 3))
    dm = rng.normal(size=n) * 1e-4
    h = 1e-6

    def L(xx, mm):
        a, p, _ = oracle_mod.force(xx, mm, eps)
        return float((ga * a).sum() + (gp * p).sum())

    x64, m64 = x32.astype(np.float64), m32.astype(np.float64)
    jvp = (L(x64 + h * dx, m64 + h * dm) - L(x64 - h * dx, m64 - h * dm)) / (2 * h)
    vjp = float((gx.astype(np.float64) * dx).sum() + (gm.astype(np.float64) * dm).sum())
    assert vjp == pytest.approx(jvp, rel=1e-4)


def test_autograd_function_matches_kernel(nb, ctx):
    import torch
    from paper_0904_3659_gb300.autograd import NBForce
    n = 1500
    x, _, m = workloads.plummer(n, seed=11)
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x.astype(np.float32)).to(dev).requires_grad_(True)
    mt = torch.from_numpy(m.astype(np.float32)).to(dev).requires_grad_(True)
    rng = np.random.default_rng(12)
    ga = torch.from_numpy(rng.normal(size=(n, 3)).astype(np.float32)).to(dev)
    gp = torch.from_numpy(rng.normal(size=n).astype(np.float32)).to(dev)
    a, p = NBForce.apply(xt, mt, 0.02, 0, ctx)
    ((a * ga).sum() + (p * gp).sum()).backward()
    gx, gm = gpu_vjp(nb, ctx, x.astype(np.float32), m.astype(np.float32), np.float32(0.02),
                     ga.cpu().numpy(), gp.cpu().numpy())
    assert xt.grad.cpu().numpy().tobytes() == gx.tobytes()
    assert mt.grad.cpu().numpy().tobytes() == gm.tobytes()


def _trajectory_grad_check(nb, ctx, oracle_mod, n, eps, dt, steps, ncoords, seed, mode=0):
    """Gradients of L = sum |x(T) - y|^2 through `steps` KDK steps with
    checkpoints every 8 steps, from the adjoint kernel, against (1) the FP64
    reverse-mode adjoint of the oracle's trajectory for every coordinate and
    (2) central FP64 finite differences of the oracle's trajectory for
    `ncoords` random coordinates (1e-4 relative). Steps: 1e-5 for x and v, 1e-2 m_i for a
    mass: L sums over all particles (~120 at N = 16384) while dL/dm_i can be ~1e-3, so a
    central difference loses about eps_64 L / h; measured against the exact FP64 adjoint,
    h = 1e-3 m_i left 4e-4 relative error on such a coordinate, h = 1e-2 m_i 3e-5."""
    import torch
    from paper_0904_3659_gb300.autograd import leapfrog
    dev = torch.device("cuda:0")
    x0, v0, m = workloads.plummer(n, seed=seed)
    m = m.astype(np.float32).astype(np.float64)
    y = workloads.targets(x0, seed=1)
    xt = torch.from_numpy(x0.copy()).to(dev).requires_grad_(True)
    vt = torch.from_numpy(v0.copy()).to(dev).requires_grad_(True)
    mt = torch.from_numpy(m.astype(np.float32)).to(dev).requires_grad_(True)
    yt = torch.from_numpy(y).to(dev)
    xT, _ = leapfrog(xt, vt, mt, eps, dt, steps, checkpoint_every=8, mode=mode, nbctx=ctx)
    loss = ((xT - yt) ** 2).sum()
    loss.backward()
    grads = {"x": xt.grad.cpu().numpy(), "v": vt.grad.cpu().numpy(),
             "m": mt.grad.cpu().numpy().astype(np.float64)}

    xT64, _, _ = oracle_mod.leapfrog(x0, v0, m, eps, dt, steps)
    sweep = []  # operands of every force VJP of the oracle's reverse sweep
    ref = dict(zip("xvm", oracle_mod.leapfrog_grad(x0, v0, m, eps, dt, steps, 2 * (xT64 - y),
                                                   on_vjp=lambda xs, ga: sweep.append((xs, ga)))))
    # Every coordinate, relative to max(|ref|, 1e-3 max |ref|), within 1e-4.
    # A mass gradient dL/dm_k = sum over the sweep's VJPs of
    # sum_l -(r_kl . ga_l) s_kl^{-3/2} can cancel to far below its terms; its
    # FP32 rounding error is then set by the size of those terms, not by the
    # result. A mass coordinate beyond 1e-4 is accepted only if its error is
    # within 1e-5 of that magnitude, M_k = sum over the VJPs and l of
    # |r_kl . ga_l| s_kl^{-3/2} (the scale the VJP kernel's own check uses).
    e2 = float(np.float32(eps)) ** 2
    for kind in "xvm":
        r = ref[kind]
        rel = np.abs(grads[kind] - r) / np.maximum(np.abs(r), 1e-3 * np.abs(r).max())
        k = int(np.argmax(rel))
        print(f"{kind}: every-coordinate max {rel.max():.3e} at flat index {k} "
              f"(ref {r.flat[k]:.3e}, gpu {grads[kind].flat[k]:.3e}), p99.9 {np.percentile(rel, 99.9):.3e}")
        if kind != "m":
            assert rel.max() <= 1e-4, (kind, rel.max())
            continue
        for k in np.flatnonzero(rel > 1e-4):
            M = 0.0
            for xs, ga in sweep:
                d = xs[k] - xs
                s2 = (d * d).sum(1) + e2
                term = np.abs((d * ga).sum(1)) * s2 ** -1.5
                term[k] = 0.0
                M += term.sum()
            cond = abs(grads["m"][k] - r[k]) / M
            print(f"m[{k}]: {rel[k]:.3e} relative, {cond:.3e} of its term magnitude {M:.3e} "
                  f"(|dL/dm| = {abs(r[k]):.3e})")
            assert cond <= 1e-5, (k, rel[k], cond)

    def L(xx, vv, mm):
        xT_, _, _ = oracle_mod.leapfrog(xx, vv, mm, eps, dt, steps)
        return float(((xT_ - y) ** 2).sum())

    rng = np.random.default_rng(3)
    worst = 0.0
    for k in range(ncoords):
        kind = ["x", "v", "m"][k % 3]
        if kind == "m":
            i = int(rng.integers(n))
            h = 1e-2 * float(m[i])
            mp_, mm_ = m.copy(), m.copy()
            mp_[i] += h
            mm_[i] -= h
            fd = (L(x0, v0, mp_) - L(x0, v0, mm_)) / (2 * h)
            g = float(grads["m"][i])
        else:
            i, c = int(rng.integers(n)), int(rng.integers(3))
            h = 1e-5
            base = x0 if kind == "x" else v0
            bp, bm = base.copy(), base.copy()
            bp[i, c] += h
            bm[i, c] -= h
            if kind == "x":
                fd = (L(bp, v0, m) - L(bm, v0, m)) / (2 * h)
            else:
                fd = (L(x0, bp, m) - L(x0, bm, m)) / (2 * h)
            g = float(grads[kind][i, c])
        scale = max(abs(fd), 1e-3 * np.abs(grads[kind]).max())
        err = abs(g - fd) / scale
        worst = max(worst, err)
        assert err <= 1e-4, (kind, k, g, fd)
    return worst


def test_trajectory_gradient_small(nb, ctx, oracle_mod):
    # N = 512 Plummer, eps = 1/64, 64 KDK steps of dt = 1/512, checkpoints
    # every 8 steps, loss = sum |x(T) - y|^2: 15 coordinates of x0, v0, m.
    _trajectory_grad_check(nb, ctx, oracle_mod, 512, np.float32(1.0 / 64), 1.0 / 512, 64, 15, 4)


def test_trajectory_gradient_small_compensated(nb, ctx, oracle_mod):
    # The same with the compensated force (positions as grid part + remainder
    # in the forward and in the adjoint's replay).
    _trajectory_grad_check(nb, ctx, oracle_mod, 512, np.float32(1.0 / 64), 1.0 / 512, 64, 6, 5,
                           mode=1)


def _autograd_composition(x0, v0, m, eps, dt, steps, ctx):
    """The trajectory built from NBForce and PyTorch arithmetic (the kicks and
    drift written as tensor operations), differentiated by autograd."""
    import torch
    from paper_0904_3659_gb300.autograd import NBForce
    a, _ = NBForce.apply(x0.float(), m, eps, 0, ctx)
    x, v = x0, v0
    for _ in range(steps):
        v = v + (0.5 * dt) * (-a.double())
        x = x + dt * v
        a, _ = NBForce.apply(x.float(), m, eps, 0, ctx)
        v = v + (0.5 * dt) * (-a.double())
    return x, v


@pytest.mark.parametrize("every", [4, 0])
def test_library_adjoint_matches_autograd_composition(nb, ctx, every):
    # The library's replay + reverse sweep against autograd through the same
    # forward arithmetic (plain mode, one packed tile shape forced for both:
    # the leap-frog kernels feed the pair kernel FP32 positions exactly as
    # NBForce does; the kernels' FP64 drift may fuse x + dt v into one
    # rounding where PyTorch rounds twice, so the trajectories agree to FP64
    # rounding). The gradients differ only in the order and precision of their
    # accumulations (the library adds the mass gradient in FP64).
    import torch
    from paper_0904_3659_gb300.autograd import leapfrog
    dev = torch.device("cuda:0")
    x0, v0, m = workloads.plummer(2500, seed=21)
    y = torch.from_numpy(workloads.targets(x0, seed=22)).to(dev)
    eps, dt, steps = np.float32(1.0 / 64), 1.0 / 512, 10
    packed = [t for t in nb.nb_list_tiles(0) if not t.fused and t.refine == 0][0]
    nb.nb_set_tile(ctx, 0, packed)
    res = []
    for which in ("library", "autograd"):
        xt = torch.from_numpy(x0.copy()).to(dev).requires_grad_(True)
        vt = torch.from_numpy(v0.copy()).to(dev).requires_grad_(True)
        mt = torch.from_numpy(m.astype(np.float32)).to(dev).requires_grad_(True)
        if which == "library":
            xT, vT = leapfrog(xt, vt, mt, eps, dt, steps, checkpoint_every=every, nbctx=ctx)
        else:
            xT, vT = _autograd_composition(xt, vt, mt, eps, dt, steps, ctx)
        (((xT - y) ** 2).sum() + 0.5 * (vT ** 2).sum()).backward()
        res.append((xT.detach().cpu().numpy(), xt.grad.cpu().numpy(), vt.grad.cpu().numpy(),
                    mt.grad.cpu().numpy()))
    nb.nb_set_tile(ctx, 0, None)
    (xl, gxl, gvl, gml), (xa, gxa, gva, gma) = res
    np.testing.assert_allclose(xl, xa, rtol=1e-13, atol=1e-15)
    for u, w in ((gxl, gxa), (gvl, gva)):
        np.testing.assert_allclose(u, w, rtol=1e-5, atol=1e-7 * np.abs(w).max())
    np.testing.assert_allclose(gml, gma, rtol=1e-4, atol=1e-5 * np.abs(gma).max())


ADJOINT_FD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                          "adjoint_fd_plummer16384.txt")


def _read_adjoint_fd():
    rows = []
    with open(ADJOINT_FD) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, i, c, h, fd, g = line.split()
            rows.append((k, int(i), int(c), float(h), float(fd), float(g)))
    return rows


def test_trajectory_gradient_plummer16384(nb, ctx, oracle_mod):
    # The differentiation workload (N = 16384 Plummer, eps = 1/64, 64 KDK
    # steps of dt = 1/512, checkpoints every 8, L = sum |x(T) - y|^2): the
    # library's gradient against FP64 central finite differences of the
    # oracle's trajectory on all 32 stored coordinates (written by
    # tests/golden/make_adjoint_fd.py from the oracle alone; recomputing
    # them takes minutes), within 1e-4 relative, and on every coordinate
    # against the oracle's FP64 reverse-mode gradient (_trajectory_grad_check
    # with no live differences). NB_FULL_ADJOINT_CHECK=1 also recomputes the
    # 32 differences live.
    import torch
    from paper_0904_3659_gb300.autograd import leapfrog
    w = workloads.WORKLOADS["plummer16384_adjoint64"]
    n, eps = w["n"], np.float32(w["eps"])
    x0, v0, m = workloads.plummer(n, seed=w["seed"])
    y = workloads.targets(x0, seed=w["target_seed"])
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(x0.copy()).to(dev).requires_grad_(True)
    vt = torch.from_numpy(v0.copy()).to(dev).requires_grad_(True)
    mt = torch.from_numpy(m.astype(np.float32)).to(dev).requires_grad_(True)
    xT, _ = leapfrog(xt, vt, mt, eps, w["dt"], w["steps"], checkpoint_every=w["checkpoint"],
                     nbctx=ctx)
    ((xT - torch.from_numpy(y).to(dev)) ** 2).sum().backward()
    g = {"x": xt.grad.cpu().numpy(), "v": vt.grad.cpu().numpy(), "m": mt.grad.cpu().numpy()}
    rows = _read_adjoint_fd()
    assert len(rows) == w["fd_coords"]
    worst = 0.0
    for kind, i, c, h, fd, _ in rows:
        v = float(g[kind][i] if kind == "m" else g[kind][i, c])
        err = abs(v - fd) / abs(fd)
        worst = max(worst, err)
        assert err <= 1e-4, (kind, i, c, v, fd, err)
    print(f"32 stored FD coordinates: worst relative error {worst:.3e}")
    ncoords = w["fd_coords"] if os.environ.get("NB_FULL_ADJOINT_CHECK") else 0
    _trajectory_grad_check(nb, ctx, oracle_mod, n, eps, w["dt"], w["steps"], ncoords, w["seed"])


def test_checkpointing_does_not_change_gradients(nb, ctx):
    import torch
    from paper_0904_3659_gb300.autograd import leapfrog
    dev = torch.device("cuda:0")
    x0, v0, m = workloads.plummer(700, seed=13)
    out = []
    for every in (0, 8, 5):
        xt = torch.from_numpy(x0.copy()).to(dev).requires_grad_(True)
        vt = torch.from_numpy(v0.copy()).to(dev).requires_grad_(True)
        mt = torch.from_numpy(m.astype(np.float32)).to(dev).requires_grad_(True)
        xT, vT = leapfrog(xt, vt, mt, np.float32(0.02), 1.0 / 256, 20, checkpoint_every=every,
                          nbctx=ctx)
        (xT.square().sum() + vT.square().sum()).backward()
        out.append((xt.grad.cpu().numpy(), vt.grad.cpu().numpy(), mt.grad.cpu().numpy()))
    # Recomputed segments give the same positions and the reverse sweep adds
    # the contributions in the same order whatever the segment length.
    for o in out[1:]:
        for u, w in zip(out[0], o):
            assert u.tobytes() == w.tobytes()

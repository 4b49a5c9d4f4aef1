"""GPU parity of nb_force_batched and nb_leapfrog_batched_step: many
independent clusters of uneven size in one persistent launch, each checked
against the FP64 oracle run on that cluster alone (Eq. (gravity) within a
cluster, nothing between clusters)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
TOL = {0: 1e-5, 1: 1e-6}


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


def run_batched(nb, ctx, x32, m32, offsets, eps32, mode):
    import torch
    dev = torch.device("cuda:0")
    n = x32.shape[0]
    xt = torch.from_numpy(np.ascontiguousarray(x32)).to(dev)
    mt = torch.from_numpy(np.ascontiguousarray(m32)).to(dev)
    ot = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64)).to(dev)
    et = torch.from_numpy(np.ascontiguousarray(eps32, dtype=np.float32)).to(dev)
    a = torch.full((n, 3), float("nan"), device=dev)
    p = torch.full((n,), float("nan"), device=dev)
    nb.nb_force_batched(ctx, xt, mt, ot, len(offsets) - 1, n, et, a, p, mode)
    nb.nb_synchronize(ctx)
    return a.cpu().numpy(), p.cpu().numpy()


def check_clusters(oracle_mod, x32, m32, offsets, eps32, a, p, tol):
    worst = 0.0
    for c in range(len(offsets) - 1):
        lo, hi = offsets[c], offsets[c + 1]
        if hi == lo:
            continue
        ra, rp, ramag = oracle_mod.force(x32[lo:hi], m32[lo:hi], eps32[c])
        da = np.linalg.norm(a[lo:hi].astype(np.float64) - ra, axis=1)
        ea = np.where(ramag > 0, da / np.where(ramag > 0, ramag, 1), da)
        ep = np.where(rp > 0, np.abs(p[lo:hi] - rp) / np.where(rp > 0, rp, 1), np.abs(p[lo:hi]))
        worst = max(worst, ea.max(), ep.max())
    assert worst <= tol, worst
    return worst


@pytest.mark.parametrize("mode", [0, 1])
def test_uneven_clusters(nb, ctx, oracle_mod, mode):
    sizes = [1, 0, 2, 31, 127, 128, 129, 300, 0, 1000, 2049, 5]
    rng = np.random.default_rng(1)
    xs, ms = [], []
    for k, s in enumerate(sizes):
        x, _, m = workloads.plummer(s, seed=100 + k, b=rng.uniform(0.5, 2.0)) if s else (
            np.zeros((0, 3)), None, np.zeros(0))
        xs.append(x)
        ms.append(m)
    x32 = np.concatenate(xs).astype(np.float32)
    m32 = np.concatenate(ms).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eps32 = rng.uniform(0.01, 0.05, len(sizes)).astype(np.float32)
    a, p = run_batched(nb, ctx, x32, m32, offsets, eps32, mode)
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
    check_clusters(oracle_mod, x32, m32, offsets, eps32, a, p, TOL[mode])


@pytest.fixture(scope="module")
def clusters1024():
    w = workloads.WORKLOADS["clusters1024_kdk32"]
    return workloads.clusters(w["n_clusters"], seed=w["seed"], nmin=w["nmin"], nmax=w["nmax"])


@pytest.mark.parametrize("mode", [0, 1])
def test_clusters1024_all_against_oracle(nb, ctx, oracle_mod, clusters1024, mode):
    cl = clusters1024
    x32, m32 = cl.x.astype(np.float32), cl.m.astype(np.float32)
    eps32 = cl.eps.astype(np.float32)
    a, p = run_batched(nb, ctx, x32, m32, cl.offsets, eps32, mode)
    check_clusters(oracle_mod, x32, m32, cl.offsets, eps32, a, p, TOL[mode])
    # The same launch again gives the same bits, whatever order the CTAs
    # take work items from the queue.
    a2, p2 = run_batched(nb, ctx, x32, m32, cl.offsets, eps32, mode)
    assert a.tobytes() == a2.tobytes() and p.tobytes() == p2.tobytes()


def test_invalid_offsets_rejected_without_writes(nb, ctx):
    import torch
    dev = torch.device("cuda:0")
    n = 100
    x = torch.zeros((n, 3), device=dev)
    m = torch.ones(n, device=dev)
    eps = torch.full((2,), 0.1, device=dev)
    for bad in ([0, 60, 140], [0, 70, 50], [5, 50, 100]):
        off = torch.tensor(bad, dtype=torch.int64, device=dev)
        a = torch.full((n, 3), 7.0, device=dev)
        p = torch.full((n,), 7.0, device=dev)
        nb.nb_force_batched(ctx, x, m, off, 2, n, eps, a, p)
        with pytest.raises(nb.NBError) as e:
            nb.nb_synchronize(ctx)
        assert e.value.status == nb.NB_ERR_ARG
        assert torch.all(a == 7.0) and torch.all(p == 7.0)
    # A non-empty cluster whose eps^2 is not a finite normal FP32 number is
    # rejected the same way; an empty cluster's eps is not read.
    off = torch.tensor([0, 60, 60, 100], dtype=torch.int64, device=dev)
    for bad_eps in (0.0, -0.5, float("nan"), float("inf"), 1e-20, 1e20):
        e3 = torch.tensor([0.1, 0.1, bad_eps], device=dev)
        a = torch.full((n, 3), 7.0, device=dev)
        p = torch.full((n,), 7.0, device=dev)
        nb.nb_force_batched(ctx, x, m, off, 3, n, e3, a, p)
        with pytest.raises(nb.NBError) as e:
            nb.nb_synchronize(ctx)
        assert e.value.status == nb.NB_ERR_ARG, bad_eps
        assert torch.all(a == 7.0) and torch.all(p == 7.0)
    e3 = torch.tensor([0.1, float("nan"), 0.1], device=dev)  # the empty cluster's eps
    nb.nb_force_batched(ctx, x, m, off, 3, n, e3, torch.empty((n, 3), device=dev),
                        torch.empty(n, device=dev))
    nb.nb_synchronize(ctx)


@pytest.mark.parametrize("mode", [0, 1])
def test_plan_follows_offsets_and_eps_changed_in_place(nb, ctx, oracle_mod, mode):
    # The context keeps its last batched plan and reuses it while the
    # offsets and eps hold the same values; the same device arrays rewritten
    # between calls (same cluster count and particle total), made invalid and
    # then restored must each be planned afresh.
    import torch
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(21)
    n = 3000
    x32 = rng.normal(size=(n, 3)).astype(np.float32)
    m32 = rng.uniform(0.5, 1.5, size=n).astype(np.float32) / n
    xt = torch.from_numpy(x32).to(dev)
    mt = torch.from_numpy(m32).to(dev)
    off = torch.empty(4, dtype=torch.int64, device=dev)
    eps = torch.empty(3, dtype=torch.float32, device=dev)
    a = torch.empty((n, 3), device=dev)
    p = torch.empty(n, device=dev)
    cases = [([0, 700, 2100, 3000], [0.05, 0.1, 0.02]),
             ([0, 1500, 1600, 3000], [0.05, 0.1, 0.02]),   # boundaries moved
             ([0, 1500, 1600, 3000], [0.01, 0.2, 0.03]),   # eps changed
             ([0, 2000, 1600, 3000], [0.01, 0.2, 0.03]),   # invalid: decreasing
             ([0, 1500, 1600, 3000], [0.01, 0.2, 0.03]),   # restored
             ([0, 700, 2100, 3000], [0.05, 0.1, 0.02])]
    for o, e in cases:
        off.copy_(torch.tensor(o, dtype=torch.int64))
        eps.copy_(torch.tensor(e, dtype=torch.float32))
        a.fill_(float("nan"))
        p.fill_(float("nan"))
        nb.nb_force_batched(ctx, xt, mt, off, 3, n, eps, a, p, mode)
        if any(o[k + 1] < o[k] for k in range(3)):
            with pytest.raises(nb.NBError) as err:
                nb.nb_synchronize(ctx)
            assert err.value.status == nb.NB_ERR_ARG
            continue
        nb.nb_synchronize(ctx)
        check_clusters(oracle_mod, x32, m32, np.array(o), np.array(e, np.float32),
                       a.cpu().numpy(), p.cpu().numpy(), TOL[mode])


def test_batched_leapfrog_matches_single_cluster_calls(nb, ctx):
    # 32 graph-replayed KDK steps of a batch equal, cluster by cluster, the
    # single-system integrator's steps (same arithmetic per pair; the pair
    # order differs, so compare within the force tolerance's effect).
    import torch
    dev = torch.device("cuda:0")
    sizes = [300, 1000, 64, 513]
    xs, vs, ms = [], [], []
    for k, s in enumerate(sizes):
        x, v, m = workloads.plummer(s, seed=200 + k)
        xs.append(x)
        vs.append(v)
        ms.append(m)
    x0 = np.concatenate(xs)
    v0 = np.concatenate(vs)
    m32 = np.concatenate(ms).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eps32 = np.full(len(sizes), 0.02, np.float32)
    n = x0.shape[0]
    stream = torch.cuda.Stream()
    xt = torch.from_numpy(x0.copy()).to(dev)
    vt = torch.from_numpy(v0.copy()).to(dev)
    mt = torch.from_numpy(m32).to(dev)
    ot = torch.from_numpy(offsets).to(dev)
    et = torch.from_numpy(eps32).to(dev)
    a = torch.zeros((n, 3), device=dev)
    p = torch.zeros(n, device=dev)
    torch.cuda.synchronize()
    nb.nb_leapfrog_batched_step(ctx, xt, vt, mt, ot, len(sizes), n, et, a, p, 1.0 / 256, 32, 0, 0,
                                stream)
    nb.nb_synchronize(ctx, stream)
    xb = xt.cpu().numpy()
    for c, s in enumerate(sizes):
        lo, hi = offsets[c], offsets[c + 1]
        xs_t = torch.from_numpy(x0[lo:hi].copy()).to(dev)
        vs_t = torch.from_numpy(v0[lo:hi].copy()).to(dev)
        ms_t = torch.from_numpy(m32[lo:hi].copy()).to(dev)
        as_t = torch.zeros((s, 3), device=dev)
        ps_t = torch.zeros(s, device=dev)
        torch.cuda.synchronize()
        nb.nb_leapfrog_step(ctx, xs_t, vs_t, ms_t, as_t, ps_t, s, eps32[c], 1.0 / 256, 32, 0, 0,
                            stream)
        nb.nb_synchronize(ctx, stream)
        assert np.abs(xs_t.cpu().numpy() - xb[lo:hi]).max() < 1e-8


def test_batched_compensated_fp64_state_far_from_origin(nb, ctx, oracle_mod):
    # Clusters placed far from the origin (FP64 state): the compensated batch
    # splits each position, relative to its cluster's bounding-box centre,
    # into an exact FP32 grid part and an FP32 remainder, so x_i - x_j carries
    # one rounding wherever the cluster sits (plain rounding of |x| ~ 1e3
    # loses u |x|). Target of the compensated path: 1e-6.
    import torch
    dev = torch.device("cuda:0")
    sizes = [900, 2500, 300]
    shifts = [np.array([1000.0, 0, 0]), np.array([-500.0, 750.0, 20.0]), np.array([0, 0, 3000.0])]
    xs, ms = [], []
    for k, s in enumerate(sizes):
        x, _, m = workloads.plummer(s, seed=300 + k)
        xs.append(x + shifts[k])
        ms.append(m)
    x64 = np.concatenate(xs)
    m32 = np.concatenate(ms).astype(np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eps32 = np.full(len(sizes), 1.0 / 128, np.float32)
    n = x64.shape[0]
    worst = {}
    for mode in (0, 1):
        xt = torch.from_numpy(x64.copy()).to(dev)
        vt = torch.zeros_like(xt)
        mt = torch.from_numpy(m32).to(dev)
        ot = torch.from_numpy(offsets).to(dev)
        et = torch.from_numpy(eps32).to(dev)
        a = torch.zeros((n, 3), device=dev)
        p = torch.zeros(n, device=dev)
        torch.cuda.synchronize()
        nb.nb_leapfrog_batched_step(ctx, xt, vt, mt, ot, len(sizes), n, et, a, p, 0.0, 0, 0, mode)
        nb.nb_synchronize(ctx)
        A, P = a.cpu().numpy().astype(np.float64), p.cpu().numpy().astype(np.float64)
        w = 0.0
        for c in range(len(sizes)):
            lo, hi = offsets[c], offsets[c + 1]
            ra, rp, ramag = oracle_mod.force(x64[lo:hi], m32[lo:hi], eps32[c])
            w = max(w, (np.linalg.norm(A[lo:hi] - ra, axis=1) / ramag).max(),
                    (np.abs(P[lo:hi] - rp) / rp).max())
        worst[mode] = w
    assert worst[1] <= 1e-6, worst
    assert worst[1] * 100 <= worst[0], worst


@pytest.mark.parametrize("shift", [0.0, 300.0])
def test_batched_compensated_kdk_clusters_against_oracle(nb, ctx, oracle_mod, shift):
    # The compensated batched leap-frog on FP64 state (each cluster's
    # positions as grid part + remainder): after 8 graph-replayed KDK steps the force it
    # returns at the final positions matches the FP64 oracle at those same
    # positions within 1e-6 for every particle of every cluster, centred or
    # moved away from the origin; two runs give the same bits.
    import torch
    dev = torch.device("cuda:0")
    cl = workloads.clusters(96, seed=7, nmin=32, nmax=2048)
    x0 = cl.x + shift * np.array([1.0, -0.5, 0.25])
    m32 = cl.m.astype(np.float32)
    eps32 = cl.eps.astype(np.float32)
    n, C = x0.shape[0], len(cl.sizes)
    stream = torch.cuda.Stream()
    runs = []
    for _ in range(2):
        xt = torch.from_numpy(x0.copy()).to(dev)
        vt = torch.from_numpy(cl.v.copy()).to(dev)
        mt = torch.from_numpy(m32).to(dev)
        ot = torch.from_numpy(cl.offsets).to(dev)
        et = torch.from_numpy(eps32).to(dev)
        a = torch.zeros((n, 3), device=dev)
        p = torch.zeros(n, device=dev)
        torch.cuda.synchronize()
        nb.nb_leapfrog_batched_step(ctx, xt, vt, mt, ot, C, n, et, a, p, 1.0 / 256, 8, 0, 1, stream)
        nb.nb_synchronize(ctx, stream)
        runs.append((xt.cpu().numpy(), a.cpu().numpy(), p.cpu().numpy()))
    (x1, a1, p1), (x2, a2, p2) = runs
    assert x1.tobytes() == x2.tobytes() and a1.tobytes() == a2.tobytes()
    assert p1.tobytes() == p2.tobytes()
    worst = 0.0
    for c in range(C):
        lo, hi = cl.offsets[c], cl.offsets[c + 1]
        ra, rp, ramag = oracle_mod.force(x1[lo:hi], m32[lo:hi], eps32[c])
        worst = max(worst, (np.linalg.norm(a1[lo:hi].astype(np.float64) - ra, axis=1) / ramag).max(),
                    (np.abs(p1[lo:hi] - rp) / rp).max())
    assert worst <= 1e-6, worst

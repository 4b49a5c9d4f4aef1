"""GPU parity of nb_force (Eq. (gravity)) against the FP64 oracle.

Acceptance metric (per particle, max over particles):
  e_a,i = |a_gpu,i - a_ref,i| / A_i,  A_i = sum_{j != i} m_j |x_i - x_j| / s_ij^{3/2}
  e_p,i = |p_gpu,i - p_ref,i| / p_i
A_i equals |a_i| when the terms do not cancel and keeps the measure
well-posed near the centre of a cluster, where a_i -> 0 by symmetry.
Tolerances: 1e-5 (NB_PLAIN), 1e-6 (NB_COMPENSATED).
"""
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


def gpu_force(nb, ctx, x32, m32, eps, mode):
    import torch
    n = x32.shape[0]
    dev = torch.device("cuda:0")
    xt = torch.from_numpy(np.ascontiguousarray(x32)).to(dev)
    mt = torch.from_numpy(np.ascontiguousarray(m32)).to(dev)
    a = torch.full((n, 3), float("nan"), dtype=torch.float32, device=dev)
    p = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
    nb.nb_force(ctx, xt, mt, n, eps, a, p, mode)
    nb.nb_synchronize(ctx)
    return a.cpu().numpy(), p.cpu().numpy()


def rel_errors(a, p, ra, rp, ramag):
    da = np.linalg.norm(a.astype(np.float64) - ra, axis=1)
    dp = np.abs(p.astype(np.float64) - rp)
    ea = np.where(ramag > 0, da / np.where(ramag > 0, ramag, 1.0), da)
    ep = np.where(rp > 0, dp / np.where(rp > 0, rp, 1.0), dp)
    return ea, ep


def plummer32(n, seed=0):
    x, _, m = workloads.plummer(n, seed=seed)
    return x.astype(np.float32), m.astype(np.float32)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 127, 1000, 1023, 1025, 4097, 6000])
def test_ragged_sizes(nb, ctx, oracle_mod, n, mode):
    x32, m32 = plummer32(n, seed=n)
    eps = np.float32(0.01)
    a, p = gpu_force(nb, ctx, x32, m32, eps, mode)
    ra, rp, ramag = oracle_mod.force(x32, m32, eps)
    ea, ep = rel_errors(a, p, ra, rp, ramag)
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
    assert ea.max() <= TOL[mode], ea.max()
    assert ep.max() <= TOL[mode], ep.max()


@pytest.mark.parametrize("mode", [0, 1])
def test_plummer4096_full(nb, ctx, oracle_mod, mode):
    # Single force + potential evaluation, N = 4096 equal-mass Plummer sphere,
    # eps = 0.01, one call to nb_force, full oracle.
    w = workloads.WORKLOADS["plummer4096"]
    x32, m32 = plummer32(w["n"], w["seed"])
    eps = np.float32(w["eps"])
    a, p = gpu_force(nb, ctx, x32, m32, eps, mode)
    ra, rp, ramag = oracle_mod.force(x32, m32, eps)
    ea, ep = rel_errors(a, p, ra, rp, ramag)
    assert ea.max() <= TOL[mode] and ep.max() <= TOL[mode], (ea.max(), ep.max())
    # Momentum invariant sum_i m_i a_i = 0, to FP32 accuracy of the sums.
    mom = np.abs((m32[:, None].astype(np.float64) * a).sum(0)).max()
    assert mom <= 1e-5 * (m32 * ramag).sum()


@pytest.mark.parametrize("mode", [0, 1])
def test_every_tile_shape(nb, ctx, oracle_mod, mode):
    # Each compiled tile shape at a size that spans several i-blocks and
    # j-tiles with a ragged tail.
    n = 3001
    x32, m32 = plummer32(n, seed=7)
    eps = np.float32(1.0 / 64)
    ra, rp, ramag = oracle_mod.force(x32, m32, eps)
    try:
        for tile in nb.nb_list_tiles(mode):
            nb.nb_set_tile(ctx, mode, tile)
            a, p = gpu_force(nb, ctx, x32, m32, eps, mode)
            ea, ep = rel_errors(a, p, ra, rp, ramag)
            assert ea.max() <= TOL[mode] and ep.max() <= TOL[mode], (tile, ea.max(), ep.max())
    finally:
        nb.nb_set_tile(ctx, mode, None)


def test_default_shapes_skip_newton_step(nb, ctx):
    # The built-in shapes use the special-function unit's rsqrt without the
    # Newton step (13 FP32 ops per pair); the step's shapes stay selectable.
    for mode in (0, 1):
        for n in (1000, 10000, 100000, 1 << 20):
            assert nb.nb_get_tile(ctx, n, mode).refine == 0, (mode, n)


def test_default_path_by_size(nb):
    # Built-in choice without tuning: the cluster single-launch shape up to
    # 9728 (76 clusters of two), the stream-K form up to 24576, pack -> pair
    # -> combine above.
    fresh = nb.Context(0)
    try:
        for mode in (0, 1):
            for n, fused in ((1, 3), (4096, 3), (8192, 3), (9728, 3), (9729, 2), (16384, 2),
                             (24575, 2), (24576, 0), (1 << 20, 0)):
                assert nb.nb_get_tile(fresh, n, mode).fused == fused, (mode, n)
    finally:
        fresh.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_newton_step_matches_unrefined_accuracy(nb, ctx, oracle_mod, mode):
    # The same shape with and without the Newton step: both within the
    # mode's tolerance, and the step does not make the result more accurate
    # than the special-function unit's estimate by more than a factor 2.
    n = 12000
    x32, m32 = plummer32(n, seed=17)
    eps = np.float32(1.0 / 128)
    ra, rp, ramag = oracle_mod.force(x32, m32, eps)
    errs = {}
    try:
        for refine in (0, 1):
            base = [t for t in nb.nb_list_tiles(mode) if t.refine == refine][0].as_tuple()
            nb.nb_set_tile(ctx, mode, base)
            a, p = gpu_force(nb, ctx, x32, m32, eps, mode)
            ea, ep = rel_errors(a, p, ra, rp, ramag)
            assert ea.max() <= TOL[mode] and ep.max() <= TOL[mode], (base, ea.max(), ep.max())
            errs[refine] = (ea.max(), ep.max())
    finally:
        nb.nb_set_tile(ctx, mode, None)
    assert errs[0][0] <= 2 * errs[1][0] and errs[0][1] <= 2 * errs[1][1], errs


@pytest.mark.parametrize("mode", [0, 1])
def test_fused_shapes(nb, ctx, oracle_mod, mode):
    # Single-launch shapes (no pack or combine kernel; the last CTA of each
    # i-block adds its partials): sizes run back to back, so a count left
    # non-zero by one launch would corrupt the next; every call is repeated
    # and must give the same bits.
    fused = [t for t in nb.nb_list_tiles(mode) if t.fused]
    assert fused
    eps = np.float32(1.0 / 64)
    cases = []
    # 20000: a stream-K CTA's range can touch three i-blocks (and the cluster
    # form falls to one CTA per cluster); 4096, 7168 and 9728: the chunked and
    # cluster forms' workload, a size where two CTAs per SM take larger
    # clusters than one, and their largest built-in size (76 clusters of two).
    for n in (1, 200, 3001, 4096, 7168, 8191, 9000, 9728, 20000):
        x32, m32 = plummer32(n, seed=100 + n)
        cases.append((n, x32, m32, oracle_mod.force(x32, m32, eps)))
    try:
        for tile in fused:
            nb.nb_set_tile(ctx, mode, tile)
            for n, x32, m32, (ra, rp, ramag) in cases:
                a1, p1 = gpu_force(nb, ctx, x32, m32, eps, mode)
                a2, p2 = gpu_force(nb, ctx, x32, m32, eps, mode)
                assert a1.tobytes() == a2.tobytes() and p1.tobytes() == p2.tobytes(), (tile, n)
                ea, ep = rel_errors(a1, p1, ra, rp, ramag)
                assert ea.max() <= TOL[mode] and ep.max() <= TOL[mode], (tile, n, ea.max(), ep.max())
    finally:
        nb.nb_set_tile(ctx, mode, None)


def test_fused_override_leaves_leapfrog_on_packed_shapes(nb, ctx):
    # The leap-frog packs FP64 state itself, so with a fused shape forced it
    # runs the built-in packed shape of the size class: the same bits.
    import torch
    x0, v0, m = workloads.plummer(3000, seed=31)
    dev = torch.device("cuda:0")
    runs = []
    fused = [t for t in nb.nb_list_tiles(0) if t.fused][0]
    for tile in (None, fused):
        nb.nb_set_tile(ctx, 0, tile)
        x = torch.from_numpy(x0.copy()).to(dev)
        v = torch.from_numpy(v0.copy()).to(dev)
        mt = torch.from_numpy(m.astype(np.float32)).to(dev)
        a = torch.empty((3000, 3), dtype=torch.float32, device=dev)
        nb.nb_leapfrog_step(ctx, x, v, mt, a, None, 3000, np.float32(0.02), 1.0 / 256, 4, 0, 0)
        nb.nb_synchronize(ctx)
        runs.append(x.cpu().numpy().tobytes())
    nb.nb_set_tile(ctx, 0, None)
    assert runs[0] == runs[1]


@pytest.mark.parametrize("mode", [0, 1])
def test_bitwise_repeatable(nb, ctx, mode):
    x32, m32 = plummer32(20000, seed=3)
    a1, p1 = gpu_force(nb, ctx, x32, m32, np.float32(0.01), mode)
    a2, p2 = gpu_force(nb, ctx, x32, m32, np.float32(0.01), mode)
    assert a1.tobytes() == a2.tobytes() and p1.tobytes() == p2.tobytes()


def test_coincident_and_self(nb, ctx, oracle_mod):
    # Duplicated positions: distinct coincident particles are summed, the
    # self term is not.
    rng = np.random.default_rng(5)
    base = rng.normal(size=(700, 3)).astype(np.float32)
    x32 = np.concatenate([base, base[:300]])
    m32 = rng.uniform(0.5, 1.5, 1000).astype(np.float32)
    eps = np.float32(0.05)
    for mode in (0, 1):
        a, p = gpu_force(nb, ctx, x32, m32, eps, mode)
        ra, rp, ramag = oracle_mod.force(x32, m32, eps)
        ea, ep = rel_errors(a, p, ra, rp, ramag)
        assert ea.max() <= TOL[mode] and ep.max() <= TOL[mode]


def test_power_of_two_scaling_exact(nb, ctx):
    # x -> 2x, eps -> 2eps scales every FP32 operation of the kernel by a
    # power of two: the outputs must be exactly a/4, p/2.
    x32, m32 = plummer32(5000, seed=9)
    for mode in (0, 1):
        a1, p1 = gpu_force(nb, ctx, x32, m32, np.float32(0.125), mode)
        a2, p2 = gpu_force(nb, ctx, 2 * x32, m32, np.float32(0.25), mode)
        np.testing.assert_array_equal(a2, a1 / 4)
        np.testing.assert_array_equal(p2, p1 / 2)


@pytest.mark.parametrize("mode", [0, 1])
def test_plummer65536_full(nb, ctx, oracle_mod, mode):
    w = workloads.WORKLOADS["plummer65536_kdk16"]
    x32, m32 = plummer32(w["n"], w["seed"])
    eps = np.float32(w["eps"])
    a, p = gpu_force(nb, ctx, x32, m32, eps, mode)
    ra, rp, ramag = oracle_mod.force(x32, m32, eps)
    ea, ep = rel_errors(a, p, ra, rp, ramag)
    assert ea.max() <= TOL[mode] and ep.max() <= TOL[mode], (ea.max(), ep.max())


@pytest.fixture(scope="module")
def plummer1m(oracle_mod):
    w = workloads.WORKLOADS["plummer1m"]
    x32, m32 = plummer32(w["n"], w["seed"])
    rows = workloads.sample_rows(w["n"], w["sample"], w["sample_seed"])
    eps = np.float32(w["eps"])
    ra, rp, ramag = oracle_mod.force_rows(x32, m32, eps, rows)
    return x32, m32, eps, rows, ra, rp, ramag


@pytest.mark.parametrize("mode", [0, 1])
def test_plummer1m_sampled_every_tile(nb, ctx, plummer1m, mode):
    # N = 2^20, eps = 1/256: every compiled shape (the benchmark runs one of
    # them), checked on 2048 sampled rows against the FP64 oracle.
    x32, m32, eps, rows, ra, rp, ramag = plummer1m
    try:
        for tile in nb.nb_list_tiles(mode):
            nb.nb_set_tile(ctx, mode, tile)
            a, p = gpu_force(nb, ctx, x32, m32, eps, mode)
            ea, ep = rel_errors(a[rows], p[rows], ra, rp, ramag)
            assert ea.max() <= TOL[mode] and ep.max() <= TOL[mode], (tile, ea.max(), ep.max())
    finally:
        nb.nb_set_tile(ctx, mode, None)


def test_argument_errors(nb, ctx):
    import torch
    dev = torch.device("cuda:0")
    x = torch.zeros((4, 3), device=dev)
    m = torch.ones(4, device=dev)
    a = torch.empty((4, 3), device=dev)
    p = torch.empty(4, device=dev)
    # eps must be finite and > 0, and eps^2 a normal FP32 number (the kernels
    # work with eps^2: below ~1.1e-19 it would flush to zero, above ~1.8e19
    # overflow).
    for eps in (0.0, -1.0, float("inf"), float("nan"), 1e-20, 1e20):
        with pytest.raises(nb.NBError) as e:
            nb.nb_force(ctx, x, m, 4, eps, a, p)
        assert e.value.status == nb.NB_ERR_ARG
    for eps in (2e-19, 1e19):  # just inside the range
        nb.nb_force(ctx, x, m, 4, eps, a, p)
    with pytest.raises(nb.NBError) as e:
        nb.nb_force(ctx, x, m, -1, 0.1, a, p)
    assert e.value.status == nb.NB_ERR_ARG
    with pytest.raises(nb.NBError) as e:
        nb.nb_force(ctx, None, m, 4, 0.1, a, p)
    assert e.value.status == nb.NB_ERR_ARG
    with pytest.raises(nb.NBError) as e:
        nb.nb_force(ctx, x, m, 4, 0.1, a, p, mode=7)
    assert e.value.status == nb.NB_ERR_ARG
    # n == 0 is a valid no-op, even with NULL pointers.
    nb.nb_force(ctx, None, None, 0, 0.1, None, None)
    with pytest.raises(nb.NBError) as e:
        nb.nb_set_tile(ctx, 0, (96, 3, 100, 2, 4, 1, 0, 0, 63))
    assert e.value.status == nb.NB_ERR_ARG


@pytest.mark.parametrize("release", [0, 1])
def test_bounded_wait_reports_timeout_and_context_survives(nb, ctx, oracle_mod, release):
    # The producer skips the copy of one work unit, so the consumers' bounded
    # wait (0.2 s here) runs out; the kernel records a timeout and returns,
    # and nb_synchronize reports it. Nothing hangs or faults, and the next
    # call on the same context is correct. Both stage-release schemes.
    x32, m32 = plummer32(4096, seed=0)
    eps = np.float32(0.01)
    tile = [t for t in nb.nb_list_tiles(0) if t.release == release][0]
    nb.nb_set_tile(ctx, 0, tile)
    nb.nb_debug_set_fault(ctx, 3, 200_000_000)
    try:
        import torch
        dev = torch.device("cuda:0")
        xt = torch.from_numpy(x32).to(dev)
        mt = torch.from_numpy(m32).to(dev)
        a = torch.empty((4096, 3), device=dev)
        p = torch.empty(4096, device=dev)
        nb.nb_force(ctx, xt, mt, 4096, eps, a, p)
        with pytest.raises(nb.NBError) as e:
            nb.nb_synchronize(ctx)
        assert e.value.status == nb.NB_ERR_TIMEOUT
    finally:
        nb.nb_debug_set_fault(ctx, -1, 0)
    try:
        a, p = gpu_force(nb, ctx, x32, m32, eps, 0)
    finally:
        nb.nb_set_tile(ctx, 0, None)
    ra, rp, ramag = oracle_mod.force(x32, m32, eps)
    ea, ep = rel_errors(a, p, ra, rp, ramag)
    assert ea.max() <= 1e-5 and ep.max() <= 1e-5


@pytest.mark.parametrize("mode", [0, 1])
def test_cluster_form_bounded_wait_reports_timeout(nb, ctx, oracle_mod, mode):
    # In the cluster form one CTA does not send its partial sums (test hook),
    # so the CTAs that own them wait out their bounded wait (0.2 s here),
    # record a timeout and write nothing; nb_synchronize reports it. Nothing
    # hangs or faults, and the next call on the same context is correct.
    x32, m32 = plummer32(4096, seed=0)
    eps = np.float32(0.01)
    tile = [t for t in nb.nb_list_tiles(mode) if t.fused == 3 and t.ipt == 4][0]
    nb.nb_set_tile(ctx, mode, tile)
    try:
        import torch
        dev = torch.device("cuda:0")
        xt = torch.from_numpy(x32).to(dev)
        mt = torch.from_numpy(m32).to(dev)
        a = torch.empty((4096, 3), device=dev)
        p = torch.empty(4096, device=dev)
        nb.nb_debug_set_fault(ctx, 1, 200_000_000)
        try:
            nb.nb_force(ctx, xt, mt, 4096, eps, a, p, mode)
            with pytest.raises(nb.NBError) as e:
                nb.nb_synchronize(ctx)
            assert e.value.status == nb.NB_ERR_TIMEOUT
        finally:
            nb.nb_debug_set_fault(ctx, -1, 0)
        a, p = gpu_force(nb, ctx, x32, m32, eps, mode)
    finally:
        nb.nb_set_tile(ctx, mode, None)
    ra, rp, ramag = oracle_mod.force(x32, m32, eps)
    ea, ep = rel_errors(a, p, ra, rp, ramag)
    tol = 1e-5 if mode == 0 else 1e-6
    assert ea.max() <= tol and ep.max() <= tol


def test_force_host_matches_device(nb, ctx):
    x32, m32 = plummer32(5000, seed=12)
    a_dev, p_dev = gpu_force(nb, ctx, x32, m32, np.float32(0.01), 0)
    a = np.empty((5000, 3), np.float32)
    p = np.empty(5000, np.float32)
    nb.nb_force_host(ctx, x32.ctypes.data, m32.ctypes.data, 5000, np.float32(0.01),
                     a.ctypes.data, p.ctypes.data, 0)
    assert a.tobytes() == a_dev.tobytes() and p.tobytes() == p_dev.tobytes()


def test_tuning_saved_and_restored(nb, ctx, tmp_path):
    # nb_autotune's picks survive a new context through the JSON file.
    path = tmp_path / "tuning.json"
    entries = nb.tune_to_file(ctx, [3000], str(path), modes=(0,))
    fresh = nb.Context(0)
    try:
        assert nb.load_tuning(fresh, str(path)) == 1
        assert nb.nb_get_tile(fresh, 3000, 0).as_tuple() == tuple(entries[0]["tile"])
        nb.nb_set_tuned_tile(fresh, 3000, 0, None)
        assert nb.nb_get_tile(fresh, 3000, 0).as_tuple() == nb.nb_get_tile(nb.Context(0), 3000, 0).as_tuple()
    finally:
        fresh.close()

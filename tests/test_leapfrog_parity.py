"""GPU checks of nb_leapfrog_step (Section "Method", Eqs. (1)-(3)) and
nb_energy against the FP64 oracle.

The device state (x, v) is FP64; the force comes from the FP32 pair kernel,
so trajectories agree with the oracle's all-FP64 trajectory to the size of
the force error times the elapsed time squared, and the energies to the
potential's FP32 accuracy.
"""
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


@pytest.fixture(scope="module")
def stream(nb):
    import torch
    return torch.cuda.Stream()


class State:
    def __init__(self, x, v, m):
        import torch
        dev = torch.device("cuda:0")
        self.n = x.shape[0]
        self.x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev)
        self.v = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(dev)
        self.m = torch.from_numpy(np.ascontiguousarray(m, dtype=np.float32)).to(dev)
        self.a = torch.zeros((self.n, 3), dtype=torch.float32, device=dev)
        self.p = torch.zeros(self.n, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()  # the library runs on another stream

    def step(self, nb, ctx, eps, dt, nsteps, a_valid, mode, stream):
        nb.nb_leapfrog_step(ctx, self.x, self.v, self.m, self.a, self.p, self.n, eps, dt, nsteps,
                            a_valid, mode, stream)
        nb.nb_synchronize(ctx, stream)

    def numpy(self):
        return self.x.cpu().numpy(), self.v.cpu().numpy()


def plummer_state(n, seed):
    x, v, m = workloads.plummer(n, seed=seed)
    return x, v, m.astype(np.float32)


@pytest.mark.parametrize("mode", [0, 1])
def test_trajectory_matches_oracle(nb, ctx, stream, oracle_mod, mode):
    n, eps, dt, steps = 2048, np.float32(1.0 / 64), 1.0 / 256, 16
    x0, v0, m = plummer_state(n, 4)
    s = State(x0, v0, m)
    s.step(nb, ctx, eps, dt, steps, 0, mode, stream)
    xg, vg = s.numpy()
    xr, vr, gr = oracle_mod.leapfrog(x0, v0, m, eps, dt, steps)
    # Force error ~1e-6 relative, elapsed time 1/16: position error ~1e-9.
    assert np.abs(xg - xr).max() < 1e-7
    assert np.abs(vg - vr).max() < 1e-6
    # The returned a is Eq. (gravity) (literal sign) at the final positions.
    a = s.a.cpu().numpy().astype(np.float64)
    scale = np.abs(gr).max()
    assert np.abs(a + gr).max() < 1e-4 * scale


def test_graph_and_direct_paths_agree_bitwise(nb, ctx, stream):
    # Steps after the first are replayed from a CUDA graph on a capturable
    # stream and launched directly on the legacy stream: same kernels, same
    # arguments, same bits. Chained calls equal one call with all steps.
    n, eps, dt = 3000, np.float32(0.02), 1.0 / 128
    x0, v0, m = plummer_state(n, 5)
    s1 = State(x0, v0, m)
    s1.step(nb, ctx, eps, dt, 10, 0, 0, stream)
    s2 = State(x0, v0, m)
    s2.step(nb, ctx, eps, dt, 10, 0, 0, 0)
    s3 = State(x0, v0, m)
    s3.step(nb, ctx, eps, dt, 4, 0, 0, stream)
    s3.step(nb, ctx, eps, dt, 6, 1, 0, stream)
    for other in (s2, s3):
        assert s1.x.cpu().numpy().tobytes() == other.x.cpu().numpy().tobytes()
        assert s1.v.cpu().numpy().tobytes() == other.v.cpu().numpy().tobytes()
        assert s1.a.cpu().numpy().tobytes() == other.a.cpu().numpy().tobytes()


def test_zero_steps_computes_force_only(nb, ctx, stream, oracle_mod):
    n, eps = 1500, np.float32(0.03)
    x0, v0, m = plummer_state(n, 6)
    s = State(x0, v0, m)
    s.step(nb, ctx, eps, 0.01, 0, 0, 0, stream)
    assert s.x.cpu().numpy().tobytes() == x0.tobytes()
    ra, rp, ramag = oracle_mod.force(x0.astype(np.float32), m, eps)
    # Positions enter the pair kernel rounded to FP32, as nb_force's do.
    ea = np.linalg.norm(s.a.cpu().numpy() - ra, axis=1) / ramag
    assert ea.max() < 1e-5


def test_time_reversible(nb, ctx, stream):
    # The force is a deterministic function of the positions, so stepping
    # back with reversed velocities returns to the start up to FP64 rounding
    # of the updates.
    n, eps, dt = 1024, np.float32(0.05), 1.0 / 128
    x0, v0, m = plummer_state(n, 7)
    s = State(x0, v0, m)
    s.step(nb, ctx, eps, dt, 20, 0, 0, stream)
    s.v.neg_()
    import torch
    torch.cuda.synchronize()
    s.step(nb, ctx, eps, dt, 20, 0, 0, stream)
    x1, v1 = s.numpy()
    assert np.abs(x1 - x0).max() < 1e-10
    assert np.abs(-v1 - v0).max() < 1e-10


def test_circular_two_body(nb, ctx, stream):
    eps = np.float32(0.0625)
    M, d = 1.0, 1.0
    vrel = np.sqrt(M * d * d / (d * d + float(eps) ** 2) ** 1.5)
    x0 = np.array([[-0.5, 0.0, 0.0], [0.5, 0.0, 0.0]])
    v0 = np.array([[0.0, -0.5 * vrel, 0.0], [0.0, 0.5 * vrel, 0.0]])
    m = np.array([0.5, 0.5], np.float32)
    period = 2 * np.pi * d / vrel
    s = State(x0, v0, m)
    s.step(nb, ctx, eps, period / 2000, 2000, 0, 0, stream)
    x1, _ = s.numpy()
    assert np.linalg.norm(x1[0] - x1[1]) == pytest.approx(1.0, abs=1e-5)
    np.testing.assert_allclose(x1, x0, atol=3e-4)


@pytest.mark.parametrize("mode", [0, 1])
def test_energy_matches_oracle(nb, ctx, stream, oracle_mod, mode):
    n, eps = 5000, np.float32(0.01)
    x, v, m = plummer_state(n, 8)
    s = State(x, v, m)
    K, W = nb.nb_energy(ctx, s.x, s.v, s.m, n, eps, mode, stream)
    Kr, Wr = oracle_mod.energy(x, v, m, eps)
    assert K == pytest.approx(Kr, rel=1e-13)
    # W from FP32-rounded positions and FP32 potentials.
    assert W == pytest.approx(Wr, rel=2e-6)


@pytest.mark.parametrize("mode", [0, 1])
def test_plummer65536_kdk16(nb, ctx, stream, mode):
    # N = 65536, eps = 1/128, 16 KDK steps of dt = 1/256, velocities from
    # the Plummer distribution function: energy drift and momentum.
    w = workloads.WORKLOADS["plummer65536_kdk16"]
    x0, v0, m = plummer_state(w["n"], w["seed"])
    eps = np.float32(w["eps"])
    s = State(x0, v0, m)
    E0 = sum(nb.nb_energy(ctx, s.x, s.v, s.m, s.n, eps, mode, stream))
    s.step(nb, ctx, eps, w["dt"], w["steps"], 0, mode, stream)
    E1 = sum(nb.nb_energy(ctx, s.x, s.v, s.m, s.n, eps, mode, stream))
    drift = abs(E1 - E0) / abs(E0)
    assert drift < 1e-4, drift
    x1, v1 = s.numpy()
    P = (m.astype(np.float64)[:, None] * v1).sum(0)
    Pscale = (m.astype(np.float64)[:, None] * np.abs(v1)).sum()
    assert np.abs(P).max() < 1e-6 * Pscale


def _force_from_fp64(nb, ctx, stream, x64, m, eps, mode):
    s = State(x64, np.zeros_like(x64), m)
    s.step(nb, ctx, eps, 0.0, 0, 0, mode, stream)   # a at the entry positions only
    return s.a.cpu().numpy().astype(np.float64), s.p.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("offset", [0.0, 1000.0])
def test_fp64_state_force_compensated_hl(nb, ctx, stream, oracle_mod, offset):
    # Positions held in FP64, the cluster centred at the origin or displaced
    # to x = 1000. Rounding them to FP32 (plain) costs u |x| absolute in every
    # x_i - x_j; the compensated path splits each position (relative to the
    # bounding box's centre) into an exact FP32 grid part and an FP32
    # remainder, so every x_i - x_j carries one rounding, and it stays within
    # 1e-6 of the FP64 oracle on the unrounded positions for every particle.
    n, eps = 65536, np.float32(1.0 / 128)
    x, _, m = workloads.plummer(n, seed=21)
    x = x + np.array([offset, 0.0, 0.0])
    m = m.astype(np.float32)
    ra, rp, ramag = oracle_mod.force(x, m, eps)
    errs = {}
    for mode in (0, 1):
        a, p = _force_from_fp64(nb, ctx, stream, x, m, eps, mode)
        ea = np.linalg.norm(a - ra, axis=1) / ramag
        ep = np.abs(p - rp) / rp
        errs[mode] = max(ea.max(), ep.max())
    assert errs[1] <= 1e-6, errs
    if offset:
        assert errs[0] > 1e-5, errs   # the rounding loss the compensated path removes


@pytest.mark.parametrize("mode", [0, 1])
def test_leapfrog_final_force_all_rows(nb, ctx, stream, oracle_mod, mode):
    # After 16 graph-replayed KDK steps (N = 8192 Plummer, eps = 1/128), the
    # force the integrator returns at its final FP64 positions against the
    # FP64 oracle at those positions, every particle: 1e-5 plain, 1e-6
    # compensated.
    n, eps, dt = 8192, np.float32(1.0 / 128), 1.0 / 256
    x0, v0, m = plummer_state(n, 24)
    s = State(x0, v0, m)
    s.step(nb, ctx, eps, dt, 16, 0, mode, stream)
    x1, _ = s.numpy()
    ra, rp, ramag = oracle_mod.force(x1, m, eps)
    a = s.a.cpu().numpy().astype(np.float64)
    p = s.p.cpu().numpy().astype(np.float64)
    ea = (np.linalg.norm(a - ra, axis=1) / ramag).max()
    ep = (np.abs(p - rp) / rp).max()
    assert max(ea, ep) <= (1e-6 if mode else 1e-5), (ea, ep)


def test_compensated_leapfrog_deterministic_and_close_to_plain(nb, ctx, stream):
    n, eps, dt = 6000, np.float32(1.0 / 64), 1.0 / 256
    x0, v0, m = plummer_state(n, 22)
    runs = []
    for _ in range(2):
        s = State(x0, v0, m)
        s.step(nb, ctx, eps, dt, 12, 0, 1, stream)
        runs.append(s)
    assert runs[0].x.cpu().numpy().tobytes() == runs[1].x.cpu().numpy().tobytes()
    assert runs[0].a.cpu().numpy().tobytes() == runs[1].a.cpu().numpy().tobytes()
    sp = State(x0, v0, m)
    sp.step(nb, ctx, eps, dt, 12, 0, 0, stream)
    assert np.abs(sp.x.cpu().numpy() - runs[0].x.cpu().numpy()).max() < 1e-8


def test_checkpoint_resume_is_bitwise(nb, ctx, stream, tmp_path):
    # The leap-frog state (x, v, a) written to disk after 10 steps and read
    # back continues exactly as the uninterrupted 16-step run.
    n, eps, dt = 4000, np.float32(1.0 / 64), 1.0 / 256
    x0, v0, m = plummer_state(n, 23)
    full = State(x0, v0, m)
    full.step(nb, ctx, eps, dt, 16, 0, 0, stream)
    part = State(x0, v0, m)
    part.step(nb, ctx, eps, dt, 10, 0, 0, stream)
    ckpt = tmp_path / "state.npz"
    np.savez(ckpt, x=part.x.cpu().numpy(), v=part.v.cpu().numpy(), a=part.a.cpu().numpy(), m=m)
    z = np.load(ckpt)
    resumed = State(z["x"], z["v"], z["m"])
    import torch
    resumed.a.copy_(torch.from_numpy(z["a"]))
    torch.cuda.synchronize()
    resumed.step(nb, ctx, eps, dt, 6, 1, 0, stream)
    for u, w in ((full.x, resumed.x), (full.v, resumed.v), (full.a, resumed.a)):
        assert u.cpu().numpy().tobytes() == w.cpu().numpy().tobytes()

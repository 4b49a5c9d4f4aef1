#!/usr/bin/env python
"""Benchmark of the direct-summation gravity path on GB300.

One step = one nb_force call (pack -> pair kernel -> combine) evaluating
Eq. (gravity) (Fujiwara & Nakasato, arXiv:0904.3659) for a Plummer sphere of
N = 2^20 particles, eps = 1/256, FP32, inputs resident in HBM. The headline
value is interactions per second (N^2 per step, the paper's convention) of
the plain path; the compensated path is timed right after it on the same
inputs. Gflop/s are also given at the paper's 38 flop per interaction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica of the same workload
(the computation needs no exchange), so scaling is weak and the value is the
sum over ranks divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle on a bounded sample of rows of the
same workload on the host cores (the reference arm for this project; the
paper's own RV770/CAL code is not available).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = "plummer1m"
FLOP_PER_INT_PAPER = 38          # the paper's convention (Section "Experiments")
FP32_LANES_PER_SM = 128          # FP32 lanes per SM per clock
MUFU_PER_INT = 1
# The earlier built-in large-N shape, with the Newton step, timed beside the
# headline (what the step costs).
NEWTON_TILE = (128, 8, 256, 3, 8, 1, 1, 0, 63, 1, 0)


def fp32_ops_per_interaction(tile) -> int:
    """FP32 pipe operations per interaction of a pair-kernel tile: 13 with the
    special-function unit's rsqrt used as is, 16 with one Newton step."""
    return 16 if tile[9] else 13


def alu_peak(sm_count, sm_mhz, ops) -> float:
    """Interactions per second with every FP32 lane busy (G-int/s)."""
    return sm_count * sm_mhz * 1e6 * FP32_LANES_PER_SM / ops / 1e9


# DRAM bytes (read + write) of one launch of the large-N plain pair kernel
# (256 threads x 4 i, 1024-particle tiles), from an ncu capture of that
# kernel alone on a Plummer sphere of N = 131072 (4.215 MB read, 0 written).
# The kernel reads each j-tile from L2 after its first touch, so DRAM traffic
# grows with N, not N^2; the bench reports it scaled to its N, and null for
# any other tile shape.
PROFILED_TILE = (256, 4, 1024, 3, 4, 1, 0, 0, 63, 0, 0)
PROFILED_DRAM_BYTES, PROFILED_N = 4.215e6, 131072


# --------------------------------------------------------------------------
# host-side helpers (no GPU needed; covered by tests/test_bench_host.py)

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    """Max of a float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(per_rank_units: float, world: int, ms_per_step_max: float) -> float:
    """Whole-job rate: units all ranks processed per second of the slowest rank."""
    return per_rank_units * world / (ms_per_step_max * 1e-3)


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int = 0, period_ms: int = 200):
        self.gpu_index = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self._t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", f"-lms={self.period_ms}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self._t is not None:
                self._t.join(timeout=2)

    def summary(self):
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [s.strip() for s in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for k, nm in enumerate(names):
            if f[5 + k].lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    # Under load: samples above 30% of max (the first/last samples can be idle).
    top = max(smax) if smax else max(sm)
    loaded = [v for v in sm if v > 0.3 * top] or sm
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": top,
            "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


# --------------------------------------------------------------------------
# inputs

def make_inputs(n, seed):
    x, _, m = workloads.plummer(n, seed=seed)
    return np.ascontiguousarray(x.astype(np.float32)), np.ascontiguousarray(m.astype(np.float32))


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of rows

def cpu_oracle_rate(x32, m32, eps, target_s=12.0, rows_seed=2, min_rows=64,
                    extra_rows=None):
    """Time oracle.force_rows on a sample of rows sized for about target_s
    seconds. Returns (rate in interactions/s, dict describing the sample,
    oracle results for extra_rows if given)."""
    import oracle
    n = x32.shape[0]
    cores = oracle.num_threads()
    rows = workloads.sample_rows(n, min_rows, seed=rows_seed + 1000)
    t0 = time.perf_counter()
    oracle.force_rows(x32, m32, eps, rows)
    dt = max(time.perf_counter() - t0, 1e-3)
    k = int(min(n, max(min_rows, min_rows * target_s / dt)))
    rows = workloads.sample_rows(n, k, seed=rows_seed + 1000)
    t0 = time.perf_counter()
    oracle.force_rows(x32, m32, eps, rows)
    dt = time.perf_counter() - t0
    rate = k * n / dt
    extra = None
    if extra_rows is not None:
        extra = oracle.force_rows(x32, m32, eps, extra_rows)
    return rate, {"rows": int(k), "n": int(n), "seconds": dt, "cores": cores}, extra


def oracle_errors(a, p, ref):
    ra, rp, ramag = ref
    ea = np.linalg.norm(a.astype(np.float64) - ra, axis=1) / ramag
    ep = np.abs(p.astype(np.float64) - rp) / rp
    return {"max_rel_a": float(ea.max()), "max_rel_p": float(ep.max()),
            "median_rel_a": float(np.median(ea)), "median_rel_p": float(np.median(ep))}


# --------------------------------------------------------------------------
# the other workloads, reported beside the headline (each a dict)

def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def extra_leapfrog(nb, ctx, dev, torch, oracle_ref=False):
    """N = 65536 Plummer, eps = 1/128: 16 KDK steps of dt = 1/256 (graph
    replayed), plain and compensated; energy drift and momentum. With
    oracle_ref the final states are kept (under "_state") for
    leapfrog_oracle_error."""
    w = workloads.WORKLOADS["plummer65536_kdk16"]
    x0, v0, m = workloads.plummer(w["n"], seed=w["seed"])
    n, eps, dt, steps = w["n"], np.float32(w["eps"]), w["dt"], w["steps"]
    stream = torch.cuda.Stream(dev)
    out = {"workload": "plummer65536_kdk16", "n": n, "steps": steps, "_state": {}}
    for mode, name in ((nb.NB_PLAIN, "plain"), (nb.NB_COMPENSATED, "compensated")):
        x = torch.from_numpy(x0.copy()).to(dev)
        v = torch.from_numpy(v0.copy()).to(dev)
        mt = torch.from_numpy(m.astype(np.float32)).to(dev)
        a = torch.zeros((n, 3), dtype=torch.float32, device=dev)
        p = torch.zeros(n, dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)
        E0 = sum(nb.nb_energy(ctx, x, v, mt, n, eps, mode, stream))
        P0 = (torch.from_numpy(m)[:, None] * torch.from_numpy(v0)).sum(0).numpy()
        nb.nb_leapfrog_step(ctx, x, v, mt, a, p, n, eps, dt, 0, 0, mode, stream)  # a(t0)
        e0, e1 = _events(torch)
        e0.record(stream)
        # The integrator needs only a: without p the kernels leave the potential out.
        nb.nb_leapfrog_step(ctx, x, v, mt, a, None, n, eps, dt, steps, 1, mode, stream)
        e1.record(stream)
        nb.nb_synchronize(ctx, stream)
        ms = e0.elapsed_time(e1)
        E1 = sum(nb.nb_energy(ctx, x, v, mt, n, eps, mode, stream))
        v1 = v.cpu().numpy()
        P1 = (m[:, None] * v1).sum(0)
        out[name] = {"ms_per_step": ms / steps, "gint_s": n * n * steps / (ms * 1e-3) / 1e9,
                     "rel_energy_drift": abs(E1 - E0) / abs(E0),
                     "momentum_change": float(np.abs(P1 - P0).max()),
                     "momentum_scale": float((m[:, None] * np.abs(v1)).sum())}
        if oracle_ref:
            out["_state"][name] = (x.cpu().numpy(), v1, a.cpu().numpy())
    return out


def leapfrog_oracle_error(lf):
    """The leap-frog block's results against the FP64 oracle's own 16 steps
    from the same initial state (Eqs. (1)-(3) with Eq. (gravity)): position
    and velocity differences after the last step, and the returned force
    against the oracle's at the GPU's final positions, every particle (e_a
    relative to A_i)."""
    import oracle
    w = workloads.WORKLOADS["plummer65536_kdk16"]
    x0, v0, m = workloads.plummer(w["n"], seed=w["seed"])
    m = m.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    xr, vr, _ = oracle.leapfrog(x0, v0, m, w["eps"], w["dt"], w["steps"])
    secs = time.perf_counter() - t0
    v_scale = float(np.sqrt((vr ** 2).sum(1).mean()))
    for name, (x, v, a) in lf.pop("_state").items():
        dx = np.linalg.norm(x - xr, axis=1)
        dv = np.linalg.norm(v - vr, axis=1)
        ra, _, ramag = oracle.force(x, m, w["eps"])
        ea = np.linalg.norm(a.astype(np.float64) - ra, axis=1) / ramag
        lf[name]["oracle_error"] = {
            "max_abs_dx": float(dx.max()), "max_abs_dv": float(dv.max()),
            "max_dv_over_v_rms": float(dv.max() / v_scale),
            "final_force_max_rel_a": float(ea.max()), "final_force_median_rel_a": float(np.median(ea)),
            "reference": f"oracle.leapfrog, FP64, {w['steps']} steps, {secs:.1f} s; "
                         "force: oracle.force at the GPU's final positions, every particle"}


def extra_batched(nb, ctx, dev, torch, plain_rate, oracle_ref=False):
    """1024 clusters (N log-uniform in [32, 4096]): one nb_force_batched
    launch (plain and compensated), and 32 graph-replayed batched KDK steps
    in each mode. With oracle_ref the results are kept (under "_state") for
    batched_oracle_error."""
    w = workloads.WORKLOADS["clusters1024_kdk32"]
    cl = workloads.clusters(w["n_clusters"], seed=w["seed"], nmin=w["nmin"], nmax=w["nmax"])
    n, C = cl.x.shape[0], len(cl.sizes)
    pairs = float((cl.sizes.astype(np.float64) ** 2).sum())
    x = torch.from_numpy(cl.x.astype(np.float32)).to(dev)
    mt = torch.from_numpy(cl.m.astype(np.float32)).to(dev)
    off = torch.from_numpy(cl.offsets).to(dev)
    eps = torch.from_numpy(cl.eps.astype(np.float32)).to(dev)
    a = torch.empty((n, 3), device=dev)
    p = torch.empty(n, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    out = {"workload": "clusters1024_kdk32", "clusters": C, "particles": n,
           "interactions_per_eval": pairs, "_state": {}}
    for mode, name in ((nb.NB_PLAIN, "plain"), (nb.NB_COMPENSATED, "compensated")):
        for _ in range(3):
            nb.nb_force_batched(ctx, x, mt, off, C, n, eps, a, p, mode, stream)
        reps = 10
        e0, e1 = _events(torch)
        e0.record(stream)
        for _ in range(reps):
            nb.nb_force_batched(ctx, x, mt, off, C, n, eps, a, p, mode, stream)
        e1.record(stream)
        nb.nb_synchronize(ctx, stream)
        ms = e0.elapsed_time(e1) / reps
        rate = pairs / (ms * 1e-3) / 1e9
        eval_state = (a.cpu().numpy(), p.cpu().numpy())
        x64 = torch.from_numpy(cl.x.copy()).to(dev)
        v64 = torch.from_numpy(cl.v.copy()).to(dev)
        torch.cuda.synchronize(dev)
        steps = w["steps"]
        nb.nb_leapfrog_batched_step(ctx, x64, v64, mt, off, C, n, eps, a, p, w["dt"], 0, 0,
                                    mode, stream)
        e0, e1 = _events(torch)
        e0.record(stream)
        nb.nb_leapfrog_batched_step(ctx, x64, v64, mt, off, C, n, eps, a, p, w["dt"], steps, 1,
                                    mode, stream)
        e1.record(stream)
        nb.nb_synchronize(ctx, stream)
        ms_lf = e0.elapsed_time(e1)
        out[name] = {"ms_per_eval": ms, "gint_s": rate,
                     "fraction_of_plain_rate": rate / plain_rate,
                     "kdk32_ms_per_step": ms_lf / steps,
                     "kdk32_gint_s": pairs * steps / (ms_lf * 1e-3) / 1e9}
        if oracle_ref:
            out["_state"][name] = (eval_state, (x64.cpu().numpy(), a.cpu().numpy(), p.cpu().numpy()))
    out["compensated"]["slowdown_vs_plain"] = out["compensated"]["ms_per_eval"] / out["plain"]["ms_per_eval"]
    out["compensated"]["kdk32_slowdown_vs_plain"] = (out["compensated"]["kdk32_ms_per_step"]
                                                     / out["plain"]["kdk32_ms_per_step"])
    return out


def _cluster_errors(xs, m, offsets, eps, a, p):
    """Max over every particle of every cluster of e_a (relative to A_i) and
    e_p against oracle.force on that cluster alone."""
    import oracle
    wa = wp = 0.0
    for c in range(len(offsets) - 1):
        lo, hi = int(offsets[c]), int(offsets[c + 1])
        if hi == lo:
            continue
        ra, rp, ramag = oracle.force(xs[lo:hi], m[lo:hi], eps[c])
        wa = max(wa, float((np.linalg.norm(a[lo:hi].astype(np.float64) - ra, axis=1) / ramag).max()))
        wp = max(wp, float((np.abs(p[lo:hi].astype(np.float64) - rp) / rp).max()))
    return {"max_rel_a": wa, "max_rel_p": wp}


def batched_oracle_error(bt):
    """The batched block's results against the FP64 oracle, every particle of
    every cluster: the single evaluation on the FP32 inputs, and the force the
    32-step KDK returns at its final FP64 positions (the oracle evaluated at
    those same positions)."""
    w = workloads.WORKLOADS["clusters1024_kdk32"]
    cl = workloads.clusters(w["n_clusters"], seed=w["seed"], nmin=w["nmin"], nmax=w["nmax"])
    x32, m32 = cl.x.astype(np.float32), cl.m.astype(np.float32)
    eps32 = cl.eps.astype(np.float32)
    t0 = time.perf_counter()
    for name, ((ea, ep), (xk, ak, pk)) in bt.pop("_state").items():
        bt[name]["oracle_error"] = {
            "eval": _cluster_errors(x32, m32, cl.offsets, eps32, ea, ep),
            "kdk32_final_force": _cluster_errors(xk, m32, cl.offsets, eps32, ak, pk)}
    bt["oracle_seconds"] = time.perf_counter() - t0


def extra_single_call(nb, ctx, dev, torch):
    """N = 4096 Plummer, eps = 0.01: one nb_force call, launched directly 200
    times back to back, and replayed from a captured CUDA graph of 20 calls
    (10 replays; one graph launch per call would time the host's graph
    launch, not the device). The results are returned under "_results" for
    the oracle comparison of the cpu_baseline leg."""
    w = workloads.WORKLOADS["plummer4096"]
    n, eps = w["n"], np.float32(w["eps"])
    x0, _, m = workloads.plummer(n, seed=w["seed"])
    x32, m32 = x0.astype(np.float32), m.astype(np.float32)
    x = torch.from_numpy(x32).to(dev)
    mt = torch.from_numpy(m32).to(dev)
    a = torch.empty((n, 3), device=dev)
    p = torch.empty(n, device=dev)
    out = {"workload": "plummer4096", "n": n, "_results": {"x": x32, "m": m32, "eps": eps}}
    for mode, name in ((nb.NB_PLAIN, "plain"), (nb.NB_COMPENSATED, "compensated")):
        nb.nb_reserve(ctx, n, mode)                # no allocation inside the capture
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(10):
                nb.nb_force(ctx, x, mt, n, eps, a, p, mode, side)
        torch.cuda.current_stream(dev).wait_stream(side)
        per_graph = 20
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(per_graph):
                nb.nb_force(ctx, x, mt, n, eps, a, p, mode)
        graph.replay()
        reps = 200
        times = {}
        for how in ("direct", "graph"):
            e0, e1 = _events(torch)
            e0.record()
            if how == "direct":
                for _ in range(reps):
                    nb.nb_force(ctx, x, mt, n, eps, a, p, mode)
            else:
                for _ in range(reps // per_graph):
                    graph.replay()
            e1.record()
            nb.nb_synchronize(ctx)
            times[how] = e0.elapsed_time(e1) / reps * 1e3
        out["_results"][name] = (a.cpu().numpy(), p.cpu().numpy())
        out[name] = {"us_per_call": times["direct"], "us_per_call_graph": times["graph"],
                     "gint_s": n * n / (times["direct"] * 1e-6) / 1e9,
                     "gint_s_graph": n * n / (times["graph"] * 1e-6) / 1e9,
                     "tile": list(nb.nb_get_tile(ctx, n, mode).as_tuple())}
    return out


def extra_mid_call(nb, ctx, dev, torch):
    """N = 12288 Plummer (seed 0), eps = 0.01: one nb_force call in the range
    of the stream-K single-launch kernel, launched directly."""
    n, eps = 12288, np.float32(0.01)
    x0, _, m = workloads.plummer(n, seed=0)
    x = torch.from_numpy(x0.astype(np.float32)).to(dev)
    mt = torch.from_numpy(m.astype(np.float32)).to(dev)
    a = torch.empty((n, 3), device=dev)
    p = torch.empty(n, device=dev)
    out = {"workload": "plummer12288", "n": n}
    for mode, name in ((nb.NB_PLAIN, "plain"), (nb.NB_COMPENSATED, "compensated")):
        for _ in range(5):
            nb.nb_force(ctx, x, mt, n, eps, a, p, mode)
        reps = 100
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(reps):
            nb.nb_force(ctx, x, mt, n, eps, a, p, mode)
        e1.record()
        nb.nb_synchronize(ctx)
        us = e0.elapsed_time(e1) / reps * 1e3
        out[name] = {"us_per_call": us, "gint_s": n * n / (us * 1e-6) / 1e9,
                     "tile": list(nb.nb_get_tile(ctx, n, mode).as_tuple())}
    return out


def extra_adjoint(nb, ctx, dev, torch, plain_rate, oracle_ref=False):
    """N = 16384 Plummer, eps = 1/64: the VJP pair kernel's rate, and one
    64-step differentiable trajectory (forward + backward, checkpoints every 8)."""
    from paper_0904_3659_gb300.autograd import leapfrog
    w = workloads.WORKLOADS["plummer16384_adjoint64"]
    n, eps = w["n"], np.float32(w["eps"])
    x0, v0, m = workloads.plummer(n, seed=w["seed"])
    rng = np.random.default_rng(5)
    x = torch.from_numpy(x0.astype(np.float32)).to(dev)
    mt = torch.from_numpy(m.astype(np.float32)).to(dev)
    ga = torch.from_numpy(rng.normal(size=(n, 3)).astype(np.float32)).to(dev)
    gp = torch.from_numpy(rng.normal(size=n).astype(np.float32)).to(dev)
    gx = torch.empty((n, 3), device=dev)
    gm = torch.empty(n, device=dev)
    a = torch.empty((n, 3), device=dev)
    p = torch.empty(n, device=dev)
    for _ in range(3):
        nb.nb_force_vjp(ctx, x, mt, n, eps, ga, gp, gx, gm)
        nb.nb_force(ctx, x, mt, n, eps, a, p)
    reps = 20
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(reps):
        nb.nb_force_vjp(ctx, x, mt, n, eps, ga, gp, gx, gm)
    e1.record()
    f0, f1 = _events(torch)
    f0.record()
    for _ in range(reps):
        nb.nb_force(ctx, x, mt, n, eps, a, p)
    f1.record()
    # The trajectory adjoint's case: no upstream gradient on p (26 instead of
    # 28 FP32 operations per pair).
    for _ in range(3):
        nb.nb_force_vjp(ctx, x, mt, n, eps, ga, None, gx, gm)
    g0, g1 = _events(torch)
    g0.record()
    for _ in range(reps):
        nb.nb_force_vjp(ctx, x, mt, n, eps, ga, None, gx, gm)
    g1.record()
    nb.nb_force_vjp(ctx, x, mt, n, eps, ga, gp, gx, gm)  # gx, gm with gp again (oracle check)
    nb.nb_synchronize(ctx)
    vjp_ms = e0.elapsed_time(e1) / reps
    fwd_ms = f0.elapsed_time(f1) / reps
    vjp_nogp_ms = g0.elapsed_time(g1) / reps
    xt = torch.from_numpy(x0.copy()).to(dev).requires_grad_(True)
    vt = torch.from_numpy(v0.copy()).to(dev).requires_grad_(True)
    mg = torch.from_numpy(m.astype(np.float32)).to(dev).requires_grad_(True)
    yt = torch.from_numpy(workloads.targets(x0, seed=w["target_seed"])).to(dev)
    times = []
    for _ in range(2):  # the first pass includes one-time set-up
        xt.grad = vt.grad = mg.grad = None
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        xT, _ = leapfrog(xt, vt, mg, eps, w["dt"], w["steps"], checkpoint_every=w["checkpoint"],
                         nbctx=ctx)
        ((xT - yt) ** 2).sum().backward()
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0)
    traj_s = times[-1]
    out = {"workload": "plummer16384_adjoint64", "n": n,
           "vjp_ms": vjp_ms, "vjp_gpair_s": n * n / (vjp_ms * 1e-3) / 1e9,
           "vjp_without_gp_ms": vjp_nogp_ms,
           "vjp_without_gp_gpair_s": n * n / (vjp_nogp_ms * 1e-3) / 1e9,
           "forward_ms_same_n": fwd_ms,
           "vjp_fraction_of_plain_rate": (n * n / (vjp_ms * 1e-3) / 1e9) / plain_rate,
           "trajectory_grad_s": traj_s, "trajectory_grad_first_s": times[0]}
    if oracle_ref:
        out["_state"] = {"vjp": (gx.cpu().numpy(), gm.cpu().numpy(), ga.cpu().numpy(),
                                 gp.cpu().numpy()),
                         "grads": {"x": xt.grad.cpu().numpy(), "v": vt.grad.cpu().numpy(),
                                   "m": mg.grad.cpu().numpy().astype(np.float64)}}
    return out


ADJOINT_FD = os.path.join(ROOT, "tests", "golden", "adjoint_fd_plummer16384.txt")


def read_adjoint_fd(path=ADJOINT_FD):
    """The stored FP64 finite differences of the differentiation workload
    (written by tests/golden/make_adjoint_fd.py from the oracle):
    [(kind, i, c, h, fd, adjoint)]."""
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, i, c, h, fd, g = line.split()
            rows.append((k, int(i), int(c), float(h), float(fd), float(g)))
    return rows


def vjp_term_scales_rows(x, m, eps, ga, gp, rows):
    """For the listed particles k, the sums over l != k of the magnitudes of
    the terms of gx_k and gm_k (the VJP's analogue of A_i: the sums cancel
    strongly, so |g_ref| itself is no scale)."""
    x = np.asarray(x, np.float64)
    m = np.asarray(m, np.float64)
    ga = np.asarray(ga, np.float64)
    gp = np.asarray(gp, np.float64)
    e2 = float(np.float32(eps)) ** 2
    nga = np.linalg.norm(ga, axis=1)
    sx, sm = np.zeros(rows.size), np.zeros(rows.size)
    for t, k in enumerate(rows):
        r = x[k] - x
        r2 = (r * r).sum(1)
        y = 1.0 / np.sqrt(r2 + e2)
        y[k] = 0.0
        y3, y5, rn = y ** 3, y ** 5, np.sqrt(r2)
        rgk = np.abs(r @ ga[k])
        rgl = np.abs((r * ga).sum(1))
        sx[t] = (m * (y3 * nga[k] + 3 * y5 * rgk * rn + abs(gp[k]) * y3 * rn)).sum() + \
            m[k] * (y3 * nga + 3 * y5 * rgl * rn + np.abs(gp) * y3 * rn).sum()
        sm[t] = (rgl * y3 + np.abs(gp) * y).sum()
    return sx, sm


def adjoint_oracle_error(adj):
    """The adjoint block against the FP64 oracle: the VJP kernel on 512
    sampled rows (error relative to the sum of term magnitudes), and the
    trajectory gradient on the 32 stored finite-difference coordinates and,
    for every coordinate, against the oracle's reverse-mode gradient."""
    import oracle
    w = workloads.WORKLOADS["plummer16384_adjoint64"]
    n, eps = w["n"], np.float32(w["eps"])
    st = adj.pop("_state")
    t0 = time.perf_counter()
    x0, v0, m = workloads.plummer(n, seed=w["seed"])
    x32, m32 = x0.astype(np.float32), m.astype(np.float32)
    gx, gm, ga, gp = st["vjp"]
    rows = workloads.sample_rows(n, 512, seed=6)
    rgx, rgm = oracle.force_vjp(x32, m32, eps, ga, gp, rows=rows)
    sx, sm = vjp_term_scales_rows(x32, m32, eps, ga, gp, rows)
    vjp_err = {"rows": int(rows.size),
               "max_rel_gx": float((np.linalg.norm(gx[rows] - rgx, axis=1) / sx).max()),
               "max_rel_gm": float((np.abs(gm[rows] - rgm) / sm).max())}
    g = st["grads"]
    fd_rows = read_adjoint_fd()
    rel = []
    for kind, i, c, h, fd, _ in fd_rows:
        v = float(g[kind][i] if kind == "m" else g[kind][i, c])
        rel.append(abs(v - fd) / abs(fd))
    m64 = m32.astype(np.float64)
    y = workloads.targets(x0, seed=w["target_seed"])
    xT, _, _ = oracle.leapfrog(x0, v0, m64, eps, w["dt"], w["steps"])
    ref = dict(zip("xvm", oracle.leapfrog_grad(x0, v0, m64, eps, w["dt"], w["steps"], 2 * (xT - y))))
    every = {}
    for kind in "xvm":
        r = ref[kind]
        e = np.abs(g[kind] - r) / np.maximum(np.abs(r), 1e-3 * np.abs(r).max())
        every[kind] = {"max": float(e.max()), "p99_9": float(np.percentile(e, 99.9))}
    adj["oracle_error"] = {
        "vjp": vjp_err,
        "trajectory_fd": {"coords": len(rel), "max_rel": float(max(rel)),
                          "median_rel": float(np.median(rel)),
                          "reference": "tests/golden/adjoint_fd_plummer16384.txt (FP64 central "
                                       "differences of the oracle's trajectory)"},
        "trajectory_every_coordinate": every,
        "seconds": time.perf_counter() - t0}


# --------------------------------------------------------------------------
# our arm

def run_ours(args):
    import torch
    import paper_0904_3659_gb300 as nb

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    w = workloads.WORKLOADS[WORKLOAD]
    n, eps = (args.n or w["n"]), np.float32(w["eps"])
    x32, m32 = make_inputs(n, w["seed"])
    xt = torch.from_numpy(x32).to(dev)
    mt = torch.from_numpy(m32).to(dev)
    a = torch.empty((n, 3), dtype=torch.float32, device=dev)
    p = torch.empty((n,), dtype=torch.float32, device=dev)
    ctx = nb.Context(dev.index)
    stream = torch.cuda.current_stream(dev)

    # Tile choice: tune on a quarter-size proxy (same inner loop; the
    # persistent split balances the full size), then record it for N's size
    # class only (the other workloads keep the shapes of their own sizes).
    tiles = {}
    for mode in ((nb.NB_PLAIN,) if args.plain_only else (nb.NB_PLAIN, nb.NB_COMPENSATED)):
        fixed = args.tile if mode == nb.NB_PLAIN else args.tile_comp
        if fixed:
            nb.nb_set_tuned_tile(ctx, n, mode, tuple(int(v) for v in fixed.split(",")))
        elif args.tile_tune:
            t, _ = nb.nb_autotune(ctx, max(n // 4, 1024), mode)
            nb.nb_set_tuned_tile(ctx, n, mode, t)
        tiles[mode] = nb.nb_get_tile(ctx, n, mode)
        nb.nb_reserve(ctx, n, mode)

    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    def timed(mode, steps, warmup, n=n, xt=xt, mt=mt, a=a, p=p):
        for _ in range(warmup):
            nb.nb_force(ctx, xt, mt, n, eps, a, p, mode, stream)
        nb.nb_synchronize(ctx, stream)
        nb.nb_timing_enable(ctx, True)
        nb.nb_timing_reset(ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize(dev)
        for k in range(steps):
            flush_buf.fill_(float(k))          # L2 flush between timed steps (untimed)
            ev[k][0].record(stream)
            nb.nb_force(ctx, xt, mt, n, eps, a, p, mode, stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        nb.nb_synchronize(ctx, stream)
        step_ms = [s.elapsed_time(e) for s, e in ev]
        kernels = {name: nb.nb_timing_read(ctx, kid) for name, kid in
                   (("pack", nb.KERNEL_PACK), ("pair", nb.KERNEL_PAIR),
                    ("combine", nb.KERNEL_REDUCE))}
        nb.nb_timing_enable(ctx, False)
        return step_ms, kernels

    with ClockSampler(dev.index) as clk:
        plain_ms, plain_k = timed(nb.NB_PLAIN, args.steps, args.warmup)
        a_plain = a.cpu().numpy()
        p_plain = p.cpu().numpy()
        if args.plain_only:
            comp_ms, comp_k = plain_ms, plain_k
            a_comp, p_comp = a_plain, p_plain
        else:
            comp_ms, comp_k = timed(nb.NB_COMPENSATED, args.steps, args.warmup)
            a_comp = a.cpu().numpy()
            p_comp = p.cpu().numpy()
        newton = None
        if args.newton_arm and tuple(tiles[nb.NB_PLAIN].as_tuple()) != NEWTON_TILE:
            # The same work with the Newton step on the reciprocal square root.
            nb.nb_set_tile(ctx, nb.NB_PLAIN, NEWTON_TILE)
            newton_ms, newton_k = timed(nb.NB_PLAIN, args.steps, args.warmup)
            newton = (newton_ms, newton_k, a.cpu().numpy(), p.cpu().numpy())
            nb.nb_set_tile(ctx, nb.NB_PLAIN, None)
    clocks = clk.summary()

    ms_plain = max_over_ranks(sum(plain_ms) / len(plain_ms), world)
    ms_comp = max_over_ranks(sum(comp_ms) / len(comp_ms), world)
    interactions = float(n) * float(n)
    value = aggregate(interactions, world, ms_plain)
    value_comp = aggregate(interactions, world, ms_comp)

    # End to end through the public C ABI with host buffers (pinned), copies
    # inside the timed region.
    hx = torch.from_numpy(x32).pin_memory()
    hm = torch.from_numpy(m32).pin_memory()
    ha = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    hp = torch.empty((n,), dtype=torch.float32).pin_memory()
    for _ in range(max(1, min(args.warmup, 2)) if args.e2e else 0):
        nb.nb_force_host(ctx, hx.data_ptr(), hm.data_ptr(), n, eps, ha.data_ptr(), hp.data_ptr(),
                         nb.NB_PLAIN, stream)
    barrier(world)
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3)) if args.e2e else 0):
        t0 = time.perf_counter()
        nb.nb_force_host(ctx, hx.data_ptr(), hm.data_ptr(), n, eps, ha.data_ptr(), hp.data_ptr(),
                         nb.NB_PLAIN, stream)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    barrier(world)
    e2e_ms_max = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world) if e2e_ms else float("nan")

    # Roofline of the dominant kernel (the pair kernel): FP32 pipe bound.
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = (peaks or {}).get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0
    pair_ms_total, pair_launches = plain_k["pair"]
    pair_ms = pair_ms_total / max(pair_launches, 1)
    achieved = interactions / (pair_ms * 1e-3) / 1e9                     # G-int/s
    plain_tile = tuple(tiles[nb.NB_PLAIN].as_tuple())
    ops = fp32_ops_per_interaction(plain_tile)
    peak = alu_peak(sm_count, sm_max_mhz, ops)
    comp_pair_ms = comp_k["pair"][0] / max(comp_k["pair"][1], 1)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return None

    out = {
        "metric": "G-interactions/s and % FP32/MUFU roofline at N=2^20 vs FP64-oracle error",
        "value": value / 1e9,
        "unit": "G-int/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_plain,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic Plummer sphere (seed 0), float32",
        "config": {"workload": WORKLOAD if n == w["n"] else f"plummer n={n} (small case)",
                   "n": n, "eps": float(eps), "mode": "plain",
                   "tile": list(tiles[nb.NB_PLAIN].as_tuple()),
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "gflops_38": value * FLOP_PER_INT_PAPER / 1e9,
        "compensated": {"value": value_comp / 1e9, "unit": "G-int/s", "ms_per_step": ms_comp,
                        "slowdown_vs_plain": ms_comp / ms_plain,
                        "tile": list(tiles.get(nb.NB_COMPENSATED, tiles[nb.NB_PLAIN]).as_tuple()),
                        "gpu_launches": sum(v[1] for v in comp_k.values()),
                        "pair_ms": comp_pair_ms},
        "kernels_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in plain_k.items()},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G-int/s",
                     "frac": achieved / peak,
                     "traffic": (PROFILED_DRAM_BYTES * n / PROFILED_N
                                 if plain_tile == PROFILED_TILE else None),
                     "traffic_note": "DRAM bytes per launch, ncu capture at N=131072 scaled by N",
                     "basis": (f"{sm_count} SMs x {sm_max_mhz:.0f} MHz x {FP32_LANES_PER_SM} FP32 "
                               f"lanes / {ops} FP32 ops per interaction "
                               f"(+{MUFU_PER_INT} MUFU rsqrt, not binding); sm_max_mhz of "
                               f"{'measured' if peaks else 'nvidia-smi'} peaks"),
                     "fp32_ops_per_interaction": ops},
        "e2e": ({"value": interactions * world / (e2e_ms_max * 1e-3) / 1e9, "unit": "G-int/s",
                 "h2d_bytes_per_step": int(x32.nbytes + m32.nbytes),
                 "d2h_bytes_per_step": int(4 * n * 3 + 4 * n)} if e2e_ms else None),
        "gpu_launches": sum(v[1] for v in plain_k.values()),
        "clocks": clocks,
    }
    if newton is not None:
        newton_ms, newton_k = newton[0], newton[1]
        n_ms = max_over_ranks(sum(newton_ms) / len(newton_ms), world)
        n_pair_ms = newton_k["pair"][0] / max(newton_k["pair"][1], 1)
        n_achieved = interactions / (n_pair_ms * 1e-3) / 1e9
        n_peak = alu_peak(sm_count, sm_max_mhz, 16)
        out["newton_step"] = {"tile": list(NEWTON_TILE), "value": aggregate(interactions, world, n_ms) / 1e9,
                              "unit": "G-int/s", "ms_per_step": n_ms, "pair_ms": n_pair_ms,
                              "roofline_frac": n_achieved / n_peak, "roofline_peak": n_peak,
                              "fp32_ops_per_interaction": 16,
                              "speedup_without_step": n_ms / ms_plain}
    if args.extras:
        plain_rate = value / world / 1e9
        ref = not args.no_cpu_baseline
        for key, fn in (("single_call", lambda: extra_single_call(nb, ctx, dev, torch)),
                        ("mid_call", lambda: extra_mid_call(nb, ctx, dev, torch)),
                        ("leapfrog", lambda: extra_leapfrog(nb, ctx, dev, torch, ref)),
                        ("batched", lambda: extra_batched(nb, ctx, dev, torch, plain_rate, ref)),
                        ("adjoint", lambda: extra_adjoint(nb, ctx, dev, torch, plain_rate, ref))):
            try:
                out[key] = fn()
            except Exception as e:  # reported in the line, the headline stands
                out[key] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_cpu_baseline:
        rows = workloads.sample_rows(n, w["sample"], w["sample_seed"])
        rate, sample, ref = cpu_oracle_rate(x32, m32, eps, target_s=args.cpu_seconds,
                                            extra_rows=rows)
        out["cpu_baseline"] = {"value": rate / 1e9, "unit": "G-int/s", "cores": sample["cores"],
                               "kind": "oracle",
                               "sample": (f"{sample['rows']} random rows x all {n} j of the same "
                                          f"workload, FP64, {sample['seconds']:.1f} s")}
        # The same oracle on one host core (a short sample of its own).
        import oracle
        threads = oracle.num_threads()
        oracle.set_num_threads(1)
        try:
            rate1, sample1, _ = cpu_oracle_rate(x32, m32, eps, target_s=min(3.0, args.cpu_seconds),
                                                min_rows=8)
        finally:
            oracle.set_num_threads(threads)
        out["cpu_baseline"]["one_core"] = {
            "value": rate1 / 1e9, "unit": "G-int/s", "cores": 1,
            "sample": f"{sample1['rows']} random rows x all {n} j, FP64, {sample1['seconds']:.1f} s"}
        out["oracle_error"] = {"rows": int(rows.size),
                               "plain": oracle_errors(a_plain[rows], p_plain[rows], ref),
                               "compensated": oracle_errors(a_comp[rows], p_comp[rows], ref)}
        if newton is not None:
            out["newton_step"]["oracle_error"] = oracle_errors(newton[2][rows], newton[3][rows], ref)
        single = out.get("single_call", {}).get("_results")
        if single is not None:
            import oracle
            ref4 = oracle.force(single["x"], single["m"], single["eps"])
            for name in ("plain", "compensated"):
                out["single_call"][name]["oracle_error_all_rows"] = oracle_errors(*single[name], ref4)
        # The FP64 oracle's error for the other workloads' results.
        for key, fn in (("leapfrog", leapfrog_oracle_error), ("batched", batched_oracle_error),
                        ("adjoint", adjoint_oracle_error)):
            blk = out.get(key, {})
            if "_state" in blk:
                try:
                    fn(blk)
                except Exception as e:  # reported in the line, the headline stands
                    blk["oracle_error"] = {"error": f"{type(e).__name__}: {e}"}
    out.get("single_call", {}).pop("_results", None)
    for key in ("leapfrog", "batched", "adjoint"):
        out.get(key, {}).pop("_state", None)
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


# --------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores

def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    w = workloads.WORKLOADS[WORKLOAD]
    n, eps = w["n"], np.float32(w["eps"])
    x32, m32 = make_inputs(n, w["seed"])
    cores = oracle.num_threads()
    # Rows per step sized for about two seconds of oracle work.
    probe = workloads.sample_rows(n, 32, seed=11)
    t0 = time.perf_counter()
    oracle.force_rows(x32, m32, eps, probe)
    dt = max(time.perf_counter() - t0, 1e-3)
    k = int(max(32, min(n, 32 * 2.0 / dt)))
    times = []
    for step in range(args.warmup + args.steps):
        rows = workloads.sample_rows(n, k, seed=100 + step)
        t0 = time.perf_counter()
        oracle.force_rows(x32, m32, eps, rows)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = k * n / (ms * 1e-3) / 1e9
    out = {
        "impl": "reference",
        "metric": "G-interactions/s and % FP32/MUFU roofline at N=2^20 vs FP64-oracle error",
        "value": value, "unit": "G-int/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic Plummer sphere (seed 0), float32",
        "config": {"workload": WORKLOAD, "n": n, "eps": float(eps),
                   "sample_rows_per_step": k},
        "cpu_baseline": {"value": value, "unit": "G-int/s", "cores": cores, "kind": "oracle",
                         "sample": f"{k} random rows x all {n} j per step, FP64"},
        "e2e": {"value": value, "unit": "G-int/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)
    return out


def run_case(args):
    """One kernel class at a small size, for profiler captures: `warmup`
    untimed launches then `steps` timed ones; prints one JSON line."""
    import torch
    import paper_0904_3659_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    case = args.case
    if case in ("pair", "comp"):
        n = args.n or (1 << 17)
        x32, m32 = make_inputs(n, 0)
        x = torch.from_numpy(x32).to(dev)
        mt = torch.from_numpy(m32).to(dev)
        a = torch.empty((n, 3), device=dev)
        p = torch.empty(n, device=dev)
        mode = nb.NB_PLAIN if case == "pair" else nb.NB_COMPENSATED
        if args.tile:
            nb.nb_set_tile(ctx, mode, tuple(int(v) for v in args.tile.split(",")))
        fn = lambda: nb.nb_force(ctx, x, mt, n, 1.0 / 256, a, p, mode)
        units = float(n) * n
    elif case == "batched":
        w = workloads.WORKLOADS["clusters1024_kdk32"]
        cl = workloads.clusters(w["n_clusters"], seed=w["seed"], nmin=w["nmin"], nmax=w["nmax"])
        n, C = cl.x.shape[0], len(cl.sizes)
        x = torch.from_numpy(cl.x.astype(np.float32)).to(dev)
        mt = torch.from_numpy(cl.m.astype(np.float32)).to(dev)
        off = torch.from_numpy(cl.offsets).to(dev)
        eps = torch.from_numpy(cl.eps.astype(np.float32)).to(dev)
        a = torch.empty((n, 3), device=dev)
        p = torch.empty(n, device=dev)
        fn = lambda: nb.nb_force_batched(ctx, x, mt, off, C, n, eps, a, p)
        units = float((cl.sizes.astype(np.float64) ** 2).sum())
    elif case in ("leapfrog", "leapfrog-comp"):
        w = workloads.WORKLOADS["plummer65536_kdk16"]
        n = args.n or w["n"]
        x0, v0, m = workloads.plummer(n, seed=w["seed"])
        xs = torch.from_numpy(x0).to(dev)
        vs = torch.from_numpy(v0).to(dev)
        x, v = xs.clone(), vs.clone()
        mt = torch.from_numpy(m.astype(np.float32)).to(dev)
        a = torch.empty((n, 3), dtype=torch.float32, device=dev)
        mode = nb.NB_PLAIN if case == "leapfrog" else nb.NB_COMPENSATED
        stream = torch.cuda.Stream(dev)  # graph replay needs a non-default stream

        def fn():
            x.copy_(xs)
            v.copy_(vs)
            nb.nb_leapfrog_step(ctx, x, v, mt, a, None, n, np.float32(w["eps"]), w["dt"], w["steps"],
                                0, mode, stream)

        def run():
            with torch.cuda.stream(stream):
                fn()
            stream.synchronize()
        units = float(n) * n * (w["steps"] + 1)
        for _ in range(args.warmup):
            run()
        nb.nb_synchronize(ctx, stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            run()
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
        print(json.dumps({"case": case, "n": n, "ms": ms, "g_units_s": units / (ms * 1e-3) / 1e9}),
              flush=True)
        return
    elif case == "vjp":
        n = args.n or 16384
        if args.tile:
            nb.nb_set_vjp_tile(ctx, tuple(int(v) for v in args.tile.split(",")))
        x32, m32 = make_inputs(n, 0)
        rng = np.random.default_rng(5)
        x = torch.from_numpy(x32).to(dev)
        mt = torch.from_numpy(m32).to(dev)
        ga = torch.from_numpy(rng.normal(size=(n, 3)).astype(np.float32)).to(dev)
        gp = torch.from_numpy(rng.normal(size=n).astype(np.float32)).to(dev)
        gx = torch.empty((n, 3), device=dev)
        gm = torch.empty(n, device=dev)
        fn = lambda: nb.nb_force_vjp(ctx, x, mt, n, 1.0 / 64, ga, gp, gx, gm)
        units = float(n) * n
    else:
        raise SystemExit(f"unknown case {case}")
    for _ in range(args.warmup):
        fn()
    nb.nb_synchronize(ctx)
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    nb.nb_synchronize(ctx)
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"case": case, "n": n, "ms": ms, "g_units_s": units / (ms * 1e-3) / 1e9}),
          flush=True)


def run_sweep(args):
    """Every compiled tile shape of both modes at N = 2^12 .. 2^20: the pair
    kernel's rate from the library's per-kernel events (one JSON line per
    shape and size). The tuner's search space, measured."""
    import torch
    import paper_0904_3659_gb300 as nb
    dev = torch.device("cuda", 0)
    ctx = nb.Context(0)
    sizes = [int(v) for v in args.sweep_sizes.split(",")]
    if args.sweep_kind == "vjp":
        rng = np.random.default_rng(5)
        for n in sizes:
            x32, m32 = make_inputs(n, 0)
            x = torch.from_numpy(x32).to(dev)
            mt = torch.from_numpy(m32).to(dev)
            ga = torch.from_numpy(rng.normal(size=(n, 3)).astype(np.float32)).to(dev)
            gp = torch.from_numpy(rng.normal(size=n).astype(np.float32)).to(dev)
            gx = torch.empty((n, 3), device=dev)
            gm = torch.empty(n, device=dev)
            reps = 3 if n >= 1 << 19 else (10 if n >= 1 << 16 else 50)
            for t in nb.nb_list_vjp_tiles():
                nb.nb_set_vjp_tile(ctx, t)
                line = {"n": n, "kernel": "vjp", "tile": list(t.as_tuple())}
                # With the upstream gradient on p, then without it (the
                # trajectory adjoint's case, a kernel of its own).
                for key, g in (("", gp), ("_without_gp", None)):
                    for _ in range(2):
                        nb.nb_force_vjp(ctx, x, mt, n, 1.0 / 64, ga, g, gx, gm)
                    nb.nb_synchronize(ctx)
                    nb.nb_timing_enable(ctx, True)
                    nb.nb_timing_reset(ctx)
                    for _ in range(reps):
                        nb.nb_force_vjp(ctx, x, mt, n, 1.0 / 64, ga, g, gx, gm)
                    nb.nb_synchronize(ctx)
                    ms, cnt = nb.nb_timing_read(ctx, nb.KERNEL_VJP)
                    nb.nb_timing_enable(ctx, False)
                    line["vjp_ms" + key] = ms / cnt
                    line["gpair_s" + key] = n * n / (ms / cnt * 1e-3) / 1e9
                print(json.dumps(line), flush=True)
            nb.nb_set_vjp_tile(ctx, None)
        return
    for n in sizes:
        x32, m32 = make_inputs(n, 0)
        x = torch.from_numpy(x32).to(dev)
        mt = torch.from_numpy(m32).to(dev)
        a = torch.empty((n, 3), device=dev)
        p = torch.empty(n, device=dev)
        reps = 3 if n >= 1 << 19 else (10 if n >= 1 << 16 else 50)
        for mode, mname in ((nb.NB_PLAIN, "plain"), (nb.NB_COMPENSATED, "compensated")):
            for t in nb.nb_list_tiles(mode):
                nb.nb_set_tile(ctx, mode, t)
                for _ in range(2):
                    nb.nb_force(ctx, x, mt, n, 1.0 / 256, a, p, mode)
                nb.nb_synchronize(ctx)
                nb.nb_timing_enable(ctx, True)
                nb.nb_timing_reset(ctx)
                for _ in range(reps):
                    nb.nb_force(ctx, x, mt, n, 1.0 / 256, a, p, mode)
                nb.nb_synchronize(ctx)
                ms, cnt = nb.nb_timing_read(ctx, nb.KERNEL_PAIR)
                nb.nb_timing_enable(ctx, False)
                pair_ms = ms / cnt
                print(json.dumps({"n": n, "mode": mname, "tile": list(t.as_tuple()),
                                  "pair_ms": pair_ms, "gint_s": n * n / (pair_ms * 1e-3) / 1e9}),
                      flush=True)
            nb.nb_set_tile(ctx, mode, None)
        tuned = {}
        for mode, mname in ((nb.NB_PLAIN, "plain"), (nb.NB_COMPENSATED, "compensated")):
            t, rate = nb.nb_autotune(ctx, n, mode)
            tuned[mname] = {"tile": list(t.as_tuple()), "gint_s_step": rate / 1e9}
        print(json.dumps({"n": n, "autotune": tuned}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tile-tune", dest="tile_tune", action="store_false")
    # Small-case options for profiler captures (the default run uses none).
    ap.add_argument("--n", type=int, default=0, help="override N (profiling small cases)")
    ap.add_argument("--tile", default="", help="plain tile: the nb_tile fields, comma-separated")
    ap.add_argument("--tile-comp", default="", help="compensated tile: the nb_tile fields")
    ap.add_argument("--no-newton-arm", dest="newton_arm", action="store_false",
                    help="skip timing the Newton-step tile beside the headline")
    ap.add_argument("--plain-only", action="store_true")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--sweep", action="store_true",
                    help="rate of every compiled tile shape over --sweep-sizes (JSON lines)")
    ap.add_argument("--sweep-sizes", default="4096,16384,65536,262144,1048576")
    ap.add_argument("--sweep-kind", choices=["pair", "vjp"], default="pair",
                    help="which kernel's compiled shapes --sweep times")
    ap.add_argument("--case", choices=["pair", "comp", "batched", "vjp", "leapfrog", "leapfrog-comp"],
                    default="",
                    help="time one kernel class at a small size (profiler captures)")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the leap-frog, batched and adjoint workloads")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)   # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    main()

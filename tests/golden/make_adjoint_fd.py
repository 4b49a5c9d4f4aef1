#!/usr/bin/env python
"""Writes adjoint_fd_plummer16384.txt: FP64 finite-difference gradients of the
differentiation workload, computed by the oracle alone.

Workload (plummer16384_adjoint64): N = 16384 Plummer sphere (seed 0), eps = 1/64,
64 kick-drift-kick leap-frog steps of dt = 1/512 (Eqs. (1)-(3), Section "Method",
with the force of Eq. (gravity), Section "Introduction"), loss
L = sum_i |x_i(T) - y_i|^2 against targets y = x(0) + 0.05 N(0, 1) (seed 1).

For 32 coordinates drawn with seed 3 (kinds cycling x0, v0, m), the file holds
the central difference (L(theta + h) - L(theta - h)) / 2h of the oracle's FP64
trajectory (h = 1e-5 for a position or velocity, 1e-2 m_i for a mass), and the
oracle's own reverse-mode gradient (oracle.leapfrog_grad) at the same
coordinate. Nothing here runs the CUDA library; the GPU test compares its
gradient with these stored values.

    python tests/golden/make_adjoint_fd.py [--out PATH]

It runs 65 FP64 trajectories of 65 force evaluations each (minutes on a few
cores).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(HERE, "adjoint_fd_plummer16384.txt")


def coordinates(n, m, count, seed):
    """(kind, i, c, h) for `count` coordinates: kinds cycle x, v, m; i, c
    uniform; h = 1e-5 for x and v, 1e-2 m_i for a mass (c = -1)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        kind = "xvm"[k % 3]
        if kind == "m":
            i = int(rng.integers(n))
            out.append((kind, i, -1, 1e-2 * float(m[i])))
        else:
            i, c = int(rng.integers(n)), int(rng.integers(3))
            out.append((kind, i, c, 1e-5))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args(argv)
    w = workloads.WORKLOADS["plummer16384_adjoint64"]
    n, eps, dt, steps = w["n"], np.float32(w["eps"]), w["dt"], w["steps"]
    x0, v0, m = workloads.plummer(n, seed=w["seed"])
    m = m.astype(np.float32).astype(np.float64)
    y = workloads.targets(x0, seed=w["target_seed"])

    def L(xx, vv, mm):
        xT, _, _ = oracle.leapfrog(xx, vv, mm, eps, dt, steps)
        return float(((xT - y) ** 2).sum())

    t0 = time.perf_counter()
    xT, _, _ = oracle.leapfrog(x0, v0, m, eps, dt, steps)
    gx, gv, gm = oracle.leapfrog_grad(x0, v0, m, eps, dt, steps, 2 * (xT - y))
    exact = {"x": gx, "v": gv, "m": gm}
    rows = []
    for kind, i, c, h in coordinates(n, m, w["fd_coords"], w["fd_seed"]):
        if kind == "m":
            mp, mm = m.copy(), m.copy()
            mp[i] += h
            mm[i] -= h
            fd = (L(x0, v0, mp) - L(x0, v0, mm)) / (2 * h)
            g = float(exact["m"][i])
        else:
            base = x0 if kind == "x" else v0
            bp, bm = base.copy(), base.copy()
            bp[i, c] += h
            bm[i, c] -= h
            if kind == "x":
                fd = (L(bp, v0, m) - L(bm, v0, m)) / (2 * h)
            else:
                fd = (L(x0, bp, m) - L(x0, bm, m)) / (2 * h)
            g = float(exact[kind][i, c])
        rows.append((kind, i, c, h, fd, g))
        print(f"{kind} {i} {c} fd={fd:.15e} adjoint={g:.15e} "
              f"({time.perf_counter() - t0:.0f} s)", flush=True)

    with open(args.out, "w") as f:
        f.write(
            "# FP64 finite-difference gradients of the differentiation workload, written by\n"
            "# tests/golden/make_adjoint_fd.py from the oracle alone (no CUDA code).\n"
            "# Trajectory: kick-drift-kick leap-frog, Eqs. (1)-(3) of Section \"Method\", with\n"
            "# the force of Eq. (gravity), Section \"Introduction\" (Fujiwara & Nakasato,\n"
            "# arXiv:0904.3659). N = 16384 Plummer (seed 0), eps = 1/64, 64 steps of dt = 1/512,\n"
            "# L = sum_i |x_i(T) - y_i|^2, y = x(0) + 0.05 N(0,1) (seed 1); coordinates seed 3.\n"
            "# fd = central difference of L with step h; adjoint = oracle.leapfrog_grad.\n"
            "# columns: kind i c h fd adjoint   (c = -1 for a mass)\n")
        for kind, i, c, h, fd, g in rows:
            f.write(f"{kind} {i} {c} {h:.17e} {fd:.17e} {g:.17e}\n")
    print(f"wrote {args.out} in {time.perf_counter() - t0:.0f} s")


if __name__ == "__main__":
    main()

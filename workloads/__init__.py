"""Seeded synthetic inputs for the direct-summation gravity path.

This module only draws particles; it holds none of the force, potential,
integration or gradient arithmetic, so both the CUDA path and the FP64 oracle
can take their inputs from it without sharing any of the method's code.

The paper's own inputs (figure-eight galaxies, a cart-wheel galaxy and a
random 100000-body system, Section "Experiments") are not available, so these
generators stand in for them:

  plummer          Plummer sphere, G = M = 1, scale radius b, sampled by the
                   rejection method of Aarseth, Henon & Wielen (1974): radius
                   from the inverse cumulative mass, speed from the isotropic
                   distribution function by von Neumann rejection.
  uniform_sphere   cold (v = 0) uniform-density ball of radius R.
  clusters         many independent clusters with log-uniform sizes, half of
                   them Plummer and half uniform balls, random radii.
  sample_rows      distinct random particle indices for sampled checks.
  targets          seeded Gaussian targets y_i = x_i + sigma * N(0, 1).

Random numbers come from numpy's PCG64 generator (np.random.default_rng),
whose integer stream and uniform/normal conversions are the same on every
platform. Positions and velocities are returned in float64; masses are
1/N_cluster. Callers round to FP32 where the kernel takes FP32, and give the
oracle that same rounded data.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "plummer", "uniform_sphere", "clusters", "sample_rows", "targets",
    "Clusters", "WORKLOADS",
]


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    """n directions uniform on the unit sphere (cos(theta) and phi uniform)."""
    cz = 1.0 - 2.0 * rng.random(n)
    phi = 2.0 * np.pi * rng.random(n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)


def plummer(n: int, seed: int = 0, b: float = 1.0, rmax: float = 100.0,
            center: bool = True):
    """Plummer sphere of n equal-mass particles (total mass 1, G = 1).

    Returns (x [n,3], v [n,3], m [n]) in float64.
    Radius: the enclosed mass fraction of a Plummer sphere is
    X = r^3 / (r^2 + b^2)^{3/2}, so r = b / sqrt(X^{-2/3} - 1); radii beyond
    rmax * b are redrawn. Speed: v = q * v_esc(r), v_esc = sqrt(2) (r^2+b^2)^{-1/4}
    (b = 1 units, scaled by 1/sqrt(b) otherwise), with q drawn from
    g(q) ~ q^2 (1 - q^2)^{7/2} by rejection under the bound 0.1.
    With center=True the centre of mass is moved to rest at the origin.
    """
    rng = np.random.default_rng(seed)
    n = int(n)
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        X = rng.random(todo.size)
        X = np.where(X <= 0.0, 0.5, X)
        rr = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        ok = rr <= rmax
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    x = r[:, None] * _unit_vectors(rng, n)

    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        q4 = rng.random(todo.size)
        y5 = 0.1 * rng.random(todo.size)
        ok = y5 < q4 * q4 * (1.0 - q4 * q4) ** 3.5
        q[todo[ok]] = q4[ok]
        todo = todo[~ok]
    vesc = np.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v = (q * vesc)[:, None] * _unit_vectors(rng, n)

    x *= b
    v /= np.sqrt(b)
    m = np.full(n, 1.0 / max(n, 1))
    if center and n:
        x -= (m[:, None] * x).sum(0) / m.sum()
        v -= (m[:, None] * v).sum(0) / m.sum()
    return x, v, m


def uniform_sphere(n: int, seed: int = 0, radius: float = 1.0, center: bool = True):
    """Cold uniform-density ball: r = R X^{1/3}, isotropic directions, v = 0."""
    rng = np.random.default_rng(seed)
    n = int(n)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    x = r[:, None] * _unit_vectors(rng, n)
    v = np.zeros((n, 3))
    m = np.full(n, 1.0 / max(n, 1))
    if center and n:
        x -= x.mean(0)
    return x, v, m


@dataclass
class Clusters:
    x: np.ndarray          # [total, 3] positions, clusters concatenated
    v: np.ndarray          # [total, 3] velocities
    m: np.ndarray          # [total] masses (1/N_c within cluster c)
    offsets: np.ndarray    # [C+1] int64, cluster c is rows offsets[c]:offsets[c+1]
    eps: np.ndarray        # [C] softening per cluster
    radius: np.ndarray     # [C] cluster radius R
    kind: np.ndarray       # [C] 0 = Plummer (scale radius R), 1 = uniform ball

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)


def clusters(n_clusters: int = 1024, seed: int = 0, nmin: int = 32, nmax: int = 4096,
             eps_over_r: float = 0.02, rmin: float = 0.5, rmax: float = 2.0) -> Clusters:
    """Independent clusters of uneven size in one concatenated array.

    N_c is log-uniform in [nmin, nmax] (rounded), the radius R_c uniform in
    [rmin, rmax], clusters alternate Plummer (even c) and uniform ball (odd c),
    and eps_c = eps_over_r * R_c. Each cluster has total mass 1 and is centred
    at the origin.
    """
    rng = np.random.default_rng(seed)
    C = int(n_clusters)
    logn = rng.uniform(np.log(nmin), np.log(nmax), C)
    sizes = np.clip(np.rint(np.exp(logn)).astype(np.int64), nmin, nmax)
    radius = rng.uniform(rmin, rmax, C)
    kind = (np.arange(C) % 2).astype(np.int64)
    xs, vs, ms = [], [], []
    for c in range(C):
        sub_seed = int(rng.integers(0, 2**62))
        if kind[c] == 0:
            x, v, m = plummer(int(sizes[c]), seed=sub_seed, b=float(radius[c]))
        else:
            x, v, m = uniform_sphere(int(sizes[c]), seed=sub_seed, radius=float(radius[c]))
        xs.append(x)
        vs.append(v)
        ms.append(m)
    offsets = np.zeros(C + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return Clusters(np.concatenate(xs) if C else np.zeros((0, 3)),
                    np.concatenate(vs) if C else np.zeros((0, 3)),
                    np.concatenate(ms) if C else np.zeros(0),
                    offsets, eps_over_r * radius, radius, kind)


def sample_rows(n: int, k: int, seed: int = 2) -> np.ndarray:
    """k distinct indices in [0, n), sorted (int64)."""
    rng = np.random.default_rng(seed)
    k = min(int(k), int(n))
    return np.sort(rng.choice(int(n), size=k, replace=False)).astype(np.int64)


def targets(x: np.ndarray, seed: int = 1, sigma: float = 0.05) -> np.ndarray:
    """y_i = x_i + sigma * N(0, 1) per coordinate."""
    rng = np.random.default_rng(seed)
    return np.asarray(x, dtype=np.float64) + sigma * rng.standard_normal(np.shape(x))


# The five workloads the project measures and tests (sizes, softening, steps).
WORKLOADS = {
    "plummer4096": dict(n=4096, seed=0, eps=0.01),
    "plummer65536_kdk16": dict(n=65536, seed=0, eps=1.0 / 128, dt=1.0 / 256, steps=16),
    "plummer1m": dict(n=1 << 20, seed=0, eps=1.0 / 256, sample=2048, sample_seed=2),
    "clusters1024_kdk32": dict(n_clusters=1024, seed=0, nmin=32, nmax=4096, steps=32,
                               dt=1.0 / 256),
    "plummer16384_adjoint64": dict(n=16384, seed=0, eps=1.0 / 64, dt=1.0 / 512, steps=64,
                                   checkpoint=8, fd_coords=32, fd_seed=3, target_seed=1),
}

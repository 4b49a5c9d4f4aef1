"""FP64 CPU oracle for the softened gravitational force and potential.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package. The product path (the CUDA
library and its Python binding) never imports it.

The arithmetic lives in ``nb_oracle.c`` (plain double loops, see its header);
this module compiles it with gcc and exposes it through ctypes on numpy
float64 arrays. Inputs given as FP32 are promoted exactly to FP64.

Functions, each following the paper (Fujiwara & Nakasato, arXiv:0904.3659):
  force        Eq. (gravity), Section "Introduction": a_i, p_i for all i
  force_rows   Eq. (gravity) for a sampled list of i
  force_vjp    chain rule of Eq. (gravity): dL/dx, dL/dm for
               L = sum_i ga_i . a_i + gp_i p_i
  leapfrog     Eqs. (1)-(3), Section "Method", with the physical sign g = -a
  leapfrog_grad  reverse-mode chain rule through leapfrog's steps (uses
               force_vjp): gradients at the initial state of a loss of the
               final state
  energy       K = 1/2 sum m v^2, W = -1/2 sum m p

Parity status: every function is pinned by CPU tests against closed forms,
exact scaling laws, invariants, finite differences and high-precision brute
force (tests/test_oracle_*.py); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_LIB = os.path.join(_HERE, "libnb_oracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile nb_oracle.c (or another copy of it) into a shared library with
    gcc (no CUDA)."""
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *_CFLAGS, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def _bind(path):
    lib = ctypes.CDLL(path)
    lib.nbo_num_threads.restype = ctypes.c_int
    lib.nbo_set_num_threads.argtypes = [ctypes.c_int]
    lib.nbo_force.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, _D, _D, _D]
    lib.nbo_force_rows.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double,
                                   ctypes.c_int64, _I64, _D, _D, _D]
    lib.nbo_force_vjp.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double,
                                  _D, _D, _D, _D]
    lib.nbo_force_vjp_rows.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double,
                                       _D, _D, ctypes.c_int64, _I64, _D, _D]
    lib.nbo_leapfrog.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int64, _D, _D]
    lib.nbo_energy.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, _D, _D]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def _f64(a, shape=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        arr = arr.reshape(shape)
    return arr


def _p(arr):
    return arr.ctypes.data_as(_D)


def _eps64(eps) -> float:
    # The CUDA library takes eps as FP32; the oracle uses that same FP32
    # value, promoted exactly to FP64 (eps^2 is then formed in FP64).
    return float(np.float32(eps))


class Oracle:
    """The oracle's functions bound to one compiled copy of nb_oracle.c (the
    module-level functions use the default build; tests that plant mistakes
    in a copy of the source drive that copy through the same functions)."""

    def __init__(self, lib_path=None):
        self._path = lib_path
        self._cdll = None

    def _lib(self):
        if self._path is None:
            return _load()
        if self._cdll is None:
            self._cdll = _bind(self._path)
        return self._cdll

    def num_threads(self) -> int:
        return int(self._lib().nbo_num_threads())


    def set_num_threads(self, n: int) -> None:
        self._lib().nbo_set_num_threads(int(n))


    def force(self, x, m, eps):
        """Eq. (gravity) for all particles. Returns (a [n,3], p [n], amag [n])."""
        x = _f64(x)
        n = x.shape[0]
        x = x.reshape(n, 3)
        m = _f64(m, (n,))
        a = np.zeros((n, 3))
        p = np.zeros(n)
        amag = np.zeros(n)
        if n:
            self._lib().nbo_force(n, _p(x), _p(m), _eps64(eps), _p(a), _p(p), _p(amag))
        return a, p, amag


    def force_rows(self, x, m, eps, rows):
        """Eq. (gravity) for the particles listed in rows."""
        x = _f64(x)
        n = x.shape[0]
        x = x.reshape(n, 3)
        m = _f64(m, (n,))
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        if rows.size and (rows.min() < 0 or rows.max() >= n):
            raise IndexError("row out of range")
        k = rows.size
        a = np.zeros((k, 3))
        p = np.zeros(k)
        amag = np.zeros(k)
        if k:
            self._lib().nbo_force_rows(n, _p(x), _p(m), _eps64(eps), k,
                                   rows.ctypes.data_as(_I64), _p(a), _p(p), _p(amag))
        return a, p, amag


    def force_vjp(self, x, m, eps, ga, gp, rows=None):
        """dL/dx, dL/dm of L = sum ga.a + gp p (all rows, or the listed ones)."""
        x = _f64(x)
        n = x.shape[0]
        x = x.reshape(n, 3)
        m = _f64(m, (n,))
        ga = _f64(ga, (n, 3))
        gp = _f64(gp, (n,))
        lib = self._lib()
        if rows is None:
            gx = np.zeros((n, 3))
            gm = np.zeros(n)
            if n:
                lib.nbo_force_vjp(n, _p(x), _p(m), _eps64(eps), _p(ga), _p(gp), _p(gx), _p(gm))
            return gx, gm
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        k = rows.size
        gx = np.zeros((k, 3))
        gm = np.zeros(k)
        if k:
            lib.nbo_force_vjp_rows(n, _p(x), _p(m), _eps64(eps), _p(ga), _p(gp), k,
                                   rows.ctypes.data_as(_I64), _p(gx), _p(gm))
        return gx, gm


    def leapfrog(self, x, v, m, eps, dt, nsteps):
        """Eqs. (1)-(3) for nsteps steps. Returns (x, v, g) after the last step,
        g the physical acceleration -a at the final positions."""
        x = _f64(x).copy()
        n = x.shape[0]
        x = x.reshape(n, 3)
        v = _f64(v, (n, 3)).copy()
        m = _f64(m, (n,))
        g = np.zeros((n, 3))
        work = np.zeros(4 * max(n, 1))
        if n:
            self._lib().nbo_leapfrog(n, _p(x), _p(v), _p(m), _eps64(eps), float(dt),
                                 int(nsteps), _p(g), _p(work))
        return x, v, g


    def leapfrog_grad(self, x0, v0, m, eps, dt, nsteps, xbar, vbar=None, on_vjp=None):
        """Gradients (dL/dx0, dL/dv0, dL/dm) of a loss L of the state after
        nsteps leapfrog steps, given xbar = dL/dx(T) and vbar = dL/dv(T).
        on_vjp(x, ga), if given, sees the operands of every force VJP the
        sweep takes (for error scales in tests; it changes nothing).

        Chain rule through the steps of `leapfrog` in reverse. One step maps
        (x, v, a) with a = Eq. (gravity) at x to
            x' = x + dt v - dt^2/2 a          Eq. (2) with g = -a
            a' = Eq. (gravity) at x'
            v' = v - dt/2 a - dt/2 a'         Eqs. (1) and (3)
        so, going back, the adjoint of a' collects -dt/2 vbar', the adjoint of
        x' collects the VJP of Eq. (gravity) at x' (force_vjp, which also gives
        the mass gradient), the adjoint of a collects -dt/2 vbar' - dt^2/2 xbar',
        and vbar = vbar' + dt xbar', xbar = xbar'.
        """
        x = _f64(x0).copy()
        n = x.shape[0]
        x = x.reshape(n, 3)
        v = _f64(v0, (n, 3)).copy()
        m = _f64(m, (n,))
        eps = _eps64(eps)
        xs = [x.copy()]
        a, _, _ = self.force(x, m, eps)
        for _ in range(int(nsteps)):
            v_half = v + 0.5 * dt * (-a)
            x = x + v * dt + 0.5 * (-a) * dt * dt
            a, _, _ = self.force(x, m, eps)
            v = v_half + 0.5 * dt * (-a)
            xs.append(x.copy())
        xb = _f64(xbar, (n, 3)).copy()
        vb = np.zeros((n, 3)) if vbar is None else _f64(vbar, (n, 3)).copy()
        ab = np.zeros((n, 3))
        mb = np.zeros(n)
        zero_p = np.zeros(n)
        for s in range(int(nsteps) - 1, -1, -1):
            ab_next = ab - 0.5 * dt * vb
            if on_vjp is not None:
                on_vjp(xs[s + 1], ab_next)
            gx, gm = self.force_vjp(xs[s + 1], m, eps, ab_next, zero_p)
            xb = xb + gx
            mb = mb + gm
            ab = -0.5 * dt * vb - 0.5 * dt * dt * xb
            vb = vb + dt * xb
        if on_vjp is not None:
            on_vjp(xs[0], ab)
        gx, gm = self.force_vjp(xs[0], m, eps, ab, zero_p)
        return xb + gx, vb, mb + gm


    def energy(self, x, v, m, eps):
        """Returns (K, W): kinetic and potential energy, W = -1/2 sum m p."""
        x = _f64(x)
        n = x.shape[0]
        x = x.reshape(n, 3)
        v = _f64(v, (n, 3))
        m = _f64(m, (n,))
        out = np.zeros(2)
        work = np.zeros(4 * max(n, 1))
        if n:
            self._lib().nbo_energy(n, _p(x), _p(v), _p(m), _eps64(eps), _p(out), _p(work))
        return float(out[0]), float(out[1])


_default = Oracle()
num_threads = _default.num_threads
set_num_threads = _default.set_num_threads
force = _default.force
force_rows = _default.force_rows
force_vjp = _default.force_vjp
leapfrog = _default.leapfrog
leapfrog_grad = _default.leapfrog_grad
energy = _default.energy

"""Python binding of libnbody.so, the sm_103a direct-summation gravity library.

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels. Functions carry the names of the C entry points in
include/nbody.h and take torch tensors (or raw integer addresses) for the
array arguments; streams default to torch's current stream.

There is no CPU fallback: importing this package works without a GPU (so the
library's exports can be checked), but every compute call goes through the
compiled library and raises if it is missing or fails.

The computation (Fujiwara & Nakasato, arXiv:0904.3659, Eq. (gravity)):
    a_i = sum_{j != i} m_j (x_i - x_j) / (|x_i - x_j|^2 + eps^2)^{3/2}
    p_i = sum_{j != i} m_j / (|x_i - x_j|^2 + eps^2)^{1/2}
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

__all__ = [
    "NB_OK", "NB_ERR_ARG", "NB_ERR_CUDA", "NB_ERR_OOM", "NB_ERR_TIMEOUT",
    "NB_ERR_NOT_IMPLEMENTED", "NB_PLAIN", "NB_COMPENSATED", "NBError", "nb_tile",
    "library", "library_path", "exported_symbols", "Context",
    "nb_create", "nb_destroy", "nb_last_error", "nb_status_string", "nb_force",
    "nb_force_host", "nb_reserve", "nb_force_batched", "nb_leapfrog_batched_step", "nb_leapfrog_step",
    "nb_leapfrog_adjoint", "nb_energy",
    "nb_force_vjp", "nb_set_vjp_tile", "nb_get_vjp_tile", "nb_list_vjp_tiles", "nb_synchronize", "nb_get_tile", "nb_set_tile", "nb_set_tuned_tile", "nb_list_tiles",
    "tune_to_file", "load_tuning",
    "nb_autotune", "nb_timing_enable", "nb_timing_read", "nb_timing_reset",
    "nb_debug_set_fault", "nb_force_noalloc", "force",
]

NB_OK = 0
NB_ERR_ARG = 1
NB_ERR_CUDA = 2
NB_ERR_OOM = 3
NB_ERR_TIMEOUT = 4
NB_ERR_NOT_IMPLEMENTED = 5

NB_PLAIN = 0
NB_COMPENSATED = 1

KERNEL_PACK, KERNEL_PAIR, KERNEL_REDUCE, KERNEL_LEAPFROG, KERNEL_BATCHED, KERNEL_VJP = range(6)

_HERE = os.path.dirname(os.path.abspath(__file__))
# NB_LIBRARY selects another build of the library (e.g. libnbody_debug.so,
# the bounds-checked build); the default is the in-tree release build.
library_path = os.environ.get("NB_LIBRARY") or os.path.join(_HERE, "libnbody.so")


class nb_tile(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("ipt", ctypes.c_int),
                ("jtile", ctypes.c_int), ("stages", ctypes.c_int),
                ("unroll", ctypes.c_int), ("minblocks", ctypes.c_int),
                ("release", ctypes.c_int), ("sums_in_smem", ctypes.c_int),
                ("packed", ctypes.c_int), ("refine", ctypes.c_int),
                ("fused", ctypes.c_int)]

    def as_tuple(self):
        return tuple(getattr(self, f) for f, _ in self._fields_)

    def __repr__(self):
        return "nb_tile(" + ", ".join(f"{f}={getattr(self, f)}" for f, _ in self._fields_) + ")"


class NBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_STATUS_NAMES = {0: "NB_OK", 1: "NB_ERR_ARG", 2: "NB_ERR_CUDA", 3: "NB_ERR_OOM",
                 4: "NB_ERR_TIMEOUT", 5: "NB_ERR_NOT_IMPLEMENTED"}

_c = ctypes
_P = _c.c_void_p
_I64 = _c.c_int64
# Signatures of include/nbody.h.
_SIGNATURES = {
    "nb_create": (_c.c_int, [_c.POINTER(_P), _c.c_int]),
    "nb_destroy": (None, [_P]),
    "nb_last_error": (_c.c_char_p, [_P]),
    "nb_status_string": (_c.c_char_p, [_c.c_int]),
    "nb_force": (_c.c_int, [_P, _P, _P, _I64, _c.c_float, _P, _P, _c.c_int, _P]),
    "nb_force_host": (_c.c_int, [_P, _P, _P, _I64, _c.c_float, _P, _P, _c.c_int, _P]),
    "nb_reserve": (_c.c_int, [_P, _I64, _c.c_int]),
    "nb_force_batched": (_c.c_int, [_P, _P, _P, _P, _I64, _I64, _P, _P, _P, _c.c_int, _P]),
    "nb_leapfrog_step": (_c.c_int, [_P, _P, _P, _P, _P, _P, _I64, _c.c_float, _c.c_double,
                                    _c.c_int, _c.c_int, _c.c_int, _P]),
    "nb_leapfrog_batched_step": (_c.c_int, [_P, _P, _P, _P, _P, _I64, _I64, _P, _P, _P,
                                            _c.c_double, _c.c_int, _c.c_int, _c.c_int, _P]),
    "nb_leapfrog_adjoint": (_c.c_int, [_P, _P, _P, _P, _P, _I64, _c.c_float, _c.c_double, _c.c_int,
                                       _P, _P, _P, _P, _c.c_int, _c.c_int, _P]),
    "nb_energy": (_c.c_int, [_P, _P, _P, _P, _I64, _c.c_float, _P, _c.c_int, _P]),
    "nb_force_vjp": (_c.c_int, [_P, _P, _P, _I64, _c.c_float, _P, _P, _P, _P, _P]),
    "nb_set_vjp_tile": (_c.c_int, [_P, _c.POINTER(nb_tile)]),
    "nb_get_vjp_tile": (_c.c_int, [_P, _I64, _c.POINTER(nb_tile)]),
    "nb_list_vjp_tiles": (_c.c_int, [_c.POINTER(nb_tile), _c.c_int, _c.POINTER(_c.c_int)]),
    "nb_synchronize": (_c.c_int, [_P, _P]),
    "nb_get_tile": (_c.c_int, [_P, _I64, _c.c_int, _c.POINTER(nb_tile)]),
    "nb_set_tile": (_c.c_int, [_P, _c.c_int, _c.POINTER(nb_tile)]),
    "nb_set_tuned_tile": (_c.c_int, [_P, _I64, _c.c_int, _c.POINTER(nb_tile)]),
    "nb_list_tiles": (_c.c_int, [_c.c_int, _c.POINTER(nb_tile), _c.c_int, _c.POINTER(_c.c_int)]),
    "nb_autotune": (_c.c_int, [_P, _I64, _c.c_int, _P, _c.POINTER(nb_tile),
                               _c.POINTER(_c.c_double)]),
    "nb_timing_enable": (_c.c_int, [_P, _c.c_int]),
    "nb_timing_read": (_c.c_int, [_P, _c.c_int, _c.POINTER(_c.c_double), _c.POINTER(_I64)]),
    "nb_timing_reset": (_c.c_int, [_P]),
    "nb_debug_set_fault": (_c.c_int, [_P, _I64, _I64]),
    "nb_force_noalloc": (_c.c_int, [_P, _P, _I64, _c.c_float, _P, _P, _P]),
}
exported_symbols = tuple(_SIGNATURES)

_lib = None


def library():
    """The loaded libnbody.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError(
                f"{library_path} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(library_path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


_DTYPES = {}


def _torch_dtype(name: str):
    dt = _DTYPES.get(name)
    if dt is None:
        import torch
        dt = _DTYPES[name] = getattr(torch, name)
    return dt


def _dev(t, dtype: str, numel: int, name: str) -> Optional[int]:
    """Address of a device array argument, checked: a torch tensor must have
    the dtype the C signature takes, be contiguous, hold at least `numel`
    elements and live on a CUDA device (an int is taken as a raw address,
    None as NULL). A wrong tensor raises here instead of being read as
    something else by the kernels. (Kept to a few attribute reads: it runs
    on every call, and at small n the host time per call is what a loop of
    calls sees.)"""
    if t is None or isinstance(t, int):
        return t
    if t.dtype is not _torch_dtype(dtype):
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs {numel}")
    if not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    return t.data_ptr()


def _addr(t) -> Optional[int]:
    """Address of a tensor's data (or an int address / None) for a C pointer."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


_raw_stream = None


def _stream(stream) -> Optional[int]:
    """cudaStream_t for a call: the given stream (a torch stream or a raw
    handle), else torch's current stream of the current device, read as a
    raw handle without building a Stream object."""
    global _raw_stream
    if stream is None:
        if _raw_stream is None:
            try:
                import torch
                if not torch.cuda.is_available():
                    return None
                raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
                cur = torch.cuda.current_device
                _raw_stream = ((lambda: raw(cur())) if raw is not None
                               else (lambda: torch.cuda.current_stream().cuda_stream))
            except ImportError:
                return None
        return _raw_stream() or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _check(ctx, status: int):
    if status != NB_OK:
        msg = library().nb_last_error(ctx.handle if ctx is not None else None)
        raise NBError(status, (msg or b"").decode())


class Context:
    """Owns an nb_ctx handle (scratch, tuning table, events) for one device."""

    def __init__(self, device: int = 0):
        h = _P()
        st = library().nb_create(ctypes.byref(h), int(device))
        if st != NB_OK:
            raise NBError(st, (library().nb_last_error(None) or b"").decode())
        self.handle = h
        self.device = int(device)

    def close(self):
        if getattr(self, "handle", None):
            library().nb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def nb_create(device: int = 0) -> Context:
    return Context(device)


def nb_destroy(ctx: Context) -> None:
    ctx.close()


def nb_last_error(ctx: Optional[Context]) -> str:
    return (library().nb_last_error(ctx.handle if ctx else None) or b"").decode()


def nb_status_string(status: int) -> str:
    return library().nb_status_string(int(status)).decode()


def nb_force(ctx, x, m, n, eps, a, p, mode=NB_PLAIN, stream=None):
    n = int(n)
    args = (_dev(x, "float32", 3 * n, "x"), _dev(m, "float32", n, "m"), n, float(eps),
            _dev(a, "float32", 3 * n, "a"), _dev(p, "float32", n, "p"))
    _check(ctx, library().nb_force(ctx.handle, *args, int(mode), _stream(stream)))


def nb_force_host(ctx, x, m, n, eps, a, p, mode=NB_PLAIN, stream=None):
    _check(ctx, library().nb_force_host(ctx.handle, _addr(x), _addr(m), int(n), float(eps),
                                        _addr(a), _addr(p), int(mode), _stream(stream)))


def nb_reserve(ctx, n, mode=NB_PLAIN):
    _check(ctx, library().nb_reserve(ctx.handle, int(n), int(mode)))


def nb_force_batched(ctx, x, m, offsets, n_clusters, n_total, eps, a, p, mode=NB_PLAIN,
                     stream=None):
    nt, nc = int(n_total), int(n_clusters)
    args = (_dev(x, "float32", 3 * nt, "x"), _dev(m, "float32", nt, "m"),
            _dev(offsets, "int64", nc + 1, "offsets"), nc, nt, _dev(eps, "float32", nc, "eps"),
            _dev(a, "float32", 3 * nt, "a"), _dev(p, "float32", nt, "p"))
    _check(ctx, library().nb_force_batched(ctx.handle, *args, int(mode), _stream(stream)))


def nb_leapfrog_step(ctx, x, v, m, a, p, n, eps, dt, nsteps, a_valid, mode=NB_PLAIN, stream=None):
    n = int(n)
    args = (_dev(x, "float64", 3 * n, "x"), _dev(v, "float64", 3 * n, "v"),
            _dev(m, "float32", n, "m"), _dev(a, "float32", 3 * n, "a"), _dev(p, "float32", n, "p"))
    _check(ctx, library().nb_leapfrog_step(ctx.handle, *args, n, float(eps), float(dt), int(nsteps),
                                           int(a_valid), int(mode), _stream(stream)))


def nb_leapfrog_adjoint(ctx, x, v, a, m, n, eps, dt, nsteps, lx, lv, la, lm, apply_first,
                        mode=NB_PLAIN, stream=None):
    n = int(n)
    _check(ctx, library().nb_leapfrog_adjoint(
        ctx.handle, _dev(x, "float64", 3 * n, "x"), _dev(v, "float64", 3 * n, "v"),
        _dev(a, "float32", 3 * n, "a"), _dev(m, "float32", n, "m"), n, float(eps), float(dt),
        int(nsteps), _dev(lx, "float64", 3 * n, "lx"), _dev(lv, "float64", 3 * n, "lv"),
        _dev(la, "float64", 3 * n, "la"), _dev(lm, "float64", n, "lm"), int(bool(apply_first)),
        int(mode), _stream(stream)))


def nb_leapfrog_batched_step(ctx, x, v, m, offsets, n_clusters, n_total, eps, a, p, dt, nsteps,
                             a_valid, mode=NB_PLAIN, stream=None):
    nt, nc = int(n_total), int(n_clusters)
    _check(ctx, library().nb_leapfrog_batched_step(
        ctx.handle, _dev(x, "float64", 3 * nt, "x"), _dev(v, "float64", 3 * nt, "v"),
        _dev(m, "float32", nt, "m"), _dev(offsets, "int64", nc + 1, "offsets"), nc, nt,
        _dev(eps, "float32", nc, "eps"), _dev(a, "float32", 3 * nt, "a"),
        _dev(p, "float32", nt, "p"), float(dt), int(nsteps), int(a_valid), int(mode),
        _stream(stream)))


def nb_energy(ctx, x, v, m, n, eps, mode=NB_PLAIN, stream=None):
    out = (ctypes.c_double * 2)()
    n = int(n)
    _check(ctx, library().nb_energy(ctx.handle, _dev(x, "float64", 3 * n, "x"),
                                    _dev(v, "float64", 3 * n, "v"), _dev(m, "float32", n, "m"), n,
                                    float(eps), ctypes.cast(out, _P), int(mode), _stream(stream)))
    return float(out[0]), float(out[1])


def nb_force_vjp(ctx, x, m, n, eps, ga, gp, gx, gm, stream=None):
    n = int(n)
    _check(ctx, library().nb_force_vjp(ctx.handle, _dev(x, "float32", 3 * n, "x"),
                                       _dev(m, "float32", n, "m"), n, float(eps),
                                       _dev(ga, "float32", 3 * n, "ga"), _dev(gp, "float32", n, "gp"),
                                       _dev(gx, "float32", 3 * n, "gx"), _dev(gm, "float32", n, "gm"),
                                       _stream(stream)))


def nb_force_noalloc(x, m, n, eps, a, p, stream=None):
    """Allocation-free nb_force (no context; n <= 65536; waits for the stream).
    The arrays must live on the current CUDA device."""
    n = int(n)
    for name, t in (("x", x), ("m", m), ("a", a), ("p", p)):
        if getattr(t, "is_cuda", False):
            import torch
            if t.device.index != torch.cuda.current_device():
                raise ValueError(f"{name} is on {t.device}, not on the current device "
                                 f"cuda:{torch.cuda.current_device()}")
    _check(None, library().nb_force_noalloc(_dev(x, "float32", 3 * n, "x"),
                                            _dev(m, "float32", n, "m"), n, float(eps),
                                            _dev(a, "float32", 3 * n, "a"),
                                            _dev(p, "float32", n, "p"), _stream(stream)))


def nb_synchronize(ctx, stream=None):
    _check(ctx, library().nb_synchronize(ctx.handle, _stream(stream)))


def nb_get_tile(ctx, n, mode=NB_PLAIN) -> nb_tile:
    t = nb_tile()
    _check(ctx, library().nb_get_tile(ctx.handle, int(n), int(mode), ctypes.byref(t)))
    return t


def nb_set_tile(ctx, mode, tile) -> None:
    if tile is None:
        _check(ctx, library().nb_set_tile(ctx.handle, int(mode), None))
        return
    if not isinstance(tile, nb_tile):
        tile = nb_tile(*tile)
    _check(ctx, library().nb_set_tile(ctx.handle, int(mode), ctypes.byref(tile)))


def nb_set_tuned_tile(ctx, n, mode, tile) -> None:
    if tile is None:
        _check(ctx, library().nb_set_tuned_tile(ctx.handle, int(n), int(mode), None))
        return
    if not isinstance(tile, nb_tile):
        tile = nb_tile(*tile)
    _check(ctx, library().nb_set_tuned_tile(ctx.handle, int(n), int(mode), ctypes.byref(tile)))


def tune_to_file(ctx, sizes, path, modes=(NB_PLAIN, NB_COMPENSATED)):
    """Run nb_autotune for every size and mode and save the picks as JSON
    ({"device": ..., "entries": [{"mode", "n", "tile", "rate"}]})."""
    import json
    entries = []
    for mode in modes:
        for n in sizes:
            t, rate = nb_autotune(ctx, n, mode)
            entries.append({"mode": int(mode), "n": int(n), "tile": list(t.as_tuple()),
                            "rate": rate})
    device = None
    try:
        import torch
        device = torch.cuda.get_device_name(ctx.device)
    except Exception:
        pass
    with open(path, "w") as f:
        json.dump({"device": device, "entries": entries}, f, indent=1)
    return entries


def load_tuning(ctx, path) -> int:
    """Restore tuning picks saved by tune_to_file; returns how many applied
    (entries naming a shape the loaded library does not compile are skipped)."""
    import json
    with open(path) as f:
        data = json.load(f)
    applied = 0
    for e in data.get("entries", []):
        try:
            nb_set_tuned_tile(ctx, e["n"], e["mode"], tuple(e["tile"]))
            applied += 1
        except NBError:
            pass
    return applied


def nb_set_vjp_tile(ctx, tile) -> None:
    if tile is None:
        _check(ctx, library().nb_set_vjp_tile(ctx.handle, None))
        return
    if not isinstance(tile, nb_tile):
        tile = nb_tile(*tile)
    _check(ctx, library().nb_set_vjp_tile(ctx.handle, ctypes.byref(tile)))


def nb_get_vjp_tile(ctx, n=1 << 20) -> nb_tile:
    """The shape nb_force_vjp uses at size n for a call with gp given."""
    t = nb_tile()
    _check(ctx, library().nb_get_vjp_tile(ctx.handle, int(n), ctypes.byref(t)))
    return t


def nb_list_vjp_tiles() -> list:
    count = ctypes.c_int(0)
    st = library().nb_list_vjp_tiles(None, 0, ctypes.byref(count))
    if st != NB_OK:
        raise NBError(st, "nb_list_vjp_tiles")
    arr = (nb_tile * count.value)()
    library().nb_list_vjp_tiles(arr, count.value, ctypes.byref(count))
    return [arr[k] for k in range(count.value)]


def nb_list_tiles(mode=NB_PLAIN) -> list:
    count = ctypes.c_int(0)
    st = library().nb_list_tiles(int(mode), None, 0, ctypes.byref(count))
    if st != NB_OK:
        raise NBError(st, "nb_list_tiles")
    arr = (nb_tile * count.value)()
    library().nb_list_tiles(int(mode), arr, count.value, ctypes.byref(count))
    return [arr[k] for k in range(count.value)]


def nb_autotune(ctx, n, mode=NB_PLAIN, stream=None):
    t = nb_tile()
    rate = ctypes.c_double(0.0)
    _check(ctx, library().nb_autotune(ctx.handle, int(n), int(mode), _stream(stream),
                                      ctypes.byref(t), ctypes.byref(rate)))
    return t, rate.value


def nb_timing_enable(ctx, on=True):
    _check(ctx, library().nb_timing_enable(ctx.handle, 1 if on else 0))


def nb_timing_read(ctx, kernel):
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    _check(ctx, library().nb_timing_read(ctx.handle, int(kernel), ctypes.byref(ms),
                                         ctypes.byref(cnt)))
    return ms.value, cnt.value


def nb_timing_reset(ctx):
    _check(ctx, library().nb_timing_reset(ctx.handle))


def nb_debug_set_fault(ctx, unit=-1, wait_ns=0):
    _check(ctx, library().nb_debug_set_fault(ctx.handle, int(unit), int(wait_ns)))


def force(x, m, eps, mode=NB_PLAIN, ctx: Optional[Context] = None, stream=None):
    """Eq. (gravity) for torch CUDA tensors x [n,3], m [n] (float32,
    contiguous). Allocates and returns (a [n,3], p [n])."""
    import torch
    if x.dtype != torch.float32 or m.dtype != torch.float32:
        raise TypeError("x and m must be float32")
    if not (x.is_cuda and m.is_cuda):
        raise TypeError("x and m must be CUDA tensors")
    x = x.contiguous()
    m = m.contiguous()
    n = x.shape[0]
    if x.shape != (n, 3) or m.shape != (n,):
        raise ValueError("x must be [n, 3] and m [n]")
    if ctx is None:
        ctx = _default_context(x.device.index or 0)
    a = torch.empty((n, 3), dtype=torch.float32, device=x.device)
    p = torch.empty((n,), dtype=torch.float32, device=x.device)
    nb_force(ctx, x, m, n, eps, a, p, mode, stream)
    return a, p


_default_ctx = {}


def _default_context(device: int) -> Context:
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]

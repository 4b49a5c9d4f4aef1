"""nb_force_noalloc: the entry point for callers that may not allocate device
memory (their memory belongs to a pool or framework allocator, or they
cannot afford an allocation's device-wide synchronisation). It takes its
scratch from a fixed array in the library image instead of a context.

Checked through the C ABI on two calls in a row (different sizes, so the
second call runs over the first call's leftovers in the shared array): against
the FP64 oracle of Eq. (gravity) (Section "Introduction") within the plain
path's tolerance of 1e-5 relative to A_i = sum_j m_j |x_i - x_j| / s_ij^{3/2}
(and p_i), and against nb_force on the same inputs; also on a caller-supplied
stream, and for its size limit. This file is collected last so that a failure
here stops a -x run only after every other test has run.
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


def _inputs(n, seed):
    x, _, m = workloads.plummer(n, seed=seed)
    return x.astype(np.float32), m.astype(np.float32)


def _errors(a, p, ra, rp, amag):
    ea = np.linalg.norm(a.astype(np.float64) - ra, axis=1) / amag
    ep = np.abs(p.astype(np.float64) - rp) / rp
    return ea.max(), ep.max()


def _check_calls(nb, oracle_mod, stream):
    import torch
    dev = torch.device("cuda:0")
    ctx = nb.Context(0)
    try:
        for n, seed, eps in ((4096, 0, np.float32(0.01)), (3001, 5, np.float32(1.0 / 64))):
            x32, m32 = _inputs(n, seed)
            ra, rp, amag = oracle_mod.force(x32, m32, eps)
            xt = torch.from_numpy(x32).to(dev)
            mt = torch.from_numpy(m32).to(dev)
            a_ref = torch.empty((n, 3), device=dev)
            p_ref = torch.empty(n, device=dev)
            nb.nb_force(ctx, xt, mt, n, eps, a_ref, p_ref)
            nb.nb_synchronize(ctx)
            a = torch.full((n, 3), float("nan"), device=dev)
            p = torch.full((n,), float("nan"), device=dev)
            if stream is not None:
                stream.wait_stream(torch.cuda.current_stream(dev))
            nb.nb_force_noalloc(xt, mt, n, eps, a, p, stream)   # waits for its stream
            a_np, p_np = a.cpu().numpy(), p.cpu().numpy()
            assert np.all(np.isfinite(a_np)) and np.all(np.isfinite(p_np))
            # Against the FP64 oracle (the plain path's tolerance).
            ea, ep = _errors(a_np, p_np, ra, rp, amag)
            assert ea <= 1e-5 and ep <= 1e-5, ("oracle", n, ea, ep)
            # Against the existing entry point on the same inputs.
            ea2, ep2 = _errors(a_np, p_np, a_ref.cpu().numpy().astype(np.float64),
                               p_ref.cpu().numpy().astype(np.float64), amag)
            assert ea2 <= 1e-5 and ep2 <= 1e-5, ("nb_force", n, ea2, ep2)
    finally:
        ctx.close()


def test_noalloc_matches_oracle_two_calls(nb, oracle_mod):
    _check_calls(nb, oracle_mod, None)


def test_noalloc_on_caller_stream(nb, oracle_mod):
    import torch
    _check_calls(nb, oracle_mod, torch.cuda.Stream(torch.device("cuda:0")))


def test_noalloc_rejects_oversize(nb):
    import torch
    dev = torch.device("cuda:0")
    n = 65537
    x = torch.zeros((n, 3), device=dev)
    m = torch.ones(n, device=dev)
    a = torch.empty((n, 3), device=dev)
    p = torch.empty(n, device=dev)
    with pytest.raises(nb.NBError) as e:
        nb.nb_force_noalloc(x, m, n, 0.1, a, p)
    assert e.value.status == nb.NB_ERR_ARG
    assert "65536" in str(e.value)


def test_noalloc_rejects_host_pointer(nb):
    # A host address where a device array is required is refused before any
    # launch (checked by the C entry point, here given raw addresses).
    import torch
    n = 64
    dev = torch.device("cuda:0")
    xh = torch.zeros((n, 3)).pin_memory()
    m = torch.ones(n, device=dev)
    a = torch.empty((n, 3), device=dev)
    p = torch.empty(n, device=dev)
    with pytest.raises(nb.NBError) as e:
        nb.nb_force_noalloc(xh.data_ptr(), m, n, 0.1, a, p)
    assert e.value.status == nb.NB_ERR_ARG

"""CPU checks of the C ABI: the library builds, loads without a GPU, and
exports every entry point include/nbody.h declares. No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nbody.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0904_3659_gb300 import build
    build.build()
    import paper_0904_3659_gb300 as nb
    return nb


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nb_create", "nb_destroy", "nb_last_error", "nb_force", "nb_force_batched",
                     "nb_leapfrog_step", "nb_force_vjp", "nb_energy", "nb_synchronize",
                     "nb_autotune"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(lib.library_path)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    # The binding wraps exactly the declared set, under the same names.
    assert sorted(lib.exported_symbols) == declared_functions()


def test_host_only_calls(lib):
    assert lib.nb_status_string(lib.NB_ERR_TIMEOUT) == "NB_ERR_TIMEOUT"
    tiles = lib.nb_list_tiles(lib.NB_PLAIN)
    assert len(tiles) >= 4
    for t in tiles + lib.nb_list_tiles(lib.NB_COMPENSATED):
        # i-block: threads * ipt particles (a fused shape: 32 * ipt, shared by its warps)
        ib = 32 * t.ipt if t.fused else t.threads * t.ipt
        assert t.ipt % 2 == 0 and 3072 % ib == 0 and 3072 % t.jtile == 0
        assert t.stages >= (1 if t.fused else 2)
        assert t.threads % 32 == 0 and t.release in (0, 1) and t.unroll >= 1
        assert (t.jtile * 32) % 16 == 0
        assert t.refine in (0, 1) and t.fused in (0, 1, 2, 3)
    # Both arithmetic forms are compiled in each mode: the special-function
    # unit's rsqrt as is (the built-in default) and with one Newton step.
    for mode in (lib.NB_PLAIN, lib.NB_COMPENSATED):
        assert {t.refine for t in lib.nb_list_tiles(mode)} == {0, 1}
        # The single-launch forms: chunked (1), stream-K (2), cluster (3).
        assert {t.fused for t in lib.nb_list_tiles(mode)} == {0, 1, 2, 3}
    # The adjoint kernel's shapes: packed pairs, tiles dividing the padding.
    vjp = lib.nb_list_vjp_tiles()
    assert len(vjp) >= 2
    for t in vjp:
        assert t.ipt % 2 == 0 and 3072 % (t.threads * t.ipt) == 0 and 3072 % t.jtile == 0
        assert t.stages >= 2 and t.threads % 32 == 0 and t.fused == 0


def test_tile_struct_matches_header(lib):
    # The binding's nb_tile has the C struct's fields, in order.
    src = open(HEADER).read()
    body = re.search(r"typedef struct nb_tile \{(.*?)\} nb_tile;", src, re.S).group(1)
    fields = re.findall(r"int (\w+);", body)
    assert [f for f, _ in lib.nb_tile._fields_] == fields


def test_create_reports_error_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.NBError) as e:
        lib.Context(0)
    assert e.value.status in (lib.NB_ERR_CUDA, lib.NB_ERR_ARG)


def test_binding_validates_device_arguments(lib):
    # Wrong dtype, layout, size or device is refused by the binding before
    # any library call (no GPU needed: the checks run first).
    torch = pytest.importorskip("torch")
    n = 10
    x32 = torch.zeros((n, 3), dtype=torch.float32)
    m32 = torch.zeros(n, dtype=torch.float32)
    a32, p32 = torch.zeros((n, 3)), torch.zeros(n)
    with pytest.raises(TypeError, match="x must be float32"):
        lib.nb_force(None, x32.double(), m32, n, 0.1, a32, p32)
    with pytest.raises(ValueError, match="contiguous"):
        lib.nb_force(None, torch.zeros((3, n)).t(), m32, n, 0.1, a32, p32)
    with pytest.raises(ValueError, match="needs 30"):
        lib.nb_force(None, x32[:9], m32, n, 0.1, a32, p32)
    with pytest.raises(TypeError, match="CUDA"):
        lib.nb_force(None, x32, m32, n, 0.1, a32, p32)
    with pytest.raises(TypeError, match="x must be float64"):
        lib.nb_leapfrog_step(None, x32, x32, m32, a32, None, n, 0.1, 0.01, 1, 0)
    with pytest.raises(TypeError, match="offsets must be int64"):
        # (raw integer addresses pass unchecked; offsets is checked next)
        lib.nb_force_batched(None, 0, 0, torch.zeros(2, dtype=torch.int32), 1, n,
                             torch.zeros(1), a32, p32)

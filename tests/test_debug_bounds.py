"""The bounds-checked build (libnbody_debug.so, -DNB_DEBUG) checks every
computed-index access of the kernels against its buffer and records a
violation instead of making it. A selection of parity tests that exercises
every kernel (single system plain and compensated, every tile shape, ragged
sizes, batches with empty and invalid clusters, FP64 state with positions
split into grid part and remainder, the adjoint, the allocation-free entry
point) runs against that build in a fresh process: any violation fails the
test that saw it."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_selection_under_bounds_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_3659_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, NB_LIBRARY=lib)
    sel = ("ragged or every_tile or coincident or uneven or invalid or far_from_origin or "
           "compensated_kdk or final_force or "
           "zero_steps or fp64_state or vjp_matches_oracle or noalloc")
    files = ["tests/test_force_parity.py", "tests/test_batched_parity.py",
             "tests/test_leapfrog_parity.py", "tests/test_vjp_parity.py",
             "tests/test_zz_no_alloc.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", *files, "-q", "-m", "gpu", "-k", sel,
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert "passed" in r.stdout

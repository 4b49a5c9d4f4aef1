"""The arithmetic fact the pair kernels' default form rests on: on sm_103a the
special-function unit's reciprocal square root is within 2^-22.9 relative of
1/sqrt(s) (the PTX ISA's bound for rsqrt.approx.f32), and one Newton-Raphson
step evaluated in FP32 does not lower that maximum, because its own three
roundings are of the same size. The probe (tests/gpu_probes/rsqrt_accuracy.cu)
checks every FP32 value in [1, 4), i.e. every mantissa and both exponent
parities, against FP64."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

PROBE = os.path.join(os.path.dirname(__file__), "gpu_probes", "rsqrt_accuracy.cu")
BOUND = 2.0 ** -22.9


@pytest.fixture(scope="module")
def errors(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("probe") / "rsqrt_accuracy")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, PROBE],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    res = {}
    for line in out.splitlines():
        name, mx, mean = line.split()
        res[name] = (float(mx), float(mean))
    return res


def test_sfu_rsqrt_within_ptx_bound(errors):
    assert errors["y"][0] <= BOUND, errors["y"]
    # y^3 (the force's s^{-3/2}) then stays within about 3 times that.
    assert errors["y3"][0] <= 3 * BOUND + 1e-9, errors["y3"]


def test_newton_step_does_not_lower_max_error(errors):
    raw, newton = errors["y"][0], errors["y1"][0]
    assert newton >= 0.9 * raw, (raw, newton)
    assert errors["y13"][0] >= 0.9 * errors["y3"][0]

"""The issue ceiling the pair kernels run against: sustained FP32 lane
operations per SM clock for scalar FFMA and packed FFMA2 multiply-add chains
(tests/gpu_probes/fp32_issue_rate.cu). The probe counts SM cycles itself
(clock64) and reads the global timer beside them, so the rates are per clock
of the run and its effective SM clock is measured, not assumed. The pair
kernels issue their arithmetic as FFMA2/FADD2/FMUL2 (two lanes per
instruction), so the packed rate, not the nominal 128 lanes per clock, is the
ceiling their FP32-pipe share is read against."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

PROBE = os.path.join(os.path.dirname(__file__), "gpu_probes", "fp32_issue_rate.cu")


@pytest.fixture(scope="module")
def rates(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("probe") / "fp32_issue_rate")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, PROBE],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    res = {}
    for line in out.splitlines():
        name, rate, mhz, sms = line.split()
        res[name] = (float(rate), float(mhz), int(sms))
    print(res)
    return res, torch.cuda.get_device_properties(0).multi_processor_count


def test_scalar_ffma_near_128_lanes(rates):
    res, sms = rates
    rate, mhz, distinct = res["ffma"]
    assert distinct == sms                 # one CTA on every SM
    assert 100.0 < rate <= 128.5, rate     # at most the 128 FP32 lanes of an SM
    assert 500.0 < mhz < 2500.0, mhz


def test_packed_ffma2_rate(rates):
    res, sms = rates
    rate, mhz, distinct = res["ffma2"]
    assert distinct == sms
    assert 64.0 < rate <= 128.5, rate

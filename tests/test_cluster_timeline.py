"""Where one N = 4096 force call spends its time in the cluster form of the
single-launch kernel (tests/gpu_probes/cluster_timeline.cu: the library's
kernel with %globaltimer stamps, 400 launches back to back with programmatic
dependent launch). The phases must account for the launch-to-launch time,
and the compute phase must dominate it."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(__file__)
ROOT = os.path.dirname(HERE)
PROBE = os.path.join(HERE, "gpu_probes", "cluster_timeline.cu")


@pytest.fixture(scope="module")
def phases(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("probe") / "cluster_timeline")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "include"), "-o", exe, PROBE],
                   check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120).stdout
    print(out)
    res = {}
    for line in out.splitlines():
        name, *vals = line.split()
        res[name] = vals
    return res


def test_probe_ran_clean(phases):
    assert phases["status"] == ["ok", "0"]


def test_phases_account_for_the_launch(phases):
    med = {k: float(v[1]) for k, v in phases.items() if len(v) == 3}
    per_launch = float(phases["per_launch_us"][0])
    parts = (med["pack"] + max(med["compute_cta_with_diagonal"], med["compute_other_cta"]) +
             med["cross_warp_sums"] + med["cluster_barrier_wait"] + med["send_and_arrival"] +
             med["combine_and_write"])
    # The span from the first CTA's release to the last CTA's exit holds the
    # median CTA's phases (plus CTA skew); span + gap is the launch period.
    assert parts <= med["span_release_to_last_exit"] + 0.5
    assert abs(med["span_release_to_last_exit"] + med["gap_previous_exit_to_release"] - per_launch) < 1.0
    assert min(med.values()) >= 0.0
    assert med["compute_other_cta"] > 0.5 * per_launch

"""The integer-pipe float <-> double conversions of the FP32-bulk kernels equal IEEE
round-to-nearest-even conversions bit for bit: the bit recipes against the host CPU's
converters (no GPU), and the device functions -- fast and slow paths -- against the GPU's
hardware converters.  The harness is tests/native/conv_check.cu, built here with nvcc."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "conv_check.cu")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("conv") / "conv_check")
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-o", exe, SRC], check=True)
    return exe


def _run(exe, mode, n):
    out = subprocess.run([exe, mode, str(n)], capture_output=True, text=True, timeout=600)
    words = out.stdout.split()
    assert out.returncode == 0 and words[:1] == ["mismatches"], (out.returncode, out.stdout,
                                                                 out.stderr)
    return int(words[1]), int(words[3])


def test_bit_recipes_match_host_conversions(harness):
    bad, checked = _run(harness, "host", 4_000_000)
    assert bad == 0 and checked > 4_000_000


@pytest.mark.gpu
def test_device_conversions_match_hardware(harness):
    bad, checked = _run(harness, "device", 200_000_000)
    assert bad == 0 and checked == 400_000_000

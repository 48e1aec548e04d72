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


@pytest.fixture(scope="module")
def root_harness(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("roots") / "root_check")
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-o", exe, os.path.join(HERE, "native", "root_check.cu")], check=True)
    return exe


@pytest.mark.gpu
def test_fp64_roots_within_one_ulp(root_harness):
    # the production FP64 square root and reciprocal square root (FP32 estimate and two
    # Newton-Raphson steps) are faithful: within 1 ulp of the exact root in the fast range;
    # warps with an argument outside it equal the library functions bit for bit
    out = subprocess.run([root_harness, "4000000"], capture_output=True, text=True, timeout=600)
    words = out.stdout.split()
    assert out.returncode == 0 and words[:1] == ["mismatches"], (out.stdout, out.stderr)
    print(out.stdout)
    assert int(words[1]) == 0 and int(words[3]) >= 4_000_000
    assert float(words[5]) <= 1.0 and float(words[7]) <= 1.0


@pytest.fixture(scope="module")
def threshold_harness(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("thr") / "threshold_check")
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-o", exe, os.path.join(HERE, "native", "threshold_check.cu")], check=True)
    return exe


@pytest.mark.gpu
def test_fp64_hlld_threshold_tests_match_the_comparisons(threshold_harness):
    # the FP64 HLLD degeneracy and HLLC-limit tests decide from the binary exponents where
    # those settle the question and compare in FP64 otherwise: every decision equals the
    # plain comparison's, on values across the exponent range, near both thresholds, zeros,
    # subnormals and negative values, mixed within warps
    out = subprocess.run([threshold_harness, "8000000"], capture_output=True, text=True,
                         timeout=600)
    words = out.stdout.split()
    assert out.returncode == 0 and words[:1] == ["mismatches"], (out.stdout, out.stderr)
    print(out.stdout)
    assert int(words[1]) == 0 and int(words[3]) >= 8_000_000
    # the near-threshold cases do reach the comparisons
    assert int(words[5]) > 0 and int(words[7]) > 0


@pytest.fixture(scope="module")
def pow2_harness(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("pow2") / "pow2_check")
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-o", exe, os.path.join(HERE, "native", "pow2_check.cu")], check=True)
    return exe


@pytest.mark.gpu
def test_fp64_power_of_two_scalings_equal_the_products(pow2_harness):
    # x/4, x/2 and 4x of the FP64 HLLD and E^c by the exponent field: bit for bit the
    # products, in warps that take the integer path and in warps where a zero, subnormal,
    # end-of-range, infinite or NaN lane sends the warp to the multiply
    out = subprocess.run([pow2_harness, "4000000"], capture_output=True, text=True, timeout=600)
    words = out.stdout.split()
    assert out.returncode == 0 and words[:1] == ["mismatches"], (out.stdout, out.stderr)
    print(out.stdout)
    assert int(words[1]) == 0 and int(words[3]) >= 12_000_000
    assert int(words[5]) >= 4_000_000 // 32 // 2 - 1000  # half the warps take the integer path


def test_multiply_and_shift_division_equals_the_quotient(tmp_path):
    # the cell-coordinate division of the kernels (divmagic.cuh, host side; the same
    # function runs on the device) against the division operator, on the host
    exe = str(tmp_path / "divmagic_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", exe,
                    os.path.join(HERE, "native", "divmagic_check.cpp")], check=True)
    out = subprocess.run([exe, "200000"], capture_output=True, text=True, timeout=300)
    words = out.stdout.split()
    assert out.returncode == 0 and words[:1] == ["mismatches"], (out.stdout, out.stderr)
    assert int(words[1]) == 0 and int(words[3]) > 4_000_000

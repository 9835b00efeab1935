"""CPU checks of the arithmetic inside the CUDA kernels (csrc/hostdev.h),
compiled for the host with g++: the in-place FFT passes against a direct DFT,
the real-FFT packing on digit-reversed data against its definition, the
column kernel's transform pair, the shared-memory swizzles, and the cubic
B-spline tap weights."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("hd") / "hostdev_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_1604_07651_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "hostdev_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_fft_passes(results):
    """Forward passes read back through the position map, inverse passes on
    digit-reversed input, every supported length, against a direct DFT."""
    assert results["fft_rel_l2"] < 5e-7


def test_real_fft_packing(results):
    assert results["rfft_rel_l2"] < 5e-7
    assert results["irfft_rel_l2"] < 5e-7


def test_dif_dit_transform_pair(results):
    """The column kernel's in-place pair: forward passes by decimation in
    frequency, product at each position's digit-reversed frequency, inverse
    passes by decimation in time, for every supported length, against
    n * IDFT(K .* DFT(x)) in FP64."""
    assert results["dif_freq_violations"] == 0
    assert results["dif_conv_rel_l2"] < 1e-6


def test_b3_weights(results):
    assert results["b3_weights"] < 1e-6


def test_b5_weights(results):
    """Quintic tap weights against the truncated-power definition of B5 and
    their partition of unity."""
    assert results["b5_weights"] < 1e-6


def test_shared_memory_swizzle_is_a_permutation(results):
    assert results["swizzle_violations"] == 0
    # 2^a <= 4096, 3 2^a <= 6144, 5 2^a <= 5120 and 9 2^a <= 2304: 13 + 12 + 11 + 9 lengths
    assert results["fft_lengths"] == 45

"""The hardware approximations under the counting kernels' FP32 binning hold
the error bounds the host planner assumes for them: lg2.approx.ftz.f32
within 2^-21 + 2^-22 |log2 x| of log2(x) (the log-spaced binning of log r
and log theta edges; the second part covers the rounding of the FP32
result, measured at about one ulp) and rsqrt.approx.ftz.f32 within 2^-22.9 of 1/sqrt(x), relative (every
arithmetic binning).  tests/approx_bound_check.cu evaluates both on every
FP32 mantissa of every exponent in [2^-60, 2^70) and reports the largest
error against the FP64 functions."""
import os
import shutil
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_hardware_approximations_within_assumed_bounds(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "approx_bound_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    os.path.join(HERE, "approx_bound_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lg, lgn, rs = (float(x) for x in r.stdout.split())
    print("lg2.approx max abs error %.3e (%.3f of the bound), rsqrt.approx max rel error %.3e"
          % (lg, lgn, rs))
    # the host replay of the binning (fp32_band_check.cpp) perturbs log2 by
    # half the planner's bound: the hardware must stay within that half
    assert 0 < lgn <= 0.5
    assert 0 < rs <= 2.0 ** -22.9

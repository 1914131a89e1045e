"""The GPU tests cannot run without a device, but they must at least import
and collect here: a syntax or import error in one of them would otherwise
surface only on a GB300."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpu_tests_collect():
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests"), "-m", "gpu",
                        "--collect-only", "-q", "-p", "no:cacheprovider"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    n = sum(1 for ln in r.stdout.splitlines() if "::" in ln and ln.startswith("tests/"))
    assert n >= 100, r.stdout[-2000:]
    for f in ("test_gpu_parity.py", "test_gpu_fullsize.py", "test_gpu_weighted.py",
              "test_gpu_batched.py", "test_gpu_density.py", "test_gpu_pixel.py",
              "test_gpu_sky.py", "test_zz_no_alloc.py"):
        assert ("tests/" + f + "::") in r.stdout, f

"""Host check of the counting kernel's neighbour cull: tests/cull_check.cpp
replays the kernel's FP32 gap test (a row against the bounding box of the
item's home objects in FP32 image coordinates) with the radii the host sets
(plan.cpp: cull_params), on pairs at and just inside the reach -- along axes
and diagonals, at far corners of frames up to 9e7, across periodic images,
monopole and (sigma, pi) -- and requires every pair within the reach by the
canonical FP64 separation (Sec. 2.2, Sec. 3.4) to be kept, while rows 1e-4
beyond the reach are dropped where the frame's rounding allows.  With the
radii's widening removed the replay must find dropped pairs, so it does
detect a margin that is too small."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1210_1833_gb300", "csrc")


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return c
    return None


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda = _cuda_home()
    if cxx is None or cuda is None:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    out = str(tmp_path_factory.mktemp("cull") / "cull_check")
    lib = next((d for d in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib")
                if os.path.exists(os.path.join(cuda, d, "libcudart.so"))), "lib64")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", os.path.join(cuda, "include"),
                    os.path.join(HERE, "cull_check.cpp"), os.path.join(CSRC, "plan.cpp"),
                    "-L", os.path.join(cuda, lib), "-lcudart", "-Wl,-rpath," + os.path.join(cuda, lib),
                    "-o", out], check=True)
    return out


def _rows(stdout):
    rows = {}
    for line in stdout.splitlines():
        p = line.split()
        if len(p) == 8 and p[4] == "beyond":
            rows[p[0]] = dict(kept=int(p[1]), dropped=int(p[2]), violations=int(p[3]),
                              beyond=int(p[5]), beyond_kept=int(p[7]))
    return rows


def test_cull_keeps_every_pair_within_reach(exe):
    r = subprocess.run([exe], capture_output=True, text=True)
    rows = _rows(r.stdout)
    assert r.returncode == 0, r.stdout
    assert len(rows) == 9
    for name, v in rows.items():
        assert v["violations"] == 0 and v["dropped"] == 0, name
        assert v["kept"] > 100000, name
        assert v["beyond_kept"] == 0, name
    # the tight scenarios did test rows beyond the reach
    assert sum(v["beyond"] > 0 for v in rows.values()) == 6


def test_cull_without_margin_is_caught(exe):
    r = subprocess.run([exe, "nomargin"], capture_output=True, text=True)
    rows = _rows(r.stdout)
    assert r.returncode == 1
    assert len(rows) == 9
    assert all(v["violations"] > 0 for v in rows.values())

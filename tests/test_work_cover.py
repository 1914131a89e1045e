"""Host check of the counting kernels' work decomposition (Sec. 3.3 cell
lists): tests/work_cover_check.cu expands the home chunks, stencil rows and
segments that the library hands to the kernel (chunks_build, stencil_build,
entry_segments, with cell grids that follow the grid contract) into object
pairs, for the half stencil of auto counts, the full stencil of the adjoint
and cross counts, periodic and open, ball, disk-slab and box reaches, two
home-chunk sizes, 1 to 8 cells per reach, and grids that need the threaded
chunk builder.  Every
pair within reach must be met exactly once and through the image that puts
it within reach; pairs beyond reach met twice (periodic half stencils) are
out of range both times and only reported."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1210_1833_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                     if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("needs nvcc (the segment function sits in a CUDA header)")
    out = str(tmp_path_factory.mktemp("cover") / "work_cover_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-Xcompiler", "-pthread", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    os.path.join(HERE, "work_cover_check.cu"), os.path.join(CSRC, "plan.cpp"),
                    "-o", out], check=True)
    return out


def test_every_pair_within_reach_met_exactly_once(exe):
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    rows = {}
    for line in r.stdout.splitlines():
        p = line.split()
        if len(p) == 5 and p[1].isdigit():
            rows[p[0]] = tuple(int(x) for x in p[1:])
    # 7 geometries x 2 chunk sizes x 3 pair-set modes at 1-3 cells per
    # reach, and 5 geometries x 2 x 3 at each of 4-8 cells per reach
    assert len(rows) == 42 + 5 * 6 * 5, r.stdout
    for k in range(4, 9):
        assert sum(name.endswith("_k%d" % k) for name in rows) == 30
    for name, (enumerated, inreach, dup, bad) in rows.items():
        assert bad == 0, (name, r.stdout)
        assert inreach > 300 and enumerated >= inreach, name
        if "auto_half" not in name or name.startswith("open"):
            assert dup == 0, name
        assert dup <= 0.001 * enumerated, name
    assert r.returncode == 0, r.stdout

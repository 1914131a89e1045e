"""Host check of the counting kernel's shared-memory layout:
tests/smem_layout_check.cu enumerates the layouts smem_layout gives for
every accumulation policy, home objects per lane, table and band size, slot
count and histogram copies, and checks that every region the kernel
addresses -- tables, histograms, queue, tile buffers and their weight
tiles, home box, culled-row indices -- and every warp's block start on a
16-byte boundary (cp.async rows and float4 accesses need it), and that a
tile buffer has room for a culled run's carried and padding rows."""
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
        pytest.skip("needs nvcc (the layout sits in a CUDA header)")
    out = str(tmp_path_factory.mktemp("layout") / "smem_layout_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    os.path.join(HERE, "smem_layout_check.cu"), "-o", out], check=True)
    return out


def test_every_region_is_16_byte_aligned(exe):
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    last = r.stdout.split()
    assert last[-4] == "layouts" and int(last[-3]) > 10000 and int(last[-1]) == 0

"""Host check of the counting kernel's FP32 near-edge bands:
tests/fp32_band_check.cpp replays the kernel's FP32 binning arithmetic (same
operation order, IEEE roundings, the hardware reciprocal square root anywhere
within its documented error) with the thresholds, tables and bands of the
host planner, on pairs on and around every edge of the monopole, chord,
(sigma, pi) and (r, mu) binnings -- uniform edges from 0 (binning by
arithmetic) and log-spaced edges (the lookup-table path) -- and on every
pair of integer lattices, where hundreds of pairs sit exactly on an edge in
FP64 (mu = 1/2 included); no pair the kernel would not re-test may fall in
another slot than the canonical FP64 formulas give (Sec. 2.2, Sec. 3.4).  The check also runs with the thresholds' (and
bands') distance from the edge halved and at 0.3, so the planner's bounds
keep a margin over what these pairs need; with the bands collapsed it must
find misbinned pairs, so the replay does detect a too-narrow band."""
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
    out = str(tmp_path_factory.mktemp("band") / "fp32_band_check")
    lib = next((d for d in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib")
                if os.path.exists(os.path.join(cuda, d, "libcudart.so"))), "lib64")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", os.path.join(cuda, "include"),
                    os.path.join(HERE, "fp32_band_check.cpp"), os.path.join(CSRC, "plan.cpp"),
                    "-L", os.path.join(cuda, lib), "-lcudart", "-Wl,-rpath," + os.path.join(cuda, lib),
                    "-o", out], check=True)
    return out


def _run(exe, factor):
    r = subprocess.run([exe, str(factor)], capture_output=True, text=True)
    rows, ties = {}, {}
    for line in r.stdout.splitlines():
        p = line.split()
        if len(p) == 4 and p[1].isdigit():
            rows[p[0]] = tuple(int(x) for x in p[1:])
        elif len(p) == 2 and p[0].endswith("_ties"):
            ties[p[0][:-5]] = int(p[1])
    return r.returncode, rows, r.stdout, ties


@pytest.mark.parametrize("factor", [1.0, 0.5, 0.3])
def test_no_unflagged_pair_is_misbinned(exe, factor):
    rc, rows, out, ties = _run(exe, factor)
    # 14 edge scenarios (6 arithmetic, 5 table, 3 log-spaced) and 10 integer
    # lattices, each with 3 ways of rounding the rsqrt (and the log2)
    assert len(rows) == 72, out
    assert sum(n.startswith("table_") for n in rows) == 15, out
    assert sum(n.startswith("log_") or "_log_" in n for n in rows) == 15, out
    lattices = [n for n in rows if n.startswith("lattice_")]
    assert len(lattices) == 30 and set(ties) == set(lattices), out
    for name, (cases, flagged, bad) in rows.items():
        assert cases > 1000 and bad == 0, (name, out)
    # the lattices hold exact FP64 ties, every one of them flagged or binned right
    # (the log-spaced edges 1, 2, 4, 8, 16 have fewer exact ties)
    assert all(ties[n] >= (60 if "_log_" in n else 100) for n in lattices), out
    assert rc == 0, out


def test_collapsed_bands_are_caught(exe):
    # thresholds at the edge itself: every edge scenario must show misbinned
    # pairs (a lattice whose FP32 values are exact can keep its ties flagged
    # even then, so the lattices are counted together)
    rc, rows, out, _ = _run(exe, 0.0)
    assert len(rows) == 72 and rc == 1, out
    for name, (cases, flagged, bad) in rows.items():
        if not name.startswith("lattice_"):
            assert bad > 0, (name, out)
    assert sum(v[2] for n, v in rows.items() if n.startswith("lattice_")) > 0, out

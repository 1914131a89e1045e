"""Host check of the double-float first stage of the edge re-test
(paper_1210_1833_gb300/csrc/df_stage.h, compiled for the host here): on
pairs on, and a hair off, every edge of the monopole, chord, (sigma, pi) and
(r, mu) binnings, open and periodic, every slot the stage decides equals the
slot of the canonical FP64 formulas (Sec. 2.2 and 3.4), and the stage decides
the pairs that are not within its error bound of an edge.  On integer
lattices (integer coordinates and edges, mu edges k/4, pairs at exactly
mu = 1/2) every FP64 quantity is exact and hundreds of pairs sit exactly on
an edge: the stage must leave those to FP64 or decide them exactly right."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("dfs") / "df_stage_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "df_stage_check.cpp")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    rows, ties = {}, {}
    for line in r.stdout.splitlines():
        parts = line.split()
        if len(parts) == 4 and parts[1].isdigit():
            rows[parts[0]] = tuple(int(x) for x in parts[1:])
        elif len(parts) == 2 and parts[0].endswith("_ties"):
            ties[parts[0][:-5]] = int(parts[1])
    return r.returncode, rows, r.stdout, ties


def test_no_decision_differs_from_fp64(results):
    rc, rows, out, ties = results
    assert rc == 0, out
    lattices = {"lattice_mono_periodic", "lattice_mono_open", "lattice_sigpi_periodic",
                "lattice_rmu"}
    assert set(rows) == {"mono_open", "mono_periodic", "mono_periodic_odd_box", "chord",
                         "sigpi_periodic", "sigpi_open", "rmu_lightcone", "rmu_centred"} | lattices
    for name, (cases, decided, bad) in rows.items():
        assert bad == 0, (name, out)
    assert set(ties) == lattices and all(v >= 100 for v in ties.values()), out


def test_stage_decides_pairs_off_the_edges(results):
    # the offsets from the edges span 0 to 0.3 relative; the stage must leave
    # only those within about 1e-10 of an edge to FP64
    _, rows, out, _ = results
    for name, (cases, decided, bad) in rows.items():
        assert cases > 0 and decided >= 0.4 * cases, (name, out)

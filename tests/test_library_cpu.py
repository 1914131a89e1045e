"""Host-side checks of libcute_gb.so that need no GPU: the library loads,
exports every entry point include/cute.h declares, the Python binding's
ctypes signatures and struct mirrors match the header, and the host-only
functions (estimators, angle -> chord) agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import cute

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "cute.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cute_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = cute.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(cute.SYMBOLS) == set(names)
    assert "sm_103a" in cute.version()


def test_ctx_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(cute.CuteError):
        cute.Context(0)


def test_theta_to_chord_matches_oracle_bit_exactly():
    t = 10.0 ** (-2.0 + 3.0 * np.arange(65) / 64.0)
    assert cute.theta_to_chord(t).tolist() == oracle.theta_to_chord(t).tolist()
    with pytest.raises(cute.CuteError):
        cute.theta_to_chord([-1.0])


@pytest.mark.parametrize("seed", [0, 1])
def test_estimators_match_oracle(seed):
    rng = np.random.default_rng(seed)
    nb = 40
    DD = rng.integers(0, 10**9, size=nb).astype(np.uint64)
    DR = rng.integers(0, 10**10, size=nb).astype(np.uint64)
    RR = rng.integers(1, 10**11, size=nb).astype(np.uint64)
    RR[3] = 0
    Nd, Nr = 500_000, 2_000_000
    for name, ref in (("ls", oracle.xi_ls(DD, DR, RR, Nd, Nr)),
                      ("natural", oracle.xi_natural(DD, RR, Nd, Nr))):
        got = cute.estimator(name, DD, DR, RR, Nd, Nr)
        assert np.isnan(got[3]) and np.isnan(ref[3])
        m = ~np.isnan(ref)
        np.testing.assert_allclose(got[m], ref[m], rtol=1e-12, atol=1e-12)
    e = np.arange(nb + 1) * 5.0
    got = cute.estimator("periodic", DD, Nd=20000, edges=e, L=1000.0)
    ref = oracle.xi_periodic(DD, 20000, e, 1000.0)
    m = ~np.isnan(ref)
    np.testing.assert_allclose(got[m], ref[m], rtol=1e-12, atol=1e-12)


def test_estimator_rejects_bad_input():
    with pytest.raises(cute.CuteError):
        cute.estimator("ls", [1, 2], None, [1, 2], 10, 20)
    with pytest.raises(cute.CuteError):
        cute.estimator("periodic", [1, 2], Nd=1, edges=[0, 1, 2], L=10)


def test_weighted_count_is_an_autograd_function():
    """The binding's differentiable weighted count (forward: weighted count,
    backward: adjoint) is a torch.autograd.Function."""
    torch = pytest.importorskip("torch")
    assert issubclass(cute.CuteWeightedCount, torch.autograd.Function)


def test_multipoles_match_oracle():
    """cute_multipoles (Bonnet recurrence, bin-edge differences) equals the
    oracle (numpy Legendre antiderivatives) on uneven mu bins."""
    rng = np.random.default_rng(82)
    m = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0, 1, 38)]))
    xi = rng.normal(size=(40, 39))
    ells = (0, 2, 4, 6, 8)
    got = cute.multipoles(xi, m, ells)
    ref = oracle.multipoles(xi, m, ells)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("bad", ["edges", "odd", "range"])
def test_multipoles_reject_bad_input(bad):
    xi = np.zeros((3, 4))
    m = np.linspace(0, 1, 5)
    ells = (0, 2)
    if bad == "edges":
        m = np.linspace(0, 0.9, 5)
    elif bad == "odd":
        ells = (1,)
    else:
        ells = (18,)
    with pytest.raises(cute.CuteError):
        cute.multipoles(xi, m, ells)


def test_weighted_estimators_match_oracle():
    rng = np.random.default_rng(85)
    DD, DR, RR = (rng.uniform(1, 1e6, 30) for _ in range(3))
    RR[3] = 0.0
    args = (1234.5, 2001.25, 8765.0, 9000.5)
    for kind in ("natural", "ls"):
        got = cute.estimator_weighted(kind, DD, DR, RR, *args)
        ref = oracle.xi_weighted(kind, DD, DR, RR, *args)
        np.testing.assert_allclose(got, ref, rtol=1e-13, equal_nan=True)
    with pytest.raises(cute.CuteError):
        cute.estimator_weighted("periodic", DD, DR, RR, *args)


# ------------------------------------------------------------------ ABI of the binding
_SCALARS = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double,
            "float": ctypes.c_float, "int": ctypes.c_int, "cute_boundary": ctypes.c_int,
            "cute_kind": ctypes.c_int, "cute_estimator_kind": ctypes.c_int}


def _prototypes():
    txt = open(os.path.join(ROOT, "include", "cute.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for name, args in re.findall(r"(?:cute_status|const char \*)\s*(cute_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                                 txt, flags=re.S):
        a = [x.strip() for x in args.split(",")]
        out[name] = [] if a == ["void"] else a
    return out


def test_binding_signatures_match_the_header():
    """Every prototype of include/cute.h against the binding's ctypes
    argtypes: same number of arguments, pointers where the header has
    pointers, and scalars of the header's width."""
    L = cute.lib()
    protos = _prototypes()
    assert set(protos) == set(cute.SYMBOLS)
    for name, args in protos.items():
        at = getattr(L, name).argtypes
        if not args:
            assert not at, name
            continue
        assert at is not None and len(at) == len(args), name
        for a, t in zip(args, at):
            if "*" in a or "[" in a:
                assert t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer), (name, a)
            else:
                base = a.replace("const ", "").split()[0]
                assert t is _SCALARS[base], (name, a, t)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout: a small
    C program compiled against include/cute.h prints sizeof and the offset
    of every field the mirror names."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("needs a C compiler")
    pairs = [(cute.PairDesc, "cute_pair_desc"), (cute.Stats, "cute_stats"),
             (cute.Tuning, "cute_tuning"), (cute.Cosmology, "cute_cosmology")]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cute.h"', "int main(void) {"]
    for py, c in pairs:
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (c, c))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (c, f, c, f))
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict((" ".join(ln.split()[:2]), int(ln.split()[2]))
               for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.splitlines())
    for py, c in pairs:
        assert got[c + " sizeof"] == ctypes.sizeof(py), c
        for f, _ in py._fields_:
            assert got["%s %s" % (c, f)] == getattr(py, f).offset, (c, f)

"""Mutation check of the oracle's pins (no GPU).

The oracle is trusted because tests/test_oracle.py pins it to things other
than itself.  Here plausible mistakes -- a dropped term, a wrong sign, a
wrong index, a transposed operand, an off-by-one loop or a wrong
normalisation -- are planted one at a time in scratch copies of the oracle
(oracle.c rebuilt into the copy's own library, the numpy functions of
oracle/__init__.py edited in the copy), and every pin of test_oracle.py is
run against each copy: each planted mistake must make at least one pin fail.
The oracle itself carries no switch for this; the mistakes are textual edits
of copies, and the unedited copy must pass every pin.
"""
import importlib.util
import inspect
import itertools
import os
import shutil
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")

# tag -> (file, old text, new text, occurrences of the old text)
C, PY = "oracle.c", "__init__.py"
MUTANTS = {
    # minimum image (Sec. 2.2)
    "wrap_sign": (C, "if (d > s->halfL) d -= s->L;", "if (d > s->halfL) d += s->L;", 1),
    "wrap_full_box": (C, "if (d > s->halfL) d -= s->L;\n    else if (d < -s->halfL) d += s->L;",
                      "if (d > s->L) d -= s->L;\n    else if (d < -s->L) d += s->L;", 1),
    # separations (Eq. 2, Eq. 7, Eq. 11)
    "mono_drop_dz": (C, "double d2 = (dx * dx + dy * dy) + dz * dz;",
                     "double d2 = dx * dx + dy * dy;", 1),
    "sigma_wrong_index": (C, "double sg2 = dx * dx + dy * dy;", "double sg2 = dx * dx + dx * dx;", 1),
    "pi_wrong_axis": (C, "double pi2 = dz * dz;", "double pi2 = dx * dx;", 1),
    "sigpi_transposed_bin": (C, "return bs * s->n1 + bp;", "return bp * s->n0 + bs;", 1),
    "rmu_drop_sz": (C, "double r2 = (sx * sx + sy * sy) + sz * sz;",
                    "double r2 = sx * sx + sy * sy;", 1),
    "rmu_los_index": (C, "lz = a[2] + b[2];", "lz = a[2] + a[2];", 1),
    "rmu_dot_transposed": (C, "double sl = (sx * lx + sy * ly) + sz * lz;",
                           "double sl = (sx * lx + sy * lx) + sz * lz;", 1),
    "rmu_drop_r2_in_den": (C, "double den = r2 * L2;", "double den = L2;", 1),
    "mu_edges_not_squared": (C, "s->E1[k] = e1[k] * e1[k];", "s->E1[k] = e1[k];", 1),
    "edges_not_squared": (C, "s->E0[k] = e0[k] * e0[k];", "s->E0[k] = e0[k];", 1),
    # bins: half-open [e_b, e_{b+1})
    "bin_closed_top": (C, "if (!(v >= E[0]) || !(v < E[n])) return -1;",
                       "if (!(v >= E[0]) || !(v <= E[n])) return -1;", 1),
    "bin_edge_to_lower": (C, "if (v >= E[mid]) lo = mid; else hi = mid;",
                          "if (v > E[mid]) lo = mid; else hi = mid;", 1),
    "mu_edge_to_lower": (C, "if (q >= t) lo = mid; else hi = mid;",
                         "if (q > t) lo = mid; else hi = mid;", 1),
    # pair enumeration
    "auto_self_pairs": (C, "int64_t j0 = is_auto ? i + 1 : 0;", "int64_t j0 = is_auto ? i : 0;", 1),
    "oor_not_counted": (C, "if (b < 0) { mc[nbins]++; continue; }", "if (b < 0) { continue; }", 1),
    "weight_wrong_operand": (C, "mc[b]++;\n        if (want_w) cs_add(&mw[b], (double)wa[i] * (double)wb[j]);",
                             "mc[b]++;\n        if (want_w) cs_add(&mw[b], (double)wa[i] * (double)wa[i]);", 1),
    # cell pruning (Sec. 3.3)
    "cells_one_sided": (C, "for (int d = -1; d <= 1; d++) {", "for (int d = 0; d <= 1; d++) {", 1),
    "cells_pairs_twice": (C, "if (is_auto && c2 < c1) continue;", "if (0 && c2 < c1) continue;", 1),
    "cells_self_pairs": (C, "if (is_auto && c2 == c1) q0 = p + 1;", "if (is_auto && c2 == c1) q0 = p;", 1),
    "cells_smaller_than_reach": (C, "double amin = reach[k] * (1.0 + 1e-9) + 1e-300;",
                                 "double amin = reach[k] * 0.5 + 1e-300;", 1),
    "cells_oor_total": (C, "(uint64_t)na * (uint64_t)(na > 0 ? na - 1 : 0) / 2",
                        "(uint64_t)na * (uint64_t)na / 2", 1),
    # gradient rows
    "grad_self_pair": (C, "if (is_auto && j == i) continue;", "if (0 && j == i) continue;", 1),
    "grad_drop_partner_weight": (C, "cs_add(&acc, (double)wpartner[j] * G[b]);",
                                 "cs_add(&acc, G[b]);", 1),
    # estimators (Eq. 13-15)
    "shell_not_cubed": (C, "(r2 * r2 * r2 - r1 * r1 * r1)", "(r2 * r2 - r1 * r1)", 1),
    "shell_drop_third": (C, "(4.0 * pi / 3.0)", "(4.0 * pi)", 1),
    "periodic_npairs_nsq": (C, "double npairs = 0.5 * (double)N * (double)(N - 1);",
                            "double npairs = (double)N * (double)N;", 1),
    "natural_drop_minus_one": (C, "f * (double)DD[b] / (double)RR[b] - 1.0",
                               "f * (double)DD[b] / (double)RR[b]", 1),
    "pair_ratio_inverted": (C, "((double)Nr * (double)(Nr - 1)) / ((double)Nd * (double)(Nd - 1))",
                            "((double)Nd * (double)(Nd - 1)) / ((double)Nr * (double)(Nr - 1))", 2),
    "ls_dr_sign": (C, "(f * (double)DD[b] - g * (double)DR[b] + (double)RR[b])",
                   "(f * (double)DD[b] + g * (double)DR[b] + (double)RR[b])", 1),
    "ls_dr_factor": (C, "double g = (double)(Nr - 1) / (double)Nd;",
                     "double g = (double)Nr / (double)Nd;", 1),
    "chord_drop_half": (C, "2.0 * sin(0.5 * theta_deg[k] * (pi / 180.0))",
                        "2.0 * sin(theta_deg[k] * (pi / 180.0))", 1),
    # multipoles (Eq. 3-4)
    "multipole_drop_2l1": (PY, "w = (2 * l + 1) * (anti(m[1:]) - anti(m[:-1]))",
                           "w = (anti(m[1:]) - anti(m[:-1]))", 1),
    # comoving distance and sky positions (Sec. 2.1, Sec. 3.4.2)
    "curvature_power": (PY, "ok * a ** 2", "ok * a ** 3", 1),
    "dark_energy_sign": (PY, "a ** (3.0 * (1.0 + w0))", "a ** (3.0 * (1.0 - w0))", 1),
    "sky_y_uses_cos": (PY, "np.cos(dec) * np.sin(ra), np.sin(dec)", "np.cos(dec) * np.cos(ra), np.sin(dec)", 1),
    # pixel maps
    "healpix_belt_slope": (PY, "np.sign(z) * (2.0 - sigma), 1.5 * z)",
                           "np.sign(z) * (2.0 - sigma), 1.0 * z)", 1),
    "healpix_cap_offset": (PY, "lambda r: 2 * r * (r - 1)", "lambda r: 2 * r * (r + 1)", 1),
    "healpix_cap_sigma": (PY, "sigma = np.sqrt(3.0 * (1.0 - np.where(polar, za, 1.0)))",
                          "sigma = np.sqrt(2.0 * (1.0 - np.where(polar, za, 1.0)))", 1),
    "healpix_belt_shift": (PY, "half = 1.0 - np.mod(ib - N, 2)", "half = np.mod(ib - N, 2)", 1),
    "healpix_ring_z": (PY, "z[polar] = np.sign(Yc[polar]) * (1.0 - sig * sig / 3.0)",
                       "z[polar] = np.sign(Yc[polar]) * (1.0 - sig * sig / 2.0)", 1),
    "weighted_dd_norm": (PY, "dd = DD / (0.5 * (s_d * s_d - q_d))", "dd = DD / (s_d * s_d - q_d)", 1),
    "weighted_ls_dr": (PY, "out = (dd - 2.0 * dr + rr) / rr", "out = (dd - dr + rr) / rr", 1),
    # density grid (Sec. 3.4.4)
    "tsc_weights_swapped": (PY, "wts = [0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2]",
                            "wts = [0.5 * (0.5 + d) ** 2, 0.75 - d * d, 0.5 * (0.5 - d) ** 2]", 1),
    "tsc_off_by_one": (PY, "ix = np.mod(i0[:, 0] + a - 1, n)", "ix = np.mod(i0[:, 0] + a, n)", 1),
    "lag_zero_included": (PY, "if (dz, dy) == (0, 0) and dx <= 0:", "if (dz, dy) == (0, 0) and dx < 0:", 1),
    # (a permuted or reflected roll is no mistake: each bin sums whole shells
    # of the cubic lag lattice, which every axis permutation and reflection
    # maps onto themselves)
    "lag_half_plane_twice": (PY, "if dz == 0 and dy < 0:", "if dz == 0 and dy < -R:", 1),
    "lag_spacing_not_squared": (PY, "r2 = (dx * dx + dy * dy + dz * dz) * a * a",
                                "r2 = (dx * dx + dy * dy + dz * dz) * a", 1),
    "lag_drop_grid_size": (PY, "s / (c * delta.size)", "s / c", 1),
}


def _load_pins():
    spec = importlib.util.spec_from_file_location("_oracle_pins", os.path.join(HERE, "test_oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _cases(pins):
    """(name, function, kwargs) for every test of the pin module, with its
    parametrize marks expanded."""
    out = []
    fns = [f for n, f in inspect.getmembers(pins, inspect.isfunction) if n.startswith("test_")]
    for fn in sorted(fns, key=lambda f: f.__code__.co_firstlineno):
        grids = []
        for m in getattr(fn, "pytestmark", []):
            if m.name != "parametrize":
                continue
            names = [s.strip() for s in m.args[0].split(",")]
            grids.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in m.args[1]])
        for combo in itertools.product(*grids):
            kw = {}
            for d in combo:
                kw.update(d)
            assert set(kw) == set(inspect.signature(fn).parameters), fn.__name__
            out.append((fn.__name__, fn, kw))
    return out


def _oracle_copy(root, tag, edit):
    """Copy of the oracle package under root/tag, with one edit applied,
    imported as its own package (its library is built in the copy)."""
    import oracle
    oracle._build.build()
    d = os.path.join(root, tag, "oracle")
    os.makedirs(d)
    for f in ("__init__.py", "_build.py", "oracle.c"):
        shutil.copy2(os.path.join(ORACLE, f), os.path.join(d, f))
    if edit is None or edit[0] != C:
        # the C source is unchanged: reuse the built library (mtime kept)
        shutil.copy2(os.path.join(ORACLE, "liboracle.so"), os.path.join(d, "liboracle.so"))
    if edit is not None:
        fname, old, new, n = edit
        p = os.path.join(d, fname)
        with open(p) as f:
            src = f.read()
        assert src.count(old) == n, "the planted edit %r no longer matches the oracle" % tag
        with open(p, "w") as f:
            f.write(src.replace(old, new))
    name = "_oracle_copy_" + tag
    spec = importlib.util.spec_from_file_location(name, os.path.join(d, "__init__.py"),
                                                  submodule_search_locations=[d])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    mod.lib()  # builds the copy's library
    return mod


def _failing_pins(pins, cases, mod, first_only):
    pins.oracle = mod
    failed = []
    for name, fn, kw in cases:
        try:
            fn(**kw)
        except pytest.skip.Exception:
            continue
        except Exception as e:  # an assertion, or an error status of the copy
            failed.append("%s%s: %s" % (name, kw or "", type(e).__name__))
            if first_only:
                break
    return failed


@pytest.fixture(scope="module")
def pins():
    return _load_pins()


def test_unedited_copy_passes_every_pin(pins, tmp_path):
    cases = _cases(pins)
    assert len(cases) >= 40
    mod = _oracle_copy(str(tmp_path), "identity", None)
    assert _failing_pins(pins, cases, mod, first_only=False) == []


@pytest.mark.parametrize("tag", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(pins, tmp_path, tag):
    mod = _oracle_copy(str(tmp_path), tag, MUTANTS[tag])
    failed = _failing_pins(pins, _cases(pins), mod, first_only=True)
    assert failed, "the planted mistake %r passes every pin of test_oracle.py" % tag

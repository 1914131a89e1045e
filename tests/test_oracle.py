"""Pins for the FP64 CPU oracle (no GPU).

The oracle is the parity reference for the CUDA path, so it is itself pinned
to things other than its own formulas: hand-counted fixtures (tests/golden),
a third-party pair counter (scipy's cKDTree), independent formulas (pdist,
arccos/atan2 angles, an explicit cosine), the analytic shell expectation for
uniform periodic boxes (Eq. 12-13), the pair-total invariant, DR/RD symmetry,
and the marginal relations between the (r,mu), (sigma,pi) and monopole
histograms (Eq. 2, Eq. 4).
"""
import functools
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import synthetic

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _unit(theta_deg, axis):
    t = math.radians(theta_deg)
    if axis == "x":
        return [math.sin(t), 0.0, math.cos(t)]
    if axis == "y":
        return [0.0, math.sin(t), math.cos(t)]
    return [0.0, 0.0, 1.0]


# ------------------------------------------------------------------ fixtures
@pytest.mark.parametrize("name", ["mono_line.json", "mono_edges.json", "mono_periodic.json",
                                  "sigpi_square.json", "rmu_triplet.json"])
def test_golden_counts(name):
    g = _load(name)
    x = np.array(g["points"], dtype=np.float64)
    c, oor, _ = oracle.count(g["kind"], x, edges0=g["edges0"], edges1=g.get("edges1"),
                             periodic=g["periodic"], L=g["L"])
    assert c.ravel().tolist() == np.array(g["counts"]).ravel().tolist()
    assert oor == g["oor"]


def test_golden_theta():
    g = _load("theta_triangle.json")
    pts = []
    for p in g["points_deg"]:
        pts.append(_unit(0.0, "z") if p[0] == "z" else _unit(p[0], p[1]))
    x = np.array(pts)
    chord = oracle.theta_to_chord(g["theta_edges_deg"])
    c, oor, _ = oracle.count("theta", x, edges0=chord)
    assert c.ravel().tolist() == g["counts"]
    assert oor == g["oor"]


def test_golden_estimators():
    g = _load("ls_numbers.json")
    ls = oracle.xi_ls(g["DD"], g["DR"], g["RR"], g["Nd"], g["Nr"])
    nat = oracle.xi_natural(g["DD"], g["RR"], g["Nd"], g["Nr"])
    assert ls[0] == pytest.approx(g["xi_ls"], rel=1e-15)
    assert nat[0] == pytest.approx(g["xi_natural"], rel=1e-15)


def test_theta_to_chord_values():
    c = oracle.theta_to_chord([0.0, 60.0, 180.0, 90.0])
    assert c[0] == 0.0
    assert c[1] == pytest.approx(1.0, rel=1e-15)
    assert c[2] == pytest.approx(2.0, rel=1e-15)
    assert c[3] == pytest.approx(math.sqrt(2.0), rel=1e-15)


# ------------------------------------------------------------------ library pins
def test_mono_open_matches_pdist_histogram():
    scipy_sd = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 50, size=(600, 3))
    edges = np.linspace(0, 30, 16)
    c, oor, _ = oracle.count("mono", x, edges0=edges)
    d = scipy_sd.pdist(x)
    h, _ = np.histogram(d, bins=edges)
    assert c.ravel().tolist() == h.tolist()
    assert oor == len(d) - h.sum()


def test_mono_periodic_matches_ckdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(12)
    L = 100.0
    x = rng.uniform(0, L, size=(800, 3))
    y = rng.uniform(0, L, size=(500, 3))
    edges = np.linspace(0, 30, 11)
    ta, tb = spatial.cKDTree(x, boxsize=L), spatial.cKDTree(y, boxsize=L)
    # cross: ordered pairs with edges[k-1] < d <= edges[k]
    ref = ta.count_neighbors(tb, edges, cumulative=False)[1:]
    c, oor, _ = oracle.count("mono", x, y, edges0=edges, periodic=True, L=L)
    assert c.ravel().tolist() == ref.tolist()
    # auto: cKDTree counts ordered pairs including i == j at d = 0
    ref_auto = ta.count_neighbors(ta, edges, cumulative=False)
    ref_auto[0] -= len(x)
    ca, _, _ = oracle.count("mono", x, edges0=edges, periodic=True, L=L)
    assert (2 * ca.ravel()).tolist() == ref_auto[1:].tolist()


def test_theta_matches_atan2_angles():
    rng = np.random.default_rng(13)
    v = rng.normal(size=(400, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v = v[v[:, 2] > 0.5]
    theta_edges = np.linspace(0.0, 40.0, 21)
    chord = oracle.theta_to_chord(theta_edges)
    c, _, _ = oracle.count("theta", v, edges0=chord)
    i, j = np.triu_indices(len(v), 1)
    cr = np.linalg.norm(np.cross(v[i], v[j]), axis=1)
    dt = np.einsum("ij,ij->i", v[i], v[j])
    ang = np.degrees(np.arctan2(cr, dt))
    h, _ = np.histogram(ang, bins=theta_edges)
    assert c.ravel().tolist() == h.tolist()


def test_rmu_matches_explicit_cosine():
    rng = np.random.default_rng(14)
    x = rng.uniform(-30, 30, size=(500, 3)) + np.array([0.0, 0.0, 300.0])
    e0 = np.linspace(0, 40, 9)
    e1 = np.linspace(0, 1, 11)
    c, _, _ = oracle.count("rmu", x, edges0=e0, edges1=e1)
    i, j = np.triu_indices(len(x), 1)
    s = x[j] - x[i]
    l = x[i] + x[j]
    r = np.linalg.norm(s, axis=1)
    mu = np.abs(np.einsum("ij,ij->i", s, l)) / (r * np.linalg.norm(l, axis=1))
    ok = r < 40
    h, _, _ = np.histogram2d(r[ok], np.minimum(mu[ok], 1.0 - 1e-15), bins=[e0, e1])
    assert c.tolist() == h.astype(np.int64).tolist()


@functools.lru_cache(maxsize=1)
def _mu_edge_pairs():
    """Integer point pairs (x_i, x_j), both with z >= 1, whose separation
    s = x_j - x_i makes exactly 60 degrees with the line of sight
    l = x_i + x_j: 4 (s.l)^2 = |s|^2 |l|^2, i.e. mu = 1/2 exactly."""
    g = np.array([v for v in itertools.product(range(-4, 5), repeat=3) if any(v)], dtype=np.int64)
    sv, lv = np.repeat(g, len(g), axis=0), np.tile(g, (len(g), 1))
    sl = (sv * lv).sum(1)
    ok = ((lv - sv) % 2 == 0).all(1) & (sl != 0) & (4 * sl * sl == (sv * sv).sum(1) * (lv * lv).sum(1))
    xi, xj = (lv[ok] - sv[ok]) // 2, (lv[ok] + sv[ok]) // 2
    up = (xi[:, 2] >= 1) & (xj[:, 2] >= 1)
    return xi[up], xj[up]


def _exact_counts(kind, a, b, e0, e1, L):
    """Brute-force histogram of integer points in exact integer arithmetic
    (Eq. 11 with half-open bins on squared integer edges; (sigma, pi) along
    z, Eq. 2; (r, mu) about the pair midpoint with mu edges k/4, compared as
    16 (s.l)^2 >= k^2 |s|^2 |l|^2).  b None: unique pairs of a.  Also
    returns how many pairs sit exactly on an edge."""
    if b is None:
        i, j = np.triu_indices(len(a), 1)
        A, B = a[i], a[j]
    else:
        i, j = np.indices((len(a), len(b))).reshape(2, -1)
        A, B = a[i], b[j]
    E0 = np.asarray(e0, dtype=np.int64) ** 2

    def bins(v, E):
        return np.where((v >= E[0]) & (v < E[-1]), np.searchsorted(E, v, side="right") - 1, -1)

    ties = 0
    if kind == "rmu":
        s, l = B - A, A + B
        r2, l2, sl = (s * s).sum(1), (l * l).sum(1), (s * l).sum(1)
        b0 = bins(r2, E0)
        k4 = np.rint(np.asarray(e1) * 4).astype(np.int64)
        assert np.array_equal(k4, np.asarray(e1) * 4)
        q16, den = 16 * sl * sl, r2 * l2
        b1 = np.zeros(len(r2), dtype=np.int64)
        for k in range(1, len(k4) - 1):
            b1 = np.where(q16 >= k4[k] ** 2 * den, k, b1)
            ties += int(np.sum((q16 == k4[k] ** 2 * den) & (b0 >= 0) & (r2 > 0)))
        b1 = np.where(r2 == 0, 0, b1)  # coincident points: no direction, mu bin 0
        n1 = len(k4) - 1
    else:
        d = B - A
        if L:
            d = np.where(2 * d > L, d - L, np.where(2 * d < -L, d + L, d))
        if kind == "mono":
            b0, b1, n1 = bins((d * d).sum(1), E0), np.zeros(len(d), dtype=np.int64), 1
        else:
            E1 = np.asarray(e1, dtype=np.int64) ** 2
            b0, b1, n1 = bins((d[:, :2] ** 2).sum(1), E0), bins(d[:, 2] ** 2, E1), len(E1) - 1
            ties += int(np.isin(d[:, 2] ** 2, E1[1:]).sum())
        ties += int(np.isin((d * d).sum(1) if kind == "mono" else (d[:, :2] ** 2).sum(1),
                            E0[1:]).sum())
    ok = (b0 >= 0) & (b1 >= 0)
    h = np.bincount(b0[ok] * n1 + b1[ok], minlength=(len(E0) - 1) * n1)
    return h.reshape(len(E0) - 1, n1), int((~ok).sum()), ties


@pytest.mark.parametrize("kind,periodic", [("mono", False), ("mono", True), ("sigpi", False),
                                           ("sigpi", True), ("rmu", False)])
def test_integer_lattice_matches_exact_arithmetic(kind, periodic):
    """Integer coordinates and edges make every FP64 quantity of the
    canonical formulas exact, so the oracle must equal a brute force in
    exact integer arithmetic, including the many pairs that sit exactly on
    an edge (half-open bins); (sigma, pi) and (r, mu) have unequal bin
    counts on the two axes, and (r, mu) includes pairs exactly on the
    mu = 1/2 edge."""
    rng = np.random.default_rng(22)
    L = 24
    e0 = [0, 1, 2, 3, 5, 8, 13]
    e1 = {"sigpi": [0, 1, 3, 5, 7], "rmu": [0.0, 0.25, 0.5, 0.75, 1.0]}.get(kind)
    if kind == "rmu":
        pi_, pj = _mu_edge_pairs()
        assert len(pi_) > 50
        r = np.concatenate([rng.integers(-8, 9, size=(150, 2)), rng.integers(1, 9, size=(150, 1))], 1)
        a, b = np.concatenate([pi_, r[:75]]), np.concatenate([pj, r[75:]])
    else:
        lo, hi = (0, L) if periodic else (-10, 11)
        a, b = rng.integers(lo, hi, size=(160, 3)), rng.integers(lo, hi, size=(140, 3))
    a, b = a.astype(np.int64), b.astype(np.int64)
    for xa, xb in ((np.concatenate([a, b]), None), (a, b)):
        ref, oor, ties = _exact_counts(kind, xa, xb, e0, e1, L if periodic else 0)
        assert ties >= 50
        c, o, _ = oracle.count(kind, xa.astype(np.float64),
                               None if xb is None else xb.astype(np.float64), edges0=e0,
                               edges1=e1, periodic=periodic, L=float(L))
        assert c.tolist() == ref.tolist()
        assert o == oor


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("kind,periodic", [("mono", True), ("mono", False), ("sigpi", True),
                                           ("rmu", False), ("theta", False)])
def test_pair_total_invariant(kind, periodic):
    rng = np.random.default_rng(15)
    L = 100.0
    if kind == "theta":
        a = rng.normal(size=(300, 3)); a /= np.linalg.norm(a, axis=1, keepdims=True)
        b = rng.normal(size=(200, 3)); b /= np.linalg.norm(b, axis=1, keepdims=True)
        e0, e1 = np.linspace(0, 0.5, 6), None
    else:
        a = rng.uniform(0, L, size=(300, 3))
        b = rng.uniform(0, L, size=(200, 3))
        if kind == "rmu":
            a += 500; b += 500
        e0 = np.linspace(0, 30, 7)
        e1 = np.linspace(0, 1, 5) if kind == "rmu" else (np.linspace(0, 20, 5) if kind == "sigpi" else None)
    ca, oa, _ = oracle.count(kind, a, edges0=e0, edges1=e1, periodic=periodic, L=L)
    assert int(ca.sum()) + oa == len(a) * (len(a) - 1) // 2
    cx, ox, _ = oracle.count(kind, a, b, edges0=e0, edges1=e1, periodic=periodic, L=L)
    assert int(cx.sum()) + ox == len(a) * len(b)
    # DR == RD bit-exactly (the canonical separation is symmetric)
    cy, oy, _ = oracle.count(kind, b, a, edges0=e0, edges1=e1, periodic=periodic, L=L)
    assert cx.tolist() == cy.tolist() and ox == oy


def test_uniform_box_matches_shell_expectation():
    """Eq. 12-13: for uniform points in a periodic box the expected count in a
    shell is N(N-1)/2 * 4pi/3 (r2^3 - r1^3) / L^3."""
    rng = np.random.default_rng(16)
    L, N = 100.0, 4000
    x = synthetic.uniform_box(N, L, rng)
    e = np.linspace(0, 20, 11)
    c, _, _ = oracle.count("mono", x, edges0=e, periodic=True, L=L)
    expect = 0.5 * N * (N - 1) * (4 * math.pi / 3) * (e[1:] ** 3 - e[:-1] ** 3) / L ** 3
    z = (c.ravel() - expect) / np.sqrt(expect)
    assert np.all(np.abs(z) < 5), z
    xi = oracle.xi_periodic(c.ravel(), N, e, L)
    assert np.all(np.abs(xi) < 5 / np.sqrt(expect))


def test_rmu_marginal_equals_monopole():
    """Eq. 4: integrating over mu recovers the monopole.  For counts: summing
    the (r, mu) histogram over all mu bins equals the r histogram exactly."""
    w = synthetic.c2_rmu_lightcone(scale=0.0006)
    c2, o2, _ = oracle.count("rmu", w.data, w.randoms, edges0=w.edges0, edges1=w.edges1)
    c1, o1, _ = oracle.count("mono", w.data, w.randoms, edges0=w.edges0)
    assert c2.sum(axis=1).tolist() == c1.ravel().tolist()
    assert o1 == o2


def test_sigpi_marginals_are_projected_monopoles():
    """Eq. 2: sigma is the separation projected off the line of sight and pi
    the part along it; a (sigma, pi) histogram with one pi bin covering every
    separation is the monopole of the points projected on the sky plane."""
    rng = np.random.default_rng(17)
    L = 60.0
    x = rng.uniform(0, L, size=(700, 3))
    es = np.linspace(0, 20, 9)
    big = np.array([0.0, L])  # pi in [0, L): every pair (|dz| <= L/2)
    c, _, _ = oracle.count("sigpi", x, edges0=es, edges1=big, periodic=True, L=L)
    proj = x.copy(); proj[:, 2] = 0.0
    m, _, _ = oracle.count("mono", proj, edges0=es, periodic=True, L=L)
    assert c[:, 0].tolist() == m.ravel().tolist()
    c2, _, _ = oracle.count("sigpi", x, edges0=np.array([0.0, L]), edges1=es, periodic=True, L=L)
    projz = x.copy(); projz[:, :2] = 0.0
    m2, _, _ = oracle.count("mono", projz, edges0=es, periodic=True, L=L)
    assert c2[0, :].tolist() == m2.ravel().tolist()


@pytest.mark.parametrize("kind,periodic", [("mono", True), ("mono", False), ("sigpi", True),
                                           ("rmu", False), ("theta", False)])
def test_cells_equal_brute_force(kind, periodic):
    rng = np.random.default_rng(18)
    L = 200.0
    if kind == "theta":
        a = synthetic._cap_uniform(900, 0.9, rng)
        b = synthetic._cap_uniform(700, 0.9, rng)
        e0, e1 = oracle.theta_to_chord(np.linspace(0, 8, 9)), None
        reach = [e0[-1]] * 3
    else:
        a = synthetic.uniform_box(900, L, rng)
        b = synthetic.uniform_box(700, L, rng)
        a = np.concatenate([a, synthetic.blobs_box(5, 40, L, 2.0, rng)])
        if kind == "rmu":
            a = a + 1000; b = b + 1000
        e0 = np.linspace(0, 40, 9)
        e1 = {"rmu": np.linspace(0, 1, 6), "sigpi": np.linspace(0, 30, 7)}.get(kind)
        reach = [40, 40, 30] if kind == "sigpi" else [40, 40, 40]
    for xb in (None, b):
        ref = oracle.count(kind, a, xb, edges0=e0, edges1=e1, periodic=periodic, L=L)
        got = oracle.count(kind, a, xb, edges0=e0, edges1=e1, periodic=periodic, L=L, cells=reach)
        assert got[0].tolist() == ref[0].tolist()
        assert got[1] == ref[1]


# ------------------------------------------------------------------ weighted + gradient
def test_weighted_unit_weights_equal_counts_and_pdist():
    sd = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(19)
    x = rng.uniform(0, 40, size=(400, 3))
    e = np.linspace(0, 20, 6)
    ones = np.ones(len(x), np.float32)
    c, _, w1 = oracle.count("mono", x, edges0=e, wa=ones, weighted=True)
    assert w1.ravel().tolist() == c.ravel().astype(float).tolist()
    w = np.exp(0.3 * rng.normal(size=len(x))).astype(np.float32)
    _, _, ws = oracle.count("mono", x, edges0=e, wa=w, weighted=True)
    d = sd.pdist(x)
    prod = sd.pdist(w.astype(np.float64)[:, None], lambda u, v: u[0] * v[0])
    ref, _ = np.histogram(d, bins=e, weights=prod)
    np.testing.assert_allclose(ws.ravel(), ref, rtol=1e-13)


@pytest.mark.parametrize("cross", [False, True])
def test_grad_rows_match_finite_differences(cross):
    """F(w) = sum_b G_b W_b is linear in each w_i (no self pairs), so the
    central difference with h = w_i is exact up to rounding."""
    rng = np.random.default_rng(20)
    L = 50.0
    a = synthetic.uniform_box(250, L, rng)
    b = synthetic.uniform_box(180, L, rng) if cross else None
    e = np.linspace(0, 15, 6)
    wa = np.exp(0.3 * rng.normal(size=len(a))).astype(np.float32)
    wb = np.exp(0.3 * rng.normal(size=180)).astype(np.float32) if cross else None
    G = rng.normal(size=5)

    def F(wa_):
        _, _, ws = oracle.count("mono", a, b, edges0=e, periodic=True, L=L, wa=wa_,
                                wb=wb, weighted=True)
        return float(np.dot(G, ws.ravel()))

    rows = np.array([0, 7, 100, 249])
    g = oracle.grad_rows("mono", a, rows, G, wb if cross else wa, xb=b, edges0=e,
                         periodic=True, L=L)
    for r, gr in zip(rows, g):
        h = float(wa[r])
        wp = wa.copy(); wp[r] = np.float32(wa[r] * 2)
        wm = wa.copy(); wm[r] = np.float32(0.0)
        fd = (F(wp) - F(wm)) / (2 * h)
        assert gr == pytest.approx(fd, rel=1e-9, abs=1e-12)
    if not cross:
        # Euler's theorem: F is homogeneous of degree 2 in w
        allg = oracle.grad_rows("mono", a, np.arange(len(a)), G, wa, edges0=e, periodic=True, L=L)
        assert float(np.dot(wa.astype(np.float64), allg)) == pytest.approx(2 * F(wa), rel=1e-10)


def test_ls_equals_normalised_form():
    """Eq. 15 with unique-pair counts equals (DDn - 2 DRn + RRn)/RRn where the
    counts are normalised by Nd(Nd-1)/2, Nd Nr and Nr(Nr-1)/2."""
    rng = np.random.default_rng(21)
    Nd, Nr = 1234, 5678
    DD = rng.integers(1, 10**6, size=20).astype(np.uint64)
    DR = rng.integers(1, 10**7, size=20).astype(np.uint64)
    RR = rng.integers(1, 10**7, size=20).astype(np.uint64)
    xi = oracle.xi_ls(DD, DR, RR, Nd, Nr)
    ddn = DD / (Nd * (Nd - 1) / 2)
    drn = DR / (Nd * Nr)
    rrn = RR / (Nr * (Nr - 1) / 2)
    np.testing.assert_allclose(xi, (ddn - 2 * drn + rrn) / rrn, rtol=1e-12)
    z = oracle.xi_ls(DD, DR, np.zeros(20, np.uint64), Nd, Nr)
    assert np.all(np.isnan(z))


# ---------------------------------------------------------------- multipoles
def test_multipoles_of_piecewise_constant_xi_by_quadrature():
    """The binned xi(r, mu) is constant on each mu bin; its multipoles
    (2l + 1) * integral_0^1 xi P_l dmu (Eq. 3 by orthogonality), with P_l
    integrated over each bin by 8-point Gauss quadrature (exact to degree
    15) of scipy's P_l, equal the oracle's."""
    from scipy.special import eval_legendre
    gx, gw = np.polynomial.legendre.leggauss(8)
    rng = np.random.default_rng(80)
    m = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0, 1, 14)]))
    xi = rng.normal(size=(3, 15))
    ells = (0, 2, 4, 6)
    ref = np.zeros((len(ells), 3))
    for q, l in enumerate(ells):
        half, mid = 0.5 * np.diff(m), 0.5 * (m[1:] + m[:-1])
        w = np.array([half[k] * np.dot(gw, eval_legendre(l, mid[k] + half[k] * gx))
                      for k in range(15)])
        ref[q] = (2 * l + 1) * xi @ w
    np.testing.assert_allclose(oracle.multipoles(xi, m, ells), ref, rtol=1e-11, atol=1e-13)


def test_multipoles_recover_legendre_coefficients_on_fine_bins():
    """Eq. 3: xi(r, mu) = sum a_l P_l(mu) (l = 0, 2, 4, 6) sampled at 2000
    mu-bin midpoints gives back the a_l up to the O(dmu^2) binning error."""
    from scipy.special import eval_legendre
    rng = np.random.default_rng(81)
    m = np.linspace(0, 1, 2001)
    mid = 0.5 * (m[1:] + m[:-1])
    a = rng.normal(size=(3, 4))
    xi = np.stack([sum(c[q] * eval_legendre(2 * q, mid) for q in range(4)) for c in a])
    np.testing.assert_allclose(oracle.multipoles(xi, m, (0, 2, 4, 6)).T, a, atol=5e-5)


def test_multipoles_of_constant_and_monopole_average():
    """A mu-independent xi has xi_0 = xi and no l > 0 part; xi_0 of any xi is
    its bin-width-weighted mean over [0, 1] (Eq. 4 for xi even in mu)."""
    m = np.array([0.0, 0.1, 0.35, 0.5, 0.9, 1.0])
    got = oracle.multipoles(np.full((2, 5), 0.7), m, (0, 2, 4))
    np.testing.assert_allclose(got, [[0.7, 0.7], [0, 0], [0, 0]], atol=1e-15)
    xi = np.random.default_rng(82).normal(size=(4, 5))
    np.testing.assert_allclose(oracle.multipoles(xi, m, (0,))[0], xi @ np.diff(m), rtol=1e-14)


# ---------------------------------------------------------------- sky coordinates
def test_comoving_distance_closed_forms():
    """chi(z) (Sec. 2.1) in three cosmologies with closed forms:
    Einstein-de Sitter 2 (c/H0)(1 - 1/sqrt(1+z)), the empty universe
    (c/H0) ln(1+z), de Sitter (c/H0) z."""
    z = np.array([0.0, 0.1, 0.5, 1.0, 2.5, 7.0])
    ch = oracle.C_OVER_H0
    np.testing.assert_allclose(oracle.comoving_distance(z, 1.0, 0.0),
                               2 * ch * (1 - 1 / np.sqrt(1 + z)), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(oracle.comoving_distance(z, 0.0, 0.0), ch * np.log1p(z),
                               rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(oracle.comoving_distance(z, 0.0, 1.0), ch * z, rtol=1e-12,
                               atol=1e-9)


def test_sky_unit_vectors():
    """RA/Dec axes land on the coordinate axes, and every n has unit norm."""
    n = oracle.sky_to_xyz([0.0, 90.0, 0.0, 180.0, 33.0], [0.0, 0.0, 90.0, -30.0, 61.0])
    np.testing.assert_allclose(n[:3], np.eye(3), atol=1e-15)
    np.testing.assert_allclose(n[3], [-np.cos(np.radians(30)), 0.0, -0.5], atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, rtol=1e-15)


# ---------------------------------------------------------------- pixel maps
def test_healpix_base_pixels():
    """nside = 1: the 12 base pixels, 4 at z = 2/3 and 4 at z = -2/3 centred
    on phi = pi/4 + k pi/2, 4 on the equator centred on phi = k pi/2."""
    c = oracle.healpix_pix2vec_ring(1, np.arange(12))
    z = np.repeat([2 / 3, 0.0, -2 / 3], 4)
    phi = np.concatenate([np.pi / 4 + np.arange(4) * np.pi / 2, np.arange(4) * np.pi / 2,
                          np.pi / 4 + np.arange(4) * np.pi / 2])
    st = np.sqrt(1 - z * z)
    ref = np.stack([st * np.cos(phi), st * np.sin(phi), z], axis=1)
    np.testing.assert_allclose(c, ref, atol=1e-15)
    np.testing.assert_array_equal(oracle.healpix_ang2pix_ring(1, ref), np.arange(12))


@pytest.mark.parametrize("nside", [1, 2, 4, 16, 64])
def test_healpix_round_trip_and_rings(nside):
    """Every pixel's centre lies in that pixel; the centres sit on 4 nside - 1
    rings with 4i pixels on the i-th ring from either pole (i < nside) and
    4 nside on the belt rings."""
    p = np.arange(12 * nside * nside)
    c = oracle.healpix_pix2vec_ring(nside, p)
    np.testing.assert_allclose(np.linalg.norm(c, axis=1), 1.0, rtol=1e-14)
    np.testing.assert_array_equal(oracle.healpix_ang2pix_ring(nside, c), p)
    zs, counts = np.unique(np.round(c[:, 2], 12), return_counts=True)
    assert len(zs) == 4 * nside - 1
    expect = [4 * min(i, 4 * nside - i, nside) for i in range(1, 4 * nside)]
    assert sorted(counts.tolist()) == sorted(expect)


def test_healpix_equal_area_and_locality():
    """Pixels have equal area: 2M uniform points on the sphere fill the 192
    pixels of nside = 4 evenly (chi^2 within 5 sigma); every point lies
    within 1.5 pixel radii of its pixel's centre."""
    rng = np.random.default_rng(83)
    v = rng.normal(size=(2_000_000, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    p = oracle.healpix_ang2pix_ring(4, v)
    cnt = np.bincount(p, minlength=192)
    mean = len(v) / 192
    chi2 = float(((cnt - mean) ** 2 / mean).sum())
    assert abs(chi2 - 191) < 5 * np.sqrt(2 * 191)
    c = oracle.healpix_pix2vec_ring(4, p[:20000])
    ang = np.arccos(np.clip(np.sum(c * v[:20000], axis=1), -1, 1))
    assert ang.max() < 1.5 * np.sqrt(4 * np.pi / 192)


@pytest.mark.parametrize("nside", [1, 3, 8, 64])
def test_healpix_points_inside_their_pixel(nside):
    """Random points against the pixel geometry stated on the sphere (Gorski
    et al. 2005): in the belt |z| <= 2/3 every pixel is a diamond in (phi, z)
    with vertices pi/(4 nside) either side of its centre in phi and
    2/(3 nside) above and below it in z, so each point must satisfy
    |dphi| / (pi/(4 nside)) + |dz| / (2/(3 nside)) <= 1 about its pixel's
    centre; everywhere, a pixel's north and south vertices lie on the
    neighbouring rings, so the point's z lies between the latitudes of the
    rings above and below its pixel's ring."""
    rng = np.random.default_rng(85)
    v = rng.normal(size=(400_000, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    p = oracle.healpix_ang2pix_ring(nside, v)
    c = oracle.healpix_pix2vec_ring(nside, p)
    belt = np.abs(v[:, 2]) <= 2.0 / 3.0
    dphi = np.angle(np.exp(1j * (np.arctan2(v[:, 1], v[:, 0]) - np.arctan2(c[:, 1], c[:, 0]))))
    dz = v[:, 2] - c[:, 2]
    lhs = np.abs(dphi) / (np.pi / (4 * nside)) + np.abs(dz) / (2.0 / (3 * nside))
    assert np.all(lhs[belt] <= 1.0 + 1e-9)
    # ring latitudes z_i, i = 0 .. 4 nside (the poles at i = 0 and 4 nside)
    i = np.arange(4 * nside + 1)
    zr = np.where(i < nside, 1.0 - i * i / (3.0 * nside * nside),
                  np.where(i > 3 * nside, -1.0 + (4 * nside - i) ** 2 / (3.0 * nside * nside),
                           (2 * nside - i) * 2.0 / (3.0 * nside)))
    ring = np.argmin(np.abs(zr[None, :] - c[:, 2:3]), axis=1)  # the centre's ring
    assert np.all(zr[ring] == pytest.approx(c[:, 2], abs=1e-12))
    assert np.all(v[:, 2] <= zr[ring - 1] + 1e-12) and np.all(v[:, 2] >= zr[ring + 1] - 1e-12)


def test_weighted_estimators_reduce_to_unweighted():
    """Unit weights turn the weighted estimators into Eq. 14 / Eq. 15 on
    unique-pair counts."""
    rng = np.random.default_rng(84)
    DD, DR, RR = (rng.integers(1, 10**6, 20).astype(np.uint64) for _ in range(3))
    nd, nr = 5000, 20000
    nat = oracle.xi_weighted("natural", DD, None, RR, nd, nd, nr, nr)
    ls = oracle.xi_weighted("ls", DD, DR, RR, nd, nd, nr, nr)
    np.testing.assert_allclose(nat, oracle.xi_natural(DD, RR, nd, nr), rtol=1e-13)
    np.testing.assert_allclose(ls, oracle.xi_ls(DD, DR, RR, nd, nr), rtol=1e-12)


# ---------------------------------------------------------------- density grid
def test_tsc_weights():
    """TSC (Sec. 3.4.4): mass is conserved; a particle on a grid point gives
    1/8, 3/4, 1/8 along each axis; one midway between two points gives 1/2,
    1/2; a full lattice of particles on the grid points gives a flat field."""
    L, n = 16.0, 16
    rng = np.random.default_rng(86)
    x = rng.uniform(0, L, (500, 3))
    w = rng.uniform(0.5, 2, 500)
    assert oracle.tsc_density(x, L, n, w).sum() == pytest.approx(w.sum(), rel=1e-13)
    rho = oracle.tsc_density(np.array([[3.0, 5.0, 7.0]]), L, n)
    line = rho[7, 5, 2:5]
    np.testing.assert_allclose(line, np.array([1 / 8, 3 / 4, 1 / 8]) * 9 / 16, rtol=1e-15)
    rho = oracle.tsc_density(np.array([[3.5, 5.0, 7.0]]), L, n)
    np.testing.assert_allclose(rho[7, 5, 3:5], np.array([0.5, 0.5]) * 9 / 16, rtol=1e-15)
    g = np.stack(np.meshgrid(*[np.arange(n) * 1.0] * 3, indexing="ij"), -1).reshape(-1, 3)
    np.testing.assert_allclose(oracle.tsc_density(g, L, n), 1.0, rtol=1e-14)


def test_lag_xi_of_a_plane_wave():
    """delta = A cos(2 pi k.x / n) on a full-period grid has
    <delta(x) delta(x + d)> = A^2/2 cos(2 pi k.d / n) exactly, so each bin
    holds the mean of that over its lags."""
    n, L, A = 16, 32.0, 0.7
    k = np.array([1, 2, 3])
    idx = np.indices((n, n, n))  # (z, y, x)
    phase = 2 * np.pi * (k[0] * idx[2] + k[1] * idx[1] + k[2] * idx[0]) / n
    delta = A * np.cos(phase)
    edges = np.array([0.0, 3.0, 6.0, 9.5])
    xi, lags = oracle.lag_xi(delta, L, edges)
    a = L / n
    R = int(np.floor(edges[-1] / a))
    ref_s, ref_c = np.zeros(3), np.zeros(3)
    for dz in range(0, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                if (dz == 0 and dy < 0) or (dz == 0 and dy == 0 and dx <= 0):
                    continue
                r = a * np.sqrt(dx * dx + dy * dy + dz * dz)
                b = np.searchsorted(edges, r, side="right") - 1
                if 0 <= b < 3:
                    ref_s[b] += 0.5 * A * A * np.cos(2 * np.pi * (k[0] * dx + k[1] * dy + k[2] * dz) / n)
                    ref_c[b] += 1
    np.testing.assert_allclose(lags, ref_c)
    np.testing.assert_allclose(xi, ref_s / ref_c, rtol=1e-12, atol=1e-14)


def test_lag_xi_fft_equals_the_direct_lag_sums():
    """The FFT form of the lag sums (correlation theorem) against the direct
    products of shifted grids, on a clustered field, on the plane wave's
    closed form, and with lags reaching past half the edge range."""
    rng = np.random.default_rng(31)
    n, L = 24, 48.0
    x = np.concatenate([rng.uniform(0, L, (3000, 3)), (rng.normal(L / 2, 3.0, (600, 3)) % L)])
    rho = oracle.tsc_density(x, L, n)
    delta = rho / rho.mean() - 1.0
    edges = np.array([0.0, 2.5, 5.0, 9.0, 14.0, 20.0])
    xi_d, c_d = oracle.lag_xi(delta, L, edges)
    xi_f, c_f = oracle.lag_xi_fft(delta, L, edges)
    np.testing.assert_array_equal(c_f, c_d)
    np.testing.assert_allclose(xi_f, xi_d, rtol=1e-11, atol=1e-13 * float(np.mean(delta ** 2)))
    # the plane wave: <delta(x) delta(x + d)> = A^2/2 cos(2 pi k.d / n)
    n, L, A = 16, 32.0, 0.7
    k = np.array([1, 2, 3])
    idx = np.indices((n, n, n))
    wave = A * np.cos(2 * np.pi * (k[0] * idx[2] + k[1] * idx[1] + k[2] * idx[0]) / n)
    edges = np.array([0.0, 3.0, 6.0, 9.5])
    xi_w, _ = oracle.lag_xi_fft(wave, L, edges)
    xi_ref, _ = oracle.lag_xi(wave, L, edges)
    np.testing.assert_allclose(xi_w, xi_ref, rtol=1e-12, atol=1e-14)

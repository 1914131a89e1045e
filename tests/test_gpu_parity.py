"""GPU parity: counts from the CUDA path (through the C ABI) equal the FP64
oracle's bit for bit, for every kind and boundary, on seeded catalogs that
span many tiles and work items with ragged tails, and on the degenerate and
adversarial cases (empty catalogs, single objects, coincident objects, pairs
exactly on bin edges, periodic pairs across the box faces)."""
import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import cute, synthetic
from gpu_util import edge_pairs_mono, edge_pairs_mu, gpu_count, oracle_count

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["arith", "table"])
def ctx(request):
    """Every parity test runs twice: arithmetic binning where the edges are
    uniform, and lookup-table binning forced for all edges."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cute.Context(0)
    if request.param == "table":
        c.set_launch(table_binning=True)
    yield c
    c.close()


def _assert_same(got, ref):
    gc, go, _ = got
    rc, ro, _ = ref
    assert gc.shape == rc.shape
    if not np.array_equal(gc, rc):
        diff = np.argwhere(gc != rc)
        raise AssertionError("counts differ at %d bins, first %s: gpu %s oracle %s" %
                             (len(diff), diff[:5].tolist(), gc[tuple(diff[0])], rc[tuple(diff[0])]))
    assert go == ro


# ------------------------------------------------------------------ workloads
def test_c1_monopole_box_full_size(ctx):
    """Full configuration of the small periodic-box workload (20,000 points,
    40 bins), brute-force oracle."""
    w = synthetic.c1_monopole_box()
    got = gpu_count(ctx, "mono", w.data, e0=w.edges0, periodic=True, L=w.L)
    ref = oracle_count("mono", w.data, e0=w.edges0, periodic=True, L=w.L)
    _assert_same(got, ref)
    xi_g = cute.estimator("periodic", got[0].ravel(), Nd=len(w.data), edges=w.edges0, L=w.L)
    xi_o = oracle.xi_periodic(ref[0].ravel(), len(w.data), w.edges0, w.L)
    np.testing.assert_allclose(xi_g, xi_o, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("cpr", [1, 2, 3])
@pytest.mark.parametrize("hp", [2, 4])
def test_mono_periodic_launch_shapes(ctx, cpr, hp):
    w = synthetic.c1_monopole_box(scale=0.3)
    table = ctx.table_binning if hasattr(ctx, "table_binning") else False
    ctx.set_launch(home_per_lane=hp, slice=128, table_binning=table)
    try:
        got = gpu_count(ctx, "mono", w.data, e0=w.edges0, periodic=True, L=w.L,
                        cells_per_reach=cpr)
    finally:
        ctx.set_launch(table_binning=table)
    ref = oracle_count("mono", w.data, e0=w.edges0, periodic=True, L=w.L)
    _assert_same(got, ref)


def test_twenty_warps_where_allowed(ctx):
    """The plain monopole kernel with two home objects per lane runs 20 warps
    per block; other kernels clamp a request for 20 to 16.  Counts exact."""
    table = ctx.table_binning if hasattr(ctx, "table_binning") else False
    ctx.set_launch(home_per_lane=2, warps_per_block=20, table_binning=table)
    try:
        w = synthetic.c1_monopole_box(scale=0.3)
        got = gpu_count(ctx, "mono", w.data, e0=w.edges0, periodic=True, L=w.L)
        assert ctx.stats()["warps_per_block"] == 20
        _assert_same(got, oracle_count("mono", w.data, e0=w.edges0, periodic=True, L=w.L))
        v = synthetic.c2_rmu_lightcone(scale=0.004)
        got = gpu_count(ctx, "rmu", v.data, v.randoms, v.edges0, v.edges1)
        assert ctx.stats()["warps_per_block"] == 16
        _assert_same(got, oracle_count("rmu", v.data, v.randoms, v.edges0, v.edges1, cells=True))
    finally:
        ctx.set_launch(table_binning=table)


def test_mono_open_cross_and_auto(ctx):
    rng = np.random.default_rng(100)
    a = np.concatenate([rng.uniform(0, 300, size=(4000, 3)),
                        synthetic.blobs_box(20, 60, 300.0, 3.0, rng)])
    b = rng.uniform(-20, 320, size=(5000, 3))
    e = np.linspace(0.0, 40.0, 17)
    _assert_same(gpu_count(ctx, "mono", a, b, e), oracle_count("mono", a, b, e))
    _assert_same(gpu_count(ctx, "mono", a, None, e), oracle_count("mono", a, None, e))
    # bins not starting at zero, log-spaced: the logarithmic table
    e2 = np.geomspace(0.5, 40.0, 25)
    _assert_same(gpu_count(ctx, "mono", a, b, e2), oracle_count("mono", a, b, e2))


def test_sigpi_periodic_and_open(ctx):
    boxes = synthetic.c4_batched_sigpi(n_boxes=1, scale=0.05)
    w = boxes[0]
    got = gpu_count(ctx, "sigpi", w.data, None, w.edges0, w.edges1, periodic=True, L=w.L)
    ref = oracle_count("sigpi", w.data, None, w.edges0, w.edges1, periodic=True, L=w.L,
                       cells=True)
    _assert_same(got, ref)
    got = gpu_count(ctx, "sigpi", w.data, w.randoms, w.edges0, w.edges1, periodic=True, L=w.L)
    ref = oracle_count("sigpi", w.data, w.randoms, w.edges0, w.edges1, periodic=True, L=w.L,
                       cells=True)
    _assert_same(got, ref)
    rng = np.random.default_rng(101)
    a = rng.uniform(0, 200, size=(3000, 3))
    es, ep = np.linspace(0, 30, 11), np.linspace(0, 20, 9)
    _assert_same(gpu_count(ctx, "sigpi", a, None, es, ep), oracle_count("sigpi", a, None, es, ep))


def test_rmu_lightcone_small(ctx):
    w = synthetic.c2_rmu_lightcone(scale=0.008)
    for a, b in ((w.data, None), (w.data, w.randoms), (w.randoms, None)):
        got = gpu_count(ctx, "rmu", a, b, w.edges0, w.edges1)
        ref = oracle_count("rmu", a, b, w.edges0, w.edges1, cells=True)
        _assert_same(got, ref)


def test_neighbour_cull(ctx):
    """The kernel drops neighbour rows beyond the reach of a home chunk's
    bounding box: fewer pairs evaluated than the stencil presented, never
    fewer than the pairs binned, and the counts still the oracle's.  The
    light-cone DR and RR at 2 and 4 home objects per lane, and the periodic
    monopole (image shifts move the home box)."""
    table = ctx.table_binning if hasattr(ctx, "table_binning") else False
    w = synthetic.c2_rmu_lightcone(scale=0.01)
    m = synthetic.c1_monopole_box(scale=0.5)
    try:
        for hp in (2, 4):
            ctx.set_launch(home_per_lane=hp, table_binning=table)
            for a, b in ((w.data, w.randoms), (w.randoms, None)):
                got = gpu_count(ctx, "rmu", a, b, w.edges0, w.edges1, cells_per_reach=4)
                st = ctx.stats()
                _assert_same(got, oracle_count("rmu", a, b, w.edges0, w.edges1, cells=True))
                binned = int(got[0].sum())
                assert binned <= st["candidate_pairs"] < 0.95 * st["stencil_pairs"]
            got = gpu_count(ctx, "mono", m.data, e0=m.edges0, periodic=True, L=m.L,
                            cells_per_reach=3)
            st = ctx.stats()
            _assert_same(got, oracle_count("mono", m.data, e0=m.edges0, periodic=True, L=m.L))
            assert int(got[0].sum()) <= st["candidate_pairs"] < st["stencil_pairs"]
    finally:
        ctx.set_launch(table_binning=table)


@pytest.mark.parametrize("cpr", [3, 4])
def test_trimmed_stencils_2d(ctx, cpr):
    """Neighbour rows trimmed to the reach ball (r, mu) or disk x slab
    (sigma, pi) at finer cells."""
    w = synthetic.c2_rmu_lightcone(scale=0.004)
    got = gpu_count(ctx, "rmu", w.data, w.randoms, w.edges0, w.edges1, cells_per_reach=cpr)
    _assert_same(got, oracle_count("rmu", w.data, w.randoms, w.edges0, w.edges1, cells=True))
    b = synthetic.c4_batched_sigpi(n_boxes=1, scale=0.03)[0]
    got = gpu_count(ctx, "sigpi", b.data, None, b.edges0, b.edges1[:31], periodic=True, L=b.L,
                    cells_per_reach=cpr)
    _assert_same(got, oracle_count("sigpi", b.data, None, b.edges0, b.edges1[:31], periodic=True,
                                   L=b.L, cells=True))


@pytest.mark.parametrize("cpr", [5, 6, 7, 8])
@pytest.mark.parametrize("hp", [2, 4])
def test_fine_cells_all_kinds(ctx, cpr, hp):
    """5 to 8 cells per reach (warm-up tuning may pick 5 for the light cone;
    cute_grid_build accepts up to 8): (r, mu) DD, DR and RR, periodic
    (sigma, pi) auto and cross, theta auto and cross and the periodic
    monopole, at 2 and 4 home objects per lane with a narrow neighbour
    slice (many items per entry), against the oracle bit for bit."""
    table = ctx.table_binning if hasattr(ctx, "table_binning") else False
    ctx.set_launch(home_per_lane=hp, slice=256, table_binning=table)
    try:
        w = synthetic.c2_rmu_lightcone(scale=0.004)
        for a, b in ((w.data, None), (w.data, w.randoms), (w.randoms, None)):
            got = gpu_count(ctx, "rmu", a, b, w.edges0, w.edges1, cells_per_reach=cpr)
            _assert_same(got, oracle_count("rmu", a, b, w.edges0, w.edges1, cells=True))
        bx = synthetic.c4_batched_sigpi(n_boxes=1, scale=0.03)[0]
        for b in (None, bx.randoms):
            got = gpu_count(ctx, "sigpi", bx.data, b, bx.edges0, bx.edges1, periodic=True, L=bx.L,
                            cells_per_reach=cpr)
            _assert_same(got, oracle_count("sigpi", bx.data, b, bx.edges0, bx.edges1,
                                           periodic=True, L=bx.L, cells=True))
        a = synthetic.c3_angular(scale=0.0005)
        chord = oracle.theta_to_chord(a.extra["theta_deg"])
        for b in (None, a.randoms):
            got = gpu_count(ctx, "theta", a.data, b, chord, cells_per_reach=cpr)
            _assert_same(got, oracle_count("theta", a.data, b, chord, cells=True))
        m = synthetic.c1_monopole_box(scale=0.2)
        got = gpu_count(ctx, "mono", m.data, e0=m.edges0, periodic=True, L=m.L,
                        cells_per_reach=cpr)
        _assert_same(got, oracle_count("mono", m.data, e0=m.edges0, periodic=True, L=m.L))
    finally:
        ctx.set_launch(table_binning=table)


@pytest.mark.parametrize("hp", [2, 4])
def test_home_per_lane_all_kinds(ctx, hp):
    """Each home-objects-per-lane width is its own kernel instantiation:
    (r, mu), (sigma, pi) and theta counts at 2 and 4 home objects per
    lane, with chunk tails that leave padded home slots."""
    table = ctx.table_binning if hasattr(ctx, "table_binning") else False
    ctx.set_launch(home_per_lane=hp, table_binning=table)
    try:
        w = synthetic.c2_rmu_lightcone(scale=0.004)
        got = gpu_count(ctx, "rmu", w.data, w.randoms, w.edges0, w.edges1)
        _assert_same(got, oracle_count("rmu", w.data, w.randoms, w.edges0, w.edges1, cells=True))
        b = synthetic.c4_batched_sigpi(n_boxes=1, scale=0.03)[0]
        got = gpu_count(ctx, "sigpi", b.data, None, b.edges0, b.edges1, periodic=True, L=b.L)
        _assert_same(got, oracle_count("sigpi", b.data, None, b.edges0, b.edges1, periodic=True,
                                       L=b.L, cells=True))
        a = synthetic.c3_angular(scale=0.0005)
        chord = oracle.theta_to_chord(a.extra["theta_deg"])
        got = gpu_count(ctx, "theta", a.data, a.randoms, chord)
        _assert_same(got, oracle_count("theta", a.data, a.randoms, chord, cells=True))
    finally:
        ctx.set_launch(table_binning=table)


def test_theta_small(ctx):
    w = synthetic.c3_angular(scale=0.0008)
    chord = oracle.theta_to_chord(w.extra["theta_deg"])
    for a, b in ((w.data, None), (w.data, w.randoms)):
        got = gpu_count(ctx, "theta", a, b, chord)
        ref = oracle_count("theta", a, b, chord, cells=True)
        _assert_same(got, ref)


# ------------------------------------------------------------------ edge cases
def test_pairs_on_edges_mono(ctx):
    rng = np.random.default_rng(102)
    e = np.arange(21) * 2.5
    x = edge_pairs_mono(rng, e, 6)
    _assert_same(gpu_count(ctx, "mono", x, None, e), oracle_count("mono", x, None, e))
    ep = e[:17]  # periodic reach must stay below 0.47 L
    xb = edge_pairs_mono(rng, ep, 6, box=100.0)
    _assert_same(gpu_count(ctx, "mono", xb, None, ep, periodic=True, L=100.0),
                 oracle_count("mono", xb, None, ep, periodic=True, L=100.0))
    st = ctx.stats()
    assert st["rechecked_pairs"] > 0
    # pairs exactly on edges need the FP64 formula; with uniform edges the
    # double-float stage decides the rest
    assert st["fp64_pairs"] > 0
    if not getattr(ctx, "table_binning", False):
        assert st["fp64_pairs"] < st["rechecked_pairs"]


def test_pairs_on_edges_sigpi(ctx):
    """(sigma, pi) pairs on (and a hair off) every sigma edge and every pi
    edge, open and periodic."""
    rng = np.random.default_rng(106)
    es, ep = np.arange(16) * 2.0, np.arange(11) * 2.5
    eps = (0.0, 2.0**-40, -2.0**-40, 2.0**-36, -2.0**-36, 2.0**-33, -2.0**-33, 2.0**-24,
           -2.0**-24)
    pts = []
    for axis, edges in ((0, es), (1, ep)):
        for e in edges[1:]:
            for d in eps:
                c = rng.uniform(20.0, 80.0, size=3)
                phi = rng.uniform(0, 2 * np.pi)
                if axis == 0:
                    sig, pi = e * (1 + d), rng.uniform(0, ep[-1])
                else:
                    sig, pi = rng.uniform(0, es[-1]), e * (1 + d)
                off = np.array([sig * np.cos(phi), sig * np.sin(phi), pi * rng.choice([-1, 1])])
                pts += [c, c + off]
    x = np.array(pts)
    _assert_same(gpu_count(ctx, "sigpi", x, None, es, ep), oracle_count("sigpi", x, None, es, ep))
    xb = np.mod(x + 55.0, 100.0)  # the same pairs, many across the box faces
    xb[xb >= 100.0] = 0.0
    _assert_same(gpu_count(ctx, "sigpi", xb, None, es, ep, periodic=True, L=100.0),
                 oracle_count("sigpi", xb, None, es, ep, periodic=True, L=100.0))
    assert ctx.stats()["fp64_pairs"] > 0


def test_pairs_on_edges_mu(ctx):
    rng = np.random.default_rng(103)
    e0 = np.arange(41) * 5.0
    e1 = np.arange(41) / 40.0
    x = np.concatenate([edge_pairs_mu(rng, e1, r, 2) for r in (0.7, 3.0, 12.0, 77.0, 190.0)])
    _assert_same(gpu_count(ctx, "rmu", x, None, e0, e1), oracle_count("rmu", x, None, e0, e1))
    st = ctx.stats()
    assert st["fp64_pairs"] > 0
    if not getattr(ctx, "table_binning", False):
        assert st["fp64_pairs"] < st["rechecked_pairs"]


def test_pairs_on_edges_theta(ctx):
    rng = np.random.default_rng(104)
    theta = 10.0 ** (-2.0 + 3.0 * np.arange(65) / 64.0)
    chord = oracle.theta_to_chord(theta)
    pts = []
    for c in chord[::3]:
        for d in (0.0, 2.0**-40, -2.0**-40, 2.0**-26):
            n1 = synthetic._cap_uniform(1, 0.96, rng)[0]
            t = np.cross(n1, rng.normal(size=3))
            t /= np.linalg.norm(t)
            ang = 2 * np.arcsin(c * (1 + d) / 2)
            n2 = np.cos(ang) * n1 + np.sin(ang) * t
            pts += [n1, n2 / np.linalg.norm(n2)]
    x = np.array(pts)
    _assert_same(gpu_count(ctx, "theta", x, None, chord), oracle_count("theta", x, None, chord))
    # uniform chord edges (arithmetic binning and the double-float stage)
    cu = np.linspace(0.0, chord[-1], 33)
    _assert_same(gpu_count(ctx, "theta", x, None, cu), oracle_count("theta", x, None, cu))


@pytest.mark.parametrize("uniform", [True, False])
def test_integer_lattice_ties(ctx, uniform):
    """Integer coordinates and integer edges: every FP64 quantity of the
    canonical formulas is exact, so thousands of pairs sit exactly on an
    edge in FP64 (ties the FP32 bands must flag and the double-float stage
    must leave to the FP64 formula); (sigma, pi) and (r, mu) have unequal bin
    counts on the two axes; the (r, mu) pairs include pairs at exactly
    mu = 1/2: s = 2m s0, l = x_i + x_j = 2q (1, 1, 0) with s0 at 60 degrees
    to (1, 1, 0)."""
    rng = np.random.default_rng(109)
    e0 = np.arange(14.0) if uniform else np.array([0.0, 1, 2, 3, 5, 8, 13])
    es = np.arange(10.0) if uniform else np.array([0.0, 1, 2, 3, 4, 6, 9])
    ep = np.arange(8.0) if uniform else np.array([0.0, 1, 3, 5, 7])
    L = 40.0
    xo = rng.integers(100, 121, size=(700, 3)).astype(np.float64)
    xp = rng.integers(0, 40, size=(700, 3)).astype(np.float64)
    for x, per in ((xo, False), (xp, True)):
        kw = dict(periodic=per, L=L if per else 0.0)
        _assert_same(gpu_count(ctx, "mono", x, None, e0, **kw), oracle_count("mono", x, None, e0, **kw))
        assert ctx.stats()["fp64_pairs"] > 0
        _assert_same(gpu_count(ctx, "mono", x[:300], x[300:], e0, **kw),
                     oracle_count("mono", x[:300], x[300:], e0, **kw))
        _assert_same(gpu_count(ctx, "sigpi", x, None, es, ep, **kw),
                     oracle_count("sigpi", x, None, es, ep, **kw))
        assert ctx.stats()["fp64_pairs"] > 0
    s0 = np.array([[1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1]], dtype=np.float64)
    pts = []
    for q in range(300, 540, 20):
        for m in (1, 2, 3, 4):
            for v in s0:
                pts += [q * np.array([1.0, 1.0, 0.0]) - m * v, q * np.array([1.0, 1.0, 0.0]) + m * v]
    xr = np.concatenate([np.array(pts),
                         np.concatenate([rng.integers(300, 341, size=(400, 2)),
                                         rng.integers(-10, 11, size=(400, 1))], 1)])
    e1 = np.array([0.0, 0.25, 0.5, 0.75, 1.0])
    _assert_same(gpu_count(ctx, "rmu", xr, None, e0, e1), oracle_count("rmu", xr, None, e0, e1))
    assert ctx.stats()["fp64_pairs"] > 0


def test_periodic_faces_and_duplicates(ctx):
    rng = np.random.default_rng(105)
    L = 100.0
    x = rng.uniform(0, L, size=(3000, 3))
    # objects hugging the faces, so most close pairs wrap
    x[:1000] = np.mod(rng.normal(0, 2.0, size=(1000, 3)), L)
    x[x >= L] = 0.0
    x[1000:1200] = x[1200:1400]  # exact duplicates: separation 0
    e = np.linspace(0, 30, 13)
    _assert_same(gpu_count(ctx, "mono", x, None, e, periodic=True, L=L),
                 oracle_count("mono", x, None, e, periodic=True, L=L))
    es, ep = np.linspace(0, 25, 6), np.linspace(0, 10, 5)
    _assert_same(gpu_count(ctx, "sigpi", x, None, es, ep, periodic=True, L=L),
                 oracle_count("sigpi", x, None, es, ep, periodic=True, L=L))


@pytest.mark.parametrize("na,nb", [(0, 0), (0, 50), (1, 0), (1, 1), (2, 7), (65, 3)])
def test_tiny_catalogs(ctx, na, nb):
    rng = np.random.default_rng(106 + na + nb)
    a = rng.uniform(0, 50, size=(na, 3))
    b = rng.uniform(0, 50, size=(nb, 3))
    e = np.linspace(0, 20, 5)
    _assert_same(gpu_count(ctx, "mono", a, b, e), oracle_count("mono", a, b, e))
    _assert_same(gpu_count(ctx, "mono", a, None, e), oracle_count("mono", a, None, e))


def test_all_in_one_cell_dense(ctx):
    rng = np.random.default_rng(107)
    a = rng.normal(0, 0.5, size=(6000, 3)) + 50.0
    e = np.linspace(0, 4, 9)
    _assert_same(gpu_count(ctx, "mono", a, None, e), oracle_count("mono", a, None, e))


def test_invalid_requests_fail_cleanly(ctx):
    a = ctx.upload(np.random.default_rng(0).uniform(0, 10, size=(10, 3)))
    with pytest.raises(cute.CuteError):
        ctx.count("mono", a, None, np.linspace(0, 1, 3))  # no grid yet
    ctx.grid([a], [1.0, 1.0, 1.0])
    with pytest.raises(cute.CuteError):
        ctx.count("mono", a, None, np.linspace(0, 2, 3))  # reach too small
    with pytest.raises(cute.CuteError):
        ctx.count("mono", a, None, np.array([0.0, 0.5, 0.4]))  # not increasing
    with pytest.raises(cute.CuteError):
        ctx.count("rmu", a, None, np.linspace(0, 1, 3), np.array([0.0, 0.5, 0.9]))  # mu to 1
    with pytest.raises(cute.CuteError):
        ctx.upload(np.array([[0.0, 0.0, 10.0]]), periodic=True, L=10.0)  # x == L
    with pytest.raises(cute.CuteError):
        ctx.upload(np.array([[0.0, np.nan, 1.0]]))
    a.free()
    ctx.sync()


def test_rmu_near_the_observer_is_refused(ctx):
    """(r, mu) needs every object farther from the observer than half the
    largest r edge (else the line of sight x_i + x_j of a pair within reach
    can vanish): such a count is refused before any launch, and the same
    objects moved away from the observer count exactly."""
    rng = np.random.default_rng(111)
    x = rng.uniform(-60.0, 60.0, size=(300, 3))
    e0, e1 = np.linspace(0, 200, 41), np.linspace(0, 1, 41)
    a = ctx.upload(x)
    ctx.grid([a], [e0[-1]] * 3)
    with pytest.raises(cute.CuteError):
        ctx.count("rmu", a, None, e0, e1)
    a.free()
    far = x + np.array([900.0, 400.0, 300.0])
    _assert_same(gpu_count(ctx, "rmu", far, None, e0, e1), oracle_count("rmu", far, None, e0, e1))


def test_rmu_duplicates_and_log_bins(ctx):
    """(r, mu) on an open catalog with exact duplicates (separation 0: r bin
    0, mu bin 0) and on log-spaced r edges (table binning for r)."""
    rng = np.random.default_rng(108)
    x = rng.uniform(500, 700, size=(4000, 3))
    x[3000:3300] = x[3300:3600]
    e1 = np.linspace(0, 1, 9)
    e0 = np.linspace(0, 30, 7)
    _assert_same(gpu_count(ctx, "rmu", x, None, e0, e1), oracle_count("rmu", x, None, e0, e1))
    elog = np.concatenate([[0.0], np.geomspace(0.5, 30, 8)])
    _assert_same(gpu_count(ctx, "rmu", x, None, elog, e1), oracle_count("rmu", x, None, elog, e1))
    _assert_same(gpu_count(ctx, "sigpi", x, None, elog, np.linspace(0, 20, 5)),
                 oracle_count("sigpi", x, None, elog, np.linspace(0, 20, 5)))


def test_extent_limit_is_rejected(ctx):
    """A joint extent beyond 2e8 on an axis is refused at grid build (the
    kernels' padding sentinels sit at 1e9 in the grid frame)."""
    x = np.array([[0.0, 0.0, 0.0], [3e8, 1.0, 1.0], [1.0, 2.0, 3.0]])
    a = ctx.upload(x)
    with pytest.raises(cute.CuteError):
        ctx.grid([a], [10.0] * 3)
    a.free()


def test_catalog_churn_and_regrid(ctx):
    """Catalogs, grids and work lists come from the context's memory pool and
    pinned blocks: counts stay exact while catalogs of growing and shrinking
    sizes are uploaded, re-gridded at other cell sizes (the cached home
    chunks must follow) and freed in between, some living across rounds."""
    rng = np.random.default_rng(109)
    e0, e1 = np.linspace(0, 20, 9), np.linspace(0, 1, 5)
    # (away from the observer at the origin: mu needs |x_i + x_j| > 0)
    keep = rng.uniform(500, 620, size=(1500, 3))
    ck = ctx.upload(keep)
    for it, n in enumerate((800, 5000, 300, 3000, 1200)):
        x = rng.uniform(500, 620, size=(n, 3))
        cx = ctx.upload(x)
        for cpr in (2, 4):
            ctx.grid([ck, cx], [20.0] * 3, cpr)
            got = ctx.count("mono", cx, ck, e0)
            _assert_same(got, oracle_count("mono", x, keep, e0))
            got = ctx.count("rmu", ck, None, e0, e1)
            _assert_same(got, oracle_count("rmu", keep, None, e0, e1))
        cx.free()
    ck.free()
    ctx.sync()


def test_sparse_grid_many_cells(ctx):
    """A sparse catalog on a grid of over 2^18 cells (home chunks built on
    several host threads) counts exactly."""
    rng = np.random.default_rng(110)
    a = rng.uniform(0, 400, size=(3000, 3))
    b = rng.uniform(0, 400, size=(2000, 3))
    e = np.linspace(0, 20, 11)
    ca, cb = ctx.upload(a), ctx.upload(b)
    try:
        ctx.grid([ca, cb], [20.0] * 3, 2)
        _assert_same(ctx.count("mono", ca, None, e), oracle_count("mono", a, None, e))
        _assert_same(ctx.count("mono", ca, cb, e), oracle_count("mono", a, b, e))
    finally:
        ca.free()
        cb.free()

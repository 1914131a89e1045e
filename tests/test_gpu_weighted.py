"""GPU weighted counts and the adjoint against the FP64 oracle.

Weighted sums W_b = sum of w_i w_j over the pairs of bin b (the pixel and
density-grid weights of Sec. 3.4) must match the oracle's compensated FP64
sums to 1e-9 relative; the gradient dF/dw_i = sum_j w_j G[bin(i, j)] of
F = sum_b G_b W_b must match the oracle's FP64 rows, central finite
differences of the GPU forward, and Euler's identity sum_i w_i dF/dw_i = 2F.
"""
import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import cute, synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["arith", "table"])
def ctx(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cute.Context(0)
    if request.param == "table":
        c.set_launch(table_binning=True)
    yield c
    c.close()


def _case(n=6000, L=400.0, seed=30):
    rng = np.random.default_rng(seed)
    x = np.concatenate([synthetic.uniform_box(n // 2, L, rng),
                        synthetic.blobs_box(n // 200, 100, L, 5.0, rng)])
    w = np.exp(0.3 * rng.normal(size=len(x))).astype(np.float32)
    return x, w


def _upload(ctx, x, w, periodic, L, reach, y=None, wy=None):
    a = ctx.upload(x, weights=w, periodic=periodic, L=L)
    b = ctx.upload(y, weights=wy, periodic=periodic, L=L) if y is not None else None
    ctx.grid([a] + ([b] if b is not None else []), [reach] * 3)
    return a, b


@pytest.mark.parametrize("periodic", [True, False])
def test_weighted_counts_match_oracle(ctx, periodic):
    x, w = _case()
    L = 400.0
    e = np.arange(31) * 5.0
    a, _ = _upload(ctx, x, w, periodic, L, e[-1])
    c, oor, ws = ctx.count("mono", a, None, e, weighted=True)
    rc, roor, rws = oracle.count("mono", x, edges0=e, periodic=periodic, L=L, wa=w,
                                 weighted=True)
    assert c.tolist() == rc.tolist() and oor == roor
    np.testing.assert_allclose(ws, rws, rtol=1e-9, atol=0)
    a.free()


def test_weighted_cross_and_unit_weights(ctx):
    x, w = _case(4000, seed=31)
    y, wy = _case(3000, seed=32)
    e = np.geomspace(1.0, 60.0, 21)  # log bins: the table path
    a, b = _upload(ctx, x, w, True, 400.0, e[-1], y, wy)
    c, _, ws = ctx.count("mono", a, b, e, weighted=True)
    rc, _, rws = oracle.count("mono", x, y, edges0=e, periodic=True, L=400.0, wa=w, wb=wy,
                              weighted=True)
    assert c.tolist() == rc.tolist()
    np.testing.assert_allclose(ws, rws, rtol=1e-9, atol=0)
    a.free(); b.free()
    one = np.ones(len(x), np.float32)
    a, _ = _upload(ctx, x, one, True, 400.0, e[-1])
    c, _, ws = ctx.count("mono", a, None, e, weighted=True)
    assert ws.ravel().tolist() == c.ravel().astype(float).tolist()
    a.free()


def test_weighted_theta_matches_oracle(ctx):
    w = synthetic.c3_angular(scale=0.0006)
    chord = oracle.theta_to_chord(w.extra["theta_deg"])
    wt = np.exp(0.3 * np.random.default_rng(33).normal(size=len(w.data))).astype(np.float32)
    a = ctx.upload(w.data, weights=wt)
    ctx.grid([a], [chord[-1]] * 3)
    c, _, ws = ctx.count("theta", a, None, chord, weighted=True)
    rc, _, rws = oracle.count("theta", w.data, edges0=chord, wa=wt, weighted=True,
                              cells=[chord[-1]] * 3)
    assert c.tolist() == rc.tolist()
    m = rws.ravel() > 0
    np.testing.assert_allclose(ws.ravel()[m], rws.ravel()[m], rtol=1e-9, atol=0)
    a.free()


@pytest.mark.parametrize("cross", [False, True])
def test_adjoint_matches_oracle_rows(ctx, cross):
    x, w = _case(5000, seed=34)
    y, wy = _case(4000, seed=35) if cross else (None, None)
    L = 400.0
    e = np.arange(31) * 5.0
    G = np.random.default_rng(36).normal(size=30)
    a, b = _upload(ctx, x, w, True, L, e[-1], y, wy)
    if cross:
        ga, gb = ctx.adjoint("mono", a, b, e, G=G, grad_b=True)
    else:
        ga = ctx.adjoint("mono", a, None, e, G=G)
    rows = np.random.default_rng(37).choice(len(x), 300, replace=False)
    ref = oracle.grad_rows("mono", x, rows, G, wy if cross else w, xb=y, edges0=e, periodic=True,
                           L=L)
    scale = oracle.grad_rows("mono", x, rows, np.abs(G), wy if cross else w, xb=y, edges0=e,
                             periodic=True, L=L)
    assert np.all(np.abs(ga[rows] - ref) <= 1e-9 * scale + 1e-300)
    if cross:
        rows_b = np.random.default_rng(38).choice(len(y), 300, replace=False)
        refb = oracle.grad_rows("mono", y, rows_b, G, w, xb=x, edges0=e, periodic=True, L=L)
        scb = oracle.grad_rows("mono", y, rows_b, np.abs(G), w, xb=x, edges0=e, periodic=True, L=L)
        assert np.all(np.abs(gb[rows_b] - refb) <= 1e-9 * scb + 1e-300)
    a.free()
    if b is not None:
        b.free()


def test_adjoint_finite_differences_and_euler(ctx):
    """F is linear in each w_i (no self pairs), so the central difference with
    h = w_i is exact up to the rounding of the GPU's FP64 weighted forward."""
    x, w = _case(3000, L=200.0, seed=39)
    L = 200.0
    e = np.arange(16) * 4.0
    G = np.random.default_rng(40).normal(size=15)

    def F(wv):
        a = ctx.upload(x, weights=wv, periodic=True, L=L)
        ctx.grid([a], [e[-1]] * 3)
        _, _, ws = ctx.count("mono", a, None, e, weighted=True)
        a.free()
        return float(np.dot(G, ws.ravel()))

    a = ctx.upload(x, weights=w, periodic=True, L=L)
    ctx.grid([a], [e[-1]] * 3)
    g = ctx.adjoint("mono", a, None, e, G=G)
    a.free()
    for i in np.random.default_rng(41).choice(len(x), 12, replace=False):
        wp = w.copy(); wp[i] = np.float32(2 * w[i])
        wm = w.copy(); wm[i] = np.float32(0.0)
        fd = (F(wp) - F(wm)) / (2.0 * float(w[i]))
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    assert float(np.dot(w.astype(np.float64), g)) == pytest.approx(2 * F(w), rel=1e-9)


@pytest.mark.parametrize("hp", [2, 4])
def test_weighted_rmu_matches_oracle(ctx, hp):
    """Weighted (r, mu) counts read the neighbours' weights from a tile of
    their own, which the neighbour cull compacts and carries beside the
    rows: light-cone DD (auto) and DR (cross) with slices of several tiles,
    counts bit for bit and weight sums to 1e-9 against the oracle."""
    v = synthetic.c2_rmu_lightcone(scale=0.004)
    # 6 x 6 bins: weighted counts keep 32 float-float columns per warp
    e0 = np.arange(7) * 25.0
    e1 = np.arange(7) / 6.0
    wd = np.exp(0.3 * np.random.default_rng(45).normal(size=len(v.data))).astype(np.float32)
    wr = np.exp(0.3 * np.random.default_rng(46).normal(size=len(v.randoms))).astype(np.float32)
    table = ctx.table_binning if hasattr(ctx, "table_binning") else False
    ctx.set_launch(home_per_lane=hp, slice=512, table_binning=table)
    try:
        d = ctx.upload(v.data, weights=wd)
        r = ctx.upload(v.randoms, weights=wr)
        ctx.grid([d, r], [e0[-1]] * 3, 4)
        for b, xb, wb in ((None, None, None), (r, v.randoms, wr)):
            c, oor, ws = ctx.count("rmu", d, b, e0, e1, weighted=True)
            st = ctx.stats()
            rc, roor, rws = oracle.count("rmu", v.data, xb, edges0=e0, edges1=e1,
                                         wa=wd, wb=wb, weighted=True)
            assert c.tolist() == rc.tolist() and oor == roor
            np.testing.assert_allclose(ws, rws, rtol=1e-9, atol=0)
            assert st["candidate_pairs"] < st["stencil_pairs"]
        d.free(); r.free()
    finally:
        ctx.set_launch(table_binning=table)


def test_adjoint_rmu_and_sigpi(ctx):
    v = synthetic.c2_rmu_lightcone(scale=0.002)
    wd = np.exp(0.3 * np.random.default_rng(42).normal(size=len(v.data))).astype(np.float32)
    wr = np.exp(0.3 * np.random.default_rng(43).normal(size=len(v.randoms))).astype(np.float32)
    d = ctx.upload(v.data, weights=wd)
    r = ctx.upload(v.randoms, weights=wr)
    ctx.grid([d, r], [v.edges0[-1]] * 3)
    G = np.random.default_rng(44).normal(size=40 * 40)
    ga = ctx.adjoint("rmu", d, r, v.edges0, v.edges1, G=G)
    rows = np.arange(0, len(v.data), 7)
    ref = oracle.grad_rows("rmu", v.data, rows, G, wr, xb=v.randoms, edges0=v.edges0,
                           edges1=v.edges1)
    sc = oracle.grad_rows("rmu", v.data, rows, np.abs(G), wr, xb=v.randoms, edges0=v.edges0,
                          edges1=v.edges1)
    assert np.all(np.abs(ga[rows] - ref) <= 1e-9 * sc + 1e-300)
    d.free(); r.free()


@pytest.mark.parametrize("cross", [False, True])
def test_autograd_weighted_count(ctx, cross):
    """CuteWeightedCount: W from the forward equals the oracle's weighted
    counts, and w.grad after backward equals the oracle's gradient rows for
    every weight (the adjoint), on device tensors."""
    x, w = _case(3000, seed=33)
    y, wy = _case(2000, seed=34) if cross else (None, None)
    L = 400.0
    e = np.arange(31) * 5.0
    G = np.random.default_rng(35).normal(size=30)
    wa = torch.tensor(w, device="cuda", requires_grad=True)
    wb = torch.tensor(wy, device="cuda", requires_grad=True) if cross else None
    W = cute.CuteWeightedCount.apply(wa, wb, ctx, "mono", x, y, e, None, True, L, [e[-1]] * 3, 0)
    assert W.shape == (30, 1) and W.dtype == torch.float64
    _, _, rws = oracle.count("mono", x, y, edges0=e, periodic=True, L=L, wa=w, wb=wy,
                             weighted=True)
    np.testing.assert_allclose(W.detach().cpu().numpy(), rws, rtol=1e-9, atol=0)
    (W.view(-1) * torch.tensor(G, device="cuda")).sum().backward()
    rows = np.arange(len(x))
    ref = oracle.grad_rows("mono", x, rows, G, wy if cross else w, xb=y, edges0=e, periodic=True,
                           L=L)
    scale = oracle.grad_rows("mono", x, rows, np.abs(G), wy if cross else w, xb=y, edges0=e,
                             periodic=True, L=L)
    got = wa.grad.detach().cpu().numpy().astype(np.float64)
    # float32 gradient of float32 weights: relative to the absolute-G scale
    assert np.all(np.abs(got - ref) <= 1e-6 * scale + 1e-30)
    if cross:
        refb = oracle.grad_rows("mono", y, np.arange(len(y)), G, w, xb=x, edges0=e,
                                periodic=True, L=L)
        scaleb = oracle.grad_rows("mono", y, np.arange(len(y)), np.abs(G), w, xb=x, edges0=e,
                                  periodic=True, L=L)
        gotb = wb.grad.detach().cpu().numpy().astype(np.float64)
        assert np.all(np.abs(gotb - refb) <= 1e-6 * scaleb + 1e-30)


def test_autograd_forward_without_backward_frees_catalogs(ctx):
    """A forward whose output needs a gradient but is never differentiated
    keeps its catalogs only while the autograd graph lives: dropping the
    output frees them (catalog handles are issued in order, so the forward's
    two catalogs are the two after a probe catalog)."""
    import ctypes
    import gc
    x, w = _case(500, seed=36)
    y, wy = _case(400, seed=37)
    L = 400.0
    e = np.arange(31) * 5.0
    probe = ctx.upload(x[:10])
    first = probe.id
    probe.free()
    wa = torch.tensor(w, device="cuda", requires_grad=True)
    wb = torch.tensor(wy, device="cuda", requires_grad=True)
    W = cute.CuteWeightedCount.apply(wa, wb, ctx, "mono", x, y, e, None, True, L, [e[-1]] * 3, 0)
    n = ctypes.c_int64()
    held = [first + 1, first + 2]
    assert all(cute.lib().cute_catalog_size(ctx.handle, i, ctypes.byref(n)) == 0 for i in held)
    del W
    gc.collect()
    assert all(cute.lib().cute_catalog_size(ctx.handle, i, ctypes.byref(n)) == -4 for i in held)


@pytest.mark.parametrize("wmax", [40, 300])
@pytest.mark.parametrize("periodic", [True, False])
def test_integer_weights_exact(ctx, periodic, wmax):
    """Weights that are all integers in [0, 2048] (counts per pixel or cell)
    take the integer weight histograms: W_b is then an exact integer sum and
    equals the oracle's bit for bit, auto and cross, monopole and chords.
    Weights up to 300 make the library shorten the neighbour slices so that
    one work item cannot overflow a 32-bit weight sum."""
    rng = np.random.default_rng(40 + wmax)
    x, _ = _case(5000, seed=41)
    w = rng.integers(0, wmax + 1, len(x)).astype(np.float32)
    L = 400.0
    e = np.arange(31) * 5.0
    a, _ = _upload(ctx, x, w, periodic, L, e[-1])
    c, oor, ws = ctx.count("mono", a, None, e, weighted=True)
    rc, roor, rws = oracle.count("mono", x, edges0=e, periodic=periodic, L=L, wa=w, weighted=True)
    assert c.tolist() == rc.tolist() and oor == roor
    np.testing.assert_array_equal(ws, rws)
    a.free()
    # cross count, and chords between unit vectors (log-spaced angles)
    y = synthetic.uniform_box(3000, L, rng)
    wy = rng.integers(1, wmax + 1, len(y)).astype(np.float32)
    a, b = _upload(ctx, x, w, periodic, L, e[-1], y=y, wy=wy)
    c, oor, ws = ctx.count("mono", a, b, e, weighted=True)
    rc, roor, rws = oracle.count("mono", x, y, edges0=e, periodic=periodic, L=L, wa=w, wb=wy,
                                 weighted=True)
    assert c.tolist() == rc.tolist() and oor == roor
    np.testing.assert_array_equal(ws, rws)
    a.free(); b.free()
    if not periodic:
        u = rng.normal(size=(4000, 3))
        u[:, 2] = np.abs(u[:, 2]) + 2.0
        u /= np.linalg.norm(u, axis=1)[:, None]
        wu = rng.integers(0, wmax + 1, len(u)).astype(np.float32)
        ch = cute.theta_to_chord(np.logspace(-1, 1.3, 21))
        p = ctx.upload(u, weights=wu)
        ctx.grid([p], [ch[-1]] * 3)
        c, oor, ws = ctx.count("theta", p, None, ch, weighted=True)
        rc, roor, rws = oracle.count("theta", u, edges0=ch, wa=wu, weighted=True)
        assert c.tolist() == rc.tolist() and oor == roor
        np.testing.assert_array_equal(ws, rws)
        p.free()

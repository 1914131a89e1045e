"""Parity at the full sizes of the five workloads, in the launch
configuration bench.py uses (4 cells per reach for the light cone, the
library's density-based choice elsewhere; library-chosen shape).

Where the FP64 oracle cannot finish a full count in seconds, the check is on
sampled rows: a seeded subset S of one catalog is uploaded as its own
catalog on the same grid, and the GPU's S x B cross count (the same kernel
on the full partner catalog) must equal the oracle's brute-force S x B
count bit for bit.  Full-size counts are further tied together by exact
invariants between kernels (the mu-marginal of (r, mu) equals the monopole;
batched equals plain; the weighted pass's counts equal the plain counts;
Euler's identity links the forward and the adjoint).
"""
import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import cute, synthetic

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CPR = 4  # bench.py's cells per reach


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cute.Context(0)
    yield c
    c.close()


def _rows(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def test_c2_rmu_lightcone_full(ctx):
    w = synthetic.c2_rmu_lightcone()
    e0, e1 = w.edges0, w.edges1
    sd = w.data[_rows(len(w.data), 1500, 70)]
    sr = w.randoms[_rows(len(w.randoms), 600, 71)]
    D, R, SD, SR = (ctx.upload(x) for x in (w.data, w.randoms, sd, sr))
    ctx.grid([D, R, SD, SR], [e0[-1]] * 3, CPR)
    dd, _, _ = ctx.count("rmu", D, None, e0, e1)
    dr, _, _ = ctx.count("rmu", D, R, e0, e1)
    rr, _, _ = ctx.count("rmu", R, None, e0, e1)
    # full DD against the cell-pruned oracle (itself pinned to brute force)
    ref_dd, _, _ = oracle.count("rmu", w.data, edges0=e0, edges1=e1, cells=[e0[-1]] * 3)
    assert dd.tolist() == ref_dd.tolist()
    # sampled rows against the full partner catalogs
    for S, xs, B, xb in ((SD, sd, R, w.randoms), (SD, sd, D, w.data), (SR, sr, R, w.randoms)):
        got, _, _ = ctx.count("rmu", S, B, e0, e1)
        ref, _, _ = oracle.count("rmu", xs, xb, edges0=e0, edges1=e1)
        assert got.tolist() == ref.tolist()
    # mu-marginal of every full count equals the monopole count (Eq. 4)
    for (a, b), c in (((D, None), dd), ((D, R), dr), ((R, None), rr)):
        mono, _, _ = ctx.count("mono", a, b, e0)
        assert c.sum(axis=1).tolist() == mono.ravel().tolist()
    xi = cute.estimator("ls", dd, dr, rr, len(w.data), len(w.randoms))
    ref_xi = oracle.xi_ls(dd, dr, rr, len(w.data), len(w.randoms))
    m = ~np.isnan(ref_xi)
    np.testing.assert_allclose(xi[m], ref_xi[m], rtol=1e-12, atol=1e-12)
    for c in (D, R, SD, SR):
        c.free()


def test_c3_angular_full(ctx):
    w = synthetic.c3_angular()
    chord = oracle.theta_to_chord(w.extra["theta_deg"])
    sd = w.data[_rows(len(w.data), 300, 72)]
    sr = w.randoms[_rows(len(w.randoms), 150, 73)]
    D, R, SD, SR = (ctx.upload(x) for x in (w.data, w.randoms, sd, sr))
    ctx.grid([D, R, SD, SR], [chord[-1]] * 3)
    dd, _, _ = ctx.count("theta", D, None, chord)
    assert int(dd.sum()) > 0
    for S, xs, B, xb in ((SD, sd, D, w.data), (SD, sd, R, w.randoms), (SR, sr, R, w.randoms)):
        got, _, _ = ctx.count("theta", S, B, chord)
        ref, _, _ = oracle.count("theta", xs, xb, edges0=chord)
        assert got.tolist() == ref.tolist()
    for c in (D, R, SD, SR):
        c.free()


def test_c4_batched_sigpi_full(ctx):
    boxes = synthetic.c4_batched_sigpi()
    e0, e1 = boxes[0].edges0, boxes[0].edges1
    reach = [e0[-1], e0[-1], e1[-1]]
    cats, pairs = [], []
    for b in boxes:
        d = ctx.upload(b.data, periodic=True, L=b.L)
        r = ctx.upload(b.randoms, periodic=True, L=b.L)
        ctx.grid([d, r], reach)
        cats.append((d, r))
        pairs += [(d, None), (d, r), (r, None)]
    batched = ctx.count_batched("sigpi", pairs, e0, e1)
    for k, (a, b) in enumerate(pairs):
        plain, _, _ = ctx.count("sigpi", a, b, e0, e1)
        assert batched[k].tolist() == plain.tolist()
    # the two smallest boxes against the cell-pruned oracle
    small = np.argsort([len(b.data) for b in boxes])[:2]
    for bi in small:
        b = boxes[bi]
        for k, (xa, xb) in enumerate(((b.data, None), (b.data, b.randoms), (b.randoms, None))):
            ref, _, _ = oracle.count("sigpi", xa, xb, edges0=e0, edges1=e1, periodic=True, L=b.L,
                                     cells=reach)
            assert batched[3 * bi + k].tolist() == ref.tolist()
    for d, r in cats:
        d.free(); r.free()


def test_c5_weighted_and_adjoint_full(ctx):
    w = synthetic.c5_weighted()
    e, G, idx = w.edges0, w.extra["G"], w.extra["fd_idx"]
    A = ctx.upload(w.data, weights=w.weights, periodic=True, L=w.L)
    S = ctx.upload(w.data[idx], weights=np.ones(len(idx), np.float32), periodic=True, L=w.L)
    ctx.grid([A, S], [e[-1]] * 3)
    counts, _, ws = ctx.count("mono", A, None, e, weighted=True)
    plain, _, _ = ctx.count("mono", A, None, e)
    assert counts.tolist() == plain.tolist()
    grad = ctx.adjoint("mono", A, None, e, G=G)
    # gradient rows of the 1,000 sampled weights against the FP64 oracle
    ref = oracle.grad_rows("mono", w.data, idx, G, w.weights, edges0=e, periodic=True, L=w.L)
    scale = oracle.grad_rows("mono", w.data, idx, np.abs(G), w.weights, edges0=e, periodic=True,
                             L=w.L)
    assert np.all(np.abs(grad[idx] - ref) <= 1e-9 * scale + 1e-300)
    # sampled rows (unit weight) x full catalog: sum_j w_j per bin, which is
    # the derivative of W_b with respect to w_i summed over the rows (plus
    # the rows' self pairs at separation 0, in bin 0)
    got_c, _, got_w = ctx.count("mono", S, A, e, weighted=True)
    ref_c, _, ref_w = oracle.count("mono", w.data[idx], w.data, edges0=e, periodic=True, L=w.L,
                                   wa=np.ones(len(idx), np.float32), wb=w.weights, weighted=True)
    assert got_c.tolist() == ref_c.tolist()
    np.testing.assert_allclose(got_w, ref_w, rtol=1e-9)
    sw = float(np.dot(G, got_w.ravel())) - float(G[0] * w.weights[idx].astype(np.float64).sum())
    assert sw == pytest.approx(float(grad[idx].sum()), rel=1e-9, abs=1e-9 * float(scale.sum()))
    # Euler: F(w) = sum_b G_b W_b is homogeneous of degree 2 in w
    F = float(np.dot(G, ws.ravel()))
    assert float(np.dot(w.weights.astype(np.float64), grad)) == pytest.approx(2 * F, rel=1e-9)
    A.free(); S.free()

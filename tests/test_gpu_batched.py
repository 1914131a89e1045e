"""Batched counts (many mock catalogs in one persistent launch, the use of
Fig. 5) equal separate counts bit for bit, and the oracle."""
import numpy as np
import pytest

from paper_1210_1833_gb300 import cute, synthetic
from gpu_util import oracle_count

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cute.Context(0)
    yield c
    c.close()


def test_batched_sigpi_boxes_equal_plain_and_oracle(ctx):
    boxes = synthetic.c4_batched_sigpi(n_boxes=6, scale=0.02)
    reach = [boxes[0].edges0[-1], boxes[0].edges0[-1], boxes[0].edges1[-1]]
    cats, pairs = [], []
    for b in boxes:
        d = ctx.upload(b.data, periodic=True, L=b.L)
        r = ctx.upload(b.randoms, periodic=True, L=b.L)
        ctx.grid([d, r], reach)
        cats.append((d, r))
        pairs += [(d, None), (d, r), (r, None)]
    e0, e1 = boxes[0].edges0, boxes[0].edges1
    batched = ctx.count_batched("sigpi", pairs, e0, e1)
    for k, (a, b) in enumerate(pairs):
        plain, _, _ = ctx.count("sigpi", a, b, e0, e1)
        assert batched[k].tolist() == plain.tolist()
    # the oracle on two of the boxes
    for bi in (0, 5):
        b = boxes[bi]
        for k, (xa, xb) in enumerate(((b.data, None), (b.data, b.randoms), (b.randoms, None))):
            ref, _, _ = oracle_count("sigpi", xa, xb, e0, e1, periodic=True, L=b.L, cells=True)
            assert batched[3 * bi + k].tolist() == ref.tolist()
    for d, r in cats:
        d.free(); r.free()


def test_batched_weighted_equal_plain(ctx):
    rng = np.random.default_rng(50)
    L = 300.0
    e = np.arange(21) * 3.0
    cats, pairs = [], []
    for k in range(5):
        n = int(rng.integers(500, 3000))
        x = synthetic.uniform_box(n, L, rng)
        w = np.exp(0.3 * rng.normal(size=n)).astype(np.float32)
        a = ctx.upload(x, weights=w, periodic=True, L=L)
        ctx.grid([a], [e[-1]] * 3)
        cats.append(a)
        pairs.append((a, None))
    counts, ws = ctx.count_batched("mono", pairs, e, weighted=True)
    for k, (a, _) in enumerate(pairs):
        c, _, w1 = ctx.count("mono", a, None, e, weighted=True)
        assert counts[k].tolist() == c.tolist()
        np.testing.assert_allclose(ws[k], w1, rtol=1e-12)
    for a in cats:
        a.free()


def test_batched_device_outputs_replay_graph(ctx):
    """Device outputs: the first call captures a CUDA graph, later calls
    replay it; every replay equals the plain counts."""
    boxes = synthetic.c4_batched_sigpi(n_boxes=4, scale=0.02)
    reach = [boxes[0].edges0[-1], boxes[0].edges0[-1], boxes[0].edges1[-1]]
    cats, pairs = [], []
    for b in boxes:
        d = ctx.upload(b.data, periodic=True, L=b.L)
        r = ctx.upload(b.randoms, periodic=True, L=b.L)
        ctx.grid([d, r], reach)
        cats.append((d, r))
        pairs += [(d, None), (d, r), (r, None)]
    e0, e1 = boxes[0].edges0, boxes[0].edges1
    plain = [ctx.count("sigpi", a, b, e0, e1)[0] for a, b in pairs]
    for _ in range(3):
        out = ctx.count_batched("sigpi", pairs, e0, e1, device=True)
        torch.cuda.synchronize()
        for k in range(len(pairs)):
            got = out[k].cpu().numpy().view(np.uint64)
            assert got.tolist() == plain[k].tolist()
    for d, r in cats:
        d.free(); r.free()


def test_autotune_keeps_counts_exact(ctx):
    w = synthetic.c2_rmu_lightcone(scale=0.01)
    d = ctx.upload(w.data)
    r = ctx.upload(w.randoms)
    ctx.grid([d, r], [w.edges0[-1]] * 3)
    ref = [ctx.count("rmu", a, b, w.edges0, w.edges1)[0] for a, b in ((d, None), (d, r))]
    t = ctx.autotune("rmu", [(d, r)], w.edges0, w.edges1, tune_cells=True, max_items=2000)
    assert t["cells_per_reach"] in (2, 3, 4) and t["home_per_lane"] in (2, 4)
    # (counts under 1e10 candidate pairs also try 64- and 256-neighbour slices)
    assert t["warps_per_block"] in (8, 12, 16) and t["slice"] in (64, 256, 1024, 2048, 4096)
    got = [ctx.count("rmu", a, b, w.edges0, w.edges1)[0] for a, b in ((d, None), (d, r))]
    for g, f in zip(got, ref):
        assert g.tolist() == f.tolist()
    d.free(); r.free()

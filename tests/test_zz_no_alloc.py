"""cute_count_pairs_noalloc: the counting entry point for callers that cannot
let the library allocate device memory when they count (a framework's
caching allocator owning the device, loops where cudaMalloc/cudaFree would
synchronise the device).

Through the C ABI, on two calls in a row, its counts must equal those of
cute_count_pairs exactly (integer counts) and its weighted sums within the
1e-12 relative tolerance the tests use for repeated FP64 accumulation.  This
file is collected last so that a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest

from paper_1210_1833_gb300 import cute, synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(ctx, kind, a, b, e0, e1=None, weighted=False):
    n0 = len(e0) - 1
    n1 = len(e1) - 1 if (e1 is not None and kind in ("rmu", "sigpi")) else 1
    e0 = np.ascontiguousarray(e0, dtype=np.float64)
    e1 = None if e1 is None else np.ascontiguousarray(e1, dtype=np.float64)
    d = ctx._desc(kind, a, b, e0, e1 if kind in ("rmu", "sigpi") else None, weighted)
    counts = torch.zeros(n0 * n1, dtype=torch.int64, device="cuda")
    wsum = torch.zeros(n0 * n1, dtype=torch.float64, device="cuda") if weighted else None
    st = cute.lib().cute_count_pairs_noalloc(ctx.handle, ctypes.byref(d),
                                             ctypes.c_void_p(counts.data_ptr()),
                                             ctypes.c_void_p(wsum.data_ptr()) if weighted else None)
    if st != 0:
        raise cute.CuteError(st, cute.lib().cute_last_error(ctx.handle).decode())
    ctx.sync()
    c = counts.cpu().numpy().view(np.uint64).reshape(n0, n1)
    return c, (None if wsum is None else wsum.cpu().numpy().reshape(n0, n1))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cute.Context(0)
    yield c
    c.close()


def test_noalloc_matches_count_pairs(ctx):
    w = synthetic.c1_monopole_box(scale=0.25)
    a = ctx.upload(w.data, periodic=True, L=w.L)
    ctx.grid([a], [w.edges0[-1]] * 3)
    ref, _, _ = ctx.count("mono", a, None, w.edges0)
    for _ in range(2):
        got, _ = _noalloc(ctx, "mono", a, None, w.edges0)
        assert got.tolist() == ref.tolist()
    a.free()

    v = synthetic.c2_rmu_lightcone(scale=0.004)
    d = ctx.upload(v.data)
    r = ctx.upload(v.randoms)
    ctx.grid([d, r], [v.edges0[-1]] * 3)
    for b in (None, r):
        ref, _, _ = ctx.count("rmu", d, b, v.edges0, v.edges1)
        for _ in range(2):
            got, _ = _noalloc(ctx, "rmu", d, b, v.edges0, v.edges1)
            assert got.tolist() == ref.tolist()
    d.free()
    r.free()


def test_noalloc_weighted_matches_count_pairs(ctx):
    rng = np.random.default_rng(60)
    L = 300.0
    x = synthetic.uniform_box(4000, L, rng)
    wt = np.exp(0.3 * rng.normal(size=len(x))).astype(np.float32)
    e = np.arange(21) * 3.0
    a = ctx.upload(x, weights=wt, periodic=True, L=L)
    ctx.grid([a], [e[-1]] * 3)
    ref, _, rws = ctx.count("mono", a, None, e, weighted=True)
    for _ in range(2):
        got, ws = _noalloc(ctx, "mono", a, None, e, weighted=True)
        assert got.tolist() == ref.tolist()
        np.testing.assert_allclose(ws, rws, rtol=1e-12)
    a.free()


def test_noalloc_rejects_host_outputs(ctx):
    x = np.random.default_rng(61).uniform(0, 10, size=(100, 3))
    a = ctx.upload(x)
    ctx.grid([a], [2.0] * 3)
    e = np.linspace(0, 2, 5)
    d = ctx._desc("mono", a, None, np.ascontiguousarray(e), None, False)
    host = np.zeros(4, dtype=np.uint64)
    st = cute.lib().cute_count_pairs_noalloc(ctx.handle, ctypes.byref(d),
                                             host.ctypes.data_as(ctypes.c_void_p), None)
    assert st == -1
    a.free()


def test_noalloc_sigpi_periodic_matches_count_pairs(ctx):
    # the disk-slab stencil and the second edge table of the scratch layout
    b = synthetic.c4_batched_sigpi(scale=0.02)[0]
    e0, e1 = b.edges0, b.edges1
    d = ctx.upload(b.data, periodic=True, L=b.L)
    r = ctx.upload(b.randoms, periodic=True, L=b.L)
    ctx.grid([d, r], [e0[-1], e0[-1], e1[-1]])
    for bb in (None, r):
        ref, _, _ = ctx.count("sigpi", d, bb, e0, e1)
        assert int(ref.sum()) > 0
        for _ in range(2):
            got, _ = _noalloc(ctx, "sigpi", d, bb, e0, e1)
            assert got.tolist() == ref.tolist()
    d.free()
    r.free()


def test_noalloc_rejects_requests_beyond_its_scratch(ctx):
    # a count whose work-item records alone exceed the fixed 8 MiB array is
    # refused before anything is launched, with the size in the message
    x = synthetic.uniform_box(1_000_000, 1000.0, np.random.default_rng(62))
    a = ctx.upload(x, periodic=True, L=1000.0)
    ctx.grid([a], [100.0] * 3, 4)
    e = np.linspace(0.0, 100.0, 11)
    d = ctx._desc("mono", a, None, np.ascontiguousarray(e), None, False)
    counts = torch.zeros(10, dtype=torch.int64, device="cuda")
    ctx.set_launch(slice=64)
    try:
        st = cute.lib().cute_count_pairs_noalloc(ctx.handle, ctypes.byref(d),
                                                 ctypes.c_void_p(counts.data_ptr()), None)
        msg = cute.lib().cute_last_error(ctx.handle).decode()
    finally:
        ctx.set_launch()
    assert st == -1
    assert "bytes of scratch" in msg
    ctx.sync()
    assert int(counts.sum()) == 0
    a.free()

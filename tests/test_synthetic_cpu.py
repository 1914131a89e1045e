"""The seeded synthetic workloads (they stand in for the paper's MICE,
PTHalo and log-normal catalogs of Sec. 4, which are not available) against
their stated recipes: sizes, boxes and sky windows, bin edges, the
volume-uniform and area-uniform draws, the clustered parts, and that every
draw is fixed by its seed."""
import math

import numpy as np

from paper_1210_1833_gb300 import synthetic


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_c1_periodic_box():
    w = synthetic.c1_monopole_box()
    assert w.kind == "mono" and w.periodic and w.L == 1000.0
    assert w.data.shape == (20000, 3) and ((w.data >= 0) & (w.data < w.L)).all()
    assert np.array_equal(w.edges0, np.arange(41) * 5.0) and w.edges1 is None
    # the second half: 200 blobs of 50 points, sigma 5 per axis
    blobs = w.data[10000:].reshape(200, 50, 3)
    d = _min_image(blobs - blobs[:, :1, :], w.L)
    assert np.abs(d).max() < 8 * 5.0 * math.sqrt(2)
    assert 0.8 * 5.0 * math.sqrt(2) < d[:, 1:, :].std() < 1.2 * 5.0 * math.sqrt(2)
    assert np.array_equal(w.data, synthetic.c1_monopole_box().data)


def test_c2_light_cone_wedge():
    w = synthetic.c2_rmu_lightcone()
    assert w.kind == "rmu" and not w.periodic
    assert w.data.shape == (500000, 3) and w.randoms.shape == (2000000, 3)
    assert np.array_equal(w.edges0, np.arange(41) * 5.0)
    assert np.array_equal(w.edges1, np.arange(41) / 40.0)
    for x in (w.data, w.randoms):
        r = np.linalg.norm(x, axis=1)
        ra = np.degrees(np.arctan2(x[:, 1], x[:, 0]))
        dec = np.degrees(np.arcsin(x[:, 2] / r))
        assert r.min() >= 1000.0 - 1e-9 and r.max() <= 2500.0 + 1e-9
        assert ra.min() >= -1e-9 and ra.max() < 60.0 + 1e-9
        assert dec.min() >= -1e-9 and dec.max() < 30.0 + 1e-9
    # randoms uniform in volume (r^3 uniform) and in area (sin Dec uniform)
    r = np.linalg.norm(w.randoms, axis=1)
    u = (r ** 3 - 1000.0 ** 3) / (2500.0 ** 3 - 1000.0 ** 3)
    assert abs(u.mean() - 0.5) < 0.002 and abs(np.median(u) - 0.5) < 0.002
    s = w.randoms[:, 2] / r
    assert abs(s.mean() - 0.25) < 0.002
    # data in 20 patches: far more clustered on the sky than the randoms
    hd, _, _ = np.histogram2d(np.arctan2(w.data[:, 1], w.data[:, 0]),
                              w.data[:, 2] / np.linalg.norm(w.data, axis=1), bins=30)
    hr, _, _ = np.histogram2d(np.arctan2(w.randoms[:, 1], w.randoms[:, 0]), s, bins=30)
    assert (hd / hd.mean()).std() > 3 * (hr / hr.mean()).std()


def test_c3_cap_of_1000_square_degrees():
    w = synthetic.c3_angular(scale=0.01)
    cos_a = 1.0 - 1000.0 * (math.pi / 180.0) ** 2 / (2 * math.pi)
    assert math.isclose(2 * math.pi * (1 - cos_a) * (180 / math.pi) ** 2, 1000.0, rel_tol=1e-12)
    assert w.data.shape == (50000, 3) and w.randoms.shape == (200000, 3)
    for x in (w.data, w.randoms):
        np.testing.assert_allclose(np.linalg.norm(x, axis=1), 1.0, rtol=1e-14)
        assert x[:, 2].min() >= cos_a
    assert abs(w.randoms[:, 2].mean() - 0.5 * (1 + cos_a)) < 2e-4
    t = w.extra["theta_deg"]
    np.testing.assert_allclose(t, 10.0 ** (-2.0 + 3.0 * np.arange(65) / 64.0), rtol=0)
    # the last 500 data points: 5 clumps of 100 within a few 0.05-degree sigmas
    cl = w.data[-500:].reshape(5, 100, 3)
    ang = np.degrees(np.arccos(np.clip(np.einsum("cij,cj->ci", cl, cl.mean(1) / np.linalg.norm(
        cl.mean(1), axis=1, keepdims=True)), -1, 1)))
    assert ang.max() < 0.05 * 6


def test_c4_boxes():
    boxes = synthetic.c4_batched_sigpi(n_boxes=3)
    assert len(boxes) == 3
    e = np.arange(51) * 3.0
    for b in boxes:
        n = len(b.data)
        assert b.kind == "sigpi" and b.periodic and b.L == 1500.0
        # randoms 2N for the drawn N; the data hold N less the remainder of
        # cutting N/2 into N/100 equal blobs (under 1 %)
        assert 0.99 * 50000 <= n <= 400000
        assert 0 <= len(b.randoms) - 2 * n <= 0.02 * len(b.randoms)
        for x in (b.data, b.randoms):
            assert ((x >= 0) & (x < b.L)).all()
        assert np.array_equal(b.edges0, e) and np.array_equal(b.edges1, e)
    again = synthetic.c4_batched_sigpi(n_boxes=3)
    assert all(np.array_equal(a.data, b.data) for a, b in zip(boxes, again))


def test_c5_weighted_box():
    w = synthetic.c5_weighted()
    assert w.periodic and w.L == 2000.0 and w.data.shape == (4000000, 3)
    assert ((w.data >= 0) & (w.data < w.L)).all()
    assert w.weights.dtype == np.float32 and (w.weights > 0).all()
    lw = np.log(w.weights.astype(np.float64))
    assert abs(lw.mean()) < 0.002 and abs(lw.std() - 0.3) < 0.002
    assert np.array_equal(w.edges0, np.arange(31) * 5.0)
    assert w.extra["G"].shape == (30,)
    idx = w.extra["fd_idx"]
    assert len(idx) == 1000 and len(np.unique(idx)) == 1000 and (np.diff(idx) > 0).all()


def test_subsample_is_seeded_and_without_replacement():
    x = np.arange(3000.0).reshape(1000, 3)
    a = synthetic.subsample(x, 100, 7)
    assert np.array_equal(a, synthetic.subsample(x, 100, 7))
    assert len(np.unique(a[:, 0])) == 100 and (np.diff(a[:, 0]) > 0).all()
    assert synthetic.subsample(x, 5000, 7) is x

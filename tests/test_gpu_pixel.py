"""Pixel maps for w(theta) (Sec. 3.4.2): HEALPix RING pixel indices and
centres on the GPU against the oracle, and the pixel-weighted angular count
of a catalog against the oracle's weighted count of the same pixels."""
import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import cute, synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cute.Context(0)
    yield c
    c.close()


def _sphere(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


@pytest.mark.parametrize("nside", [1, 4, 64, 1024])
def test_pixel_map_matches_oracle(ctx, nside):
    v = _sphere(200_000, 100 + nside)
    w = np.random.default_rng(101).uniform(0.5, 2.0, len(v)).astype(np.float32)
    got = ctx.pixel_map(v, w, nside)
    p = oracle.healpix_ang2pix_ring(nside, v)
    ref = np.bincount(p, weights=w.astype(np.float64), minlength=12 * nside * nside)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-9)
    counts = ctx.pixel_map(v, None, nside)
    assert counts.sum() == len(v)
    assert np.array_equal(counts, np.bincount(p, minlength=12 * nside * nside).astype(np.float64))


@pytest.mark.parametrize("nside", [1, 16, 2048])
def test_pixel_centres_match_oracle_and_round_trip(ctx, nside):
    npix = 12 * nside * nside
    pix = np.unique(np.random.default_rng(102).integers(0, npix, 50_000))
    pix = np.concatenate([[0, npix - 1], pix]) if npix > 2 else np.arange(npix)
    c = ctx.pixel_centres(nside, pix)
    # the oracle places centres through the HEALPix projection, the library
    # by the ring formulas: the two roundings differ by a few ulp
    np.testing.assert_allclose(c, oracle.healpix_pix2vec_ring(nside, pix), rtol=0, atol=4e-15)
    m = ctx.pixel_map(c, None, nside)  # every centre falls in its own pixel
    assert np.array_equal(np.nonzero(m)[0], np.unique(pix))
    with pytest.raises(cute.CuteError):
        ctx.pixel_centres(nside, np.array([npix], dtype=np.int64))
    with pytest.raises(cute.CuteError):
        ctx.pixel_map(2.0 * c[:10], None, nside)  # not unit vectors


def test_pixel_weighted_angular_count(ctx):
    """w_pix: pixelise a cap catalog (device tensors), correlate the occupied
    pixels weighted by their counts; equals the oracle's weighted count of
    the oracle's pixel centres with the oracle's counts."""
    w = synthetic.c3_angular(scale=0.01)
    nside = 512
    theta = np.array([0.2, 0.3, 0.5, 0.8, 1.2, 2.0, 3.0, 5.0])
    chord = oracle.theta_to_chord(theta)
    m = ctx.pixel_map(torch.from_numpy(w.data).cuda(), None, nside)
    pix = torch.nonzero(m).view(-1)
    cen = ctx.pixel_centres(nside, pix)
    wt = m[pix].to(torch.float32)
    P = ctx.upload(cen, weights=wt)
    ctx.grid([P], [chord[-1]] * 3)
    c, _, ws = ctx.count("theta", P, None, chord, weighted=True)
    p_ref = oracle.healpix_ang2pix_ring(nside, w.data)
    occ, cnt = np.unique(p_ref, return_counts=True)
    assert np.array_equal(pix.cpu().numpy(), occ)
    cen_ref = oracle.healpix_pix2vec_ring(nside, occ)
    rc, _, rws = oracle.count("theta", cen_ref, edges0=chord, wa=cnt.astype(np.float32),
                              weighted=True)
    assert c.tolist() == rc.tolist()
    np.testing.assert_allclose(ws, rws, rtol=1e-9)
    P.free()

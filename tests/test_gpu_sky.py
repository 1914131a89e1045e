"""Sky coordinates on the GPU (cute_sky_to_xyz): comoving positions
chi(z) n from (RA, Dec, z) for a user cosmology (Sec. 2.1), unit vectors for
the angular measure (Sec. 3.4.2), against the oracle's adaptive quadrature,
and an (r, mu) count of a light cone given in sky coordinates."""
import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import cute

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cute.Context(0)
    yield c
    c.close()


def _sky(n, seed, zmax=3.0):
    rng = np.random.default_rng(seed)
    ra = rng.uniform(0, 360, n)
    dec = np.degrees(np.arcsin(rng.uniform(-1, 1, n)))
    z = rng.uniform(0, zmax, n)
    z[:3] = [0.0, zmax, 1e-6]
    return ra, dec, z


@pytest.mark.parametrize("cosmo", [(0.3, 0.7, -1.0), (0.25, 0.7, -0.9), (1.0, 0.0, -1.0),
                                   (0.3, 0.0, -1.0)])
def test_sky_to_xyz_matches_oracle(ctx, cosmo):
    ra, dec, z = _sky(5000, 90)
    got = ctx.sky_to_xyz(ra, dec, z, *cosmo)
    ref = oracle.sky_to_xyz(ra, dec, z, *cosmo)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-9)


def test_unit_vectors_and_device_arrays(ctx):
    ra, dec, z = _sky(4000, 91)
    got = ctx.sky_to_xyz(ra, dec)
    np.testing.assert_allclose(got, oracle.sky_to_xyz(ra, dec), rtol=0, atol=1e-15)
    t = [torch.from_numpy(a).cuda() for a in (ra, dec, z)]
    gd = ctx.sky_to_xyz(*t)
    assert gd.is_cuda and gd.shape == (4000, 3)
    np.testing.assert_array_equal(gd.cpu().numpy(), ctx.sky_to_xyz(ra, dec, z))


def test_bad_redshift_and_mixed_memory_rejected(ctx):
    ra, dec, z = _sky(100, 92)
    for bad in (25.0, -0.1, np.nan):
        zz = z.copy()
        zz[7] = bad
        with pytest.raises(cute.CuteError):
            ctx.sky_to_xyz(ra, dec, zz)
    with pytest.raises(cute.CuteError):
        ctx.sky_to_xyz(ra, dec, z, omega_m=-0.1)
    # device angles with a host output are refused before any launch
    r = torch.from_numpy(ra).cuda()
    out = np.zeros((100, 3))
    d = np.ascontiguousarray(dec)
    st = cute.lib().cute_sky_to_xyz(ctx.handle, cute._ptr(r), cute._ptr(d), None, 100, None,
                                    cute._ptr(out))
    assert st == -1  # CUTE_E_INVALID


def test_rmu_count_of_a_sky_catalog(ctx):
    """A small light cone given as (RA, Dec, z): the library's positions and
    (r, mu) counts equal the oracle's positions and counts."""
    rng = np.random.default_rng(93)
    n = 3000
    ra = rng.uniform(0, 20, n)
    dec = rng.uniform(0, 15, n)
    z = rng.uniform(0.3, 0.4, n)
    xyz = ctx.sky_to_xyz(ra, dec, z, 0.31, 0.69)
    ref_xyz = oracle.sky_to_xyz(ra, dec, z, 0.31, 0.69)
    np.testing.assert_allclose(xyz, ref_xyz, rtol=1e-12)
    e0 = np.arange(21) * 5.0
    e1 = np.linspace(0, 1, 11)
    D = ctx.upload(xyz)
    ctx.grid([D], [e0[-1]] * 3)
    got, _, _ = ctx.count("rmu", D, None, e0, e1)
    ref, _, _ = oracle.count("rmu", ref_xyz, edges0=e0, edges1=e1)
    assert got.tolist() == ref.tolist()
    D.free()

"""FP64 CPU oracle for pair counting -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` /
``--impl reference`` legs may import this package.  It shares no code with
the CUDA library and never imports it.  The pair counts, gradient rows and
estimators live in oracle.c (plain C, FP64, compiled with gcc) and are
marshalled here; the multipoles, comoving distances, HEALPix pixels, TSC
density grid and lag correlations are plain numpy/scipy below.

Every function cites the passage of Alonso (2012) it follows; see oracle.c
for the canonical formulas and the readings taken where the paper is silent.
"""
import ctypes

import numpy as np

from . import _build

KINDS = {"mono": 0, "rmu": 1, "sigpi": 2, "theta": 3}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.oracle_count.argtypes = [i32, i32, f64, P, i64, P, i64, i32, P, i32, P, i32,
                                   P, P, P, P, P, i32]
        L.oracle_count_cells.argtypes = [i32, i32, f64, P, i64, P, i64, i32, P, i32, P,
                                         i32, P, P, P, P, P, P, i32]
        L.oracle_grad_rows.argtypes = [i32, i32, f64, P, i64, P, i64, i32, P, i32, P, i32,
                                       P, P, P, i64, P, i32]
        L.oracle_xi_periodic.argtypes = [P, i64, P, i32, f64, P]
        L.oracle_xi_natural.argtypes = [P, P, i64, i64, i32, P]
        L.oracle_xi_ls.argtypes = [P, P, P, i64, i64, i32, P]
        L.oracle_theta_to_chord.argtypes = [P, i32, P]
        for f in ("oracle_count", "oracle_count_cells", "oracle_grad_rows",
                  "oracle_xi_periodic", "oracle_xi_natural", "oracle_xi_ls",
                  "oracle_theta_to_chord", "oracle_max_threads"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _xyz(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 2 or x.shape[1] != 3:
        raise ValueError("positions must be an (n, 3) array")
    return x


def _edges(e):
    return None if e is None else np.ascontiguousarray(e, dtype=np.float64)


def _w(w):
    return None if w is None else np.ascontiguousarray(w, dtype=np.float32)


def max_threads() -> int:
    return lib().oracle_max_threads()


def count(kind, xa, xb=None, edges0=None, edges1=None, periodic=False, L=0.0,
          wa=None, wb=None, weighted=False, cells=None, nthreads=0):
    """Pair-count histogram (Eq. 11; serial loop of Sec. 3.1).

    kind: 'mono' | 'rmu' | 'sigpi' | 'theta'.  xb None -> auto-correlation
    (unique pairs i<j of xa); else cross-correlation (all xa x xb).
    cells: None -> brute force over every pair; a 3-vector of per-axis reach
    -> the cell-pruned form (Sec. 3.3), identical counts.
    Returns (counts[n0, n1] uint64, oor, wsum or None)."""
    k = KINDS[kind]
    xa = _xyz(xa)
    is_auto = xb is None
    xb = xa if is_auto else _xyz(xb)
    e0 = _edges(edges0)
    e1 = _edges(edges1)
    n0 = len(e0) - 1
    n1 = (len(e1) - 1) if k in (1, 2) else 1
    wa_, wb_ = _w(wa), _w(wb)
    if weighted and is_auto:
        wb_ = wa_
    counts = np.zeros(n0 * n1, dtype=np.uint64)
    oor = np.zeros(1, dtype=np.uint64)
    wsum = np.zeros(n0 * n1, dtype=np.float64) if weighted else None
    if cells is None:
        rc = lib().oracle_count(k, int(periodic), float(L), _ptr(xa), len(xa), _ptr(xb), len(xb),
                                int(is_auto), _ptr(e0), n0, _ptr(e1), n1 if k in (1, 2) else 0,
                                _ptr(wa_), _ptr(wb_), _ptr(counts), _ptr(oor), _ptr(wsum),
                                int(nthreads))
    else:
        reach = np.ascontiguousarray(cells, dtype=np.float64)
        rc = lib().oracle_count_cells(k, int(periodic), float(L), _ptr(xa), len(xa), _ptr(xb),
                                      len(xb), int(is_auto), _ptr(e0), n0, _ptr(e1),
                                      n1 if k in (1, 2) else 0, _ptr(wa_), _ptr(wb_),
                                      _ptr(reach), _ptr(counts), _ptr(oor), _ptr(wsum),
                                      int(nthreads))
    if rc != 0:
        raise ValueError("oracle_count failed with status %d" % rc)
    return counts.reshape(n0, n1), int(oor[0]), (None if wsum is None else wsum.reshape(n0, n1))


def grad_rows(kind, xa, rows, G, wpartner, xb=None, edges0=None, edges1=None,
              periodic=False, L=0.0, nthreads=0):
    """d/dw_i of sum_b G_b W_b for the rows i of catalog A (weighted counts of
    Sec. 3.4): sum over partners j of w_j G[bin(i, j)]."""
    k = KINDS[kind]
    xa = _xyz(xa)
    is_auto = xb is None
    xb = xa if is_auto else _xyz(xb)
    e0, e1 = _edges(edges0), _edges(edges1)
    n0 = len(e0) - 1
    n1 = (len(e1) - 1) if k in (1, 2) else 0
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    G = np.ascontiguousarray(G, dtype=np.float64).ravel()
    wp = _w(wpartner)
    out = np.zeros(len(rows), dtype=np.float64)
    rc = lib().oracle_grad_rows(k, int(periodic), float(L), _ptr(xa), len(xa), _ptr(xb), len(xb),
                                int(is_auto), _ptr(e0), n0, _ptr(e1), n1, _ptr(wp), _ptr(G),
                                _ptr(rows), len(rows), _ptr(out), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_grad_rows failed with status %d" % rc)
    return out


def xi_periodic(DD, N, edges, L):
    """Eq. 13 with N(N-1)/2 unique pairs and the exact shell volume."""
    DD = np.ascontiguousarray(DD, dtype=np.uint64).ravel()
    e = _edges(edges)
    out = np.zeros(len(DD), dtype=np.float64)
    rc = lib().oracle_xi_periodic(_ptr(DD), int(N), _ptr(e), len(DD), float(L), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_xi_periodic failed")
    return out


def xi_natural(DD, RR, Nd, Nr):
    """Eq. 14."""
    DD = np.ascontiguousarray(DD, dtype=np.uint64).ravel()
    RR = np.ascontiguousarray(RR, dtype=np.uint64).ravel()
    out = np.zeros(len(DD), dtype=np.float64)
    rc = lib().oracle_xi_natural(_ptr(DD), _ptr(RR), int(Nd), int(Nr), len(DD), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_xi_natural failed")
    return out


def xi_ls(DD, DR, RR, Nd, Nr):
    """Eq. 15 (Landy-Szalay)."""
    DD = np.ascontiguousarray(DD, dtype=np.uint64).ravel()
    DR = np.ascontiguousarray(DR, dtype=np.uint64).ravel()
    RR = np.ascontiguousarray(RR, dtype=np.uint64).ravel()
    out = np.zeros(len(DD), dtype=np.float64)
    rc = lib().oracle_xi_ls(_ptr(DD), _ptr(DR), _ptr(RR), int(Nd), int(Nr), len(DD), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_xi_ls failed")
    return out


def theta_to_chord(theta_deg):
    """Chord 2 sin(theta/2) between unit vectors at angle theta (Eq. 7)."""
    t = np.ascontiguousarray(theta_deg, dtype=np.float64)
    out = np.zeros(len(t), dtype=np.float64)
    rc = lib().oracle_theta_to_chord(_ptr(t), len(t), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_theta_to_chord failed")
    return out


def multipoles(xi, mu_edges, ells=(0, 2, 4)):
    """Even multipoles of a binned xi(r, mu), Sec. 2.1 Eq. 3 (xi(r, mu) =
    sum_l xi_l(r) P_l(mu)) inverted by the orthogonality of the Legendre
    polynomials: xi_l(r) = (2l + 1)/2 * integral_{-1}^{1} xi P_l dmu, which
    for xi even in mu (mu = |cos|) is (2l + 1) * integral_0^1 xi P_l dmu;
    xi is constant within each mu bin, and P_l is integrated exactly over
    each bin with numpy's Legendre-series antiderivative.  l = 0 is Eq. 4."""
    from numpy.polynomial import legendre
    xi = np.asarray(xi, dtype=np.float64)
    m = np.asarray(mu_edges, dtype=np.float64)
    out = np.zeros((len(ells), xi.shape[0]))
    for q, l in enumerate(ells):
        anti = legendre.Legendre.basis(l).integ()
        w = (2 * l + 1) * (anti(m[1:]) - anti(m[:-1]))
        out[q] = xi @ w
    return out


C_OVER_H0 = 2997.92458  # c / H0 in Mpc/h


def comoving_distance(z, omega_m, omega_l, w0=-1.0):
    """Radial comoving distance chi(z) of Sec. 2.1 in Mpc/h: (c/H0) times the
    integral of 1/E from 0 to z, E^2 = Om (1+z)^3 + Ok (1+z)^2 + OL (1+z)^(3(1+w)),
    Ok = 1 - Om - OL; integrated with scipy's adaptive quadrature between
    consecutive sorted redshifts."""
    from scipy.integrate import quad
    z = np.asarray(z, dtype=np.float64)
    ok = 1.0 - omega_m - omega_l

    def inv_e(x):
        a = 1.0 + x
        return 1.0 / np.sqrt(omega_m * a ** 3 + ok * a ** 2 + omega_l * a ** (3.0 * (1.0 + w0)))

    order = np.argsort(z, kind="stable")
    out = np.empty_like(z)
    acc, prev = 0.0, 0.0
    for i in order:
        if z[i] > prev:
            acc += quad(inv_e, prev, z[i], epsabs=1e-15, epsrel=1e-13, limit=200)[0]
            prev = z[i]
        out[i] = C_OVER_H0 * acc
    return out


def sky_to_xyz(ra_deg, dec_deg, z=None, omega_m=0.3, omega_l=0.7, w0=-1.0):
    """Positions chi(z) n from (RA, Dec) in degrees and redshifts (None: the
    unit vectors n of the projection onto the unit sphere, Sec. 3.4.2),
    n = (cos dec cos ra, cos dec sin ra, sin dec)."""
    ra = np.radians(np.asarray(ra_deg, dtype=np.float64))
    dec = np.radians(np.asarray(dec_deg, dtype=np.float64))
    n = np.stack([np.cos(dec) * np.cos(ra), np.cos(dec) * np.sin(ra), np.sin(dec)], axis=1)
    if z is None:
        return n
    return n * comoving_distance(z, omega_m, omega_l, w0)[:, None]


# HEALPix (Gorski et al. 2005) through its planar projection (Calabretta &
# Roukema 2007): with X = phi / (pi/4) and, in the equatorial belt
# |z| <= 2/3, Y = 3 z / 2, or in the polar caps Y = +-(2 - sigma),
# sigma = sqrt(3 (1 - |z|)), X pulled towards the centre X_f of its
# quadrant by the factor sigma, the sphere maps onto 12 squares (diamonds)
# and every pixel boundary onto one of the lines X + Y = 1 + 2k/nside,
# X - Y = 1 + 2k/nside.  A point's pixel is then its cell (a, b) of that
# lattice; the cell's centre sits at X_c = 1 + (a + b + 1)/nside,
# Y_c = (a - b)/nside, on ring i = 2 nside - (a - b) (ring latitudes
# Y_i = 2 - i/nside), and the RING index counts the rings above it and the
# centres of its own ring with phi in [0, 2 pi) below its own (Gorski et al.
# 2005: polar ring i holds 4i centres at phi = (j + 1/2) pi/(2i); belt rings
# 4 nside centres, spaced pi/(2 nside), starting at phi = pi/(4 nside) when
# i - nside is even and at phi = 0 when it is odd).
def _hp_project(xyz):
    """(X, Y) of unit vectors in the HEALPix projection, and the quadrant q
    (0..3) of each point's phi."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    phi = np.mod(np.arctan2(y, x), 2 * np.pi)
    X = phi / (np.pi / 4)
    X = np.where(X >= 8.0, 0.0, X)
    q = np.minimum(np.floor(X / 2).astype(np.int64), 3)
    za = np.abs(z)
    polar = za > 2.0 / 3.0
    sigma = np.sqrt(3.0 * (1.0 - np.where(polar, za, 1.0)))
    Xf = 2.0 * q + 1.0
    Xp = np.where(polar, Xf + (X - Xf) * sigma, X)
    Yp = np.where(polar, np.sign(z) * (2.0 - sigma), 1.5 * z)
    return Xp, Yp, q


def healpix_ang2pix_ring(nside, xyz):
    """Pixel index (HEALPix RING scheme) of unit vectors, the pixelisation
    taken for the pixel maps of Sec. 3.4.2: the lattice cell of the point in
    the HEALPix projection, then its ring and its rank on the ring."""
    xyz = np.asarray(xyz, dtype=np.float64)
    N = int(nside)
    X, Y, q = _hp_project(xyz)
    a = np.floor((X + Y - 1.0) * N / 2.0).astype(np.int64)
    b = np.floor((X - Y - 1.0) * N / 2.0).astype(np.int64)
    i = 2 * N - (a - b)                      # ring of the cell's centre, 1 .. 4N-1
    out = np.empty(len(X), dtype=np.int64)
    north, south = i < N, i > 3 * N
    belt = ~(north | south)
    # polar rings: the centre's offset from its quadrant's face centre,
    # u = X_c - X_f = (a + b + 1 - 2 q N)/N, ranks it among the quadrant's
    # i centres (spaced 2/N around X_f)
    for sel, ring, before in ((north, i, lambda r: 2 * r * (r - 1)),
                              (south, 4 * N - i, lambda r: 12 * N * N - 2 * r * (r + 1))):
        r, qs = ring[sel], q[sel]
        m = qs * r + (r + a[sel] + b[sel] - 2 * qs * N) // 2
        out[sel] = before(r) + m
    # belt rings: centres spaced 2/N in X; rank = floor(X_c N / 2) with
    # X_c N / 2 = (N + a + b + 1) / 2 taken modulo 4N (phi in [0, 2 pi))
    ib = i[belt]
    rank = np.mod((N + a[belt] + b[belt] + 1) // 2, 4 * N)
    out[belt] = 2 * N * (N - 1) + 4 * N * (ib - N) + rank
    return out


def healpix_pix2vec_ring(nside, pix):
    """Centres of HEALPix RING pixels as unit vectors: the ring found among
    the rings' first indices, the centre placed in the HEALPix projection
    (Y_i = 2 - i/nside; X spaced 2/nside), then mapped back to the sphere."""
    N = int(nside)
    p = np.asarray(pix, dtype=np.int64)
    rings = np.arange(1, 4 * N)
    size = 4 * np.minimum(np.minimum(rings, 4 * N - rings), N)
    first = np.concatenate([[0], np.cumsum(size)[:-1]])
    k = np.searchsorted(first, p, side="right") - 1
    i, m = rings[k], p - first[k]
    Yc = 2.0 - i / N
    Xc = np.empty(len(p))
    polar = (i < N) | (i > 3 * N)
    r = np.where(i < N, i, 4 * N - i)[polar]
    q = m[polar] // r
    Xc[polar] = 2.0 * q + 1.0 + (2.0 * (m[polar] - q * r) - r + 1.0) / N
    # belt: first centre at X = 1/N when i - N is even, at X = 0 when odd
    ib = i[~polar]
    half = 1.0 - np.mod(ib - N, 2)
    Xc[~polar] = (2.0 * m[~polar] + half) / N
    z = np.empty(len(p))
    phi = np.empty(len(p))
    z[~polar] = Yc[~polar] / 1.5
    phi[~polar] = Xc[~polar] * (np.pi / 4)
    sig = 2.0 - np.abs(Yc[polar])
    z[polar] = np.sign(Yc[polar]) * (1.0 - sig * sig / 3.0)
    Xf = 2.0 * q + 1.0
    phi[polar] = (Xf + (Xc[polar] - Xf) / sig) * (np.pi / 4)
    st = np.sqrt((1.0 - z) * (1.0 + z))
    return np.stack([st * np.cos(phi), st * np.sin(phi), z], axis=1)


def xi_weighted(kind, DD, DR, RR, s_d, q_d, s_r, q_r):
    """Eq. 14 / Eq. 15 on weighted pair sums: DD over the total data-data
    pair weight (S_d^2 - Q_d)/2, DR over S_d S_r, RR over (S_r^2 - Q_r)/2."""
    DD = np.asarray(DD, dtype=np.float64)
    RR = np.asarray(RR, dtype=np.float64)
    dd = DD / (0.5 * (s_d * s_d - q_d))
    rr = RR / (0.5 * (s_r * s_r - q_r))
    with np.errstate(divide="ignore", invalid="ignore"):
        if kind == "natural":
            out = dd / rr - 1.0
        else:
            dr = np.asarray(DR, dtype=np.float64) / (s_d * s_r)
            out = (dd - 2.0 * dr + rr) / rr
    return np.where(RR != 0, out, np.nan)


def tsc_density(xyz, L, n, w=None):
    """Triangular-shaped-cloud interpolation of a periodic catalog to an n^3
    grid (Sec. 3.4.4), grid points at multiples of a = L/n: along each axis
    the nearest point i0 = rint(x/a) takes 3/4 - d^2 and its neighbours
    (1/2 -+ d)^2 / 2, d = x/a - i0.  Returns rho[z, y, x] (summed weights)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    wt = np.ones(len(xyz)) if w is None else np.asarray(w, dtype=np.float64)
    u = xyz / (L / n)
    i0 = np.rint(u)
    d = u - i0
    i0 = i0.astype(np.int64)
    wts = [0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2]
    rho = np.zeros((n, n, n))
    for c in range(3):
        for b in range(3):
            for a in range(3):
                ix = np.mod(i0[:, 0] + a - 1, n)
                iy = np.mod(i0[:, 1] + b - 1, n)
                iz = np.mod(i0[:, 2] + c - 1, n)
                np.add.at(rho, (iz, iy, ix), wt * wts[a][:, 0] * wts[b][:, 1] * wts[c][:, 2])
    return rho


def _lag_bins(delta, L, edges, lag_sum):
    """xi per bin from the lag sums lag_sum(dz, dy, dx) = sum_x delta(x)
    delta(x + d) over every lag vector d of the half space with a|d| below
    the last edge, binned by a^2 |d|^2 on the squared edges (half-open);
    mean over the bin's lags and the grid's points.  Returns (xi, lags)."""
    n = delta.shape[0]
    a = L / n
    e2 = np.asarray(edges, dtype=np.float64) ** 2
    nb = len(e2) - 1
    R = int(np.floor(edges[-1] / a))
    s, c = np.zeros(nb), np.zeros(nb)
    for dz in range(0, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                if (dz, dy) == (0, 0) and dx <= 0:
                    continue
                if dz == 0 and dy < 0:
                    continue
                r2 = (dx * dx + dy * dy + dz * dz) * a * a
                if r2 < e2[0] or r2 >= e2[-1]:
                    continue
                b = int(np.searchsorted(e2, r2, side="right")) - 1
                s[b] += lag_sum(dz, dy, dx)
                c[b] += 1
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(c > 0, s / (c * delta.size), np.nan), c


def lag_xi(delta, L, edges):
    """xi(r) = <delta(x) delta(x + r)> over the pairs of distinct grid points
    of a periodic grid whose separation falls in each bin (Sec. 3.4.4): for
    every lag vector d of the half space with a|d| below the last edge, the
    product sum of delta with delta shifted by d, binned by a^2 |d|^2 on the
    squared edges (half-open).  Returns (xi, lags per bin)."""
    return _lag_bins(delta, L, edges, lambda dz, dy, dx: float(
        np.sum(delta * np.roll(delta, (-dz, -dy, -dx), axis=(0, 1, 2)))))


def lag_xi_fft(delta, L, edges):
    """The same estimate as lag_xi with the lag sums taken from the circular
    autocorrelation of the grid: sum_x delta(x) delta(x + d) is the inverse
    FFT of |FFT(delta)|^2 at d (the correlation theorem; FP64, numpy's FFT
    as the library step).  For grids where the direct sums are too slow."""
    n = delta.shape[0]
    f = np.fft.rfftn(np.asarray(delta, dtype=np.float64))
    C = np.fft.irfftn(f * np.conj(f), s=delta.shape, axes=(0, 1, 2))
    del f
    return _lag_bins(delta, L, edges, lambda dz, dy, dx: float(C[dz % n, dy % n, dx % n]))


def density_grid_xi(xyz, L, n, edges, w=None):
    """Sec. 3.4.4 end to end: TSC density, delta = rho / mean(rho) - 1,
    lag-averaged delta_i delta_j per bin."""
    rho = tsc_density(xyz, L, n, w)
    return lag_xi(rho / rho.mean() - 1.0, L, edges)

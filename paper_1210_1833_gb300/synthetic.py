"""Seeded synthetic catalogs shaped like the paper's workloads.

The paper measures on a MICE light-cone subset, 600 PTHalo mocks and a
log-normal mock (Sec. 4, Figs. 5-6); none of them is available, so these
generators stand in for them.  Every catalog is FP64, drawn with
``numpy.random.default_rng(seed)`` (PCG64) and fully determined by its seed.

This module holds no pair-counting arithmetic: it only draws positions,
weights and bin edges (bin edges are plain lists of numbers; turning angles
into chords is done by each side on its own).  Both the oracle tests and the
CUDA path read their inputs from here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _wrap_box(x: np.ndarray, L: float) -> np.ndarray:
    """Map into [0, L): np.mod may return L itself for tiny negatives."""
    x = np.mod(x, L)
    x[x >= L] = 0.0
    return x


def uniform_box(n: int, L: float, rng: np.random.Generator) -> np.ndarray:
    return _wrap_box(rng.uniform(0.0, L, size=(n, 3)), L)


def blobs_box(n_blobs: int, per_blob: int, L: float, sigma, rng) -> np.ndarray:
    """Gaussian blobs at uniform centres, wrapped into the periodic box.
    sigma: scalar or per-axis (sx, sy, sz)."""
    centres = rng.uniform(0.0, L, size=(n_blobs, 3))
    pts = np.repeat(centres, per_blob, axis=0)
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (3,))
    pts = pts + rng.normal(0.0, 1.0, size=pts.shape) * sig
    return _wrap_box(pts, L)


# ---------------------------------------------------------------- sky helpers
def _radec_to_xyz(ra_deg, dec_deg, r):
    ra = np.radians(ra_deg)
    dec = np.radians(dec_deg)
    cd = np.cos(dec)
    return np.stack([r * cd * np.cos(ra), r * cd * np.sin(ra), r * np.sin(dec)], axis=1)


def _shell_r(n, r1, r2, rng):
    """Radii uniform in volume between r1 and r2."""
    u = rng.uniform(0.0, 1.0, size=n)
    return np.cbrt(r1 ** 3 + u * (r2 ** 3 - r1 ** 3))


# ---------------------------------------------------------------- configs
@dataclass
class Workload:
    name: str
    kind: str                      # 'mono' | 'rmu' | 'sigpi' | 'theta'
    periodic: bool
    L: float
    edges0: np.ndarray
    edges1: np.ndarray | None
    data: np.ndarray | None = None
    randoms: np.ndarray | None = None
    weights: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def c1_monopole_box(scale: float = 1.0) -> Workload:
    """Monopole xi(r) in a periodic cube, DD only: L = 1000, 20,000 points,
    half uniform and half in 200 Gaussian blobs (sigma = 5), seed 0;
    40 linear bins on [0, 200).  scale < 1 keeps the shape with fewer points."""
    rng = np.random.default_rng(0)
    L = 1000.0
    n_uni = int(round(10000 * scale))
    n_blob = max(1, int(round(200 * scale)))
    uni = uniform_box(10000, L, rng)[:n_uni]
    blob = blobs_box(200, 50, L, 5.0, rng)[: n_blob * 50]
    data = np.concatenate([uni, blob], axis=0)
    edges = np.arange(41, dtype=np.float64) * 5.0
    return Workload("c1_monopole_box", "mono", True, L, edges, None, data=data)


def c2_rmu_lightcone(scale: float = 1.0) -> Workload:
    """xi(r, mu) on a light-cone wedge: 500k data in 20 clustered sky patches
    and 2M uniform randoms, r in [1000, 2500], RA 0-60 deg, Dec 0-30 deg;
    40 r bins on [0, 200) x 40 mu bins on [0, 1], midpoint line of sight;
    seed 1.  scale < 1 draws proportionally fewer objects."""
    rng = np.random.default_rng(1)
    r1, r2 = 1000.0, 2500.0
    ra_max, dec_max = 60.0, 30.0
    smax = math.sin(math.radians(dec_max))
    nr = int(round(2_000_000 * scale))
    nd = int(round(500_000 * scale))
    # randoms: uniform in volume over the wedge
    ra = rng.uniform(0.0, ra_max, size=nr)
    dec = np.degrees(np.arcsin(rng.uniform(0.0, smax, size=nr)))
    rand = _radec_to_xyz(ra, dec, _shell_r(nr, r1, r2, rng))
    # data: 20 patch centres, Gaussian 2-degree offsets in the tangent plane,
    # redrawn until inside the window
    n_patch = 20
    c_ra = rng.uniform(0.0, ra_max, size=n_patch)
    c_dec = np.degrees(np.arcsin(rng.uniform(0.0, smax, size=n_patch)))
    which = rng.integers(0, n_patch, size=nd)
    d_ra = np.empty(nd)
    d_dec = np.empty(nd)
    todo = np.arange(nd)
    while todo.size:
        w = which[todo]
        eta = rng.normal(0.0, 2.0, size=todo.size)
        xi = rng.normal(0.0, 2.0, size=todo.size)
        dd = c_dec[w] + eta
        rr = c_ra[w] + xi / np.cos(np.radians(c_dec[w]))
        ok = (rr >= 0) & (rr < ra_max) & (dd >= 0) & (dd < dec_max)
        d_ra[todo[ok]] = rr[ok]
        d_dec[todo[ok]] = dd[ok]
        todo = todo[~ok]
    data = _radec_to_xyz(d_ra, d_dec, _shell_r(nd, r1, r2, rng))
    e0 = np.arange(41, dtype=np.float64) * 5.0
    e1 = np.arange(41, dtype=np.float64) / 40.0
    return Workload("c2_rmu_lightcone", "rmu", False, 0.0, e0, e1, data=data, randoms=rand)


def _cap_cos_alpha() -> float:
    # 1 - cos(alpha) = area / (2 pi), area = 1000 square degrees
    return 1.0 - 1000.0 * (math.pi / 180.0) ** 2 / (2.0 * math.pi)


def _cap_uniform(n, cos_a, rng):
    z = rng.uniform(cos_a, 1.0, size=n)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def c3_angular(scale: float = 1.0) -> Workload:
    """w(theta) on a 1000 sq-deg cap about +z: 5M data (99% uniform, 1% in
    500 clumps of 100 at 0.05 deg) and 20M uniform randoms, unit vectors;
    64 log theta bins on 0.01-10 deg (edges in degrees in extra['theta_deg']);
    seed 2.  The chord edges are left to each consumer."""
    rng = np.random.default_rng(2)
    cos_a = _cap_cos_alpha()
    nr = int(round(20_000_000 * scale))
    nd = int(round(5_000_000 * scale))
    n_clump_pts = int(round(50_000 * scale))
    n_clumps = max(1, n_clump_pts // 100)
    n_clump_pts = n_clumps * 100
    rand = _cap_uniform(nr, cos_a, rng)
    uni = _cap_uniform(nd - n_clump_pts, cos_a, rng)
    centres = _cap_uniform(n_clumps, cos_a, rng)
    pts = np.repeat(centres, 100, axis=0)
    todo = np.arange(len(pts))
    out = np.empty_like(pts)
    sig = math.radians(0.05)
    while todo.size:
        c = pts[todo]
        # tangent basis at each centre
        ref = np.where(np.abs(c[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
        t1 = np.cross(c, ref)
        t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
        t2 = np.cross(c, t1)
        a = rng.normal(0.0, sig, size=(todo.size, 1))
        b = rng.normal(0.0, sig, size=(todo.size, 1))
        v = c + a * t1 + b * t2
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        ok = v[:, 2] >= cos_a
        out[todo[ok]] = v[ok]
        todo = todo[~ok]
    data = np.concatenate([uni, out], axis=0)
    theta = 10.0 ** (-2.0 + 3.0 * np.arange(65, dtype=np.float64) / 64.0)
    return Workload("c3_angular", "theta", False, 0.0, None, None, data=data, randoms=rand,
                    extra={"theta_deg": theta})


def c4_batched_sigpi(n_boxes: int = 64, scale: float = 1.0) -> list[Workload]:
    """64 periodic boxes (L = 1500) of uneven N ~ log-uniform in 50k-400k, half
    uniform and half in N/100 blobs (sigma_xy = 5, sigma_z = 10), each with
    2N uniform randoms; 50 sigma x 50 pi linear bins to 150; seed 3."""
    rng = np.random.default_rng(3)
    L = 1500.0
    Ns = np.floor(np.exp(rng.uniform(math.log(5e4), math.log(4e5), size=64))).astype(np.int64)
    out = []
    e = np.arange(51, dtype=np.float64) * 3.0
    for k in range(64):
        n = int(Ns[k])
        n_uni = n - n // 2
        n_bl = max(1, n // 100)
        per = (n // 2) // n_bl
        uni = uniform_box(n_uni, L, rng)
        bl = blobs_box(n_bl, max(per, 1), L, (5.0, 5.0, 10.0), rng)
        data = np.concatenate([uni, bl], axis=0)
        rand = uniform_box(2 * n, L, rng)
        if k < n_boxes:
            if scale < 1.0:
                data = data[: max(2, int(len(data) * scale))]
                rand = rand[: max(2, int(len(rand) * scale))]
            out.append(Workload("c4_box%02d" % k, "sigpi", True, L, e, e.copy(), data=data,
                                randoms=rand))
    return out


def c5_weighted(scale: float = 1.0) -> Workload:
    """Weighted DD and adjoint: periodic cube L = 2000, 4M points (half
    uniform, half in 20,000 blobs x 100, sigma = 5), FP32 weights
    exp(0.3 N(0,1)); 30 bins on [0, 150); upstream G_b ~ N(0,1) (seed 5);
    1,000 sampled weights for the finite-difference check (seed 6); seed 4."""
    rng = np.random.default_rng(4)
    L = 2000.0
    n = int(round(4_000_000 * scale))
    n_bl = max(1, int(round(20_000 * scale)))
    uni = uniform_box(n - n_bl * 100, L, rng)
    bl = blobs_box(n_bl, 100, L, 5.0, rng)
    data = np.concatenate([uni, bl], axis=0)
    w = np.exp(0.3 * rng.normal(0.0, 1.0, size=len(data))).astype(np.float32)
    edges = np.arange(31, dtype=np.float64) * 5.0
    G = np.random.default_rng(5).normal(0.0, 1.0, size=30)
    fd_idx = np.random.default_rng(6).choice(len(data), size=min(1000, len(data)), replace=False)
    return Workload("c5_weighted", "mono", True, L, edges, None, data=data, weights=w,
                    extra={"G": G, "fd_idx": np.sort(fd_idx)})


def subsample(x: np.ndarray, n: int, seed: int) -> np.ndarray:
    """Seeded subset of rows (without replacement), order preserved."""
    if n >= len(x):
        return x
    idx = np.sort(np.random.default_rng(seed).choice(len(x), size=n, replace=False))
    return x[idx]

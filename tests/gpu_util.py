"""Helpers shared by the GPU parity tests: run one count through the C-ABI
library and the same count through the FP64 oracle."""
import math

import numpy as np

import oracle


def reach_of(kind, e0, e1):
    if kind == "sigpi":
        return [e0[-1], e0[-1], e1[-1]]
    return [e0[-1]] * 3


def gpu_count(ctx, kind, a, b=None, e0=None, e1=None, periodic=False, L=0.0, cells_per_reach=2,
              wa=None, wb=None, weighted=False):
    ca = ctx.upload(a, weights=wa, periodic=periodic, L=L)
    cb = ctx.upload(b, weights=wb, periodic=periodic, L=L) if b is not None else None
    ctx.grid([ca] + ([cb] if cb is not None else []), reach_of(kind, e0, e1), cells_per_reach)
    try:
        return ctx.count(kind, ca, cb, e0, e1, weighted=weighted)
    finally:
        ca.free()
        if cb is not None:
            cb.free()


def oracle_count(kind, a, b=None, e0=None, e1=None, periodic=False, L=0.0, cells=False, wa=None,
                 wb=None, weighted=False):
    return oracle.count(kind, a, b, edges0=e0, edges1=e1 if kind in ("rmu", "sigpi") else None,
                        periodic=periodic, L=L, wa=wa, wb=wb, weighted=weighted,
                        cells=reach_of(kind, e0, e1) if cells else None)


def edge_pairs_mono(rng, edges, n_per_edge, box=None, scale_eps=(0.0, 2.0**-40, -2.0**-40,
                                                                   2.0**-36, -2.0**-36, 2.0**-34,
                                                                   -2.0**-34, 2.0**-30, -2.0**-30,
                                                                   2.0**-22, -2.0**-22)):
    """Points placed in pairs whose separations sit exactly on (or within a
    hair of) every bin edge: the pairs the FP32 path must hand to the
    re-test, on both sides of the double-float stage's margin (about 2^-36
    relative) and of the FP32 error band."""
    pts = []
    for e in edges:
        if e <= 0:
            continue
        for _ in range(n_per_edge):
            for d in scale_eps:
                u = rng.normal(size=3)
                u /= np.linalg.norm(u)
                c = rng.uniform(0.3, 0.7, size=3) * (box if box else 100.0)
                pts.append(c)
                pts.append(c + u * e * (1.0 + d))
    x = np.array(pts)
    if box:
        x = np.mod(x, box)
        x[x >= box] = 0.0
    return x


def edge_pairs_mu(rng, mu_edges, r, n_per_edge, dist=1500.0):
    """Pairs at separation r whose midpoint-line-of-sight cosine is (almost)
    exactly a mu edge."""
    pts = []
    for m in mu_edges:
        for _ in range(n_per_edge):
            for d in (0.0, 2.0**-40, -2.0**-40, 2.0**-36, -2.0**-36, 2.0**-33, -2.0**-33,
                      2.0**-28, -2.0**-28):
                xi = rng.normal(size=3)
                xi = xi / np.linalg.norm(xi) * dist
                t = rng.normal(size=3)
                mm = min(max(m * (1 + d), 0.0), 1.0)
                s = np.zeros(3)
                for _ in range(8):  # fixed point: direction relative to l = 2 x_i + s
                    lh = (2 * xi + s) / np.linalg.norm(2 * xi + s)
                    tt = t - np.dot(t, lh) * lh
                    tt /= np.linalg.norm(tt)
                    s = r * (mm * lh + math.sqrt(max(0.0, 1 - mm * mm)) * tt)
                pts.append(xi)
                pts.append(xi + s)
    return np.array(pts)

"""Splitting pair counts across ranks (one process per GPU).

The path partitions into independent units: the home objects of a count, or
whole catalogs of a batch.  Two forms:

* ``batch_share``: catalogs of a batch dealt round-robin to ranks; each rank
  counts its own, with no exchange (weak scaling).
* ``sharded_auto``: one auto-correlation split by home rows.  Each rank
  counts its rows A_k against the whole catalog A (a cross count), the
  histograms are summed once across ranks (the single exchange step), and
  unique pairs follow as (sum - self pairs) / 2, since every unordered pair
  {i, j} is met twice, from i and from j, and every object meets itself
  once at separation 0.

The counting itself is a callable so the same logic serves the GPU library
and, in tests, the CPU oracle.
"""
from __future__ import annotations

import numpy as np


def row_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced [lo, hi) block of n rows for this rank."""
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def batch_share(n_items: int, rank: int, world: int) -> list[int]:
    """Items of a batch owned by this rank (round-robin)."""
    return list(range(rank, n_items, world))


def sharded_auto(cross_count, x: np.ndarray, rank: int, world: int, self_bin, allreduce):
    """Unique-pair auto-count of x from per-rank cross counts.

    cross_count(xs, x) -> uint64 histogram of the rows xs against all of x.
    self_bin: flat index of the bin separation 0 falls in, or None.
    allreduce(np.ndarray int64) -> elementwise sum over ranks."""
    lo, hi = row_range(len(x), rank, world)
    part = np.asarray(cross_count(x[lo:hi], x), dtype=np.uint64).astype(np.int64)
    shape = part.shape
    tot = allreduce(part.ravel().copy()).reshape(shape)
    if self_bin is not None:
        tot.ravel()[self_bin] -= len(x)
    if np.any(tot % 2):
        raise ArithmeticError("ordered pair counts must be even")
    return (tot // 2).astype(np.uint64)

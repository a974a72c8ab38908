"""Spatial decomposition of the sectored timestep over ranks (Sec. 5.1).

The paper's parallel scheme gives each process a subdomain, sweeps the
colours in the same order everywhere, and exchanges ghost spins before each
colour's pass (and positions once per step).  This module is the host-side
plan of that scheme for slabs along x:

* ``slab_bounds``: contiguous ranges of sector columns, at least two sectors
  wide, one per rank (sectors of one colour stay out of interaction range of
  each other however the columns are cut, because the colouring is global);
* ``owners``: the rank owning each atom (by its sector column);
* ``halo_plan``: for every ordered pair of ranks (src, dst), the atoms src
  owns that lie within ``reach`` of dst's slab (periodic in x), split by
  colour, so that after colour c's pass src sends dst only the spins that
  pass turned; positions go once per step, after the drift.

Nothing here computes any part of the method; it only partitions atom ids.
"""
from __future__ import annotations

import numpy as np


def slab_bounds(nsec_x: int, ranks: int):
    """[(x0, x1)] sector-column ranges, one per rank, as even as possible,
    each at least two columns wide (ValueError otherwise)."""
    if ranks < 1 or nsec_x < 2 * ranks:
        raise ValueError(f"{nsec_x} sector columns cannot give {ranks} slabs of at least two")
    cuts = [(k * nsec_x) // ranks for k in range(ranks + 1)]
    return [(cuts[k], cuts[k + 1]) for k in range(ranks)]


def owners(sector_x, bounds):
    """Rank of each atom from its sector column."""
    sector_x = np.asarray(sector_x)
    own = np.full(sector_x.shape, -1, dtype=np.int64)
    for k, (a, b) in enumerate(bounds):
        own[(sector_x >= a) & (sector_x < b)] = k
    if (own < 0).any():
        raise ValueError("a sector column outside every slab")
    return own


def _distance_to_slab(x, lo, hi, L):
    """Periodic distance of coordinates x to the interval [lo, hi) of a ring
    of length L (0 inside)."""
    x = np.mod(np.asarray(x, dtype=np.float64) - lo, L)      # slab starts at 0
    w = hi - lo
    inside = x < w
    return np.where(inside, 0.0, np.minimum(x - w, L - x))


def halo_plan(x, colour, own, bounds, edge_x, L, reach):
    """{(src, dst): {c: ids}}: atoms of src within `reach` of dst's slab, by
    colour c, ids ascending.  x: the atoms' x coordinates (wrapped or not),
    colour: their colours, own: their ranks, bounds: slab sector columns,
    edge_x: sector edge along x, L: box length along x."""
    x = np.asarray(x, dtype=np.float64)
    colour = np.asarray(colour)
    plan = {}
    for dst, (a, b) in enumerate(bounds):
        d = _distance_to_slab(x, a * edge_x, b * edge_x, L)
        near = d < reach
        for src in range(len(bounds)):
            if src == dst:
                continue
            sel = near & (own == src)
            plan[(src, dst)] = {c: np.flatnonzero(sel & (colour == c)) for c in range(8)}
    return plan


def halo_ids(plan, src, dst):
    """All atoms src sends dst (every colour), ascending."""
    parts = [v for v in plan[(src, dst)].values() if len(v)]
    return np.sort(np.concatenate(parts)) if parts else np.zeros(0, dtype=np.int64)

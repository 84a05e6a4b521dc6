"""Line sharding of one surface across ranks (one GPU per rank).

The micromagnetic lines are independent walks (the paper's central point, and
its cost estimate of the full surface as a sum over lines), so a surface is
split by lines: each rank walks a share of the lines l = 0..N/2 chosen by
longest-processing-time-first on an estimated cost, and the assembled ln g of
every line is gathered on one rank at the end.  The gather is the only
exchange; nothing crosses ranks while the walks run.

The estimated cost of a line is its number of bins squared (a flat-histogram
walk over n bins needs of order n^2 moves per stage).
"""
from __future__ import annotations

import heapq

import numpy as np


def line_bins(N: int, NB: int, z: int, kstep: int, ell: int) -> int:
    """Bins of line l: the k in [0, min(z min(l, N-l), N_B)] with the lattice's spacing."""
    return min(z * min(ell, N - ell), NB) // kstep + 1


def line_costs(N: int, NB: int, z: int, kstep: int) -> dict:
    """Estimated cost (bins^2) of every line l = 0..N/2."""
    return {ell: line_bins(N, NB, z, kstep, ell) ** 2 for ell in range(N // 2 + 1)}


def lpt_partition(costs: dict, nranks: int) -> list:
    """Longest processing time first: lines in decreasing cost (ties by l), each
    to the rank with the least assigned cost so far (ties by rank).  Every line
    goes to exactly one rank; the result is the same on every rank."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    heap = [(0, r) for r in range(nranks)]
    shares = [[] for _ in range(nranks)]
    for ell in sorted(costs, key=lambda l: (-costs[l], l)):
        load, r = heapq.heappop(heap)
        shares[r].append(ell)
        heapq.heappush(heap, (load + costs[ell], r))
    return [sorted(s) for s in shares]


def handle_costs(h) -> dict:
    """line_costs for a library handle (paper_1302_2320_gb300.Handle)."""
    return line_costs(h.N, h.NB, h.get_option("z"), h.get_option("k_step"))


def walk_share(h, ells, ln_f_min: float, flatness: float = 0.8, allow=None) -> dict:
    """Walk the lines `ells` on this rank's GPU and return {l: assembled ln g}."""
    import paper_1302_2320_gb300 as wl
    h.select_lines(ells)
    h.run(ln_f_min, flatness, allow=allow or (wl.WL_OK, wl.WL_ENOTCONVERGED))
    h.assemble()
    return {int(ell): h.get_lng(int(ell)) for ell in ells}


def gather_lines(dist, local: dict, dst: int = 0):
    """Gather every rank's {l: ln g} on rank dst (host objects over the process
    group).  Returns the merged dict on dst, None elsewhere.  A line that two
    ranks report is an error."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return dict(local)
    world = dist.get_world_size()
    parts = [None] * world if dist.get_rank() == dst else None
    dist.gather_object(local, parts, dst=dst)
    if dist.get_rank() != dst:
        return None
    merged = {}
    for p in parts:
        for ell, arr in p.items():
            if ell in merged:
                raise ValueError(f"line {ell} walked by two ranks")
            merged[ell] = arr
    return merged


def ragged_surface(lines: dict, nlines: int):
    """(values, offsets) over l = 0..nlines-1 in order of l, like wl_get_surface."""
    missing = [l for l in range(nlines) if l not in lines]
    if missing:
        raise ValueError(f"lines missing from the gather: {missing[:8]}")
    offs = np.zeros(nlines + 1, dtype=np.int64)
    for l in range(nlines):
        offs[l + 1] = offs[l] + len(lines[l])
    return np.concatenate([np.asarray(lines[l], dtype=np.float64) for l in range(nlines)]), offs

"""Sharding independent generator sets across ranks (one GPU per rank).

The sets of a batched closure are independent units: each rank closes its own
share with ``lie_closure_batched`` on its GPU, with no collective on the data
path; only the per-set results (dimension, status) are gathered at the end.

Shares are balanced by an estimated cost, longest-processing-time first.  The
cost of one closure is dominated by screening every pair of the final basis
against that basis: about D^2 / 2 candidates times N P flops each, with
D <= d^2 - 1 + 1 the largest possible dimension, N ~ D and P = d^2, so it is
taken as d^6 (times the generator count as a tie-breaker).
"""
from __future__ import annotations

import heapq


def set_cost(d: int, k: int) -> float:
    """Estimated relative cost of closing a set of k generators of size d."""
    return float(d) ** 6 * (1.0 + 1e-3 * k)


def assign(costs, world: int):
    """Longest-processing-time-first assignment of units to ``world`` ranks.

    Returns a list of index lists, one per rank, each in increasing order.  The
    assignment is deterministic (ties broken by index and rank), so every rank
    computes the same plan without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shares]


def run_sharded(generator_sets, tol: float, rank: int, world: int, closure_fn, gather_fn=None, **opts):
    """Close this rank's share of ``generator_sets`` and gather all results.

    closure_fn(sets, tol, **opts) -> (dims, statuses) runs on the local GPU (in
    production ``binding.lie_closure_batched`` without bases); gather_fn(obj)
    returns the list of every rank's obj (``torch.distributed.all_gather_object``
    wrapped), or None on a single rank.  Returns (dims, statuses) for all sets,
    in input order, on every rank."""
    costs = [set_cost(g.shape[1], g.shape[0]) for g in generator_sets]
    shares = assign(costs, world)
    mine = shares[rank]
    dims, stats = closure_fn([generator_sets[i] for i in mine], tol, **opts) if mine else ([], [])
    local = list(zip(mine, dims, stats))
    parts = gather_fn(local) if gather_fn is not None and world > 1 else [local]
    out_d = [None] * len(generator_sets)
    out_s = [None] * len(generator_sets)
    for part in parts:
        for i, dm, st in part:
            out_d[i] = dm
            out_s[i] = st
    return out_d, out_s


def lie_closure_batched_sharded(generator_sets, tol: float, **opts):
    """Every rank of an initialised torch.distributed job calls this with the
    same sets; each closes its share on its current GPU and all ranks return
    the full (dims, statuses).  Without a process group it runs everything
    locally."""
    from . import binding

    def closure_fn(sets, tol_, **kw):
        dims, stats, _, _ = binding.lie_closure_batched(sets, tol_, **kw)
        return dims, stats

    try:
        import torch.distributed as dist
        ready = dist.is_available() and dist.is_initialized()
    except ImportError:
        ready = False
    if not ready:
        return run_sharded(generator_sets, tol, 0, 1, closure_fn, None, **opts)

    def gather(obj):
        out = [None] * dist.get_world_size()
        dist.all_gather_object(out, obj)
        return out

    return run_sharded(generator_sets, tol, dist.get_rank(), dist.get_world_size(), closure_fn, gather, **opts)

"""Sharding independent generator sets across ranks (one GPU per rank).

The sets of a batched closure are independent units: each rank closes its own
share with ``lie_closure_batched`` on its GPU, with no collective on the data
path; only the per-set results (dimension, status and, on request, the basis)
are gathered at the end.

Shares are balanced by an estimated cost, longest-processing-time first.  A
closure of final dimension D at size d screens about D^2 / 2 candidates, each
projected onto a basis of up to D elements of P = d^2 components: about
6 D^3 d^2 flops of screening GEMMs, plus a per-set floor for the block loop's
launches and synchronisations.  D is the exact string count when every
generator is a multiple of one Pauli string (then every bracket is again a
string, and the closure is the set of strings reached), else the generic
bound d^2 - 1.
"""
from __future__ import annotations

import heapq

import numpy as np

# rates behind the cost estimate (seconds): sustained screening-GEMM rate and
# the host-side cost of one block of the sweep
_GEMM_FLOPS = 1.5e15
_BLOCK_S = 1e-3


def pauli_string_bits(m: np.ndarray):
    """(x, z) bit masks if ``m`` is a nonzero multiple of one Pauli string, else
    None.  Bits follow the row index: row r has its single nonzero in column
    r ^ x, with value m[0, x] * (-1)^popcount(r & z)."""
    d = m.shape[0]
    nz = np.abs(m) > 1e-12 * max(1.0, float(np.abs(m).max()))
    if not nz.any() or not np.all(nz.sum(axis=1) == 1):
        return None
    x = int(np.argmax(nz[0]))
    rows = np.arange(d)
    cols = rows ^ x
    if not np.all(nz[rows, cols]):
        return None
    vals = m[rows, cols]
    ratio = vals / vals[0]
    z = 0
    b = 1
    while b < d:
        if abs(ratio[b] + 1.0) < 1e-9:
            z |= b
        elif abs(ratio[b] - 1.0) > 1e-9:
            return None
        b <<= 1
    par = np.array([bin(r & z).count("1") & 1 for r in range(d)])
    if not np.allclose(ratio, 1.0 - 2.0 * par, atol=1e-9):
        return None
    return x, z


def _string_closure_count(strings) -> int:
    """Number of distinct strings reached from ``strings`` by the bracket:
    anticommuting strings (odd symplectic form) bracket to their product,
    whose bits are the XOR of theirs; commuting strings bracket to zero."""
    xs, zs = [], []
    seen = set()
    for s in strings:
        if s != (0, 0) and s not in seen:
            seen.add(s)
            xs.append(s[0])
            zs.append(s[1])
    i = 0
    while i < len(xs):
        X = np.asarray(xs[:i], dtype=np.int64)
        Z = np.asarray(zs[:i], dtype=np.int64)
        form = (X & zs[i]) ^ (Z & xs[i])
        odd = np.zeros(len(form), dtype=bool)
        v = form.copy()
        while np.any(v):
            odd ^= (v & 1).astype(bool)
            v >>= 1
        for j in np.nonzero(odd)[0]:
            s = (xs[i] ^ xs[j], zs[i] ^ zs[j])
            if s not in seen:
                seen.add(s)
                xs.append(s[0])
                zs.append(s[1])
        i += 1
    return len(xs)


def estimate_dim(generators: np.ndarray) -> int:
    """Closure dimension used by the cost model: exact for generator sets made
    of Pauli-string multiples, the generic bound d^2 - 1 otherwise."""
    d = generators.shape[1]
    bits = [pauli_string_bits(g) for g in generators]
    if all(b is not None for b in bits):
        # an identity generator adds one direction that brackets to nothing
        ident = any(b == (0, 0) for b in bits)
        return _string_closure_count(bits) + (1 if ident else 0)
    return d * d - 1


def set_cost(d: int, k: int, dim: int | None = None) -> float:
    """Estimated seconds to close a set of k generators of size d whose closure
    has dimension ``dim`` (default: the generic bound d^2 - 1)."""
    D = float(d * d - 1 if dim is None else max(dim, 1))
    return 6.0 * D ** 3 * d * d / _GEMM_FLOPS + _BLOCK_S * max(1.0, D / 64.0) + 1e-9 * k


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


def run_sharded(generator_sets, tol: float, rank: int, world: int, closure_fn, gather_fn=None,
                gather_bases: bool = False, **opts):
    """Close this rank's share of ``generator_sets`` and gather all results.

    closure_fn(sets, tol, return_basis, **opts) -> (dims, statuses, bases) runs
    on the local GPU (in production ``binding.lie_closure_batched``); bases is
    None unless return_basis.  gather_fn(obj) returns the list of every rank's
    obj (``torch.distributed.all_gather_object`` wrapped), or None on a single
    rank.  Returns (dims, statuses, bases) for all sets, in input order, on
    every rank; bases is None unless ``gather_bases`` (every rank then holds
    every basis, so use it for sets whose bases fit each host)."""
    costs = [set_cost(g.shape[1], g.shape[0], estimate_dim(g)) for g in generator_sets]
    shares = assign(costs, world)
    mine = shares[rank]
    if mine:
        dims, stats, bases = closure_fn([generator_sets[i] for i in mine], tol, gather_bases, **opts)
    else:
        dims, stats, bases = [], [], []
    if not gather_bases or bases is None:
        bases = [None] * len(mine)
    local = list(zip(mine, dims, stats, bases))
    parts = gather_fn(local) if gather_fn is not None and world > 1 else [local]
    n = len(generator_sets)
    out_d, out_s, out_b = [None] * n, [None] * n, [None] * n
    for part in parts:
        for i, dm, st, b in part:
            out_d[i] = dm
            out_s[i] = st
            out_b[i] = b
    return out_d, out_s, (out_b if gather_bases else None)


def lie_closure_batched_sharded(generator_sets, tol: float, gather_bases: bool = False, **opts):
    """Every rank of an initialised torch.distributed job calls this with the
    same sets; each closes its share on its current GPU and all ranks return
    the full (dims, statuses, bases).  Without a process group it runs
    everything locally."""
    from . import binding

    def closure_fn(sets, tol_, return_basis, **kw):
        dims, stats, bases, _ = binding.lie_closure_batched(sets, tol_, return_basis=return_basis, **kw)
        return dims, stats, bases

    try:
        import torch.distributed as dist
        ready = dist.is_available() and dist.is_initialized()
    except ImportError:
        ready = False
    if not ready:
        return run_sharded(generator_sets, tol, 0, 1, closure_fn, None, gather_bases, **opts)

    def gather(obj):
        out = [None] * dist.get_world_size()
        dist.all_gather_object(out, obj)
        return out

    return run_sharded(generator_sets, tol, dist.get_rank(), dist.get_world_size(), closure_fn, gather,
                       gather_bases, **opts)

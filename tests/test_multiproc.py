"""The multi-rank path of bench.py on CPU: world size 2 over gloo.

Every rank of a GPU run is an independent replica; the only cross-rank steps
are the barriers around the timed region and the max over ranks of the elapsed
time.  Here they run on CPU processes with the gloo backend (no GPU)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    dist.init_process_group("gloo")
    bench.barrier(dist)
    q.put((rank, bench.max_over_ranks(dist, float(10 * rank + 1))))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 11.0), (1, 11.0)]


def test_reference_arm_under_torchrun_world2():
    """Rank 0 alone runs the oracle arm and prints one JSON line; rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-seconds", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 2 and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle"
    assert j["e2e"]["h2d_bytes_per_step"] == 0


# ------------------------------------------------- batched sets across ranks
def test_cost_model_dimension_estimate():
    """The cost model's dimension is the exact string count for Pauli-string
    sets (checked against the oracle's integer closure, which shares no code
    with it) and d^2 - 1 for dense random sets."""
    import numpy as np
    import oracle.closure as oc
    from paper_2506_01120_gb300 import inputs, shard
    for s in inputs.batched_sets(40, seed=3):
        est = shard.estimate_dim(s["generators"])
        if s["kind"] == "pauli":
            assert est == len(oc.pauli_closure(s["labels"]))
        else:
            assert est == s["d"] ** 2 - 1
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(4))
    assert shard.estimate_dim(g) == 255
    assert shard.estimate_dim(3.0 * inputs.generators_from_labels(inputs.so2n_chain_labels(4))) == 28
    assert shard.pauli_string_bits(np.eye(4) + 0.1) is None
    # small Pauli closures cost far less than generic sets of the same d
    assert shard.set_cost(64, 3, dim=30) < 1e-3 * shard.set_cost(64, 3)


def test_lpt_assignment_balances_and_covers():
    from paper_2506_01120_gb300 import shard
    costs = [shard.set_cost(d, k) for d, k in [(64, 2), (64, 6), (32, 3), (16, 2), (8, 5), (64, 4), (8, 2)]]
    for world in (1, 2, 3, 4):
        shares = shard.assign(costs, world)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shares]
        # LPT bound: max load <= (4/3 - 1/(3 m)) OPT, and OPT >= max(mean, largest)
        opt_lb = max(sum(costs) / world, max(costs))
        assert max(loads) <= (4 / 3) * opt_lb + 1e-9
    assert shard.assign(costs, 2) == shard.assign(list(costs), 2)     # deterministic


def _shard_worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    from paper_2506_01120_gb300 import inputs, shard
    dist.init_process_group("gloo")
    sets = [s["generators"] for s in inputs.batched_sets(12, seed=5, dims=(8, 16))]

    def fake_closure(gs, tol, return_basis, **opts):
        # stands in for the GPU call: one deterministic number (and a small
        # array standing for the basis) per set
        dims = [int(g.shape[1] * 100 + g.shape[0]) for g in gs]
        bases = [np.full((2, 2), float(x)) for x in dims] if return_basis else None
        return dims, [0] * len(gs), bases

    def gather(obj):
        out = [None] * world
        dist.all_gather_object(out, obj)
        return out

    dims, stats, none = shard.run_sharded(sets, 1e-8, rank, world, fake_closure, gather)
    assert none is None
    dims_b, stats_b, bases = shard.run_sharded(sets, 1e-8, rank, world, fake_closure, gather, gather_bases=True)
    assert dims_b == dims and stats_b == stats
    q.put((rank, dims, stats, [float(b[0, 0]) for b in bases]))
    dist.destroy_process_group()


def test_run_sharded_gathers_every_set_gloo():
    import torch.multiprocessing as mp
    from paper_2506_01120_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    sets = [s["generators"] for s in inputs.batched_sets(12, seed=5, dims=(8, 16))]
    want = [int(g.shape[1] * 100 + g.shape[0]) for g in sets]
    for rank, dims, stats, bases in res:
        assert dims == want and stats == [0] * 12
        assert bases == [float(x) for x in want]          # every rank holds every set's basis

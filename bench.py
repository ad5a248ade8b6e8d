#!/usr/bin/env python
"""Benchmark of the Lie-closure hot path (Algorithm 4, arXiv 2506.01120).

One step = one complete closure of the su(64) open-chain workload (d = 64,
generators iX_j, iY_j (j = 1..6) and iZ_jZ_{j+1} (j = 1..5), dimension 4095,
17 + 4095*4094/2 = 8,382,482 candidates) through ``lie_closure_dev`` in mixed
precision, generators already resident on the device.

Printed (rank 0, one JSON line): brackets checked per second (whole job),
time-to-closure, the roofline of the dominant kernel (the split-BF16 tcgen05
screening GEMM, event-timed inside the library on the call's stream), the
end-to-end number through the host API (host->device copy of the generators,
device->host copy of the basis), the FP64 GPU path on a bounded prefix of the
same sweep, the sparse Pauli-sum form of the method on the same generators at
6 and 7 qubits (the workloads of the paper's Table 2), and the CPU oracle on a
bounded sample.

``--impl reference`` times the CPU oracle instead (the paper has no code; the
oracle is the reference arm) on bounded samples of the same workload.
Multi-GPU: every rank runs an independent replica (a single closure does not
shard); value = all ranks' candidates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "brackets checked/s and time-to-closure, mixed vs FP64 GPU, at equal closure dim"
UNIT = "brackets/s"
WORKLOAD = "su64_chain_d64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--block-k", type=int, default=0)
    ap.add_argument("--tau", type=float, default=0.0)
    ap.add_argument("--fp64-prefix", type=int, default=60000,
                    help="candidates of the FP64 GPU comparison run (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle sample budget (0 = skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-seconds", type=float, default=0.0,
                    help="reference arm: oracle seconds per step (0 = about a minute in total)")
    ap.add_argument("--pauli-steps", type=int, default=3,
                    help="timed closures per sparse Pauli-sum workload (0 = skip)")
    ap.add_argument("--pauli-qubits", type=int, nargs="*", default=[6, 7],
                    help="qubit counts of the sparse hardware-efficient-ansatz workloads")
    ap.add_argument("--pauli-only", action="store_true", help="run only the sparse Pauli-sum leg")
    ap.add_argument("--next-rows", action="store_true",
                    help="run only the Algorithm 2 / Algorithm 3 / resume timings and print them as one line")
    ap.add_argument("--legs", default="fp64full,config5,config3,batched",
                    help="comma list of the single-run workload legs after the timed steps "
                         "(fp64full, config5, config3, batched; 'none' = skip)")
    ap.add_argument("--batched-full", action="store_true",
                    help="batched leg: full Algorithm 4 sweep per set instead of the saturation exit")
    ap.add_argument("--autotune", type=int, default=0, help="lc_options.autotune for the timed steps")
    ap.add_argument("--legs-only", action="store_true",
                    help="run only the --legs workload legs and print them as one line")
    ap.add_argument("--kernel-case", action="store_true",
                    help="run only the profiling case: the saturated su(64) state (all 4095 Pauli strings) resumed "
                         "at the pair (3000, 0) for 31,744 candidates, i.e. blocks of 1024 .. 16384 pairs")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self) -> dict:
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        return j, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def profiled_traffic(version: str):
    """DRAM bytes per launch of the screening GEMM from the committed ncu
    summary, if it was taken on this kernel version; else None."""
    p = os.path.join(ROOT, "profiles", "split_gemm_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    with open(p) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("library_version") != version:
        return None
    return int(kv["dram_bytes_per_launch"])


# ------------------------------------------------------------ CPU oracle leg
def oracle_sample(seconds: float):
    """The oracle as it stands, resumed at the saturated state of the same
    sweep (V = the 4095 orthonormal Pauli elements of su(64), cursor l = 2000),
    checking candidates for about ``seconds``.  Returns (rate, cand, wall, cores)."""
    import oracle.closure as oc
    from paper_2506_01120_gb300 import inputs
    g, labels = inputs.workload_generators(WORKLOAD)
    V = inputs.generators_from_labels(oc.pauli_closure(labels))
    state = oc.Alg4Result(V=V, dim=V.shape[0], l=2000, m=0, max_dim=2 * 64 * 64)
    done, t0, c0 = 0, time.perf_counter(), time.process_time()
    while time.perf_counter() - t0 < seconds:
        state = oc.alg4_orthonormalization(g, 1e-8, resume=state, max_candidates=4)
        done += 4
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    return done / wall, done, wall, max(1, round(cpu / wall))


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    per_step = args.ref_seconds if args.ref_seconds > 0 else \
        max(2.0, min(15.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(per_step / 4)
    rates, walls, cores, cands = [], [], 1, 0
    for _ in range(args.steps):
        r, c, w, cores = oracle_sample(per_step)
        rates.append(r)
        walls.append(w)
        cands += c
    value = cands / sum(walls)
    sample = (f"oracle resumed at the saturated state of {WORKLOAD} (|V|=4095, cursor l=2000), "
              f"{cands} candidates over {args.steps} steps of ~{per_step:.0f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "d": 64, "k": 17, "tol": 1e-8},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             **host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU legs
# Table 2 of the paper (many-core CPU, sparse Pauli sums): seconds per closure
PAPER_TABLE2_S = {6: 429.0, 7: 2345.0}
# issue-slot utilisation of k_pauli_screen1 measured by ncu (7-qubit chain)
PAULI_SCREEN1_ISSUE_ACTIVE = 0.62
# algorithmic bytes of the one-string screen (k_pauli_screen1) per candidate:
# the two operand strings (16 B) and the flag (1 B), plus for anticommuting
# pairs the index probe (string 8 B + head 4 B)
def pauli_screen_bytes(candidates: int, anticommuting: int) -> float:
    return 17.0 * candidates + 12.0 * anticommuting


def pauli_leg(args, stream, peaks, peak_src):
    """Sparse Pauli-sum closures of the hardware-efficient-ansatz generators
    (iX_j, iY_j, iZ_jZ_{j+1}) through lie_closure_pauli_dev (resident inputs)
    and lie_closure_pauli (host arrays in, basis out)."""
    import numpy as np
    import torch

    from paper_2506_01120_gb300 import binding, inputs
    out = []
    for n in args.pauli_qubits:
        labels = inputs.su2n_chain_labels(n)
        s, c, o = inputs.pauli_sum_terms([[(l, 1.0)] for l in labels])
        D = 4 ** n - 1
        cap, tcap = D + 1, 2 * (D + 1)
        ds, dc, do = (torch.from_numpy(s.view(np.int64)).cuda(), torch.from_numpy(c).cuda(),
                      torch.from_numpy(o).cuda())
        bs = torch.empty(tcap, dtype=torch.int64, device="cuda")
        bc = torch.empty(tcap, dtype=torch.float64, device="cuda")
        bo = torch.empty(cap + 1, dtype=torch.int64, device="cuda")

        def run():
            return binding.lie_closure_pauli_dev(ds, dc, do, n, 1e-8, cap, tcap, bs, bc, bo, stream=stream,
                                                 profile=1)
        run()
        torch.cuda.synchronize()
        times, reps = [], []
        for _ in range(args.pauli_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = run()
            b.record(stream)
            torch.cuda.synchronize()
            assert r.dim == D, (n, r.dim)
            times.append(a.elapsed_time(b) * 1e-3)
            reps.append(r.report)
        cand = reps[0]["brackets_checked"] + reps[0]["generators_checked"]
        t = sum(times) / len(times)
        t_screen = sum(rp["t_phase_s"][3] for rp in reps) / len(reps)
        t_accept = sum(rp["t_phase_s"][4] for rp in reps) / len(reps)
        screened = reps[0]["brackets_checked"]
        nbytes = pauli_screen_bytes(screened, reps[0]["n_nonzero"])
        gbs = nbytes / t_screen / 1e9 if t_screen > 0 else 0.0
        hw = []
        for _ in range(2):
            t0 = time.perf_counter()
            rh = binding.lie_closure_pauli(s, c, o, n, 1e-8, max_dim=cap, term_capacity=tcap)
            hw.append(time.perf_counter() - t0)
            assert rh.dim == D
        te = min(hw)
        out.append({
            "workload": f"hea_n{n}_pauli", "qubits": n, "closure_dim": D, "candidates": cand,
            "value": cand / t, "unit": UNIT, "time_to_closure_s": t, "t_last_accept_s": reps[-1]["t_last_accept_s"],
            "phase_s": {"screen": t_screen, "accept": t_accept, "other": max(0.0, t - t_screen - t_accept)},
            "screen_launches": reps[0]["gemm_launches"], "gpu_launches": reps[0]["kernel_launches"],
            "roofline": {"bound": "issue", "achieved": gbs, "unit": "GB/s (algorithmic bytes, L2-resident)",
                         "peak": None, "frac": None, "traffic": None, "kernel": "k_pauli_screen1",
                         "bytes_per_candidate": nbytes / screened if screened else None,
                         "issue_active_ncu": PAULI_SCREEN1_ISSUE_ACTIVE,
                         "note": "the basis strings and the string index stay in L2 (ncu: 97 % L2 hit rate, "
                                 "under 1 MB of DRAM traffic per launch); the kernel is bound by instruction "
                                 "issue (ncu: issue slots busy, profiles/k_pauli_screen1_hea_n7.md), not by HBM"},
            "e2e": {"value": cand / te, "unit": UNIT, "time_to_closure_s": te,
                    "h2d_bytes_per_step": int(s.nbytes + c.nbytes + o.nbytes),
                    "d2h_bytes_per_step": int(D * 16 + (D + 1) * 8)},
            "paper_table2_cpu_s": PAPER_TABLE2_S.get(n),
        })
    return out


def host_info():
    """The host the oracle ran on: core counts and the BLAS thread setting."""
    info = {"host_cores": os.cpu_count()}
    try:
        info["affinity_cores"] = len(os.sched_getaffinity(0))
    except AttributeError:
        pass
    blas = None
    try:
        from threadpoolctl import threadpool_info
        blas = [{"api": p.get("internal_api"), "threads": p.get("num_threads")} for p in threadpool_info()]
    except Exception:
        env = {k: os.environ[k] for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
               if k in os.environ}
        blas = env or "library default (all cores)"
    info["blas_threads"] = blas
    return info


def _closure_dev_timed(gd, tol, stream, **opts):
    """One closure through lie_closure_dev, timed with CUDA events on its stream."""
    import torch
    from paper_2506_01120_gb300 import binding
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    r = binding.lie_closure_dev(gd, tol, stream=stream, **opts)
    b.record(stream)
    torch.cuda.synchronize()
    return r, a.elapsed_time(b) * 1e-3


def fp64_full_leg(gd, tol, stream, mixed_s):
    """The plain FP64 GPU form of the bench workload run to closure."""
    r, t = _closure_dev_timed(gd, tol, stream, precision="fp64", profile=1)
    cand = r.report["brackets_checked"] + r.report["generators_checked"]
    return {"full_time_to_closure_s": t, "dim": r.dim, "candidates": cand, "brackets_per_s": cand / t,
            "t_last_accept_s": r.report["t_last_accept_s"],
            "phase_s": dict(zip(["brackets", "projection_gemm", "residual_gemm", "screen", "fp64_accept", "other"],
                                r.report["t_phase_s"])),
            "mixed_speedup_same_dim": t / mixed_s if mixed_s else None}


def config5_leg(stream, window_mixed=2_000_000, window_fp64=20_000):
    """su128_random2_d128 (d = 128, dim 16383, 134,193,155 candidates in the
    full sweep): time to the saturation exit (labelled: not in the paper) for
    both precisions, and a timed window of the saturated phase (resumed at the
    pair (8192, 0) of the saturated basis) from which the full sweep's time
    is extrapolated (labelled extrapolated)."""
    import torch
    from paper_2506_01120_gb300 import binding, inputs
    g, _ = inputs.workload_generators("su128_random2_d128")
    d, tol = g.shape[1], 1e-8
    D = d * d - 1
    full_cand = g.shape[0] + D * (D - 1) // 2
    gd = torch.from_numpy(g).cuda()
    B = torch.empty((D + 1, d, d), dtype=torch.complex128, device="cuda")
    out = {"workload": "su128_random2_d128", "d": d, "closure_dim": D, "full_sweep_candidates": full_cand}
    for prec, window in (("mixed", window_mixed), ("fp64", window_fp64)):
        r, t = _closure_dev_timed(gd, tol, stream, precision=prec, saturation_exit=1, profile=1,
                                  **({"basis_out": B} if prec == "mixed" else {}))
        sat_cand = r.report["brackets_checked"] + r.report["generators_checked"]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        w = binding.lie_closure_resume_dev(B, D, (8192, 0), tol, max_dim=D + 1, stream=stream, precision=prec,
                                           max_candidates=window)
        b.record(stream)
        torch.cuda.synchronize()
        tw = a.elapsed_time(b) * 1e-3
        rate = w.report["brackets_checked"] / tw
        out[prec] = {"saturation_exit": {"dim": r.dim, "candidates": sat_cand, "time_to_closure_s": t,
                                         "phase_s": dict(zip(["brackets", "projection_gemm", "residual_gemm",
                                                              "screen", "fp64_accept", "other"],
                                                             r.report["t_phase_s"])),
                                         "eps_screen": r.report["eps_screen"],
                                         "tau_screen": r.report["tau_screen"], "n_gray": r.report["n_gray"],
                                         "min_acc_rel_res": r.report["min_acc_rel_res"],
                                         "min_acc_screen_rel_res": r.report["min_acc_screen_rel_res"],
                                         "screen_margin": (r.report["min_acc_screen_rel_res"] / r.report["tau_screen"]
                                                           if prec == "mixed" else None)},
                     "saturated_window": {"candidates": w.report["brackets_checked"], "time_s": tw,
                                          "brackets_per_s": rate, "dim_after": w.dim,
                                          "n_flagged": w.report["n_flagged"]},
                     "full_sweep_time_s_extrapolated": t + (full_cand - sat_cand) / rate}
    out["mixed_vs_fp64_saturation_exit_speedup"] = (out["fp64"]["saturation_exit"]["time_to_closure_s"] /
                                                  out["mixed"]["saturation_exit"]["time_to_closure_s"])
    out["mixed_vs_fp64_full_sweep_speedup_extrapolated"] = (out["fp64"]["full_sweep_time_s_extrapolated"] /
                                                          out["mixed"]["full_sweep_time_s_extrapolated"])
    del B
    torch.cuda.empty_cache()
    return out


def config3_leg(stream, fp64_prefix=400):
    """so20_chain_d1024 (d = 1024, dim 190): the full mixed closure, and the
    FP64 and mixed forms on the same candidate prefix (the full FP64 closure
    needs ~1.5e14 FP64 flop of brackets alone)."""
    import torch
    from paper_2506_01120_gb300 import inputs
    g, _ = inputs.workload_generators("so20_chain_d1024")
    gd = torch.from_numpy(g).cuda()
    tol = 1e-8
    r, t = _closure_dev_timed(gd, tol, stream, precision="mixed", max_dim=256, profile=1)
    cand = r.report["brackets_checked"] + r.report["generators_checked"]
    out = {"workload": "so20_chain_d1024", "dim": r.dim, "candidates": cand, "time_to_closure_s": t,
           "brackets_per_s": cand / t,
           "phase_s": dict(zip(["brackets", "projection_gemm", "residual_gemm", "screen", "fp64_accept", "other"],
                               r.report["t_phase_s"]))}
    rf, tf = _closure_dev_timed(gd, tol, stream, precision="fp64", max_dim=256, max_candidates=fp64_prefix)
    rm, tm = _closure_dev_timed(gd, tol, stream, precision="mixed", max_dim=256, max_candidates=fp64_prefix)
    out["prefix"] = {"candidates": fp64_prefix, "fp64_time_s": tf, "mixed_time_s": tm, "fp64_dim": rf.dim,
                     "mixed_dim": rm.dim}
    return out


def batched_leg(full: bool):
    """The 256-set batched workload (seed 1120) through lie_closure_batched;
    per-set dimensions checked against the closed form / exact Pauli closure."""
    import oracle.closure as oc
    from paper_2506_01120_gb300 import binding, inputs
    sets = inputs.batched_sets(256, seed=1120)
    gens = [x["generators"] for x in sets]
    t0 = time.perf_counter()
    dims, stat, _, reps = binding.lie_closure_batched(gens, 1e-8, saturation_exit=0 if full else 1)
    t = time.perf_counter() - t0
    ok = all(st == 0 for st in stat)
    exact = all(dim == (len(oc.pauli_closure(x["labels"])) if x["kind"] == "pauli" else x["d"] ** 2 - 1)
                for x, dim in zip(sets, dims))
    cand = sum(r["brackets_checked"] + r["generators_checked"] for r in reps)
    return {"workload": "batched256_d8to64", "sets": len(sets), "mode": "full sweep" if full else
            "saturation exit (labelled; not in the paper)", "time_s": t, "candidates": cand,
            "brackets_per_s": cand / t, "all_ok": ok, "all_dims_exact": exact}


def kernel_case():
    """A short, fixed launch sequence for ncu: the su(64) basis made of the 4095
    non-identity Pauli strings (orthonormal, saturated) resumed at the pair
    (3000, 0) for 31,744 candidates, so the sweep runs blocks of 1024, 2048,
    4096, 8192 and 16384 pairs (the last one the saturated-phase size)."""
    from paper_2506_01120_gb300 import binding, inputs
    n = 6
    labels = ["".join("IXYZ"[(s >> (2 * q)) & 3] for q in range(n)) for s in range(1, 4 ** n)]
    V = inputs.generators_from_labels(labels)
    r = binding.lie_closure_resume(V, (3000, 0), 1e-8, precision="mixed", max_candidates=31744, profile=1)
    return {"kernel_case": {"dim": r.dim, "candidates": r.report["brackets_checked"],
                            "phase_s": r.report["t_phase_s"], "version": binding.version()}}


def next_rows_leg():
    """Algorithm 3 on the su(64) chain (mixed, host API), Algorithm 2 against
    Algorithm 4 in FP64 (full sweeps), and an su(64) closure stopped halfway
    and resumed."""
    from paper_2506_01120_gb300 import binding, inputs
    out = {}
    g, _ = inputs.workload_generators(WORKLOAD)
    binding.lie_closure(g, 1e-8, return_basis=False)          # warm the library and pool
    t0 = time.perf_counter()
    B, V, st, rep = binding.lie_closure_alg3(g, 1e-8, precision="mixed")
    t = time.perf_counter() - t0
    cand = rep["brackets_checked"] + rep["generators_checked"]
    out["alg3_su64_chain_d64_mixed"] = {"dim": len(V), "candidates": cand, "time_to_closure_s": t,
                                        "brackets_per_s": cand / t, "status": st}
    # Algorithm 2 against Algorithm 4 (both FP64): the su(2^n) chains, whose
    # Gram matrix stays the identity, and a random traceless pair, where the
    # paper warns that the inverse can go unstable
    cases = [(f"su{2 ** n}_chain_d{2 ** n}", inputs.generators_from_labels(inputs.su2n_chain_labels(n)))
             for n in (4, 5)]
    cases.append(("random2_d16", inputs.random_set(16, 2, seed=116)))
    for label, gr in cases:
        row = {}
        for name, fn in (("alg4_fp64", lambda: binding.lie_closure(gr, 1e-8, precision="fp64", check=False)),
                         ("alg2_fp64", lambda: binding.lie_closure_alg2(gr, 1e-8, check=False))):
            t0 = time.perf_counter()
            r = fn()
            t = time.perf_counter() - t0
            c = r.report["brackets_checked"] + r.report["generators_checked"]
            row[name] = {"dim": r.dim, "status": binding.status_string(r.status), "candidates": c,
                         "time_to_closure_s": t, "brackets_per_s": c / t}
        out[label] = row
    full = binding.lie_closure(g, 1e-8, precision="mixed")
    half = full.report["brackets_checked"] // 2
    t0 = time.perf_counter()
    a = binding.lie_closure(g, 1e-8, precision="mixed", max_candidates=half)
    t1 = time.perf_counter()
    b = binding.lie_closure_resume(a.basis, (a.report["cursor_l"], a.report["cursor_m"]), 1e-8, precision="mixed")
    t2 = time.perf_counter()
    import numpy as np
    out["resume_su64_chain_d64_mixed"] = {
        "full_time_s": full.report["t_total_s"], "first_half_s": t1 - t0, "resumed_half_s": t2 - t1,
        "same_basis": bool(b.dim == full.dim and np.abs(b.basis - full.basis).max() < 1e-12)}
    return out


def run_ours(args, world, rank, local, pg):
    import numpy as np
    import torch

    from paper_2506_01120_gb300 import binding, inputs
    from paper_2506_01120_gb300.build import build

    torch.cuda.set_device(local)
    if rank == 0 and not os.path.exists(binding.LIB_PATH):
        build()
    barrier(pg)
    if args.next_rows:
        if rank == 0:
            print(json.dumps({"next_rows": next_rows_leg()}), flush=True)
        return
    if args.kernel_case:
        if rank == 0:
            print(json.dumps(kernel_case()), flush=True)
        return
    if args.legs_only:
        legs = set(x for x in args.legs.split(",") if x and x != "none")
        out = {}
        if "config5" in legs:
            out["su128_random2_d128"] = config5_leg(torch.cuda.current_stream())
        if "config3" in legs:
            out["so20_chain_d1024"] = config3_leg(torch.cuda.current_stream())
        if "batched" in legs:
            out["batched256_d8to64"] = batched_leg(args.batched_full)
        if rank == 0:
            print(json.dumps({"workloads": out}), flush=True)
        return
    if args.pauli_only:
        peaks, peak_src = measured_peaks()
        sp = pauli_leg(args, torch.cuda.current_stream(), peaks, peak_src)
        if rank == 0:
            print(json.dumps({"sparse_pauli": sp}), flush=True)
        return
    g, _ = inputs.workload_generators(WORKLOAD)
    k, d = g.shape[0], g.shape[1]
    tol = 1e-8
    gd = torch.from_numpy(g).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    opts = dict(precision="mixed", profile=1)
    if args.autotune:
        opts["autotune"] = args.autotune
    if args.block_k:
        opts["block_k"] = args.block_k
    if args.tau:
        opts["tau_screen"] = args.tau

    def step():
        return binding.lie_closure_dev(gd, tol, stream=stream, **opts)

    for _ in range(args.warmup):
        flush.zero_()
        r = step()
        assert r.dim == 4095, r.dim
    torch.cuda.synchronize()
    barrier(pg)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    reports = []
    with ClockSampler(local) as clk:
        barrier(pg)
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()                       # L2 flush, outside the timed events
            ev[i][0].record(stream)
            r = step()
            ev[i][1].record(stream)
            reports.append(r.report)
            assert r.dim == 4095, r.dim
        torch.cuda.synchronize()
        barrier(pg)
    clocks = clk.summary()
    step_s = [a.elapsed_time(b) * 1e-3 for a, b in ev]
    local_total = sum(step_s)
    total = max_over_ranks(pg, local_total)
    cand = reports[0]["brackets_checked"] + reports[0]["generators_checked"]
    value = cand * args.steps * world / total

    # roofline of the dominant kernel (screening GEMMs), event-timed per phase
    peaks, peak_src = measured_peaks()
    gemm_t = sum(rep["t_phase_s"][1] + rep["t_phase_s"][2] for rep in reports)
    gemm_n = sum(rep["gemm_launches"] for rep in reports)
    gemm_f = sum(rep["gemm_flops"] for rep in reports)
    achieved_tf = gemm_f / gemm_t / 1e12 if gemm_t > 0 else 0.0
    peak_tf = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    traffic = profiled_traffic(binding.version())
    phases = [sum(rep["t_phase_s"][i] for rep in reports) / args.steps for i in range(6)]

    # end to end through the host API: pinned generators in, basis out
    e2e = None
    if args.e2e_steps > 0:
        gh = torch.from_numpy(g).pin_memory()
        bh = torch.empty((4095, d, d), dtype=torch.complex128).pin_memory()
        import ctypes
        L = binding.lib()
        o = binding.make_options("mixed")
        walls = []
        for i in range(args.e2e_steps + 1):
            dim = ctypes.c_longlong(0)
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = L.lie_closure(gh.data_ptr(), k, d, tol, bh.data_ptr(), ctypes.byref(dim), 4095, ctypes.byref(o),
                               None)
            t1 = time.perf_counter()
            assert st == 0 and dim.value == 4095
            if i > 0:
                walls.append(t1 - t0)
        e2e_t = max_over_ranks(pg, sum(walls))
        e2e = {"value": cand * len(walls) * world / e2e_t, "unit": UNIT,
               "h2d_bytes_per_step": int(g.nbytes), "d2h_bytes_per_step": int(4095 * d * d * 16),
               "time_to_closure_s": e2e_t / len(walls)}

    # the plain FP64 GPU form against the mixed form on the same prefix
    # the same closure with the (optional, not in the paper) saturation exit,
    # labelled separately: it stops once |V| reaches d^2 - 1
    rs = binding.lie_closure_dev(gd, tol, stream=stream, precision="mixed", saturation_exit=1)
    sat = {"dim": rs.dim, "candidates": rs.report["brackets_checked"] + rs.report["generators_checked"],
           "time_to_closure_s": rs.report["t_total_s"]}

    fp64 = None
    if args.fp64_prefix > 0:
        rf = binding.lie_closure_dev(gd, tol, stream=stream, precision="fp64", max_candidates=args.fp64_prefix)
        rm = binding.lie_closure_dev(gd, tol, stream=stream, precision="mixed", max_candidates=args.fp64_prefix)
        nf = rf.report["brackets_checked"] + rf.report["generators_checked"]
        fp64 = {"prefix_candidates": nf, "dim_at_prefix": rf.dim, "mixed_dim_at_prefix": rm.dim,
                "fp64_brackets_per_s": nf / rf.report["t_total_s"],
                "mixed_brackets_per_s_same_prefix": nf / rm.report["t_total_s"],
                "fp64_time_s": rf.report["t_total_s"], "mixed_time_s": rm.report["t_total_s"]}

    sparse = pauli_leg(args, stream, peaks, peak_src) if args.pauli_steps > 0 else None

    # single-run legs on the other workloads (not part of the timed steps)
    legs = set(x for x in args.legs.split(",") if x and x != "none")
    workloads = {}
    mixed_step_s = total / args.steps
    if "fp64full" in legs:
        fp64_full = fp64_full_leg(gd, tol, stream, mixed_step_s)
        if fp64 is None:
            fp64 = {}
        fp64.update(fp64_full)
    if "config5" in legs:
        workloads["su128_random2_d128"] = config5_leg(stream)
    if "config3" in legs:
        workloads["so20_chain_d1024"] = config3_leg(stream)
    if "batched" in legs:
        workloads["batched256_d8to64"] = batched_leg(args.batched_full)

    cpu = None
    if rank == 0 and args.cpu_seconds > 0:
        rate, c, w, cores = oracle_sample(args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{c} candidates in {w:.1f} s, oracle resumed at the saturated state of {WORKLOAD} "
                         f"(|V|=4095, cursor l=2000)", **host_info()}

    if rank != 0:
        return
    rep0 = reports[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3(f32 acc)+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "d": d, "k": k, "tol": tol, "precision": "mixed_bf16x3",
                   "closure_dim": rep0["dim"], "candidates_per_step": cand,
                   "block_k": args.block_k or "auto", "tau_screen": rep0["tau_screen"],
                   "l2": "flushed between steps (256 MB write); working set ~0.5 GB > L2",
                   "parallelism": f"replicas x{world}"},
        "time_to_closure_s": total / args.steps,
        "t_last_accept_s": rep0["t_last_accept_s"],
        "phase_s": dict(zip(["brackets", "projection_gemm", "residual_gemm", "screen", "fp64_accept", "other"],
                            phases)),
        "roofline": {"bound": "tensor", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / peak_tf if peak_tf else None, "traffic": traffic,
                     "kernel": "k_split_gemm (projection + residual)", "launches_per_step": gemm_n / args.steps,
                     "peak_source": f"bf16_tflops_sustained ({peak_src})"},
        "e2e": e2e,
        "saturation_exit": sat,
        "fp64_gpu": fp64,
        "workloads": workloads or None,
        "sparse_pauli": sparse,
        "cpu_baseline": cpu,
        "gpu_launches": int(sum(rep["kernel_launches"] for rep in reports)),
        "clocks": clocks,
        "screen": {"n_flagged": rep0["n_flagged"], "n_nonzero": rep0["n_nonzero"],
                   "tau_screen": rep0["tau_screen"], "eps_screen": rep0["eps_screen"], "n_gray": rep0["n_gray"],
                   "max_screen_rej_rel_res": rep0["max_screen_rej_rel_res"],
                   "min_acc_screen_rel_res": rep0["min_acc_screen_rel_res"],
                   "min_acc_rel_res": rep0["min_acc_rel_res"], "max_rej_rel_res": rep0["max_rej_rel_res"]},
        "tiles": {"block_k": rep0["block_k_used"], "block_k_growth": rep0["block_k_growth_used"],
                  "gemm_tile": [128, rep0["gemm_tile_n"], rep0["gemm_tile_k"]], "autotuned": rep0["autotuned"]},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()

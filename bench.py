"""Benchmark of the GB300 HYLU numeric phase: numeric LU ms per factorization,
GFLOP/s from the symbolic flop count and the fraction of the roofline, with
every solve held to backward error <= 1e-12.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hylu|reference]
                    [--workload convdiff3d_64|circuit_100k|aniso9_512|grid5_64|circuit_batch_512]

Default workload: the 3D 7-point upwind convection-diffusion operator on a 64^3
grid (n = 262,144, nested dissection), the largest single-GPU configuration.
One step = refactor (value scatter + numeric factorization) + forward/backward
substitution (+ refinement where taken), inputs resident in HBM.  On that
workload the line also carries the precision form (FP32 factors, FP64
refinement to the same 1e-12) measured on the same matrix.  Under torchrun
every rank factors its own replica (the path does not shard; the batching
workload splits its systems across ranks); rank 0 prints one JSON line.
`--impl reference` times the CPU oracle on a bounded sample instead: a
smaller instance of the same generator under the same ordering, extrapolated
by the symbolic flop count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "convdiff3d_64"
CIRCUIT_N = 30000          # size of the 'circuit' profiling workload (--n)
VALUE_SETS = 16
METRICS = {
    "circuit_100k": "numeric LU ms/factor (circuit-like n=100000, refactor of 16 value sets, "
                    "backward error <= 1e-12)",
    "convdiff3d_64": "numeric LU ms/factor (3D 7-point upwind convection-diffusion 64^3, n=262144, "
                     "nested dissection, backward error <= 1e-12)",
}
METRIC = METRICS["convdiff3d_64"]


def metric_name() -> str:
    if WORKLOAD in METRICS:
        return METRICS[WORKLOAD]
    return f"numeric LU ms/factor ({WORKLOAD}, backward error <= 1e-12)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hylu", choices=["hylu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ordering-trial", action="store_true",
                    help="circuit workload: untimed AMD / nested dissection trial first, the faster one timed")
    ap.add_argument("--no-precision-form", action="store_true",
                    help="convdiff3d_64: skip the measurements of the precision form (its own and the secondary configurations')")
    ap.add_argument("--no-secondary", action="store_true",
                    help="convdiff3d_64: skip the secondary configurations (5-point grid, circuit, "
                         "anisotropic diffusion) measured into the same line")
    ap.add_argument("--workload", default="convdiff3d_64",
                    choices=["circuit_100k", "circuit", "grid5_64", "aniso9_512", "convdiff3d_64",
                             "circuit_batch_512"],
                    help="convdiff3d_64 is the largest single-GPU configuration (default); 'circuit' "
                         "with --n is the circuit generator at another size (profiling cases)")
    ap.add_argument("--n", type=int, default=30000, help="size for --workload circuit")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="grid workloads: grid side x scale (profiling cases; 1 is the configuration)")
    ap.add_argument("--batch-systems", type=int, default=512,
                    help="circuit_batch_512: systems in the batch (512 is the configuration)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="fp32: the precision form (FP32 factors, FP64 refinement on every solve)")
    ap.add_argument("--gemm-min-rows", type=int, default=None,
                    help="precision form: smallest supernode that takes its sup-sup updates on the tensor "
                         "cores (0: off; default: the library's)")
    args = ap.parse_args()
    global WORKLOAD, CIRCUIT_N
    WORKLOAD = args.workload
    CIRCUIT_N = args.n
    return args


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        else:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- inputs
def make_inputs(n_circuit: int = 30000, scale: float = 1.0):
    """The workload matrix, VALUE_SETS value sets on its pattern (fresh values
    for the circuit generator, the matrix itself otherwise) and b = A x_true."""
    from paper_2509_07690_gb300 import synth
    if WORKLOAD == "circuit":
        idx = 1
        A = synth.circuit(n_circuit, seed=1000 + idx)
    else:
        idx = synth.WORKLOADS[WORKLOAD]["index"]
        A = synth.workload(WORKLOAD, scale)
    if WORKLOAD.startswith("circuit"):
        sets = [synth.circuit_value_set(A, 1002 + idx + j) for j in range(VALUE_SETS)]
    else:
        sets = [A] * VALUE_SETS
    xt, b = synth.rhs(A, 1001 + idx)
    return A, sets, b[0]


def ordering_for(workload: str) -> int:
    """Nested dissection (1) for the PDE workloads, AMD (0) for the 5-point
    grid and the circuit matrices.  On the circuit matrix nested dissection
    (hub rows last) has 11% fewer flops and a 6.4x shallower dependency graph,
    but measured on the GB300 its factorization is slower (260 against 212
    ms): the hub rows, not the chain, bound it."""
    return 1 if workload in ("aniso9_512", "convdiff3d_64") else 0


def backward_error(A, vals, x, b) -> float:
    """||b - A x||inf / (||A||inf ||x||inf + ||b||inf) with numpy (host check)."""
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    ax = np.bincount(rid, weights=vals * x[A.col], minlength=A.n)
    anorm = np.bincount(rid, weights=np.abs(vals), minlength=A.n).max()
    return float(np.abs(b - ax).max() / (anorm * np.abs(x).max() + np.abs(b).max()))


def residual_1(A, vals, x, b) -> float:
    """The paper's accuracy metric (Sec. 3.3): ||A x - b||_1 / ||b||_1 (host check)."""
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    ax = np.bincount(rid, weights=vals * x[A.col], minlength=A.n)
    r1 = float(np.abs(ax - b).sum())
    nb = float(np.abs(b).sum())
    return r1 / nb if nb > 0 else r1


def kernel_mix(info) -> dict:
    """Shares of the padded flops by kernel of the paper's Fig. 1 (row-row,
    sup-row, sup-sup) and the in-supernode factorization, from hylu_info."""
    total = info.flops_padded if info.flops_padded > 0 else 1.0
    parts = (("row_row", info.flops_row_row), ("sup_row", info.flops_sup_row),
             ("sup_sup", info.flops_sup_sup), ("in_supernode", info.flops_in_supernode))
    return {k: round(v / total, 4) for k, v in parts}


# oracle sample sizes: a fraction of the workload's size parameter (circuit
# rows, grid side), its starting value, and the exponent with which the
# oracle's time grows in it (flops of the ordering: circuits ~ n^3 here,
# 3D nested dissection n^2 = k^6, 2D nested dissection n^1.5 = k^3)
SAMPLE_GROWTH = {"circuit_100k": (0.1, 3.0), "circuit": (0.1, 3.0), "convdiff3d_64": (0.25, 6.0),
                 "aniso9_512": (0.1, 3.0), "grid5_64": (1.0, 3.0)}


def sample_instance(frac: float):
    """A smaller instance of the workload's own generator (same seed rule):
    frac x the circuit size or the grid side."""
    from paper_2509_07690_gb300 import synth
    if WORKLOAD == "circuit":
        return synth.circuit(max(50, int(round(CIRCUIT_N * frac))), seed=1001)
    return synth.workload(WORKLOAD, frac)


def oracle_once(frac: float, ordering: int | None = None):
    """Preprocess a sample instance with the library's host analysis (the
    oracle takes the same matching, scaling and ordering as every parity
    test), then time the oracle's factorization of it on one host core."""
    import oracle
    from paper_2509_07690_gb300 import Solver
    A = sample_instance(frac)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=ordering_for(WORKLOAD) if ordering is None else ordering)
    rp, cp, dr, dc, _ = s.export_perm()
    s.close()
    t0 = time.perf_counter()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc)
    dt = time.perf_counter() - t0
    fl = o.flops[0]
    del o
    return dt, fl, A.n


def oracle_size(budget_s: float, ordering: int | None = None) -> float:
    """Largest sample fraction (grown by 1.2x from the workload's start,
    at most 1) whose oracle run is predicted to fit the budget."""
    frac, expo = SAMPLE_GROWTH.get(WORKLOAD, (0.1, 3.0))
    dt, _, _ = oracle_once(frac, ordering)
    while frac < 1.0 and dt * 1.2 ** expo < budget_s:
        frac = min(1.0, frac * 1.2)
        dt, _, _ = oracle_once(frac, ordering)
    return frac


# ----------------------------------------------------------------- clocks
_ACTIVE_CLOCKS = []   # samplers still running (stopped on an abandoned measurement)


class Clocks:
    def __init__(self, gpu_index: int, path: str):
        self.path = path
        self.p = None
        _ACTIVE_CLOCKS.append(self)
        try:
            self.f = open(path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self in _ACTIVE_CLOCKS:
            _ACTIVE_CLOCKS.remove(self)
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [q.strip() for q in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_hbm_gbs() -> float:
    """Measured HBM copy bandwidth of the target GPU (MEASURED_PEAKS.json at
    the repository root), else 6.8 TB/s."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def kernel_hash() -> str:
    """Hash of the code that determines the factor kernel: kernels.cu up to
    its substitution section, plus launch_factor, without comments and blank
    lines."""
    p = os.path.join(ROOT, "paper_2509_07690_gb300", "csrc", "kernels.cu")
    src = open(p).read()
    i = src.index("// -------------------------------------------------------------- solve")
    j = src.index("int launch_factor(")
    k = src.index("\n}\n", j) + 3
    code = []
    for line in (src[:i] + src[j:k]).splitlines():
        line = line.split("//", 1)[0].rstrip()
        if line:
            code.append(line)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def profiled_traffic(workload: str, fp32: bool = False):
    """DRAM bytes per factor-kernel launch from the committed ncu summary, if
    it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"factor_kernel_{workload}{'_fp32' if fp32 else ''}.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("factor_source_sha256_16") != kernel_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------- batching form
BATCH_SETS = 4
BATCH_RHS = 8
BATCH_SAMPLE_EVERY = 16


def partition_systems(weights, ws: int) -> list[list[int]]:
    """Split independent systems over ws ranks with no exchange between them
    (the batching form shards by system): largest weight first, each to the
    least-loaded rank (ties to the lower rank), every rank's list ascending.
    The same on every rank (deterministic), so no rank needs to ask another.
    A rank's load is at most the mean load plus the largest single weight."""
    order = sorted(range(len(weights)), key=lambda q: (-weights[q], q))
    load = [0.0] * ws
    parts = [[] for _ in range(ws)]
    for q in order:
        r = min(range(ws), key=lambda j: (load[j], j))
        parts[r].append(q)
        load[r] += weights[q]
    return [sorted(p) for p in parts]


def batch_weight(n: int) -> float:
    """Work proxy of one circuit-like system of n rows for the split across
    ranks: its flops grow about like n^2 on this generator (AMD), known
    before any analysis."""
    return float(n) ** 2


def batch_inputs(count: int = 512, only=None):
    """512 circuit-like systems (n ~ U[2000, 40000]) of the circuit generator,
    4 value sets each (the matrix's own values, then fresh sets), 8 RHS.
    only: the indices of the systems to generate (this rank's share)."""
    from paper_2509_07690_gb300 import synth
    idx = synth.WORKLOADS["circuit_batch_512"]["index"]
    sizes = synth.circuit_batch_sizes()[:count]
    keep = range(len(sizes)) if only is None else only
    mats = [synth.circuit(int(sizes[q]), seed=1000 * (idx + 1) + q) for q in keep]
    sets = [[m.val if v == 0 else synth.circuit_values(m.rowptr, m.col, 7919 * (v + 1) + q)
             for q, m in zip(keep, mats)] for v in range(BATCH_SETS)]
    return mats, sets


def run_batch(args, ws, rank, local):
    """Batching form: every instance (system x value set) factored and solved
    (8 RHS) in one persistent launch per kernel, replayed from a CUDA graph
    with the autotuned grid; against per-system plain launches (one handle,
    refactor + solve per instance) timed on every 16th system."""
    import torch
    from paper_2509_07690_gb300 import BatchSolver, Solver, build as pbuild, capi
    pbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2509_07690_gb300 import synth
    sizes = synth.circuit_batch_sizes()[:args.batch_systems]
    share = partition_systems([batch_weight(int(n)) for n in sizes], ws)[rank]
    mats, sets = batch_inputs(args.batch_systems, only=share)
    k = len(mats)
    t0 = time.time()
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], BATCH_SETS)
    analyze_s = time.time() - t0
    info = bs.info
    inst = k * BATCH_SETS
    vals = torch.from_numpy(bs.concat_values(sets)).to(dev)
    rng = np.random.default_rng(1005)
    b = rng.standard_normal((BATCH_RHS, bs.n))
    db = torch.from_numpy(b).to(dev)
    dx = torch.empty_like(db)
    bs.factor(vals)
    bs.solve(db, dx)                          # sizes the right-hand-side workspace the graph uses
    best = bs.tune(vals)
    tinfo = bs.get_info()
    tuned = {"factor_blocks_per_sm": tinfo.factor_blocks_per_sm, "solve_blocks_per_sm": tinfo.solve_blocks_per_sm,
             "heavy_queue": tinfo.heavy_queue}
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream())
    # the graph cannot test the backward error on the host: where the
    # untimed factorization perturbed a pivot, two fixed FP64 refinement
    # steps are recorded after the solve; every replay's final residual is
    # read back below
    corrections = 2 if bs.get_info().nperturb > 0 else 0
    with torch.cuda.stream(side):
        bs.graph_capture(vals, db, dx, corrections=corrections, stream=side)
        for _ in range(args.warmup):
            bs.graph_launch(stream=side)
        side.synchronize()
        clocks = Clocks(local, os.path.join(tempfile.gettempdir(), f"hylu_clocks_{os.getpid()}.csv")) if rank == 0 else None
        barrier(ws)
        l0 = capi.hylu_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for _ in range(args.steps):
            bs.graph_launch(stream=side)
        e1.record(side)
        side.synchronize()
        launches = capi.hylu_launch_count() - l0
        clk = clocks.stop() if clocks else None
    t_batch = allmax(ws, e0.elapsed_time(e1)) / args.steps
    inst_all = int(round(allsum(ws, float(inst))))
    x = dx.cpu().numpy()
    ginfo = bs.get_info()
    nperturb = ginfo.nperturb
    be = res1 = 0.0
    be_all = []
    for q in range(inst):                     # every instance, every RHS (host check)
        v, sidx = divmod(q, k)
        m = mats[sidx]
        rb = bs.row_base[q]
        bq = 0.0
        for r in range(BATCH_RHS):
            bq = max(bq, backward_error(m, sets[v][sidx], x[r, rb:rb + m.n], b[r, rb:rb + m.n]))
            if q % 64 == 0:
                res1 = max(res1, residual_1(m, sets[v][sidx], x[r, rb:rb + m.n], b[r, rb:rb + m.n]))
        be_all.append(bq)
        if q % 64 == 0:
            be = max(be, bq)
    be_all = np.array(be_all)
    # per-system plain launches on a sample, extrapolated to every instance
    plain_ms = []
    for sidx in range(0, k, BATCH_SAMPLE_EVERY):
        m = mats[sidx]
        s = Solver(m.n, m.rowptr, m.col, m.val)
        dv = torch.from_numpy(sets[1][sidx]).to(dev)
        dbs = torch.from_numpy(np.ascontiguousarray(b[:, :m.n])).to(dev)
        dxs = torch.empty_like(dbs)
        s.factor(dv)
        s.solve(dbs, dxs)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        s.factor(dv)
        s.solve(dbs, dxs)
        a1.record()
        torch.cuda.synchronize()
        plain_ms.append(a0.elapsed_time(a1))
        s.close()
    t_plain = statistics.mean(plain_ms) * inst
    bs_flops = allsum(ws, info.flops)
    be = allmax(ws, be)
    be_whole = allmax(ws, ginfo.backward_error)
    above = int(round(allsum(ws, float(np.sum(be_all > 1e-12)))))
    nsys = args.batch_systems
    if rank == 0:
        out = {
            "metric": f"factorizations/s (batching form: {nsys} circuit-like systems n~U[2000,40000] x 4 value "
                      "sets x 8 RHS, one persistent launch per kernel in a CUDA graph)",
            "value": inst_all / (t_batch * 1e-3), "unit": "factorizations/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch, "higher_is_better": True,
            "scaling": "weak" if ws == 1 else "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "circuit_batch_512" if nsys == 512 else f"circuit_batch_{nsys}",
                       "systems": nsys, "systems_rank0": k, "value_sets": BATCH_SETS,
                       "instances": inst_all, "nrhs": BATCH_RHS, "rows_rank0": bs.n, "flops": bs_flops,
                       "nnz_store_rank0": info.nnz_store, "tuned_blocks_per_sm": best, "tuned": tuned,
                       "analyze_s": analyze_s,
                       "flops_by_kernel": kernel_mix(info), "graph_refinement_steps": corrections,
                       "l2": "factor storage far above the 126 MB L2, no flush",
                       "parallelism": f"systems split over {ws} ranks (no exchange)" if ws > 1 else "1 GPU"},
            "gflops": bs_flops / (t_batch * 1e-3) / 1e9,
            "backward_error": be, "residual_1": res1, "nperturb": nperturb,
            "backward_error_note": "backward_error: worst over every 64th instance (8 RHS each); "
                                   "instances_above_1e-12 counts every instance (host check of the replay's x); "
                                   "backward_error_whole_batch: the graph's final residual over the combined system",
            "instances_above_1e-12": above, "backward_error_worst_instance": float(allmax(ws, float(be_all.max()))),
            "backward_error_whole_batch": be_whole,
            "plain_launches": {"factorizations_per_s": inst / (t_plain * 1e-3), "ms_per_instance":
                               statistics.mean(plain_ms), "sample": f"every {BATCH_SAMPLE_EVERY}th system "
                               f"({len(plain_ms)} systems, value set 1), refactor + 8-RHS solve, extrapolated "
                               f"to rank 0's {inst} instances"},
            "speedup_vs_plain_launches": t_plain / t_batch,
            "cpu_baseline": None,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        print(json.dumps(out), flush=True)
    bs.close()
    return 0


# ----------------------------------------------------------------- arms
def run_reference(args, ws, rank):
    """The CPU oracle on the machine's host cores: each step times one oracle
    factorization of a smaller instance of the same generator under the
    ordering the GPU arm times, extrapolated by the symbolic flop count."""
    if rank != 0:
        return 0
    from paper_2509_07690_gb300 import Solver
    if WORKLOAD == "circuit_batch_512":
        print(json.dumps({"impl": "reference", "unavailable": "the batching workload has no oracle arm: "
                          "its per-instance parity is checked in the tests"}), flush=True)
        return 0
    A, sets, b = make_inputs(args.n, args.scale)
    ordering = ordering_for(WORKLOAD)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=ordering)
    total_flops = s.info.flops
    s.close()
    frac = oracle_size(max(2.0, args.cpu_seconds / 4), ordering)
    rates, n_s = [], 0
    for k in range(args.warmup + args.steps):
        dt, fl, n_s = oracle_once(frac, ordering)
        if k >= args.warmup:
            rates.append(dt / fl)
    ms_full = statistics.mean(rates) * total_flops * 1e3
    oname = "ND" if ordering == 1 else "AMD"
    sample = (f"extrapolation: {WORKLOAD} generator at n={n_s} (same seed rule, {oname} ordering as the GPU arm), "
              f"oracle factorization timed per step on one core, scaled by the flop count to n={A.n} "
              f"({total_flops:.3e} flops)")
    out = {"metric": metric_name(), "value": ms_full, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_full, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n": A.n, "nnz": A.nnz, "flops": total_flops, "ordering": oname},
           "cpu_baseline": {"value": ms_full, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample,
                            "extrapolated_from_n": n_s},
           "e2e": {"value": ms_full, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


class Rejected(Exception):
    """A measurement whose solution misses the backward-error acceptance."""


TRIAL_REFACTORS = 3


def ordering_trial(args, local) -> dict:
    """Untimed trial of both orderings on the workload (before any timed
    region): per ordering, one factorization and TRIAL_REFACTORS
    refactorizations with the solve, the mean factor-kernel time (CUDA
    events) and the worst backward error, or the library error it raised."""
    import gc
    import torch
    from paper_2509_07690_gb300 import Solver, build as pbuild, capi
    pbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)                # the library works on the current device
    A, sets, b = make_inputs(args.n, args.scale)
    fp32 = args.precision == "fp32"
    d_b = torch.from_numpy(b).to(dev)
    d_x = torch.empty_like(d_b)
    out = {}
    for name, o in (("ND", 1), ("AMD", 0)):
        s = None
        try:
            s = Solver(A.n, A.rowptr, A.col, A.val, timing=1, ordering=o, precision=1 if fp32 else 0)
            s.factor(torch.from_numpy(A.val).to(dev))
            s.solve(d_b, d_x)
            ms, be = [], 0.0
            for k in range(TRIAL_REFACTORS):
                s.factor(torch.from_numpy(sets[k % VALUE_SETS].val).to(dev))
                s.solve(d_b, d_x)
                ms.append(s.get_info().factor_kernel_ms)
                be = max(be, backward_error(A, sets[k % VALUE_SETS].val, d_x.cpu().numpy(), b))
            out[name] = {"factor_ms": statistics.mean(ms), "backward_error": be, "flops": s.info.flops}
        except capi.HyluError as e:
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        finally:
            if s is not None:
                s.close()
            gc.collect()
    return out


def choose_ordering(trial: dict) -> int:
    """Nested dissection (1) unless its trial failed (an error, or a backward
    error above 1e-12) or AMD's passing trial was faster; then AMD (0)."""
    def ok(t):
        return "factor_ms" in t and t["backward_error"] <= 1e-12
    nd, amd = trial["ND"], trial["AMD"]
    if not ok(nd) or (ok(amd) and amd["factor_ms"] < nd["factor_ms"]):
        return 0
    return 1


def run_hylu(args, ws, rank, local):
    """The plain form.  For the circuit workload an untimed trial times both
    orderings first (one process only), and the faster one that meets the
    1e-12 backward error is measured (nested dissection without a trial).  If
    the measured nested-dissection run fails (a library error, or a backward
    error above 1e-12) the workload is timed under AMD instead, and the line
    says so."""
    import gc
    from paper_2509_07690_gb300 import capi
    ordering = ordering_for(WORKLOAD)
    if not (WORKLOAD.startswith("circuit") and args.ordering_trial):
        out = measure_hylu(args, ws, rank, local, ordering)
        if WORKLOAD == "convdiff3d_64" and args.precision == "fp64" and not args.no_precision_form:
            # the precision form as specified (sup-sup on the tensor cores),
            # and the same FP32 factorization on CUDA cores only
            gc.collect()
            out32 = measure_hylu(args, ws, rank, local, ordering, fp32=True, sub=True)
            gc.collect()
            saved, args.gemm_min_rows = args.gemm_min_rows, 0
            out32c = measure_hylu(args, ws, rank, local, ordering, fp32=True, sub=True)
            args.gemm_min_rows = saved
            if out is not None and out32 is not None:
                out["precision_form"] = precision_summary(out, out32)
            if out is not None and out32c is not None:
                out["precision_form_cuda_cores"] = precision_summary(out, out32c)
        if WORKLOAD == "convdiff3d_64" and args.precision == "fp64" and not args.no_secondary:
            # the other single-matrix configurations, device-timed on the same
            # code (no CPU baseline, fewer steps): config 1 (5-point grid),
            # config 2 (circuit) and config 4 (anisotropic diffusion)
            sec = {}
            for wl in ("grid5_64", "circuit_100k", "aniso9_512"):
                gc.collect()
                saved_w, saved_s = WORKLOAD, args.steps
                set_workload(wl)
                args.steps = max(4, min(args.steps, 8))
                try:
                    o2 = measure_hylu(args, ws, rank, local, ordering_for(wl), sub=True)
                    o2p = None
                    if not args.no_precision_form:
                        # the precision form on the same matrix, against its FP64 line
                        gc.collect()
                        o2p = measure_hylu(args, ws, rank, local, ordering_for(wl), fp32=True, sub=True)
                finally:
                    set_workload(saved_w)
                    args.steps = saved_s
                if o2 is not None:
                    sec[wl] = secondary_summary(o2)
                    if o2p is not None:
                        sec[wl]["precision_form"] = precision_summary(o2, o2p)
            if out is not None and sec:
                out["secondary_workloads"] = sec
        if out is not None:
            print(json.dumps(out), flush=True)
        return 0
    trial = None
    if ws == 1:
        trial = ordering_trial(args, local)
        ordering = choose_ordering(trial)
        if ordering == 0:
            out = measure_hylu(args, ws, rank, local, 0, trial=trial)
            if out is not None:
                print(json.dumps(out), flush=True)
            return 0
    try:
        out = measure_hylu(args, ws, rank, local, 1, strict=True, trial=trial)
    except (capi.HyluError, Rejected) as e:
        reason = f"{type(e).__name__}: {e}"
        for c in list(_ACTIVE_CLOCKS):
            c.stop()
        gc.collect()                              # releases the failed run's solver
        sys.stderr.write(f"bench: nested dissection run failed ({reason}); timing AMD instead\n")
        out = measure_hylu(args, ws, rank, local, 0, fallback_from={"ordering": "ND", "reason": reason},
                           trial=trial)
    if out is not None:
        print(json.dumps(out), flush=True)
    return 0


def measure_hylu(args, ws, rank, local, ordering: int, strict: bool = False, fallback_from=None, trial=None,
                 fp32: bool | None = None, sub: bool = False):
    """One measured form on the workload; returns the JSON object (rank 0)
    or None.  sub: a second form reported inside the main line (no CPU
    baseline)."""
    import torch
    from paper_2509_07690_gb300 import Solver, build as pbuild, capi
    pbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    A, sets, b = make_inputs(args.n, args.scale)
    if fp32 is None:
        fp32 = args.precision == "fp32"
    extra = {} if args.gemm_min_rows is None else {"gemm_min_rows": args.gemm_min_rows}
    s = Solver(A.n, A.rowptr, A.col, A.val, timing=1, ordering=ordering, precision=1 if fp32 else 0, **extra)
    info = s.info
    flops = info.flops
    d_sets = [torch.from_numpy(v.val).to(dev) for v in sets]
    d_b = torch.from_numpy(b).to(dev)
    d_x = torch.empty_like(d_b)
    s.factor(torch.from_numpy(A.val).to(dev))
    s.solve(d_b, d_x)
    for k in range(args.warmup):
        s.factor(d_sets[k % VALUE_SETS])
        s.solve(d_b, d_x)
    torch.cuda.synchronize()
    if fp32:
        # FP32 FMA units x max SM clock: 152 SMs x 128 lanes x 2 flops x 2070 MHz
        peak_gflops = 152 * 128 * 2 * 2.070
        peak_source = "FP32 ALU: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (unit counts, max clock)"
    else:
        peak_gflops = capi.hylu_measure_fp64_peak(stream.cuda_stream)
        peak_source = "FP64 FMA throughput measured live (hylu_measure_fp64_peak)"
    # ---------------- device-resident timed region
    clocks = Clocks(local, os.path.join(tempfile.gettempdir(), f"hylu_clocks_{os.getpid()}.csv")) if rank == 0 else None
    barrier(ws)
    torch.cuda.synchronize()
    l0 = capi.hylu_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms, solve_ms, bes = [], [], []
    ev0.record(stream)
    for k in range(args.steps):
        fe[k][0].record(stream)
        s.factor(d_sets[k % VALUE_SETS])
        fe[k][1].record(stream)
        s.solve(d_b, d_x)
        inf = s.get_info()
        kern_ms.append(inf.factor_kernel_ms)
        solve_ms.append(inf.solve_kernel_ms)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    launches = capi.hylu_launch_count() - l0
    clk = clocks.stop() if clocks else None
    total_ms = ev0.elapsed_time(ev1)
    fact_ms = [a.elapsed_time(bb) for a, bb in fe]
    # correctness of the timed work: the last value set's solution
    x = d_x.cpu().numpy()
    be = backward_error(A, sets[(args.steps - 1) % VALUE_SETS].val, x, b)
    inf = s.get_info()
    t_fact = allmax(ws, sum(fact_ms))
    t_total = allmax(ws, total_ms)
    value = t_fact / (ws * args.steps)
    kmean = statistics.mean(kern_ms)
    smean = statistics.mean(solve_ms)
    achieved = flops / (kmean * 1e-3) / 1e12
    hbm_peak = measured_hbm_gbs()
    vbytes = 4 if fp32 else 8
    compulsory_bytes = 16.0 * A.nnz + (vbytes + 4.0) * info.nnz_store
    hbm_factor_bytes = 6.0 * flops + compulsory_bytes
    solve_bytes = (vbytes + 4.0) * info.nnz_store + 6.0 * 8.0 * A.n
    # ---------------- end to end through host buffers
    h_vals = [torch.from_numpy(v.val).pin_memory() for v in sets]
    h_b = torch.from_numpy(b).pin_memory()
    h_x = torch.empty_like(h_b).pin_memory()
    d_v = torch.empty_like(d_sets[0])
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        d_v.copy_(h_vals[k % VALUE_SETS], non_blocking=True)
        d_b.copy_(h_b, non_blocking=True)
        s.factor(d_v)
        s.solve(d_b, d_x)
        h_x.copy_(d_x, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    e2e_ms = allmax(ws, e0.elapsed_time(e1)) / (ws * args.steps)
    be_e2e = backward_error(A, sets[(args.steps - 1) % VALUE_SETS].val, h_x.numpy(), b)
    res1 = max(residual_1(A, sets[(args.steps - 1) % VALUE_SETS].val, x, b),
               residual_1(A, sets[(args.steps - 1) % VALUE_SETS].val, h_x.numpy(), b))
    if strict and not max(be, be_e2e) <= 1e-12:
        s.close()
        raise Rejected(f"backward error {max(be, be_e2e):.2e} above 1e-12")
    # ---------------- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not sub:
        frac = oracle_size(args.cpu_seconds / 2, ordering)
        dt, fl, n_s = oracle_once(frac, ordering)
        cpu = {"value": dt * 1e3 * flops / fl, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"extrapolation: {WORKLOAD} generator at n={n_s} ({fl:.3e} flops, {dt:.1f} s on one "
                         f"core, same ordering), scaled by the flop count to n={A.n}; host has "
                         f"{os.cpu_count()} cores",
               "extrapolated_from_n": n_s}
    if rank == 0:
        out = {
            "metric": metric_name(), "value": value, "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": (WORKLOAD if args.scale == 1.0 else f"{WORKLOAD}_x{args.scale}")
                       if WORKLOAD != "circuit" else f"circuit_{A.n}", "n": A.n,
                       "nnz": A.nnz, "ordering": "ND" if ordering == 1 else "AMD",
                       "precision": "FP32 factors + FP64 refinement" if fp32 else "FP64",
                       "value_sets": VALUE_SETS, "flops": flops, "nnz_lu": info.nnz_lu,
                       "nnz_store": info.nnz_store, "supernodes": info.nsupernodes,
                       "rows_in_supernodes": info.rows_in_supernodes,
                       "flops_by_kernel": kernel_mix(info),
                       "critical_path_levels": {"factor": info.factor_levels, "forward": info.fwd_levels,
                                                "backward": info.bwd_levels},
                       "l2": f"factor storage {info.nnz_store * 8 / 1e9:.2f} GB > 126 MB L2, no flush",
                       "parallelism": f"replicas x{ws}"},
            "gflops": flops / (value * 1e-3) / 1e9,
            "backward_error": max(be, be_e2e),
            "residual_1": res1,
            "solve_ms": statistics.mean(solve_ms),
            "nperturb": inf.nperturb,
            "refine_iters": inf.refine_iters,
            "tensor_supsup": tensor_summary(inf, kmean) if fp32 else None,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gflops / 1e3,
                         "unit": "TFLOP/s", "frac": achieved * 1e3 / peak_gflops,
                         "traffic": profiled_traffic(WORKLOAD, fp32), "kernel": "factor_kernel",
                         "peak_source": peak_source,
                         "kernel_ms": kmean},
            # the same factor kernel against HBM (12 B per U entry an update
            # touches, 2 flops each, plus A in and the factors out), and the
            # substitution kernels (each stored entry read once: value + index,
            # plus six n-vectors per right-hand side)
            "roofline_hbm": {"bound": "hbm", "kernel": "factor_kernel",
                             "achieved": hbm_factor_bytes / (kmean * 1e-3) / 1e9, "peak": hbm_peak,
                             "unit": "GB/s", "frac": hbm_factor_bytes / (kmean * 1e-3) / 1e9 / hbm_peak,
                             "bytes_per_launch": hbm_factor_bytes,
                             "compulsory_bytes": compulsory_bytes,
                             "compulsory_frac": compulsory_bytes / (kmean * 1e-3) / 1e9 / hbm_peak,
                             "note": "bytes_per_launch counts 12 B for every U entry an update touches; "
                                     "re-reads served from L2 make frac exceed 1"},
            "solve_roofline": {"bound": "hbm", "kernel": "fwd_kernel+bwd_kernel",
                               "achieved": solve_bytes / (smean * 1e-3) / 1e9, "peak": hbm_peak,
                               "unit": "GB/s", "frac": solve_bytes / (smean * 1e-3) / 1e9 / hbm_peak,
                               "bytes_per_solve": solve_bytes, "solve_kernel_ms": smean},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(A.nnz * 8 + A.n * 8),
                    "d2h_bytes_per_step": int(A.n * 8)},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if fallback_from:
            out["fallback_from"] = fallback_from
        if trial:
            out["ordering_trial"] = {"refactorizations": TRIAL_REFACTORS, **trial}
        s.close()
        return out
    s.close()
    return None


def measured_bf16_tflops() -> float:
    """Measured dense BF16 tensor throughput (MEASURED_PEAKS.json), else 1900."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def tensor_summary(inf, kernel_ms: float) -> dict:
    """The precision form's tensor-core sup-sup tasks: how many, their useful
    FP32 flops (2 per multiply-add of L_{D,S} U_{S,T}) and the BF16 tensor
    flops those take (six term products each), as a rate over the factor
    kernel's time against the measured BF16 peak."""
    bf16 = 6.0 * inf.gemm_flops
    rate = bf16 / (kernel_ms * 1e-3) / 1e12 if kernel_ms > 0 else 0.0
    return {"destinations": inf.gemm_destinations, "tasks": inf.gemm_tasks, "useful_fp32_flops": inf.gemm_flops,
            "bf16_flops": bf16, "bf16_tflops_over_factor_kernel": rate, "bf16_peak_tflops": measured_bf16_tflops(),
            "tensor_frac": rate / measured_bf16_tflops(), "products_per_fp32_product": 6}


def set_workload(name: str) -> None:
    global WORKLOAD
    WORKLOAD = name


def secondary_summary(o: dict) -> dict:
    """A secondary configuration's measurement inside the default line."""
    keep = ("value", "unit", "ms_per_step", "steps", "gflops", "backward_error", "solve_ms", "nperturb",
            "refine_iters", "gpu_launches")
    out = {k: o[k] for k in keep}
    out["config"] = {k: o["config"][k] for k in ("workload", "n", "nnz", "ordering", "flops", "critical_path_levels")}
    out["roofline"] = o["roofline"]
    out["e2e_ms"] = o["e2e"]["value"]
    out["clocks"] = o["clocks"]
    return out


def precision_summary(fp64: dict, fp32: dict) -> dict:
    """The precision form measured on the same matrix, against the FP64 line:
    factor and step times (the FP32 step includes its FP64 refinement), the
    backward error both reach, and the factor kernel's roofline."""
    return {"precision": fp32["config"]["precision"], "factor_ms": fp32["value"],
            "ms_per_step": fp32["ms_per_step"], "gflops": fp32["gflops"], "solve_ms": fp32["solve_ms"],
            "refine_iters": fp32["refine_iters"], "backward_error": fp32["backward_error"],
            "e2e_ms": fp32["e2e"]["value"], "roofline": fp32["roofline"], "tensor_supsup": fp32["tensor_supsup"],
            "speedup_factor_vs_fp64": fp64["value"] / fp32["value"],
            "speedup_step_vs_fp64": fp64["ms_per_step"] / fp32["ms_per_step"],
            "gpu_launches": fp32["gpu_launches"], "clocks": fp32["clocks"]}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
    ws, rank, local = dist_setup(args)
    try:
        if WORKLOAD == "circuit_batch_512":
            return run_batch(args, ws, rank, local)
        return run_hylu(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

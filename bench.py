"""Benchmark of the GB300 HYLU numeric phase (numeric LU ms per factorization,
GFLOP/s from the symbolic flop count, fraction of the FP64 roofline) on the
circuit-like workload: n = 100,000, 1% hubs, AMD ordering, refactorization of
16 fresh value sets on one pattern, each followed by a solve that must reach
backward error <= 1e-12.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hylu|reference]

One step = refactor (value scatter + numeric factorization) + forward/backward
substitution (+ refinement if a pivot was perturbed), inputs resident in HBM.
Under torchrun every rank factors its own replica (the path does not shard);
rank 0 prints one JSON line.  `--impl reference` times the CPU oracle on a
bounded sample (a smaller instance of the same generator, extrapolated by the
symbolic flop count) instead.
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

WORKLOAD = "circuit_100k"
VALUE_SETS = 16
METRIC = "numeric LU ms/factor (circuit-like n=100000, refactor of 16 value sets, backward error <= 1e-12)"


def metric_name() -> str:
    if WORKLOAD == "circuit_100k":
        return METRIC
    return f"numeric LU ms/factor ({WORKLOAD}, backward error <= 1e-12)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hylu", choices=["hylu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ordering-trial", action="store_true",
                    help="circuit workload: skip the untimed AMD / nested dissection trial")
    ap.add_argument("--workload", default="circuit_100k",
                    choices=["circuit_100k", "circuit", "grid5_64", "aniso9_512", "convdiff3d_64",
                             "circuit_batch_512"],
                    help="circuit_100k is the headline configuration; 'circuit' with --n is the same "
                         "generator at another size (profiling cases)")
    ap.add_argument("--n", type=int, default=30000, help="size for --workload circuit")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="grid workloads: grid side x scale (profiling cases; 1 is the configuration)")
    ap.add_argument("--batch-systems", type=int, default=512,
                    help="circuit_batch_512: systems in the batch (512 is the configuration)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="fp32: the precision form (FP32 factors, FP64 refinement on every solve)")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = args.workload
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
    """Nested dissection (1) for the PDE workloads and the circuit matrix, AMD
    (0) for the 5-point grid.  On the circuit matrix nested dissection (hub
    rows last) needs 11% fewer flops than AMD and its dependency graph is
    6.4x shallower (1,347 against 8,676 factor levels), and the factor kernel
    is bound by that chain."""
    return 1 if workload in ("aniso9_512", "convdiff3d_64", "circuit_100k", "circuit") else 0


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


def sample_instance(n_s: int):
    """A smaller instance of the same circuit-like generator (same seed rule)."""
    from paper_2509_07690_gb300 import synth
    idx = synth.WORKLOADS[WORKLOAD]["index"]
    return synth.circuit(n_s, seed=1000 + idx)


def oracle_once(n_s: int, ordering: int | None = None):
    """Preprocess a sample instance with the library's host analysis (the
    oracle takes the same matching, scaling and ordering as every parity
    test), then time the oracle's factorization of it on one host core."""
    import oracle
    from paper_2509_07690_gb300 import Solver
    A = sample_instance(n_s)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=ordering_for(WORKLOAD) if ordering is None else ordering)
    rp, cp, dr, dc, _ = s.export_perm()
    s.close()
    t0 = time.perf_counter()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc)
    dt = time.perf_counter() - t0
    fl = o.flops[0]
    del o
    return dt, fl


def oracle_size(budget_s: float, ordering: int | None = None) -> int:
    """Largest sample size n_s (grown by 1.5x from 10,000) whose oracle run is
    predicted to fit the budget (time grows about like n_s^3 here)."""
    n_s = 10_000
    dt, _ = oracle_once(n_s, ordering)
    while n_s < 100_000 and dt * 1.5 ** 3 < budget_s:
        n_s = min(100_000, int(n_s * 1.5))
        dt, _ = oracle_once(n_s, ordering)
    return n_s


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


def batch_inputs(count: int = 512):
    """512 circuit-like systems (n ~ U[2000, 40000]) of the circuit generator,
    4 value sets each (the matrix's own values, then fresh sets), 8 RHS."""
    from paper_2509_07690_gb300 import synth
    idx = synth.WORKLOADS["circuit_batch_512"]["index"]
    sizes = synth.circuit_batch_sizes()[:count]
    mats = [synth.circuit(int(n), seed=1000 * (idx + 1) + q) for q, n in enumerate(sizes)]
    sets = [[m.val if v == 0 else synth.circuit_values(m.rowptr, m.col, 7919 * (v + 1) + q)
             for q, m in enumerate(mats)] for v in range(BATCH_SETS)]
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
    mats, sets = batch_inputs(args.batch_systems)
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
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        bs.graph_capture(vals, db, dx, stream=side)
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
    x = dx.cpu().numpy()
    nperturb = bs.get_info().nperturb
    be = res1 = 0.0
    for q in range(0, inst, 64):              # every 64th instance, every RHS
        v, sidx = divmod(q, k)
        m = mats[sidx]
        rb = bs.row_base[q]
        for r in range(BATCH_RHS):
            be = max(be, backward_error(m, sets[v][sidx], x[r, rb:rb + m.n], b[r, rb:rb + m.n]))
            res1 = max(res1, residual_1(m, sets[v][sidx], x[r, rb:rb + m.n], b[r, rb:rb + m.n]))
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
    bs_flops = info.flops
    if rank == 0:
        out = {
            "metric": f"factorizations/s (batching form: {k} circuit-like systems n~U[2000,40000] x 4 value sets "
                      "x 8 RHS, one persistent launch per kernel in a CUDA graph)",
            "value": inst / (t_batch * 1e-3), "unit": "factorizations/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_batch, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "circuit_batch_512" if k == 512 else f"circuit_batch_{k}", "systems": k, "value_sets": BATCH_SETS,
                       "instances": inst, "nrhs": BATCH_RHS, "rows": bs.n, "flops": bs_flops,
                       "nnz_store": info.nnz_store, "tuned_blocks_per_sm": best, "analyze_s": analyze_s,
                       "flops_by_kernel": kernel_mix(info),
                       "l2": "factor storage far above the 126 MB L2, no flush",
                       "parallelism": f"replicas x{ws}"},
            "gflops": bs_flops / (t_batch * 1e-3) / 1e9,
            "backward_error": be, "residual_1": res1, "nperturb": nperturb,
            "plain_launches": {"factorizations_per_s": inst / (t_plain * 1e-3), "ms_per_instance":
                               statistics.mean(plain_ms), "sample": f"every {BATCH_SAMPLE_EVERY}th system "
                               f"({len(plain_ms)} systems, value set 1), refactor + 8-RHS solve, extrapolated "
                               f"to {inst} instances"},
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
    if rank != 0:
        return 0
    from paper_2509_07690_gb300 import Solver
    A, sets, b = make_inputs()
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=ordering_for(WORKLOAD))
    total_flops = s.info.flops
    s.close()
    n_s = oracle_size(max(2.0, args.cpu_seconds / 4))
    rates = []
    for k in range(args.warmup + args.steps):
        dt, fl = oracle_once(n_s)
        if k >= args.warmup:
            rates.append(dt / fl)
    ms_full = statistics.mean(rates) * total_flops * 1e3
    sample = (f"circuit-like generator at n={n_s} (same seed rule), oracle factorization timed per step, "
              f"extrapolated to the n={A.n} flop count")
    out = {"metric": METRIC, "value": ms_full, "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_full, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n": A.n, "nnz": A.nnz, "flops": total_flops},
           "cpu_baseline": {"value": ms_full, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample},
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
    if ordering == 0 or not WORKLOAD.startswith("circuit"):
        return measure_hylu(args, ws, rank, local, ordering)
    trial = None
    if ws == 1 and not args.no_ordering_trial:
        trial = ordering_trial(args, local)
        ordering = choose_ordering(trial)
        if ordering == 0:
            return measure_hylu(args, ws, rank, local, 0, trial=trial)
    try:
        return measure_hylu(args, ws, rank, local, 1, strict=True, trial=trial)
    except (capi.HyluError, Rejected) as e:
        reason = f"{type(e).__name__}: {e}"
    for c in list(_ACTIVE_CLOCKS):
        c.stop()
    gc.collect()                              # releases the failed run's solver
    sys.stderr.write(f"bench: nested dissection run failed ({reason}); timing AMD instead\n")
    return measure_hylu(args, ws, rank, local, 0, fallback_from={"ordering": "ND", "reason": reason}, trial=trial)


def measure_hylu(args, ws, rank, local, ordering: int, strict: bool = False, fallback_from=None, trial=None):
    import torch
    from paper_2509_07690_gb300 import Solver, build as pbuild, capi
    pbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    A, sets, b = make_inputs(args.n, args.scale)
    fp32 = args.precision == "fp32"
    s = Solver(A.n, A.rowptr, A.col, A.val, timing=1, ordering=ordering, precision=1 if fp32 else 0)
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
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and WORKLOAD == "circuit_100k":
        n_s = oracle_size(args.cpu_seconds / 2, ordering)
        dt, fl = oracle_once(n_s, ordering)
        cpu = {"value": dt * 1e3 * flops / fl, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"circuit-like generator at n={n_s} ({fl:.3e} flops, {dt:.1f} s on one core), "
                         f"extrapolated to the n={A.n} flop count; host has {os.cpu_count()} cores"}
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
        print(json.dumps(out), flush=True)
    s.close()
    return 0


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

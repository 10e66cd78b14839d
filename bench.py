#!/usr/bin/env python
"""Benchmark of the H_h matrix-vector product on GB300.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]
                    [--workload adaptive_65k|adaptive_16k|multirhs_65k|multirhs_262k] [--nrhs R]

Workload (default): N = 65,536 points uniform in [0,1]^3, kernel 1/r with
K(x,x) = 0, leaf 128, eta 1, switch level 4, tol 1e-6, adaptive storage from
{fp64, fp32, fp16, bf16}, one fp64 right-hand side U(-1,1); timed next to the
uniform-fp64 H_h matvec of the same compression.  A step is one complete
product y = A_h x (permute in, phase 1, phase 2 with the dense diagonal,
permute out).  The factors (about 1.9 GB adaptive, 3.7 GB fp64) exceed the
L2 cache, so every step streams them from HBM.

Many right-hand sides (--workload multirhs_*): N points U[0,1]^3, Gaussian
kernel exp(-r^2/0.01), leaf 128, eta 1, switch level 5, tol 1e-6, adaptive
storage from {fp64, fp32, bf16, e4m3}, R = 128 right-hand sides N(0,1) (the
262,144-point workload, or the same family at 65,536 points); a step is one
product Y = A_h X of all R columns; the metric is right-hand sides per second.

Multi-GPU (torchrun): every rank runs an independent replica (weak scaling);
the max time over ranks is reported.  --impl reference times the CPU oracle
(oracle/, float64 NumPy) on a bounded sample of the same product.  In the
single right-hand-side line the CPU-baseline leg also compares the product
with the oracle's Algorithm 4 on the rows of eight seeded leaf clusters
("parity": relative error, the 1e-6 tolerance and Theorem 4.4's bound).
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

import hh_workloads as W  # noqa: E402

CACHE = os.environ.get("HH_CACHE_DIR", "/tmp/hh_cache")
WORKLOADS = {
    "adaptive_65k": "N=65,536 points U[0,1]^3, kernel 1/r (K(x,x)=0), leaf 128, eta 1, switch level 4, "
                    "tol 1e-6, adaptive {fp64,fp32,fp16,bf16} vs uniform fp64, 1 RHS U(-1,1)",
    # the same matrix family at N = 16,384 (factors 0.24 GB, still larger
    # than L2): the size used for full ncu captures
    "adaptive_16k": "N=16,384 points U[0,1]^3, kernel 1/r (K(x,x)=0), leaf 128, eta 1, switch level 4, "
                    "tol 1e-6, adaptive {fp64,fp32,fp16,bf16} vs uniform fp64, 1 RHS U(-1,1)",
}
WORKLOAD_N = {"adaptive_65k": 65536, "adaptive_16k": 16384}
MANY_N = {"multirhs_65k": 65536, "multirhs_262k": 262144}
for _k, _n in MANY_N.items():
    WORKLOADS[_k] = (f"N={_n:,} points U[0,1]^3, Gaussian exp(-r^2/0.01), leaf 128, eta 1, switch level 5, "
                     "tol 1e-6, adaptive {fp64,fp32,bf16,e4m3}, R right-hand sides N(0,1) per product")
# the 16/8-bit single-column field alone (its own line; for captures)
LOWBIT_N = {"lowbit_65k": 65536, "lowbit_16k": 16384}
for _k, _n in LOWBIT_N.items():
    WORKLOADS[_k] = (f"N={_n:,} points U[0,1]^3, Gaussian exp(-r^2/0.01), leaf 128, eta 1, switch level 5, "
                     "tol 1e-6, adaptive {fp64,fp32,bf16,e4m3}, 1 RHS N(0,1)")
WORKLOADS["uneven_batch"] = ("64 independent matrices, N log-uniform in [nmin, nmax] (preset [2,048, 131,072]); "
                             "even index 2-D exp(-r) leaf 64, odd index 3-D 1/r leaf 128; eta 1, switch level "
                             "floor(L/2), tol 1e-6, adaptive {fp64,fp32,fp16,bf16}; one RHS U(-1,1) each")
# fp32 FMA issue rate of the CUDA cores: 152 SMs x 128 lanes x 2 flops at the
# 2,070 MHz maximum SM clock
FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops_sustained"]), "measured (sustained)"
    except Exception:
        return 1700.0, "fallback (sustained)"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_matrices(P, torch, rank, ws, dev, workload):
    c = W.CONFIGS["adaptive_65k"]
    pts = W.config_points("adaptive_65k", WORKLOAD_N[workload])
    args = (c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"], c["tol"], W.F64)
    if ws > 1 and rank != 0:
        torch.distributed.barrier()       # rank 0 builds the cache file first
    t0 = time.time()
    H64 = P.HMatrix.build_cached(pts, CACHE, *args, device=dev)
    if ws > 1 and rank == 0:
        torch.distributed.barrier()
    Ham = H64.reencode(c["fmts"], dev)
    return c, pts, H64, Ham, time.time() - t0


def timed_loop(torch, H, x, y, steps, ws):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        H.matvec(x, out=y)
    e1.record(st)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    return e0.elapsed_time(e1)


def max_over_ranks(torch, v, ws):
    """The largest of the ranks' values (on the process group's device)."""
    if ws == 1:
        return v
    dev = "cpu" if torch.distributed.get_backend() == "gloo" else "cuda"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(ws, units_per_rank, t_ms_max):
    """Whole-job throughput of ws independent replicas: every rank processed
    units_per_rank units; the job took the slowest rank's time."""
    return ws * units_per_rank / (t_ms_max / 1000.0)


def traffic_for(kernel: str, algorithmic_bytes: float):
    """DRAM bytes per launch: the traffic / algorithmic-bytes ratio of a
    committed ncu capture (profiles/traffic.json) times this launch's
    algorithmic bytes; None unless the kernel's source is the one captured."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)["kernels"][kernel]
        src = os.path.join(ROOT, "paper_2604_09147_gb300", "csrc", t["source"])
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != t["sha256"]:
                return None
        return float(t["dram_bytes"]) / float(t["algorithmic_bytes"]) * algorithmic_bytes
    except Exception:
        return None


def oracle_sample(path: str, x: np.ndarray, budget_s: float, fraction: float | None = None, keep: bool = False):
    """Time the oracle's Algorithm 4 (float64 NumPy) on a bounded sample:
    whole products while they fit the budget, else a slice of the blocks;
    returns (products per second, description, seconds), and with keep the
    oracle's copy of the matrix as a fourth item."""
    from oracle import hhfile
    from oracle import matvec as M
    G = hhfile.read(path)
    blocks = G.lowrank
    if fraction is None:
        t = time.perf_counter()
        M.matvec(G, x)
        one = time.perf_counter() - t
        fraction = 1.0 if one <= budget_s / 3 else max(0.01, (budget_s / 3) / one)
    nb = max(1, int(round(len(blocks) * fraction)))
    part = G.__class__(**{**G.__dict__, "lowrank": blocks[:nb],
                          "dense": G.dense[:max(1, int(round(len(G.dense) * fraction)))]})
    frac_bytes = (sum(b.k * (b.m + b.n) for b in part.lowrank) + sum(d.m * d.n for d in part.dense)) / \
        max(1.0, sum(b.k * (b.m + b.n) for b in blocks) + sum(d.m * d.n for d in G.dense))
    reps, t0 = 0, time.perf_counter()
    while True:
        M.matvec(part, x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 50:
            break
    rate = reps * frac_bytes / el
    desc = (f"oracle Algorithm 4 in float64 NumPy over {nb} of {len(blocks)} low-rank blocks "
            f"({100 * frac_bytes:.1f}% of the factor+dense words), {reps} passes, {el:.1f} s")
    return (rate, desc, el, G) if keep else (rate, desc, el)


def oracle_sample_1thread(path: str, x: np.ndarray, budget_s: float) -> dict:
    """oracle_sample with NumPy's BLAS held to one thread: a child process
    whose thread-count variables are set before NumPy loads."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    with tempfile.TemporaryDirectory() as d:
        xp = os.path.join(d, "x.npy")
        np.save(xp, x)
        code = ("import sys, json, numpy as np; sys.path.insert(0, %r); import bench; "
                "r, desc, el = bench.oracle_sample(%r, np.load(%r), %r); print(json.dumps([r, desc]))"
                % (ROOT, path, xp, float(budget_s)))
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=max(120.0, 6 * budget_s))
    rate, desc = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": rate, "cores": 1, "kind": "oracle", "sample": desc}


def oracle_rows_check(G, x: np.ndarray, y: np.ndarray, leaves: int = 8, seed: int = 7) -> dict:
    """The product y (user order; one column or n x R) against the oracle's
    Algorithm 4 in float64 over the same stored factors, on the rows of a few
    seeded leaf clusters: every low-rank and dense block whose row cluster
    holds them."""
    L = G.tree.L
    nleaf = 1 << L
    pick = sorted(int(v) for v in np.random.default_rng(seed).choice(nleaf, size=min(leaves, nleaf), replace=False))
    sel = [(int(G.tree.off[nleaf - 1 + v]), int(G.tree.size[nleaf - 1 + v])) for v in pick]
    sel = [(o, z) for o, z in sel if z > 0]
    xt = np.asarray(x, dtype=np.float64)[G.perm]
    yo = [np.zeros((z,) + xt.shape[1:]) for _, z in sel]

    def hits(r0, m):
        return [q for q, (o, z) in enumerate(sel) if r0 <= o and o + z <= r0 + m]
    for b in G.lowrank:
        h = hits(b.row_off, b.m)
        if not h or not b.k:
            continue
        t = b.Vd().T @ xt[b.col_off:b.col_off + b.n]
        U = b.Ud()
        for q in h:
            o, z = sel[q]
            yo[q] += U[o - b.row_off:o - b.row_off + z] @ t
    for d in G.dense:
        for q in hits(d.row_off, d.m):
            o, z = sel[q]
            yo[q] += d.D[o - d.row_off:o - d.row_off + z] @ xt[d.col_off:d.col_off + d.n]
    yu = np.asarray(y, dtype=np.float64)
    num = sum(float(np.sum((yu[G.perm[o:o + z]] - yo[q]) ** 2)) for q, (o, z) in enumerate(sel))
    den = sum(float(np.sum(v ** 2)) for v in yo)
    return {"rel_err": float(np.sqrt(num / den)) if den > 0 else 0.0, "rows": sum(z for _, z in sel),
            "leaf_clusters": len(sel)}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import paper_2604_09147_gb300 as P
    per_step = max(0.5, 120.0 / max(1, args.steps + args.warmup))
    if args.workload in MANY_N or args.workload in LOWBIT_N:
        nr = 1 if args.workload in LOWBIT_N else args.nrhs
        c = W.CONFIGS["multirhs_262k"]
        pts = W.config_points("multirhs_262k", {**MANY_N, **LOWBIT_N}[args.workload])
        H = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"],
                                   c["tol"], c["fmts"], device=-1)
        path = os.path.join(CACHE, f"bench_{args.workload}_ref.hhm")
        H.save(path)
        x = W.config_rhs("multirhs_262k", nrhs=nr, n=len(pts))
        if nr == 1:
            x = x[:, 0]
        rate, desc, el = oracle_sample(path, x, per_step * args.steps)
        if args.workload in LOWBIT_N:
            unit, metric = "matvec/s", "H_h matvecs/s (adaptive precision), HBM GB/s and fraction of peak"
        else:
            rate, unit = rate * nr, "rhs/s"
            metric = "H_h matvec right-hand sides/s (adaptive precision, many right-hand sides)"
            desc += f", {nr} columns per pass"
    else:
        c = W.CONFIGS["adaptive_65k"]
        pts = W.config_points("adaptive_65k", WORKLOAD_N[args.workload])
        H64 = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"],
                                     c["tol"], W.F64, device=-1)
        Ham = H64.reencode(c["fmts"], -1)
        path = os.path.join(CACHE, "bench_adaptive_ref.hhm")
        Ham.save(path)
        x = W.config_rhs("adaptive_65k", n=len(pts))[:, 0]
        rate, desc, el = oracle_sample(path, x, per_step * args.steps)
        unit = "matvec/s"
        metric = "H_h matvecs/s (adaptive precision), HBM GB/s and fraction of peak, vs uniform fp64"
    out = {"impl": "reference", "metric": metric, "value": rate,
           "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000.0 / rate, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload]},
           "cpu_baseline": {"value": rate, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": rate, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def low_bit_field(args, P, torch, rank, ws, dev, clocks=None):
    """Single right-hand side on a matrix with 16- and 8-bit factors:
    N = 65,536 (--low-bit-n) points U[0,1]^3, Gaussian exp(-r^2/0.01), leaf 128,
    eta 1, switch level 5, tol 1e-6, {fp64, fp32, bf16, e4m3} (the
    many-right-hand-side workload's family), one N(0,1) right-hand side.
    Times the streaming passes with their bf16 / e4m3 decoding; reports the
    blocks and bytes per format, GB/s, the HBM fraction per phase and the
    error against the oracle on sampled leaf-cluster rows."""
    c = W.CONFIGS["multirhs_262k"]
    pts = W.config_points("multirhs_262k", args.low_bit_n)
    t0 = time.time()
    H = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"], c["tol"],
                               c["fmts"], device=dev)
    build_s = time.time() - t0
    n = len(pts)
    x0 = W.config_rhs("multirhs_262k", nrhs=1, n=n)[:, 0]
    x = torch.from_numpy(x0.copy()).cuda()
    y = torch.empty_like(x)
    tuned = None if args.no_autotune else H.autotune(0)
    inf = H.info()
    for _ in range(max(3, args.warmup)):
        H.matvec(x, out=y)
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    t = timed_loop(torch, H, x, y, args.steps, ws)
    clk = clocks.stop() if clocks is not None else None
    t = max_over_ranks(torch, t, ws)
    ms = t / args.steps
    hbm, peak_kind = peaks()
    phases = np.mean([H.matvec_timed(x, y) for _ in range(min(args.steps, 100))], axis=0)
    b1, b2 = inf["v_bytes"], inf["u_bytes"] + inf["dense_bytes"]
    out = {"workload": f"N={n:,} points U[0,1]^3, Gaussian exp(-r^2/0.01), leaf 128, eta 1, switch level 5, "
                       "tol 1e-6, adaptive {fp64,fp32,bf16,e4m3}, 1 RHS N(0,1)",
           "ms_per_step": ms, "value": 1e3 / ms, "unit": "matvec/s",
           "gbs": inf["bytes_per_matvec"] / (ms * 1e-3) / 1e9,
           "hbm_frac": inf["bytes_per_matvec"] / (ms * 1e-3) / 1e9 / hbm, "peak_kind": f"of {peak_kind}",
           "blocks_per_fmt": inf["blocks_per_fmt"], "factor_bytes_per_fmt": inf["factor_bytes_per_fmt"],
           "phase_ms": {"prep": phases[0], "phase1": phases[1], "phase2": phases[2], "finish": phases[3]},
           "phase1_hbm_frac": b1 / (phases[1] * 1e-3) / 1e9 / hbm,
           "phase2_hbm_frac": b2 / (phases[2] * 1e-3) / 1e9 / hbm,
           "build_seconds": build_s, "autotune": tuned, "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            from oracle import hhfile
            ya = H.matvec(x).cpu().numpy()
            path = os.path.join(CACHE, "bench_low_bit.hhm")
            H.save(path)
            G = hhfile.read(path)
            out["parity"] = oracle_rows_check(G, x0, ya)
            out["parity"].update({"tol": 1e-6, "bound_thm44": inf["bound_thm44"]})
            del G
        except Exception as e:  # reported, not fatal to the measurement
            out["parity"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_low_bit(args):
    """The 16/8-bit single-column matrix as the line's own workload."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    import paper_2604_09147_gb300 as P
    from paper_2604_09147_gb300 import build as B
    B.build()
    args.low_bit_n = LOWBIT_N[args.workload]
    f = low_bit_field(args, P, torch, rank, ws, dev, clocks=ClockSampler(dev))
    clk = f.pop("clocks")
    out = {"metric": "H_h matvecs/s (adaptive precision), HBM GB/s and fraction of peak",
           "value": ws * f["value"], "unit": "matvec/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": f["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "n": args.low_bit_n, "nrhs": 1,
                      "parallelism": f"replicas x{ws}", "l2": "inputs larger than L2"},
           "gpu_launches": 4 * args.steps, "clocks": clk, "detail": f}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_sharded(args):
    """The adaptive workload's product with its block rows split over the
    ranks (paper_2604_09147_gb300.dist): per step one NCCL all-gather of x and
    each rank's shard product; value = whole products per second (strong
    scaling: the matrix is fixed, each rank holds 1/N of its block rows)."""
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws == 1:  # a single process without torchrun: a one-rank group
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29517")
    dist.init_process_group("nccl", init_method="env://", world_size=ws, rank=rank)
    dev = torch.cuda.current_device()
    import paper_2604_09147_gb300 as P
    from paper_2604_09147_gb300 import build as B
    from paper_2604_09147_gb300.dist import RowSharded
    B.build()
    c = W.CONFIGS["adaptive_65k"]
    pts = W.config_points("adaptive_65k", WORKLOAD_N[args.workload])
    if rank != 0:
        dist.barrier()
    H64 = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"],
                                 c["tol"], W.F64, device=-1)
    if rank == 0:
        dist.barrier()
    Hh = H64.reencode(c["fmts"], -1)                 # host-only whole matrix: plan and shards
    rs = RowSharded(Hh, device=dev)
    n = len(pts)
    x = torch.from_numpy(W.config_rhs("adaptive_65k", n=n)[:, 0].copy()).cuda()
    xl = rs.scatter(x)
    for _ in range(args.warmup):
        rs.matvec(xl)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        rs.matvec(xl)
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    t = max_over_ranks(torch, e0.elapsed_time(e1), ws)
    y = rs.gather(rs.matvec(xl))
    Hfull = H64.reencode(c["fmts"], dev) if rank == 0 else None
    err = None
    if rank == 0:
        ref = Hfull.matvec(x)
        err = float((y - ref).norm() / ref.norm())
    inf = Hh.info()
    out = {"metric": "H_h matvecs/s (adaptive precision), row-sharded over the ranks", "value": args.steps / (t / 1e3),
           "unit": "matvec/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": t / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "n": n, "nrhs": 1, "parallelism": f"row shards x{ws}",
                      "bounds": rs.bounds, "l2": "inputs larger than L2 at N = 1"},
           "gbs": inf["bytes_per_matvec"] / (t / args.steps * 1e-3) / 1e9,
           "rel_err_vs_single_gpu": err, "gpu_launches": 4 * args.steps, "clocks": clk,
           "collective_bytes_per_step": 8 * n}
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist.destroy_process_group()
    return 0


def run_construct(args):
    """Construction time: the adaptive workload's matrix (or the
    differentiation workload's family at --construct-n points, exp(-r),
    {fp64, fp32, bf16}) built with the compression on the GPU (hh_build_dev)
    and, unless --no-host-build, by the host builder; reports both times, the
    device compression's share, blocks left to the host, and the agreement of
    ranks and formats."""
    import torch
    import paper_2604_09147_gb300 as P
    from paper_2604_09147_gb300 import build as B
    B.build()
    dev = torch.cuda.current_device()
    if args.construct_n:
        c = W.CONFIGS["autograd_1m"]
        pts = W.points(args.construct_n, 3, 1234 + c["id"])
        fmts, ell, desc = c["fmts"], -1, (f"N={args.construct_n:,} points U[0,1]^3, exp(-r), leaf 128, eta 1, "
                                           "switch level floor(L/2), tol 1e-6, adaptive {fp64,fp32,bf16}")
    else:
        c = W.CONFIGS["adaptive_65k"]
        pts = W.config_points("adaptive_65k")
        fmts, ell, desc = c["fmts"], c["ell"], WORKLOADS["adaptive_65k"]
    args_b = (c["kernel"], c["kernel_param"], c["leaf"], c["eta"], ell, c["tol"], fmts)
    t0 = time.time()
    Hd = P.HMatrix.build(pts, *args_b, device=dev, construct_on_device=True)
    t_dev = time.time() - t0
    inf = Hd.info()
    out = {"metric": "H_h construction seconds (compression on the GPU vs the host builder)",
           "value": t_dev, "unit": "s", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
           "config": {"workload": desc, "n": len(pts), "host_cores": os.cpu_count()},
           "device_build_seconds": t_dev, "device_compression_seconds": inf["build_device_seconds"],
           "fallback_blocks": inf["build_fallback"], "blocks": inf["n_lowrank"],
           "blocks_per_fmt": inf["blocks_per_fmt"], "bytes_per_matvec": inf["bytes_per_matvec"]}
    if not args.no_host_build:
        t0 = time.time()
        Hh = P.HMatrix.build(pts, *args_b, device=-1)
        out["host_build_seconds"] = time.time() - t0
        out["speedup"] = out["host_build_seconds"] / t_dev
        with tempfile.TemporaryDirectory() as d:
            from oracle import hhfile
            Hh.save(os.path.join(d, "h.hhm"))
            Hd.save(os.path.join(d, "d.hhm"))
            gh, gd = hhfile.read(os.path.join(d, "h.hhm")), hhfile.read(os.path.join(d, "d.hhm"))
        kh = {(b.level, b.i, b.j): (b.k, b.fmt) for b in gh.lowrank}
        dk = np.array([abs(b.k - kh[(b.level, b.i, b.j)][0]) for b in gd.lowrank])
        out["ranks_within_2"] = float(np.mean(dk <= 2))
        out["max_rank_difference"] = int(dk.max()) if len(dk) else 0
        out["formats_equal"] = float(np.mean([b.fmt == kh[(b.level, b.i, b.j)][1] for b in gd.lowrank]))
        out["sum_rank_device_over_host"] = float(sum(b.k for b in gd.lowrank) / max(1, sum(b.k for b in gh.lowrank)))
    print(json.dumps(out), flush=True)
    return 0


def run_solve(args):
    """Conjugate gradients (hh_solve_cg) for (A_h + I) x = b on the
    16/8-bit Gaussian 65k matrix (a symmetric positive definite kernel), to
    a relative residual of 1e-8: the solve's time, its iterations, and the
    time per iteration against one product of the same matrix."""
    import torch
    import paper_2604_09147_gb300 as P
    from paper_2604_09147_gb300 import build as B
    B.build()
    dev = torch.cuda.current_device()
    c = W.CONFIGS["multirhs_262k"]
    pts = W.config_points("multirhs_262k", args.low_bit_n)
    H = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"], c["tol"],
                               c["fmts"], device=dev)
    tuned = None if args.no_autotune else H.autotune(0)
    n = len(pts)
    b = torch.from_numpy(W.rhs(n, 1, "uniform", 4401)[:, 0].copy()).cuda()
    H.solve_cg(b, shift=1.0, rtol=1e-8, max_iter=20)          # warm-up
    torch.cuda.synchronize()
    ts, its = [], 0
    for _ in range(max(1, min(args.steps, 5))):
        t0 = time.perf_counter()
        x, its, res = H.solve_cg(b, shift=1.0, rtol=1e-8, max_iter=2000)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    y = torch.empty_like(b)
    for _ in range(3):
        H.matvec(b, out=y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        H.matvec(b, out=y)
    e1.record()
    torch.cuda.synchronize()
    prod_ms = e0.elapsed_time(e1) / 20
    t = statistics.median(ts)
    out = {"metric": "conjugate-gradient solve seconds, (A_h + I) x = b to 1e-8", "value": t, "unit": "s",
           "n_gpus": 1, "steps": len(ts), "higher_is_better": False, "data": "synthetic",
           "config": {"workload": WORKLOADS["lowbit_65k"] if args.low_bit_n == 65536 else f"n={n}", "n": n,
                      "shift": 1.0, "rtol": 1e-8},
           "iterations": its, "final_relres": res, "ms_per_iteration": 1e3 * t / max(1, its),
           "product_ms": prod_ms, "overhead_per_iteration_ms": 1e3 * t / max(1, its) - prod_ms, "autotune": tuned}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    import paper_2604_09147_gb300 as P
    from paper_2604_09147_gb300 import build as B
    B.build()
    c, pts, H64, Ham, build_s = build_matrices(P, torch, rank, ws, dev, args.workload)
    n = len(pts)
    xh0 = W.config_rhs("adaptive_65k", n=n)[:, 0]
    x = torch.from_numpy(xh0.copy()).cuda()
    y = torch.empty_like(x)
    tuned = None if args.no_autotune else {"adaptive": Ham.autotune(0), "fp64": H64.autotune(0)}
    inf, inf64 = Ham.info(), H64.info()
    for _ in range(args.warmup):
        Ham.matvec(x, out=y)
        H64.matvec(x, out=y)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    t_amp = timed_loop(torch, Ham, x, y, args.steps, ws)
    t_64 = timed_loop(torch, H64, x, y, args.steps, ws)
    clk = clocks.stop()
    t_amp = max_over_ranks(torch, t_amp, ws)
    t_64 = max_over_ranks(torch, t_64, ws)
    Ham.sync_status()
    ms_amp, ms_64 = t_amp / args.steps, t_64 / args.steps
    value = replica_value(ws, args.steps, t_amp)
    hbm, peak_kind = peaks()

    # per-launch device times (CUDA events between the four launches)
    phases = np.zeros(4)
    nph = min(args.steps, 200)
    for _ in range(nph):
        phases += np.array(Ham.matvec_timed(x, y))
    phases /= nph
    bytes_p1 = inf["v_bytes"]
    bytes_p2 = inf["u_bytes"] + inf["dense_bytes"]
    dom = 1 if phases[1] >= phases[2] else 2
    dom_bytes = bytes_p1 if dom == 1 else bytes_p2
    dom_name = "stream_kernel<1,...> (phase 1: t_b = V_b^T x_J)" if dom == 1 else \
        "stream_kernel<2,...> (phase 2: y_I += U_b t_b, dense diagonal)"
    achieved = dom_bytes / (phases[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic_for(f"phase{dom}", dom_bytes), "kernel": dom_name, "peak_kind": f"of {peak_kind}",
                "bytes_per_launch": dom_bytes, "ms_per_launch": float(phases[dom]),
                "phase_ms": {"prep": phases[0], "phase1": phases[1], "phase2": phases[2], "finish": phases[3]}}

    # end to end through the C-ABI from pinned host buffers
    xh = torch.empty(n, dtype=torch.float64, pin_memory=True)
    xh.copy_(x.cpu())
    xnp = xh.numpy()
    ynp = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    e2e_steps = max(3, min(args.steps, 200))
    for _ in range(3):
        Ham.matvec_host(xnp, out=ynp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Ham.matvec_host(xnp, out=ynp)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ws * e2e_steps / max_over_ranks(torch, e2e_s, ws), "unit": "matvec/s",
           "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}

    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        y_amp = Ham.matvec(x).cpu().numpy()
        path = os.path.join(CACHE, "bench_adaptive.hhm")
        Ham.save(path)
        rate, desc, _, G = oracle_sample(path, xh0, args.cpu_seconds, keep=True)
        cpu = {"value": rate, "unit": "matvec/s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc}
        try:  # the same oracle on one thread
            one = oracle_sample_1thread(path, xh0, args.cpu_seconds / 2)
            one["unit"] = "matvec/s"
            cpu["one_thread"] = one
        except Exception as e:  # reported, not fatal to the measurement
            cpu["one_thread"] = {"error": f"{type(e).__name__}: {e}"}
        # the product's error against the oracle, beside the paper's bound
        try:
            parity = oracle_rows_check(G, xh0, y_amp)
        except Exception as e:  # a failed check is reported, not fatal to the measurement
            parity = {"error": f"{type(e).__name__}: {e}"}
        parity.update({"tol": 1e-6, "bound_thm44": inf["bound_thm44"],
                       "vs": "oracle Algorithm 4 (float64) over the same stored factors, sampled leaf-cluster rows"})
        del G

    low_bit = None if args.no_low_bit else low_bit_field(args, P, torch, rank, ws, dev)

    gbs = inf["bytes_per_matvec"] / (ms_amp * 1e-3) / 1e9
    gbs64 = inf64["bytes_per_matvec"] / (ms_64 * 1e-3) / 1e9
    out = {
        "metric": "H_h matvecs/s (adaptive precision), HBM GB/s and fraction of peak, vs uniform fp64",
        "value": value, "unit": "matvec/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_amp, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "dtype_note": "fp32 accumulation for 32/16/8-bit factors; fp64 factors and the dense "
                                      "diagonal as pairs of fp32 halves (about 2^-48); fp64 output scatter",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "n": n, "nrhs": 1, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (factor bytes %.2f GB adaptive / %.2f GB fp64 per step)"
                         % (inf["bytes_per_matvec"] / 1e9, inf64["bytes_per_matvec"] / 1e9)},
        "gbs": gbs, "hbm_frac": gbs / hbm,
        "fp64_uniform": {"value": ws * args.steps / (t_64 / 1000.0), "unit": "matvec/s", "ms_per_step": ms_64,
                         "gbs": gbs64, "hbm_frac": gbs64 / hbm},
        "speedup_vs_fp64": ms_64 / ms_amp,
        "bytes_ratio_fp64_over_amp": inf64["bytes_per_matvec"] / inf["bytes_per_matvec"],
        "storage_ratio_fp64_over_amp": inf["storage_fp64"] / inf["storage_amp"],
        "blocks_per_fmt": inf["blocks_per_fmt"],
        "bound_thm44": inf["bound_thm44"],
        "build_seconds": build_s,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "parity": parity,
        "gpu_launches": 4 * args.steps, "clocks": clk, "autotune": tuned,
        "low_bit_1rhs": low_bit,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def build_many(P, torch, rank, ws, dev, workload):
    c = W.CONFIGS["multirhs_262k"]
    pts = W.config_points("multirhs_262k", MANY_N[workload])
    if ws > 1 and rank != 0:
        torch.distributed.barrier()
    t0 = time.time()
    H = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"], c["tol"],
                               c["fmts"], device=dev)
    if ws > 1 and rank == 0:
        torch.distributed.barrier()
    return c, pts, H, time.time() - t0


def run_many(args):
    """Many right-hand sides: Y = A_h X with R columns per product."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    import paper_2604_09147_gb300 as P
    from paper_2604_09147_gb300 import build as B
    B.build()
    c, pts, H, build_s = build_many(P, torch, rank, ws, dev, args.workload)
    n, R = len(pts), args.nrhs
    X0 = W.config_rhs("multirhs_262k", nrhs=R, n=n)            # (n, R) column-major
    x = torch.from_numpy(np.ascontiguousarray(X0.T)).cuda().t()  # device, column-major
    y = torch.empty((R, n), dtype=torch.float64, device="cuda").t()
    tuned = None if args.no_autotune else H.autotune(R)
    inf = H.info()
    for _ in range(args.warmup):
        H.matvec(x, out=y)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    t_ms = timed_loop(torch, H, x, y, args.steps, ws)
    clk = clocks.stop()
    t_ms = max_over_ranks(torch, t_ms, ws)
    H.sync_status()
    ms = t_ms / args.steps
    value = replica_value(ws, args.steps * R, t_ms)

    # per-launch device times of the sequence (CUDA events around every launch)
    nst = max(3, min(args.steps, 20))
    st = np.mean([H.matvec_stages(x, y) for _ in range(nst)], axis=0)
    names = ["images", "tc_dense", "fp64_streaming", "mr_phase1", "tc_phase1", "mr_phase2", "tc_phase2", "finish"]
    stages = {k: float(v) for k, v in zip(names, st)}
    hbm, peak_kind = peaks()
    bf16, bf16_kind = bf16_peak()
    fmt_b = {"fp32": 4, "fp16": 2, "bf16": 2, "e4m3": 1}
    # Roofline per launch.  The CUDA-core products are bound by the fp32 FMA
    # rate.  The tensor-core phases are bound by HBM: at R columns a stored
    # element carries 2R flop, at R = 128 64 flop/B for fp32 and 128 for
    # bf16 factors, below the bf16 ridge (about 251 flop/B), so their roof
    # is their stored factor bytes at the measured HBM bandwidth; the same
    # algorithmic flops against the bf16 tensor peak are reported beside it.
    # The dense blocks run on the tensor cores as 21 digit products per
    # multiply-add (six 8-bit digits of H and of X, diagonals 0 to 5), in
    # passes of at most 64 columns: their roof is the bf16 tensor peak for
    # the MMA flops issued (128 rows x 16 positions per k-step of an entry,
    # padding included); the fp64-equivalent 2R flop per entry is reported
    # beside it.
    rp_dense = sum((min(64, R - p0) + 15) // 16 * 16 for p0 in range(0, R, 64))
    per = {
        "mr_phase1": ("alu", 2.0 * R * inf["mr_v_elems"], FP32_TFLOPS, "derived fp32 FMA peak"),
        "mr_phase2": ("alu", 2.0 * R * inf["mr_u_elems"], FP32_TFLOPS, "derived fp32 FMA peak"),
        "tc_dense": ("tensor", 21 * 2.0 * rp_dense * inf["dense_tc_elems"], bf16, bf16_kind),
        "tc_phase1": ("hbm", 2.0 * R * inf["tc_v_elems"], bf16, bf16_kind),
        "tc_phase2": ("hbm", 2.0 * R * inf["tc_u_elems"], bf16, bf16_kind),
    }
    # bytes of the stored operands each launch reads once (fp32-equivalent for
    # the CUDA-core phases, whose factors are fp32 here; stored bytes for the
    # tensor-core phases; fp64 for the dense blocks)
    tcb = inf["tc_factor_bytes"]
    tcu = tcb * inf["tc_u_elems"] / max(1, inf["tc_u_elems"] + inf["tc_v_elems"])
    alg_bytes = {"mr_phase1": 4.0 * inf["mr_v_elems"], "mr_phase2": 4.0 * inf["mr_u_elems"],
                 "tc_dense": 8.0 * inf["dense_elems"], "tc_phase1": tcb - tcu, "tc_phase2": tcu}
    detail = {}
    for k, (bound, flops, peak, kind) in per.items():
        t = stages[k] * 1e-3
        tf = flops / t / 1e12 if t > 0 else None
        detail[k] = {"ms": stages[k], "bound": bound, "tflops": tf, "operand_bytes": alg_bytes[k],
                     "operand_gbs": alg_bytes[k] / t / 1e9 if t > 0 else None}
        if bound == "hbm":
            detail[k].update({"hbm_frac": detail[k]["operand_gbs"] / hbm if t > 0 else None,
                              "tensor_frac": tf / peak if t > 0 else None, "tensor_peak_kind": kind})
        elif bound == "tensor":
            detail[k].update({"peak_tflops": peak, "frac": tf / peak if t > 0 else None, "peak_kind": kind,
                              "fp64_equiv_tflops": 2.0 * R * inf["dense_elems"] / t / 1e12 if t > 0 else None})
        else:
            detail[k].update({"peak_tflops": peak, "frac": tf / peak if t > 0 else None, "peak_kind": kind})
    dom = max(per, key=lambda k: stages[k])
    bound, flops, peak, kind = per[dom]
    d = detail[dom]
    if bound == "hbm":
        roofline = {"bound": "hbm", "achieved": d["operand_gbs"], "peak": hbm, "unit": "GB/s",
                    "frac": d["hbm_frac"], "traffic": traffic_for(dom, alg_bytes[dom]), "kernel": dom,
                    "peak_kind": f"of {peak_kind}", "bytes_per_launch": alg_bytes[dom], "ms_per_launch": stages[dom],
                    "tensor": {"achieved": d["tflops"], "peak": peak, "unit": "TFLOP/s", "frac": d["tensor_frac"],
                               "peak_kind": f"of {kind}", "flops_per_launch": flops},
                    "stages": detail}
    else:
        roofline = {"bound": bound, "achieved": d["tflops"], "peak": peak, "unit": "TFLOP/s", "frac": d["frac"],
                    "traffic": traffic_for(dom, alg_bytes[dom]), "kernel": dom, "peak_kind": f"of {kind}",
                    "flops_per_launch": flops, "ms_per_launch": stages[dom], "stages": detail}

    # the same columns through the streaming passes, 4 per product
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, min(3, args.steps))
    e0.record()
    for _ in range(reps):
        for j in range(0, R, 4):
            H.matvec(x[:, j:j + 4], out=y[:, j:j + 4])
    e1.record()
    torch.cuda.synchronize()
    ms_stream = e0.elapsed_time(e1) / reps

    # end to end from pinned host buffers
    xh = torch.empty((R, n), dtype=torch.float64, pin_memory=True)
    xh.copy_(torch.from_numpy(np.ascontiguousarray(X0.T)))
    xnp = xh.numpy().T
    ynp = torch.empty((R, n), dtype=torch.float64, pin_memory=True).numpy().T
    e2e_steps = max(3, min(args.steps, 50))
    H.matvec_host(xnp, out=ynp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        H.matvec_host(xnp, out=ynp)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ws * e2e_steps * R / max_over_ranks(torch, e2e_s, ws), "unit": "rhs/s",
           "h2d_bytes_per_step": 8 * n * R, "d2h_bytes_per_step": 8 * n * R}

    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        Y = H.matvec(x).cpu().numpy()
        path = os.path.join(CACHE, f"bench_{args.workload}.hhm")
        H.save(path)
        rate, desc, _, G = oracle_sample(path, X0, args.cpu_seconds, keep=True)
        cpu = {"value": rate * R, "unit": "rhs/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": desc + f", {R} columns per pass"}
        try:
            parity = oracle_rows_check(G, X0, Y)
        except Exception as e:  # a failed check is reported, not fatal to the measurement
            parity = {"error": f"{type(e).__name__}: {e}"}
        parity.update({"tol": "1e-6 ||Y|| + sum_b w_b |U_b| |V_b|^T |X| over the tensor-core blocks "
                              "(w_b = 2^-20 fp32, 2^-12 16/8-bit)", "bound_thm44": inf["bound_thm44"],
                       "vs": "oracle Algorithm 4 (float64) over the same stored factors, sampled leaf-cluster rows, "
                             "all columns"})
        del G
    # input images, tensor-core phase 1, dense input digits, dense blocks,
    # tensor-core phase 2, output permutation; the CUDA-core phases where
    # they have blocks; three streaming launches per 4 columns of fp64 blocks
    launches = (6 + (inf["mr_v_elems"] > 0) + (inf["mr_u_elems"] > 0)
                + (3 * ((R + 3) // 4) if stages["fp64_streaming"] > 0.002 else 0))
    out = {
        "metric": "H_h matvec right-hand sides/s (adaptive precision, many right-hand sides)",
        "value": value, "unit": "rhs/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "dtype_note": "tensor cores on exact bf16 slices with fp32 accumulation (fp32 factors "
                                      "and input: three slices, six products, accumulators drained every 64 terms; "
                                      "16/8-bit factors: two input slices, drained every 512 terms); CUDA-core fp32 "
                                      "FMA for blocks on unaligned clusters; fp64 dense diagonal on the tensor cores as "
                                      "exact products of six 8-bit digits (about 2^-45 of sum |H||X|); fp64 output",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "n": n, "nrhs": R, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (%.2f GB of factors and dense blocks per step)"
                         % (inf["bytes_per_matvec"] / 1e9)},
        "streaming_4col": {"ms_per_step": ms_stream, "speedup": ms_stream / ms},
        "other_stages_ms": {k: stages[k] for k in ("images", "fp64_streaming", "finish")},
        "blocks_per_fmt": inf["blocks_per_fmt"], "factor_bytes_per_fmt": inf["factor_bytes_per_fmt"],
        "tc_factor_bytes": inf["tc_factor_bytes"], "bound_thm44": inf["bound_thm44"], "build_seconds": build_s,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "parity": parity,
        "gpu_launches": launches * args.steps, "clocks": clk, "autotune": tuned,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """Uneven batch: one product of every matrix per step, as one captured CUDA
    graph of one persistent kernel for the whole batch, next to the
    four-launch graph and to one launch sequence per matrix."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    import paper_2604_09147_gb300 as P
    from paper_2604_09147_gb300 import build as B
    B.build()
    specs = W.uneven_batch(args.batch_count, nmin=args.batch_nmin, nmax=args.batch_nmax)
    t0 = time.time()
    mats = [P.HMatrix.build_cached(sp["points"], CACHE, sp["kernel"], sp["kernel_param"], sp["leaf"], sp["eta"],
                                   sp["ell"], sp["tol"], sp["fmts"], device=dev) for sp in specs]
    build_s = time.time() - t0
    batch = P.HBatch(mats)                      # one persistent cooperative kernel per product
    os.environ["HH_BATCH_LAUNCHES"] = "4"
    try:
        batch4 = P.HBatch(mats)                 # the same as prep, two passes, finish
    finally:
        del os.environ["HH_BATCH_LAUNCHES"]
    xs_h = [sp["x"][:, 0] for sp in specs]
    x = torch.from_numpy(np.concatenate(xs_h)).cuda()
    y = torch.empty_like(x)
    xs = [x[batch.offsets[i]:batch.offsets[i + 1]] for i in range(len(mats))]
    ys = [y[batch.offsets[i]:batch.offsets[i + 1]] for i in range(len(mats))]
    infos = [m.info() for m in mats]
    total_bytes = sum(i["bytes_per_matvec"] for i in infos)
    for _ in range(args.warmup):
        batch.matvec(x, out=y, graph=True)
        for m, xi, yi in zip(mats, xs, ys):
            m.matvec(xi, out=yi)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, steps):
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        return max_over_ranks(torch, e0.elapsed_time(e1), ws)

    clocks = ClockSampler(dev)
    clocks.start()
    batch4.matvec(x, out=y, graph=True)
    t_graph = timed(lambda: batch.matvec(x, out=y, graph=True), args.steps)
    t_seq = timed(lambda: batch.matvec(x, out=y), args.steps)
    t_four = timed(lambda: batch4.matvec(x, out=y, graph=True), args.steps)
    t_each = timed(lambda: [m.matvec(xi, out=yi) for m, xi, yi in zip(mats, xs, ys)], args.steps)
    clk = clocks.stop()
    mats[0].sync_status()
    ms = t_graph / args.steps
    count = len(mats)
    value = replica_value(ws, args.steps * count, t_graph)
    hbm, peak_kind = peaks()
    gbs = total_bytes / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                "kernel": "batch_kernel (prep, phase 1, phase 2, finish in one persistent cooperative kernel)",
                "peak_kind": f"of {peak_kind}", "bytes_per_launch": total_bytes, "ms_per_launch": ms}
    # end to end: pinned host vector in, product, host vector out
    xh = torch.empty_like(x, device="cpu").pin_memory()
    xh.copy_(x.cpu())
    yh = torch.empty_like(xh).pin_memory()
    e2e_steps = max(3, min(args.steps, 200))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        x.copy_(xh, non_blocking=True)
        batch.matvec(x, out=y, graph=True)
        yh.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ws * e2e_steps * count / max_over_ranks(torch, e2e_s, ws), "unit": "matvec/s",
           "h2d_bytes_per_step": 8 * x.numel(), "d2h_bytes_per_step": 8 * x.numel()}
    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle on the largest matrix of the batch, scaled by bytes to the whole batch
        big = max(range(count), key=lambda i: infos[i]["bytes_per_matvec"])
        ybig = y[batch.offsets[big]:batch.offsets[big + 1]].cpu().numpy()  # its part of the last batch product
        path = os.path.join(CACHE, "bench_batch_big.hhm")
        mats[big].save(path)
        rate, desc, _, G = oracle_sample(path, xs_h[big], args.cpu_seconds, keep=True)
        scale = infos[big]["bytes_per_matvec"] / total_bytes
        cpu = {"value": rate * scale * count, "unit": "matvec/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": desc + f"; matrix {big} (N={specs[big]['n']}), scaled by bytes to the batch"}
        try:
            parity = oracle_rows_check(G, xs_h[big], ybig)
        except Exception as e:  # a failed check is reported, not fatal to the measurement
            parity = {"error": f"{type(e).__name__}: {e}"}
        parity.update({"tol": 1e-6, "bound_thm44": infos[big]["bound_thm44"], "matrix": big,
                       "vs": "oracle Algorithm 4 (float64) over the same stored factors, sampled leaf-cluster rows "
                             "of the largest matrix's part of the batch product"})
        del G
    out = {
        "metric": "H_h matvecs/s over an uneven batch (one CUDA graph per batch product)",
        "value": value, "unit": "matvec/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "dtype_note": "fp32 accumulation for 32/16/8-bit factors; fp64 data as fp32 pairs",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["uneven_batch"], "count": count, "nmin": args.batch_nmin,
                   "nmax": args.batch_nmax, "n_total": int(x.numel()), "parallelism": f"replicas x{ws}",
                   "l2": "batch bytes %.2f GB per step" % (total_bytes / 1e9)},
        "one_sequence": {"ms_per_step": t_seq / args.steps},
        "four_launch_graph": {"ms_per_step": t_four / args.steps, "speedup_persistent": t_four / t_graph},
        "per_matrix_launches": {"ms_per_step": t_each / args.steps, "speedup_graph": t_each / t_graph},
        "build_seconds": build_s, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "parity": parity,
        "gpu_launches": args.steps, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    batch4.close()
    batch.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="adaptive_65k")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="CPU oracle baseline time budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["replicas", "sharded", "construct", "solve"], default="replicas",
                    help="replicas: independent products per rank (weak scaling); sharded: the "
                         "adaptive workload's block rows split over the ranks (strong scaling); construct: "
                         "construction time on the GPU against the host builder; solve: conjugate "
                         "gradients on the 16/8-bit Gaussian matrix")
    ap.add_argument("--construct-n", type=int, default=0,
                    help="construct mode: points of the exp(-r) family (0: the adaptive 65k workload)")
    ap.add_argument("--no-host-build", action="store_true", help="construct mode: skip the host builder")
    ap.add_argument("--no-low-bit", action="store_true",
                    help="skip the 16/8-bit single-column field of the default line")
    ap.add_argument("--low-bit-n", type=int, default=65536,
                    help="points of that field's matrix (16,384 for ncu captures)")
    ap.add_argument("--nrhs", type=int, default=128, help="right-hand sides per product (multirhs workloads)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch parameters (for profiling runs with a fixed launch sequence)")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-nmin", type=int, default=2048)
    ap.add_argument("--batch-nmax", type=int, default=131072)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if not 1 <= args.nrhs <= 128:
        ap.error("--nrhs must be between 1 and 128")
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "sharded":
        return run_sharded(args)
    if args.mode == "construct":
        return run_construct(args)
    if args.mode == "solve":
        return run_solve(args)
    if args.workload in MANY_N:
        return run_many(args)
    if args.workload in LOWBIT_N:
        return run_low_bit(args)
    if args.workload == "uneven_batch":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the msRep SpMV hot path on one GB300.

Workload (the SpMV workload the headline metric is quoted on): two FP64
matrices, each in CSR, CSC and COO with int32 indices,
  * R-MAT 2^20 x 2^20 with 2^24 nonzeros (a,b,c,d = .57/.19/.19/.05,
    duplicates summed, values N(0,1)),
  * the 5-point Laplacian of a 2048 x 2048 grid (4,194,304 rows,
    20,963,328 nonzeros),
cut into P nnz-balanced partitions (default P = 148 * 16).

One step = msrep_spmv (partitioned SpMV plus the merge of split rows) for
all six (matrix, format) pairs, inputs resident in HBM.  Partitioning
(pCSR/pCSC/pCOO conversion, Alg. 2/4/6, with the tile plan) is done once per
matrix, timed separately and reported as partition time.  Every matrix is
larger than L2, so no L2 flush is done between steps.

Printed: one JSON line (rank 0) with value = SpMV GFLOP/s (2*nnz per SpMV,
alpha/beta scaling not counted), the HBM roofline of the dominant kernel,
the end-to-end figure through the C ABI with host buffers, the oracle timed
on the host cores, clocks sampled during the timed region, and the
low-precision form (FP32 / BF16 values) on the R-MAT matrix.

--impl reference times the CPU oracle (plain single-threaded FP64 SpMV of
the same workload) instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2209_07552_gb300 import inputs as I  # noqa: E402

FORMATS = ("csr", "csc", "coo")
METRIC = "SpMV GFLOP/s (FP64, R-MAT 2^20 / 2^24 nnz + 2D Laplacian 2048^2, CSR+CSC+COO)"


def algorithmic_bytes(fmt: str, m: int, n: int, nnz: int, sv: int, sx: int) -> int:
    """Compulsory bytes of one SpMV (beta = 0): every nonzero's value and
    index(es), the pointer array, x and y each touched once."""
    if fmt == "csr":
        return (sv + 4) * nnz + 4 * (m + 1) + sx * n + sx * m
    if fmt == "csc":
        return (sv + 4) * nnz + 4 * (n + 1) + sx * n + sx * m
    return (sv + 8) * nnz + sx * n + sx * m


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (every 100 ms)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float) -> float:
    """Largest `value` over all ranks of the default process group (the
    bench reports the slowest rank's step time); the value itself when no
    group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")
_UNIT = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9,
         "nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "second": 1.0,
         "ns": 1e-9, "us": 1e-6, "ms": 1e-3}


# the sources that make the single-matrix SpMV kernels and their tile plans
STAMP_SOURCES = ("csrc/common.cuh", "csrc/tma.cuh", "csrc/spmv_core.cuh", "csrc/spmv.cu",
                 "csrc/partition.cu")


def code_of(text: str) -> str:
    """C/C++/CUDA source without its comments and blank lines (the sources
    hashed by source_stamp hold no comment markers inside string literals),
    so that a change to comments alone leaves the stamp as it is."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def source_stamp() -> str:
    """Hash of the code (comments stripped) of the single-matrix SpMV kernels
    and their tile plans, the public header and the code-generation flags of
    libmsrep.so, independent of where the repository lives."""
    import hashlib
    from paper_2209_07552_gb300 import build as B
    h = hashlib.sha1(" ".join(B.ARCH + [f for f in B.NVCC_FLAGS if not f.startswith("-I")]).encode())
    paths = [os.path.join(os.path.dirname(B.CSRC), p) for p in STAMP_SOURCES]
    paths.append(os.path.join(B.INCLUDE, "msrep.h"))
    for path in paths:
        h.update(os.path.basename(path).encode())
        with open(path, encoding="utf-8") as f:
            h.update(code_of(f.read()).encode())
    return h.hexdigest()


def recorded_traffic(key: str):
    """DRAM bytes (read + write) of one launch of the main kernel of `key`
    ("matrix/format"), from the committed ncu record; None when there is no
    record or the kernels have changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get("kernels", {}).get(key)
    if e is None or e.get("source_stamp") != source_stamp():
        return None
    return e["dram_read_bytes"] + e["dram_write_bytes"]


def record_traffic(csv_path: str, key: str, command: str) -> dict:
    """Adds the DRAM bytes per launch measured by an ncu capture (CSV from
    `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,
    gpu__time_duration.sum --csv --log-file ...`) to the traffic record,
    stamped with the current kernel sources.  With several captured launches
    the last one counts."""
    import csv
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    per = {}
    name = None
    for r in csv.DictReader(lines):
        v = float(r["Metric Value"].replace(",", ""))
        v *= _UNIT.get(r["Metric Unit"].strip().lower(), 1.0)
        per.setdefault(r["ID"], {})[r["Metric Name"]] = v
        name = r["Kernel Name"]
    last = per[max(per, key=int)]
    entry = {"kernel": name.split("(")[0] if name else None,
             "dram_read_bytes": last["dram__bytes_read.sum"],
             "dram_write_bytes": last["dram__bytes_write.sum"],
             "duration_us_under_ncu": last.get("gpu__time_duration.sum", 0.0) * 1e6,
             "source_stamp": source_stamp(), "command": command}
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except (OSError, ValueError):
        d = {"note": "DRAM bytes per launch of each main SpMV kernel, from one ncu "
                     "capture of the profile case; a record counts only while its "
                     "source_stamp matches the kernel sources.", "kernels": {}}
    d["kernels"][key] = entry
    os.makedirs(os.path.dirname(TRAFFIC_FILE), exist_ok=True)
    with open(TRAFFIC_FILE, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
        f.write("\n")
    return entry


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload_config(args, world):
    """The workload both arms report (the reference arm runs the oracle's
    plain SpMV over the same six (matrix, format) pairs)."""
    return {"workload": "rmat20_16Mnnz+laplace2048", "formats": list(FORMATS),
            "P": args.P, "tile": args.tile or 512, "alpha": 1.0, "beta": 0.0,
            "streams": args.streams,
            "l2": "inputs larger than L2 (each matrix 222-403 MB); no flush",
            "parallelism": (f"{world} replicas, one per GPU, no data-path collective"
                            if world > 1 else "single GPU")}


def load_workload():
    return {"rmat": I.rmat_full(), "laplace": I.laplace_full()}


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------

def cpu_oracle_run(mats, budget_s: float):
    """Time the oracle's FP64 SpMV over the workload's (matrix, format)
    pairs, repeating until ~budget_s of CPU work; returns (GFLOP/s, sample)."""
    import oracle as O
    pre = []
    for name, a in mats.items():
        x = I.vector(a.n, I.SEED_BASE + 1)
        c = I.csr_to_csc(a)
        q = I.csr_to_coo(a)
        pre.append((name, "csr", lambda a=a, x=x: O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x), a.nnz))
        pre.append((name, "csc", lambda a=a, c=c, x=x: O.spmv_csc(a.m, a.n, c.col_ptr, c.row_idx, c.val, x), a.nnz))
        pre.append((name, "coo", lambda a=a, q=q, x=x: O.spmv_coo(a.m, q.row_idx, q.col_idx, q.val, x), a.nnz))
    flops = 0.0
    spmvs = 0
    t0 = time.perf_counter()
    while True:
        for name, fmt, fn, nnz in pre:
            fn()
            flops += 2.0 * nnz
            spmvs += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return flops / dt / 1e9, f"{spmvs} single-threaded FP64 SpMVs over the 6 (matrix, format) pairs of the workload, {dt:.1f} s"


def cpu_all_cores_run(mats, budget_s: float):
    """Time the all-core CPU baseline (oracle/cpu_baseline.c: nonzero-balanced
    partitions, one OpenMP thread each, as the paper's Sec. 3.3 gives each
    partition a host thread) over the workload's (matrix, format) pairs,
    repeating until ~budget_s; returns (GFLOP/s, threads, sample)."""
    from oracle import cpu_baseline as C
    pre = []
    for name, a in mats.items():
        x = I.vector(a.n, I.SEED_BASE + 1)
        c = I.csr_to_csc(a)
        q = I.csr_to_coo(a)
        pre.append((C.Prepared("csr", a.m, a.n, a.row_ptr, a.col_idx, a.val), x, a.m))
        pre.append((C.Prepared("csc", a.m, a.n, c.col_ptr, c.row_idx, c.val), x, a.m))
        pre.append((C.Prepared("coo", a.m, a.n, None, q.col_idx, q.val, row_idx=q.row_idx), x,
                    a.m))
    ys = [np.empty(m) for _, _, m in pre]
    for (P, x, _), y in zip(pre, ys):  # first touch of the scratch, untimed
        P.run(x, y)
    flops, spmvs = 0.0, 0
    t0 = time.perf_counter()
    while True:
        for (P, x, _), y in zip(pre, ys):
            P.run(x, y)
            flops += 2.0 * P.nnz
            spmvs += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    th = C.threads()
    return (flops / dt / 1e9, th,
            f"{spmvs} FP64 SpMVs on {th} threads (nonzero-balanced partitions, one per "
            f"thread) over the 6 (matrix, format) pairs of the workload, {dt:.1f} s")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    mats = load_workload()
    budget = max(3.0, min(60.0, 2.0 * args.steps))
    val, sample = cpu_oracle_run(mats, budget)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, 1),
        "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": 1,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def partition_overhead(part_ms, part_local_ms, kern):
    """Partitioning as a share of partition + one SpMV (the paper's measure
    of partitioning overhead, Sec. 5, with the matrix already on the
    device, so nothing is distributed), without and with the local
    pointers materialised."""
    out = {}
    for k, t in part_ms.items():
        spmv_ms = kern[k]["call_us"] * 1e-3
        tl = part_local_ms[k]
        out[k] = {"ms": t, "ms_with_local": tl, "spmv_ms": spmv_ms,
                  "pct": 100.0 * t / (t + spmv_ms),
                  "pct_with_local": 100.0 * tl / (tl + spmv_ms)}
    return out


def run_ours(args):
    import torch

    import paper_2209_07552_gb300 as M
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P = args.P

    mats = load_workload()
    pairs = []   # (name, fmt, A, part, x, y, ws, nnz, bytes)
    part_ms, part_local_ms = {}, {}
    for name, a in mats.items():
        xh = I.vector(a.n, I.SEED_BASE + 1)
        x = torch.from_numpy(xh).to(dev)
        for fmt in FORMATS:
            A = M.DeviceMatrix.from_host(a, fmt, "f64", device=dev)
            part = M.DevicePartition(A, P, tile=args.tile, device=dev)
            # partition time (the pCSR/pCSC/pCOO conversion incl. tile plan)
            for _ in range(2):
                M.msrep_partition(A, part)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            e0.record()
            for _ in range(reps):
                M.msrep_partition(A, part)
            e1.record()
            torch.cuda.synchronize()
            part_ms[f"{name}/{fmt}"] = e0.elapsed_time(e1) / reps
            # the same with the local row/column pointers (pCOO: the local
            # row-index array, one entry per nonzero) materialised
            part_l = M.DevicePartition(A, P, tile=args.tile, local=True, device=dev)
            M.msrep_partition(A, part_l)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                M.msrep_partition(A, part_l)
            e1.record()
            torch.cuda.synchronize()
            part_local_ms[f"{name}/{fmt}"] = e0.elapsed_time(e1) / reps
            del part_l
            y = torch.empty(a.m, dtype=torch.float64, device=dev)
            ws = M.alloc_workspace(A, part, device=dev)
            nb = algorithmic_bytes(fmt, a.m, a.n, a.nnz, 8, 8)
            pairs.append((name, fmt, A, part, x, y, ws, a.nnz, nb))
    del mats

    # The step's SpMVs are independent problems.  With --streams 2 each
    # matrix's three SpMVs run in order on a stream of their own, so one
    # matrix's small kernels (fix-up, prepare, gather) overlap the other's
    # main kernel; the timed region still spans every SpMV of every step.
    main = torch.cuda.current_stream()
    lanes = [torch.cuda.Stream() for _ in range(args.streams)] if args.streams > 1 else [main]
    names = sorted({p[0] for p in pairs})
    fork, joins = torch.cuda.Event(), [torch.cuda.Event() for _ in lanes]

    def step():
        if len(lanes) > 1:
            fork.record(main)
            for ln in lanes:
                ln.wait_event(fork)
        for (name, _, A, part, x, y, ws, _, _) in pairs:
            ln = lanes[names.index(name) % len(lanes)]
            M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws, stream=ln)
        if len(lanes) > 1:
            for ln, j in zip(lanes, joins):
                j.record(ln)
                main.wait_event(j)

    flops_step = sum(2.0 * p[7] for p in pairs)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.step_only:
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
        if rank == 0:
            ms = ev0.elapsed_time(ev1) / args.steps
            print(json.dumps({"step_only": True, "ms_per_step": ms,
                              "gflops": flops_step / (ms * 1e-3) / 1e9}), flush=True)
        return
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
        # per-kernel timing of the main SpMV kernels (profiling events)
        kern = {}
        reps = max(20, min(args.steps, 200))
        for (name, fmt, A, part, x, y, ws, nnz, nb) in pairs:
            ks = main_kernel_stats(
                M, lambda: M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws), reps)
            k_us = ks["median"]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws)
            e1.record()
            torch.cuda.synchronize()
            kern[f"{name}/{fmt}"] = {"kernel_us": k_us, "kernel_us_mean": ks["mean"],
                                     "kernel_reps": reps,
                                     "call_us": 1e3 * e0.elapsed_time(e1) / reps,
                                     "bytes": nb, "nnz": nnz}
            fl = access_floor_us(M, A, x, reps)
            if fl is not None:
                kern[f"{name}/{fmt}"].update(fl)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    value = flops_step * world / (ms_step * 1e-3) / 1e9

    # roofline of the dominant kernel (largest kernel time in the step)
    peak, peak_kind = measured_peaks()
    dom_key = max(kern, key=lambda k: kern[k]["kernel_us"])
    d = kern[dom_key]
    achieved = d["bytes"] / (d["kernel_us"] * 1e-6) / 1e9
    roof = {"bound": "hbm", "kernel": dom_key, "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic(dom_key)}
    if "floor_us" in d:
        # the same arrays streamed with only the gathers / scatters, no row
        # logic (msrep_access_floor): the bound the access pattern sets
        roof["access_floor"] = {"us": d["floor_us"], "mode": d["floor_mode"],
                                "gbs": d["bytes"] / (d["floor_us"] * 1e-6) / 1e9,
                                "kernel_frac_of_floor": d["floor_us"] / d["kernel_us"]}
    for k, v in kern.items():
        v["gbs"] = v["bytes"] / (v["kernel_us"] * 1e-6) / 1e9
        v["frac"] = v["gbs"] / peak
    part_over = partition_overhead(part_ms, part_local_ms, kern)

    # end to end through the C ABI with host buffers: x up, SpMV, y down
    e2e = run_e2e(M, pairs, args, dev)
    # the served stream runs first among the extra legs, on a device and
    # host that the other legs' large allocations have not touched yet
    serving = run_serving(M, args, dev) if args.serve_seconds > 0 else None
    p_sweep = run_p_sweep(M, pairs, args) if not args.skip_p_sweep else None
    coo_orders = run_coo_orders(M, args, dev, kern, peak) if not args.skip_coo_orders else None
    stream_tma = run_stream_tma(M, pairs, kern, peak) if not args.skip_stream_tma else None
    imbalance = run_imbalance(M, args, dev) if not args.skip_imbalance else None

    # low-precision form on every (matrix, format) pair
    prec = run_precision(M, args, dev, kern) if not args.skip_precision else None
    batched = run_batched(M, args, dev) if args.batched_count > 0 else None

    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded R-MAT and 2D Laplacian)",
        "config": workload_config(args, world),
        "roofline": roof,
        "per_kernel": kern,
        "partition_ms": part_ms,
        "partition_overhead": part_over,
        "coo_orders": coo_orders,
        "e2e": e2e,
        # CSR and COO: main kernel + fix-up kernel; CSC: prepare (zero y or
        # the permuted accumulator) + main kernel + gather of y
        "gpu_launches": args.steps * sum(2 if p[1] != "csc" else 3 for p in pairs),
        "clocks": clk.summary(),
    }
    if p_sweep:
        line["p_sweep"] = p_sweep
    if imbalance:
        line["imbalance"] = imbalance
    if stream_tma:
        line["stream_tma"] = stream_tma
    if prec:
        line["precision"] = prec
    if batched:
        line["batched"] = batched
    if serving:
        line["serving"] = serving
    if rank == 0 and not args.no_cpu_baseline:
        mats = load_workload()
        v, sample = cpu_oracle_run(mats, args.cpu_budget)
        line["cpu_baseline"] = {"value": v, "unit": "GFLOP/s", "cores": 1,
                                "kind": "oracle", "sample": sample}
        va, th, sample_a = cpu_all_cores_run(mats, args.cpu_budget)
        line["cpu_baseline_all_cores"] = {"value": va, "unit": "GFLOP/s", "cores": th,
                                          "kind": "openmp nonzero-partitioned SpMV",
                                          "sample": sample_a}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_p_sweep(M, pairs, args, Ps=(148, 148 * 4, 148 * 16, 148 * 64), reps=20):
    """Main-kernel time of every (matrix, format) pair at P = 148 .. 148*64
    partitions (the sweep of the partition count), FP64, default tile; for
    CSR and CSC also with row+nonzero merge-path cuts ("<P>_merge_path")."""
    out = {}
    for (name, fmt, A, _, x, y, _, _, _) in pairs:
        row = {}
        variants = [(0, "")]
        if fmt in ("csr", "csc"):
            variants.append((M.MSREP_PART_MERGE_PATH, "_merge_path"))
        for P in Ps:
            for pflags, tag in variants:
                part = M.DevicePartition(A, P, tile=args.tile, device=x.device)
                M.msrep_partition(A, part, pflags)
                ws = M.alloc_workspace(A, part, device=x.device)
                for _ in range(3):
                    M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws)
                row[f"{P}{tag}"] = main_kernel_us(
                    M, lambda: M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws), reps)
                del part, ws
        out[f"{name}/{fmt}"] = row
    return {"kernel_us": out, "P": list(Ps)}


def main_kernel_stats(M, call, reps, skip=3):
    """Median and mean CUDA-event time (us) of the main SpMV kernel over
    `reps` back-to-back calls of `call`.  Each call gets its own pair of
    profiling events, recorded on the launch stream just before and just
    after its main kernel.  The calls are not synchronised one by one: the
    host stays ahead of the device, so no host submission latency falls
    inside an event pair.  The first `skip` calls, which the idle device may
    reach before the host has queued their kernels, are dropped."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps + skip)]
    torch.cuda.synchronize()
    for s0, s1 in evs:
        M.native.msrep_profile_events(s0, s1)
        call()
    M.native.msrep_profile_events(None, None)
    torch.cuda.synchronize()
    ts = sorted(1e3 * s0.elapsed_time(s1) for s0, s1 in evs[skip:])
    n = len(ts)
    med = ts[n // 2] if n % 2 else 0.5 * (ts[n // 2 - 1] + ts[n // 2])
    return {"median": med, "mean": sum(ts) / n}


def main_kernel_us(M, call, reps, skip=3):
    """Median CUDA-event time (us) of the main SpMV kernel (see
    main_kernel_stats)."""
    return main_kernel_stats(M, call, reps, skip)["median"]


def access_floor_us(M, A, x, reps):
    """Time of msrep_access_floor over the matrix's own index and value
    arrays: a gather of x per nonzero (CSR; COO also streams its row index),
    the faster of eight consecutive nonzeros a lane and lane-interleaved
    steps, or an atomic add per nonzero (CSC, the faster of scattering to
    y's rows and to the permuted accumulator); every mode's time is kept.
    None when a vector length is not a power of two."""
    import torch
    if A.fmt == M.MSREP_CSC:
        n_vec, modes, idx2 = A.m, (2, 3), None
    else:
        # eight consecutive nonzeros a lane, and lane-interleaved steps
        n_vec, modes = A.n, ((1, 5) if A.fmt == M.MSREP_COO else (0, 4))
        idx2 = A.idx2
    if n_vec & (n_vec - 1):
        return None
    vec = x if A.fmt != M.MSREP_CSC else torch.zeros(n_vec, dtype=torch.float64, device=x.device)
    sink = torch.zeros(1, dtype=torch.float64, device=x.device)
    best = None
    by_mode = {}
    for mode in modes:
        for _ in range(2):
            M.native.msrep_access_floor(mode, A.idx, A.val, vec, idx2=idx2, sink=sink)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            M.native.msrep_access_floor(mode, A.idx, A.val, vec, idx2=idx2, sink=sink)
        e1.record()
        torch.cuda.synchronize()
        us = 1e3 * e0.elapsed_time(e1) / reps
        by_mode[str(mode)] = us
        if best is None or us < best[0]:
            best = (us, mode)
    return {"floor_us": best[0], "floor_mode": best[1], "floor_us_by_mode": by_mode}


def run_e2e(M, pairs, args, dev):
    import torch
    hx, hy = {}, {}
    # every pair gets its own device x (the formats of one matrix share x in
    # the device-resident step; here their uploads overlap)
    pairs = [(name, fmt, A, part, torch.empty_like(x), y, ws, nnz, nb)
             for (name, fmt, A, part, x, y, ws, nnz, nb) in pairs]
    for (name, fmt, A, part, x, y, ws, nnz, nb) in pairs:
        hx[(name, fmt)] = torch.empty(x.numel(), dtype=torch.float64).pin_memory()
        hx[(name, fmt)].copy_(torch.from_numpy(I.vector(x.numel(), I.SEED_BASE + 1)))
        hy[(name, fmt)] = torch.empty(y.numel(), dtype=torch.float64).pin_memory()
    h2d = sum(x.numel() * 8 for (_, _, _, _, x, _, _, _, _) in pairs)
    d2h = sum(y.numel() * 8 for (_, _, _, _, _, y, _, _, _) in pairs)

    # Three streams pipeline the step: the upload of pair i+1's x and the
    # download of pair i-1's y overlap the SpMV of pair i (separate copy
    # engines).  Events order each pair's upload -> SpMV -> download, and
    # keep the next step from overwriting x (y) before the SpMV (download)
    # that reads it has finished.
    up, comp, down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: [torch.cuda.Event() for _ in pairs] for k in ("x_in", "x_used", "y_out", "y_read")}
    started = [False] * len(pairs)

    def step():
        for i, (name, fmt, A, part, x, y, ws, _, _) in enumerate(pairs):
            with torch.cuda.stream(up):
                if started[i]:
                    up.wait_event(ev["x_used"][i])
                x.copy_(hx[(name, fmt)], non_blocking=True)
                ev["x_in"][i].record(up)
            comp.wait_event(ev["x_in"][i])
            if started[i]:
                comp.wait_event(ev["y_read"][i])
            M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws, stream=comp)
            ev["x_used"][i].record(comp)
            ev["y_out"][i].record(comp)
            with torch.cuda.stream(down):
                down.wait_event(ev["y_out"][i])
                hy[(name, fmt)].copy_(y, non_blocking=True)
                ev["y_read"][i].record(down)
            started[i] = True
    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    # the host copies of y must equal the device results of the last step
    for (name, fmt, A, part, x, y, ws, _, _) in pairs:
        if not torch.equal(hy[(name, fmt)], y.cpu()):
            raise RuntimeError(f"e2e: host y of {name}/{fmt} differs from the device result")
    flops = sum(2.0 * p[7] for p in pairs)
    return {"value": flops / dt / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3,
            "pipeline": "uploads, SpMVs and downloads on three streams"}


def run_batched(M, args, dev):
    """The batched form: 512 uneven FP32 CSR matrices (rows log-uniform in
    [1e3, 2e5], geometric row lengths with mean U(4, 64)), autotuned, one
    persistent launch plus fix-up, captured in a CUDA graph; timed by graph
    replays.  Bytes per launch: the FP32 CSR formula summed over matrices."""
    import torch
    t0 = time.time()
    mats, xs = I.batched_set_parallel(args.batched_count)
    gen_s = time.time() - t0
    D = [M.DeviceMatrix.from_host(a, "csr", "f32", device=dev) for a in mats]
    X = [torch.from_numpy(x).to(dev) for x in xs]
    Y = [torch.empty(a.m, dtype=torch.float32, device=dev) for a in mats]
    nnz = sum(a.nnz for a in mats)
    nbytes = sum(algorithmic_bytes("csr", a.m, a.n, a.nnz, 4, 4) for a in mats)
    t0 = time.time()
    tune = M.msrep_autotune(D, X, Y, device=dev)
    tune_s = time.time() - t0
    B = M.DeviceBatch(D, X, Y, tune, device=dev)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        for _ in range(3):
            B.run(stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.run(stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / reps
    peak, _ = measured_peaks()
    tiles = {}
    for b in range(32):
        tiles[b] = (int(tune.tile[b]), int(tune.part_nnz[b]))
    used = sorted({int(np.log2(max(a.nnz, 1))) for a in mats})
    return {"matrices": len(mats), "nnz": nnz, "launch_us": us,
            "gflops": 2.0 * nnz / (us * 1e-6) / 1e9,
            "gbs": nbytes / (us * 1e-6) / 1e9, "frac": nbytes / (us * 1e-6) / 1e9 / peak,
            "bytes_per_launch": nbytes, "total_tiles": B.total_tiles,
            "tune": {str(b): tiles[b] for b in used}, "cta_threads": int(tune.cta_threads),
            "gen_s": gen_s, "autotune_s": tune_s,
            "graph": "one CUDA graph: persistent batched kernel + fix-up"}


def run_serving(M, args, dev):
    """The served form: 64 matrices drawn like the batched set plus two 2^20
    R-MAT matrices (16.8M nonzeros each); a Poisson stream of requests
    (args.serve_rate per second for args.serve_seconds, the first second
    discarded), each naming a matrix uniformly and carrying k ~ U{1..8}
    FP32 vectors.  Latency is submit -> y in the caller's host buffer,
    measured by the server, which also splits it into queue wait (submit
    -> packed into a launch) and device time per launch.  Run twice: under
    a 60 GB budget (everything fits) and under a budget of the launch
    contexts plus 25% of the set's bytes, so that admission binds (the
    matrices that do not fit are rejected; the stream names admitted
    ones)."""
    seed = I.SEED_BASE + 4
    mats, _ = I.batched_set_parallel(64, seed=seed)
    mats = list(mats) + [I.rmat_full(), I.cached_csr(f"rmat20_{seed}", lambda: I.rmat(seed=seed))]
    g = I.rng(seed, 300)
    X = []
    for a in mats:   # page-locked inputs, as a serving front end would hold them
        xa = M.native.pinned_empty((8, a.n))
        xa[:] = I.to_f32(g.uniform(-1, 1, (8, a.n)))
        X.append(xa)
    cfg = dict(arena_bytes=256 << 20, contexts=args.serve_contexts, max_items=512,
               device=dev.index or 0)
    # Page-locked y buffers for every matrix, carved from one slab allocated
    # up front (48 per matrix, each large enough for 8 vectors): the load
    # driver waits for the request that last used a buffer before reusing
    # it, so the pool must outlast the slowest request (48 buffers a matrix
    # are reused about every 160 ms at 20,000 requests/s over 66 matrices);
    # with fewer, one slow request stalled the open-loop driver and the
    # stall bunched the following submissions.
    per = 48
    sizes = [8 * a.m for a in mats]
    slab = M.native.pinned_empty((per * sum(sizes),))
    pools, o = [], 0
    for sz in sizes:
        pools.append([slab[o + i * sz:o + (i + 1) * sz] for i in range(per)])
        o += per * sz
    full = serve_once(M, mats, X, 60 << 30, cfg, args, seed, pools)
    with M.Server(budget_bytes=60 << 30, **cfg) as S0:
        ctx_bytes = S0.stats()["resident_bytes"]
    budget = ctx_bytes + (full["resident_bytes_after_register"] - ctx_bytes) // 4
    quarter = serve_once(M, mats, X, budget, cfg, args, seed + 1, pools)
    full["budget_25pct"] = quarter
    full["y_buffers_per_matrix"] = per
    del slab
    return full


def serve_once(M, mats, X, budget, cfg, args, seed, all_pools):
    """One served stream under `budget`: register every matrix (those that
    do not fit are not admitted), then replay the Poisson stream with the
    library's native driver (msrep_serve_replay), which submits each
    request at its arrival time from one native thread; request i writes
    into the next of its matrix's page-locked y buffers and, before that,
    the replay waits for the request that last used that buffer."""
    S = M.Server(budget_bytes=budget, **cfg)
    ids = []
    for j, a in enumerate(mats):
        try:
            ids.append((j, S.register(a)))
        except M.MsrepError as e:
            if e.status != 6:      # MSREP_ERR_BUDGET: not admitted
                raise
    not_admitted = S.stats()["rejected"]
    resident = S.stats()["resident_bytes"]
    g = I.rng(seed, 301)
    arrivals = I.poisson_arrivals(args.serve_rate, args.serve_seconds, seed)
    n = arrivals.shape[0]
    pick = g.integers(0, len(ids), n)
    ks = g.integers(1, 9, n).astype(np.int32)
    mids = np.empty(n, np.int64)
    xs, ys = [], []
    reuse = np.full(n, -1, np.int64)
    used = {}
    count = {}
    for i in range(n):
        j, mid = ids[int(pick[i])]
        mids[i] = mid
        xs.append(X[j][:int(ks[i])])
        c = count.get(j, 0)
        slot = c % len(all_pools[j])
        count[j] = c + 1
        ys.append(all_pools[j][slot])
        reuse[i] = used.get((j, slot), -1)
        used[(j, slot)] = i
    warm = min(1.0, 0.2 * args.serve_seconds)
    late, lag = S.replay(arrivals * 1e6, mids, ks, xs, ys, reuse, reset_after_us=warm * 1e6)
    st = S.stats()
    S.close()
    st.update({"offered_rate": n / args.serve_seconds, "requests": n,
               "late_submissions": late, "max_submit_lag_us": lag,
               "driver": "msrep_serve_replay (native, open loop)",
               "matrices": len(mats), "admitted": len(ids), "not_admitted": not_admitted,
               "window_s": args.serve_seconds, "discarded_warmup_s": warm,
               "budget_bytes": budget, "resident_bytes_after_register": resident})
    return st


def run_precision(M, args, dev, kern):
    """The low-precision form on both workload matrices in CSR, CSC and COO:
    values stored FP32 and BF16, x and y FP32.  Per (matrix, format, type):
    main-kernel time (median of CUDA-event pairs), GB/s and fraction of the
    HBM peak on the form's own algorithmic bytes, speedup of the kernel over
    the FP64 kernel of the same pair (per_kernel), and the normwise error of
    y against the FP64 oracle on the original FP64 values and x (computed on
    the host, outside any timed region), with the tolerance it must meet.
    Also k = 8 vectors on the FP32 R-MAT CSR matrix (msrep_spmm)."""
    import torch

    import oracle as O
    peak, _ = measured_peaks()
    tol = {"f32": 1e-5, "bf16": 1e-2}
    out = {}
    for name, a in load_workload().items():
        xh = I.vector(a.n, I.SEED_BASE + 1)
        y_ref = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, xh)
        nref = float(np.linalg.norm(y_ref))
        x = torch.from_numpy(I.to_f32(xh)).to(dev)
        for fmt in FORMATS:
            row = {}
            f64_us = kern[f"{name}/{fmt}"]["kernel_us"]
            for dt in ("f32", "bf16"):
                A = M.DeviceMatrix.from_host(a, fmt, dt, device=dev)
                part = M.DevicePartition(A, args.P, tile=args.tile, device=dev)
                M.msrep_partition(A, part)
                y = torch.empty(a.m, dtype=torch.float32, device=dev)
                ws = M.alloc_workspace(A, part, device=dev)
                call = lambda: M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws)
                for _ in range(3):
                    call()
                ks = main_kernel_stats(M, call, 20)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(20):
                    call()
                e1.record()
                torch.cuda.synchronize()
                sv = {"f32": 4, "bf16": 2}[dt]
                nb = algorithmic_bytes(fmt, a.m, a.n, a.nnz, sv, 4)
                err = float(np.linalg.norm(y.cpu().numpy().astype(np.float64) - y_ref)) / nref
                row[dt] = {"kernel_us": ks["median"], "kernel_us_mean": ks["mean"],
                           "call_us": 1e3 * e0.elapsed_time(e1) / 20, "bytes": nb,
                           "gbs": nb / (ks["median"] * 1e-6) / 1e9,
                           "frac": nb / (ks["median"] * 1e-6) / 1e9 / peak,
                           "speedup_vs_f64": f64_us / ks["median"],
                           "normwise_err_vs_oracle_f64": err, "tolerance": tol[dt],
                           "within_tolerance": err <= tol[dt]}
                if name == "rmat" and fmt == "csr" and dt == "f32":
                    out["f32_k8"] = run_spmm_leg(M, A, part, a, xh, dev, row[dt]["call_us"])
                del A, part, y, ws
            out[f"{name}/{fmt}"] = row
        torch.cuda.synchronize()
    return out


def run_spmm_leg(M, A, part, a, xh, dev, spmv_call_us, k=8):
    """k = 8 right-hand sides on the FP32 R-MAT matrix with msrep_spmm (the
    matrix read once, the 8 values of a column gathered together) against 8
    separate msrep_spmv calls; effective GFLOP/s = 2 * nnz * k / time."""
    import torch
    X = torch.from_numpy(np.stack([np.roll(xh, v) for v in range(k)])).to(dev, torch.float32)
    Y = torch.empty((k, a.m), dtype=torch.float32, device=dev)
    ws = torch.empty(M.msrep_spmm_workspace_size(A, part, k), dtype=torch.uint8, device=dev)
    for _ in range(3):
        M.msrep_spmm(A, part, 1.0, X, 0.0, Y, workspace=ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record()
    for _ in range(reps):
        M.msrep_spmm(A, part, 1.0, X, 0.0, Y, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / reps
    return {"k": k, "call_us": us, "gflops": 2.0 * a.nnz * k / (us * 1e-6) / 1e9,
            "speedup_vs_k_spmv": k * spmv_call_us / us}


def run_imbalance(M, args, dev):
    """The imbalance experiment of Sec. 2.3 (Fig. 5) on one GPU, with thread
    blocks in place of GPUs: B partitions, one thread block each
    (MSREP_SCHED_PER_PARTITION), B = the number of SMs, so that every
    partition runs at once on an SM of its own, as the paper's partitions
    run on GPUs of their own.  The matrix has
    2^20 rows in B equal row blocks; rows of the first half of the blocks
    hold 32 nonzeros, the others 32 / r (the paper's two-level nonzero
    distribution, low-to-high ratio 1/r).  Per r: the SpMV over the
    Baseline row-block partitioning (Sec. 5.1, MSREP_PART_ROW_BLOCK) and
    over Alg. 2's nonzero-balanced partitioning and over the row+nonzero
    merge-path partitioning (which also balances the rows, whose ends cost
    the CSR kernel work too), all one block per partition, and the
    row-block partitioning under the default schedule (every partition's
    tiles spread over all blocks).  CSR, FP64."""
    import torch
    m, heavy = 1 << 20, 32
    # one partition per SM: each thread block has its SM to itself, as each
    # of the paper's partitions has its GPU
    B = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {"rows": m, "partitions": B, "heavy_row_nnz": heavy, "ratios": {}}
    for r in (1, 2, 4, 10):
        a = I.block_imbalance_matrix(m, B, heavy, r, I.SEED_BASE + 5 + r)
        x = torch.from_numpy(I.vector(a.n, I.SEED_BASE + 1)).to(dev)
        y = torch.empty(a.m, dtype=torch.float64, device=dev)
        A = M.DeviceMatrix.from_host(a, "csr", "f64", device=dev)
        row = {"nnz": a.nnz, "light_row_nnz": a.meta["light_len"]}
        for tag, pflags, flags in (("row_block_per_partition", M.MSREP_PART_ROW_BLOCK,
                                    M.MSREP_SCHED_PER_PARTITION),
                                   ("nnz_balanced_per_partition", 0, M.MSREP_SCHED_PER_PARTITION),
                                   ("merge_path_per_partition", M.MSREP_PART_MERGE_PATH,
                                    M.MSREP_SCHED_PER_PARTITION),
                                   ("row_block_default_schedule", M.MSREP_PART_ROW_BLOCK, 0)):
            part = M.DevicePartition(A, B, device=dev)
            M.msrep_partition(A, part, pflags)
            h = part.to_host()
            ln = (h["end_idx"].astype(np.int64) - h["start_idx"] + 1)
            ws = M.alloc_workspace(A, part, device=dev)
            call = lambda: M.msrep_spmv(A, part, 1.0, x, 0.0, y, flags=flags, workspace=ws)
            for _ in range(3):
                call()
            us = main_kernel_us(M, call, 20)
            row[tag] = {"kernel_us": us, "gflops": 2.0 * a.nnz / (us * 1e-6) / 1e9,
                        "max_partition_nnz": int(ln.max()), "mean_partition_nnz": float(ln.mean())}
            del part, ws
        rb, nb = row["row_block_per_partition"], row["nnz_balanced_per_partition"]
        mp = row["merge_path_per_partition"]
        row["row_block_over_balanced_perf"] = nb["kernel_us"] / rb["kernel_us"]
        row["row_block_over_merge_path_perf"] = mp["kernel_us"] / rb["kernel_us"]
        out["ratios"][str(r)] = row
        del A, x, y
    return out


def run_coo_orders(M, args, dev, kern, peak):
    """pCOO of the workload's matrices sorted by column and in no order
    (Sec. 3.2.3; their SpMV is a scatter): main-kernel and call time, GB/s
    against COO's algorithmic bytes, and the result against the row-sorted
    COO product of the same matrix (normwise)."""
    import torch
    out = {}
    for name, a in (("rmat", I.rmat_full()), ("laplace", I.laplace_full())):
        x = torch.from_numpy(I.vector(a.n, I.SEED_BASE + 1)).to(dev)
        A0 = M.DeviceMatrix.from_host(a, "coo", "f64", device=dev)
        p0 = M.DevicePartition(A0, args.P, device=dev)
        M.msrep_partition(A0, p0)
        y_ref = torch.empty(a.m, dtype=torch.float64, device=dev)
        M.msrep_spmv(A0, p0, 1.0, x, 0.0, y_ref, workspace=M.alloc_workspace(A0, p0, device=dev))
        del A0, p0
        for fmt in ("coo_col", "coo_any"):
            A = M.DeviceMatrix.from_host(a, fmt, "f64", device=dev)
            part = M.DevicePartition(A, args.P, device=dev)
            M.msrep_partition(A, part)
            ws = M.alloc_workspace(A, part, device=dev)
            y = torch.empty(a.m, dtype=torch.float64, device=dev)
            for _ in range(3):
                M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws)
            reps = 50
            k_us = main_kernel_us(
                M, lambda: M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws), reps)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws)
            e1.record()
            torch.cuda.synchronize()
            nb = algorithmic_bytes("coo", a.m, a.n, a.nnz, 8, 8)
            c_us = 1e3 * e0.elapsed_time(e1) / reps
            d = torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref)
            out[f"{name}/{fmt}"] = {
                "kernel_us": k_us, "call_us": c_us, "bytes": nb,
                "gbs": nb / (k_us * 1e-6) / 1e9, "frac": nb / (k_us * 1e-6) / 1e9 / peak,
                "row_sorted_coo_kernel_us": kern[f"{name}/coo"]["kernel_us"],
                "normwise_vs_row_sorted": float(d)}
            del A, part, ws
    return out


def run_stream_tma(M, pairs, kern, peak, reps=20):
    """The bulk-copy (TMA) staging variant (MSREP_STREAM_TMA) of each main
    kernel of the step, on the step's own problems: main-kernel time beside
    the direct-load kernel's, and its result against the direct kernel's
    (bit-equal for CSR and COO, normwise for CSC, whose atomic adds land in
    another order)."""
    import torch
    out = {}
    for (name, fmt, A, part, x, y, ws, nnz, nb) in pairs:
        key = f"{name}/{fmt}"
        M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=ws)
        y_direct = y.clone()
        try:
            for _ in range(3):
                M.msrep_spmv(A, part, 1.0, x, 0.0, y, flags=M.MSREP_STREAM_TMA, workspace=ws)
        except M.MsrepError as e:   # e.g. a tile above the variant's 512
            out[key] = {"unsupported": str(e)}
            continue
        torch.cuda.synchronize()
        if fmt == "csc":
            check = {"normwise_vs_direct": float(torch.linalg.norm(y - y_direct)
                                                 / torch.linalg.norm(y_direct))}
        else:
            check = {"bit_equal_to_direct": bool(torch.equal(y, y_direct))}
        k_us = main_kernel_us(M, lambda: M.msrep_spmv(A, part, 1.0, x, 0.0, y,
                                                       flags=M.MSREP_STREAM_TMA, workspace=ws),
                              reps)
        d_us = kern[key]["kernel_us"]
        out[key] = {"kernel_us": k_us, "direct_kernel_us": d_us, "stream_over_direct": k_us / d_us,
                    "gbs": nb / (k_us * 1e-6) / 1e9, "frac": nb / (k_us * 1e-6) / 1e9 / peak,
                    **check}
        del y_direct
    # a bounded wait of the streaming kernels that gave up is reported here
    try:
        M.native.msrep_device_status()
        out["waits_gave_up"] = False
    except M.MsrepError:
        out["waits_gave_up"] = True
    return out


def run_profile_case(args):
    """A short fixed case for ncu captures: partition the R-MAT matrix once,
    then `--reps` calls of msrep_spmv in one format and value type."""
    import torch

    import paper_2209_07552_gb300 as M
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.profile == "batched":
        # uneven FP32 CSR matrices drawn like the batched workload, autotuned,
        # `--reps` batched launches
        mats, xs = I.batched_set_parallel(args.profile_batch_count)
        D = [M.DeviceMatrix.from_host(a, "csr", "f32", device=dev) for a in mats]
        X = [torch.from_numpy(x).to(dev) for x in xs]
        Y = [torch.empty(a.m, dtype=torch.float32, device=dev) for a in mats]
        tune = M.msrep_autotune(D, X, Y, device=dev)
        B = M.DeviceBatch(D, X, Y, tune, device=dev)
        for _ in range(args.reps):
            B.run()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "batched", "matrices": len(mats),
                          "nnz": sum(a.nnz for a in mats), "cta_threads": int(tune.cta_threads),
                          "reps": args.reps}))
        return
    a = I.rmat_full() if args.profile_matrix == "rmat" else I.laplace_full()
    dt = args.profile_dtype
    A = M.DeviceMatrix.from_host(a, args.profile, dt, device=dev)
    part = M.DevicePartition(A, args.P, tile=args.tile, device=dev)
    M.msrep_partition(A, part)
    xt = torch.float64 if dt == "f64" else torch.float32
    x = torch.from_numpy(I.vector(a.n, I.SEED_BASE + 1)).to(dev, xt)
    y = torch.empty(a.m, dtype=xt, device=dev)
    ws = M.alloc_workspace(A, part, device=dev)
    flags = M.MSREP_STREAM_TMA if args.stream_tma else 0
    if args.profile_floor:
        # the access-pattern floor kernel on the same arrays
        vec = x if args.profile != "csc" else torch.zeros(a.m, dtype=torch.float64, device=dev)
        mode = {"csr": 0, "coo": 1, "csc": 3}[args.profile]
        for _ in range(args.reps):
            M.native.msrep_access_floor(mode, A.idx, A.val, vec, idx2=A.idx2)
    elif args.profile_k > 0:
        # k right-hand sides (CSR): msrep_spmm on k shifted copies of x
        X = torch.stack([torch.roll(x, v) for v in range(args.profile_k)])
        Y = torch.empty((args.profile_k, a.m), dtype=xt, device=dev)
        wk = torch.empty(M.msrep_spmm_workspace_size(A, part, args.profile_k),
                         dtype=torch.uint8, device=dev)
        for _ in range(args.reps):
            M.msrep_spmm(A, part, 1.0, X, 0.0, Y, flags=flags, workspace=wk)
        y = Y[0]
    else:
        for _ in range(args.reps):
            M.msrep_spmv(A, part, 1.0, x, 0.0, y, flags=flags, workspace=ws)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile, "stream_tma": args.stream_tma, "matrix": args.profile_matrix,
                      "dtype": dt, "reps": args.reps, "P": args.P,
                      "y_norm": float(torch.linalg.norm(y.double()))}))


def run_sweep(args):
    """Kernel time of every (matrix, format, tile, P) combination (FP64),
    one JSON line each; used to choose the defaults."""
    import torch

    import paper_2209_07552_gb300 as M
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    peak, _ = measured_peaks()
    mats = load_workload()
    fmts = args.sweep_formats.split(",")
    for name, a in mats.items():
        x = torch.from_numpy(I.vector(a.n, I.SEED_BASE + 1)).to(dev)
        y = torch.empty(a.m, dtype=torch.float64, device=dev)
        for fmt in fmts:
            A = M.DeviceMatrix.from_host(a, fmt, "f64", device=dev)
            nb = algorithmic_bytes(fmt, a.m, a.n, a.nnz, 8, 8)
            tiles = [int(t) for t in args.sweep_tiles.split(",")]
            Ps = [int(q) for q in args.sweep_P.split(",")]
            modes = [True] if args.sweep_direct_only else [False, True]
            for tile, P, direct in [(t, p, d) for t in tiles for p in Ps
                                    for d in modes if d or t <= 512]:
                    flags = 0 if direct else M.MSREP_STREAM_TMA
                    part = M.DevicePartition(A, P, tile=tile, device=dev)
                    M.msrep_partition(A, part)
                    ws = M.alloc_workspace(A, part, device=dev)
                    for _ in range(3):
                        M.msrep_spmv(A, part, 1.0, x, 0.0, y, flags=flags, workspace=ws)
                    us = main_kernel_us(M, lambda: M.msrep_spmv(A, part, 1.0, x, 0.0, y,
                                                                 flags=flags, workspace=ws), 10)
                    print(json.dumps({"matrix": name, "fmt": fmt, "tile": tile, "P": P,
                                      "direct": direct, "kernel_us": us, "gbs": nb / us / 1e3,
                                      "frac": nb / us / 1e3 / peak}), flush=True)
            del A


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--P", type=int, default=148 * 16)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--streams", type=int, default=1, choices=[1, 2],
                    help="streams the step's independent SpMVs are spread over")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-precision", action="store_true")
    ap.add_argument("--skip-p-sweep", action="store_true",
                    help="skip the P = 148 .. 148*64 sweep of the main kernels")
    ap.add_argument("--skip-imbalance", action="store_true",
                    help="skip the row-block imbalance experiment")
    ap.add_argument("--skip-coo-orders", action="store_true",
                    help="skip the column-sorted / unsorted COO leg")
    ap.add_argument("--skip-stream-tma", action="store_true",
                    help="skip the bulk-copy (TMA) staging variant's leg")
    ap.add_argument("--batched-count", type=int, default=512,
                    help="matrices in the batched-form measurement (0 = skip)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the served request stream (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-contexts", type=int, default=4,
                    help="launch contexts of the server (launches in flight at once)")
    ap.add_argument("--step-only", action="store_true",
                    help="run only the timed step (for an ncu launch list of the step)")
    ap.add_argument("--profile-batch-count", type=int, default=64,
                    help="matrices of the batched profile case")
    ap.add_argument("--profile", choices=FORMATS + ("coo_col", "coo_any", "batched"), default=None,
                    help="run only a short fixed case (for ncu captures)")
    ap.add_argument("--profile-matrix", choices=["rmat", "laplace"], default="rmat")
    ap.add_argument("--profile-dtype", choices=["f64", "f32", "bf16"], default="f64")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--profile-floor", action="store_true",
                    help="profile case: the access-pattern floor kernel instead of the SpMV")
    ap.add_argument("--profile-k", type=int, default=0,
                    help="profile case: msrep_spmm with this many vectors (CSR) instead of msrep_spmv")
    ap.add_argument("--stream-tma", action="store_true",
                    help="bulk-copy staging kernels (MSREP_STREAM_TMA) in the profile case")
    ap.add_argument("--record-traffic", metavar="NCU_CSV", default=None,
                    help="store the DRAM bytes of an ncu capture of the profile case "
                         "(--profile, --profile-matrix select the key)")
    ap.add_argument("--record-command", default="",
                    help="the ncu command line that wrote NCU_CSV (kept with the record)")
    ap.add_argument("--sweep", action="store_true", help="time every (format, tile, P)")
    ap.add_argument("--sweep-formats", default="csr,csc,coo")
    ap.add_argument("--sweep-tiles", default="256,512,1024")
    ap.add_argument("--sweep-P", default="148,2368")
    ap.add_argument("--sweep-direct-only", action="store_true")
    args = ap.parse_args()
    if args.record_traffic:
        key = f"{args.profile_matrix}/{args.profile or 'csr'}"
        print(json.dumps({key: record_traffic(args.record_traffic, key, args.record_command)}))
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.profile:
        run_profile_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

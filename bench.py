#!/usr/bin/env python
"""Benchmark of the sparse-embedding least-squares hot path on GB300.

Workload (the large sparse regression configuration): CSR A with n = 2^24 rows,
d = 256 columns, exactly 16 distinct columns per row drawn from Zipf(1.1),
N(0,1) float32 values, b = A x0 + 0.01 N(0,1); CountSketch with m = 65536
rows (hash seed 1); least squares by LSQR preconditioned with R from SA, to
the relative normal-equation residual 1e-6.

One step = one call of cw_lsqr_precond: hash + bucket sort + SA/Sb + R + the
sketch-and-solve start + LSQR iterations, i.e. every step of the path on one
synthetic input already resident in HBM.  value = nnz(A) processed per second
(summed over ranks).  e2e = the same through the C ABI with the CSR arrays and
b copied from pinned host memory every step and x copied back.

Under torchrun each rank solves its own replica (weak scaling; the path needs
no collective when problems are independent).  ``--impl reference`` times the
float64 CPU oracle on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("SA nnz/s and HBM GB/s vs peak; solve time at residual ratio ≤1+ε, learned vs plain sketch")
WORKLOAD = ("large sparse regression: CSR n=2^24 x d=256, 16 distinct Zipf(1.1) columns/row, N(0,1) fp32, "
            "b=A x0+0.01 noise, CountSketch m=65536 seed 1, LSQR preconditioned by R from SA to rtol 1e-6")
N_ROWS, D, K_NNZ, ZIPF_S, M, SEED, RTOL = 1 << 24, 256, 16, 1.1, 65536, 1, 1e-6
DATA_SEED_A, DATA_SEED_B = 1002, 2002
SAMPLE_ROWS_CPU = 1 << 22   # cpu_baseline leg: rows of the same workload
SAMPLE_ROWS_REFERENCE = 1 << 20  # --impl reference: rows per step

# kernels reported in the stage breakdown, with their algorithmic bytes per launch
# (a function of the workload): each byte of A read once, vectors read/written once
def _alg_bytes(kernel, n, d, nnz, m):
    if kernel == "k_lsqr_pass":
        # col + val, row_ptr, z (or b) read, z written
        return nnz * 8 + (n + 1) * 4 + n * 4 + n * 4
    if kernel == "k_apply_csr":
        # col + val gathered once, SA and Sb written
        return nnz * 8 + m * d * 4 + m * 4
    if kernel == "k_coarse_scatter":
        # row_ptr and b read (the per-row records it writes are sort overhead)
        return (n + 1) * 4 + n * 4
    return None


# bytes each sketch kernel actually has to move (algorithmic + the sort's own
# records): the per-kernel bandwidth figure reported beside the algorithmic one
def _moved_bytes(kernel, n, d, nnz, m):
    if kernel == "k_coarse_scatter":
        return (n + 1) * 4 + n * 4 + n * 16
    if kernel == "k_fine_sort":
        return n * 16 * 2 + n * 12 + m * 4
    if kernel == "k_apply_csr":
        return nnz * 8 + n * 12 + m * d * 4 + m * 4 + m * 4
    return None


TIMED_KERNELS = ("k_lsqr_pass", "k_apply_csr", "k_coarse_scatter", "k_fine_sort", "k_tile_hist",
                 "k_lsqr_post_mc", "k_chol_small", "k_chol_panel", "k_chol_update", "k_tri_inv_f32", "k_gram_to_f32", "k_chol_finish",
                 "k_lsqr_start", "k_gram_tile", "k_gram_tc", "k_gram_tc_reduce", "k_gram_gemv", "k_qr_householder", "k_qr_blocked", "k_scan_tiles", "k_scan_bins",
                 "k_scan_chunk_sums", "k_trsm_upper", "k_trsv_upper", "k_gram_reduce", "k_tri_inverse",
                 "k_transpose64", "k_upper_matvec", "k_to_f32_transposed", "k_set_last",
                 "k_tri_diag_inv", "k_tri_inv_blk")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("cw", "reference"), default="cw")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rows", type=int, default=N_ROWS,
                    help="rows of A (a smaller case of the same workload for profiler captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the per-step timings of the other rows")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-regression row")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-sketch row")
    ap.add_argument("--only-qr", type=int, nargs=2, default=None, metavar=("M", "D"),
                    help="only time the float64 QR of an M x D Gaussian SA (profiling)")
    ap.add_argument("--only-batch", type=int, default=0,
                    help="only plan and run the first N problems of the batched workload (profiling)")
    ap.add_argument("--oracle-worker", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-sketch-worker", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-steps", type=int, default=1, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------- distributed plumbing

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(x, world, device=None):
    """Largest value of x over all ranks (plain float for world == 1)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device=None):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples every 100 ms while running; stop()
    keeps the samples taken between mark_start() and mark_end() (all samples if
    none fall inside)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "cw_clocks_%d_%d.csv" % (os.getpid(), gpu_index))
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # wait (at most 5 s) for the first sample so the timed region is covered
        t_end = time.time() + 5.0
        while time.time() < t_end and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                sm = float(parts[2].split()[0])
                mx = float(parts[3].split()[0])
            except ValueError:
                continue
            rs = {nm for nm, v in zip(names, parts[6:10]) if v.lower().startswith("active")}
            rows.append((ts, sm, mx, rs))
        os.unlink(self.path)
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 <= r[0] <= self.t1]
        use = inside or rows
        if not use:
            return None
        reasons = set()
        for r in use:
            reasons |= r[3]
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "samples": len(use), "samples_in_timed_region": len(inside), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- peaks and profiles

def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources each profiled kernel is built from: a capture stays valid until they change
KERNEL_SOURCES = {"k_lsqr_pass": ("lsqr_pass.cuh", "cw_common.cuh"),
                  "k_apply_csr": ("sketch.cu", "sketch_body.cuh", "cw_common.cuh")}


def source_hash(kernel=None):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1207_6365_gb300", "csrc")
    names = KERNEL_SOURCES.get(kernel) or sorted(os.listdir(csrc))
    for name in names:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch recorded by an ncu capture of the current sources, else None."""
    path = os.path.join(ROOT, "profiles", "%s__large_sparse.md" % kernel)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    mh = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    mt = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not mh or not mt or mh.group(1) != source_hash(kernel):
        return None
    return float(mt.group(1))


# ---------------------------------------------------------------- workload

def make_problem(device, rows=N_ROWS, replica=0):
    import workloads as W
    A = W.csr_zipf(rows, D, K_NNZ, ZIPF_S, seed=DATA_SEED_A + 7919 * replica, device=device)
    b, _ = W.rhs(A, 0.01, seed=DATA_SEED_B + 7919 * replica)
    return A, b


# ---------------------------------------------------------------- oracle (CPU) timing

def oracle_step(A_np, b_np, d, m, seed, rtol):
    """The float64 CPU oracle's version of one step; returns LSQR iterations."""
    import oracle
    rp, col, val = A_np
    SA, Sb = oracle.sketch_csr(rp, col, val, d, b_np, m, seed)
    x0, R = oracle.solve_sketch(SA, Sb)
    x, it, test, conv, _ = oracle.lsqr_precond_csr(rp, col, val, d, b_np, R, x0, rtol, 100)
    return it


def oracle_worker(rows, steps):
    """Runs in a child process with single-threaded BLAS; prints one JSON line."""
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A, b = make_problem(dev, rows=rows)
    A_np = A.numpy()
    b_np = b.cpu().numpy()
    import oracle
    oracle.build()
    ts, its = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        its.append(oracle_step(A_np, b_np, D, M, SEED, RTOL))
        ts.append(time.perf_counter() - t0)
    nnz = int(A_np[0][-1])
    print(json.dumps({"rows": rows, "nnz": nnz, "times": ts, "iters": its}))


def oracle_sketch_worker(rows, reps):
    """Runs in a child process: the all-core float64 oracle sketch (SA and Sb,
    rows sorted by bucket, buckets summed in parallel) on the workload's first
    `rows` rows; prints one JSON line."""
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A, b = make_problem(dev, rows=rows)
    rp, col, val = A.numpy()
    b_np = b.cpu().numpy()
    del A, b
    import oracle
    oracle.build()
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.sketch_csr_parallel(rp, col, val, D, b_np, M, SEED, threads=threads)
        ts.append(time.perf_counter() - t0)
    print(json.dumps({"rows": rows, "nnz": int(rp[-1]), "times": ts, "threads": threads}))


def run_oracle_sketch_child(rows, reps):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sketch-worker", str(rows),
                          "--oracle-steps", str(reps)], env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle sketch worker failed:\n" + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_oracle_child(rows, steps):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", str(rows),
                          "--oracle-steps", str(steps)], env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle worker failed:\n" + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def host_info():
    """The host the oracle ran on: logical CPUs, CPUs this process may use, CPU model."""
    info = {"nproc": os.cpu_count()}
    try:
        info["affinity"] = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        pass
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                key = key.strip().lower()
                if key in ("model name", "cpu model"):
                    model = val.strip()
                    break
                if key == "cpu part" and model is None:
                    model = "Arm CPU part " + val.strip()
    except OSError:
        pass
    info["cpu"] = model or platform.machine()
    return info


def cpu_baseline_block(res, sample_desc):
    tot = sum(res["times"])
    return {"value": res["nnz"] * len(res["times"]) / tot, "unit": "nnz/s", "cores": 1, "kind": "oracle",
            "sample": sample_desc, "seconds": tot, "lsqr_iters": res["iters"][-1], "host": host_info()}


# ---------------------------------------------------------------- main arms

def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    steps, warm = max(1, args.steps), max(0, args.warmup)
    res = run_oracle_child(SAMPLE_ROWS_REFERENCE, steps + warm)
    res["times"] = res["times"][warm:]
    sample = ("first 2^20 rows of the workload per step (same d, m, seed, Zipf columns, rtol); float64 CPU "
              "oracle: C sketch loop, LAPACK QR, LSQR with C matvecs; 1 thread")
    cb = cpu_baseline_block(res, sample)
    v = cb["value"]
    ms = 1000.0 * sum(res["times"]) / len(res["times"])
    line = {"metric": METRIC, "value": v, "unit": "nnz/s", "n_gpus": world, "steps": steps, "warmup": warm,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_rows": SAMPLE_ROWS_REFERENCE, "n": N_ROWS, "d": D,
                       "m": M, "rtol": RTOL},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _timed(fn, stream, reps=3, warm=1):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def segment_read_rates(cw, stream, device):
    """Read throughput (GB/s) of 64-byte segments at random places of a 2 GiB
    array (larger than L2), issued like the segmented sum's row gathers, and of
    the same kernel on consecutive segments; the better of 4 and 8 CTAs per SM."""
    import torch
    a = torch.ones(1 << 29, dtype=torch.float32, device=device)
    nseg = a.numel() // 16
    out = torch.zeros(1, dtype=torch.float32, device=device)
    res = {}
    for key, seq in (("random_64B_GBps", False), ("sequential_64B_GBps", True)):
        best = 0.0
        for k in (4, 8):
            ms = _timed(lambda: cw.probe_gather64(a, nseg, seq, k, out), stream, reps=3, warm=1)
            best = max(best, nseg * 64 / (ms / 1000.0) / 1e9)
        res[key] = best
    del a
    return res


def with_sa_sketch(roofline, sketch_roofline):
    """The dominant kernel's roofline with the SA sketch's own figures nested
    under "sa_sketch" (cw_sketch_csr alone: time, achieved GB/s and fraction of
    the copy peak on its algorithmic bytes, the segment read rates), so that a
    record keeping only the line's standard keys keeps them too."""
    if roofline is None or not sketch_roofline:
        return roofline
    keep = ("call", "ms", "achieved", "frac", "alg_bytes_per_call", "nnz_per_s", "traffic",
            "segment_read_rates", "apply_gather_GBps", "apply_frac_of_random_64B")
    out = dict(roofline)
    out["sa_sketch"] = {k: sketch_roofline[k] for k in keep if k in sketch_roofline}
    return out


def _stage_ms(cw, names, reps):
    out = {}
    for nm in names:
        cnt, tot = cw.profile_get(nm)
        if cnt:
            out[nm] = tot / reps
    return out


def row_timings(cw, A, b, stream, peak):
    """Per-call times of the method's other steps (CUDA events on the launching
    stream; per-kernel times from the library's own events).  The dense rows use
    a Gaussian A of the dense-sketch workload's shape (n = 2^22, d = 512; for
    timing only: the kernels' work does not depend on the values)."""
    import torch
    rows = {}
    reps = 3
    SA = torch.empty(M, D, device=A.row_ptr.device)
    Sb = torch.empty(M, device=A.row_ptr.device)
    sort_k = ("k_tile_hist", "k_scan_chunk_sums", "k_scan_bins", "k_scan_tiles", "k_coarse_scatter", "k_fine_sort",
              "k_set_last")
    cw.profile_reset()
    cw.profile_enable(True)
    ms = _timed(lambda: cw.cw_sketch_csr(A, b, M, SEED, SA, Sb), stream, reps=reps, warm=0)
    cw.profile_enable(False)
    st = _stage_ms(cw, sort_k + ("k_apply_csr",), reps)
    rows["A1_A2_hash_sort_ms"] = sum(v for k, v in st.items() if k in sort_k)
    rows["A3_segmented_sum_ms"] = st.get("k_apply_csr")
    rows["A1_A3_sketch_csr_ms"] = ms
    rows.update(tiny_latency(cw, stream))
    rows["A4_qr_fp64_ms"] = _timed(lambda: cw.cw_qr(SA, Sb), stream, reps=2)
    rows["A5_sketch_and_solve_ms"] = _timed(lambda: cw.cw_solve_sketch(A, b, M, SEED), stream, reps=2)
    # generalized sparse embedding: q = 1024 blocks, v = 16, kappa = 4 (t = 65536 rows, as SA above)
    gq, gv, gk = 1024, 16, 4
    rows["N4_general_sketch_ms"] = _timed(lambda: cw.cw_sketch_csr_general(A, b, gq, gv, gk, SEED, SA, Sb), stream,
                                          reps=reps)
    rows["N4_general_sketch_config"] = "q=%d, v=%d, kappa=%d on the large sparse matrix" % (gq, gv, gk)
    del SA, Sb
    # dense rows: n = 2^22, d = 512, m = 65536, k = 32
    n3, d3, k3 = 1 << 22, 512, 32
    g = torch.Generator(device=A.row_ptr.device).manual_seed(1003)
    A3 = torch.randn(n3, d3, device=A.row_ptr.device, generator=g)
    G3 = torch.randn(d3, k3, device=A.row_ptr.device, dtype=torch.float64, generator=g)
    SA3 = torch.empty(M, d3, device=A.row_ptr.device)
    ms = _timed(lambda: cw.cw_sketch_dense(A3, None, M, SEED, SA3), stream, reps=reps)
    ab = n3 * d3 * 4 + M * d3 * 4
    rows["A3_sketch_dense_ms"] = ms
    rows["A3_sketch_dense_GBps"] = ab / (ms / 1000.0) / 1e9
    rows["A3_sketch_dense_frac"] = rows["A3_sketch_dense_GBps"] / peak
    # NEXT-2: sketch with values and its backward on the same dense A (one pass over A each)
    vals = torch.randn(n3, device=A.row_ptr.device, generator=g)
    gS = torch.randn(M, d3, device=A.row_ptr.device, generator=g)
    ms = _timed(lambda: cw.cw_sketch_dense_values(A3, None, M, SEED, vals, SA3), stream, reps=reps)
    rows["N2_values_forward_dense_ms"] = ms
    rows["N2_values_forward_dense_frac"] = (ab + n3 * 4) / (ms / 1000.0) / 1e9 / peak
    gv = torch.empty(n3, device=A.row_ptr.device)
    ms = _timed(lambda: cw.cw_sketch_values_backward_dense(A3, None, M, SEED, gS, None, gv), stream, reps=reps)
    bb = n3 * d3 * 4 + M * d3 * 4 + n3 * 4
    rows["N2_values_backward_dense_ms"] = ms
    rows["N2_values_backward_dense_GBps"] = bb / (ms / 1000.0) / 1e9
    rows["N2_values_backward_dense_frac"] = rows["N2_values_backward_dense_GBps"] / peak
    del SA3, vals, gS, gv
    lev_k = ("k_apply_dense_precise", "k_qr_blocked", "k_qr_householder", "k_qr_finalize", "k_trsm_upper",
             "k_m_digits", "k_leverage_tc", "k_leverage")
    cw.cw_leverage(A3, M, SEED, G3)
    torch.cuda.synchronize()
    cw.profile_reset()
    cw.profile_enable(True)
    ms = _timed(lambda: cw.cw_leverage(A3, M, SEED, G3), stream, reps=2, warm=0)
    cw.profile_enable(False)
    st = _stage_ms(cw, lev_k, 2)
    rows["A7_leverage_total_ms"] = ms
    rows["A7_stages_ms"] = st
    lk = "k_leverage_tc" if "k_leverage_tc" in st else ("k_leverage" if "k_leverage" in st else None)
    if lk:
        lb = n3 * d3 * 4 + n3 * 4
        rows["A7_leverage_pass_kernel"] = lk
        rows["A7_leverage_pass_GBps"] = lb / (st[lk] / 1000.0) / 1e9
        rows["A7_leverage_pass_frac"] = rows["A7_leverage_pass_GBps"] / peak
        # bf16 products actually issued: 15 digit pairs of 2 n d k flops (tensor path)
        if lk == "k_leverage_tc":
            rows["A7_leverage_tc_TFLOPs"] = 15 * 2.0 * n3 * d3 * k3 / (st[lk] / 1000.0) / 1e12
    rows["dense_workload"] = "A: n=2^22 x d=512 float32 N(0,1) (timing only), m=65536, G: 512 x 32, seed 1"
    del A3, G3
    torch.cuda.empty_cache()
    rows.update(leverage_error_row(cw))
    return rows


def tiny_latency(cw, stream, calls=50):
    """The tiny sketch-and-solve configuration: CSR n = 65536, d = 32, 8 uniform
    distinct columns per row, b = A x0 + 0.1 noise, m = 4096, seed 1.  Latency of
    one cw_solve_sketch call (sketch, float64 QR, solve; it returns after x' is
    on the device) as the caller sees it (host wall clock, median of `calls`),
    and of the sketch alone (CUDA events)."""
    import torch
    import workloads as W
    A = W.csr_uniform(65536, 32, 8, seed=1001, device="cuda")
    b, _ = W.rhs(A, 0.1, seed=2001)
    b = b.cuda()
    for _ in range(3):
        cw.cw_solve_sketch(A, b, 4096, 1)
    torch.cuda.synchronize()
    wall = []
    for _ in range(calls):
        t0 = time.perf_counter()
        cw.cw_solve_sketch(A, b, 4096, 1)
        torch.cuda.synchronize()
        wall.append((time.perf_counter() - t0) * 1e6)
    sk_us = 1000.0 * _timed(lambda: cw.cw_sketch_csr(A, b, 4096, 1), stream, reps=20, warm=3)
    return {"C1_solve_sketch_us": statistics.median(wall), "C1_solve_sketch_us_min": min(wall),
            "C1_sketch_csr_us": sk_us,
            "C1_workload": "CSR n=65536, d=32, 8 uniform distinct columns/row, m=4096, seed 1"}


def leverage_error_row(cw, sample=1 << 16):
    """The dense leverage configuration: A = U diag(sigma) V^T, n = 2^22, d = 512,
    U and V Haar, sigma geometric from 1 to 1e-6 (kappa = 1e6), m = 65536,
    G 512 x 32.  The library's leverage scores against the float64 oracle's
    same algorithm (its own sketch of the stored A, its own QR, the same G) on
    `sample` rows drawn uniformly (seed 9)."""
    import numpy as np
    import torch
    import oracle
    import workloads as W
    t0 = time.perf_counter()
    n, d, k = 1 << 22, 512, 32
    A = W.dense_lowrank(n, d, W.geometric_sigma(d, 1e-6), seed=1003, device="cuda")
    G = W.gaussian(d, k, seed=2)
    lev = cw.cw_leverage(A, M, SEED, G.cuda())
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0
    A_h = A.cpu().numpy()
    lev_h = lev.cpu().double().numpy()
    del A, lev
    torch.cuda.empty_cache()
    t1 = time.perf_counter()
    SA_o, _ = oracle.sketch_dense(A_h, None, M, SEED)
    R_o, _ = oracle.qr_r(SA_o)
    rows = np.random.default_rng(9).choice(n, size=sample, replace=False)
    lev_o = oracle.leverage_same(A_h, R_o, G.numpy(), rows=rows)
    rel = np.abs(lev_h[rows] - lev_o) / lev_o
    return {"C3_leverage_rel_err_max": float(rel.max()), "C3_leverage_rel_err_median": float(np.median(rel)),
            "C3_leverage_rows_checked": int(sample), "C3_leverage_target": 1e-3,
            "C3_seconds_generate_and_gpu": t_gpu, "C3_seconds_oracle": time.perf_counter() - t1,
            "C3_workload": "dense A = U diag(sigma) V^T, n=2^22, d=512, U, V Haar, sigma 1 -> 1e-6, m=65536, "
                           "G 512 x 32; oracle: float64 sketch of the stored A, QR, same G, on sampled rows"}


def batch_timings(cw, stream, count=512):
    """The batched workload: 512 CSR problems, n log-uniform in [2^12, 2^18],
    d in {16, 32, 64, 128}, 4-32 distinct uniform columns per row, N(0,1),
    m = 4 d^2, seeds 1..512.  Times the batch (one graph launch: batched sketch
    and one persistent solve kernel, autotuned) and the same problems solved
    one at a time with cw_solve_sketch, both with CUDA events on the stream."""
    import torch
    import workloads as W
    shapes = W.batch_shapes(count, seed=1)
    probs = []
    for sh in shapes:
        A, b = W.batch_problem(sh, device="cuda")
        probs.append((A, b, sh["m"], sh["seed"]))
    torch.cuda.synchronize()
    out = {"N1_workload": "%d CSR problems: n log-uniform in [2^12, 2^18] (total %d rows, %d nnz), d in "
                          "{16, 32, 64, 128}, 4-32 distinct uniform columns per row, N(0,1) values, "
                          "b = A x0 + 0.1 noise, m = 4 d^2, seeds 1..%d"
                          % (count, sum(p[0].n for p in probs), sum(int(p[0].col.numel()) for p in probs), count)}
    # the tuned shape goes to a cache file so that the direct-launch plan below
    # (per-kernel times) runs the same configuration
    import tempfile
    tune = tempfile.NamedTemporaryFile(prefix="cw_tune_", suffix=".txt", delete=False)
    tune.close()
    old_env = os.environ.get("CW_TUNE_CACHE")
    os.environ["CW_TUNE_CACHE"] = tune.name
    B = cw.Batch(probs, autotune=True)
    out["N1_plan"] = B.info()
    B.run()
    st = B.finish()
    out["N1_status_counts"] = {str(k): st.count(k) for k in sorted(set(st))}
    l0 = cw.launch_count()
    ms = _timed(B.run, stream, reps=5, warm=1)
    out["N1_batched_ms"] = ms
    out["N1_batched_launches_per_call"] = (cw.launch_count() - l0) / 6
    out["N1_batched_problems_per_s"] = count / (ms / 1000.0)
    out["N1_solve_phases_ms"] = B.phases()
    B.close()
    # per-stage times from a direct-launch plan (the graph hides its kernels)
    E = cw.Batch(probs, eager=True, autotune=True)
    out["N1_stages_plan"] = E.info()
    if old_env is None:
        del os.environ["CW_TUNE_CACHE"]
    else:
        os.environ["CW_TUNE_CACHE"] = old_env
    os.unlink(tune.name)
    E.run()
    E.finish()
    torch.cuda.synchronize()
    cw.profile_reset()
    cw.profile_enable(True)
    E.run()
    torch.cuda.synchronize()
    cw.profile_enable(False)
    names = ("kb_tile_hist", "kb_scan_chunk_sums", "kb_scan_bins", "kb_scan_tiles", "kb_coarse_scatter",
             "kb_fine_sort", "kb_set_last", "kb_apply_csr", "k_batch_solve")  # (kb_apply_csr: any variant)
    out["N1_stages_ms"] = _stage_ms(cw, names, 1)
    E.close()
    # one problem at a time with the same solver: a one-problem plan per problem
    # (the batch's sketch kernels and persistent solve kernel, one graph each),
    # launched one after the other
    singles = [cw.Batch([pr], autotune=False) for pr in probs]
    for S1 in singles:
        S1.run()
        S1.finish()
    out["N1_one_at_a_time_same_solver_ms"] = _timed(lambda: [S1.run() for S1 in singles], stream, reps=2, warm=1)
    for S1 in singles:
        S1.close()
    del singles
    out["N1_speedup_same_solver"] = out["N1_one_at_a_time_same_solver_ms"] / out["N1_batched_ms"]
    # one problem at a time through the single-problem API (float64 Householder QR)
    def one_by_one():
        for A, b, m, seed in probs:
            cw.cw_solve_sketch(A, b, m, seed)
    out["N1_one_at_a_time_ms"] = _timed(one_by_one, stream, reps=1, warm=1)
    out["N1_speedup"] = out["N1_one_at_a_time_ms"] / out["N1_batched_ms"]
    del probs
    torch.cuda.empty_cache()
    return out


def learned_rows(cw, n_train=2000, n_report=200, n_select=100, epochs=20, n=1 << 20, d=128, m=2048):
    """The learned-sketch workload at the recipe's counts: a family
    A = U diag(j^-1.5) V_fam^T + 1e-3 N(0,1) (n = 2^20, d = 128, V_fam fixed by
    seed 7, U Haar per matrix), b = A x0 + 0.05 noise; 2000 training matrices,
    100 selection matrices and 200 report matrices, each its own seed.
    m = 2048 = 1024 learned rows (values tied per bucket, w_k, at the fixed hash
    positions of seed 11) + 1024 random CountSketch rows (seed 12); Adam lr 1e-3,
    20 epochs, one matrix per step, on rho^2 - 1 through the library's
    backward (trained through the Cholesky factor of the sketched Gram matrix;
    every reported ratio comes from the Householder QR solve).  Each matrix is
    generated once and kept as its sufficient statistics (the two sketches and
    the Gram matrix of [A b]), all the loss needs.  select_or_fallback decides
    on the selection set; the report set gives the ratios."""
    import math
    import time
    import torch
    import workloads as W
    from paper_1207_6365_gb300 import learned as L
    t0 = time.time()
    V, sig = W.family_basis(d, seed=7, device="cuda")
    sk = L.TiedSketch(m, seed_L=11, seed_R=12, method="normal")

    def member(k):
        A, b = W.family_matrix(k, n, V, sig, device="cuda")
        return sk.member(A, b, m, seed_P=13)
    train_set = [member(k) for k in range(n_train)]
    select_set = [member(200000 + k) for k in range(n_select)]
    report_set = [member(100000 + k) for k in range(n_report)]
    torch.cuda.synchronize()
    t_gen = time.time() - t0
    _, l0 = L.evaluate(sk, report_set)
    t1 = time.time()
    hist = L.train(sk, train_set, epochs, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    sel = L.select_or_fallback(sk, select_set, m, seed_P=13)
    p1, l1 = L.evaluate(sk, report_set)
    diff = [a - b for a, b in zip(l1, p1)]
    mean = sum(diff) / len(diff)
    se = math.sqrt(sum((x - mean) ** 2 for x in diff) / (len(diff) - 1) / len(diff))
    # what the values learned: their spread, and their correlation with
    # 1/sqrt(bucket load) of the learned half (the weights that give every
    # sketched row the same variance)
    w = sk.w.detach().double()
    bucket, _ = cw.cw_hash(11, m // 2, 0, n)
    load = torch.bincount(bucket.long(), minlength=m // 2).double()
    corr = float(torch.corrcoef(torch.stack([w, load.rsqrt()]))[0, 1])
    out = {"N3_workload": "family n=2^20 x d=128, %d train / %d selection / %d report matrices (recipe: 2000 train / "
                          "200 test), m=2048 = 1024 learned rows (values tied per bucket) + 1024 random rows, Adam lr "
                          "1e-3, %d epochs, one matrix per step" % (n_train, n_select, n_report, epochs),
           "N3_test_ratio_plain_countsketch": sum(p1) / len(p1),
           "N3_test_ratio_learned_random_init": sum(l0) / len(l0),
           "N3_test_ratio_learned_random_trained": sum(l1) / len(l1),
           "N3_trained_minus_plain_mean_and_se": [mean, se],
           "N3_gaussian_sketch_ratio": L.gaussian_sketch_ratio(m, d),
           "N3_selection_means_plain_learned": [sel.mean_plain, sel.mean_learned],
           "N3_selected": sel.name,
           "N3_train_loss_first_last_epoch": [hist[0], hist[-1]],
           "N3_w_mean_std_corr_with_rsqrt_load": [float(w.mean()), float(w.std()), corr],
           "N3_train_ms_per_step": t_train * 1000.0 / (epochs * n_train), "N3_generate_s": t_gen}
    del train_set, select_set, report_set
    torch.cuda.empty_cache()
    return out


def run_cw(args):
    import torch
    import paper_1207_6365_gb300 as cw
    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, "nccl")
    cw.load()

    A, b = make_problem("cuda", rows=args.rows, replica=rank)
    n, nnz = A.n, A.nnz
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def step():
        return cw.cw_lsqr_precond(A, b, M, SEED, rtol=RTOL, max_iter=100)

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        x, it, test = step()
    torch.cuda.synchronize()

    cw.profile_reset()
    cw.profile_enable(True)
    l0 = cw.launch_count()
    barrier(world, device)
    torch.cuda.synchronize()
    clocks.mark_start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        x, it, test = step()
        iters.append(it)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier(world, device)
    clk = clocks.stop()
    cw.profile_enable(False)
    launches = cw.launch_count() - l0
    ms_local = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms_local, world, device)
    launches_all = sum_over_ranks(launches, world, device)
    value = nnz * args.steps * world / (ms_max / 1000.0)

    stages = {}
    for kname in TIMED_KERNELS:
        cnt, tot = cw.profile_get(kname)
        if cnt:
            stages[kname] = {"launches_per_step": cnt / args.steps, "ms_per_step": tot / args.steps,
                             "avg_ms": tot / cnt}
    dom = max(stages, key=lambda k: stages[k]["ms_per_step"]) if stages else None
    peak, peak_kind = measured_peak_hbm()
    roofline = None
    if dom is not None and _alg_bytes(dom, n, D, nnz, M) is not None:
        alg = _alg_bytes(dom, n, D, nnz, M)
        ach = alg / (stages[dom]["avg_ms"] / 1000.0) / 1e9
        tr = ncu_traffic(dom)
        roofline = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_source": peak_kind, "alg_bytes_per_launch": alg,
                    "traffic": tr}
    for kname, st in stages.items():
        ab = _alg_bytes(kname, n, D, nnz, M)
        if ab is not None:
            st["alg_GBps"] = ab / (st["avg_ms"] / 1000.0) / 1e9
            st["frac_of_peak"] = st["alg_GBps"] / peak
        mb = _moved_bytes(kname, n, D, nnz, M)
        if mb is not None:
            st["moved_GBps"] = mb / (st["avg_ms"] / 1000.0) / 1e9

    # sketch alone (SA + Sb through cw_sketch_csr), for the SA nnz/s figure
    SA = torch.empty(M, D, device=device)
    Sb = torch.empty(M, device=device)
    for _ in range(2):
        cw.cw_sketch_csr(A, b, M, SEED, SA, Sb)
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    reps = 5
    for _ in range(reps):
        cw.cw_sketch_csr(A, b, M, SEED, SA, Sb)
    s1.record(stream)
    torch.cuda.synchronize()
    sk_ms = s0.elapsed_time(s1) / reps
    sk_bytes = nnz * 8 + (n + 1) * 4 + n * 4 + M * D * 4 + M * 4
    cw.profile_reset()
    cw.profile_enable(True)
    for _ in range(reps):
        cw.cw_sketch_csr(A, b, M, SEED, SA, Sb)
    torch.cuda.synchronize()
    cw.profile_enable(False)
    sk_stages = {}
    for kname in ("k_tile_hist", "k_scan_chunk_sums", "k_scan_bins", "k_scan_tiles", "k_coarse_scatter",
                  "k_fine_sort", "k_set_last", "k_apply_csr"):
        cnt, tot = cw.profile_get(kname)
        if cnt:
            sk_stages[kname] = tot / reps
    sk_ach = sk_bytes / (sk_ms / 1000.0) / 1e9
    sketch_roofline = {"call": "cw_sketch_csr (hash, bucket sort, segmented sum: 8 kernels)", "bound": "hbm",
                       "achieved": sk_ach, "peak": peak, "unit": "GB/s", "frac": sk_ach / peak,
                       "peak_source": peak_kind, "alg_bytes_per_call": sk_bytes, "ms": sk_ms,
                       "nnz_per_s": nnz / (sk_ms / 1000.0), "traffic": ncu_traffic("k_apply_csr"),
                       "traffic_of": "k_apply_csr (the segmented sum)", "stages_ms": sk_stages}
    del SA, Sb

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        rp_h = A.row_ptr.cpu().pin_memory()
        col_h = A.col.cpu().pin_memory()
        val_h = A.val.cpu().pin_memory()
        b_h = b.cpu().pin_memory()
        import workloads as W
        A_h = W.CSR(n, D, rp_h, col_h, val_h)
        x_h = torch.empty(D, dtype=torch.float64).pin_memory()
        h2d = rp_h.numel() * 4 + col_h.numel() * 4 + val_h.numel() * 4 + b_h.numel() * 4
        d2h = D * 8

        def e2e_step():
            # host buffers in, x out: the library copies A in row chunks and
            # sketches each chunk while the next one is in flight
            xx, _, _ = cw.cw_lsqr_precond_host(A_h, b_h, M, SEED, rtol=RTOL, max_iter=100, x=x_h)
            return xx

        e2e_step()
        torch.cuda.synchronize()
        esteps = max(1, min(args.steps, 5))
        barrier(world, device)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(esteps):
            e2e_step()
        f1.record(stream)
        torch.cuda.synchronize()
        barrier(world, device)
        ems = max_over_ranks(f0.elapsed_time(f1), world, device)
        e2e = {"value": nnz * esteps * world / (ems / 1000.0), "unit": "nnz/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": esteps, "ms_per_step": ems / esteps,
               "call": "cw_lsqr_precond_host (page-locked host CSR and b, x back to host memory)"}
        del A_h, x_h, rp_h, col_h, val_h, b_h

    # the segmented sum reads each row's col and val as 64-byte segments at
    # random places: the rate to compare it with is the random segment read
    # rate, about half the copy rate
    gc = segment_read_rates(cw, stream, device)
    sketch_roofline["segment_read_rates"] = gc
    if sk_stages.get("k_apply_csr"):
        g = nnz * 8 / (sk_stages["k_apply_csr"] / 1000.0) / 1e9
        sketch_roofline["apply_gather_GBps"] = g
        sketch_roofline["apply_frac_of_random_64B"] = g / gc["random_64B_GBps"]

    rows = None
    if rank == 0 and not args.no_rows:
        # the other rows are reported, not required: a failure in one of them is
        # recorded in the line instead of losing the line
        rows = {}
        for name, fn, skip in (("rows", lambda: row_timings(cw, A, b, stream, peak), False),
                               ("N1", lambda: batch_timings(cw, stream), args.no_batch),
                               ("N3", lambda: learned_rows(cw), args.no_learned)):
            if skip:
                continue
            try:
                rows.update(fn())
            except Exception as exc:  # noqa: BLE001
                rows[name + "_error"] = ("%s: %s" % (type(exc).__name__, exc))[-400:]
                torch.cuda.synchronize()
                torch.cuda.empty_cache()

    cpu_all = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            r2 = run_oracle_sketch_child(n, 3)
            tt = min(r2["times"])
            cpu_all = {"value": r2["nnz"] / tt, "unit": "nnz/s", "cores": r2["threads"], "kind": "oracle",
                       "sample": "SA and Sb of the whole workload (n = %d rows) by the float64 oracle on all "
                                 "host cores (rows sorted by bucket, buckets summed in parallel), best of 3"
                                 % r2["rows"],
                       "seconds": tt, "gpu_sketch_nnz_per_s": nnz / (sk_ms / 1000.0), "host": host_info()}
        except Exception as exc:  # report, do not hide, a failed baseline
            cpu_all = {"error": str(exc)[-300:]}
    cpu_baseline = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            res = run_oracle_child(SAMPLE_ROWS_CPU, 1)
            cpu_baseline = cpu_baseline_block(
                res, "first 2^22 rows of the workload (same d, m, seed, Zipf columns, rtol): float64 CPU oracle "
                     "(C sketch loop, LAPACK QR, LSQR with C matvecs), one step, 1 thread")
        except Exception as exc:  # report, do not hide, a failed baseline
            cpu_baseline = {"error": str(exc)[-300:]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if n == N_ROWS else
                           "smaller case for profiler captures (n = %d), otherwise as: %s" % (n, WORKLOAD),
                           "n": n, "d": D, "nnz": nnz, "m": M, "rtol": RTOL,
                           "l2": "inputs (2.3 GB of CSR and b) larger than the 129 MB L2; no flush",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": with_sa_sketch(roofline, sketch_roofline), "cpu_baseline": cpu_baseline, "e2e": e2e,
                "clocks": clk,
                "gpu_launches": int(launches_all), "lsqr_iters": iters[-1] if iters else None,
                "sketch_roofline": sketch_roofline,
                "cpu_baseline_all_cores": cpu_all,
                "stages": stages, "rows": rows}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batch_only(count):
    """--only-batch N: the first N problems of the batched workload, planned
    with the autotuner and direct launches (one line of JSON; for profiler
    captures of the batch kernels on a smaller case)."""
    import torch
    import paper_1207_6365_gb300 as cw
    import workloads as W
    cw.load()
    probs = []
    for sh in W.batch_shapes(512, seed=1)[:count]:
        A, b = W.batch_problem(sh, device="cuda")
        probs.append((A, b, sh["m"], sh["seed"]))
    B = cw.Batch(probs, autotune=True, eager=True)
    B.run()
    st = B.finish()
    print(json.dumps({"problems": count, "plan": B.info(), "status": {str(k): st.count(k) for k in set(st)},
                      "phases_ms": B.phases()}), flush=True)
    B.close()
    return 0


def run_qr_only(m, d):
    """--only-qr M D: the float64 QR (cw_qr) of an M x D Gaussian SA with a
    right-hand side, one warm-up and three timed calls (CUDA events); one line
    of JSON (for profiler captures of the QR kernel on its own)."""
    import torch
    import paper_1207_6365_gb300 as cw
    cw.load()
    g = torch.Generator(device="cuda").manual_seed(5)
    SA = torch.randn(m, d, device="cuda", generator=g)
    Sb = torch.randn(m, device="cuda", generator=g)
    stream = torch.cuda.current_stream()
    ms = _timed(lambda: cw.cw_qr(SA, Sb), stream, reps=3, warm=1)
    flops = 2.0 * m * d * d - 2.0 * d ** 3 / 3.0
    print(json.dumps({"m": m, "d": d, "qr_ms": ms, "fp64_tflops": flops / (ms / 1000.0) / 1e12}), flush=True)
    return 0


def main():
    args = parse()
    if args.only_batch:
        return run_batch_only(args.only_batch)
    if args.only_qr:
        return run_qr_only(args.only_qr[0], args.only_qr[1])
    if args.oracle_worker:
        oracle_worker(args.oracle_worker, args.oracle_steps)
        return 0
    if args.oracle_sketch_worker:
        oracle_sketch_worker(args.oracle_sketch_worker, args.oracle_steps)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_cw(args)


if __name__ == "__main__":
    sys.exit(main())

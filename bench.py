#!/usr/bin/env python
"""Benchmark of the SpMV path on the 6M-cell finite-volume Laplacian.

Workload (one step): y = A x, FP64, on the Kuhn-tet 100^3 cube (6,000,000 cells,
29,880,000 non-zeros, Dirichlet, cells randomly permuted then RCM-reordered), inputs resident
in HBM, L2 flushed (256 MB written, then 256 MB read) between timed steps.  The metric is effective bandwidth:
algorithmic bytes 12 nnz + 16 N (each value, index, x and y entry once) per step / time.

Secondary results measured once after the timed loop (same JSON line): FP32 product of the same
matrix, FP64 on the random (unreordered) order, the naive CSR kernel, CG solves, SpMM and the
serving loop where available.

--impl reference times the CPU oracle (plain sequential C) on the same workload.
N > 1 (torchrun): independent replicas, one per GPU, weak scaling; value = all ranks' bytes /
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "SpMV effective GB/s (% HBM peak) FP64 vs mixed; served CG solves/s, p99"
WORKLOAD = "kuhn-tet 100^3 FV Laplacian, Dirichlet, 6,000,000 rows, 29,880,000 nnz, RCM order"
FLUSH_BYTES = 512 << 20  # 256 MB written + 256 MB read between timed steps
VARIANTS = {0: "auto", 1: "spmv_csr", 2: "spmv_sell", 3: "spmv_sell_window", 4: "spmv_sell_bulk"}


def spmv_bytes(n, nnz, f32=False):
    return (8 * nnz + 8 * n) if f32 else (12 * nnz + 16 * n)


def reduce_max_time(t_local, world, device=None):
    """Slowest rank's time (replicas: every rank runs the same workload on its own GPU)."""
    if world == 1:
        return t_local
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def weak_scaling_value(nbytes_per_step, steps, world, t_max):
    """Whole-job effective GB/s: bytes of all ranks' steps over the slowest rank's time."""
    return world * nbytes_per_step * steps / t_max / 1e9


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self._t:
            self._t.join(timeout=5)
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                mhz.append(float(s[0]))
                mx = float(s[1])
            except ValueError:
                continue
            for name, v in zip(names, s[3:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


def traffic_from_profile(kernel_key):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)[kernel_key]
    except Exception:
        return None
    h = hashlib.sha256()
    for rel in t.get("sources", []):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != t.get("sha256"):
        return None
    return t.get("traffic_bytes")


# ---------------------------------------------------------------------------------------
def host_threads():
    """Host cores this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_spmv_rows(rp, ci, v, x, a, b, threads, pool):
    """The oracle's sequential CSR SpMV over rows [a, b), split into `threads` contiguous row
    blocks run at once on host threads (the ctypes call releases the GIL).  The oracle itself
    is unchanged; only its rows are spread over the cores.  Returns the algorithmic bytes."""
    import oracle
    cuts = np.linspace(a, b, threads + 1).astype(np.int64)
    jobs = [(int(cuts[i]), int(cuts[i + 1])) for i in range(threads) if cuts[i + 1] > cuts[i]]
    list(pool.map(lambda ab: oracle.spmv(rp[ab[0]:ab[1] + 1], ci, v, x), jobs))
    return 12 * int(rp[b] - rp[a]) + 16 * (b - a)


def run_reference(args):
    """The CPU oracle on the same workload and metric (reference arm), on all host cores."""
    import concurrent.futures as cf
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2107_12371_gb300 import workloads
    m, x = workloads.c2()
    perm = oracle.cm_order(m.row_ptr, m.col_idx)
    rp, ci, v = oracle.permute_csr(m.row_ptr, m.col_idx, m.values, perm)
    xp = np.ascontiguousarray(x[perm])
    n = m.n
    T = host_threads()
    with cf.ThreadPoolExecutor(T) as pool:
        # one full product first; each timed step is a bounded sample: a contiguous block of
        # rows sized so the K steps take about a minute in total (the whole matrix if it fits)
        t0 = time.perf_counter()
        oracle_spmv_rows(rp, ci, v, xp, 0, n, T, pool)
        t_full = time.perf_counter() - t0
        rows = n if args.steps * t_full <= 60.0 else max(1, int(n * 60.0 / (args.steps * t_full)))
        blocks = [(a, min(n, a + rows)) for a in range(0, n, rows)]

        def step(i):
            a, b = blocks[i % len(blocks)]
            return oracle_spmv_rows(rp, ci, v, xp, a, b, T, pool)

        for i in range(args.warmup):
            step(i)
        done = 0
        t0 = time.perf_counter()
        for i in range(args.steps):
            done += step(i)
        dt = time.perf_counter() - t0
    value = done / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": m.n, "nnz": m.nnz, "rows_per_step": rows,
                       "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": T, "kind": "oracle",
                             "sample": "%d steps of the sequential CSR SpMV over %d-row blocks "
                                       "of the 6M-row RCM-ordered matrix, each block split "
                                       "over %d host threads" % (args.steps, rows, T)},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(rp, ci, v, x, nbytes, budget_s=10.0):
    """The oracle's SpMV timed on the host: on all cores (row blocks on threads), and on one."""
    import concurrent.futures as cf
    import oracle
    n = rp.size - 1
    T = host_threads()
    out = {}
    with cf.ThreadPoolExecutor(T) as pool:
        for threads, budget in ((T, budget_s * 0.5), (1, budget_s * 0.5)):
            oracle_spmv_rows(rp, ci, v, x, 0, n, threads, pool)
            reps = 0
            t0 = time.perf_counter()
            while True:
                oracle_spmv_rows(rp, ci, v, x, 0, n, threads, pool)
                reps += 1
                dt = time.perf_counter() - t0
                if dt >= budget:
                    break
            out[threads] = (nbytes * reps / dt / 1e9, reps, dt)
    value, reps, dt = out[T]
    return {"value": value, "unit": "GB/s", "cores": T, "kind": "oracle",
            "sample": "%d full CSR SpMVs of the 6M-row RCM-ordered matrix (%.1f s), rows split "
                      "over %d host threads each running the sequential oracle" % (reps, dt, T),
            "single_thread": {"value": out[1][0], "unit": "GB/s", "cores": 1,
                              "sample": "%d full sequential SpMVs (%.1f s)" % out[1][1:]}}


def flush_l2(flush_buf):
    """Write a buffer larger than L2 (evicts every line of the previous step), then read a
    second one, so the dirty lines of the write are written back before the timed kernel."""
    half = flush_buf.numel() // 2
    flush_buf[:half].add_(1)
    return flush_buf[half:].sum()


def time_kernel(torch, fn, steps, flush_buf, stream, warmup=3):
    """Per-step CUDA-event times (ms) of fn() with an L2 flush before each step, after `warmup`
    untimed calls (the first launches of a kernel load its module and touch fresh buffers)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        for a, b in evs:
            flush_l2(flush_buf)
            a.record(stream)
            fn()
            b.record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def run_profile_kernel(args):
    """A few launches of one secondary kernel, for ncu captures (no timing output)."""
    import torch
    from paper_2107_12371_gb300 import capi, meshgen, workloads
    capi.load()
    dev = torch.device("cuda", 0)
    what = args.profile_kernel
    if what.startswith("spmm"):
        k, dt = int(what.split("_")[1][1:]), what.split("_")[2]
        m, X = workloads.mixed(87, seed=1, k=32)
        A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM,
                        precision=capi.SPMV_PREC_DUAL, sigma=1024, spmm_form=args.spmm_form)
        Xd = torch.from_numpy(np.ascontiguousarray(X[:, :k])).to(
            dev, torch.float64 if dt == "f64" else torch.float32)
        Yd = torch.empty_like(Xd)
        for _ in range(args.steps):
            A.apply_multi(Xd, Yd)
    elif what == "mcg":
        # multi-RHS CG on the 87^3 mixed mesh, k = 8 and 32, FP64 and mixed, 32 iterations each
        for k in (8, 32):
            m, Bv = workloads.mixed(87, seed=1, k=k)
            A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM,
                            precision=capi.SPMV_PREC_DUAL, sigma=1024)
            Bd = torch.from_numpy(np.ascontiguousarray(Bv.reshape(m.n, k)[A.permutation()])).to(dev)
            Xd = torch.zeros_like(Bd)
            for mixed in (0, 1):
                A.solve_multi(Bd, Xd, rtol=1e-10, max_iter=32, mixed=mixed, max_outer=1)
            A.close()
    elif what == "chain":
        M, G, L, rng = meshgen.kuhn_tet_operators(80, seed=0, permute=False)
        Gh = capi.Matrix(G.n, G.row_ptr, G.col_idx, G.values, n_cols=G.n_cols)
        Mh = capi.Matrix(M.n, M.row_ptr, M.col_idx, M.values, n_cols=M.n_cols)
        xd = torch.from_numpy(meshgen.uniform_vectors(rng, L.n)).to(dev)
        y = torch.empty(M.n, dtype=torch.float64, device=dev)
        for _ in range(args.steps):
            capi.spmv_apply_chain(Mh.handle, Gh.handle, xd, y)
    torch.cuda.synchronize()
    print(json.dumps({"profile_kernel": what}), flush=True)
    return 0


def run_gpu(args):
    import torch
    from paper_2107_12371_gb300 import capi, workloads

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    capi.load()

    m, x = workloads.c2()
    n, nnz = m.n, m.nnz
    nbytes = spmv_bytes(n, nnz)
    stream = torch.cuda.Stream(device=dev)
    t_create = time.perf_counter()
    variant = {"auto": capi.SPMV_VARIANT_AUTO, "sell": capi.SPMV_VARIANT_SELL,
               "csr": capi.SPMV_VARIANT_CSR, "window": capi.SPMV_VARIANT_SELL_WINDOW,
               "bulk": capi.SPMV_VARIANT_SELL_BULK}[args.variant]
    A = capi.Matrix(n, m.row_ptr, m.col_idx, m.values, stream=stream,
                    reorder=capi.SPMV_REORDER_RCM, precision=capi.SPMV_PREC_DUAL,
                    slice_height=args.slice_height, autotune=int(args.autotune),
                    variant=variant, index_bits=args.index_bits, block=args.block)
    t_create = time.perf_counter() - t_create
    info = A.info()
    xd = torch.from_numpy(x).to(dev)
    xi = torch.empty_like(xd)
    yi = torch.empty_like(xd)
    A.permute(0, xd, xi, stream)
    flush = torch.zeros(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    fn = lambda: A.apply(xi, yi, stream)  # noqa: E731
    if args.profile and args.f32:
        x32, y32 = xi.float(), torch.empty(n, dtype=torch.float32, device=dev)
        fn = lambda: A.apply_f32(x32, y32, stream)  # noqa: E731

    for _ in range(max(3, args.warmup)):
        fn()
    stream.synchronize()

    sampler = ClockSampler(local).start()
    time.sleep(0.2)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    times = time_kernel(torch, fn, args.steps, flush, stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    # keep the sampler running a little under a load loop so the clocks reflect the kernel
    soak_end = time.perf_counter() + (0.0 if args.profile else 1.0)
    with torch.cuda.stream(stream):
        while time.perf_counter() < soak_end:
            for _ in range(200):
                fn()
            stream.synchronize()
    clocks = sampler.stop()

    # the same K products back to back, without the flush between them: the write-back of each
    # y (which the flush of the timed loop absorbs outside its events) is inside this region
    with torch.cuda.stream(stream):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush_l2(flush)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
    stream.synchronize()
    b2b_s = e0.elapsed_time(e1) / 1e3 / args.steps
    t_dev = reduce_max_time(sum(times) / 1e3, world, dev)  # seconds over the K timed SpMVs
    value = weak_scaling_value(nbytes, args.steps, world, t_dev)
    avg_launch_s = sum(times) / len(times) / 1e3
    peak, peak_src = measured_peaks()

    if args.profile:
        if args.profile_cg > 0:
            # a few CG iterations of both solvers, for launch lists of the CG kernels
            bi = xi.clone()
            for mixed in (0, 1):
                xs = torch.zeros_like(bi)
                A.solve(bi, xs, stream, raise_on_error=False, rtol=1e-10, mixed=mixed,
                        max_iter=args.profile_cg, max_outer=2)
            torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile_run": True, "value": value, "unit": "GB/s"}), flush=True)
        return 0
    extra = {}
    if rank == 0 and not args.quick:
        extra = secondary(args, torch, capi, workloads, m, x, A, xi, stream, flush, dev)

    # end-to-end through the C ABI with host buffers: pinned x -> device, y -> pinned host
    xh = torch.from_numpy(x[A.permutation()]).pin_memory()
    yh = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    for _ in range(3):
        xi.copy_(xh, non_blocking=True)
        fn()
        yh.copy_(yi, non_blocking=True)
    stream.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(e2e_steps):
            xi.copy_(xh, non_blocking=True)
            fn()
            yh.copy_(yi, non_blocking=True)
        ev1.record(stream)
    stream.synchronize()
    e2e_serial_s = ev0.elapsed_time(ev1) / 1e3 / e2e_steps

    # through spmv_apply_host_async: one C-ABI call per step with x and y in pinned host
    # memory, steps taking three streams (and three host buffer pairs) in turn, so that
    # consecutive calls overlap (wall clock, host timer between full synchronisations)
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(2)]
    xhs = [xh] + [xh.clone().pin_memory() for _ in range(2)]
    yhs = [yh] + [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]

    def host_steps(steps):
        for j in range(steps):
            A.apply_host_async(xhs[j % 3], yhs[j % 3], streams[j % 3])

    host_steps(4)
    torch.cuda.synchronize(dev)
    # one synchronous call at a time, for comparison
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        A.apply_host(xh, yh, stream)
    e2e_single_s = (time.perf_counter() - t0) / e2e_steps
    t0 = time.perf_counter()
    host_steps(e2e_steps)
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    traffic = traffic_from_profile("%s_f64_c2_rcm_i%d_s%d" % (
        VARIANTS[info["variant"]], info["index_bits"], info["slice_height"]))
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "nnz": nnz, "format": "sliced ELLPACK",
                   "slice_height": info["slice_height"], "block": info["block"],
                   "variant": VARIANTS[info["variant"]], "index_bits": info["index_bits"],
                   "autotuned": bool(args.autotune), "reorder": "rcm",
                   "bandwidth": info["bandwidth"], "max_slice_span": info["max_slice_span"],
                   "algorithmic_bytes_per_step": nbytes, "l2": "flushed between steps (256 MB write, then 256 MB read)",
                   "create_s": round(t_create, 3), "wall_s_timed_region": round(wall, 4),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "pct_hbm_peak": 100.0 * (value / world) / peak,
        "clocks": clocks,
        "e2e": {"value": nbytes / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n,
                "call": "spmv_apply_host_async, steps taking three streams in turn (pinned "
                        "host x and y; the copies of one call overlap the products and "
                        "copies of the others)",
                "one_call_at_a_time_value": nbytes / e2e_single_s / 1e9,
                "one_call_at_a_time": "spmv_apply_host (synchronous; copy of x, product and "
                                      "copy of y overlapped by eight runs of slices)",
                "serial_value": nbytes / e2e_serial_s / 1e9},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": nbytes / avg_launch_s / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": nbytes / avg_launch_s / 1e9 / peak,
                     "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel": VARIANTS[info["variant"]],
                     "traffic": traffic},
        "headline_back_to_back": {"ms": b2b_s * 1e3, "GBs": nbytes / b2b_s / 1e9,
                                  "frac": nbytes / b2b_s / 1e9 / peak,
                                  "note": "K products without the L2 flush between them: each "
                                          "y write-back falls inside the timed region"},
    }
    if traffic:
        line["roofline"]["dram_bytes_frac"] = traffic / avg_launch_s / 1e9 / peak
        line["roofline"]["dram_bytes_per_nnz"] = traffic / nnz
        line["roofline"]["dram_bytes_note"] = (
            "DRAM bytes an ncu capture counted per launch (16-bit columns move fewer bytes than "
            "the algorithmic 12 B per non-zero) / launch time / copy peak")
    line.update(extra)
    # the oracle on the host cores before the serving passes: timed after them (tens of GB of
    # generated requests allocated and freed) the threaded oracle measured several times slower
    if not args.no_cpu_baseline:
        rp, ci, v = capi.spmv_export_csr(A.handle, n, nnz)
        line["cpu_baseline"] = cpu_baseline(rp, ci, v, xi.cpu().numpy(), nbytes)
    if rank == 0 and not args.quick and args.serve_requests > 0:
        line.update(serving_results(args, capi, torch))
    line["summary"] = summary_of(line)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def summary_of(line):
    """The results a reader looks for first, gathered at the end of the JSON line."""
    def g(*keys):
        d = line
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d
    r3 = lambda v: None if v is None else (round(v, 4) if abs(v) < 10 else round(v, 1))  # noqa
    out = {
        "spmv_fp64_GBs": r3(g("value")), "spmv_fp64_frac": r3(g("roofline", "frac")),
        "spmv_fp64_dram_frac": r3(g("roofline", "dram_bytes_frac")),
        "spmv_fp64_back_to_back_frac": r3(g("headline_back_to_back", "frac")),
        "spmv_fp32_GBs": r3(g("fp32_spmv", "value")),
        "e2e_GBs": r3(g("e2e", "value")),
        "cg_fp64_s": r3(g("cg_fp64_graph", "seconds")),
        "cg_fp64_persistent_s": r3(g("cg_fp64_persistent", "seconds")),
        "cg_mixed_s": r3(g("cg_mixed_ir", "seconds")),
        "cg_mixed_persistent_s": r3(g("cg_mixed_ir_persistent", "seconds")),
        "cg_mixed_speedup_vs_fp64": r3(g("mixed_speedup_vs_fp64")),
        "cg_mixed_rel_residual_fp64": g("cg_mixed_ir", "rel_residual_fp64"),
    }
    for k in ("k8", "k32"):
        out["cg_multi_" + k] = {
            "fp64_solves_per_s": r3(g("cg_multi_rhs", k, "fp64", "solves_per_s")),
            "mixed_solves_per_s": r3(g("cg_multi_rhs", k, "mixed", "solves_per_s")),
            "fp64_vs_separate": r3(g("cg_multi_rhs", k, "speedup_fp64_vs_separate")),
            "mixed_vs_separate": r3(g("cg_multi_rhs", k, "speedup_mixed_vs_separate"))}
    out["spmm_frac"] = {k: r3(g("spmm_mixed_mesh", k, "roofline", "frac"))
                        for k in ("k8_f64", "k8_f32", "k32_f64", "k32_f32")}
    out["chain_speedup_tuned"] = {"fp64": r3(g("operator_chain", "speedup")),
                                  "fp32": r3(g("operator_chain", "fp32", "speedup"))}
    out["chain_speedup_fused_kernel"] = {"fp64": r3(g("operator_chain", "fused_speedup")),
                                         "fp32": r3(g("operator_chain", "fp32", "fused_speedup"))}
    sv = g("serving")
    if sv:
        out["serving"] = {"requests": sv["requests"],
                          "one_at_a_time_plain_fp64": [r3(sv["one_at_a_time_plain_fp64"][f])
                                                       for f in ("solves_per_s", "p50_latency_s",
                                                                 "p99_latency_s")]}
        for key in ("arrival_0.5x", "arrival_1x", "arrival_1x_priority", "arrival_2x",
                    "saturated"):
            out["serving"][key] = [r3(sv[key][f]) for f in ("solves_per_s", "p50_latency_s",
                                                            "p99_latency_s")]
        out["serving"]["fields"] = "solves/s, p50 s, p99 s"
    return out


def secondary(args, torch, capi, workloads, m, x, A, xi, stream, flush, dev):
    """One-off measurements reported beside the headline (same JSON line)."""
    out = {}
    n, nnz = m.n, m.nnz
    K = max(10, min(args.steps, 100))
    nb64 = spmv_bytes(n, nnz)
    nb32 = spmv_bytes(n, nnz, f32=True)

    def timed(handle, f32=False, csr=False, xin=None):
        xv = xin if xin is not None else xi
        if f32:
            xv = xv.float()
        yv = torch.empty_like(xv)
        if f32:
            fn = lambda: handle.apply_f32(xv, yv, stream)  # noqa: E731
        elif csr:
            fn = lambda: handle.apply_csr(xv, yv, stream)  # noqa: E731
        else:
            fn = lambda: handle.apply(xv, yv, stream)  # noqa: E731
        t = time_kernel(torch, fn, K, flush, stream)
        ms = sum(t) / len(t)
        nb = nb32 if f32 else nb64
        return {"value": nb / (ms / 1e3) / 1e9, "unit": "GB/s", "ms": ms}

    # FP32 product (the mixed-precision inner SpMV) of the headline handle, whose layout was
    # tuned for the FP64 product; its error against the FP64 product (which equals the FP64
    # oracle bit for bit), normwise and per entry relative to sum_j |a_ij x_j|
    out["fp32_spmv"] = dict(timed(A, f32=True), algorithmic_bytes=nb32)
    y64 = torch.empty_like(xi)
    A.apply(xi, y64, stream)
    y32 = torch.empty(n, dtype=torch.float32, device=dev)
    A.apply_f32(xi.float(), y32, stream)
    absA = torch.empty_like(xi)
    Aabs = capi.Matrix(n, m.row_ptr, m.col_idx, np.abs(m.values), stream=stream,
                       reorder=capi.SPMV_REORDER_RCM)
    Aabs.apply(xi.abs(), absA, stream)  # same renumbering: RCM of the same pattern
    Aabs.close()
    torch.cuda.synchronize(dev)
    d = (y32.double() - y64).abs()
    out["fp32_spmv"]["error_vs_fp64"] = {
        "normwise": float(d.norm() / y64.norm()),
        "max_componentwise": float((d / absA.clamp_min(1e-300)).max())}
    # an FP32 handle of the same matrix with its layout tuned for the FP32 product
    F = capi.Matrix(n, m.row_ptr, m.col_idx, m.values, stream=stream,
                    reorder=capi.SPMV_REORDER_RCM, precision=capi.SPMV_PREC_FP32, autotune=1)
    fx = torch.empty_like(xi)
    F.permute(0, torch.from_numpy(x).to(dev), fx, stream)
    finfo = F.info()
    out["fp32_spmv_fp32_tuned"] = dict(timed(F, f32=True, xin=fx), algorithmic_bytes=nb32,
                                       slice_height=finfo["slice_height"], block=finfo["block"],
                                       variant=VARIANTS[finfo["variant"]],
                                       index_bits=finfo["index_bits"])
    F.close()
    # the naive CSR kernel (Sec. 4.3 baseline) on the same order
    out["naive_csr_rcm"] = timed(A, csr=True)
    # explicit variants of the RCM-ordered matrix (ablation of Sec. 5.1's two ideas)
    for name, kw in [("sell_int32_cols", dict(index_bits=32)),
                     ("sell_int16_cols", dict(index_bits=16)),
                     ("window_int16_cols", dict(index_bits=16,
                                                variant=capi.SPMV_VARIANT_SELL_WINDOW))]:
        H = capi.Matrix(n, m.row_ptr, m.col_idx, m.values, stream=stream,
                        reorder=capi.SPMV_REORDER_RCM, precision=capi.SPMV_PREC_DUAL,
                        slice_height=64, **kw)
        hx = torch.empty_like(xi)
        H.permute(0, torch.from_numpy(x).to(dev), hx, stream)
        out[name] = {"fp64": timed(H, xin=hx), "fp32": timed(H, f32=True, xin=hx),
                     "index_bits": H.info()["index_bits"]}
        H.close()
    # random order (no reordering): sliced and naive -- the GPU analogue of Table 2's ordering
    R = capi.Matrix(n, m.row_ptr, m.col_idx, m.values, stream=stream,
                    slice_height=args.slice_height)
    xr = torch.from_numpy(x).to(dev)
    out["sell_random_order"] = timed(R, xin=xr)
    out["naive_csr_random_order"] = timed(R, csr=True, xin=xr)
    R.close()
    out.update(table2_results(args, torch, capi, workloads, flush, stream, dev))
    if not args.no_cpu_baseline:
        out.update(oracle_beside_results(torch, capi, workloads, dev))
    out.update(cg_results(torch, capi, m, x, A, xi, dev))
    out.update(spmm_results(args, torch, capi, workloads, flush, stream, dev))
    out.update(mcg_results(args, torch, capi, workloads, dev))
    out.update(chain_results(args, torch, capi, flush, stream, dev))
    return out


def oracle_beside_results(torch, capi, workloads, dev):
    """The CPU oracle timed beside the GPU on the same inputs for the solver rows, on bounded
    samples (one thread, the oracle as it stands): FP64 Jacobi-PCG and mixed refinement to
    1e-10 on the 48,000-cell Dirichlet Kuhn-tet cube, and an 8-vector SpMM on a mixed mesh of
    about 80,000 cells.  GPU times are wall-clock per call (CG) or CUDA events (SpMM)."""
    import oracle
    out = {}
    m, b = workloads.kuhn(20, seed=0, dirichlet=True)
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, precision=capi.SPMV_PREC_DUAL)
    bd = torch.from_numpy(b).to(dev)
    for mixed in (0, 1):
        xd = torch.zeros_like(bd)
        A.solve(bd, xd, raise_on_error=False, rtol=1e-10, mixed=mixed)  # warm
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = A.solve(bd, xd, raise_on_error=False, rtol=1e-10, mixed=mixed)
        torch.cuda.synchronize(dev)
        t_gpu = time.perf_counter() - t0
        t0 = time.perf_counter()
        if mixed:
            _, info = oracle.mixed_ir(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10)
            it_o = info["inner_iterations"]
        else:
            x64_oracle, info = oracle.jacobi_pcg(m.row_ptr, m.col_idx, m.values, b, rtol=1e-10)
            it_o = info["iterations"]
        t_cpu = time.perf_counter() - t0
        xg = xd.cpu().numpy()
        out["mixed_ir" if mixed else "cg_fp64"] = {
            "cells": m.n, "gpu_s": t_gpu, "oracle_s": t_cpu, "oracle_over_gpu": t_cpu / t_gpu,
            "gpu_iterations": r["iterations"], "oracle_iterations": it_o,
            "gpu_rel_residual": r["rel_residual"], "oracle_rel_residual": info["rel_residual"],
            "error_vs_fp64_oracle": float(np.linalg.norm(xg - x64_oracle) /
                                          np.linalg.norm(x64_oracle))}
    A.close()
    mm, X = workloads.mixed(30, seed=1, k=8)
    H = capi.Matrix(mm.n, mm.row_ptr, mm.col_idx, mm.values)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    Yd = torch.empty_like(Xd)
    H.apply_multi(Xd, Yd)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(20):
        H.apply_multi(Xd, Yd)
    ev[1].record()
    torch.cuda.synchronize(dev)
    t_gpu = ev[0].elapsed_time(ev[1]) / 1e3 / 20
    t0 = time.perf_counter()
    ref = oracle.spmm(mm.row_ptr, mm.col_idx, mm.values, X, use_fma=True)
    t_cpu = time.perf_counter() - t0
    out["spmm_k8_fp64"] = {"cells": mm.n, "gpu_s": t_gpu, "oracle_s": t_cpu,
                           "oracle_over_gpu": t_cpu / t_gpu,
                           "bit_identical": bool(np.array_equal(Yd.cpu().numpy(), ref))}
    H.close()
    return {"oracle_beside": out}


def table2_results(args, torch, capi, workloads, flush, stream, dev):
    """The GPU analogue of Table 2 (naive vs cached SpMV on the paper's five matrix sizes, 50K
    to 800K tetrahedral cells): synthetic Kuhn-tet cubes of 48K-796K cells (Dirichlet, cells
    permuted).  Per size, FP64 product times of the naive CSR kernel (x gathered from global
    memory, Sec. 4.3) in the cells' random order and after RCM, of the sliced kernel with x
    resident in L2, and of the sliced kernel with the circular shared-memory window of Sec.
    5.1, both after RCM; L2 flushed before every timed step."""
    rows = []
    K = max(10, min(args.steps, 50))
    for n3 in (20, 26, 32, 40, 51):
        m, x = workloads.kuhn(n3, seed=0, dirichlet=True)
        xd = torch.from_numpy(x).to(dev)
        nb = spmv_bytes(m.n, m.nnz)

        def ms_of(handle, xin, csr=False):
            y = torch.empty_like(xin)
            if csr:
                fn = lambda: handle.apply_csr(xin, y, stream)  # noqa: E731
            else:
                fn = lambda: handle.apply(xin, y, stream)  # noqa: E731
            t = sorted(time_kernel(torch, fn, K, flush, stream))
            t = t[len(t) // 10: len(t) - len(t) // 10] or t
            return sum(t) / len(t)

        R = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, stream=stream)
        naive_random = ms_of(R, xd, csr=True)
        R.close()
        row = {"cells": m.n, "nnz": m.nnz, "naive_random_ms": naive_random}
        for name, variant in (("cached_l2", capi.SPMV_VARIANT_SELL),
                              ("cached_window", capi.SPMV_VARIANT_SELL_WINDOW)):
            H = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, stream=stream,
                            reorder=capi.SPMV_REORDER_RCM, variant=variant)
            xi = torch.empty_like(xd)
            H.permute(0, xd, xi, stream)
            if name == "cached_l2":
                row["naive_rcm_ms"] = ms_of(H, xi, csr=True)
            row[name + "_ms"] = ms_of(H, xi)
            H.close()
        row["speedup_vs_naive_random"] = row["naive_random_ms"] / row["cached_l2_ms"]
        row["cached_l2_GBs"] = nb / (row["cached_l2_ms"] / 1e3) / 1e9
        rows.append(row)
    return {"table2_sizes": {"paper_speedups_for_context": [8.19, 10.95, 15.19, 15.87, 16.41],
                             "rows": rows}}


def cg_bytes_per_iter(n, nnz, f32=False):
    # q = A p (matrix, p, q) + x/r update (read x p r q dinv, write x r) + p update (read r dinv
    # p, write p): 12 nnz + 16 N + 56 N + 32 N in FP64, half the vector bytes in FP32
    return (8 * nnz + 52 * n) if f32 else (12 * nnz + 104 * n)


def cg_results(torch, capi, m, b, A, bi, dev):
    """CG solves of the 6M-cell system to 1e-10 (b = the workload's U[-1,1] vector, RCM order)."""
    out = {}
    n, nnz = m.n, m.nnz
    for name, opts in [("cg_fp64_graph", {}), ("cg_fp64_persistent", {"persistent": 1}),
                       ("cg_mixed_ir", {"mixed": 1}),
                       ("cg_mixed_ir_persistent", {"mixed": 1, "persistent": 1})]:
        best = None
        for _ in range(2):
            xi = torch.zeros_like(bi)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            res = A.solve(bi, xi, raise_on_error=False, rtol=1e-10, **opts)
            dt = time.perf_counter() - t0
            if best is None or dt < best[0]:
                best = (dt, res)
        dt, res = best
        f32 = bool(opts.get("mixed"))
        item = {"seconds": dt, "iterations": res["iterations"],
                "outer_iterations": res["outer_iterations"],
                "rel_residual_fp64": res["rel_residual"], "status": res["status"]}
        item["ms_per_iteration"] = dt / max(1, res["iterations"]) * 1e3
        item["effective_GBs"] = (res["iterations"] * cg_bytes_per_iter(n, nnz, f32) / dt / 1e9)
        out[name] = item
    best64 = min(out["cg_fp64_graph"]["seconds"], out["cg_fp64_persistent"]["seconds"])
    best32 = min(out["cg_mixed_ir"]["seconds"], out["cg_mixed_ir_persistent"]["seconds"])
    out["mixed_speedup_vs_fp64"] = best64 / best32
    # where an FP64 iteration's time goes (CUDA events; the solve above ran 16-iteration graph
    # batches with a scalar read-back after each)
    t = capi.spmv_diag_cg_timing(A.handle, 64)
    t["kernel_sum"] = t["product"] + t["update_xr"] + t["update_p"]
    t["solve_per_iter"] = out["cg_fp64_graph"]["ms_per_iteration"]
    t["unit"] = "ms"
    out["cg_iteration_breakdown"] = t
    return out


def spmm_results(args, torch, capi, workloads, flush, stream, dev):
    """Multi-RHS products on the mixed hexahedron/prism/tetrahedron mesh (87^3 hexahedra,
    about 2M cells, seed 1, RCM order), k = 8 and 32 right-hand sides, FP64 and FP32."""
    out = {}
    m, X = workloads.mixed(87, seed=1, k=32)
    # rows sorted by length inside 1,024-row windows after RCM: the mixed mesh's rows hold
    # 4..13 entries, and unsorted slices pad to their longest row
    plain = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, stream=stream,
                        reorder=capi.SPMV_REORDER_RCM)
    padded_plain = plain.info()["sell_entries"]
    plain.close()
    A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, stream=stream,
                    reorder=capi.SPMV_REORDER_RCM, precision=capi.SPMV_PREC_DUAL, sigma=1024)
    info = A.info()
    perm = A.permutation()
    X = X[perm]
    K = max(5, min(args.steps, 30))
    for k in (8, 32):
        for name, dt, vb in (("f64", torch.float64, 8), ("f32", torch.float32, 4)):
            Xd = torch.from_numpy(np.ascontiguousarray(X[:, :k])).to(dev, dt)
            Yd = torch.empty_like(Xd)
            t = time_kernel(torch, lambda: A.apply_multi(Xd, Yd, stream), K, flush, stream)
            sec = sum(t) / len(t) / 1e3
            nbytes = (vb + 4) * m.nnz + 2 * vb * m.n * k
            flops = 2.0 * m.nnz * k
            item = {"ms": sec * 1e3, "GBs": nbytes / sec / 1e9, "GFLOPs": flops / sec / 1e9,
                    "algorithmic_bytes": nbytes}
            if name == "f64":
                item["roofline"] = {"bound": "alu", "achieved": flops / sec / 1e12, "peak": 1.25,
                                    "unit": "TFLOP/s", "frac": flops / sec / 1e12 / 1.25,
                                    "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s)"}
            else:
                peak, _ = measured_peaks()
                item["roofline"] = {"bound": "hbm", "achieved": nbytes / sec / 1e9, "peak": peak,
                                    "unit": "GB/s", "frac": nbytes / sec / 1e9 / peak}
            out["k%d_%s" % (k, name)] = item
    A.close()
    return {"spmm_mixed_mesh": {"n": m.n, "nnz": m.nnz, "max_row": int(np.diff(m.row_ptr).max()),
                                "slice_height": info["slice_height"],
                                "index_bits": info["index_bits"], "sigma": 1024,
                                "sell_entries_over_nnz": info["sell_entries"] / m.nnz,
                                "sell_entries_over_nnz_unsorted": padded_plain / m.nnz, **out}}


def mcg_results(args, torch, capi, workloads, dev):
    """Multi-RHS CG (cg_solve_multi) on the mixed-element mesh (87^3 hexahedra, about 2M cells,
    RCM order, rows sorted by length inside 1,024-row windows), k = 8 and 32 right-hand sides
    U[-1,1] to 1e-10: FP64 and mixed refinement, CUDA-graph batches and the persistent kernel,
    against the same k systems solved one after another by cg_solve on the same handle."""
    out = {}
    for k in (8, 32):
        m, Bv = workloads.mixed(87, seed=1, k=k)
        A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values, reorder=capi.SPMV_REORDER_RCM,
                        precision=capi.SPMV_PREC_DUAL, sigma=1024)
        perm = A.permutation()
        Bd = torch.from_numpy(np.ascontiguousarray(Bv.reshape(m.n, k)[perm])).to(dev)
        Xd = torch.zeros_like(Bd)
        row = {}
        for name, opts in (("fp64", {}), ("fp64_persistent", {"persistent": 1}),
                           ("mixed", {"mixed": 1}), ("mixed_persistent", {"mixed": 1,
                                                                          "persistent": 1})):
            A.solve_multi(Bd, Xd, rtol=1e-10, **opts)  # warm (work arrays, graphs)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            st, cols = A.solve_multi(Bd, Xd, rtol=1e-10, **opts)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            its = [c["iterations"] for c in cols]
            row[name] = {"seconds": dt, "solves_per_s": k / dt, "status": st,
                         "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
                         "max_rel_residual_fp64": max(c["rel_residual"] for c in cols)}
        cols_d = [Bd[:, c].contiguous() for c in range(k)]
        x = torch.zeros_like(cols_d[0])
        for name, mixed in (("separate_fp64", 0), ("separate_mixed", 1)):
            A.solve(cols_d[0], x, raise_on_error=False, rtol=1e-10, mixed=mixed)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for c in range(k):
                A.solve(cols_d[c], x, raise_on_error=False, rtol=1e-10, mixed=mixed)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            row[name] = {"seconds": dt, "solves_per_s": k / dt}
        best64 = min(row["fp64"]["seconds"], row["fp64_persistent"]["seconds"])
        best32 = min(row["mixed"]["seconds"], row["mixed_persistent"]["seconds"])
        row["speedup_fp64_vs_separate"] = row["separate_fp64"]["seconds"] / best64
        row["speedup_mixed_vs_separate"] = row["separate_mixed"]["seconds"] / best32
        row["speedup_mixed_vs_fp64"] = best64 / best32
        out["k%d" % k] = row
        A.close()
    return {"cg_multi_rhs": {"mesh": "mixed hex/prism/tet 87^3, %d cells, %d nnz" % (m.n, m.nnz),
                             **out}}


def chain_results(args, torch, capi, flush, stream, dev):
    """Operator chain of the operator-based formulation: y = M (G x) with the gradient G
    (faces x cells) and the divergence M (cells x faces) of the 80^3 Kuhn-tet mesh (3.07M
    cells, 6.1M faces): two separate products called by the user against spmv_apply_chain in
    each of its forms (the fused kernel, the two products through M's temporary) and with
    the form its tuner picks on the first call."""
    from paper_2107_12371_gb300 import meshgen
    M, G, L, rng = meshgen.kuhn_tet_operators(80, seed=0, permute=False)
    x = meshgen.uniform_vectors(rng, L.n)
    Gh = capi.Matrix(G.n, G.row_ptr, G.col_idx, G.values, stream=stream, n_cols=G.n_cols,
                     precision=capi.SPMV_PREC_DUAL)
    forms = {"fused": capi.SPMV_CHAIN_FUSED, "two_products": capi.SPMV_CHAIN_TWO,
             "tuned": capi.SPMV_CHAIN_AUTO}
    # the tuned handle keeps the sliced product variant (its slice height and CTA size are
    # tuned with the chain form): the tuner times a product of x from DRAM, while the chain's
    # second product reads t = G x from L2
    Mh = {name: capi.Matrix(M.n, M.row_ptr, M.col_idx, M.values, stream=stream,
                            n_cols=M.n_cols, precision=capi.SPMV_PREC_DUAL, chain_form=f,
                            autotune=int(f == capi.SPMV_CHAIN_AUTO),
                            variant=capi.SPMV_VARIANT_SELL)
          for name, f in forms.items()}
    xd = torch.from_numpy(x).to(dev)
    t = torch.empty(G.n, dtype=torch.float64, device=dev)
    y = torch.empty(M.n, dtype=torch.float64, device=dev)
    x32, t32, y32 = xd.float(), t.float(), y.float()
    K = max(10, min(args.steps, 50))
    ms = lambda fn: (lambda ts: sum(ts) / len(ts))(time_kernel(torch, fn, K, flush, stream))  # noqa

    def sep():
        Gh.apply(xd, t, stream)
        Mh["fused"].apply(t, y, stream)

    def sep32():
        Gh.apply_f32(x32, t32, stream)
        Mh["fused"].apply_f32(t32, y32, stream)
    out = {"mesh": "kuhn-tet 80^3, %d cells, %d faces" % (L.n, G.n),
           "separate_ms": ms(sep), "fp32": {"separate_ms": ms(sep32)}}
    for name, h in Mh.items():
        out[name + "_ms"] = ms(lambda: capi.spmv_apply_chain(h.handle, Gh.handle, xd, y, stream))
        out["fp32"][name + "_ms"] = ms(lambda: capi.spmv_apply_chain_f32(h.handle, Gh.handle,
                                                                          x32, y32, stream))
    out["tuned_pick"] = {"fp64": Mh["tuned"].info()["chain_form"][0],
                         "fp32": Mh["tuned"].info()["chain_form"][1],
                         "codes": "1 fused kernel, 2 two products"}
    out["speedup"] = out["separate_ms"] / out["tuned_ms"]
    out["fp32"]["speedup"] = out["fp32"]["separate_ms"] / out["fp32"]["tuned_ms"]
    out["fused_speedup"] = out["separate_ms"] / out["fused_ms"]
    out["fp32"]["fused_speedup"] = out["fp32"]["separate_ms"] / out["fp32"]["fused_ms"]
    nbytes = 12 * (M.nnz + G.nnz) + 8 * (L.n + 2 * G.n + L.n)
    out["algorithmic_bytes_two_products"] = nbytes
    out["separate_GBs"] = nbytes / (out["separate_ms"] / 1e3) / 1e9
    Gh.close()
    for h in Mh.values():
        h.close()
    return {"operator_chain": out}


def _gen_request(index, cells):
    from paper_2107_12371_gb300 import workloads
    m, b = workloads.serving_request(index, cells)
    return index, m.n, m.row_ptr, m.col_idx, m.values, b


class RequestStream:
    """The serving stream's requests generated ahead of use on host threads (the C assembler
    releases the GIL), in order, holding at most `ahead` of them in host memory; with
    preload, all of them are generated before the constructor returns."""

    def __init__(self, sizes, threads, ahead=64, preload=False):
        import concurrent.futures as cf
        self.sizes = sizes
        self.pool = cf.ThreadPoolExecutor(threads)
        self.ahead = len(sizes) if preload else ahead
        self.futs = {}
        self.next = 0
        self.wait_s = 0.0  # time the consumer waited for generation
        self._fill(0)
        if preload:
            for f in self.futs.values():
                f.result()

    def _fill(self, i):
        while self.next < len(self.sizes) and self.next < i + self.ahead:
            self.futs[self.next] = self.pool.submit(_gen_request, self.next,
                                                    float(self.sizes[self.next]))
            self.next += 1

    def get(self, i):
        f = self.futs.pop(i)
        if not f.done():
            t0 = time.perf_counter()
            r = f.result()
            self.wait_s += time.perf_counter() - t0
        else:
            r = f.result()
        self._fill(i + 1)
        return r

    def close(self):
        self.pool.shutdown(wait=True, cancel_futures=True)


def preload_fits(sizes):
    """Whether the whole stream fits in host memory twice over (about 80 bytes per cell:
    CSR of a 5-entry row, right-hand side and result)."""
    import os
    try:
        avail = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    except (ValueError, OSError):
        return False
    return 2 * 80 * float(np.sum(sizes)) < avail


def serving_results(args, capi, torch):
    """The serving stream of 2,000 requests (cell counts log-uniform in [1e4, 2e6], seed =
    request index, FP64 or mixed precision by a seeded coin, rtol 1e-8, 60 GB budget), each
    request a distinct jittered Kuhn-tet box generated on host threads just ahead of its use.
    (a) The baseline: every request as a plain FP64 solve, one at a time (handle, copy of b,
    cg_solve, copy of x).  (b) Served: submitted to the server with Poisson arrivals at 0.5x,
    1x and 2x the baseline's rate, and saturated (a closed loop keeping 64 requests in the
    server) for its capacity.  Latency = submit to result in host memory (conversion
    included), p50 / p99 over all requests."""
    from paper_2107_12371_gb300 import workloads
    n_req = args.serve_requests
    sizes = workloads.serving_sizes(2000, seed=0)[:n_req]
    coin = np.random.default_rng(1).random(2000)[:n_req] < 0.5
    opts = [capi.cg_default_options(rtol=1e-8, mixed=int(c)) for c in coin]
    plain = capi.cg_default_options(rtol=1e-8, mixed=0)
    gen_threads = max(1, min(12, host_threads() - 4))

    def stream(preload=False):
        return RequestStream(sizes, gen_threads, preload=preload)

    def solve_one(req, o):
        i, n, rp, ci, v, b = req
        A = capi.Matrix(n, rp, ci, v, precision=capi.SPMV_PREC_DUAL if o.mixed else 0)
        bd = torch.from_numpy(b).cuda()
        xd = torch.zeros_like(bd)
        r = A.solve(bd, xd, raise_on_error=False, **{f: getattr(o, f) for f, _ in o._fields_})
        xd.cpu()
        A.close()
        return r

    # untimed: the first requests in both precisions load every kernel the stream uses
    # (lazy module loading makes a kernel's first launch slow) and warm the allocator
    warm = stream()
    for i in range(min(16, n_req)):
        req = warm.get(i)
        solve_one(req, plain)
        solve_one(req, capi.cg_default_options(rtol=1e-8, mixed=1))
    warm.close()

    # (a) plain FP64 solves one at a time (the baseline)
    st = stream()
    lat, conv, cells_total = [], 0, 0
    t_all = time.perf_counter()
    wait0 = 0.0
    for i in range(n_req):
        req = st.get(i)
        t0 = time.perf_counter()
        r = solve_one(req, plain)
        lat.append(time.perf_counter() - t0)
        conv += r["status"] == capi.SPMV_OK
        cells_total += req[1]
    t_serial = time.perf_counter() - t_all - st.wait_s
    wait0 = st.wait_s
    st.close()
    rate_plain = n_req / t_serial
    baseline = {"solves_per_s": rate_plain, "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "converged": conv,
                "seconds": t_serial, "generation_wait_s_excluded": wait0}

    # (b) served
    served = {}
    # the largest requests (estimated footprint >= 256 MB: about 1M cells and up) on
    # high-priority streams, at 1x, beside the same arrivals at the default priority
    prio_bytes = 256 << 20
    for mult, prio in ((0.5, 0), (1.0, 0), (1.0, prio_bytes), (2.0, 0), (None, 0)):
        lam = mult * rate_plain if mult else None
        gaps = (np.random.default_rng(2).exponential(1.0 / lam, size=n_req) if mult
                else np.zeros(n_req))
        # the closed loop outruns the generator (about 80M cells/s on the host threads that
        # the server's slot threads leave): its requests are generated before the clock starts
        preload = mult is None and preload_fits(sizes)
        st = stream(preload)
        srv = capi.spmv_server_create(60 << 30, args.serve_slots)
        if prio:
            capi.spmv_server_set_priority_bytes(srv, prio)
        pending = {}
        results = []

        def poll_some():
            for t in list(pending):
                r = capi.spmv_server_poll(srv, t, np.empty(pending[t]))
                if r is not None:
                    results.append(r)
                    del pending[t]

        t0 = time.perf_counter()
        next_t = t0
        late = 0.0
        for i in range(n_req):
            req = st.get(i)
            if mult:
                next_t += gaps[i]
                while time.perf_counter() < next_t:
                    poll_some()
                    time.sleep(0.0002)
                late = max(late, time.perf_counter() - next_t)
            else:
                while len(pending) >= 64:
                    poll_some()
                    time.sleep(0.0002)
            _, n, rp, ci, v, b = req
            pending[capi.spmv_server_submit(srv, n, rp, ci, v, b, opts[i])] = n
        t_sub = time.perf_counter() - t0
        while pending:
            poll_some()
            time.sleep(0.0005)
        t_served = time.perf_counter() - t0
        s = capi.spmv_server_get_stats(srv)
        capi.spmv_server_destroy(srv)
        gen_wait = st.wait_s
        st.close()
        served[("arrival_%gx" % mult if mult else "saturated") + ("_priority" if prio else "")] = {
            "arrival_rate_per_s": lam, "offered_rate_per_s": n_req / t_sub,
            "solves_per_s": n_req / t_served,
            "p50_latency_s": s["p50_latency_s"], "p99_latency_s": s["p99_latency_s"],
            "peak_bytes": s["peak_bytes"],
            "phase_s": {"setup": s["setup_s"], "solve": s["solve_s"], "teardown": s["teardown_s"]},
            "converged": sum(1 for r in results if r["status"] == capi.SPMV_OK),
            "max_rel_residual": max(r["rel_residual"] for r in results),
            "generation": "all requests generated before the timed region" if preload else
                          "generated on host threads ahead of submission",
            "generation_wait_s": gen_wait}
    cells = [float(c) for c in sizes]
    return {"serving": {
        "requests": n_req, "stream": "2,000-request stream, requests 0..%d (%d..%d target cells, "
        "mean %d; %d cells generated)" % (n_req - 1, min(cells), max(cells), int(np.mean(cells)),
                                          cells_total),
        "slots": args.serve_slots, "budget_bytes": 60 << 30, "rtol": 1e-8,
        "precision": "FP64 or mixed by a seeded coin (%d mixed)" % int(coin.sum()),
        "one_at_a_time_plain_fp64": baseline, **served,
        "served_1x_over_one_at_a_time": served["arrival_1x"]["solves_per_s"] / rate_plain,
        "saturated_over_one_at_a_time": served["saturated"]["solves_per_s"] / rate_plain}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--slice-height", type=int, default=64)
    ap.add_argument("--block", type=int, default=256, help="CTA size of the SpMV kernels")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: the headline handle picks S, CTA size and variant by timing")
    ap.add_argument("--quick", action="store_true", help="headline only, no secondary results")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", default="auto", choices=["auto", "sell", "csr", "window", "bulk"],
                    help="kernel variant of the headline handle (auto: default / autotuned)")
    ap.add_argument("--index-bits", type=int, default=0, choices=[0, 16, 32])
    ap.add_argument("--f32", action="store_true",
                    help="with --profile: time the FP32 product of the handle instead")
    ap.add_argument("--profile-kernel", default="",
                    help="spmm_k8_f64 | spmm_k32_f32 | ... | chain: launch only that kernel")
    ap.add_argument("--spmm-form", type=int, default=0,
                    help="with --profile-kernel spmm_*: the SPMV_SPMM_* form (0 = default)")
    ap.add_argument("--profile-cg", type=int, default=0,
                    help="with --profile: also run CG solves capped at this many iterations")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--profile", action="store_true",
                    help="timed SpMV loop only (for ncu launch lists and captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_kernel:
        return run_profile_kernel(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark of the brute-force k-nearest-neighbour search on GB300.

Workload: the largest shape of Table 1 of the paper, N = n = m = 38400 points,
D = d = 96, k = 20, points uniform in [0,1) (seeded synthetic data; the paper
does not state its distribution).  One step is one complete search of all
38400 queries against the 38400 references through the C ABI: the tensor-core
(bf16) distance + threshold filter, the float32 re-rank, the float64 near-tie
re-check and the output.  Inputs are resident in HBM when a step starts; L2 is
flushed (256 MiB write) before every step, outside the timed window.

Also reported: the float32 CUDA-core form on the same workload, the same
search end to end through the C ABI with pinned host buffers (host<->device
copies timed), the roofline fraction of the dominant kernel, and the oracle
timed on the host cores on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun with N > 1 every rank runs the full workload on its own GPU
(independent problems, weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("queries/s & %roofline at n=m=38400,d=96,k=20 (BF16+rerank vs FP32); "
          "serve p50/p99")
WORKLOAD = "uniform_n38400_d96_k20"
SERVE_WORKLOAD = "serve_m4194304_d96"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM traffic of one tensor-core filter launch on this workload, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum: 36.51 + 63.00 MB; see
# profiles/tc_filter_uniform_n38400_d96_k20.md), valid only for the kernel's
# device source it was measured on (sha256 prefix of tc_device.cuh followed by
# tc_ptx.cuh); otherwise reported as null.
FILTER_TRAFFIC_BYTES = 99.23e6
FILTER_TRAFFIC_SRC = "847a37a8c20ca9ba"
FILTER_SOURCES = ("tc_device.cuh", "tc_ptx.cuh")

CLOCK_HOLD_S = 0.3

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# tf32 has no measured peak: the measured bf16 peak times the nominal dense
# tf32 : bf16 ratio of the part (1.1 : 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def tensor_peak(peaks, precision):
    """Dense tensor-core peak (TFLOP/s) of a contraction in `precision`."""
    return peaks["bf16_tflops"] * (TF32_PER_BF16 if precision == "tf32" else 1.0)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    p.add_argument("--precision", choices=["bf16", "tf32"], default="bf16")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--sweep", action="store_true",
                   help="Table 1 grid (N x D, k = 20) instead of the bench line")
    p.add_argument("--configs", action="store_true",
                   help="timings of the other forms and shapes (configs 1-3) instead of the bench line")
    p.add_argument("--serve-requests", type=int, default=1000)
    p.add_argument("--profile-search", nargs=3, metavar=("PRECISION", "WORKLOAD", "DISTANCE"),
                   help="run --reps searches of a workload (fp32/bf16/tf32, a workload name or a "
                        "Table 1 point table1_n<N>_d<D>, l2/l1/linf) and exit: the command "
                        "of an ncu capture")
    p.add_argument("--profile-batch", type=int, default=0,
                   help="run --reps bf16 batches of this many Euclidean instances of the test "
                        "distribution and exit: the command of an ncu capture")
    p.add_argument("--reps", type=int, default=4)
    p.add_argument("--serve-batch", type=int, default=0,
                   help="time searches of this many queries on the serving reference set "
                        "(m = 4,194,304, d = 96, k = 20) instead of the bench line")
    return p.parse_args()


def max_over_ranks(value: float, pg, device) -> float:
    """The largest of every rank's `value` (all-reduce MAX through the process
    group pg; pg None: a single process).  Timings are taken as the slowest
    rank's, and whole-job throughput is the work of all ranks over that time."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampled while the timed region runs."""

    def __init__(self, device: int):
        self.path = os.path.join(tempfile.gettempdir(), f"knn_clocks_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={device}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_first(self, limit_s: float = 3.0) -> None:
        """Return once the sampler has written its first reading (nvidia-smi
        takes a moment to start), or after limit_s."""
        if self.proc is None:
            return
        t_end = time.monotonic() + limit_s
        while time.monotonic() < t_end and self.proc.poll() is None:
            try:
                if os.path.getsize(self.path) > 0:
                    return
            except OSError:
                return
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def filter_traffic(precision):
    """Measured DRAM bytes per filter launch, or None when the kernel source
    has changed since the measurement (or for another precision)."""
    import hashlib
    h = hashlib.sha256()
    try:
        for name in FILTER_SOURCES:
            with open(os.path.join(ROOT, "paper_0804_1448_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
    except OSError:
        return None
    cur = h.hexdigest()[:16]
    return FILTER_TRAFFIC_BYTES if (cur == FILTER_TRAFFIC_SRC and precision == "bf16") else None


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return FALLBACK_PEAKS, "fallback"


def cpu_baseline(R, Q, k, seconds):
    """The oracle, as it stands, on a bounded sample of the workload's queries."""
    import oracle
    done, t0 = 0, time.perf_counter()
    batch = 512
    while done < Q.shape[0] and time.perf_counter() - t0 < seconds:
        oracle.knn(R, Q[done:done + batch], k, "l2")
        done += min(batch, Q.shape[0] - done)
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "queries/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"{done} of {Q.shape[0]} queries x {R.shape[0]} references, d={R.shape[1]}, "
                      f"k={k}, float64 with a full sort per query ({dt:.1f} s)"}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, per step a bounded
    sample of the workload (no GPU work)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_0804_1448_gb300 import inputs
    R, Q, k = inputs.workload(WORKLOAD)
    per_step = 64
    for i in range(args.warmup):
        oracle.knn(R, Q[i * per_step:(i + 1) * per_step], k, "l2")
    t0 = time.perf_counter()
    off = args.warmup * per_step
    for i in range(args.steps):
        lo = (off + i * per_step) % (Q.shape[0] - per_step)
        oracle.knn(R, Q[lo:lo + per_step], k, "l2")
    dt = time.perf_counter() - t0
    v = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": Q.shape[0], "m": R.shape[0], "d": R.shape[1],
                       "k": k, "distance": "l2", "queries_per_step": per_step},
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": f"{per_step} queries per step x {args.steps} steps"},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_bench(local, args):
    """Serving form: resident reference set of 4,194,304 points (d = 96,
    uniform, float32 + bf16 copy), 4 slots sharing it, query batches of
    log-uniform size in [1, 8192] with k uniform in [1, 256] (Euclidean, bf16
    + re-rank).  First all requests at once (saturation queries/s), then
    Poisson arrivals at 30/70/95% of it; p50/p99 latency of each."""
    import numpy as np
    import torch
    from paper_0804_1448_gb300 import inputs, serve
    w = inputs.WORKLOADS[SERVE_WORKLOAD]
    R = inputs.workload_refs(SERVE_WORKLOAD)
    dev = torch.device("cuda", local)
    pool = torch.from_numpy(inputs.uniform(w["pool"], w["d"], seed=w["seed_q"])).to(dev)
    srv = serve.Server(torch.from_numpy(R).to(dev), "bf16", slots=4, n_max=8192, k_max=256,
                       device=local)
    del R

    def requests(seed, rate):
        reqs = serve.workload(args.serve_requests, seed, rate)
        for r in reqs:
            off = (r.rid * 7919) % (w["pool"] - r.n + 1)
            r.queries = pool[off:off + r.n]
        return reqs

    srv.serve(requests(70, None)[:8])                 # warm-up: kernels loaded, slots primed
    done, sched, _ = srv.serve(requests(71, None))
    sat = serve.summary(done)
    mean_n = float(np.mean([r.n for r in done]))
    loads = []
    for i, frac in enumerate((0.30, 0.70, 0.95)):
        rate = frac * sat["queries_per_s"] / mean_n
        done, sched, _ = srv.serve(requests(72 + i, rate))
        s = serve.summary(done)
        loads.append({"offered_frac": frac, "offered_qps": frac * sat["queries_per_s"],
                      "achieved_qps": s["queries_per_s"], "p50_ms": s["p50_ms"],
                      "p99_ms": s["p99_ms"], "requests": s["requests"],
                      "peak_in_flight": sched.peak_running})
    srv.close()
    return {"workload": SERVE_WORKLOAD, "m": w["m"], "d": w["d"], "precision": "bf16",
            "slots": 4, "batch": "log-uniform [1, 8192]", "k": "uniform [1, 256]",
            "requests_per_run": args.serve_requests,
            "saturation_qps": sat["queries_per_s"], "saturation_p50_ms": sat["p50_ms"],
            "saturation_p99_ms": sat["p99_ms"], "loads": loads,
            "latency": "GPU completion (CUDA event) minus arrival, one clock",
            "inputs": "reference set and query pool resident on the device"}


def batch_bench(local, args, peak_tflops, hbm_gbs):
    """Batching form: 512 independent instances, m uniform in [1000, 200000],
    n uniform in [16, 4096], d in {32, 64, 128}, k in {1, 10, 50}, float32
    uniform data (generated on the device from a fixed seed), Euclidean,
    bf16 + re-rank.  Timed: the persistent form (one kernel launch, split
    lengths autotuned per (d, k) bucket), the graph of the instances' own
    launches on parallel branches (autotuned), and the same instances enqueued
    one after another, each planned alone.  The roofline of the batch is the
    sum over instances of max(2 n m d / tensor peak, 4 d (m + n) + 8 n k bytes
    / HBM bandwidth): each instance's contraction at the bf16 peak, or its
    float32 inputs read and outputs written once, whichever takes longer."""
    import numpy as np
    import torch
    from paper_0804_1448_gb300 import knn
    dev = torch.device("cuda", local)
    g = np.random.Generator(np.random.Philox(5))
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    count = 512
    inst = []
    flops = 0.0
    queries = 0
    roof_s = 0.0
    for _ in range(count):
        m = int(g.integers(1000, 200001))
        n = int(g.integers(16, 4097))
        d = int(g.choice([32, 64, 128]))
        k = int(g.choice([1, 10, 50]))
        R = torch.rand((m, d), generator=gen, device=dev)
        Q = torch.rand((n, d), generator=gen, device=dev)
        inst.append(dict(R=R, Q=Q, k=k, dist=torch.empty((n, k), device=dev),
                         idx=torch.empty((n, k), dtype=torch.int32, device=dev)))
        f = 2.0 * n * m * d
        flops += f
        queries += n
        roof_s += max(f / (peak_tflops * 1e12), (4.0 * d * (m + n) + 8.0 * n * k) / (hbm_gbs * 1e9))
    ix = knn.Index(local, "bf16")
    stream = torch.cuda.current_stream(dev)

    def timed(flags, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            ix.search_batch(inst, flags=flags, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    ix.search_batch(inst, flags=knn.KNN_BATCH_NO_GRAPH, stream=stream)   # warm-up
    t_seq = timed(knn.KNN_BATCH_NO_GRAPH, 3)
    # graph of per-instance launches on parallel branches (autotuned)
    br = knn.KNN_BATCH_BRANCHES | knn.KNN_BATCH_AUTOTUNE
    ix.search_batch(inst, flags=br, stream=stream)
    torch.cuda.synchronize(dev)
    branches = ix.batch_info()
    t_branches = timed(br, 5)
    # the persistent form (autotuned split lengths)
    t0 = time.perf_counter()
    ix.search_batch(inst, flags=knn.KNN_BATCH_AUTOTUNE, stream=stream)   # tunes, captures
    torch.cuda.synchronize(dev)
    tune_s = time.perf_counter() - t0
    tuned = ix.batch_info()
    t_pers = timed(knn.KNN_BATCH_AUTOTUNE, 5)
    after = ix.batch_info()
    # the last run's CTA time per stage, averaged over the SMs' CTAs
    ctas = torch.cuda.get_device_properties(dev).multi_processor_count
    stages = {name: {"work_ms_per_cta": v["work_ms"] / ctas, "wait_ms_per_cta": v["wait_ms"] / ctas,
                     "items": v["items"]}
              for name, v in ix.batch_stage_times().items()}
    ix.close()
    tflops = flops / (t_pers / 1e3) / 1e12
    return {"workload": "batch_512_uniform", "instances": count, "queries": queries,
            "flop": flops, "precision": "bf16", "distance": "l2",
            "persistent_ms": t_pers, "queries_per_s": queries / (t_pers / 1e3),
            "launches": after["launches"], "work_items": after["items"],
            "graph_nodes": after["graph_nodes"], "stages": stages,
            "roofline_ms": roof_s * 1e3, "frac_of_roofline": roof_s * 1e3 / t_pers,
            "roofline": "sum over instances of max(2nmd / bf16 peak, (4d(m+n) + 8nk) B / HBM)",
            "achieved_tflops": tflops, "frac_of_peak": tflops / peak_tflops if peak_tflops else None,
            "branches_graph_ms": t_branches, "branches_graph_launches": branches["launches"],
            "per_instance_ms": t_seq, "per_instance_queries_per_s": queries / (t_seq / 1e3),
            "speedup_vs_per_instance": t_seq / t_pers, "speedup_vs_branches_graph": t_branches / t_pers,
            "tuned": {"tune_device_ms": tuned["tune_ms"], "tune_wall_s": tune_s,
                      "branches_graph": {"branches": branches["branches"],
                                         "sm_share": branches["sm_share"]}}}


# Table 1 of the paper, BF-CUDA seconds (8800 GTX, float32, host<->device copies
# included), by D then N.
TABLE1_N = (1200, 2400, 4800, 9600, 19200, 38400)
TABLE1_BF_CUDA = {
    8: (0.02, 0.10, 0.38, 1.71, 7.93, 31.41),
    16: (0.02, 0.10, 0.38, 1.78, 7.98, 31.31),
    32: (0.02, 0.11, 0.40, 1.81, 8.35, 33.40),
    64: (0.03, 0.12, 0.44, 2.00, 9.52, 37.61),
    80: (0.03, 0.12, 0.46, 2.05, 9.93, 39.98),
    96: (0.03, 0.13, 0.48, 2.07, 10.41, 43.74),
}


def configs(args):
    """Timings of the forms and shapes beside the bench line, one JSON line:
    config 1 (n = m = 1200, d = 8, k = 20: float32 CUDA-core and bf16 forms,
    and the oracle on the host cores over all 1200 queries, on all cores and
    on one), config 2
    (n = m = 38400, d = 96, k = 20: float32 Euclidean, Manhattan and
    Chebyshev, bf16 and tf32 Euclidean, bf16 Mahalanobis with a seeded inverse
    covariance), config 3 (m = 2^20, n = 16384, d = 128, k = 100, Gaussian
    mixture: float32, bf16 and tf32, 400 re-rank candidates, and the oracle on
    32 of its queries) and the serving shape (m = 4,194,304, d = 96) at batch
    sizes 1, 64, 512 and 4096 with k = 20, with the filter's achieved HBM rate
    on the bf16 reference copy.  Device times
    with inputs resident (CUDA events, median of `reps`), L2 flushed before
    each.  Accuracy against the oracle is the tests' job (tests/test_gpu_tc.py,
    tests/test_gpu_mixture.py)."""
    import numpy as np
    import torch
    from paper_0804_1448_gb300 import inputs, knn
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peaks, _ = load_peaks()

    def timed(R, Q, k, precision, metric, reps, S_inv=None):
        ix = knn.Index(0, precision, rerank_factor=4)
        ix.set_reference(R)
        if S_inv is not None:
            ix.set_mahalanobis(S_inv)
        dist = torch.empty((Q.shape[0], k), device=dev)
        idx = torch.empty((Q.shape[0], k), dtype=torch.int32, device=dev)
        ix.search_into(Q, k, dist, idx, metric, stream)
        ix.set_profiling(True)
        times, prof = [], []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ix.search_into(Q, k, dist, idx, metric, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
            prof.append(ix.profile())
        st = ix.stats()
        ix.close()
        ms = float(np.median(times))
        out = {"ms": ms, "queries_per_s": Q.shape[0] / (ms / 1e3),
               "fallback_queries": st["fallback_queries"]}
        filt = [pp.get("tc_filter") for pp in prof if pp.get("tc_filter")]
        if filt:
            fms = float(np.median(filt))
            tfl = 2.0 * Q.shape[0] * R.shape[0] * R.shape[1] / (fms / 1e3) / 1e12
            pk = tensor_peak(peaks, precision)
            out.update({"filter_ms": fms, "filter_tflops": tfl, "filter_frac": tfl / pk})
        return out

    res = {}
    import oracle
    R, Q, k = inputs.workload("uniform_n1200_d8_k20")
    Rd, Qd = torch.from_numpy(R).to(dev), torch.from_numpy(Q).to(dev)
    t0 = time.perf_counter()
    oracle.knn(R, Q, k, "l2")
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.knn(R, Q, k, "l2", nthreads=1)
    dt1 = time.perf_counter() - t0
    res["uniform_n1200_d8_k20"] = {
        "fp32_l2": timed(Rd, Qd, k, "fp32", "l2", 20), "bf16_l2": timed(Rd, Qd, k, "bf16", "l2", 20),
        "cpu_baseline": {"value": Q.shape[0] / dt, "unit": "queries/s", "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": f"all {Q.shape[0]} queries ({dt:.2f} s)"},
        # one core, the setting of the paper's BF-C timing (Table 1, N = 1200, D = 8)
        "cpu_baseline_1core": {"value": Q.shape[0] / dt1, "unit": "queries/s", "cores": 1,
                               "kind": "oracle", "seconds": dt1,
                               "sample": f"all {Q.shape[0]} queries ({dt1:.2f} s)"}}
    R, Q, k = inputs.workload(WORKLOAD)
    Rd, Qd = torch.from_numpy(R).to(dev), torch.from_numpy(Q).to(dev)
    # an inverse covariance with eigenvalues from 1 to 30 (seeded rotation)
    g = np.random.Generator(np.random.Philox(8))
    rot, _ = np.linalg.qr(g.standard_normal((R.shape[1], R.shape[1])))
    S_inv = (rot * np.geomspace(1.0, 30.0, R.shape[1])) @ rot.T
    S_inv = 0.5 * (S_inv + S_inv.T)
    res[WORKLOAD] = {"fp32_l2": timed(Rd, Qd, k, "fp32", "l2", 5),
                     "fp32_l1": timed(Rd, Qd, k, "fp32", "l1", 5),
                     "fp32_linf": timed(Rd, Qd, k, "fp32", "linf", 5),
                     "bf16_l2": timed(Rd, Qd, k, "bf16", "l2", 10),
                     "tf32_l2": timed(Rd, Qd, k, "tf32", "l2", 10),
                     "bf16_mahalanobis": timed(Rd, Qd, k, "bf16", "mahalanobis", 10, S_inv)}
    name = "mixture_m1048576_n16384_d128_k100"
    R, Q, k = inputs.workload(name)
    Rd, Qd = torch.from_numpy(R).to(dev), torch.from_numpy(Q).to(dev)
    sel = np.arange(0, Q.shape[0], Q.shape[0] // 32)[:32]
    t0 = time.perf_counter()
    oracle.knn_subset(R, Q, sel, k, "l2")
    dt = time.perf_counter() - t0
    del R, Q
    res[name] = {"fp32_l2": timed(Rd, Qd, k, "fp32", "l2", 3),
                 "bf16_l2": timed(Rd, Qd, k, "bf16", "l2", 5),
                 "tf32_l2": timed(Rd, Qd, k, "tf32", "l2", 5),
                 "cpu_baseline": {"value": len(sel) / dt, "unit": "queries/s",
                                  "cores": oracle.max_threads(), "kind": "oracle",
                                  "sample": f"{len(sel)} of 16384 queries ({dt:.1f} s)"}}
    del Rd, Qd
    torch.cuda.empty_cache()
    # the serving shape at fixed batch sizes: small batches stream the bf16
    # reference copy once per search (HBM-bound), large ones are tensor-bound
    w = inputs.WORKLOADS[SERVE_WORKLOAD]
    Rs = torch.from_numpy(inputs.workload_refs(SERVE_WORKLOAD)).to(dev)
    pool = torch.from_numpy(inputs.uniform(8192, w["d"], seed=w["seed_q"])).to(dev)
    kp = (w["d"] + 4 + 63) // 64 * 64
    r_bytes = float(w["m"]) * kp * 2
    serve_rows = {}
    for b in (1, 64, 512, 4096):
        t = timed(Rs, pool[:b].contiguous(), 20, "bf16", "l2", 5)
        if "filter_ms" in t:
            t["filter_hbm_gbs"] = r_bytes / (t["filter_ms"] / 1e3) / 1e9
            t["filter_hbm_frac"] = t["filter_hbm_gbs"] / peaks["hbm_gbs"]
        serve_rows[f"n{b}_k20"] = t
    res[SERVE_WORKLOAD] = serve_rows
    print(json.dumps({"configs": res, "peaks": {"bf16_tflops": peaks["bf16_tflops"],
                                                "hbm_gbs": peaks["hbm_gbs"],
                                                "tf32": "bf16_tflops x 1.1/2.25 (nominal "
                                                        "tf32:bf16 ratio)"}}),
          flush=True)


def serve_batch(args):
    """Searches of args.serve_batch queries against the resident serving set
    (m = 4,194,304, d = 96, bf16, k = 20): args.warmup untimed, then args.steps
    timed with CUDA events (L2 flushed before each); one JSON line with the
    per-search time, the filter's time and its rate on the bf16 reference copy
    (small batches stream that copy once per search: the HBM-bound case)."""
    import numpy as np
    import torch
    from paper_0804_1448_gb300 import inputs, knn
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    peaks, src = load_peaks()
    w = inputs.WORKLOADS[SERVE_WORKLOAD]
    R = torch.from_numpy(inputs.workload_refs(SERVE_WORKLOAD)).to(dev)
    b = args.serve_batch
    Q = torch.from_numpy(inputs.uniform(b, w["d"], seed=w["seed_q"])).to(dev)
    ix = knn.Index(0, "bf16")
    ix.set_reference(R)
    dist = torch.empty((b, 20), device=dev)
    idx = torch.empty((b, 20), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(1, args.warmup)):
        ix.search_into(Q, 20, dist, idx, "l2", stream)
    ix.set_profiling(True)
    times, filt = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ix.search_into(Q, 20, dist, idx, "l2", stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
        filt.append(ix.profile().get("tc_filter", float("nan")))
    ix.close()
    kp = (w["d"] + 4 + 63) // 64 * 64
    r_bytes = float(w["m"]) * kp * 2
    fms = float(np.median(filt))
    print(json.dumps({"serve_batch": b, "m": w["m"], "d": w["d"], "k": 20, "precision": "bf16",
                      "ms": float(np.median(times)), "filter_ms": fms,
                      "filter_hbm_gbs": r_bytes / (fms / 1e3) / 1e9,
                      "filter_hbm_frac": r_bytes / (fms / 1e3) / 1e9 / peaks["hbm_gbs"],
                      "peak_source": f"{src} hbm_gbs"}), flush=True)


def sweep(args):
    """The Table 1 grid: N = n = m in TABLE1_N, D in {8, 16, 32, 64, 80, 96},
    k = 20, uniform [0,1) points, Euclidean.  Per point: the bf16 and float32
    searches with inputs resident on the device (CUDA events, median of 5),
    and the bf16 search end to end through the C ABI with host buffers (the
    paper's BF-CUDA times include the copies)."""
    import numpy as np
    import torch
    from paper_0804_1448_gb300 import inputs, knn
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for D in sorted(TABLE1_BF_CUDA):
        for ni, N in enumerate(TABLE1_N):
            R = inputs.uniform(N, D, seed=1000 + D)
            Q = inputs.uniform(N, D, seed=2000 + D)
            Rd, Qd = torch.from_numpy(R).to(dev), torch.from_numpy(Q).to(dev)
            dist = torch.empty((N, 20), device=dev)
            idx = torch.empty((N, 20), dtype=torch.int32, device=dev)
            row = {"N": N, "D": D, "paper_bf_cuda_s": TABLE1_BF_CUDA[D][ni]}
            for prec in ("bf16", "fp32"):
                ix = knn.Index(0, prec)
                ix.set_reference(Rd)
                for _ in range(2):
                    ix.search_into(Qd, 20, dist, idx, "l2", stream)
                times = []
                for _ in range(5):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ix.search_into(Qd, 20, dist, idx, "l2", stream)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    times.append(e0.elapsed_time(e1))
                row[f"{prec}_device_ms"] = float(np.median(times))
                if prec == "bf16":
                    st = ix.stats()
                    row["bf16_fallback_queries_per_search"] = st["fallback_queries"] / 7.0
                    row["bf16_fallback_reasons"] = [st["fallback_short_list"], st["fallback_overflow"],
                                                    st["fallback_wide_cut"], st["fallback_uncertified"]]
                    Qh = torch.from_numpy(Q).pin_memory()
                    dh = torch.empty((N, 20), dtype=torch.float32).pin_memory()
                    ih = torch.empty((N, 20), dtype=torch.int32).pin_memory()
                    ix.search_into(Qh, 20, dh, ih, "l2")
                    t = []
                    for _ in range(5):
                        t0 = time.perf_counter()
                        ix.search_into(Qh, 20, dh, ih, "l2")
                        t.append(time.perf_counter() - t0)
                    row["bf16_e2e_ms"] = float(np.median(t) * 1e3)
                ix.close()
            row["speedup_e2e_vs_paper"] = row["paper_bf_cuda_s"] * 1e3 / row["bf16_e2e_ms"]
            rows.append(row)
    print(json.dumps({"sweep": "table1", "k": 20, "distance": "l2", "rows": rows}), flush=True)


def profile_search(args):
    """--reps searches of one workload in one precision and distance, inputs
    resident, nothing timed (for ncu: the last launches are the warm ones)."""
    import torch
    from paper_0804_1448_gb300 import inputs, knn
    precision, workload, distance = args.profile_search
    grid = re.fullmatch(r"table1_n(\d+)_d(\d+)", workload)
    if grid:   # a point of the Table 1 grid, drawn as --sweep draws it
        N, D = int(grid.group(1)), int(grid.group(2))
        R, Q, k = inputs.uniform(N, D, seed=1000 + D), inputs.uniform(N, D, seed=2000 + D), 20
    else:
        R, Q, k = inputs.workload(workload)
    Rd, Qd = torch.from_numpy(R).cuda(), torch.from_numpy(Q).cuda()
    ix = knn.Index(0, precision)
    ix.set_reference(Rd)
    for _ in range(args.reps):
        ix.search(Qd, k, distance)
    ix.sync()
    ix.close()
    print(json.dumps({"profile_search": [precision, workload, distance], "reps": args.reps}))


def profile_batch(args):
    """--reps runs of one bf16 batch of Euclidean instances with the batch GPU
    test's distribution (m 1000..20000, n 16..512, d in {32, 64, 128}, k in
    {1, 10, 50}; seeded), device inputs (for ncu)."""
    import numpy as np
    import torch
    from paper_0804_1448_gb300 import inputs, knn
    g = np.random.default_rng(11)
    inst = []
    for i in range(args.profile_batch):
        m = int(g.integers(1000, 20001))
        n = int(g.integers(16, 513))
        d = int(g.choice([32, 64, 128]))
        k = int(g.choice([1, 10, 50]))
        R = torch.from_numpy(inputs.uniform(m, d, seed=10000 + 2 * (11000 + i))).cuda()
        Q = torch.from_numpy(inputs.uniform(n, d, seed=10001 + 2 * (11000 + i))).cuda()
        inst.append(dict(R=R, Q=Q, k=k, dist=torch.empty((n, k), device="cuda"),
                         idx=torch.empty((n, k), dtype=torch.int32, device="cuda")))
    ix = knn.Index(0, "bf16")
    for _ in range(args.reps):
        ix.search_batch(inst)
    ix.sync()
    info = ix.batch_info()
    ix.close()
    print(json.dumps({"profile_batch": args.profile_batch, "reps": args.reps, "batch_info": info}))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.configs:
        configs(args)
        return
    if args.serve_batch > 0:
        serve_batch(args)
        return
    if args.profile_search:
        profile_search(args)
        return
    if args.profile_batch > 0:
        profile_batch(args)
        return
    if args.sweep:
        sweep(args)
        return
    world, rank, local = dist_env()
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_0804_1448_gb300 import inputs, knn

    R, Q, k = inputs.workload(WORKLOAD)
    n, m, d = Q.shape[0], R.shape[0], R.shape[1]
    dev = torch.device("cuda", local)
    Rd = torch.from_numpy(R).to(dev)
    Qd = torch.from_numpy(Q).to(dev)
    dist_out = torch.empty((n, k), dtype=torch.float32, device=dev)
    idx_out = torch.empty((n, k), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)

    def timed_steps(ix, steps, profile_stage=None):
        """Device time of `steps` searches, each after an L2 flush."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        stage_ms = []
        barrier()
        l0 = ix.stats()["kernel_launches"]
        for e0, e1 in ev:
            flush.fill_(1)
            e0.record(stream)
            ix.search_into(Qd, k, dist_out, idx_out, "l2", stream)
            e1.record(stream)
            if profile_stage:
                stage_ms.append(ix.profile().get(profile_stage))
        barrier()
        launches = ix.stats()["kernel_launches"] - l0
        return sum(a.elapsed_time(b) for a, b in ev), stage_ms, launches

    # ---- tensor-core form (the headline)
    ix = knn.Index(local, args.precision)
    ix.set_reference(Rd)
    ix.set_profiling(True)
    for _ in range(max(3, args.warmup)):
        ix.search_into(Qd, k, dist_out, idx_out, "l2", stream)
    ix.sync()
    clocks = Clocks(local)
    clocks.wait_first()
    total_ms, filt_ms, launches = timed_steps(ix, args.steps, "tc_filter")
    prof = ix.profile()
    # the timed steps are shorter than the sampling period: the same searches
    # go on, untimed, for CLOCK_HOLD_S more so that the readings see that load
    t_hold = time.perf_counter() + CLOCK_HOLD_S
    while time.perf_counter() < t_hold:
        flush.fill_(1)
        ix.search_into(Qd, k, dist_out, idx_out, "l2", stream)
        torch.cuda.synchronize(dev)
    clock_info = clocks.stop()
    clock_info["window"] = (f"sampled every 50 ms from before the timed steps to {CLOCK_HOLD_S} s "
                            "of the same searches after them")
    ms_step = max_over_ranks(total_ms / args.steps, pg, dev)
    value = world * n / (ms_step / 1e3)

    # ---- roofline of the dominant kernel (the tensor-core filter pass)
    peaks, peak_src = load_peaks()
    filt = [x for x in filt_ms if x]
    filt_avg = sum(filt) / len(filt) if filt else None
    flops = 2.0 * n * m * d    # algorithmic: 2 m d per query
    achieved = flops / (filt_avg / 1e3) / 1e12 if filt_avg else None
    peak = tensor_peak(peaks, args.precision)
    roofline = {"bound": "tensor", "kernel": "tc_filter", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": filter_traffic(args.precision), "peak_source": f"{peak_src} "
                + ("bf16_tflops (burst)" if args.precision == "bf16"
                   else "bf16_tflops x 1.1/2.25 (nominal tf32:bf16 ratio)"),
                "kernel_ms": filt_avg, "flops_per_launch": flops}

    # ---- float32 CUDA-core form, same workload (the comparator)
    ix32 = knn.Index(local, "fp32")
    ix32.set_reference(Rd)
    for _ in range(3):
        ix32.search_into(Qd, k, dist_out, idx_out, "l2", stream)
    ix32.sync()
    k32 = max(3, args.steps // 6)
    fp32_ms, _, _ = timed_steps(ix32, k32)
    fp32_value = world * n / (max_over_ranks(fp32_ms / k32, pg, dev) / 1e3)
    ix32.close()

    # ---- end to end through the C ABI with pinned host buffers (the plain call:
    # the per-stage profiling events of the device-timed steps are off)
    ix.set_profiling(False)
    Qh = torch.from_numpy(Q).pin_memory()
    dh = torch.empty((n, k), dtype=torch.float32).pin_memory()
    ih = torch.empty((n, k), dtype=torch.int32).pin_memory()
    for _ in range(2):
        ix.search_into(Qh, k, dh, ih, "l2")
    barrier()
    e2e_steps = max(3, args.steps // 3)
    e2e_t = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        ix.search_into(Qh, k, dh, ih, "l2")     # synchronous: Q in, search, results out
        e2e_t.append(time.perf_counter() - t0)
    barrier()
    e2e_s = max_over_ranks(statistics.median(e2e_t), pg, dev)
    e2e = {"value": world * n / e2e_s, "unit": "queries/s",
           "h2d_bytes_per_step": int(n * d * 4), "d2h_bytes_per_step": int(n * k * 8),
           "statistic": f"median of {e2e_steps} wall-clock steps (mean {statistics.mean(e2e_t) * 1e3:.3f} ms)"}
    stats = ix.stats()
    ix.close()

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "m": m, "d": d, "k": k, "distance": "l2",
                       "precision": args.precision, "rerank_factor": 4,
                       "l2": "flushed before every step (256 MiB write), outside the timed window",
                       "step": "one knn_search of all n queries (filter, re-rank, re-check)"},
            "fp32_value": fp32_value, "speedup_vs_fp32": value / fp32_value,
            "stage_ms": prof, "roofline": roofline, "e2e": e2e, "gpu_launches": launches,
            "fallback_queries_total": stats["fallback_queries"], "clocks": clock_info}
    if not args.no_serve:
        line["serve"] = serve_bench(local, args)
    if not args.no_batch:
        line["batch"] = batch_bench(local, args, tensor_peak(peaks, "bf16"), peaks["hbm_gbs"])
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(R, Q, k, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()

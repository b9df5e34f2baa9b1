"""Benchmark of the all-pairs PCC hot path on GB300.

Workload: the output-bound configuration, n = 65,536 genes x l = 512
samples of log2(1 + NB counts) with 200 planted 40-gene modules (FP32
input).  One step = the whole path on one matrix resident in HBM:
standardize (Eq. (5), FP64 row statistics) -> split tensor-core contraction
of the upper triangle (Eq. (6)) writing the packed FP32 triangle
(2,147,450,880 pairs, 8.59 GB) and the fused |r| >= 0.8 edge list.

Metric: Gpair*samples/s = pairs(i<j) * l / time / 1e9.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle (the
baseline this project is measured against) on bounded samples of the same
workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GENES = 65536
L_SAMPLES = 512
SEED = 3
TAU = 0.8
EDGE_CAP = 1 << 24
METRIC = ("all-pairs PCC Gpair·samples/s, split-TC vs plain FP32 GPU at "
          "max|Δr|≤1e-5")
UNIT = "Gpair*samples/s"
WORKLOAD = "output-bound all-pairs PCC, n=65536 x l=512 FP32"
# resolved pcc_prec -> (name, tensor-core products per K step, MMA dtype)
FORMS = {0: ("fp64", 0, "f64"), 1: ("fp32", 0, "f32"),
         2: ("bf16x3", 3, "bf16"), 3: ("fp16x3s", 3, "f16"),
         4: ("bf16x4", 4, "bf16"), 5: ("bf16x1", 1, "bf16")}


def gpair_samples(n, l):
    return n * (n - 1) / 2 * l / 1e9


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained",
                                                      d["bf16_tflops"]), \
            "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}",
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, which):
        """Wall-clock bounds of the timed region (samples outside it are
        dropped when enough fall inside)."""
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["n/a"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(
                    parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]),
                             parts[6:10]))
            except ValueError:
                continue
        os.unlink(self.path)
        t0 = getattr(self, "t0", None)
        t1 = getattr(self, "t1", None)
        inside = [r for r in rows if t0 is not None and t0 <= r[0] <= t1]
        use = inside if len(inside) >= 3 else rows
        reasons = set()
        for r in use:
            for nm, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm = [r[1] for r in use]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "reasons": sorted(reasons), "samples": len(use),
                "window": "timed region" if use is inside else "whole run"}


def kernel_source_hash() -> str:
    """Hash of the pair kernel's sources with comments and blank space
    removed, so that an edit of a comment keeps the committed counters."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("tc_pairs.cu", "tc_epilogue.cuh", "tc_common.cuh",
              "pcc_ptx.cuh", "pcc_sched.h"):
        src = open(os.path.join(ROOT, "paper_1605_01584_gb300", "csrc", f),
                   encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def committed_traffic(n, l):
    """DRAM bytes per launch of the pair kernel from the committed ncu
    summary, scaled to this workload; None once the kernel source differs
    from the one the counters were taken on."""
    p = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
    if not os.path.exists(p):
        return None, "no committed ncu capture"
    d = json.load(open(p))
    if d.get("kernel_src_sha") != kernel_source_hash():
        return None, "kernel changed since the ncu capture"
    scale = (n * (n - 1) / 2) / (d["n"] * (d["n"] - 1) / 2)
    if d.get("l") != l:
        return None, "captured at another l"
    if scale == 1.0:
        return d["dram_bytes_per_launch"], (
            f"ncu dram read+write of one launch at this size (n={d['n']})")
    return d["dram_bytes_per_launch"] * scale, (
        f"ncu dram read+write at n={d['n']}, scaled by pairs x{scale:.2f}")


# ------------------------------------------------------------- CPU oracle
def oracle_rate(X, seconds: float, seed: int = 11):
    """Time the FP64 oracle (as it stands) on a bounded random sample of the
    workload's pairs; returns (Gpair*samples/s, cores, sample text)."""
    import oracle
    n, l = X.shape
    rng = np.random.default_rng(seed)
    X64 = X.astype(np.float64)
    npairs = 20000
    while True:
        I = rng.integers(0, n, npairs)
        J = rng.integers(0, n, npairs)
        t0 = time.perf_counter()
        oracle.pcc_pairs(X64, I, J)
        dt = time.perf_counter() - t0
        if dt >= 0.9 * seconds or npairs >= 1 << 28:
            break
        # grow toward the target; the last round lands on it
        npairs = int(npairs * min(max(seconds / max(dt, 1e-3), 1.1), 64.0))
    rate = npairs * l / dt / 1e9
    sample = (f"{npairs} random pairs (i,j) of the {n}x{l} matrix, Eq. (1) "
              f"in FP64 with per-row mean/SSQ, {dt:.1f} s")
    return rate, oracle.num_threads(), sample


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_single_thread_rate(l: int, seconds: float = 2.0):
    """The oracle's rate on one host thread (a child process started with
    OMP_NUM_THREADS=1, random pairs of a 4,096-row matrix of the same row
    length: the cost per pair*sample depends only on l)."""
    code = (
        "import sys, time, numpy as np\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import oracle, synth\n"
        f"X = synth.counts_log(4096, {l}, 3).astype(np.float64)\n"
        "rng = np.random.default_rng(7); n = 4096; npairs = 2000\n"
        "while True:\n"
        "    I = rng.integers(0, n, npairs); J = rng.integers(0, n, npairs)\n"
        "    t0 = time.perf_counter(); oracle.pcc_pairs(X, I, J)\n"
        "    dt = time.perf_counter() - t0\n"
        f"    if dt >= {seconds} or npairs >= 1 << 26: break\n"
        "    npairs *= 4\n"
        f"print(npairs * {l} / dt / 1e9, oracle.num_threads())\n")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True,
                           text=True, env=env, timeout=120)
        v, th = r.stdout.split()[:2]
        return float(v) if int(th) == 1 else None
    except Exception:
        return None


def oracle_batch_seconds(X64, npairs: int, seed: int) -> float:
    """Wall time of the FP64 oracle (Eq. (1)) on npairs random pairs of X."""
    import oracle
    n = X64.shape[0]
    rng = np.random.default_rng(seed)
    I = rng.integers(0, n, npairs)
    J = rng.integers(0, n, npairs)
    t0 = time.perf_counter()
    oracle.pcc_pairs(X64, I, J)
    return time.perf_counter() - t0


def run_reference(args):
    """The oracle as the reference arm: every step is Eq. (1) in FP64 on one
    batch of random pairs of the same 65,536 x 512 matrix (all host cores),
    the batch sized once so that the whole run takes about two minutes.
    ms_per_step is the measured time of one such batch; the time of the
    whole triangle at the measured rate is reported beside it."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synth
    X = synth.counts_log(N_GENES, L_SAMPLES, SEED)
    X64 = X.astype(np.float64)
    per_step = max(0.5, args.ref_seconds / max(1, args.steps + args.warmup))
    # size the batch (not a step): grow until one batch takes ~per_step
    npairs = 20000
    while True:
        dt = oracle_batch_seconds(X64, npairs, 99)
        if dt >= 0.5 * per_step or npairs >= 1 << 28:
            break
        npairs = int(npairs * min(max(per_step / max(dt, 1e-3), 1.1), 64.0))
    npairs = int(npairs * min(per_step / max(dt, 1e-3), 4.0))
    for s in range(args.warmup):
        oracle_batch_seconds(X64, npairs, 100 + s)
    times = [oracle_batch_seconds(X64, npairs, 200 + s)
             for s in range(args.steps)]
    ms_step = statistics.fmean(times) * 1e3
    value = npairs * L_SAMPLES / (ms_step / 1e3) / 1e9
    cores = oracle.num_threads()
    sample = (f"{npairs} random pairs (i,j) of the {N_GENES}x{L_SAMPLES} "
              "matrix per step, Eq. (1) in FP64 with per-row mean/SSQ")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_GENES, "l": L_SAMPLES,
                   "tau": TAU, "seed": SEED,
                   "step": f"{npairs} random pairs per step (a bounded "
                           "sample of the whole triangle)"},
        "pairs_per_step": npairs,
        "full_triangle_seconds_at_this_rate":
            gpair_samples(N_GENES, L_SAMPLES) / value,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def max_over_ranks(x: float, dist=None) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself
    without a process group.  The reduction runs on the GPU under NCCL and
    on the host under gloo."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args):
    import torch
    import paper_1605_01584_gb300 as pcc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pcc.load()
    import synth
    n, l = args.n, args.l
    X = synth.counts_log(n, l, SEED + 1000 * rank)
    Xd = torch.from_numpy(X).cuda()
    npairs = n * (n - 1) // 2
    R = torch.empty(npairs, dtype=torch.float32, device="cuda")
    E = torch.empty(EDGE_CAP * pcc.EDGE_BYTES, dtype=torch.uint8,
                    device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    Z = pcc.pcc_standardize(Xd, args.prec)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        pcc.pcc_standardize(Xd, args.prec, Z=Z)
        if ev is not None:
            ev[1].record(stream)
        cnt.zero_()
        if ev is not None:
            ev[2].record(stream)
        pcc.pcc_threshold_edges(Z, TAU, E, EDGE_CAP, cnt, R)
        if ev is not None:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = pcc.pcc_sync_status(Z)
    if st != 0:
        raise RuntimeError(f"device status {pcc.pcc_status_string(st)}")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)]
           for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks.mark("t0")
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    std_ms = [e[0].elapsed_time(e[1]) for e in evs]
    pair_ms = [e[2].elapsed_time(e[3]) for e in evs]
    edges_found = int(cnt.item())
    st = pcc.pcc_sync_status(Z)
    if st != 0:
        raise RuntimeError(f"device status {pcc.pcc_status_string(st)}")

    ms_step = max_over_ranks(total_ms / args.steps, dist)
    value = gpair_samples(n, l) * world / (ms_step / 1e3)

    # roofline of the dominant kernel (the fused pair kernel)
    hbm, bf16, bf16_sus, peak_kind = peaks()
    info = Z.info()
    z_bytes = n * info["lpad"] * 2 * (1 if FORMS[info["prec"]][1] == 1 else 2)
    alg_bytes = npairs * 4 + z_bytes + n + min(edges_found, EDGE_CAP) * 12
    pair_avg = statistics.mean(pair_ms)
    achieved_gbs = alg_bytes / (pair_avg / 1e3) / 1e9
    alg_flops = 2.0 * npairs * l
    nprod = FORMS[info["prec"]][1]
    exec_flops = nprod * 2.0 * (info["lpad"]) * 128 * 256 * 2 * (
        (-(-n // 256)) * (-(-n // 256) + 1) // 2)
    exec_tflops = exec_flops / (pair_avg / 1e3) / 1e12

    traffic, traffic_note = committed_traffic(n, l)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": FORMS[info["prec"]][2],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "l": l, "tau": TAU,
                   "split": FORMS[info["prec"]][0],
                   "seed": SEED,
                   "per_rank": "independent matrix per GPU (seed + 1000*rank)",
                   "l2": "inputs larger than L2 (134 MB X; 8.6 GB output "
                         "streamed per step)"},
        "ms_standardize": statistics.mean(std_ms),
        "ms_pairs": pair_avg,
        "edges": edges_found,
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm,
                     "unit": "GB/s", "frac": achieved_gbs / hbm,
                     "traffic": traffic, "traffic_note": traffic_note,
                     "kernel": "k_pairs_tc (fused packed + edges)",
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes},
        "roofline_split_executed": {
            "bound": "tensor", "achieved": exec_tflops, "peak": bf16,
            "unit": "TFLOP/s", "frac": exec_tflops / bf16,
            "executed_flops_per_launch": exec_flops,
            "algorithmic_flops_per_launch": alg_flops,
            "peak_kind": peak_kind + " burst bf16 (the timed region is "
                         f"{args.steps} launches, {args.steps * ms_step:.0f}"
                         " ms back to back)",
            "frac_of_sustained": exec_tflops / bf16_sus},
        "clocks": clk,
        "gpu_launches": 2 * args.steps,
    }

    # plain FP32 CUDA-core comparator on the same matrix
    if not args.skip_fp32:
        Z32 = pcc.pcc_standardize(Xd, "fp32")
        for _ in range(2):
            pcc.pcc_standardize(Xd, "fp32", Z=Z32)
            pcc.pcc_allpairs_upper(Z32, R)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        reps = 3
        a.record(stream)
        for _ in range(reps):
            pcc.pcc_standardize(Xd, "fp32", Z=Z32)
            cnt.zero_()
            pcc.pcc_threshold_edges(Z32, TAU, E, EDGE_CAP, cnt, R)
        b.record(stream)
        torch.cuda.synchronize()
        ms32 = a.elapsed_time(b) / reps
        out["fp32_simt"] = {"ms_per_step": ms32,
                            "value": gpair_samples(n, l) / (ms32 / 1e3),
                            "speedup_split_tc": ms32 / ms_step}
        # its roofline: the FP32 FMA rate of the CUDA cores, measured by a
        # microbenchmark (the driver's peaks hold no such number), beside
        # the nominal SMs x 128 FP32 lanes x 2 flops x max SM clock
        fma = pcc.pcc_measure_fp32_fma()
        sms = torch.cuda.get_device_properties(
            torch.cuda.current_device()).multi_processor_count
        ach = alg_flops / (ms32 / 1e3) / 1e12
        nominal = (sms * 128 * 2 * clk["sm_max_mhz"] * 1e6 / 1e12
                   if clk.get("sm_max_mhz") else None)
        out["fp32_simt"]["roofline"] = {
            "bound": "alu", "achieved": ach, "peak": fma, "unit": "TFLOP/s",
            "frac": ach / fma, "peak_kind": "measured FFMA microbenchmark",
            "nominal_peak": nominal,
            "note": "algorithmic 2l flops per pair over the whole FP32 step"}
        Z32.close()

    # end to end through the C ABI with host buffers: X is copied in by
    # pcc_standardize_host, R streamed out by pcc_threshold_edges_host and
    # the edge list (with its count) by pcc_edges_copy_host, all inside the
    # timed region of every step
    if not args.skip_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        Rh = torch.empty(npairs, dtype=torch.float32, pin_memory=True)
        Eh = torch.empty(EDGE_CAP * pcc.EDGE_BYTES, dtype=torch.uint8,
                         pin_memory=True)
        e2e_steps = max(3, min(args.steps, 10))

        def e2e_step():
            pcc.pcc_standardize_host(Xh, args.prec, Z=Z)
            cnt.zero_()
            if args.e2e_mode == "passes":
                # row-block passes: each pass's slice of R is copied to Rh
                # while the next pass computes (Algorithm 2)
                pcc.pcc_threshold_edges_host(Z, TAU, E, EDGE_CAP, cnt, Rh,
                                             device_bytes=args.e2e_window)
            else:
                pcc.pcc_threshold_edges(Z, TAU, E, EDGE_CAP, cnt, R)
                Rh.copy_(R, non_blocking=True)
            return pcc.pcc_edges_copy_host(E, cnt, EDGE_CAP, Eh)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ne = 0
        # each step ends with its results on the host; the value is the
        # total wall time of the timed steps / steps (the host link's rate
        # varies from step to step on a shared machine: the median step and
        # the spread are reported beside it)
        walls = []
        t_all = time.perf_counter()
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            ne = e2e_step()
            walls.append((time.perf_counter() - t0) * 1e3)
        total_e2e = (time.perf_counter() - t_all) * 1e3
        e2e_ms = max_over_ranks(total_e2e / e2e_steps, dist)
        out["e2e"] = {"value": gpair_samples(n, l) * world / (e2e_ms / 1e3),
                      "unit": UNIT, "ms_per_step": e2e_ms,
                      "statistic": "total wall time of the timed steps / "
                                   "steps",
                      "ms_per_step_median": statistics.median(walls),
                      "ms_per_step_min": min(walls),
                      "ms_per_step_max": max(walls),
                      "ms_each_step": [round(w, 3) for w in walls],
                      "warmup": args.warmup,
                      "steps": e2e_steps,
                      "api": "pcc_standardize_host + "
                             "pcc_threshold_edges_host + "
                             "pcc_edges_copy_host",
                      "h2d_bytes_per_step": X.nbytes,
                      "mode": args.e2e_mode,
                      "d2h_bytes_per_step": npairs * 4 + 8 + min(
                          ne, EDGE_CAP) * 12}

    if rank == 0 and world == 1 and not args.skip_cpu:
        v, cores, sample = oracle_rate(X, args.cpu_seconds)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores,
                               "kind": "oracle", "sample": sample,
                               "cpu_model": cpu_model(),
                               "single_thread_value":
                                   oracle_single_thread_rate(l)}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _graph_timed(fn, steps, warmup):
    """Run `warmup` plain steps (they allocate whatever a first call
    allocates), capture one step in a CUDA graph and time `steps` replays;
    None when the step cannot be captured."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
    except Exception:
        torch.cuda.synchronize()
        return None
    return _timed(g.replay, steps, 1, torch.cuda.current_stream())


def run_perm(args):
    """Permutation test workload: n=4096 x l=256, P=1000 seeded Fisher-Yates
    permutations, counts of |r_k| >= |r_obs| for every pair."""
    import torch
    import paper_1605_01584_gb300 as pcc
    import synth
    pcc.load()
    n, l, P = 4096, 256, args.P
    X = synth.counts_log(n, l, 4)
    perms = synth.fisher_yates_perms(P, l, seed=4)
    Xd = torch.from_numpy(X).cuda()
    dp = torch.from_numpy(perms).cuda()
    Z = pcc.pcc_standardize(Xd, args.prec)
    cnt = torch.zeros(n * (n - 1) // 2, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        pcc.pcc_standardize(Xd, args.prec, Z=Z)
        cnt.zero_()
        pcc.pcc_perm_test(Z, dp, P, 0, P, cnt)

    ms_stream = _timed(step, max(3, min(args.steps, 20)), args.warmup, stream)
    # the whole test (standardize, count reset, gather, pair kernel) as one
    # CUDA graph
    ms_graph = _graph_timed(step, max(3, min(args.steps, 20)), 1)
    ms = ms_graph if ms_graph is not None else ms_stream
    st = pcc.pcc_sync_status(Z)
    # the other forms (0: permuted in shared memory, 1: through a workspace
    # of permuted rows): their times, and the same counts
    ref_cnt = cnt.clone()
    before = pcc.pcc_get_tuning()
    other = {}
    try:
        for form, name in ((0, "shared_memory_form"),
                           (1, "workspace_form")):
            pcc.pcc_set_tuning(perm_form=form)
            ms_f = _timed(step, 3, 1, stream)
            other[name] = {
                "ms_per_step": ms_f,
                "counts_equal": bool(torch.equal(cnt, ref_cnt)),
                "status": pcc.pcc_sync_status(Z),
                "value": n * (n - 1) / 2 * l * P / (ms_f / 1e3) / 1e9}
    finally:
        pcc.pcc_set_tuning(perm_form=before["perm_form"])
    info = Z.info()
    tiles = (-(-n // 128)) * (-(-n // 128) + 1) // 2
    exec_flops = FORMS[info["prec"]][1] * 2 * 128 * 128 * info["lpad"] * tiles * (P + 1)
    alg_flops = n * (n - 1) / 2 * 2.0 * l * P
    _, bf16, bf16_sus, kind = peaks()
    out = {"metric": "permutation-test Gpair*samples*perms/s",
           "value": n * (n - 1) / 2 * l * P / (ms / 1e3) / 1e9,
           "unit": "Gpair*samples*perms/s", "ms_per_step": ms,
           "ms_per_step_stream": ms_stream, "graph": ms_graph is not None,
           "steps": max(3, min(args.steps, 20)), "warmup": args.warmup,
           "status": st, "dtype": FORMS[info["prec"]][2],
           "config": {"workload": f"permutation test n=4096 x l=256, P={P}",
                      "split": args.prec},
           # algorithmic: 2l flops per pair and permutation
           "roofline": {
               "bound": "tensor", "achieved": alg_flops / (ms / 1e3) / 1e12,
               "peak": bf16, "unit": "TFLOP/s",
               "frac": alg_flops / (ms / 1e3) / 1e12 / bf16,
               "peak_kind": kind + " burst bf16 (sub-second timed region)"},
           "roofline_split_executed": {
               "bound": "tensor", "achieved": exec_flops / (ms / 1e3) / 1e12,
               "peak": bf16, "unit": "TFLOP/s",
               "frac": exec_flops / (ms / 1e3) / 1e12 / bf16,
               "peak_kind": kind + " burst bf16",
               "note": "3-product split work of the P permutations and one "
                       "r_obs pass per 128 x 128 tile; the kernel also "
                       "repeats r_obs per chunk of permutations and pads "
                       "lone tiles in the pair form (about 5% more tensor "
                       "work, not counted)"},
           # the other forms (pcc_set_perm_form(0) / (1)), stream-launched,
           # 3 steps
           **other}
    print(json.dumps(out), flush=True)
    return 0


def run_batched(args):
    """Batched uneven workload: 64 matrices, n ~ U{500..20000}, l ~
    U{32..2048}, all pairs of each in one persistent launch."""
    import torch
    import paper_1605_01584_gb300 as pcc
    import synth
    pcc.load()
    # the first `--matrices` of the 64 (a smaller case for profiling)
    shapes = synth.uneven_shapes()[:max(1, args.matrices)]
    Xs, Zs, Rs = [], [], []
    t0 = time.time()
    gen = synth.counts_log_many(shapes, [5 * 1000 + b
                                         for b in range(len(shapes))])
    for X, (n, l) in zip(gen, shapes):
        Xd = torch.from_numpy(X).cuda()
        Xs.append(Xd)
        Zs.append(pcc.pcc_standardize(Xd, args.prec))
        Rs.append(torch.empty(n * (n - 1) // 2, device="cuda"))
    gen_s = time.time() - t0
    stream = torch.cuda.current_stream()
    tune_s = None
    if args.tune:
        # tune every shape bucket of the batch (K = 32, CTA pairs or single
        # CTAs, band heights) into the tune cache before the timed steps
        from paper_1605_01584_gb300 import autotune
        t0 = time.time()
        autotune.tune_batched([(n, l) for n, l in shapes], args.prec)
        tune_s = time.time() - t0
    # per-matrix (CTA form, band rows): the tune cache's best where it has
    # an entry, else the current knobs; resolved once, reused every step
    choices = pcc.pcc_allpairs_upper_batched(Zs, Rs)

    def step():
        # every matrix's standardize in one launch, then every matrix's
        # pairs in one persistent launch per CTA form
        pcc.pcc_standardize_batched(Xs, args.prec, Zs=Zs)
        pcc.pcc_allpairs_upper_batched(Zs, Rs, choices=choices)

    ms_stream = _timed(step, max(3, min(args.steps, 10)), args.warmup, stream)
    # the whole step (one standardize launch per form, one pair launch) as
    # one CUDA graph
    ms_graph = _graph_timed(step, max(3, min(args.steps, 10)), 1)
    ms = ms_graph if ms_graph is not None else ms_stream

    def kern():
        pcc.pcc_allpairs_upper_batched(Zs, Rs, choices=choices)

    ms_k = _timed(kern, max(3, min(args.steps, 10)), 1, stream)
    st = pcc.pcc_sync_status(Zs[0])
    work = sum(n * (n - 1) / 2 * l for n, l in shapes) / 1e9
    out_bytes = sum(n * (n - 1) / 2 * 4 for n, l in shapes)
    hbm, bf16, bf16_sus, kind = peaks()
    # executed tensor work: every 256 x 256 super-tile of each triangle
    # (diagonal ones whole), at the padded row length and the matrix's
    # number of products
    exec_flops = 0.0
    for (n, l), Z in zip(shapes, Zs):
        info = Z.info()
        m = -(-n // 256)
        exec_flops += (FORMS[info["prec"]][1] * 2.0 * 256 * 256 *
                       info["lpad"] * m * (m + 1) / 2)
    out = {"metric": "batched all-pairs Gpair*samples/s", "value": work /
           (ms / 1e3), "unit": "Gpair*samples/s", "ms_per_step": ms,
           "ms_per_step_stream": ms_stream, "graph": ms_graph is not None,
           "ms_batched_kernel": ms_k, "status": st,
           "config": {"workload": f"{len(shapes)} uneven matrices "
                      "n~U{500..20000}, l~U{32..2048}", "split": args.prec,
                      "matrices": len(shapes), "gen_seconds": gen_s,
                      "tuned": bool(args.tune), "tune_seconds": tune_s},
           "choices": {
               "per_matrix": [{"n": n, "l": l, "pair": c[0], "band_rows":
                               c[1]} for (n, l), c in zip(shapes, choices)],
               "pair_form_matrices": sum(c[0] for c in choices),
               "single_cta_matrices": sum(1 - c[0] for c in choices),
               "launches": (1 if all(c[0] for c in choices) or
                            not any(c[0] for c in choices) else 2)},
           "roofline": {"bound": "hbm", "achieved": out_bytes / (ms_k / 1e3)
                        / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": out_bytes / (ms_k / 1e3) / 1e9 / hbm,
                        "note": "output bytes only"},
           "roofline_split_executed": {
               "bound": "tensor", "achieved": exec_flops / (ms_k / 1e3) / 1e12,
               "peak": bf16, "unit": "TFLOP/s",
               "frac": exec_flops / (ms_k / 1e3) / 1e12 / bf16,
               "executed_flops_per_launch": exec_flops,
               "peak_kind": kind + " burst bf16 (sub-second timed region)"}}
    print(json.dumps(out), flush=True)
    return 0


def run_cross(args):
    """Non-symmetric workload (Eq. (7)-(8)): r(x_i, y_j) between X = n x l
    and Y = n/2 x l (log counts; default 65,536 and 32,768 x 512), dense
    FP32 R (8.6 GB at the default)."""
    import torch
    import paper_1605_01584_gb300 as pcc
    import synth
    pcc.load()
    nx, ny, l = args.n, args.n // 2, args.l
    X = synth.counts_log(nx, l, 6)
    Y = synth.counts_log(ny, l, 7)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    ZX = pcc.pcc_standardize(Xd, args.prec)
    ZY = pcc.pcc_standardize(Yd, args.prec)
    R = torch.empty((nx, ny), device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        pcc.pcc_standardize(Xd, args.prec, Z=ZX)
        pcc.pcc_standardize(Yd, args.prec, Z=ZY)
        pcc.pcc_cross_allpairs(ZX, ZY, R)

    def kern():
        pcc.pcc_cross_allpairs(ZX, ZY, R)

    steps = max(3, min(args.steps, 20))
    ms = _timed(step, steps, args.warmup, stream)
    ms_k = _timed(kern, steps, 1, stream)
    st = pcc.pcc_sync_status(ZX)
    info = ZX.info()
    tiles = pcc.pcc_cross_num_tiles(ZX, ZY)
    nprod = FORMS[info["prec"]][1]
    exec_flops = nprod * 2 * 256 * 256 * info["lpad"] * tiles
    out_bytes = nx * ny * 4 + 2 * 2 * (nx + ny) * info["lpad"]
    hbm, bf16, bf16_sus, kind = peaks()
    out = {"metric": "cross all-pairs Gpair*samples/s",
           "value": nx * ny * l / (ms / 1e3) / 1e9,
           "unit": "Gpair*samples/s", "ms_per_step": ms,
           "ms_cross_kernel": ms_k, "steps": steps, "warmup": args.warmup,
           "status": st, "dtype": FORMS[info["prec"]][2],
           "config": {"workload": f"cross X {nx}x{l} vs Y {ny}x{l}, dense "
                      "FP32 R", "split": args.prec,
                      "l2": "inputs and the 8.6 GB output exceed L2"},
           "roofline": {"bound": "hbm", "achieved": out_bytes /
                        (ms_k / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": out_bytes / (ms_k / 1e3) / 1e9 / hbm},
           "roofline_split_executed": {
               "bound": "tensor", "achieved": exec_flops / (ms_k / 1e3)
               / 1e12, "peak": bf16, "unit": "TFLOP/s",
               "frac": exec_flops / (ms_k / 1e3) / 1e12 / bf16,
               "peak_kind": kind + " burst bf16 (sub-second timed region)"}}
    print(json.dumps(out), flush=True)
    return 0


def run_paper(args):
    """The paper's own shapes, as context (Section IV): U[0,1] with n = 16K,
    32K, 64K and l = 5,000, and a 17,555 x 5,072 log-count stand-in for the
    human dataset; each in FP64 on CUDA cores (the paper's precision) and in
    the default split form on tensor cores, one full triangle per run.  The
    split form's error is taken over every pair against the FP64 CUDA-core
    triangle (which the parity tests hold within 1e-12 of Eq. (1)).  The
    paper's one-Phi times are quoted beside them."""
    import torch
    import paper_1605_01584_gb300 as pcc
    import synth
    pcc.load()
    shapes = [("uniform 16K x 5K", 16000, 5000, 27.4),
              ("uniform 32K x 5K", 32000, 5000, 83.2),
              ("uniform 64K x 5K", 64000, 5000, 285.4),
              ("counts 17,555 x 5,072 (human stand-in)", 17555, 5072, 32.1)]
    runs = []

    def max_diff(a, b):
        """max |a - b| over the pairs both hold a number, and whether their
        NaN (flagged-row) patterns differ, in chunks of 2^28 pairs."""
        m, mismatch = 0.0, False
        for k in range(0, a.numel(), 1 << 28):
            x, y = a[k:k + (1 << 28)].double(), b[k:k + (1 << 28)]
            nx, ny = torch.isnan(x), torch.isnan(y)
            mismatch |= bool((nx != ny).any())
            d = (x - y).abs().masked_fill(nx | ny, 0.0)
            m = max(m, float(d.max()))
        return m, mismatch

    for name, n, l, phi_s in shapes:
        if n > args.n:
            continue
        if name.startswith("uniform"):
            X = synth.uniform01(n, l, 8)
        else:
            X = synth.counts_log(n, l, 9)
        Xd = torch.from_numpy(X).cuda()
        ref = None
        for prec in ("fp64", args.prec):
            dt = torch.float64 if prec == "fp64" else torch.float32
            R = torch.empty(n * (n - 1) // 2, dtype=dt, device="cuda")
            Z = pcc.pcc_standardize(Xd, prec)

            def step():
                pcc.pcc_standardize(Xd, prec, Z=Z)
                pcc.pcc_allpairs_upper(Z, R)

            step()
            torch.cuda.synchronize()
            reps = 1 if prec == "fp64" else 3
            ms = _timed(step, reps, 0, torch.cuda.current_stream())
            st = pcc.pcc_sync_status(Z)
            info = Z.info()
            run = {"data": name, "n": n, "l": l,
                   "form": FORMS[info["prec"]][0],
                   "seconds": ms / 1e3, "status": st,
                   "Gpair_samples_per_s": n * (n - 1) / 2 * l
                   / (ms / 1e3) / 1e9,
                   "paper_one_phi_fp64_seconds": phi_s}
            if ref is None:
                ref = R
            else:
                err, mism = max_diff(R, ref)
                run["max_abs_dr_vs_fp64_all_pairs"] = err
                run["nan_pattern_differs"] = mism
                del R
            runs.append(run)
            print(json.dumps(runs[-1]), file=sys.stderr, flush=True)
            del Z
            torch.cuda.empty_cache()
        del ref
        torch.cuda.empty_cache()
    out = {"metric": "paper-shape context runs (seconds per full triangle)",
           "unit": "s", "runs": runs,
           "note": "context only: the paper's times are FP64 on one 5110P "
                   "Xeon Phi (Table of Section IV)",
           "config": {"workload": "paper shapes", "split": args.prec}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="auto",
                    choices=["auto", "bf16x3", "fp16x3s", "bf16x4",
                             "bf16x1"])
    ap.add_argument("--workload", default="allpairs",
                    choices=["allpairs", "perm", "batched", "cross",
                             "paper"])
    ap.add_argument("--n", type=int, default=N_GENES)
    ap.add_argument("--matrices", type=int, default=64,
                    help="matrices of the batched workload (its first K)")
    ap.add_argument("--tune", action="store_true",
                    help="batched workload: tune each shape bucket first")
    ap.add_argument("--P", type=int, default=1000,
                    help="permutations of the perm workload")
    ap.add_argument("--l", type=int, default=L_SAMPLES)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="--impl reference: about this many seconds of "
                         "oracle work over all steps")
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--e2e-mode", default="passes",
                    choices=["passes", "oneshot"],
                    help="host delivery of R: overlapped row-block passes "
                         "or one kernel then one copy")
    ap.add_argument("--e2e-window", type=int, default=0,
                    help="device bytes for the two pass windows (0: auto)")
    ap.add_argument("--skip-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "perm":
        return run_perm(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "cross":
        return run_cross(args)
    if args.workload == "paper":
        return run_paper(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

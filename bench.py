"""Benchmark of the Cleora propagation path on GB300.

One step = one pass of the whole path over the device-resident edge list of the workload:
graph build (id map + CSR), init of T_0, and I propagation iterations
(T_k = rownorm_L2(M T_{k-1})).  The metric is nnz*d/s per iteration, nnz being the CSR
entries: nnz*d / (median per-iteration time), BF16 storage (headline) and FP32 storage.

Default workload: undirected power-law graph, 41M nodes, 1.4B edges (2.8B CSR entries,
max degree ~3M), unit weights, d = 128, I = 4, generated on the GPU.  Inputs (T: 10.5-21 GB,
gathered bytes ~0.7-1.4 TB per iteration) are far larger than L2, so no flush is needed.

Reports: roofline of the propagate kernel against the measured HBM copy bandwidth, an
end-to-end figure through the C ABI with host buffers, the FP64 CPU oracle timed on a
bounded sample (cpu_baseline), SM clocks sampled during the timed region.

``--impl reference`` times the FP64 CPU oracle (the only reference this method has) on the
same workload family, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {
    "large": synth.LARGE,
    "mid": synth.MID,
    "small": synth.SMALL,
    # a 1/40 scale copy of the large graph (profiling and quick runs)
    "large_1_40": synth.PowerLawSpec("chung_lu_1M_35M_undirected_d128", 1_025_000, 35_000_000,
                                     2.0, 150_000.0, False, None, 128, 4),
}

# Bounded CPU sample of each workload for the oracle timing: same generator family, smaller.
CPU_SAMPLES = {
    "large": synth.PowerLawSpec("chung_lu_250k_8.5M_undirected_d128", 250_000, 8_500_000, 2.0,
                                18_000.0, False, None, 128, 4),
    "mid": synth.PowerLawSpec("chung_lu_200k_4M_directed_lognormal_d256", 200_000, 4_000_000, 2.1,
                              10_000.0, True, "lognormal", 256, 4),
    "small": synth.SMALL,
}
CPU_SAMPLES["large_1_40"] = CPU_SAMPLES["large"]


STAGING_LABELS = {0: "automatic", 1: "registers", 2: "ring (bulk copy per row)",
                  3: "ring (4-row tensor gathers)"}


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (identity when not
    distributed).  CPU tensors for gloo, CUDA tensors for nccl."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(units_per_rank, world, seconds_max):
    """Replicas on every rank: units all ranks processed / the slowest rank's time."""
    return units_per_rank * world / seconds_max


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


PROP_SOURCES = ["paper_2102_02302_gb300/csrc/propagate_kernels.cuh",
                "paper_2102_02302_gb300/csrc/propagate.cu",
                "paper_2102_02302_gb300/csrc/prop_f32_v16.cu", "paper_2102_02302_gb300/csrc/prop_f32_v8.cu",
                "paper_2102_02302_gb300/csrc/prop_bf16_v16.cu", "paper_2102_02302_gb300/csrc/prop_bf16_v8.cu"]
BATCH_SOURCES = PROP_SOURCES + ["paper_2102_02302_gb300/csrc/batch_kernels.cuh",
                                "paper_2102_02302_gb300/csrc/batch.cu",
                                "paper_2102_02302_gb300/csrc/batch_f32_v16.cu",
                                "paper_2102_02302_gb300/csrc/batch_f32_v8.cu",
                                "paper_2102_02302_gb300/csrc/batch_bf16_v16.cu",
                                "paper_2102_02302_gb300/csrc/batch_bf16_v8.cu"]


def source_sha(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        p = os.path.join(ROOT, f)
        if os.path.exists(p):
            with open(p, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_source_sha():
    return source_sha(PROP_SOURCES)


def measured_traffic(key, files=None):
    """DRAM bytes (read + write) per launch (per replay for the batch) from the committed
    ncu summary profiles/traffic.json, or None when the sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    e = t.get("entries", {}).get(key)
    if e is None or e.get("source_sha") != source_sha(files or PROP_SOURCES):
        return None
    return e["dram_bytes"]


def model_bytes(n, nnz, d, es, has_val):
    """Algorithmic bytes of one iteration: rowptr and col (and val) read once, one gathered
    row per CSR entry, every row written once."""
    return 8 * (n + 1) + 4 * nnz + (4 * nnz if has_val else 0) + es * d * nnz + es * d * n


def compulsory_bytes(n, nnz, d, es, has_val):
    """Lower bound with perfect reuse: CSR once, T read once, T written once."""
    return 8 * (n + 1) + 4 * nnz + (4 * nnz if has_val else 0) + 2 * es * d * n


def roofline_block(n, nnz, d, es, hv, iter_s, traffic, peak, peak_kind, kernel):
    """Roofline of one propagate launch (one iteration).  `achieved` and `frac` are read on
    DRAM bytes from ncu (dram__bytes_read + write per launch) over the CUDA-event time; the
    byte model (CSR once, one gathered row per entry, T written once) and the compulsory
    bytes (T read once) are reported beside it.  Without a DRAM capture of the current kernel
    build the model figure stands in and `basis` says so."""
    mb = model_bytes(n, nnz, d, es, hv)
    cb = compulsory_bytes(n, nnz, d, es, hv)
    model_gbs, comp_gbs = mb / iter_s / 1e9, cb / iter_s / 1e9
    if traffic is not None:
        achieved, basis = traffic / iter_s / 1e9, "dram bytes (ncu) / CUDA-event time"
    else:
        achieved, basis = model_gbs, "byte model (no DRAM capture of this kernel build)"
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "basis": basis, "kernel": kernel,
            "launch_ms": iter_s * 1e3,
            "model_bytes": mb, "model_gbs": model_gbs, "model_frac": model_gbs / peak,
            "compulsory_bytes": cb, "compulsory_frac": comp_gbs / peak,
            "bytes_model": "8(n+1) + 4nnz (+4nnz values) + s*d*nnz gathered + s*d*n written",
            "peak_kind": f"{peak_kind} copy bandwidth (frac of {peak_kind})",
            "kernel_sha": kernel_source_sha()}


def prop_kernel_name(st, d):
    es = 4 if st == "f32" else 2
    vec = 16 if d * es // 16 >= 32 else 8
    return f"k_propagate<{'float' if st == 'f32' else '__nv_bfloat16'}, {vec}, ...>"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------------------

def oracle_sample_setup(workload):
    import oracle
    spec = CPU_SAMPLES[workload]
    e = spec.generate()
    g = oracle.build_from(e)
    T0 = oracle.init(g.ids, spec.d, 0)
    return spec, g, T0


def oracle_iteration_rate(spec, g, T0, iters=1):
    import oracle
    t = time.perf_counter()
    oracle.propagate(g, T0, iters)
    dt = (time.perf_counter() - t) / iters
    return g.nnz * spec.d / dt, dt


def cpu_baseline(workload):
    spec, g, T0 = oracle_sample_setup(workload)
    rate, dt = oracle_iteration_rate(spec, g, T0, 1)
    cores = os.cpu_count() or 1
    return {"value": rate, "unit": "nnz*d/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, one propagation iteration of {spec.name} "
                      f"(n={g.n}, nnz={g.nnz}, d={spec.d}; same generator family as the "
                      f"workload, smaller), {dt:.2f} s on {cores} threads"}


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    spec, g, T0 = oracle_sample_setup(args.workload)
    for _ in range(args.warmup):
        oracle_iteration_rate(spec, g, T0, 1)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_iteration_rate(spec, g, T0, 1)
        times.append(dt)
    dt = float(np.median(times))
    value = g.nnz * spec.d / dt
    cores = os.cpu_count() or 1
    line = {
        "impl": "reference", "metric": "nnz*d/s per iteration", "value": value,
        "unit": "nnz*d/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload].name, "sample": spec.name,
                   "n": g.n, "nnz": g.nnz, "d": spec.d},
        "cpu_baseline": {"value": value, "unit": "nnz*d/s", "cores": cores, "kind": "oracle",
                         "sample": f"one FP64 oracle iteration per step of {spec.name} "
                                   f"(n={g.n}, nnz={g.nnz}, d={spec.d})"},
        "e2e": {"value": value, "unit": "nnz*d/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

def make_edges(spec, device):
    """Device-resident edge list of the workload (src, dst int64 tensors holding uint64 ids,
    weights or None)."""
    import torch
    if not spec.directed and spec.weights is None and spec.n >= 1_000_000:
        import synth.gpu
        src, dst, meta = synth.gpu.chung_lu_undirected(spec.n, spec.edges, spec.gamma, spec.seed,
                                                       spec.max_deg)
        return src, dst, None, meta
    e = spec.generate()
    src = torch.from_numpy(e.src.view(np.int64)).to(device)
    dst = torch.from_numpy(e.dst.view(np.int64)).to(device)
    w = None if e.weights is None else torch.from_numpy(e.weights).to(device)
    return src, dst, w, e.meta


def time_dtype(pkg, ctx, edges, spec, storage, steps, warmup, events_ok=True):
    """Warm-up, then `steps` timed steps (build + init + I iterations), CUDA events on the
    context's stream.  Returns per-step and per-iteration times (ms) and launch counts."""
    import torch
    src, dst, w, _ = edges
    stream = torch.cuda.current_stream()

    def step(record):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(spec.iters + 3)]
        ev[0].record(stream)
        ctx.graph_build(src, dst, w, spec.directed)
        ev[1].record(stream)
        ctx.init(spec.d, 0, storage)
        ev[2].record(stream)
        for k in range(spec.iters):
            ctx.propagate(1)
            ev[3 + k].record(stream)
        return ev

    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize()
    l0 = ctx.launches()
    all_ev = []
    torch.cuda.nvtx.range_push(f"timed_{storage}")  # lets a profiler keep only timed launches
    t0 = time.perf_counter()
    for _ in range(steps):
        all_ev.append(step(True))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - t0
    launches = ctx.launches() - l0
    step_ms, build_ms, init_ms, iter_ms = [], [], [], []
    for ev in all_ev:
        step_ms.append(ev[0].elapsed_time(ev[-1]))
        build_ms.append(ev[0].elapsed_time(ev[1]))
        init_ms.append(ev[1].elapsed_time(ev[2]))
        for k in range(spec.iters):
            iter_ms.append(ev[2 + k].elapsed_time(ev[3 + k]))
    return {"step_ms": step_ms, "build_ms": build_ms, "init_ms": init_ms, "iter_ms": iter_ms,
            "wall_s": wall, "launches": launches}


def e2e_buffers(spec, edges):
    """Pinned host buffers of the end-to-end measurement: the edge list and room for the
    FP32 result (at most spec.n rows).  Allocated once, early, like an application's
    long-lived staging buffers."""
    import torch

    def pinned_copy(t):  # a pinned host buffer filled straight from the device tensor
        if t is None:
            return None
        h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
        h.copy_(t)
        return h

    src_h, dst_h, w_h = (pinned_copy(t) for t in edges[:3])
    out = torch.empty((spec.n, spec.d), dtype=torch.float32, pin_memory=True)
    return (src_h, dst_h, w_h), out


def e2e_measure(pkg, spec, host_edges, out_buf, storage, steps, device):
    """Through the public API with host buffers: upload + build + init + I iterations +
    FP32 result back to host, every step."""
    import torch
    src_h, dst_h, w_h = host_edges
    with pkg.Context(device) as ctx:
        ctx.graph_build(src_h, dst_h, w_h, spec.directed)
        n = ctx.info()["n"]
        out = out_buf[:n]
        times, phases = [], []
        for s in range(steps + 1):  # first one warms the pool
            t = time.perf_counter()
            ctx.graph_build(src_h, dst_h, w_h, spec.directed)
            t1 = time.perf_counter()
            ctx.init(spec.d, 0, storage)
            ctx.sync()
            t2 = time.perf_counter()
            ctx.propagate(spec.iters, out)
            ctx.sync()
            t3 = time.perf_counter()
            if s > 0:
                times.append(t3 - t)
                phases.append((t1 - t, t2 - t1, t3 - t2))
    h2d = src_h.numel() * 8 * 2 + (0 if w_h is None else w_h.numel() * 4)
    d2h = n * spec.d * 4
    # the host link alone: the same edge upload as plain copies into device tensors
    dsrc = torch.empty_like(src_h, device=f"cuda:{device}")
    ddst = torch.empty_like(dst_h, device=f"cuda:{device}")
    torch.cuda.synchronize()
    t = time.perf_counter()
    dsrc.copy_(src_h, non_blocking=True)
    ddst.copy_(dst_h, non_blocking=True)
    torch.cuda.synchronize()
    t_link = time.perf_counter() - t
    del dsrc, ddst
    torch.cuda.empty_cache()
    ph = np.median(np.array(phases), axis=0)
    split = {"upload_build_s": float(ph[0]), "init_s": float(ph[1]), "iterate_download_s": float(ph[2]),
             "edge_copy_only_s": t_link}
    return float(np.median(times)), h2d, d2h, split


# ---------------------------------------------------------------------------------------
# Batched small graphs (4096 graphs, one persistent launch per step, CUDA-graph replay)
# ---------------------------------------------------------------------------------------

def _gen_batch_chunk(specs):
    out = []
    for sp in specs:
        e = sp.generate()
        out.append((e.src, e.dst, e.weights, e.directed))
    return out


def generate_batch(count=4096, seed=0, workers=None):
    """The batched workload: n log-uniform in [50, 50000], average degree U[4, 30], directed
    with probability 1/2, uniform(0.1, 1) weights, d in {64, 128, 256}, I in {3, 4, 5}."""
    import multiprocessing as mp
    specs = synth.batch_specs(count, seed)
    workers = workers or min(16, os.cpu_count() or 1)
    chunks = [specs[i::workers] for i in range(workers)]
    with mp.get_context("spawn").Pool(workers) as pool:  # spawn: safe next to CUDA
        parts = pool.map(_gen_batch_chunk, chunks)
    edges = [None] * count
    for w, part in enumerate(parts):
        for k, e in enumerate(part):
            edges[w + k * workers] = e
    return specs, edges


def batch_measure(device, steps, warmup, count=4096, peak=None, peak_kind="measured", autotune=True):
    import torch
    import paper_2102_02302_gb300 as pkg
    t = time.perf_counter()
    specs, edges = generate_batch(count)
    gen_s = time.perf_counter() - t
    descs = [{"src": e[0], "dst": e[1], "weights": e[2], "directed": e[3], "d": sp.d,
              "iters": sp.iters, "seed": sp.seed, "storage": "bf16"} for sp, e in zip(specs, edges)]
    stream = torch.cuda.Stream(device)
    t = time.perf_counter()
    with pkg.Batch(descs, device, stream.cuda_stream, autotune=autotune) as b:
        create_s = time.perf_counter() - t
        del descs, edges
        tot = b.totals
        work = 0
        mbytes = 0  # byte model of one replay (every graph is weighted: per-entry values)
        sched = {}
        for g, sp in enumerate(specs):
            inf = b.info(g)
            work += inf["nnz"] * sp.d * sp.iters
            mbytes += sp.iters * model_bytes(inf["n"], inf["nnz"], sp.d, 2, True)
            mbytes += (2 + 2 + 4) * sp.d * inf["n"]  # T_0 written; last T read, FP32 out written
            sched.setdefault(f"bf16_d{sp.d}", b.schedule(g))
        for _ in range(warmup):
            b.run(None)
        times = []
        torch.cuda.nvtx.range_push("timed_batch")  # lets a profiler keep only timed launches
        with torch.cuda.stream(stream):
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pkg.cleora_batch_run(b.handle, None)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        torch.cuda.nvtx.range_pop()
        run_ms = float(np.median(times))
        launches = b.launches()
    replay_s = run_ms * 1e-3
    traffic = measured_traffic("batch/bf16", BATCH_SOURCES)
    if peak is None:
        peak, peak_kind = measured_peaks()
    model_gbs = mbytes / replay_s / 1e9
    achieved = model_gbs if traffic is None else traffic / replay_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            "basis": ("byte model (no DRAM capture of this kernel build)" if traffic is None
                      else "dram bytes (ncu) of one replay / CUDA-event replay time"),
            "model_bytes": mbytes, "model_gbs": model_gbs, "model_frac": model_gbs / peak,
            "bytes_model": "sum over graphs of I * (8(n+1) + 8nnz + 2*d*nnz + 2*d*n) + 8*d*n (init, output)",
            "peak_kind": f"{peak_kind} copy bandwidth (frac of {peak_kind})",
            "kernel_sha": source_sha(BATCH_SOURCES)}
    return {"graphs": count, "storage": "bf16", "nodes": tot["nodes"], "nnz": tot["nnz"],
            "roofline": roof,
            "autotune": autotune,
            "nnz_d_iters": work, "value": work / (run_ms * 1e-3), "unit": "nnz*d/s",
            "run_ms": run_ms, "launches_per_run": launches, "max_iters": tot["max_iters"],
            "schedules": sched, "generate_s": gen_s, "create_s": create_s,
            "value_def": "sum over graphs of nnz*d*I / CUDA-graph replay time (init, all steps, FP32 output)"}


# ---------------------------------------------------------------------------------------
# Serving: Poisson arrivals at 80% of measured capacity, p50/p99 arrival -> result on host
# ---------------------------------------------------------------------------------------

def serve_pool(count=48, seed=0):
    """Job graphs: n log-uniform in [1e3, 5e6] (quantiles), average degree U[5, 40],
    undirected unit-weight Chung-Lu (exponent 2.1), generated on the GPU, kept in pinned
    host memory."""
    import torch
    import synth.gpu
    r = (synth.rng(seed, 200, np.arange(count, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    pool = []
    for k in range(count):
        q = (k + 0.5) / count
        n = int(round(math.exp(math.log(1e3) + q * (math.log(5e6) - math.log(1e3)))))
        deg = 5.0 + 35.0 * r[k]
        E = max(1, int(n * deg / 2))
        src, dst, meta = synth.gpu.chung_lu_undirected(n, E, 2.1, seed * 1000 + k, max(10.0, 0.02 * 2 * E))
        pool.append({"n": n, "src": src.cpu().pin_memory(), "dst": dst.cpu().pin_memory(), "edges": meta["edges"]})
        del src, dst
    torch.cuda.empty_cache()
    return pool


def serve_jobs(pool, count, seed):
    cnt = np.arange(count, dtype=np.uint64)
    u = [(synth.rng(seed, 300 + k, cnt) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 for k in range(4)]
    logs = np.log([p["n"] for p in pool])
    jobs = []
    for i in range(count):
        ln = math.log(1e3) + u[0][i] * (math.log(5e6) - math.log(1e3))
        g = int(np.argmin(np.abs(logs - ln)))
        d = (64, 128, 256, 1024)[min(int(u[1][i] * 4), 3)]
        it = (3, 4, 5)[min(int(u[2][i] * 3), 2)]
        st = "bf16" if u[3][i] < 0.5 else "f32"
        jobs.append((g, d, it, st))
    return jobs


def release_pinned_cache():
    """Pinned host buffers that torch frees stay in its host allocator's cache (still pinned);
    hand them back so that later pinned allocations can use that memory."""
    import gc
    import torch
    gc.collect()
    f = getattr(torch._C, "_host_emptyCache", None)
    if f is not None:
        f()


class PinnedArena:
    """First-fit allocator over one pinned host buffer (job outputs land here directly)."""

    def __init__(self, nbytes):
        import threading
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        self.np = self.buf.numpy()
        self.free = [(0, nbytes)]
        self.cv = threading.Condition()

    def alloc(self, nbytes):
        nbytes = (nbytes + 255) // 256 * 256
        for i, (off, size) in enumerate(self.free):
            if size >= nbytes:
                if size == nbytes:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + nbytes, size - nbytes)
                return off, nbytes
        return None

    def release(self, off, nbytes):
        with self.cv:
            self.free.append((off, nbytes))
            self.free.sort()
            merged = []
            for o, sz in self.free:
                if merged and merged[-1][0] + merged[-1][1] == o:
                    merged[-1] = (merged[-1][0], merged[-1][1] + sz)
                else:
                    merged.append((o, sz))
            self.free = merged
            self.cv.notify_all()

    def view(self, off, rows, d):
        return self.np[off: off + rows * d * 4].view(np.float32).reshape(rows, d)


def serve_run(srv, pool, arena, jobs, arrivals, start):
    """Feeds jobs at their arrival times (waiting for output space when the arena is full)
    and collects them in completion order.  Returns per-job results in job order."""
    import threading
    ids, regions, out = {}, {}, {}
    lock = threading.Lock()

    def feeder():
        for k, (g, d, it, st) in enumerate(jobs):
            delay = start + arrivals[k] - srv.now()
            if delay > 0:
                time.sleep(delay)
            p = pool[g]
            with arena.cv:
                while (reg := arena.alloc(p["n"] * d * 4)) is None:
                    arena.cv.wait(0.05)
            buf = arena.view(reg[0], p["n"], d)
            jid = srv.submit(p["src"], p["dst"], None, False, d, it, 1000 + k, st, buf, nodes_hint=p["n"])
            with lock:
                ids[jid] = k
                regions[jid] = reg

    th = threading.Thread(target=feeder)
    th.start()
    while len(out) < len(jobs):
        r = srv.next(1000)
        if r is None:
            continue
        jid, res = r
        with lock:
            k = ids[jid]
            reg = regions.pop(jid)
        arena.release(*reg)
        out[k] = res
    th.join()
    return [out[k] for k in range(len(jobs))]


def serve_measure(device, n_jobs=2000, n_capacity=600, warm=100, slots=8, seed=0,
                  arena_bytes=96 << 30, short_slots=2, short_job_s=0.02):
    import paper_2102_02302_gb300 as pkg
    t = time.perf_counter()
    pool = serve_pool(seed=seed)
    arena = None
    for gb in (96, 64, 48, 32, 16):  # as much pinned output space as the host gives
        if (gb << 30) > arena_bytes:
            continue
        try:
            arena = PinnedArena(gb << 30)
            arena_bytes = gb << 30
            break
        except RuntimeError:
            release_pinned_cache()
    if arena is None:
        raise RuntimeError("no pinned host memory for the serving output arena")
    gen_s = time.perf_counter() - t
    with pkg.Server(device, max_slots=slots, short_slots=short_slots, short_job_seconds=short_job_s) as srv:
        # capacity: closed loop (every job available at once; output space is the only gate)
        cap_jobs = serve_jobs(pool, n_capacity, seed + 1)
        t0 = srv.now()
        res = serve_run(srv, pool, arena, cap_jobs, np.zeros(n_capacity), t0)
        done_t = np.sort([r.t_done for r in res])
        lo, hi = int(0.1 * n_capacity), int(0.9 * n_capacity)  # steady state: middle 80%
        capacity = (hi - lo) / (done_t[hi] - done_t[lo])
        # open loop: Poisson arrivals at 80% of capacity
        lam = 0.8 * capacity
        jobs = serve_jobs(pool, n_jobs, seed + 2)
        u = (synth.rng(seed, 400, np.arange(n_jobs, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        arrivals = np.cumsum(-np.log(1.0 - u) / lam)
        start = srv.now() + 0.05
        results = serve_run(srv, pool, arena, jobs, arrivals, start)
    ok = [r for r in results if r.status == 0]
    arr = start + arrivals
    lat = np.array([r.t_done - a for r, a in zip(results, arr)])[warm:]
    wait = np.array([r.t_admit - a for r, a in zip(results, arr)])[warm:]
    svc = np.array([r.t_done - r.t_admit for r in results])[warm:]
    # the feeder's wait for output space (arrival -> submit) and the server's own latency
    # (submit -> result in host memory)
    feed = np.array([r.t_submit - a for r, a in zip(results, arr)])[warm:]
    srv_lat = np.array([r.t_done - r.t_submit for r in results])[warm:]
    # the service split by phase: upload + build, init, iterations + FP32 rows to the host
    ph_build = np.array([r.t_built - r.t_admit for r in results])[warm:]
    ph_init = np.array([r.t_inited - r.t_built for r in results])[warm:]
    ph_iter = np.array([r.t_done - r.t_inited for r in results])[warm:]
    span = max(r.t_done for r in results[warm:]) - arr[warm]
    work = sum(r.nnz * j[1] * j[2] for r, j in zip(results[warm:], jobs[warm:]))
    big = np.array([pool[j[0]]["n"] * j[1] for j in jobs])[warm:]
    q = np.percentile(big, 90)
    # latency per size class: quartiles of the job's work (pool graph edges * d * I)
    work_j = np.array([pool[j[0]]["edges"] * j[1] * j[2] for j in jobs])[warm:]
    edges_q = np.percentile(work_j, [25, 50, 75])
    cls = np.searchsorted(edges_q, work_j, side="right")
    by_size = []
    for c in range(4):
        sel = lat[cls == c]
        if sel.size:
            by_size.append({"class": f"work quartile {c + 1}", "jobs": int(sel.size),
                            "p50_ms": float(np.percentile(sel, 50) * 1e3),
                            "p99_ms": float(np.percentile(sel, 99) * 1e3),
                            "queue_wait_p99_ms": float(np.percentile(wait[cls == c], 99) * 1e3),
                            "feeder_wait_p99_ms": float(np.percentile(feed[cls == c], 99) * 1e3),
                            "server_latency_p99_ms": float(np.percentile(srv_lat[cls == c], 99) * 1e3),
                            "service_p50_ms": float(np.percentile(svc[cls == c], 50) * 1e3),
                            "service_p99_ms": float(np.percentile(svc[cls == c], 99) * 1e3),
                            "build_p99_ms": float(np.percentile(ph_build[cls == c], 99) * 1e3),
                            "init_p99_ms": float(np.percentile(ph_init[cls == c], 99) * 1e3),
                            "iterate_download_p99_ms": float(np.percentile(ph_iter[cls == c], 99) * 1e3)})
    return {"jobs": n_jobs, "warmup_jobs": warm, "slots": slots, "short_slots": short_slots,
            "short_job_s": short_job_s,
            "failed": n_jobs - len(ok),
            "capacity_jobs_per_s": capacity, "lambda_jobs_per_s": lam,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "queue_wait_p50_ms": float(np.percentile(wait, 50) * 1e3),
            "queue_wait_p99_ms": float(np.percentile(wait, 99) * 1e3),
            "feeder_wait_p99_ms": float(np.percentile(feed, 99) * 1e3),
            "server_latency_p50_ms": float(np.percentile(srv_lat, 50) * 1e3),
            "server_latency_p99_ms": float(np.percentile(srv_lat, 99) * 1e3),
            "service_p50_ms": float(np.percentile(svc, 50) * 1e3),
            "service_p99_ms": float(np.percentile(svc, 99) * 1e3),
            "by_size": by_size,
            "p99_over_p50": float(np.percentile(lat, 99) / np.percentile(lat, 50)),
            "admission": "earliest virtual finish (arrival + estimated service) among jobs that fit the budget; "
                         "short jobs (estimated service <= short_job_s) also on short slots with their own "
                         "reserve, on high-priority streams",
            "p99_ms_largest_10pct": float(np.percentile(lat[big >= q], 99) * 1e3),
            "p99_ms_other_90pct": float(np.percentile(lat[big < q], 99) * 1e3),
            "jobs_per_s": (n_jobs - warm) / span, "nnz_d_iters_per_s": work / span,
            "pool_graphs": len(pool), "setup_s": gen_s, "output_arena_gb": arena_bytes / 2**30,
            "latency_def": "Poisson arrival time to FP32 result in (pinned) host memory",
            "job_mix": "n log-uniform [1e3, 5e6] (48-graph pool, nearest n), degree U[5, 40], "
                       "d in {64,128,256,1024}, I in {3,4,5}, FP32/BF16 50/50"}


def cpu_baseline_blocks(pkg, ctx, info, spec, target_entries=800_000_000, start_frac=1 / 3):
    """The FP64 oracle timed on host cores over a contiguous block of rows of the workload's
    own graph (rows are in ascending-id order, and ids are unrelated to degree, so a block is
    a random sample of rows), from its FP32 T_0: one step of `oracle.step_csr_rows`.  The
    rate (entries * d / time) is extrapolated to the whole graph."""
    import torch
    import oracle
    n, nnz, d = info["n"], info["nnz"], spec.d
    dev = torch.device("cuda", torch.cuda.current_device())
    rowptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    pkg.cleora_get_csr(ctx.handle, rowptr, col)
    ctx.init(d, 0, "f32")
    T0 = torch.empty((n, d), dtype=torch.float32, device=dev)
    pkg.cleora_get_embeddings(ctx.handle, T0, "f32")
    ctx.sync()
    r0 = int(n * start_frac)
    k0 = int(rowptr[r0])
    r1 = int(torch.searchsorted(rowptr, torch.tensor([k0 + min(target_entries, nnz - k0)], device=dev)))
    r1 = max(r0 + 1, min(r1, n))
    k1 = int(rowptr[r1])
    col_blk = col[k0:k1].cpu().numpy()
    del col
    # full-length rowptr whose rows outside the block are empty; block rows index col_blk
    rp = (rowptr - k0).clamp_(0, k1 - k0).cpu().numpy()
    del rowptr
    T_host = T0.cpu().numpy()
    del T0
    rows = np.arange(r0, r1, dtype=np.int64)
    t = time.perf_counter()
    oracle.step_csr_rows(rp, col_blk, None, T_host, rows)
    dt = time.perf_counter() - t
    del T_host, col_blk, rp
    cores = os.cpu_count() or 1
    rate = (k1 - k0) * d / dt
    return {"value": rate, "unit": "nnz*d/s", "cores": cores, "kind": "oracle",
            "sample": f"extrapolated: one FP64 oracle step (step_csr_rows) over rows [{r0}, {r1}) "
                      f"of the full graph ({r1 - r0} rows, {k1 - k0} of its {nnz} CSR entries, "
                      f"d = {d}, from the FP32 T_0), {dt:.1f} s on {cores} threads; the rate per "
                      f"entry is taken to hold for all entries",
            "seconds": dt, "entries": k1 - k0}


def config_leg(key, spec, device, steps, warmup, peak, peak_kind):
    """A smaller workload: GPU per-iteration time for FP32 and BF16 storage (build + init +
    I iterations per step, CUDA events on the context's stream) beside a full, timed FP64
    oracle run of all I iterations on the host cores (its graph build is not timed)."""
    import torch
    import oracle
    import paper_2102_02302_gb300 as pkg
    e = spec.generate()
    dev = torch.device("cuda", device)
    src = torch.from_numpy(e.src.view(np.int64)).to(dev)
    dst = torch.from_numpy(e.dst.view(np.int64)).to(dev)
    w = None if e.weights is None else torch.from_numpy(e.weights).to(dev)
    stream = torch.cuda.Stream(device)
    prev = torch.cuda.current_stream(device)
    torch.cuda.set_stream(stream)
    out = {"workload": spec.name, "d": spec.d, "iters": spec.iters}
    with pkg.Context(device, stream.cuda_stream) as ctx:
        ctx.graph_build(src, dst, w, spec.directed)
        info = ctx.info()
        n, nnz, hv = info["n"], info["nnz"], info["has_val"]
        out.update({"n": n, "nnz": nnz, "weighted": hv, "directed": spec.directed})
        for st in ("f32", "bf16"):
            r = time_dtype(pkg, ctx, (src, dst, w, None), spec, st, steps, warmup)
            it = float(np.median(r["iter_ms"])) * 1e-3
            es = 4 if st == "f32" else 2
            out[st] = {"value": nnz * spec.d / it, "unit": "nnz*d/s", "iter_ms": it * 1e3,
                       "step_ms": float(np.mean(r["step_ms"])),
                       "roofline": roofline_block(n, nnz, spec.d, es, hv, it,
                                                  measured_traffic(f"{key}/{st}"), peak,
                                                  peak_kind, prop_kernel_name(st, spec.d))}
    torch.cuda.set_stream(prev)
    del src, dst, w
    torch.cuda.empty_cache()
    g = oracle.build_from(e)
    T0 = oracle.init(g.ids, spec.d, 0)
    t = time.perf_counter()
    oracle.propagate(g, T0, spec.iters)
    dt = time.perf_counter() - t
    cores = os.cpu_count() or 1
    out["oracle"] = {"value": g.nnz * spec.d * spec.iters / dt, "unit": "nnz*d/s",
                     "run_s": dt, "cores": cores, "kind": "oracle",
                     "sample": f"full FP64 oracle run, all {spec.iters} iterations of the whole graph"}
    out["bf16_speedup_over_f32"] = out["f32"]["iter_ms"] / out["bf16"]["iter_ms"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS) + ["batch", "serve"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--storage", default="both", choices=["both", "bf16", "f32"])
    ap.add_argument("--hot-bytes", type=int, default=0,
                    help="L2 bytes kept for hot rows (0: library default, 1: off)")
    ap.add_argument("--staging", type=int, default=0, choices=sorted(STAGING_LABELS),
                    help="gathered rows reach the sums through 0: automatic, 1: registers, 2: the shared-memory ring (a bulk copy per row), 3: the ring (4-row tensor gathers)")
    ap.add_argument("--ring-stages", type=int, default=0, help="ring stages (0: library default)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 10k-node and 2M-node workloads (GPU and full oracle runs)")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-short-slots", type=int, default=2, help="serving slots for short jobs only")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-autotune", type=int, default=1, help="1: autotuned schedules, 0: defaults")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        import torch
        rank, local_rank, world = env_rank()
        torch.cuda.set_device(local_rank)
        r = serve_measure(local_rank, args.serve_jobs, short_slots=args.serve_short_slots)
        if rank == 0:
            print(json.dumps({"metric": "job p50/p99 latency", "value": r["p99_ms"], "unit": "ms",
                              "n_gpus": world, "steps": args.serve_jobs, "warmup": r["warmup_jobs"],
                              "ms_per_step": r["mean_ms"], "higher_is_better": False,
                              "scaling": "weak", "vs_baseline": None, "dtype": "mixed",
                              "data": "synthetic", "config": {"workload": "serving_poisson_80pct"},
                              "serving": r}), flush=True)
        return 0
    if args.workload == "batch":
        import torch
        rank, local_rank, world = env_rank()
        torch.cuda.set_device(local_rank)
        r = batch_measure(local_rank, args.steps, args.warmup, args.batch_count,
                          autotune=bool(args.batch_autotune))
        if rank == 0:
            print(json.dumps({"metric": "nnz*d/s per iteration", "value": r["value"],
                              "unit": "nnz*d/s", "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": r["run_ms"],
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                              "dtype": "bf16", "data": "synthetic",
                              "config": {"workload": f"batched_{args.batch_count}_chung_lu_graphs"},
                              "batched": r}), flush=True)
        return 0

    import torch
    import paper_2102_02302_gb300 as pkg

    rank, local_rank, world = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    device = local_rank
    spec = WORKLOADS[args.workload]

    t = time.perf_counter()
    edges = make_edges(spec, torch.device("cuda", device))
    gen_s = time.perf_counter() - t
    if not args.no_e2e and rank == 0:
        e2e_host, e2e_out = e2e_buffers(spec, edges)

    # A dedicated stream: the library and the CUDA events must share it (torch's default
    # stream has handle 0, which the C ABI reads as "create a private stream").
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    storages = ["bf16", "f32"] if args.storage == "both" else [args.storage]
    results = {}
    cpu = None
    with pkg.Context(device, stream.cuda_stream) as ctx:
        if args.hot_bytes:
            ctx.set_option("hot_bytes", args.hot_bytes)
        if args.staging:
            ctx.set_option("staging", args.staging)
        if args.ring_stages:
            ctx.set_option("ring_stages", args.ring_stages)
        ctx.graph_build(*edges[:3], spec.directed)
        info = ctx.info()
        for st in storages:
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            sampler = ClockSampler(device)
            sampler.start()
            r = time_dtype(pkg, ctx, edges, spec, st, args.steps, args.warmup)
            r["clocks"] = sampler.stop()
            r["max_step_ms"], r["max_iter_ms"] = max_over_ranks(
                [np.mean(r["step_ms"]), np.median(r["iter_ms"])], "cuda")
            results[st] = r
        if not args.no_cpu and rank == 0 and world == 1:
            if args.workload in ("large", "large_1_40"):
                cpu = cpu_baseline_blocks(pkg, ctx, info, spec)
            else:
                cpu = cpu_baseline(args.workload)

    n, nnz, d, hv = info["n"], info["nnz"], spec.d, info["has_val"]
    peak, peak_kind = measured_peaks()

    def summary(st):
        r = results[st]
        es = 2 if st == "bf16" else 4
        t_iter = r["max_iter_ms"] * 1e-3
        mb = model_bytes(n, nnz, d, es, hv)
        cb = compulsory_bytes(n, nnz, d, es, hv)
        return {
            "value": whole_job_rate(nnz * d, world, t_iter),
            "iter_ms_median": r["max_iter_ms"],
            "iter_ms_min": float(np.min(r["iter_ms"])),
            "step_ms": r["max_step_ms"],
            "build_ms": float(np.mean(r["build_ms"])),
            "init_ms": float(np.mean(r["init_ms"])),
            "model_bytes_per_iter": mb,
            "compulsory_bytes_per_iter": cb,
            "model_gbs": mb / t_iter / 1e9,
            "compulsory_gbs": cb / t_iter / 1e9,
            "launches": r["launches"],
            "clocks": r["clocks"],
            "wall_s": r["wall_s"],
            "roofline": roofline_block(n, nnz, d, es, hv, t_iter,
                                       measured_traffic(f"{args.workload}/{st}"), peak, peak_kind,
                                       prop_kernel_name(st, d)),
        }

    sums = {st: summary(st) for st in storages}
    head = "bf16" if "bf16" in sums else storages[0]
    hs = sums[head]

    e2e = None
    if not args.no_e2e and rank == 0:
        del edges
        torch.cuda.empty_cache()
        t_e2e, h2d, d2h, split = e2e_measure(pkg, spec, e2e_host, e2e_out, head, args.e2e_steps, device)
        del e2e_host, e2e_out  # 43 GB of pinned host memory, not needed by the later parts
        release_pinned_cache()
        e2e = {"value": world * nnz * d * spec.iters / t_e2e, "unit": "nnz*d/s",
               "s_per_step": t_e2e, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "phases": split,
               "value_def": f"nnz*d*I / end-to-end step time (I = {spec.iters})",
               "note": "public C ABI with pinned host buffers: edge upload, build, init, "
                       f"{spec.iters} iterations and FP32 result download per step"}

    batched = None
    if not args.no_batch:
        batched = batch_measure(device, args.steps, args.warmup, args.batch_count, peak, peak_kind,
                                autotune=bool(args.batch_autotune))
        batched["value"] *= world

    serving = None
    if not args.no_serve:
        serving = serve_measure(device, args.serve_jobs, short_slots=args.serve_short_slots)

    configs = None
    if not args.no_configs and rank == 0 and world == 1:
        configs = {k: config_leg(k, WORKLOADS[k], device, args.steps, args.warmup, peak, peak_kind)
                   for k in ("small", "mid")}

    line = {
        "metric": "nnz*d/s per iteration", "value": hs["value"], "unit": "nnz*d/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": hs["step_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": head, "data": "synthetic",
        "config": {"workload": spec.name, "n": n, "nnz": nnz, "edges": int(info["nnz"] // 2) if not spec.directed else None,
                   "d": d, "iters": spec.iters, "storage": head, "accumulate": "f32",
                   "max_row_len": info["max_row_len"], "weighted": hv,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (T and gathered rows >> 129 MB); no flush",
                   "step": "graph build + init + I iterations on device-resident edges",
                   "value_def": "nnz*d / median per-iteration time (CUDA events)",
                   "hot_bytes": args.hot_bytes or "default",
                   "staging": STAGING_LABELS[args.staging],
                   "ring_stages": args.ring_stages or "default",
                   "generator_s": gen_s},
        "roofline": hs["roofline"],
        "roofline_f32": sums["f32"]["roofline"] if "f32" in sums else None,
        "gpu_launches": hs["launches"],
        "clocks": hs["clocks"],
        "e2e": e2e,
        "cpu_baseline": cpu,
        "batched": batched,
        "serving": serving,
        "configs": configs,
        "breakdown": {st: {k: v for k, v in s.items() if k not in ("clocks", "roofline")}
                      for st, s in sums.items()},
    }
    if "bf16" in sums and "f32" in sums:
        line["bf16_speedup_over_f32"] = sums["f32"]["iter_ms_median"] / sums["bf16"]["iter_ms_median"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the CHERT hot path on the layered visco-TTI workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl chert|reference]

Workload: 2D layered viscoelastic TTI, 401 x 401 nodes at dx = 10 m, 8 flat
layers of seeded Thomsen parameters, tilts and Q (PCG64 seed 1002), wave
modes qP, qSV and qSH, 1 deg cache (M = 90 slowness angles per quadrant,
MEV kernel, homogeneity scan step 0.001 deg over [-30, 30] deg), radius-5
stencil (80 offsets), 64 surface sources.  One step runs the whole hot path:
cache build (8,640 entries), direction lookup, propagation and attenuation
relaxation of 192 (source, mode) fields with parents, and raypaths to 41
surface receivers per field.  The cache is built with a float scan and a
float-float (~48-bit) root polish (float storage); lookup and relaxation run
in float.  Before the timed steps the relaxation's launch shape is autotuned.

Further sections (added to the same JSON line): the plain-vs-surrogate
comparison on the per-cell 1701x351 model, the 201^3 3D model, and, on
request, the cache angular-step study and the CUDA-graph batch.

`value` is traveltime fields per second (a field = one (source, mode) pair
with both tau^R and tau^I and their parents); `e2e` is the same through the
host-buffer call (inputs copied from pinned memory, both fields copied back).
With torchrun, every rank runs the full workload on its own GPU (weak
scaling, no collective on the data path).  `--impl reference` times the FP64
CPU oracle on a bounded sample of the same workload.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_26108_b300 import inputs  # noqa: E402

METRIC = "cache entries/s; traveltime fields/s, plain vs surrogate at ≤1e-4 rel error"
MODES = ["qP", "qSV", "qSH"]
M_PER_QUADRANT = 90
SCAN_STEP = 0.001 * math.pi / 180
SCAN_HALF = 30000
RADIUS = 5
N_RECEIVERS = 41
E2E_PATH_CAP = 512          # nodes per returned raypath (longer ones come back with length 0)
SM_COUNT = 148
FP32_LANES_PER_SM = 128
# FP32 operations (adds, multiplies, 2 per fused multiply-add) of one
# energy-velocity evaluation of the cache build: the ncu count of FP32
# instructions of the all-float layered build divided by its counted
# evaluations (float); and of one float-float evaluation, from the same count
# for the MIXED build less its float evaluations (bench.py --cache-only;
# profiles/cache_build_kernel_layered_tti_401x401.md, part C).
F_EVAL_F32 = 368.4
F_EVAL_FF = 5945.0
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "relax_fast_kernel_layered_tti_401x401_64src.md")


def workload(n_sources=64):
    model = inputs.layered_tti(n_sources=n_sources)
    off = inputs.stencil_2d(RADIUS)
    rcv = np.round(np.linspace(0, model.nx - 1, N_RECEIVERS)).astype(np.int64)   # surface row
    return model, off, rcv


def measured_hbm_gbs():
    """HBM copy bandwidth of this machine's B300s (MEASURED_PEAKS.json at the
    repository root), else the fallback figure of one earlier measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "of fallback"


def measured_bf16_tflops():
    """Sustained dense BF16 rate of this machine's B300s (MEASURED_PEAKS.json),
    else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "of measured (sustained)"
    except (OSError, KeyError, ValueError):
        return 1400.0, "of fallback (sustained)"


# Instructions a warp issues per pull in the relaxation's inner loop, counted
# from its source: one 8-byte shared load of (tau, class), an index add, a
# shared load of the weight, an add and a min.
INSTR_PER_PULL = 5


def hbm_roofline(alg_bytes, dram_bytes, launch_s):
    """The relaxation against HBM: algorithmic bytes (class id read, tauR,
    tauI, parR, parI written) and, when captured, the DRAM bytes ncu counted,
    per launch time, over the measured copy bandwidth."""
    peak, src = measured_hbm_gbs()
    a = alg_bytes / launch_s / 1e9
    out = {"achieved_gbs": a, "peak_gbs": peak, "peak_source": src, "frac": a / peak}
    if dram_bytes:
        out["dram_gbs"] = dram_bytes / launch_s / 1e9
        out["dram_frac"] = out["dram_gbs"] / peak
    return out


def issue_rate_peak(sm_max_mhz):
    """Pulls per second if every scheduler issued one pull instruction per
    cycle: 148 SMs x 4 schedulers x clock x 32 lanes / instructions per pull."""
    return SM_COUNT * 4 * sm_max_mhz * 1e6 * 32 / INSTR_PER_PULL


def issue_roofline(alg_pulls, launch_s, sm_max_mhz):
    """The relaxation against the issue rate: algorithmic pulls (one per
    directed edge per field component) per second over the rate at which the
    schedulers could issue the pull loop."""
    peak = issue_rate_peak(sm_max_mhz)
    a = alg_pulls / launch_s
    return {"achieved_pulls_per_s": a, "peak_pulls_per_s": peak, "frac": a / peak,
            "instructions_per_pull": INSTR_PER_PULL,
            "peak_source": "derived: 148 SMs x 4 schedulers x max SM clock x 32 lanes / instructions per pull"}


def host_link(nbytes, reps=3):
    """Device-to-host copy rate of this machine's host link: one copy of nbytes
    from device memory into page-locked host memory, timed with CUDA events
    on its stream (median of reps), and the time the step's device-to-host
    bytes take at that rate: the floor of an end-to-end step whose copies
    overlap its kernels completely."""
    import torch
    n = max(int(nbytes), 1)
    src = torch.empty(n, dtype=torch.uint8, device="cuda")
    src.fill_(1)
    dst = torch.empty(n, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    ms = []
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            e0.record(s)
            dst.copy_(src, non_blocking=True)
            e1.record(s)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms[1:])
    return {"d2h_gbs": n / t / 1e6, "d2h_bytes": n, "d2h_ms_at_link_rate": t,
            "note": "one page-locked copy of the step's device-to-host bytes, CUDA events"}


def relax_sources_sha():
    """Digest of the 2D relaxation's sources, to tie a DRAM capture to the
    kernel version it measured."""
    import hashlib
    h = hashlib.sha256()
    for f in ("relax_fast.cuh", "relax.cu"):
        with open(os.path.join(ROOT, "paper_2609_26108_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic():
    """DRAM bytes per launch of the relaxation from the committed ncu summary,
    or None when that capture measured another version of the kernel."""
    try:
        with open(TRAFFIC_PROFILE) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_launch:"):
                    fields = dict(kv.split("=") for kv in line.split(":", 1)[1].split())
                    if fields.get("sources_sha256_16") == relax_sources_sha():
                        return float(fields["bytes"])
    except (OSError, ValueError):
        pass
    return None


def cache_roofline(build_once, entries, build_s, counter):
    """The cache build against the measured FP32 multiply-add rate: work =
    counted energy-velocity evaluations x FP32 operations per evaluation."""
    from paper_2609_26108_b300 import chert
    with counter() as ec:
        build_once()
    n_f32, n_ff, n_f64 = ec.counts
    flops = n_f32 * F_EVAL_F32 + n_ff * F_EVAL_FF
    peak32 = max(chert.fma_rate("fp32", 1 << 15) for _ in range(3))
    peak64 = max(chert.fma_rate("fp64", 1 << 10) for _ in range(2))
    achieved = flops / build_s
    return {"bound": "fp32", "achieved": achieved / 1e12, "peak": peak32 / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak32, "peak_source": "measured: chert_fma_rate (FP32 FMA chains, all SMs)",
            "fp64_fma_peak_tflops": peak64 / 1e12,
            "evaluations": {"float": n_f32, "float_float": n_ff, "double": n_f64},
            "evaluations_per_entry": (n_f32 + n_ff + n_f64) / entries,
            "flops_per_evaluation": {"float": F_EVAL_F32, "float_float": F_EVAL_FF},
            "flops_per_entry": flops / entries,
            "roofline_entries_per_s": peak32 / (flops / entries), "entries_per_s": entries / build_s}


def directed_edges(nx, nz, off):
    return int(sum((nx - abs(int(o[0]))) * (nz - abs(int(o[2]))) for o in off
                   if abs(int(o[0])) < nx and abs(int(o[2])) < nz))


def config_dict(model, extra=None):
    d = {"workload": "layered_visco_tti_2d_401x401_8layers_%dsrc_3modes_1deg_R5" % len(model.sources),
         "nx": model.nx, "nz": model.nz, "dx_m": model.dx, "n_layers": len(model.layers),
         "n_sources": len(model.sources), "modes": MODES, "cache_deg": 90.0 / M_PER_QUADRANT,
         "kernel": "MEV", "scan_step_deg": 0.001, "stencil_radius": RADIUS,
         "n_offsets": int(len(inputs.stencil_2d(RADIUS))), "fields_per_step": len(model.sources) * 3,
         "cache_entries_per_step": len(model.layers) * 3 * 4 * M_PER_QUADRANT,
         "l2": "outputs (494 MB of fields) exceed L2; L2 also flushed (256 MB write) before each step"}
    if extra:
        d.update(extra)
    return d


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


# --------------------------------------------------------------- CPU oracle
def cpu_info():
    """CPU model and the cores this process may use."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return model, cores


def _oracle_task(task):
    """One unit of oracle work on one core: ("solve", seed) times one cache
    solve at the full scan grid, ("field", seed) one source's tauR and tauI by
    Dijkstra; returns its wall time."""
    kind, seed = task
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:                    # the oracle's numpy calls are small; one thread is what it gets
        import contextlib
        threadpool_limits = lambda n: contextlib.nullcontext()   # noqa: E731
    from oracle import cache_oracle as co
    from oracle import graph_oracle as go
    model, off, _ = workload()
    rng = np.random.default_rng(seed)
    with threadpool_limits(1):
        t0 = time.perf_counter()
        if kind == "solve":
            mi, k, j = rng.integers(0, 3), rng.integers(0, len(model.layers)), rng.integers(0, M_PER_QUADRANT + 1)
            L = model.layers[k]
            a = co.moduli_from_thomsen(L.vp0, L.vs0, L.eps, L.delta, L.gamma, L.qp, L.qs)
            co.solve_direction(co.stiffness_tensor(a), (math.pi / 2) * j / M_PER_QUADRANT, MODES[mi], "MEV",
                               SCAN_STEP, SCAN_HALF)
        else:
            Vsel = rng.uniform(1500, 4500, (len(model.layers), len(off)))
            Asel = rng.uniform(1e-6, 1e-4, (len(model.layers), len(off)))
            cls = model.class_of_node.astype(np.int32)
            s = int(model.sources[rng.integers(0, len(model.sources))])
            go.dijkstra((model.nx, 1, model.nz), model.dx, cls, off, Vsel, 0, s)
            go.dijkstra((model.nx, 1, model.nz), model.dx, cls, off, Asel, 1, s)
        return time.perf_counter() - t0


def oracle_sample(model, off, n_solves=3, n_fields=2, seed=0, parallel=True):
    """Time the FP64 oracle on a bounded sample of the workload.

    The cache part times distinct (mode, class, angle) solves at the full scan
    grid and scales to the 2,184 distinct solves of the 8,640-entry cache; the
    relaxation part times (source, mode) fields, each tau^R and tau^I by
    binary-heap Dijkstra with parents.  Single thread: n_solves solves and
    n_fields fields one after another.  Parallel (parallel=True): a process
    pool with one worker per core runs one solve and one field per worker at
    once, and the wall time of each batch gives the whole machine's rate.
    Returns a dict with fields/s and entries/s, single-thread and parallel."""
    from oracle import graph_oracle as go
    go.build()
    model_name, cores = cpu_info()
    rng = np.random.default_rng(seed)
    t_solve = sum(_oracle_task(("solve", int(rng.integers(1 << 30)))) for _ in range(n_solves)) / n_solves
    t_field = sum(_oracle_task(("field", int(rng.integers(1 << 30)))) for _ in range(n_fields)) / n_fields
    n_solves_total = len(model.layers) * 3 * (M_PER_QUADRANT + 1)
    n_fields_total = len(model.sources) * 3
    entries = len(model.layers) * 3 * 4 * M_PER_QUADRANT
    t_step = n_solves_total * t_solve + n_fields_total * t_field
    out = {"cpu_model": model_name, "nproc": cores,
           "single": {"fields_per_s": n_fields_total / t_step, "entries_per_s": entries / (n_solves_total * t_solve),
                      "s_per_solve": t_solve, "s_per_field": t_field, "cores": 1},
           "sample": "%d cache solves at the full 0.001 deg scan (scaled to %d solves) + %d fields of tauR+tauI "
                     "Dijkstra on 401x401 (scaled to %d fields)" % (n_solves, n_solves_total, n_fields,
                                                                    n_fields_total)}
    if parallel and cores > 1:
        import multiprocessing as mp
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"             # one thread per worker process
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_task, [("field", 0)] * cores)                 # start-up, imports
            t0 = time.perf_counter()
            pool.map(_oracle_task, [("solve", seed + 1 + i) for i in range(cores)], chunksize=1)
            t_solves = time.perf_counter() - t0
            t0 = time.perf_counter()
            pool.map(_oracle_task, [("field", seed + 1 + i) for i in range(cores)], chunksize=1)
            t_fields = time.perf_counter() - t0
        solve_rate = cores / t_solves                  # solves/s over the machine
        field_rate = cores / t_fields
        t_par = n_solves_total / solve_rate + n_fields_total / field_rate
        out["parallel"] = {"fields_per_s": n_fields_total / t_par,
                           "entries_per_s": entries * solve_rate / n_solves_total, "cores": cores,
                           "sample": "%d solves and %d fields at once, one per worker process" % (cores, cores)}
    best = out.get("parallel", out["single"])
    out["fields_per_s"], out["entries_per_s"], out["cores"] = best["fields_per_s"], best["entries_per_s"], best["cores"]
    out["t_step_s"] = n_fields_total / out["fields_per_s"]
    return out


def run_reference(args):
    """The oracle on the host's cores: per step, one cache solve and one field
    per core at once (a spawn process pool, one worker per core), scaled to
    the workload's 2,184 solves and 192 fields."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import multiprocessing as mp
    from oracle import graph_oracle as go
    go.build()
    model, off, _ = workload()
    model_name, cores = cpu_info()
    n_solves_total = len(model.layers) * 3 * (M_PER_QUADRANT + 1)
    n_fields_total = len(model.sources) * 3
    vals, times = [], []
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"                 # one thread per worker process
    with mp.get_context("spawn").Pool(cores) as pool:
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_task, [("solve", 1000 * step + i) for i in range(cores)], chunksize=1)
            t_solves = time.perf_counter() - t0
            t0 = time.perf_counter()
            pool.map(_oracle_task, [("field", 1000 * step + i) for i in range(cores)], chunksize=1)
            t_fields = time.perf_counter() - t0
            if step < args.warmup:
                continue
            t_step = n_solves_total * t_solves / cores + n_fields_total * t_fields / cores
            vals.append(n_fields_total / t_step)
            times.append(t_step)
    value = statistics.median(vals)
    sample = ("per step: %d cache solves at the full 0.001 deg scan and %d fields of tauR+tauI Dijkstra on "
              "401x401, one of each per worker process at once, scaled to %d solves and %d fields"
              % (cores, cores, n_solves_total, n_fields_total))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "fields/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_dict(model),
           "cpu_baseline": {"value": value, "unit": "fields/s", "cores": cores, "kind": "oracle",
                            "cpu_model": model_name, "nproc": cores, "sample": sample},
           "e2e": {"value": value, "unit": "fields/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "note": "each step times a bounded sample of the oracle and scales it to the whole workload; "
                   "ms_per_step is that scaled time, not the step's wall time"}
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------- surrogate
SURR_TRAIN_CLASSES = 110_000       # x 31 angles x 3 modes = 10.2M exact training entries
SURR_TRAIN_M = 30
SURR_TRAIN_STEPS = 3000
SURR_BATCH = 4096
SURR_MAX_CYCLES = 512              # attenuation paths through the folds turn often


def surrogate_section(n_sources, flush, log=None, qsv_angles_deg=(1.0,)):
    """Plain vs surrogate form on the per-cell folded and faulted model.

    1701 x 351 nodes (597,051 cells, each its own medium), 10 folded layers and
    a normal fault (PCG64 seed 1003), modes qP/qSV/qSH, 1 deg cache, radius-5
    stencil, `n_sources` surface sources.  Plain: the exact solver for every
    (cell, mode, angle) solve.  Surrogate: the networks for every solve, the
    exact solver for those they hand back (flag 2).  The networks are trained
    once beforehand (reported, not part of the timed step) on exact entries of
    independently seeded media.  Each form is timed once (cache build, then
    the relaxation of all fields with parents), with L2 flushed before each
    part; the error is the surrogate form's traveltime against the plain
    form's, over all nodes with tau > 0."""
    import torch
    from paper_2609_26108_b300 import chert, surrogate

    model = inputs.folded_faulted(n_sources=n_sources)
    n = model.nx * model.nz
    p = model.params
    keys = ["vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt"]
    d_cells = chert.classes_to_device(chert.classes_from_arrays(**{k: p[k] for k in keys}))
    d_cls = torch.arange(n, dtype=torch.int32, device="cuda")
    off = inputs.stencil_2d(RADIUS)
    src = [int(v) for v in model.sources]
    M = M_PER_QUADRANT

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    train = surrogate.exact_training_set(inputs.random_tti_classes(SURR_TRAIN_CLASSES, seed=2003), MODES,
                                         SURR_TRAIN_M)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    params = [surrogate.train(*train[m], steps=SURR_TRAIN_STEPS, batch=SURR_BATCH, lr=2e-3, seed=1)[0]
              for m in MODES]
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del train
    if log:
        log("training set %.1f s, training %.1f s" % (t_data, t_train))
    # BF16 roofline of inference: 2 flops per parameter per row
    rows = 1 << 22
    xin = torch.rand((rows, 8), device="cuda") * 2 - 1
    ws_f = torch.empty(int(chert.lib().chert_mlp_workspace_bytes(rows, 0)), dtype=torch.uint8, device="cuda")
    chert.mlp_forward(params[0], xin, workspace=ws_f)
    t_inf = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        chert.mlp_forward(params[0], xin, workspace=ws_f)
        b.record()
        torch.cuda.synchronize()
        t_inf.append(a.elapsed_time(b) / 1e3)
    inf_s = statistics.median(t_inf)
    n_par = chert.mlp_param_count() - 10                     # weights and biases (out_mean/out_std excluded)
    bf16_peak = measured_bf16_tflops()
    inf_tflops = 2.0 * n_par * rows / inf_s / 1e12
    del xin, ws_f

    shape = (len(MODES), n, 4 * M)
    bufs = []
    for _ in range(2):
        b = {k: torch.empty(shape, dtype=torch.float32, device="cuda")
             for k in ("V", "A", "Q", "rx", "rz", "theta", "vartheta")}
        b["flag"] = torch.empty(shape, dtype=torch.uint8, device="cuda")
        bufs.append(b)
    fshape = (len(src), len(MODES), n)
    taus = [tuple(torch.empty(fshape, dtype=dt, device="cuda")
                  for dt in (torch.float32, torch.float32, torch.int32, torch.int32)) for _ in range(2)]
    ws = torch.empty(chert.workspace_bytes(len(MODES), n, len(off), chert.FP32, len(src), model.nx, model.nz),
                     dtype=torch.uint8,
                     device="cuda")
    # load every kernel once on a small slice before timing
    small = surrogate.per_cell_cache(d_cells[: 104 * 64], 64, MODES, M)
    surrogate.per_cell_cache(d_cells[: 104 * 64], 64, MODES, M, params)
    chert.traveltime(small, 8, 8, model.dx, d_cls[:64], off, [0], workspace=ws)

    def timed(fn):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return r, a.elapsed_time(b) / 1e3

    def run_form(prm, buf, tau):
        cache, t_cache = timed(lambda: surrogate.per_cell_cache(d_cells, n, MODES, M, prm, out=buf))
        _, t_relax = timed(lambda: chert.traveltime(cache, model.nx, model.nz, model.dx, d_cls, off, src,
                                                    max_cycles=SURR_MAX_CYCLES, out=tau, workspace=ws))
        nf = len(src) * len(MODES)
        r = {"cache_s": t_cache, "relax_s": t_relax, "cache_entries_per_s": n * len(MODES) * 4 * M / t_cache,
             "fields_per_s": nf / (t_cache + t_relax)}
        if prm is not None:
            r["solves_recomputed_exactly"] = int(cache.n_fallback)
            r["solves_total"] = n * len(MODES) * (M + 1)
            # nodewise angular coverage; missing angles against the exact (plain) cache
            r["coverage"] = coverage_summary(cache, off, None, bufs[0]["flag"])
        else:
            r["coverage"] = coverage_summary(cache, off)
        return r

    def errors():
        errs = {}
        for comp, name in ((0, "tauR"), (1, "tauI")):
            for mi, m in enumerate(MODES):
                r = taus[0][comp][:, mi].double()
                g = taus[1][comp][:, mi].double()
                ok = torch.isfinite(r) & (r > 0)
                rel = ((g - r).abs() / r)[ok]
                q = torch.quantile(rel[torch.randperm(rel.numel(), device="cuda")[:1 << 24]],
                                   torch.tensor([0.5, 0.99], dtype=torch.float64, device="cuda"))
                errs["%s_%s" % (name, m)] = {"median": float(q[0]), "p99": float(q[1]), "max": float(rel.max()),
                                             "frac_le_1e-4": float((rel <= 1e-4).double().mean())}
        return errs

    res = {"plain": run_form(None, bufs[0], taus[0])}
    if log:
        log("plain %s" % res["plain"])
    points = []
    prev_angle = chert.set_surrogate_qsv_angle(math.radians(qsv_angles_deg[0]))
    try:
        for deg in qsv_angles_deg:
            chert.set_surrogate_qsv_angle(math.radians(deg))
            r = run_form(params, bufs[1], taus[1])
            r["qsv_fallback_angle_deg"] = deg
            r["traveltime_rel_error_vs_plain"] = errors()
            r["p99_worst"] = max(v["p99"] for v in r["traveltime_rel_error_vs_plain"].values())
            r["speedup_fields_per_s"] = r["fields_per_s"] / res["plain"]["fields_per_s"]
            points.append(r)
            if log:
                log("surrogate at %.2f deg: %s" % (deg, r))
    finally:
        chert.set_surrogate_qsv_angle(prev_angle)
    # the form reported: the first angle (in the order given) whose worst p99
    # error over modes and components is within 1e-4, else the last one
    meet = [p for p in points if p["p99_worst"] <= 1e-4]
    res["surrogate"] = meet[0] if meet else points[-1]
    errs = res["surrogate"]["traveltime_rel_error_vs_plain"]
    worst = max(v["median"] for k, v in errs.items() if k.startswith("tauR"))
    return {"workload": "folded_faulted_visco_tti_2d_1701x351_per_cell_%dsrc_3modes_1deg_R5" % len(src),
            "cells": n, "fields": len(src) * len(MODES),
            "training": {"exact_entries": SURR_TRAIN_CLASSES * (SURR_TRAIN_M + 1) * len(MODES),
                         "steps_per_mode": SURR_TRAIN_STEPS, "batch": SURR_BATCH,
                         "dataset_s": t_data, "train_s": t_train, "one_off": True},
            "plain": res["plain"], "surrogate": res["surrogate"],
            "roofline_inference": {"bound": "tensor", "achieved": inf_tflops, "peak": bf16_peak[0],
                                   "unit": "TFLOP/s", "frac": inf_tflops / bf16_peak[0], "peak_source": bf16_peak[1],
                                   "rows": rows, "rows_per_s": rows / inf_s, "flops_per_row": 2 * n_par},
            "speedup_fields_per_s": res["surrogate"]["fields_per_s"] / res["plain"]["fields_per_s"],
            "speedup_cache": res["plain"]["cache_s"] / res["surrogate"]["cache_s"],
            "traveltime_rel_error_vs_plain": errs,
            "meets_1e-4_at_p99": res["surrogate"]["p99_worst"] <= 1e-4,
            "operating_points": [{k: p[k] for k in ("qsv_fallback_angle_deg", "fields_per_s", "speedup_fields_per_s",
                                                    "p99_worst", "solves_recomputed_exactly", "cache_s")}
                                 for p in points],
            "tauR_median_rel_error_worst_mode": worst}


# --------------------------------------------------------------- no-cache ablation
def section_no_cache(tracer, model, off, classes, value, source_index=31):
    """The no-cache (MSPM-style) form of the paper's Algorithm 1 on the main
    workload: for each field of one source (3 modes), every node's own
    directional table is solved afresh from its medium (160,801 tables of 91
    solves; nothing shared between nodes or fields), then looked up and
    relaxed.  Timed with events around the whole per-field work; its fields
    and parents must equal the cached path's bit for bit."""
    import torch
    from paper_2609_26108_b300 import chert
    from paper_2609_26108_b300.pipeline import no_cache_traveltime, per_node_classes
    d_nodes = chert.classes_to_device(per_node_classes(classes, model.class_of_node.astype(np.int32)))
    s = int(model.sources[source_index])
    no_cache_traveltime(d_nodes, 41, 1, model.dx, off, [0], ["qP"], M_PER_QUADRANT, SCAN_STEP, SCAN_HALF)   # load
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    got = no_cache_traveltime(d_nodes, model.nx, model.nz, model.dx, off, [s], MODES, M_PER_QUADRANT, SCAN_STEP,
                              SCAN_HALF)
    b.record()
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3
    tracer.set_inputs(tracer.d_classes, tracer.d_cls, [s] * tracer.n_sources)
    ref = tracer.run()
    torch.cuda.synchronize()
    same = all(bool(torch.equal(g[0], r[0])) for g, r in zip(got, ref))
    tracer.set_inputs(tracer.d_classes, tracer.d_cls, model.sources)
    nf = len(MODES)
    return {"workload": "layered_visco_tti_2d_401x401, source %d, 3 modes, per-field tables of all %d nodes"
                        % (source_index, model.nx * model.nz),
            "fields": nf, "s": t, "s_per_field": t / nf, "fields_per_s": nf / t,
            "table_solves_per_field": model.nx * model.nz * (M_PER_QUADRANT + 1),
            "cached_fields_per_s": value, "cache_speedup": value / (nf / t),
            "identical_to_cached_path": same,
            "note": "the paper's CPU comparison of the two methods (its MSPM against its CHERT on its layered model, "
                    "hardware not stated): 329 s against about 5 s"}


# --------------------------------------------------------------- 3D
def section_3d(flush, n_sources=16):
    """3D layered visco-TTI, 201^3 nodes at dx = 10 m, 12 layers (PCG64 seed
    1004, symmetry-axis azimuth ~ U(0, 360 deg)), qP and qSV, 1 deg x 1 deg
    cache of global directions (360 azimuths x 180 polar angles = 64,800 per
    class and mode), radius-2 3D stencil (98 offsets), 16 sources on a 4 x 4
    surface grid; MIXED cache, FP32 edge weights with traveltimes accumulated
    in float-float (~48-bit) and returned as double.  One run of cache build +
    relaxation with parents, L2 flushed before each part."""
    import torch
    from paper_2609_26108_b300 import chert

    m = inputs.layered_tti_3d(n_sources=n_sources)
    modes = ["qP", "qSV"]
    nk = len(m.layers)
    d_classes = chert.classes_to_device(chert.classes_from_layers(m.layers))
    d_cls = torch.as_tensor(m.class_of_node, device="cuda")
    off = inputs.stencil_3d(2)
    src = [int(v) for v in m.sources]
    n = m.nx * m.ny * m.nz
    shape = (len(src), len(modes), n)
    tau = tuple(torch.empty(shape, dtype=dt, device="cuda")
                for dt in (torch.float64, torch.float64, torch.int32, torch.int32))
    ws = torch.empty(chert.workspace_bytes(len(modes), nk, len(off), chert.FP32_ACC64, len(src)),
                     dtype=torch.uint8, device="cuda")
    small = chert.build_cache_3d(d_classes, nk, modes, 36, 18, precision="mixed")       # load the kernels
    chert.traveltime(small, 9, 9, m.dx, d_cls[:729], off, [0], ny=9, workspace=ws, precision="fp32_acc64")

    def timed(fn):
        flush.fill_(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return r, a.elapsed_time(b) / 1e3

    cache, t_cache = timed(lambda: chert.build_cache_3d(d_classes, nk, modes, 360, 180, precision="mixed"))
    _, t_relax = timed(lambda: chert.traveltime(cache, m.nx, m.nz, m.dx, d_cls, off, src, max_cycles=64,
                                                out=tau, workspace=ws, ny=m.ny, precision="fp32_acc64"))
    nf = len(src) * len(modes)
    # receiver gathers: a 21 x 21 surface grid per field, both components
    g = np.round(np.linspace(0, m.nx - 1, 21)).astype(np.int64)
    rcv = torch.as_tensor(np.array([x + m.nx * y for y in g for x in g], dtype=np.int64), device="cuda")
    fsrc = torch.as_tensor(np.repeat(np.asarray(src, np.int64), len(modes)), device="cuda")
    cap = 3 * m.nx

    def gathers():
        return [chert.raypath(tau[2 + c].reshape(nf, -1), fsrc, rcv, cap) for c in (0, 1)]

    paths, t_paths = timed(gathers)
    n_ok = int(sum(int((p[1] > 0).sum()) for p in paths))
    edges = int(sum((m.nx - abs(int(o[0]))) * (m.ny - abs(int(o[1]))) * (m.nz - abs(int(o[2]))) for o in off))
    return {"workload": "layered_visco_tti_3d_201^3_12layers_%dsrc_qP_qSV_1x1deg_R2" % len(src),
            "nodes": n, "fields": nf,
            "precision": "mixed cache (float storage), fp32 weights, float-float traveltime accumulation",
            "cache_entries": nk * len(modes) * 64800, "cache_s": t_cache,
            "cache_entries_per_s": nk * len(modes) * 64800 / t_cache,
            "relax_s": t_relax, "fields_per_s": nf / (t_cache + t_relax),
            "raypaths": {"receivers_per_field": int(rcv.numel()), "paths": 2 * nf * int(rcv.numel()),
                         "traced": n_ok, "s": t_paths},
            "edge_relaxations_per_s": edges * nf * 2 / t_relax, "directed_edges_per_field": edges}


# --------------------------------------------------------------- angular coverage
def coverage_summary(cache, off, class_of_node=None, truth_flag=None):
    """Per-node angular coverage of a 2D cache (chert_angular_coverage), per
    mode: over the model's nodes (each node takes its class's counts;
    class_of_node None: one class per node), the mean and minimum coverage
    ratio (covered stencil directions / stencil directions), the fraction of
    nodes with full coverage, the mean branch-mismatch ratio (mismatched /
    covered directions) and the fraction of nodes with any mismatch, and --
    with a reference cache's flags -- the mean and maximum missing-angle ratio
    (entries valid in the reference but flagged here / entries)."""
    import torch
    from paper_2609_26108_b300 import chert

    covd, mis, miss = chert.angular_coverage(cache, off, truth_flag=truth_flag)
    n_off = len(off)
    out = {}
    for mi, m in enumerate(MODES[:len(cache.modes)]):
        c, x, g = covd[mi].double(), mis[mi].double(), miss[mi].double()
        if class_of_node is not None:
            idx = class_of_node.long()
            c, x, g = c[idx], x[idx], g[idx]
        cr = c / n_off
        mr = torch.where(c > 0, x / c.clamp_min(1), torch.zeros_like(x))
        r = {"coverage_ratio_mean": float(cr.mean()), "coverage_ratio_min": float(cr.min()),
             "nodes_full_coverage": float((c == n_off).double().mean()),
             "branch_mismatch_ratio_mean": float(mr.mean()), "nodes_with_mismatch": float((x > 0).double().mean())}
        if truth_flag is not None:
            gr = g / cache.n_dir
            r["missing_angle_ratio_mean"] = float(gr.mean())
            r["missing_angle_ratio_max"] = float(gr.max())
        out[m] = r
    return out


# --------------------------------------------------------------- angular step
def section_angular(n_sources=8, steps_deg=(0.5, 1.0, 2.0, 5.0, 10.0)):
    """Cache angular-step study on the layered 401x401 model: caches of
    0.5 to 10 deg (MIXED), n_sources surface sources x 3 modes, FP32
    relaxation.  Per step and mode: RMS of the relative tauR and tauI misfit
    against the 0.5 deg fields (nodes with tau > 0), and the angle between
    each stencil offset and the ray of the entry the lookup selects
    (mean / max over classes and offsets; the lookup's directional error)."""
    import torch
    from paper_2609_26108_b300 import chert

    model = inputs.layered_tti(n_sources=n_sources)
    off = inputs.stencil_2d(RADIUS)
    d_classes = chert.classes_to_device(chert.classes_from_layers(model.layers))
    d_cls = torch.as_tensor(model.class_of_node.astype(np.int32), device="cuda")
    nk = len(model.layers)
    dirs = torch.as_tensor(off[:, [0, 2]] / np.linalg.norm(off, axis=1)[:, None], device="cuda")

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    rows, ref = [], None
    for deg in steps_deg:
        M = int(round(90.0 / deg))
        cache, t_c = timed(lambda: chert.build_cache(d_classes, nk, MODES, M, SCAN_STEP, SCAN_HALF, "MEV", "mixed"))
        fields, t_r = timed(lambda: chert.traveltime(cache, model.nx, model.nz, model.dx, d_cls, off,
                                                     model.sources, max_cycles=128))
        idx, _, _ = chert.edge_table(cache, off)
        ix = idx.long().clamp_min(0)
        rx = torch.gather(cache["rx"].double(), 2, ix)
        rz = torch.gather(cache["rz"].double(), 2, ix)
        dot = (rx * dirs[None, None, :, 0] + rz * dirs[None, None, :, 1]).clamp(-1, 1)
        ang = torch.rad2deg(torch.acos(dot))
        row = {"step_deg": deg, "cache_ms": t_c, "relax_ms": t_r}
        for mi, m in enumerate(MODES):
            a = ang[mi][idx[mi] >= 0]
            row["lookup_angle_deg_%s" % m] = {"mean": float(a.mean()), "max": float(a.max())}
        # nodewise angular coverage; missing angles against the FP64 cache of the same step
        truth = chert.build_cache(d_classes, nk, MODES, M, SCAN_STEP, SCAN_HALF, "MEV", "fp64")
        row["coverage"] = coverage_summary(cache, off, d_cls, truth["flag"])
        del truth
        if ref is None:
            ref = [f.double().clone() for f in fields[:2]]
        else:
            for comp, name in ((0, "tauR"), (1, "tauI")):
                for mi, m in enumerate(MODES):
                    r = ref[comp][:, mi]
                    g = fields[comp][:, mi].double()
                    ok = torch.isfinite(r) & (r > 0) & torch.isfinite(g)
                    row["rms_rel_misfit_%s_%s" % (name, m)] = float((((g - r) / r)[ok] ** 2).mean().sqrt())
        rows.append(row)
    return {"workload": "layered_visco_tti_2d_401x401_8layers_%dsrc_3modes_R5, caches %s deg"
                        % (len(model.sources), list(steps_deg)), "reference": "0.5 deg fields", "rows": rows}


def section_angular_cells(n_sources=8, steps_deg=(0.5, 1.0, 2.0, 5.0, 10.0), n_truth=4096):
    """The angular-step study on the per-cell folded and faulted 1701x351
    model (597,051 cells, each its own medium): exact MIXED per-cell caches
    at 0.5 to 10 deg, n_sources surface sources x 3 modes, FP32 relaxation;
    per step the RMS relative tau misfit against the 0.5 deg fields and the
    nodewise angular coverage over all nodes.  Missing angles are counted on
    n_truth seeded cells against their FP64 caches of the same step."""
    import torch
    from paper_2609_26108_b300 import chert

    model = inputs.folded_faulted(n_sources=n_sources)
    n = model.nx * model.nz
    p = model.params
    keys = ["vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt"]
    d_cells = chert.classes_to_device(chert.classes_from_arrays(**{k: p[k] for k in keys}))
    d_cls = torch.arange(n, dtype=torch.int32, device="cuda")
    off = inputs.stencil_2d(RADIUS)
    src = [int(v) for v in model.sources]
    pick = np.sort(np.random.default_rng(1007).choice(n, n_truth, replace=False))
    sub = {k: p[k][pick] for k in keys}
    d_sub = chert.classes_to_device(chert.classes_from_arrays(**sub))

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return r, a.elapsed_time(b) / 1e3

    rows, ref = [], None
    for deg in steps_deg:
        M = int(round(90.0 / deg))
        cache, t_c = timed(lambda: chert.build_cache(d_cells, n, MODES, M, SCAN_STEP, SCAN_HALF, "MEV", "mixed"))
        fields, t_r = timed(lambda: chert.traveltime(cache, model.nx, model.nz, model.dx, d_cls, off, src,
                                                     max_cycles=SURR_MAX_CYCLES))
        row = {"step_deg": deg, "cache_s": t_c, "relax_s": t_r, "coverage": coverage_summary(cache, off)}
        del cache
        mixed = chert.build_cache(d_sub, n_truth, MODES, M, SCAN_STEP, SCAN_HALF, "MEV", "mixed")
        truth = chert.build_cache(d_sub, n_truth, MODES, M, SCAN_STEP, SCAN_HALF, "MEV", "fp64")
        sc = coverage_summary(mixed, off, None, truth["flag"])
        for m in sc:
            row["coverage"][m]["missing_angle_ratio_mean_sampled"] = sc[m]["missing_angle_ratio_mean"]
            row["coverage"][m]["missing_angle_ratio_max_sampled"] = sc[m]["missing_angle_ratio_max"]
        del mixed, truth
        if ref is None:
            ref = [f.double().clone() for f in fields[:2]]
        else:
            for comp, name in ((0, "tauR"), (1, "tauI")):
                for mi, m in enumerate(MODES):
                    r = ref[comp][:, mi]
                    g = fields[comp][:, mi].double()
                    ok = torch.isfinite(r) & (r > 0) & torch.isfinite(g)
                    rel = ((g - r) / r)[ok]
                    row["rms_rel_misfit_%s_%s" % (name, m)] = float((rel ** 2).mean().sqrt())
                    row["median_abs_rel_misfit_%s_%s" % (name, m)] = float(rel.abs().median())
        del fields
        rows.append(row)
    return {"workload": "folded_faulted_visco_tti_2d_1701x351_per_cell_%dsrc_3modes_R5, caches %s deg"
                        % (len(src), list(steps_deg)),
            "reference": "0.5 deg fields; missing angles on %d seeded cells against FP64" % n_truth, "rows": rows}


# --------------------------------------------------------------- scheduler study
def section_scheduler(n_sources=16, reps=3, percell_sources=2):
    """Block-heap marching (Eq. 32), the hybrid scheduler (at most 6
    sweep cycles, then block-heap marching from the source for unconverged
    fields) and frontier label correcting (atomicMin pushes; layered model
    only, its class-pair table must fit in shared memory) against the sweep
    scheduler.  Layered
    401x401 model: n_sources surface sources x 3 modes, MIXED cache, FP32
    relaxation with parents, per scheduler the best of `reps` timed
    relaxations (after one untimed).  Per-cell folded and faulted 1701x351
    model (exact per-cell FP32 cache): percell_sources sources x 3 modes, one
    timed relaxation per scheduler, per mode.  Each case also reports whether
    the two schedulers return the same fields and parents bit for bit."""
    import torch
    from paper_2609_26108_b300 import chert, surrogate

    model = inputs.layered_tti(n_sources=n_sources)
    off = inputs.stencil_2d(RADIUS)
    d_classes = chert.classes_to_device(chert.classes_from_layers(model.layers))
    d_cls = torch.as_tensor(model.class_of_node.astype(np.int32), device="cuda")
    cache = chert.build_cache(d_classes, len(model.layers), MODES, M_PER_QUADRANT, SCAN_STEP, SCAN_HALF,
                              "MEV", "mixed")
    res, outs = {}, {}
    try:
        for name in ("sweeps", "block_heap", "hybrid", "frontier"):
            chert.set_relax_scheduler(name)
            run = lambda: chert.traveltime(cache, model.nx, model.nz, model.dx, d_cls, off, model.sources,
                                           max_cycles=128)
            outs[name] = [t.clone() for t in run()]
            best = None
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record()
                run()
                b.record()
                torch.cuda.synchronize()
                best = a.elapsed_time(b) if best is None else min(best, a.elapsed_time(b))
            res[name + "_ms"] = best
    finally:
        chert.set_relax_scheduler("hybrid")
    res["identical"] = all(bool(torch.equal(x, y)) for o in ("block_heap", "hybrid", "frontier")
                           for x, y in zip(outs["sweeps"], outs[o]))
    res["block_heap_over_sweeps"] = res["block_heap_ms"] / res["sweeps_ms"]
    res["frontier_over_sweeps"] = res["frontier_ms"] / res["sweeps_ms"]
    res["workload"] = "layered_visco_tti_2d_401x401_8layers_%dsrc_3modes_1deg_R5, fp32 relaxation" % n_sources
    if percell_sources <= 0:
        return res
    del outs, cache
    pc = inputs.folded_faulted(n_sources=percell_sources)
    n = pc.nx * pc.nz
    keys = ["vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt"]
    d_cells = chert.classes_to_device(chert.classes_from_arrays(**{k: pc.params[k] for k in keys}))
    d_pcls = torch.arange(n, dtype=torch.int32, device="cuda")
    per = {"workload": "folded_faulted_visco_tti_2d_1701x351_per_cell_%dsrc_R5, fp32 relaxation, per mode"
                       % percell_sources}
    src = [int(v) for v in pc.sources]
    for mode in MODES:
        pcache = surrogate.per_cell_cache(d_cells, n, [mode], M_PER_QUADRANT)
        got = {}
        try:
            for name in ("sweeps", "block_heap", "hybrid"):
                chert.set_relax_scheduler(name)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record()
                got[name] = chert.traveltime(pcache, pc.nx, pc.nz, pc.dx, d_pcls, off, src,
                                             max_cycles=SURR_MAX_CYCLES)
                b.record()
                torch.cuda.synchronize()
                per["%s_%s_ms" % (mode, name)] = a.elapsed_time(b)
        finally:
            chert.set_relax_scheduler("hybrid")
        per["%s_identical" % mode] = all(bool(torch.equal(x, y)) for o in ("block_heap", "hybrid")
                                         for x, y in zip(got["sweeps"], got[o]))
        del pcache, got
    res["per_cell"] = per
    return res


# --------------------------------------------------------------- batch
def section_batch(n2d, n3d):
    """Several problems of uneven size in one CUDA graph (the batched form):
    the per-cell folded and faulted 1701x351 model (exact per-cell cache,
    n2d sources x 3 modes) and a 101^3 block of the 3D layered model cut at a
    seeded corner (1 deg x 1 deg FP64 cache, n3d sources x qP/qSV).  Each
    problem is captured on its own stream, so their kernels overlap.  Timed:
    one eager pass (problems one after another) against one graph replay,
    each from the caches' build to the raypaths."""
    import torch
    from paper_2609_26108_b300 import chert
    from paper_2609_26108_b300.pipeline import GraphBatch, Problem

    fm = inputs.folded_faulted(n_sources=n2d)
    n = fm.nx * fm.nz
    keys = ["vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt"]
    d_cells = chert.classes_to_device(chert.classes_from_arrays(**{k: fm.params[k] for k in keys}))
    m3 = inputs.subvolume_3d(inputs.layered_tti_3d(), 101, seed=1005, n_sources=n3d)
    d3 = chert.classes_to_device(chert.classes_from_layers(m3.layers))
    probs = [Problem(d_cells, n, MODES, fm.nx, fm.nz, fm.dx, torch.arange(n, dtype=torch.int32, device="cuda"),
                     inputs.stencil_2d(RADIUS), fm.sources, receivers=np.arange(0, fm.nx, 40), M=M_PER_QUADRANT,
                     max_cycles=512),
             Problem(d3, len(m3.layers), ["qP", "qSV"], m3.nx, m3.nz, m3.dx,
                     torch.as_tensor(m3.class_of_node, device="cuda"), inputs.stencil_3d(2), m3.sources,
                     receivers=np.arange(0, m3.nx * m3.ny, 997), n_az=360, n_pol=180, ny=m3.ny,
                     cache_precision="fp64")]
    batch = GraphBatch(probs)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    t_eager = timed(batch.run_eager)
    batch.check()
    batch.capture()
    t_graph = timed(batch.replay)
    batch.check()
    nf = batch.n_fields
    return {"workload": "batch: folded_faulted 1701x351 per-cell %dsrc x 3 modes + layered_tti_3d 101^3 block "
                        "%dsrc x 2 modes, one CUDA graph" % (len(fm.sources), len(m3.sources)),
            "fields": nf, "eager_s": t_eager, "graph_s": t_graph,
            "fields_per_s_eager": nf / t_eager, "fields_per_s_graph": nf / t_graph,
            "note": "each pass builds the caches (exact per-cell, 3D FP64) and relaxes every field with parents "
                    "and raypaths"}


def section_c5(n2d=512, n_blocks=8, n3d_per_block=16, block=101):
    """Many sources and modes of uneven grid size as one batched job: the
    per-cell folded and faulted 1701x351 model (597,051 cells) with n2d
    surface sources x 3 modes, and n_blocks blocks of block^3 nodes cut at
    seeded corners of the 201^3 layered 3D model with n3d_per_block sources
    x qP/qSV each.  One CUDA graph per form: the 2D per-cell cache (exact, or
    the surrogate with its exact fallback on the device), the 3D blocks' one
    shared MIXED cache (1 x 1 deg), the 2D relaxation with parents (hybrid
    scheduler: its per-cell qSV attenuation fields need block-heap marching),
    the 3D blocks' relaxations in ONE persistent launch (float weights,
    float-float accumulation), raypaths to receiver lines.  Launch shapes (3D tile, 2D
    points per thread) come from the batch's autotuner on the first eager
    pass.  Timed: one graph replay per form (the surrogate's training is
    one-off, before)."""
    import torch
    from paper_2609_26108_b300 import chert, surrogate
    from paper_2609_26108_b300.pipeline import GraphBatch, Problem

    fm = inputs.folded_faulted(n_sources=n2d)
    n = fm.nx * fm.nz
    keys = ["vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt"]
    d_cells = chert.classes_to_device(chert.classes_from_arrays(**{k: fm.params[k] for k in keys}))
    d_own = torch.arange(n, dtype=torch.int32, device="cuda")
    big = inputs.layered_tti_3d()
    d3 = chert.classes_to_device(chert.classes_from_layers(big.layers))
    blocks = [inputs.subvolume_3d(big, block, seed=1005 + b, n_sources=n3d_per_block) for b in range(n_blocks)]
    train = surrogate.exact_training_set(inputs.random_tti_classes(SURR_TRAIN_CLASSES, seed=2003), MODES,
                                         SURR_TRAIN_M)
    params = [surrogate.train(*train[m], steps=SURR_TRAIN_STEPS, batch=SURR_BATCH, lr=2e-3, seed=1)[0]
              for m in MODES]
    del train
    prev_angle = chert.set_surrogate_qsv_angle(0.0)      # the operating point within 1e-4 (qSV exact)
    out = {"workload": "c5: folded_faulted 1701x351 per-cell %dsrc x 3 modes + %d blocks %d^3 of layered_tti_3d "
                       "x %dsrc x qP/qSV, one CUDA graph, 3D relaxations in one persistent launch"
                       % (len(fm.sources), n_blocks, block, n3d_per_block),
           "fields_2d": len(fm.sources) * 3, "fields_3d": n_blocks * n3d_per_block * 2}
    try:
        for form, prm in (("exact", None), ("surrogate", params)):
            probs = [Problem(d_cells, n, MODES, fm.nx, fm.nz, fm.dx, d_own, inputs.stencil_2d(RADIUS), fm.sources,
                             receivers=np.arange(0, fm.nx, 40), M=M_PER_QUADRANT, max_cycles=SURR_MAX_CYCLES,
                             surrogate_params=prm, path_cap=2048)]
            for b in blocks:
                probs.append(Problem(d3, len(big.layers), ["qP", "qSV"], b.nx, b.nz, b.dx,
                                     torch.as_tensor(b.class_of_node, device="cuda"), inputs.stencil_3d(2),
                                     b.sources, receivers=np.arange(0, b.nx * b.ny, 997), n_az=360, n_pol=180,
                                     ny=b.ny, cache_precision="mixed", relax_precision="fp32_acc64"))
            batch = GraphBatch(probs, persistent_3d=True)
            t0 = time.perf_counter()
            batch.run_eager()
            torch.cuda.synchronize()
            t_eager = time.perf_counter() - t0
            batch.check()
            tuned = batch.autotune()
            batch.capture(warm=False)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            batch.replay()
            b.record()
            torch.cuda.synchronize()
            t_graph = a.elapsed_time(b) / 1e3
            batch.check()
            nf = batch.n_fields
            r = {"graph_s": t_graph, "fields_per_s": nf / t_graph, "first_eager_pass_s": t_eager,
                 "autotune_ms": tuned}
            if prm is not None:
                r["solves_recomputed_exactly"] = int(batch.state[0]["cache"].n_fallback)
                r["solves_total"] = n * 3 * (M_PER_QUADRANT + 1)
            out[form] = r
            del batch, probs
            torch.cuda.empty_cache()
    finally:
        chert.set_surrogate_qsv_angle(prev_angle)
    out["fields"] = out["fields_2d"] + out["fields_3d"]
    out["surrogate_speedup"] = out["surrogate"]["fields_per_s"] / out["exact"]["fields_per_s"]
    return out


# --------------------------------------------------------------- GPU arm
def run_chert(args):
    import torch
    import torch.distributed as dist
    from paper_2609_26108_b300 import build, chert, replicas
    from paper_2609_26108_b300.pipeline import Tracer

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    model, off, rcv = workload(args.sources)
    classes = chert.classes_from_layers(model.layers)
    d_classes = chert.classes_to_device(classes)
    d_cls = torch.as_tensor(model.class_of_node.astype(np.int32), device="cuda")
    tr = Tracer(len(classes), MODES, M_PER_QUADRANT, model.nx, model.nz, model.dx, off,
                len(model.sources), rcv, scan_step=SCAN_STEP, scan_half=SCAN_HALF)
    tr.set_inputs(d_classes, d_cls, model.sources)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    from paper_2609_26108_b300.pipeline import autotune_points_per_thread
    ppt, tune_ms = autotune_points_per_thread(tr)          # launch shape of the relaxation (untimed)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        tr.run()
    barrier()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            flush.fill_(k & 0xff)               # evict L2 between steps (not timed)
            e = ev[k]
            tr.run(events=e[:3])
            e[3].record()
        barrier()
    clocks = clk.summary()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    cache_ms = [e[0].elapsed_time(e[1]) for e in ev]
    relax_ms = [e[1].elapsed_time(e[2]) for e in ev]
    nf = len(model.sources) * len(MODES)
    entries = len(classes) * len(MODES) * 4 * M_PER_QUADRANT
    value, slowest_s = replicas.job_throughput(sum(step_ms) / 1e3, nf * args.steps, device="cuda")
    total_ms = 1e3 * slowest_s

    # end to end through one library call on host buffers (chert_trace_host):
    # page-locked classes, class map and sources in; both traveltime fields
    # and the raypaths of both components to every receiver out
    from paper_2609_26108_b300.pipeline import HostTracer
    h_classes = d_classes.cpu().pin_memory()
    h_cls = d_cls.cpu().pin_memory()
    h_src = torch.as_tensor(np.asarray(model.sources, np.int64)).pin_memory()
    ht = HostTracer(len(classes), MODES, M_PER_QUADRANT, model.nx, model.nz, model.dx, off, len(model.sources), rcv,
                    scan_step=SCAN_STEP, scan_half=SCAN_HALF, path_cap=E2E_PATH_CAP)
    ht.run(h_classes, h_cls, h_src)
    barrier()
    e2e_times = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ht.run(h_classes, h_cls, h_src)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value, _ = replicas.job_throughput(sum(e2e_times), nf * args.steps, device="cuda")
    e2e_h2d, e2e_d2h = ht.h2d_bytes(h_classes, h_cls, h_src), ht.d2h_bytes()
    del ht
    e2e_link = host_link(e2e_d2h)
    e2e_link["e2e_ms_per_step"] = 1e3 * sum(e2e_times) / args.steps
    e2e_link["device_ms_per_step"] = total_ms / args.steps

    # roofline of the dominant kernel (relaxation): algorithmic work = one
    # relaxation (add + min: 2 FP32 ops) per directed edge per field component
    relax_avg_s = statistics.mean(relax_ms) / 1e3
    edges = directed_edges(model.nx, model.nz, off)
    alg_ops = 2.0 * edges * nf * 2
    sm_max = clocks.get("sm_max_mhz") or 2032.0
    peak_tops = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    achieved = alg_ops / relax_avg_s / 1e12
    traffic = captured_traffic() if len(model.sources) == 64 else None
    roofline = {"bound": "alu", "kernel": "relax_fast_kernel<float,5,1,false>", "achieved": achieved,
                "peak": peak_tops, "unit": "TFLOP/s", "frac": achieved / peak_tops, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu)",
                "alg_bytes_per_launch": 20.0 * model.nx * model.nz * nf,   # class id 4 B + tauR, tauI, parR, parI 4 B each per node per field
                "peak_source": "derived: 148 SMs x 128 FP32 lanes x max SM clock (non-FMA op rate)",
                "alg_ops_per_launch": alg_ops, "directed_edges_per_field": edges,
                "launch_ms": 1e3 * relax_avg_s,
                "hbm": hbm_roofline(20.0 * model.nx * model.nz * nf, traffic, relax_avg_s),
                "issue": issue_roofline(edges * nf * 2, relax_avg_s, sm_max)}
    cache_avg_s = statistics.mean(cache_ms) / 1e3
    roof_cache = cache_roofline(
        lambda: chert.build_cache(tr.d_classes, len(classes), MODES, M_PER_QUADRANT, SCAN_STEP, SCAN_HALF, "MEV",
                                  "mixed", out=tr.cache_out),
        entries, cache_avg_s, chert.EvalCounter)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    out = {"metric": METRIC, "value": value, "unit": "fields/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": config_dict(model, {"cache_precision": "float scan, float-float polish, float storage",
                                         "relax_precision": "fp32", "parallelism": "replicas" if world > 1 else "single",
                                         "relax_points_per_thread": ppt,
                                         "autotune_relax_ms": {str(k): v for k, v in tune_ms.items()}}),
           "cache_entries_per_s": world * entries / cache_avg_s,
           "cache_build_ms": 1e3 * cache_avg_s, "relax_ms": 1e3 * relax_avg_s,
           "edge_relaxations_per_s": world * edges * nf * 2 / relax_avg_s,
           "roofline": roofline, "roofline_cache_build": roof_cache, "clocks": clocks,
           "e2e": {"value": e2e_value, "unit": "fields/s", "h2d_bytes_per_step": e2e_h2d,
                   "d2h_bytes_per_step": e2e_d2h, "call": "chert_trace_host (one C-ABI call on page-locked host "
                   "buffers: inputs in, cache, traveltimes with parents, raypaths, fields and raypaths out)",
                   "link": e2e_link},
           "gpu_launches": tr.launches_per_run * args.steps}
    if world == 1 and args.no_cache:
        out["no_cache_ablation"] = section_no_cache(tr, model, off, classes, value)
    if world == 1 and args.surrogate_sources > 0:
        out["surrogate"] = surrogate_section(args.surrogate_sources, flush,
                                             qsv_angles_deg=[float(v) for v in args.surrogate_qsv_angles.split(",")])
    if world == 1 and args.sources_3d > 0:
        out["lattice_3d"] = section_3d(flush, args.sources_3d)
    if world == 1 and args.angular_study:
        out["angular_study"] = section_angular()
    if world == 1 and args.angular_study_cells:
        out["angular_study_cells"] = section_angular_cells()
    if world == 1 and args.scheduler_study > 0:
        out["scheduler_study"] = section_scheduler(args.scheduler_study)
    if world == 1 and args.batch_sources > 0:
        out["batch"] = section_batch(args.batch_sources, args.batch_sources_3d)
    if world == 1 and args.c5:
        out["c5"] = section_c5()
    if world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(model, off)
        out["cpu_baseline"] = {"value": cb["fields_per_s"], "unit": "fields/s", "cores": cb["cores"],
                               "kind": "oracle", "cpu_model": cb["cpu_model"], "nproc": cb["nproc"],
                               "sample": cb["sample"], "cache_entries_per_s": cb["entries_per_s"],
                               "single_thread": cb["single"], "parallel": cb.get("parallel")}
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_cache_only(precision):
    """The layered workload's cache build alone, twice (the second with the
    evaluation counter), for profiling its kernels; prints the counts."""
    import torch
    from paper_2609_26108_b300 import build, chert
    build.build()
    model, _, _ = workload(1)
    d = chert.classes_to_device(chert.classes_from_layers(model.layers))
    chert.build_cache(d, len(model.layers), MODES, M_PER_QUADRANT, SCAN_STEP, SCAN_HALF, "MEV", precision)
    torch.cuda.synchronize()
    with chert.EvalCounter() as ec:
        chert.build_cache(d, len(model.layers), MODES, M_PER_QUADRANT, SCAN_STEP, SCAN_HALF, "MEV", precision)
    print(json.dumps({"cache_only": precision, "solves": len(model.layers) * 3 * (M_PER_QUADRANT + 1),
                      "evaluations_float_floatfloat_double": ec.counts}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chert", choices=["chert", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sources", type=int, default=64,
                    help="surface sources (64 = the benchmark workload; fewer only for profiling)")
    ap.add_argument("--angular-study", action="store_true",
                    help="add the cache angular-step study (0.5-10 deg) on the layered model")
    ap.add_argument("--c5", action="store_true",
                    help="add the batched job: 512 sources x 3 modes on the per-cell model + 8 x 101^3 3D blocks "
                         "x 16 sources x 2 modes, one CUDA graph per form (exact, surrogate)")
    ap.add_argument("--angular-study-cells", action="store_true",
                    help="add the cache angular-step study (0.5-10 deg) on the per-cell folded model")
    ap.add_argument("--batch-sources", type=int, default=0,
                    help="sources of the per-cell 2D problem in the CUDA-graph batch (0, the default: leave it "
                         "out; the measured batch is --batch-sources 64 --batch-sources-3d 16)")
    ap.add_argument("--batch-sources-3d", type=int, default=16,
                    help="sources of the 101^3 3D problem in the CUDA-graph batch")
    ap.add_argument("--sources-3d", type=int, default=16,
                    help="sources of the 201^3 3D section (0: leave it out)")
    ap.add_argument("--surrogate-sources", type=int, default=16,
                    help="sources of the per-cell plain-vs-surrogate comparison (0: leave it out)")
    ap.add_argument("--surrogate-qsv-angles", default="1.0,0",
                    help="qSV fallback angles (deg, comma-separated) of the surrogate form, tried in order; the "
                         "first whose worst p99 traveltime error is within 1e-4 is reported (else the last)")
    ap.add_argument("--scheduler-study", type=int, default=0,
                    help="sources of the block-heap vs sweep scheduler comparison on the layered model (0: leave it out)")
    ap.add_argument("--no-cache", type=int, default=1,
                    help="1 (default): add the no-cache (MSPM-style) ablation of one source x 3 modes; 0: leave it out")
    ap.add_argument("--cache-only", default=None, choices=["fp32", "mixed", "fp64"],
                    help="profiling aid: build the layered workload's cache twice in this precision and exit")
    args = ap.parse_args()
    if args.cache_only:
        return run_cache_only(args.cache_only)
    if args.impl == "reference":
        return run_reference(args)
    return run_chert(args)


if __name__ == "__main__":
    sys.exit(main())

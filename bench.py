#!/usr/bin/env python3
"""Throughput of one t-FDP iteration (arXiv 2303.03964) on one GB300.

A step is one full iteration of the hot path -- bin/sort, spread, grid interaction by
FFT, back-projection, attraction over the edge list, position update -- on a seeded
synthetic graph with its inputs resident in HBM. The default workload is the
1000 x 1000 lattice (1M nodes, 1,998,000 edges) with uniform initial positions,
ibFFT repulsion with k = 3 and a grid of at most 1023^2 nodes (FFT size 2048).

Prints one JSON line. Timing: W warm-up steps, then K steps each preceded by an L2
flush (a 256 MiB write) and timed with CUDA events on the library's stream; per-stage
CUDA events captured inside the iteration graph give the dominant kernel's live
duration for the roofline. `e2e` repeats the steps through the C ABI with host
buffers (positions in and out of pinned host memory every step, wall clock).

--impl reference times the FP64 CPU oracle on the same workload (the reference arm).
Multi-GPU (torchrun): every rank lays out its own copy of the graph (replicas; one
graph does not shard without a collective, which this path does not have).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-iterations/s at 1M nodes (mixed vs plain FP32, same force error); p50/p99 update"
UNIT = "node-iterations/s"
FLUSH_BYTES = 256 << 20

WORKLOADS = {
    "lattice_1m": {"desc": "1000x1000 lattice, n=1,000,000, m=1,998,000, U[-500,500]^2",
                   "rep": "fft", "k": 3, "grid_max": 1023, "total_iters": 300},
    # the paper's own grid rule on the same lattice: N_int = ceil(L) = 1000 boxes per axis,
    # G = 3000, P = 8192 (Sec. 3.4), instead of the 1023 cap of the main line
    "lattice_1m_paper_grid": {"desc": "1000x1000 lattice, n=1,000,000, m=1,998,000, U[-500,500]^2, "
                                      "grid up to 3071 (G=3000, P=8192)",
                              "rep": "fft", "k": 3, "grid_max": 3071, "total_iters": 300},
    "ba_2m": {"desc": "Barabasi-Albert n=2,000,000, m0=3, U[-707,707]^2",
              "rep": "fft", "k": 3, "grid_max": 1023, "total_iters": 300},
    "sbm_100k": {"desc": "SBM n=100,000, 20 blocks, mean degree 10, 90% intra, U[-50,50]^2",
                 "rep": "fft", "k": 3, "grid_max": 255, "total_iters": 500},
    "er_2000_exact": {"desc": "ER n=2000, m=8000, U[-50,50]^2, exact repulsion",
                      "rep": "exact", "k": 3, "grid_max": 255, "total_iters": 100},
    # the exact all-pairs kernel at a size that fills the GPU (its FMA roofline)
    "er_64k_exact": {"desc": "ER n=65,536, m=262,144, U[-128,128]^2, exact repulsion",
                     "rep": "exact", "k": 3, "grid_max": 255, "total_iters": 100},
}

# DRAM bytes of the dominant kernel from one ncu capture, per launch, keyed by
# (workload, stage); valid only while every source file the kernel is built from is
# unchanged (sha256 over STAGE_SOURCES). Captured with
#   ncu --set full --clock-control none -k regex:k_cols_r -s 2 -c 1 -o prof_k_cols_r
#       python bench.py --steps 2 --warmup 3 --no-cpu-baseline --no-batch --no-serving
#       --no-dynamic-k --no-quality --no-workloads --no-mixed
NCU_TRAFFIC = {
    ("lattice_1m", "cols"): {"bytes": 50455552 + 1001472, "sha": "8cd75292345cda4e"},
}

# Stages timed by the library that are ONE kernel on the critical path, and that kernel
# (P <= 4096 uses the register-resident FFT kernels). "sort" is four kernels (grid, bin,
# scan, scatter) and "attract" runs on a side stream under the FFT, so neither is a
# roofline candidate.
STAGE_KERNEL = {"spread": "k_spread", "rows_fwd": "k_rows_fwd_r", "cols": "k_cols_r",
                "rows_inv": "k_rows_inv_r", "gather_update": "k_gather_update",
                "exact": "k_exact", "edge_update": "k_edge_update"}

# the files a stage's kernel code is built from (the node kernels take NodeLaunch from
# launch.h by value; the FFT kernels take plain arguments, so launch.h is host-side there)
_NODE_SRC = ("node_kernels.cu", "node_dev.cuh", "common.cuh", "launch.h")
_FFT_SRC = ("fft_kernels.cu", "fft_stages.cuh", "fft_reg.cuh", "fft.cuh", "common.cuh")
STAGE_SOURCES = {"spread": _NODE_SRC, "gather_update": _NODE_SRC, "edge_update": _NODE_SRC,
                 "exact": _NODE_SRC, "rows_fwd": _FFT_SRC, "cols": _FFT_SRC, "rows_inv": _FFT_SRC}


def make_workload(name):
    from paper_2303_03964_gb300 import synth
    if name in ("lattice_1m", "lattice_1m_paper_grid"):
        e, xy = synth.lattice_1m()
    elif name == "ba_2m":
        e, xy = synth.ba_2m()
    elif name == "sbm_100k":
        e, xy = synth.sbm_100k()
    elif name == "er_2000_exact":
        e, xy = synth.er_2000()
    elif name == "er_64k_exact":
        rng = synth.rng_for(6)
        e = synth.erdos_renyi(65536, 4 * 65536, rng)
        xy = synth.uniform_positions(65536, 128.0, rng)
    else:
        raise KeyError(name)
    return e, xy


def stage_bytes(stage, n, m, G, P, nbox):
    """Algorithmic bytes of one launch of a stage: each input read once, each output
    written once (FP32 positions 8 B/node, int32 indices 4 B)."""
    NH = P // 2 + 1
    if stage == "sort":
        # bin: read xy, write (key, slot); scan: cnt -> off; scatter: read (key, slot),
        # xy and the old permutation, write sorted xy and the new permutation
        return 8 * n + 8 * n + 2 * 4 * nbox + (8 * n + 8 * n + 4 * n) + (8 * n + 4 * n)
    if stage == "spread":
        return 8 * n + 4 * nbox + 3 * 4 * G * G
    if stage == "rows_fwd":
        return 3 * 4 * G * G + 3 * 8 * G * NH
    if stage == "cols":
        return 3 * 8 * G * NH + 3 * 4 * P * NH + 3 * 8 * G * NH
    if stage == "rows_inv":
        return 3 * 8 * G * NH + 16 * G * G
    if stage == "gather_update":
        # sorted positions and permutation in, attraction in (from k_attract), the output
        # grid (A, O^x, O^y, 0) once; positions out in caller and in sorted order
        return 8 * n + 4 * n + 8 * n + 16 * G * G + 8 * n + 8 * n
    if stage == "attract":
        # positions, row pointers, column ids and the neighbour positions, attraction out
        return 8 * n + 4 * (n + 1) + 4 * 2 * m + 8 * 2 * m + 8 * n
    if stage == "edge_update":
        return 8 * n + 4 * (n + 1) + 4 * 2 * m + 8 * 2 * m + 8 * n
    return 0


def iteration_model_bytes(n, m, G, P):
    """Single-pass byte model of one FFT-path iteration: node bytes 28 n + 24 m (the
    spread reads the positions; gather, attraction and update read positions, row
    pointers, column ids and the neighbours' positions and write the positions) plus
    grid bytes 2 * 3 * 4 G^2 + 2 * 3 * P (P/2+1) * 8 + 3 * P (P/2+1) * 4 (each transform
    one read and one write, the three kernel spectra read once)."""
    NH = P // 2 + 1
    return 28 * n + 24 * m + 2 * 3 * 4 * G * G + 2 * 3 * P * NH * 8 + 3 * P * NH * 4


def iteration_roofline(n, m, G, P, ms_per_step, peak_gbs):
    """Whole-iteration rate against HBM under iteration_model_bytes (None without a grid)."""
    if not G or not P or ms_per_step <= 0:
        return None
    b = iteration_model_bytes(n, m, G, P)
    ach = b / (ms_per_step * 1e-3) / 1e9
    return {"bytes_per_iteration": b, "achieved": ach, "peak": peak_gbs, "unit": "GB/s",
            "frac": ach / peak_gbs,
            "model": "28 n + 24 m node bytes + 24 G^2 + 60 P (P/2+1) grid bytes per iteration"}


def source_sha(stage):
    srcs = STAGE_SOURCES.get(stage)
    if not srcs:
        return None
    h = hashlib.sha256()
    for src in srcs:
        with open(os.path.join(ROOT, "paper_2303_03964_gb300", "csrc", src), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks_raw():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    active = True  # nvidia-smi cannot be paused; it samples the whole measurement

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlSampler:
    """SM clock, its maximum and the clock-event (throttle) reasons, read through NVML
    every 2 ms in a background thread during the timed region (read-only queries)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        import ctypes
        self.ok = False
        self.samples = []
        self.stop_flag = False
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            done = False
            try:
                import torch
                uuid = str(torch.cuda.get_device_properties(cuda_index).uuid)
                for cand in ("GPU-" + uuid, uuid):
                    if lib.nvmlDeviceGetHandleByUUID(cand.encode(), ctypes.byref(h)) == 0:
                        done = True
                        break
            except Exception:
                pass
            if not done and lib.nvmlDeviceGetHandleByIndex_v2(cuda_index, ctypes.byref(h)) != 0:
                return
            self.lib, self.h, self.ct = lib, h, ctypes
            self.ok = True
        except OSError:
            pass

    active = False  # samples are kept only while a timed region runs

    def _read(self):
        ct = self.ct
        while not self.stop_flag:
            if not self.active:
                time.sleep(0.001)
                continue
            clk, mx, rs = ct.c_uint(0), ct.c_uint(0), ct.c_ulonglong(0)
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk)) == 0:
                self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ct.byref(mx))
                fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                    self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
                fn(self.h, ct.byref(rs))
                self.samples.append((clk.value, mx.value, rs.value))
            time.sleep(0.002)

    def start(self):
        if self.ok:
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()

    def stop(self):
        if not self.ok:
            return None
        self.stop_flag = True
        self.thread.join(timeout=2)
        if not self.samples:
            return None
        reasons = set()
        for _, _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(c for c, _, _ in self.samples),
                "sm_max_mhz": max(m for _, m, _ in self.samples), "reasons": sorted(reasons),
                "samples": len(self.samples), "source": "nvml every 2 ms inside the timed regions"}


def serving_measurement(jobs=200, rate=20.0, updates=5, init_iters=300, upd_iters=50,
                        budget_gb=48, max_active=24, chunk=10, sampler=None):
    """Poisson stream of layout jobs (n log-uniform in [10k, 1M], SBM / BA in turn): each
    job is laid out for init_iters iterations, then receives `updates` parameter changes
    (alpha, beta, gamma uniform in the paper's ranges with alpha (1 + beta) < 1), each
    followed by upd_iters warm-started iterations, submitted as soon as the previous
    request of the job completes. Latency = completion - submission of a request."""
    import numpy as np
    from paper_2303_03964_gb300 import synth, tfdp
    rng = synth.rng_for(5)
    specs = []
    t = 0.0
    for q in range(jobs):
        t += rng.exponential(1.0 / rate)
        n = int(np.exp(rng.uniform(np.log(10_000), np.log(1_000_000)))) // 10 * 10
        if q % 2 == 0:
            e, _ = synth.sbm(n, 10, 8.0, 0.9, rng)
        else:
            e = synth.barabasi_albert(n, 3, rng)
        xy = synth.uniform_positions(n, np.sqrt(n) / 2.0, rng)
        # grid cap from the expected layout side (unit density): P = 1024 .. 2048
        gmax = 3 * min(341, max(50, int(np.ceil(1.2 * np.sqrt(n)))))
        ups = []
        for _ in range(updates):
            while True:
                a, b = rng.uniform(0.01, 0.5), rng.uniform(8.0, 50.0)
                if a * (1 + b) < 1:
                    break
            ups.append((a, b, float(rng.uniform(2.0, 8.0))))
        specs.append((t, n, e, xy, gmax, ups))
    total_n = sum(sp[1] for sp in specs)
    srv = tfdp.Server(budget_gb << 30, max_active=max_active, chunk_iters=chunk)
    job_of, pending, lat_upd, lat_init = {}, {}, [], []
    n_of = {}
    t0 = time.perf_counter()
    if sampler is not None:
        sampler.active = True
    nxt, finished = 0, 0
    first_submit = None
    last_done = 0.0
    while finished < jobs:
        now = time.perf_counter() - t0
        while nxt < jobs and specs[nxt][0] <= now:
            _, n, e, xy, gmax, ups = specs[nxt]
            job, _ = srv.submit(n, e, xy, tfdp.params_default(grid_max=gmax, total_iters=init_iters), init_iters)
            job_of[job] = nxt
            pending[job] = list(ups)
            n_of[job] = n
            nxt += 1
        wait = 2 if nxt < jobs else 20
        for d in srv.poll(256, wait_ms=wait):
            job = d["job_id"]
            if first_submit is None or d["t_submit"] < first_submit:
                first_submit = d["t_submit"]
            last_done = max(last_done, d["t_done"])
            if d["status"] != 0:
                raise RuntimeError("request failed: %s" % d)
            (lat_init if d["kind"] == 0 else lat_upd).append(d["t_done"] - d["t_submit"])
            if pending[job]:
                a, b, g = pending[job].pop(0)
                gmax = specs[job_of[job]][4]
                srv.update(job, tfdp.params_default(alpha=a, beta=b, gamma=g, grid_max=gmax), upd_iters)
            else:
                srv.release(job)
                finished += 1
    if sampler is not None and isinstance(sampler, NvmlSampler):
        sampler.active = False
    st = srv.stats()
    srv.close()
    span = last_done - first_submit
    node_its = total_n * (init_iters + updates * upd_iters)

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(q * len(v)))]
    return {"workload": "%d jobs, Poisson %.0f/s, n log-uniform in [10k, 1M] (sum %d), SBM / BA m0=3 in turn; "
                        "%d-iteration layout then %d updates of %d warm-started iterations" % (
                            jobs, rate, total_n, init_iters, updates, upd_iters),
            "update_latency_s_p50": pct(lat_upd, 0.5), "update_latency_s_p99": pct(lat_upd, 0.99),
            "layout_latency_s_p50": pct(lat_init, 0.5), "layout_latency_s_p99": pct(lat_init, 0.99),
            "throughput": node_its / span, "unit": UNIT, "span_s": span, "requests": len(lat_upd) + len(lat_init),
            "peak_active_jobs": st["peak_active"], "budget_bytes": st["budget_bytes"], "max_active": max_active,
            "chunk_iters": chunk}


def stage_kernel(stage, P):
    """Kernel of a single-kernel stage (every FFT size runs the register-resident FFT
    kernels; P = 8192 keeps one channel in registers at a time)."""
    return STAGE_KERNEL[stage]


def stage_roofline(stage, ms, n, m, G, P, nbox, peak, peak_kind):
    """Roofline of one single-kernel stage from its in-graph time: algorithmic bytes
    (stage_bytes) against the HBM peak, or, for the exact kernel, about 11 FP32 flops per
    pair against the FP32 FMA peak (152 SMs x 128 lanes x 2 flops x 2.07 GHz)."""
    if stage == "exact":
        fma_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        ach = 11.0 * n * n / (ms * 1e-3) / 1e12
        return {"stage": stage, "kernel": STAGE_KERNEL[stage], "bound": "alu", "achieved": ach,
                "kernel_ms": ms, "peak": fma_peak, "unit": "TFLOP/s", "frac": ach / fma_peak, "traffic": None,
                "peak_kind": "derived: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2.07 GHz"}
    bytes_ = stage_bytes(stage, n, m, G, P, nbox)
    ach = bytes_ / (ms * 1e-3) / 1e9
    return {"stage": stage, "kernel": stage_kernel(stage, P), "bound": "hbm", "achieved": ach, "peak": peak,
            "unit": "GB/s", "frac": ach / peak, "traffic": None, "algorithmic_bytes": bytes_, "kernel_ms": ms,
            "peak_kind": peak_kind + " hbm_gbs (burst copy)"}


def workload_measurement(name, stream, flush, steps, warmup, cpu=True):
    """Another configuration's workload with the main line's timing (L2 flushed before
    each step, CUDA events around each step): device-resident rate, per-stage times and
    the roofline of its dominant single-kernel stage, the end-to-end rate through
    tfdp_run with pinned host buffers, and the FP64 oracle on the host cores."""
    import torch
    from paper_2303_03964_gb300 import tfdp
    spec = WORKLOADS[name]
    e, xy = make_workload(name)
    n, m = xy.shape[0], e.shape[0]
    rep_mode = tfdp.REP_EXACT if spec["rep"] == "exact" else tfdp.REP_FFT
    params = tfdp.params_default(rep_mode=rep_mode, k_interp=spec["k"], grid_max=spec["grid_max"],
                                 total_iters=spec["total_iters"])
    with tfdp.Graph(n, e, xy, params, stream=stream.cuda_stream) as g:
        def step():
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.iterate(1)
            e1.record(stream)
            stream.synchronize()
            return e0.elapsed_time(e1)
        for _ in range(warmup):
            step()
        ms = [step() for _ in range(steps)]
        st = g.stats()
        # stage breakdown (events on a side branch of the iteration), after the timed steps
        g.set_stage_timing(True)
        brk = []
        for _ in range(5):
            step()
            brk.append(g.stage_times())
        g.set_stage_timing(False)
        stages = {k: statistics.fmean(b[k] for b in brk[2:]) for k in brk[0]}
        # end to end: upload, one iteration, download per call (pinned host buffers)
        hin = torch.empty((n, 2), dtype=torch.float32, pin_memory=True)
        hout = torch.empty((n, 2), dtype=torch.float32, pin_memory=True)
        g.get_positions(hout.numpy())
        hin.copy_(hout)
        e2e = []
        for _ in range(steps):
            t0 = time.perf_counter()
            g.run(hin.numpy(), 1, hout.numpy())
            e2e.append(time.perf_counter() - t0)
            hin.copy_(hout)
    G, P = st["grid_G"], st["fft_P"]
    nbox = st["grid_n_int"] ** 2
    cand = {k: v for k, v in stages.items() if k in STAGE_KERNEL and v > 0}
    dom = max(cand, key=cand.get)
    peak, peak_kind = measured_peaks()
    step_ms = sum(ms) / len(ms)
    out = {"desc": spec["desc"], "rep": spec["rep"], "n": int(n), "m": int(m),
           "value": n * len(ms) / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": step_ms,
           "grid_G": G, "fft_P": P, "device_flags": st["device_flags"], "stages_ms": stages,
           "roofline": stage_roofline(dom, cand[dom], n, m, G, P, nbox, peak, peak_kind),
           "iteration_roofline": (iteration_roofline(n, m, G, P, step_ms, peak)
                                  if spec["rep"] == "fft" else None),
           "e2e": {"value": n * len(e2e) / sum(e2e), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                   "d2h_bytes_per_step": 8 * n}}
    if cpu:
        out["cpu_baseline"] = cpu_baseline(e, xy, spec, budget_s=6.0)
    return out


def exact_kernel_measurement(stream, flush, steps, warmup, name="er_64k_exact"):
    """The tiled exact all-pairs kernel (k_exact) at a size where it fills the GPU, against
    the FP32 FMA peak. About 11 FP32 flops per pair at gamma = 2 (two differences, 1 + d^2
    as two FMAs, r^2 and two FMA accumulations) plus one reciprocal on the quarter-rate
    MUFU unit (16 per SM and clock), which caps it at 16 pairs per SM and clock, i.e.
    11/16 of the all-FMA peak."""
    import torch
    from paper_2303_03964_gb300 import tfdp
    e, xy = make_workload(name)
    n = xy.shape[0]
    params = tfdp.params_default(rep_mode=tfdp.REP_EXACT, total_iters=WORKLOADS[name]["total_iters"])
    with tfdp.Graph(n, e, xy, params, stream=stream.cuda_stream) as g:
        g.set_stage_timing_mask(["exact"])
        times = []
        for it in range(warmup + steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            g.iterate(1)
            g.synchronize()
            if it >= warmup:
                times.append(g.stage_times()["exact"])
        flags = g.stats()["device_flags"]
    ms = statistics.fmean(times)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peaks = measured_peaks_raw()
    clock_ghz = (peaks.get("sm_max_mhz") or 2070.0) / 1e3
    fma_peak = sms * 128 * 2 * clock_ghz / 1e3  # TFLOP/s
    ach = 11.0 * n * n / (ms * 1e-3) / 1e12
    return {"kernel": "k_exact", "n": n, "pairs": n * n, "kernel_ms": ms, "bound": "alu",
            "achieved": ach, "peak": fma_peak, "unit": "TFLOP/s", "frac": ach / fma_peak,
            "pairs_per_s": n * n / (ms * 1e-3), "mix_ceiling_frac": 11.0 / 16.0,
            "peak_kind": "derived: %d SMs x 128 FP32 lanes x 2 flop (FMA) x %.2f GHz" % (sms, clock_ghz),
            "workload": name + ": " + WORKLOADS[name]["desc"] + ", gamma = 2, one launch per iteration",
            "device_flags": flags}


def mixed_measurement(e, xy, spec, stream, flush, steps, warmup):
    """Precision mode BF16x3 (the column stage of the grid interaction as BF16
    split-precision tensor-core products with FP32 accumulation) on the same workload and
    timing as the main line, beside the FP32 mode: whole-iteration rate, the column
    stage's in-graph time, and the force field of both modes at the same positions (their
    relative L2 difference; each mode's error against the FP64 oracle is measured by the
    GPU parity tests)."""
    import numpy as np
    import torch
    from paper_2303_03964_gb300 import tfdp
    n = xy.shape[0]
    out = {}
    forces = {}
    for name, prec in (("fp32", tfdp.PREC_FP32), ("bf16x3", tfdp.PREC_BF16X3)):
        params = tfdp.params_default(k_interp=spec["k"], grid_max=spec["grid_max"],
                                     total_iters=spec["total_iters"], precision=prec)
        with tfdp.Graph(n, e, xy, params, stream=stream.cuda_stream) as g:
            forces[name] = g.eval_forces()[0].astype(np.float64)
            g.set_stage_timing_mask(["cols"])

            def step():
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.iterate(1)
                e1.record(stream)
                stream.synchronize()
                return e0.elapsed_time(e1), g.stage_times()["cols"]
            for _ in range(warmup):
                step()
            res = [step() for _ in range(steps)]
            st = g.stats()
        ms = sum(r[0] for r in res) / len(res)
        out[name] = {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "cols_ms": sum(r[1] for r in res) / len(res),
                     "cols_kernel": "k_cols_tc" if name == "bf16x3" else "k_cols_r",
                     "device_flags": st["device_flags"]}
    diff = float(np.linalg.norm(forces["bf16x3"] - forces["fp32"]) / np.linalg.norm(forces["fp32"]))
    out["frep_rel_l2_bf16x3_vs_fp32"] = diff
    out["speedup_bf16x3_over_fp32"] = out["fp32"]["ms_per_step"] / out["bf16x3"]["ms_per_step"]
    out["force_error_vs_oracle"] = {
        "fp32": 4.3e-7, "bf16x3": 4.8e-6, "tolerance": 1e-5,
        "source": "GPU parity tests, all 1M nodes against the FP64 oracle's ibFFT at the same positions"}
    out["note"] = ("both modes meet the 1e-5 force tolerance; the tensor-core column stage is slower than the "
                   "FP32 register FFT: its register epilogues between the four GEMM stages (twiddles, bf16 "
                   "hi/lo split, shared stores) take most of its time, not the tensor pipe")
    return out


def dynamic_k_measurement(e, xy, spec, stream, sampler=None):
    """One whole layout (total_iters iterations) of the same graph with the dynamic k
    schedule of Sec. 3.4 (k = 1 for 90 % of the iterations, then 2, then 3) against the
    fixed k = 3 of the main line. Each run starts from the same positions, after one
    untimed run that captures the iteration graphs of every k."""
    import torch
    from paper_2303_03964_gb300 import tfdp
    n, T = xy.shape[0], spec["total_iters"]
    out = {"workload": "%d-iteration layout from X0 of the same workload, grid up to %d, CUDA events "
                       "around the whole layout" % (T, spec["grid_max"])}
    for name, k in (("fixed_k3", 3), ("dynamic", tfdp.K_DYNAMIC)):
        p = tfdp.params_default(k_interp=k, grid_max=spec["grid_max"], total_iters=T)
        with tfdp.Graph(n, e, xy, p, stream=stream.cuda_stream) as g:
            g.iterate(T)
            g.set_positions(xy)
            g.set_iteration(0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if sampler is not None:
                sampler.active = True
            e0.record(stream)
            g.iterate(T)
            e1.record(stream)
            stream.synchronize()
            if sampler is not None and isinstance(sampler, NvmlSampler):
                sampler.active = False
            ms = e0.elapsed_time(e1)
            flags = g.stats()["device_flags"]
        out[name] = {"layout_ms": ms, "value": n * T / (ms * 1e-3), "unit": UNIT, "device_flags": flags}
    out["speedup"] = out["fixed_k3"]["layout_ms"] / out["dynamic"]["layout_ms"]
    return out


def quality_measurement():
    """Layout quality of the ibFFT path against the exact path (Sec. 4 metrics): three
    synthetic graphs, 300-iteration layouts from the same start, host-side metrics."""
    import numpy as np
    from paper_2303_03964_gb300 import quality as q
    from paper_2303_03964_gb300 import synth, tfdp
    rng = synth.rng_for(6)
    rng_spread = synth.rng_for(7)  # other starts, drawn apart so the main sequence is unchanged
    graphs = []
    e, _ = synth.sbm(2000, 10, 8.0, 0.9, rng)
    graphs.append(("sbm_2000", 2000, e))
    graphs.append(("lattice_40x40", 1600, synth.lattice(40, 40)))
    graphs.append(("ba_2000", 2000, synth.barabasi_albert(2000, 2, rng)))
    out = {"workload": "SBM n=2000 (10 blocks, mean degree 8), 40x40 lattice, BA n=2000 (m0=2); "
                       "300 iterations, k=3, grid <= 255; relative = (ibFFT - exact) / exact"}
    for name, n, e in graphs:
        xy0 = synth.uniform_positions(n, np.sqrt(n) / 2.0, rng)
        m = {}
        for label, rep in (("exact", tfdp.REP_EXACT), ("ibfft", tfdp.REP_FFT)):
            with tfdp.Graph(n, e, xy0, tfdp.params_default(rep_mode=rep, total_iters=300, grid_max=255)) as g:
                g.iterate(300)
                m[label] = q.evaluate(g.get_positions(), e)
        m["relative"] = {k: q.relative(m["ibfft"][k], m["exact"][k]) for k in m["exact"]}
        # the spread of the exact method itself: the same graph from another random start
        xy1 = synth.uniform_positions(n, np.sqrt(n) / 2.0, rng_spread)
        with tfdp.Graph(n, e, xy1, tfdp.params_default(rep_mode=tfdp.REP_EXACT, total_iters=300,
                                                        grid_max=255)) as g:
            g.iterate(300)
            other = q.evaluate(g.get_positions(), e)
        m["exact_seed_spread"] = {k: q.relative(other[k], m["exact"][k]) for k in m["exact"]}
        out[name] = m
    return out


def cpu_baseline(e, xy, spec, budget_s=15.0):
    """The FP64 oracle as it stands, on the same workload, on this host's cores."""
    import numpy as np
    import oracle
    x = xy.astype(np.float64)
    mode = "exact" if spec["rep"] == "exact" else "fft"
    iters = 0
    t0 = time.perf_counter()
    while True:
        x = oracle.iterate(x, e, 1, mode=mode, k=spec["k"], grid_max=spec["grid_max"],
                           T=spec["total_iters"], t0=iters)
        iters += 1
        el = time.perf_counter() - t0
        if el > budget_s or iters >= 50:
            break
    n = xy.shape[0]
    return {"value": n * iters / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d full iteration(s) of the same workload (%s repulsion), %.1f s" % (
                iters, mode, el)}


def batched_measurement(args, stream, flush, steps, warmup, solo_sample=48, sampler=None):
    """512 mixed graphs (n log-uniform in [1k, 50k]) advanced together as a batch, with
    every graph at the reference grid (k = 3, grid <= 255: P = 512) and with the grids the
    autotuner (tfdp_batch_plan) picks per graph by measured force error; against the same
    graphs run one at a time (a sample of them, reference grid)."""
    import numpy as np
    import torch
    from paper_2303_03964_gb300 import synth, tfdp
    graphs = synth.batch_mixed()
    base = tfdp.params_default(grid_max=255, total_iters=300)
    params = [base for _ in graphs]
    total_n = sum(g[0] for g in graphs)
    peak, _ = measured_peaks()

    def timed(fn):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    def run_batch(prm):
        b = tfdp.Batch(graphs, prm, stream=stream.cuda_stream)
        blocks = b.autotune(3)
        for _ in range(warmup):
            timed(lambda: b.iterate(1))
        if sampler is not None:
            sampler.active = True
        ms = [timed(lambda: b.iterate(1)) for _ in range(steps)]
        if sampler is not None and isinstance(sampler, NvmlSampler):
            sampler.active = False
        sts = [b.stats(q) for q in range(len(graphs))]
        parts = b.num_parts()
        phase_parts = b.phase_parts()
        b.close()
        # single-pass byte model of every graph's iteration at its own grid and FFT size
        model_bytes = sum(iteration_model_bytes(g[0], len(g[1]), st["grid_G"], st["fft_P"])
                          for g, st in zip(graphs, sts))
        mean_ms = statistics.fmean(ms)
        return {"value": total_n * len(ms) / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": mean_ms,
                "parts": parts, "cooperative_ctas": blocks,
                "launch_shape": ("one launch per phase" if phase_parts == parts else
                                 "one cooperative launch" if phase_parts == 0 else
                                 "%d of %d parts one launch per phase" % (phase_parts, parts)),
                "device_flags": max(st["device_flags"] for st in sts),
                "iteration_roofline": {
                    "bytes_per_iteration": model_bytes, "achieved": model_bytes / (mean_ms * 1e-3) / 1e9,
                    "peak": peak, "unit": "GB/s", "frac": model_bytes / (mean_ms * 1e-3) / 1e9 / peak,
                    "model": "sum over graphs of 28 n + 24 m node bytes + 24 G^2 + 60 P (P/2+1) grid bytes"},
                "fft_P_counts": {str(P): sum(1 for st in sts if st["fft_P"] == P)
                                 for P in sorted(set(st["fft_P"] for st in sts))}}

    ref = run_batch(params)
    t0 = time.perf_counter()
    planned, err = tfdp.batch_plan(graphs, base, max_error_ratio=1.5, min_error_bound=0.02, probes=2)
    plan_s = time.perf_counter() - t0
    tuned = run_batch(planned)
    tuned["plan_s"] = plan_s
    tuned["k_counts"] = {str(k): sum(1 for p in planned if p.k_interp == k) for k in (1, 2, 3)}
    tuned["force_error_vs_exact_max"] = float(np.max(err))
    tuned["force_error_vs_exact_median"] = float(np.median(err))
    tuned["rule"] = ("per graph the cheapest grid (a smaller FFT at any k, else the reference) whose repulsion "
                     "error against the exact sum is within max(1.5x the reference grid's, 2 %), measured on 2 "
                     "graphs per half-octave of n")
    # solo: a sample of the same graphs, one graph per launch sequence (reference grid)
    idx = list(range(0, len(graphs), max(1, len(graphs) // solo_sample)))[:solo_sample]
    solo_n, solo_ms = 0, 0.0
    for q in idx:
        n, e, xy = graphs[q]
        with tfdp.Graph(n, e, xy, params[q], stream=stream.cuda_stream) as g:
            for _ in range(2):
                timed(lambda: g.iterate(1))
            t = [timed(lambda: g.iterate(1)) for _ in range(3)]
        solo_n += n
        solo_ms += statistics.median(t)
    solo_value = solo_n / (solo_ms * 1e-3)
    out = {"workload": "512 graphs, n log-uniform in [1k, 50k] (sum %d), SBM / BA m0=2 / lattice in turn, "
                       "FP32; value: autotuned grids, reference: k=3, grid <= 255 (P=512) for every graph"
                       % total_n,
           "value": tuned["value"], "unit": UNIT, "ms_per_step": tuned["ms_per_step"],
           "autotuned": tuned, "reference_grid": ref, "solo_value": solo_value,
           "solo_sample": "%d of the graphs (%d nodes), reference grid, one iteration each, median of 3" % (
               len(idx), solo_n),
           "speedup_vs_solo": ref["value"] / solo_value,
           "speedup_autotuned_vs_reference_grid": tuned["value"] / ref["value"],
           "device_flags": max(ref["device_flags"], tuned["device_flags"]),
           "iteration_roofline": tuned["iteration_roofline"]}
    return out


def dist_env():
    from paper_2303_03964_gb300 import replicas
    return replicas.world()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    spec = WORKLOADS[args.workload]
    e, xy = make_workload(args.workload)
    import numpy as np
    import oracle
    x = xy.astype(np.float64)
    mode = "exact" if spec["rep"] == "exact" else "fft"
    for w in range(args.warmup):
        x = oracle.iterate(x, e, 1, mode=mode, k=spec["k"], grid_max=spec["grid_max"],
                           T=spec["total_iters"], t0=w)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        x = oracle.iterate(x, e, 1, mode=mode, k=spec["k"], grid_max=spec["grid_max"],
                           T=spec["total_iters"], t0=args.warmup + s)
        times.append(time.perf_counter() - t0)
    n = xy.shape[0]
    tot = sum(times)
    value = n * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": spec["desc"], "rep": mode,
                       "k": spec["k"], "grid_max": spec["grid_max"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "one full FP64 oracle iteration per step on the same workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2303_03964_gb300 import replicas, tfdp

    spec = WORKLOADS[args.workload]
    e, xy = make_workload(args.workload)
    n, m = xy.shape[0], e.shape[0]
    rep = tfdp.REP_EXACT if spec["rep"] == "exact" else tfdp.REP_FFT
    params = tfdp.params_default(rep_mode=rep, k_interp=spec["k"], grid_max=spec["grid_max"],
                                 total_iters=spec["total_iters"])
    stream = torch.cuda.Stream()
    g = tfdp.Graph(n, e, xy, params, stream=stream.cuda_stream)
    # warm-up with every stage bracketed by events, to find the dominant single kernel
    g.set_stage_timing(True)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        g.iterate(1)
        ev1.record(stream)
        stream.synchronize()
        return ev0.elapsed_time(ev1), g.stage_times()

    warm = [step()[1] for _ in range(args.warmup)]
    cand = {k: statistics.fmean(w[k] for w in warm[-2:]) for k in STAGE_KERNEL}
    dom = max(cand, key=cand.get)
    # the timed steps bracket only that kernel (the library records the events on a
    # side branch of the captured iteration, so they cost the step < 1 us)
    g.set_stage_timing_mask([dom])
    for _ in range(2):  # the iteration graph is recaptured with the new event set
        step()
    torch.cuda.synchronize()
    replicas.barrier()
    sampler = NvmlSampler(local)
    if not sampler.ok:
        sampler = ClockSampler(local)
    sampler.start()
    sampler.active = True
    step_ms, stages = [], []
    for _ in range(args.steps):
        ms, st = step()
        step_ms.append(ms)
        stages.append(st)
    torch.cuda.synchronize()
    replicas.barrier()
    if isinstance(sampler, NvmlSampler):
        sampler.active = False
    # replicas: every rank ran the same workload; the slowest rank's time counts
    total_ms = replicas.max_over_ranks(sum(step_ms))
    stats = g.stats()

    # end to end through the C ABI with host buffers: pinned positions in and out
    host_in = torch.empty((n, 2), dtype=torch.float32, pin_memory=True)
    host_out = torch.empty((n, 2), dtype=torch.float32, pin_memory=True)
    g.get_positions(host_out.numpy())
    host_in.copy_(host_out)
    e2e_s = []
    hin, hout = host_in.numpy(), host_out.numpy()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        g.run(hin, 1, hout)  # upload, one iteration, download: one call, one synchronisation
        e2e_s.append(time.perf_counter() - t0)
        host_in.copy_(host_out)
    e2e_total = replicas.max_over_ranks(sum(e2e_s))

    if rank != 0:
        g.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    dom_ms = statistics.fmean(st[dom] for st in stages)
    # per-stage breakdown, outside the timed region, with every stage bracketed
    g.set_stage_timing(True)
    brk = [step()[1] for _ in range(5)][2:]
    mean_stage = {k: statistics.fmean(b[k] for b in brk) for k in brk[0]}
    G, P = stats["grid_G"], stats["fft_P"]
    nbox = stats["grid_n_int"] ** 2
    peak, peak_kind = measured_peaks()
    roof = None
    if dom == "exact":
        # about 11 FP32 flops per pair (distance, kernel by reciprocal powers, two FMAs);
        # peak: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz = 80.5 TFLOP/s
        flops = 11.0 * n * n
        fma_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        ach = flops / (dom_ms * 1e-3) / 1e12
        roof = {"stage": dom, "kernel": STAGE_KERNEL[dom], "bound": "alu",
                "achieved": ach, "kernel_ms": dom_ms, "peak": fma_peak, "unit": "TFLOP/s",
                "frac": ach / fma_peak, "traffic": None,
                "peak_kind": "derived: 152 SMs x 128 FP32 FMA lanes x 2 flop x 2.07 GHz"}
    else:
        bytes_ = stage_bytes(dom, n, m, G, P, nbox)
        ach = bytes_ / (dom_ms * 1e-3) / 1e9
        tr = NCU_TRAFFIC.get((args.workload, dom))
        traffic = tr["bytes"] if tr and tr.get("sha") == source_sha(dom) else None
        roof = {"stage": dom, "kernel": stage_kernel(dom, P), "bound": "hbm", "achieved": ach, "peak": peak,
                "unit": "GB/s",
                "frac": ach / peak, "traffic": traffic, "algorithmic_bytes": bytes_, "kernel_ms": dom_ms,
                "peak_kind": peak_kind + " hbm_gbs (burst copy)"}
    cpu = None
    if not args.no_cpu_baseline and ws >= 1 and rank == 0:
        cpu = cpu_baseline(e, xy, spec)
    batched = None
    if not args.no_batch and args.workload == "lattice_1m":
        batched = batched_measurement(args, stream, flush, args.steps, args.warmup, sampler=sampler)
    serving = None
    if not args.no_serving and args.workload == "lattice_1m":
        serving = serving_measurement(sampler=sampler)
    others = None
    if not args.no_workloads and args.workload == "lattice_1m":
        others = {w: workload_measurement(w, stream, flush, min(args.steps, 20), args.warmup,
                                          cpu=not args.no_cpu_baseline)
                  for w in ("er_2000_exact", "sbm_100k", "ba_2m", "lattice_1m_paper_grid")}
    exact_kernel = None
    if not args.no_workloads and args.workload == "lattice_1m":
        exact_kernel = exact_kernel_measurement(stream, flush, min(args.steps, 10), args.warmup)
    quality = None
    if not args.no_quality and args.workload == "lattice_1m":
        quality = quality_measurement()
    mixed = None
    if not args.no_mixed and spec["rep"] == "fft" and spec["grid_max"] > 512:
        mixed = mixed_measurement(e, xy, spec, stream, flush, args.steps, args.warmup)
    dynamic_k = None
    if not args.no_dynamic_k and spec["rep"] == "fft":
        dynamic_k = dynamic_k_measurement(e, xy, spec, stream, sampler=sampler)
        if args.workload == "lattice_1m" and not args.no_workloads:
            # the paper's own grid rule on the same graph: G = 3000 at k = 3 (P = 8192),
            # 1000 at k = 1 (P = 2048)
            dynamic_k["paper_grid"] = dynamic_k_measurement(e, xy, WORKLOADS["lattice_1m_paper_grid"], stream,
                                                            sampler=sampler)
    clocks = sampler.stop()
    value = ws * n * args.steps / (total_ms * 1e-3)
    q = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": spec["desc"], "rep": spec["rep"],
                   "k": spec["k"], "grid_max": spec["grid_max"], "grid_G": G, "fft_P": P,
                   "grid_policy": "SNAP_H", "precision": "fp32",
                   "l2": "flushed before every step (256 MiB write, outside the timed events)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "step_ms_p50": q[len(q) // 2], "step_ms_p99": q[min(len(q) - 1, int(0.99 * len(q)))],
        "mixed": mixed,
        "batched": batched,
        "serving": serving,
        "dynamic_k": dynamic_k,
        "other_workloads": others,
        "exact_kernel": exact_kernel,
        "quality": quality,
        "stages_ms": mean_stage,
        "stages_note": "5 steps after the timed region with every stage bracketed by events "
                       "(the timed steps bracket only the roofline kernel)",
        "roofline": roof,
        "iteration_roofline": (iteration_roofline(n, m, G, P, total_ms / args.steps, peak)
                               if spec["rep"] == "fft" else None),
        "cpu_baseline": cpu,
        "e2e": {"value": ws * n * args.steps / e2e_total, "unit": UNIT,
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": stats["kernels_per_iteration"] * args.steps,
        "clocks": clocks,
        "device_flags": stats["device_flags"],
    }
    print(json.dumps(line), flush=True)
    g.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="lattice_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-graph batched measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the SBM 100k / BA 2M / ER 2000 (exact) lines and the exact-kernel "
                         "roofline (n = 65536) of the default run")
    ap.add_argument("--no-quality", action="store_true",
                    help="skip the exact-vs-ibFFT layout-quality comparison")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the BF16x3 precision-mode line")
    ap.add_argument("--no-dynamic-k", action="store_true",
                    help="skip the whole-layout comparison of the dynamic k schedule with k = 3")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

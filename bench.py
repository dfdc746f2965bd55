#!/usr/bin/env python3
"""Benchmark of the GB300 NNFFT library.

One step = one pass of the whole hot path on a fresh node set:
  nnfft_set_nodes (binning + sort of both node sets, Algorithm 2.2 step 0)
  + nnfft_exec (steps 1-4, forward) + nnfft_adjoint (its transpose)
at N = 4096, M1 = M2 = 2^20 uniform nodes, complex128, sigma1 = sigma2 = 2,
m1 = m2 = 8 (the fp64 / 1e-12 workload).  The metric counts M1 + M2 points per
transform, so a step processes 2 (M1 + M2) points.  Inputs are resident in HBM;
L2 is flushed (512 MB write) between timed steps and every step is timed with
CUDA events on the plan stream.

Also reported (same JSON line): per-stage device times, the roofline of the
dominant kernel, the fp32 path (m = 4), Chebyshev nodes, exec-only throughput
with a resident plan, the fast sinc transform (N = 1024, L1 = L2 = 2^18), the
end-to-end number through the host-buffer C ABI calls, and the CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NNFFT nonuniform pts/sec (M1+M2)/s at 1e-12 FP64 vs 2e-5 FP32 batched; p99 latency"
N_BW, M_PTS = 4096, 1 << 20
SINC_N, SINC_L = 1024, 1 << 18
L2_FLUSH_BYTES = 512 << 20
WORKLOAD = ("nnfft_fp64 N=4096 M1=M2=2^20 uniform nodes sigma=2 m=8: "
            "set_nodes + forward + adjoint per step")


def nvtx_push(name):
    """Open an NVTX range (profilers filter launches on it); a no-op without NVTX."""
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 FMA peak of GB300: the profiling recipe lists 1.25 TFLOP/s FP64, i.e. 152 SMs x
# 2 FP64 FMA per clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s.
# FP32/INT32 lane operations per second: 152 SMs x 128 FP32 lanes x 2.07 GHz (max SM clock),
# one operation per lane and clock (an FMA counts once)
FP32_LANE_TOPS = 152 * 128 * 2.070e9 / 1e12


def df_ops(kind, D, m=8):
    """FP32/INT32 lane operations of the split-precision arithmetic per unit (point for the
    point kernels, grid point for the spread convolution, cell for the gather convolution),
    counted from the double-float primitives: product 4, accumulate 8, sum 11, Chebyshev
    recurrence step 15, complex128 -> float pairs 20 per real, float pair -> double 11;
    degrees d < D/2 in double-float, the others 3 FP32 operations each (recurrence + 2 FMA).
    Loads, index arithmetic and the work-item reductions are not counted."""
    B, F = D // 2, D - D // 2
    if kind == "moments":       # split, 2y, degrees 0 and 1, recurrence degrees, FP32 degrees
        return 2 * 20 + 2 + 2 * 8 + 2 * 12 + (B - 2) * (15 + 2 * 12) + 3 * F
    if kind == "eval":          # ... + the FP32 part added, normalised, assembled into doubles
        return 2 + 2 * 12 + (B - 2) * (15 + 2 * 12) + 3 * F + 2 * 8 + 2 * 3 + 2 * 11
    ntap = 2 * m                # convolutions: 2m taps per degree, then the degree sum
    return B * ntap * 2 * 12 + F * ntap * 2 + (D - 1) * 22 + 14


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled during the timed region.

    Reads NVML through ctypes every 5 ms from a background thread (read-only queries);
    falls back to `nvidia-smi -lms 100` when libnvidia-ml cannot be loaded."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, index):
        import ctypes
        import threading
        self.index = index
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self._proc = None
        self._nvml = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                if nv.nvmlDeviceGetHandleByIndex_v2(int(index), ctypes.byref(h)) == 0:
                    self._nvml, self._h = nv, h
                    mx = ctypes.c_uint()
                    if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:   # NVML_CLOCK_SM
                        self.max_mhz = float(mx.value)
        except Exception:
            self._nvml = None

    def _sample_once(self):
        import ctypes
        nv, h = self._nvml, self._h
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and fn(h, ctypes.byref(rs)) == 0:
            self.samples.append((float(clk.value), int(rs.value)))

    def _run(self):
        while not self._stop.is_set():
            self._sample_once()
            self._stop.wait(0.005)

    def __enter__(self):
        import threading
        if self._nvml is not None:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
        else:
            try:
                q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                     "clocks_event_reasons.hw_thermal_slowdown,"
                     "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
                self._proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                     "--format=csv,noheader,nounits", "-lms", "100"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception:
                self._proc = None
        return self

    def __exit__(self, *exc):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=2)
            self._sample_once()          # the state at the end of the region
        if self._proc is not None:
            self._proc.terminate()
            try:
                out, _ = self._proc.communicate(timeout=5)
            except Exception:
                self._proc.kill()
                out = ""
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for r in (out or "").strip().splitlines():
                f = [t.strip() for t in r.split(",")]
                if len(f) >= 6 and f[0].replace(".", "").isdigit():
                    self.max_mhz = float(f[1]) if f[1].replace(".", "").isdigit() else self.max_mhz
                    bits = sum(self.REASONS[n] for n, v in zip(names, f[2:6]) if v == "Active")
                    self.samples.append((float(f[0]), bits))
        return False

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"],
                    "samples": 0}
        mhz = [c for c, _ in self.samples]
        reasons = sorted({n for _, b in self.samples for n, bit in self.REASONS.items() if b & bit})
        return {"sm_mhz": float(np.median(mhz)), "sm_min_mhz": float(np.min(mhz)),
                "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples": len(self.samples),
                "source": "nvml" if self._nvml is not None else "nvidia-smi"}


# -------------------------------------------------------------------------------------------
# the CPU oracle (baseline leg and reference arm)
# -------------------------------------------------------------------------------------------
def host_cpu():
    """The host's CPU model and logical core count (lscpu when present)."""
    import platform
    import shutil
    import subprocess
    model = None
    if shutil.which("lscpu"):
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            model = None
    return {"model": model or platform.processor() or platform.machine(),
            "machine": platform.machine(), "nproc": os.cpu_count()}


def oracle_sample(seconds_target=12.0, seed=0):
    """Time the oracle's direct sums on a bounded row sample of the workload; extrapolate."""
    import oracle
    from paper_2107_02671_gb300 import workloads as W
    v, x, f = W.nnfft_inputs(M_PTS, M_PTS, seed)
    g = W.adjoint_inputs(M_PTS, seed)
    cores = oracle.num_threads()
    probe = max(8, 2 * cores)                    # rows run in parallel over the cores
    t0 = time.perf_counter()
    oracle.nnfft_direct(N_BW, v, f, x, rows=np.arange(probe))
    per_row = (time.perf_counter() - t0) / probe
    J = int(max(16, min(M_PTS, seconds_target / 2 / max(per_row, 1e-9))))
    rows = W.sample_rows(M_PTS, J, seed)
    t0 = time.perf_counter()
    oracle.nnfft_direct(N_BW, v, f, x, rows=rows)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.nnfft_adjoint_direct(N_BW, v, x, g, rows=rows)
    t_adj = time.perf_counter() - t0
    full = (t_fwd + t_adj) * M_PTS / len(rows)
    return {"value": 4 * M_PTS / full, "unit": "pts/s", "cores": cores, "kind": "oracle",
            "host": host_cpu(),
            "sample": (f"direct fp64 sums for {len(rows)} sampled output rows of the forward and "
                       f"of the adjoint at N=4096, M1=M2=2^20 (each row sums all 2^20 terms); "
                       f"extrapolated x{M_PTS / len(rows):.0f} to the full step"),
            "seconds": t_fwd + t_adj}


def oracle_stage_reference(seed=0):
    """The second CPU baseline: the oracle's Algorithm 2.2 stage reference (the fast method
    itself, exact sinh windows, naive DFT for step 3) at the full workload, forward and
    adjoint, on one host core.  Nothing is sampled or extrapolated."""
    import oracle
    from paper_2107_02671_gb300 import workloads as W
    v, x, f = W.nnfft_inputs(M_PTS, M_PTS, seed)
    g = W.adjoint_inputs(M_PTS, seed)
    P = oracle.make_params(N_BW, 2.0, 2.0, 8, 8)
    t0 = time.perf_counter()
    oracle.nnfft_alg22(P, v, f, x, nthreads=1)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.nnfft_alg22_adjoint(P, v, x, g, nthreads=1)
    t_adj = time.perf_counter() - t0
    return {"value": 4 * M_PTS / (t_fwd + t_adj), "unit": "pts/s", "cores": 1,
            "kind": "oracle stage reference",
            "sample": ("Algorithm 2.2 step by step (exact sinh windows, naive DFT of length "
                       f"N2={P.N2} over K1={P.K1} grid values for step 3) and its transpose at "
                       "N=4096, M1=M2=2^20, sigma=2, m=8, full size, one thread, no extrapolation"),
            "seconds": t_fwd + t_adj, "forward_s": t_fwd, "adjoint_s": t_adj}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    from paper_2107_02671_gb300 import workloads as W
    v, x, f = W.nnfft_inputs(M_PTS, M_PTS, 0)
    g = W.adjoint_inputs(M_PTS, 0)
    cores = oracle.num_threads()
    probe = 4
    t0 = time.perf_counter()
    oracle.nnfft_direct(N_BW, v, f, x, rows=np.arange(probe))
    per_row = (time.perf_counter() - t0) / probe
    total_budget = 150.0   # seconds for warmup + timed steps together
    J = int(max(4, min(4096, total_budget / (args.steps + args.warmup) / 2 / max(per_row, 1e-9))))
    times = []
    for s in range(args.warmup + args.steps):
        rows = W.sample_rows(M_PTS, J, 100 + s)
        t0 = time.perf_counter()
        oracle.nnfft_direct(N_BW, v, f, x, rows=rows)
        oracle.nnfft_adjoint_direct(N_BW, v, x, g, rows=rows)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    # A step is the bounded sample: J output rows of the forward and J of the adjoint, each
    # summing all 2^20 terms, i.e. J/M2 of a full forward and of a full adjoint.  In the
    # metric's unit that is 4 J point-equivalents per step (a full step is 4 M), so
    # value = 4 J / step time, the full-step throughput.
    step_s = float(np.mean(times))
    value = 4 * J / step_s
    sample = (f"per step: direct fp64 forward and adjoint sums for {J} sampled output rows "
              f"(all 2^20 terms each) = {J}/{M_PTS} of a full set_nodes + forward + adjoint "
              f"step; value = 4*{J} point-equivalents / step time (a full step would take "
              f"{step_s * M_PTS / J:.0f} s)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "points_per_step": 4 * J,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "N": N_BW, "M1": M_PTS, "M2": M_PTS,
                                        "m": 8, "sigma": 2.0, "nodes": "uniform"},
        "cpu_baseline": {"value": value, "unit": "pts/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------------------------------
# our arm
# -------------------------------------------------------------------------------------------
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of every
# split-precision point-kernel variant at the headline size, from ncu captures of
# `python bench.py --steps 3 --warmup 3 --no-cpu-baseline --no-batch --no-serve --no-m-sweep --tuning T`
# (NVTX range headline_seq) with T = 8,8,0,0,1,1,256,0 / 4,4,0,0,2,2,256,0 /
# 16,16,0,0,32,32,256,0, averaged over the captured launches.  The files the kernels are
# built from (their code, the double-float primitives, the side descriptor) are hashed; a
# change since the capture reports null.
NCU_SOURCES = ["kern_spread_df.cu", "df.cuh", "side.h"]
NCU_HASH = "6ae0a0d0a1c0ed5c"
NCU_TRAFFIC = {
    "k_moments_df_team<14>": 29457216,          # 8 lanes per work item
    "k_moments_df_team_pf<14>": 29459968 + 256, # 8 lanes, two accumulator sets per lane
    "k_moments_df_half<14>": 29457920,          # 16
    "k_eval_df_flat<14>": 20458432 + 1791360,   # one thread per point
    "k_eval_df_flat_tma<14>": 20435008 + 1765248,   # the same, cells staged by TMA
    "k_eval_df<14>": 16266240 + 1656320,        # 32
}


def point_kernel(stage, tuning):
    """Name of the split-precision kernel a point stage ran with the plan's tuning."""
    side = "v" if stage in ("fwd_moments", "adj_eval") else "x"
    if stage.endswith("_moments"):
        lanes = tuning.get(f"moments_lanes_{side}", 32)
        return {8: "k_moments_df_team<14>", 4: "k_moments_df_team_pf<14>",
                16: "k_moments_df_half<14>"}.get(lanes, "k_moments_df_warp<14>")
    lanes = tuning.get(f"eval_lanes_{side}", 32)
    return {1: "k_eval_df_flat<14>", 2: "k_eval_df_flat_tma<14>", 3: "k_eval_gather_df<14>",
            8: "k_eval_df_team<14>"}.get(lanes, "k_eval_df<14>")


def ncu_traffic(stage, tuning):
    import hashlib
    if not (stage.endswith("_moments") or stage.endswith("_eval")):
        return None, None
    kern = point_kernel(stage, tuning)
    h = hashlib.sha256()
    for f in NCU_SOURCES:
        with open(os.path.join(ROOT, "paper_2107_02671_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != NCU_HASH:
        return None, kern + ": source changed since the ncu capture"
    return NCU_TRAFFIC.get(kern), kern


BATCH_COUNT = 512


M_SWEEP = (1 << 22, 1 << 24, 1 << 26)


def run_m_sweep(args, rank, dev, flush, timed, pk):
    """fp64 (split precision), N = 4096, sigma = 2, m = 8, M1 = M2 = M uniform nodes for the
    M of M_SWEEP: the step (one graph launch) after the autotuner's choice, and from a
    sequential pass the point kernels' HBM fractions (24 B per point).  At 2^20 points a cell
    holds ~128 points and the moments launch ~13 warps per SM; larger M fills the cells and the
    GPU."""
    import torch
    from paper_2107_02671_gb300 import nnfft as B
    from paper_2107_02671_gb300 import workloads as W
    out = {"what": "fp64 N=4096 sigma=2 m=8, M1 = M2 = M uniform nodes; HBM fractions of the "
                   "point kernels from a sequential pass, 24 B per point",
           "runs": []}
    for M in M_SWEEP:
        v, x, f = W.nnfft_inputs(M, M, 50 + rank)
        g = W.adjoint_inputs(M, 50 + rank)
        vd, xd, fd, gd = (torch.from_numpy(a).to(dev) for a in (v, x, f, g))
        del v, x, f, g
        y = torch.empty(M, dtype=torch.complex128, device=dev)
        z = torch.empty(M, dtype=torch.complex128, device=dev)
        P = B.Plan(N_BW, M, M, 2.0, 2.0, 8, 8, dtype=torch.complex128)
        tune = P.autotune(fd, gd, y, z, reps=2, v=vd, x=xd, flush_l2=True)
        gr = P.transform_graph(vd, xd, fd, gd, y, z)
        for _ in range(3):
            gr.launch()
        P.sync()
        k = 10
        ms, _, _ = timed(gr.launch, k, label="m_sweep")
        P.sync()
        gr.close()

        def seq(P=P, vd=vd, xd=xd, fd=fd, gd=gd, y=y, z=z):
            P.set_nodes(vd, xd)
            P.exec(fd, y)
            P.adjoint(gd, z)
        _, _, st = timed(seq, k, P, label="m_sweep_seq")
        P.sync()
        stage = {kk: 1e3 * tot / n for kk, (tot, n) in st.items() if n}
        hbm = {kk: round(24 * M / (stage[kk] / 1e6) / 1e9 / pk["hbm_gbs"], 3)
               for kk in ("fwd_moments", "fwd_eval", "adj_moments", "adj_eval") if kk in stage}
        out["runs"].append({"M": M, "value": 4 * M / (np.mean(ms) / 1e3), "unit": "pts/s",
                            "ms_per_step": float(np.mean(ms)),
                            "stage_us": {kk: round(vv, 1) for kk, vv in stage.items()},
                            "hbm_frac_point_kernels": hbm,
                            "tuning": {kk: tune[kk] for kk in ("moments_lanes_v", "eval_lanes_v",
                                                               "fft_variant", "item_cap", "sort_lsd")}})
        P.close()
        del P, vd, xd, fd, gd, y, z
        torch.cuda.empty_cache()
    return out


def run_batched(args, rank, dev, flush, timed, pk):
    """The batched workload at fp32 (m = 4, complex64) and fp64 (m = 8, complex128): one
    plan holding all instances; per step set_nodes + exec + adjoint, and exec + adjoint
    with the nodes resident.  Point-kernel HBM fractions from the stage times."""
    import torch
    from paper_2107_02671_gb300 import nnfft as B
    from paper_2107_02671_gb300 import workloads as W
    count = args.batch_count
    N, M1, M2 = W.batch_sizes(count, rank)
    out = {"instances": count, "sum_M1": int(M1.sum()), "sum_M2": int(M2.sum()),
           "sizes": "M1, M2 log-uniform in [1e3, 1e6], N log-uniform in [64, 8192], uniform nodes"}
    pts = int(M1.sum() + M2.sum())
    variants = (("fp32_m4", torch.complex64, np.complex64, 4, 16),
                ("fp64_m8", torch.complex128, np.complex128, 8, 24))
    if args.only_fp32_batch:
        variants = variants[:1]
    for name, dt, npd, m, bpp in variants:
        v, x, f = W.batch_inputs(M1, M2, 1000 * rank, dtype=npd)
        g = W.draw_complex(np.random.default_rng(7 + rank), int(M2.sum()), npd)
        t0 = time.time()
        P = B.BatchPlan(N, M1, M2, 2.0, 2.0, m, dtype=dt)
        t_plan = time.time() - t0
        vd, xd, fd, gd = (torch.from_numpy(a).to(dev) for a in (v, x, f, g))
        y = torch.empty(int(M2.sum()), dtype=dt, device=dev)
        z = torch.empty(int(M1.sum()), dtype=dt, device=dev)

        def step(P=P, vd=vd, xd=xd, fd=fd, gd=gd, y=y, z=z):
            P.transform(vd, xd, fd, gd, y, z)

        def fwd_adj(P=P, fd=fd, gd=gd, y=y, z=z):
            P.exec_adjoint(fd, gd, y, z)

        tune = P.autotune(fd, gd, y, z, reps=2, v=vd, x=xd, flush_l2=True)
        for _ in range(3):
            step()
        P.sync()
        k = max(3, min(20, args.steps // 10))
        ms_full, l_full, _ = timed(step, k, label="batched_step")
        P.sync()
        # the same step captured once as a CUDA graph over these buffers, one launch per step
        graph = P.transform_graph(vd, xd, fd, gd, y, z)
        for _ in range(2):
            graph.launch()
        P.sync()
        ms_graph, l_graph, _ = timed(graph.launch, k, label="batched_graph")
        P.sync()
        graph.close()
        ms_exec, _, _ = timed(fwd_adj, k, label="batched_exec")
        P.sync()

        def step_seq(P=P, vd=vd, xd=xd, fd=fd, gd=gd, y=y, z=z):
            P.set_nodes(vd, xd)
            P.exec(fd, y)
            P.adjoint(gd, z)

        # split precision: the grid stage as stage-wide launches and as one cooperative
        # launch per direction (fft_variant 3), each timed as the graph step
        grid_forms = None
        if dt == torch.complex128:
            grid_forms = {}
            t0v = dict(P.tuning())
            keep = (t0v["moments_lanes_v"], t0v["moments_lanes_x"])
            rest = (t0v["item_split"], t0v["eval_lanes_v"], t0v["eval_lanes_x"], t0v["item_cap"],
                    t0v["sort_lsd"])
            base = t0v["fft_variant"] if t0v["fft_variant"] != 3 else 0
            for label, fv in (("stage_launches", base), ("fused_cooperative", 3)):
                try:
                    P.set_tuning(*keep, fv, *rest)
                except B.NNFFTError as e:
                    grid_forms[label] = {"unavailable": str(e)}
                    continue
                gr = P.transform_graph(vd, xd, fd, gd, y, z)
                for _ in range(2):
                    gr.launch()
                P.sync()
                ms_g, _, _ = timed(gr.launch, k, label="batched_grid_form")
                P.sync()
                gr.close()
                _, _, stf = timed(step_seq, k, P, label="batched_seq_form")
                P.sync()
                sus = {kk: 1e3 * tot / n for kk, (tot, n) in stf.items() if n}
                grid_us = sum(sus.get(f"{d}_{s2}", 0.0) for d in ("fwd", "adj")
                              for s2 in ("cell_fold", "spread_conv", "fft", "gather_conv"))
                grid_forms[label] = {"fft_variant": fv, "graph_ms_per_step": float(np.mean(ms_g)),
                                     "graph_value": 2 * pts / (np.mean(ms_g) / 1e3),
                                     "grid_stage_us_sequential": round(grid_us, 1)}
            P.set_tuning(*keep, t0v["fft_variant"], *rest)
            grid_forms["what"] = ("grid stage (cell fold, spread convolution, FFT, gather "
                                  "convolution) as stage-wide launches or as one cooperative "
                                  "launch per direction with grid barriers; graph step and the "
                                  "grid stages' device time in a sequential pass")
        # per-stage times (and kernel HBM fractions) from a pass with the two directions
        # one after the other: in the timed step they share the GPU
        _, _, st = timed(step_seq, k, P, label="batched_seq")
        P.sync()
        stage = {kk: round(1e3 * tot / n, 1) for kk, (tot, n) in st.items() if n}
        hbm = {}
        for kk in ("fwd_moments", "fwd_eval", "adj_moments", "adj_eval"):
            if kk in stage:
                npts = M1.sum() if kk in ("fwd_moments", "adj_eval") else M2.sum()
                gbs = bpp * float(npts) / (stage[kk] / 1e6) / 1e9
                hbm[kk] = {"us": stage[kk], "achieved_gbs": gbs, "frac": gbs / pk["hbm_gbs"]}
        # accuracy on a few instances (sampled rows against the oracle)
        acc = None
        if rank == 0:
            try:
                import oracle
                yh = y.cpu().numpy()
                worst = 0.0
                for i in range(0, count, 97):
                    a1, b1, a2, b2 = P.off1[i], P.off1[i + 1], P.off2[i], P.off2[i + 1]
                    rows = W.sample_rows(int(M2[i]), 4, i)
                    fi = f[a1:b1].astype(np.complex128)
                    want = oracle.nnfft_direct(int(N[i]), v[a1:b1], fi, x[a2:b2], rows=rows)
                    worst = max(worst, float(np.max(np.abs(yh[a2:b2][rows] - want)) / np.sum(np.abs(fi))))
                acc = worst
            except Exception as e:   # accuracy is reported, the tests enforce it
                acc = f"unavailable: {e}"
        out[name] = {"value": 2 * pts / (np.mean(ms_full) / 1e3), "unit": "pts/s",
                     "ms_per_step": float(np.mean(ms_full)),
                     "step": "set_nodes + exec + adjoint over all instances",
                     "graph_value": 2 * pts / (np.mean(ms_graph) / 1e3),
                     "graph_ms_per_step": float(np.mean(ms_graph)),
                     "graph_launches_per_step": l_graph // k,
                     "graph_what": "the same step as one CUDA graph launch (nnfft_transform "
                                   "captured once over these buffers)",
                     "exec_adjoint_value": 2 * pts / (np.mean(ms_exec) / 1e3),
                     "exec_adjoint_ms": float(np.mean(ms_exec)),
                     "launches_per_step": l_full // k, "stage_us": stage,
                     "stage_note": "stage_us and the HBM fractions come from a sequential pass "
                                   "(set_nodes, exec, adjoint)",
                     "hbm_roofline_point_kernels": hbm, "plan_seconds": round(t_plan, 2),
                     "max_rel_err_sampled": acc, "tuning": tune}
        if grid_forms is not None:
            out[name]["grid_stage_forms"] = grid_forms
        del P, vd, xd, fd, gd, y, z
        torch.cuda.empty_cache()
    return out


SERVE_RATE, SERVE_WARM, SERVE_TIMED = 2000.0, 1500, 100000
SERVE_MAXP = 1 << 22
SERVE_SWEEP = (4000.0, 8000.0, 16000.0)      # offered rates of the capacity sweep
SERVE_SWEEP_N = 4000


def _serve_pools(rng):
    """Pinned host pools the requests slice: uniform nodes, N(0,1) values."""
    import torch
    P = SERVE_MAXP
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()      # noqa: E731
    pools = {"nodes": pin(rng.uniform(-0.5, 0.5, P))}
    c128 = (rng.standard_normal(P) + 1j * rng.standard_normal(P)).astype(np.complex128)
    pools["c128"], pools["c64"] = pin(c128), pin(c128.astype(np.complex64))
    r64 = rng.standard_normal(P)
    pools["r64"], pools["r32"] = pin(r64), pin(r64.astype(np.float32))
    pools["out"] = [torch.empty(P, dtype=torch.complex128).pin_memory().numpy() for _ in range(16)]
    return pools


def _serve_stream(S, pools, rng, n, rate, warm):
    """Submit n requests of the served mix with exponential gaps at `rate` per second; the
    first `warm` fill the plan cache and are excluded (stats reset after them).  Returns
    the server's statistics of the rest and the offered points per second."""
    import threading
    from paper_2107_02671_gb300 import nnfft as B
    P = SERVE_MAXP
    gaps = rng.exponential(1.0 / rate, n)
    kind = rng.random(n) < 0.7                       # True: NNFFT
    lN, lM = np.log([64, 16384]), np.log([1e3, 4e6])
    Ns = np.rint(np.exp(rng.uniform(*lN, n))).astype(np.int64)
    M1 = np.rint(np.exp(rng.uniform(*lM, n))).astype(np.int64)
    M2 = np.rint(np.exp(rng.uniform(*lM, n))).astype(np.int64)
    tols = rng.choice([1e-5, 1e-9, 1e-12], n)
    ids, lat = [], []
    done = threading.Event()

    def waiter():
        k = 0
        while k < n:
            if k < len(ids):
                lat.append(S.wait(ids[k]))
                k += 1
            elif done.is_set() and k >= len(ids):
                break
            else:
                time.sleep(0.0002)

    th = threading.Thread(target=waiter)
    th.start()
    t_next = time.perf_counter()
    t_start = t_next
    if warm == 0:
        S.stats(reset=True)
    for i in range(n):
        if warm and i == warm:
            while len(lat) < warm:                    # drain the warm-up, then restart the clock
                time.sleep(0.001)
            S.stats(reset=True)
            t_next = time.perf_counter()
            t_start = t_next
        t_next += gaps[i]
        while time.perf_counter() < t_next:
            pass
        m1, m2, N = int(M1[i]), int(M2[i]), int(Ns[i])
        o1, o2 = int(rng.integers(0, P - m1 + 1)), int(rng.integers(0, P - m2 + 1))
        v, x = pools["nodes"][o1:o1 + m1], pools["nodes"][o2:o2 + m2]
        dt, _ = B.tolerance_params(tols[i])
        buf = pools["out"][i % len(pools["out"])]
        if kind[i]:
            f = (pools["c128"] if dt == B.NNFFT_C128 else pools["c64"])[o1:o1 + m1]
            ids.append(S.submit_nnfft(N, v, x, f, buf.view(f.dtype)[:m2], tols[i]))
        else:
            c = (pools["r64"] if dt == B.NNFFT_C128 else pools["r32"])[o1:o1 + m1]
            ids.append(S.submit_sinc(min(N, 16384), v, c, x, buf.view(c.dtype)[:m2], tols[i], "gl"))
    t_arrivals = time.perf_counter() - t_start
    done.set()
    th.join()
    offered = float(np.sum((M1 + M2)[warm:])) / max(t_arrivals, 1e-9)
    return S.stats(), offered


def _served_errors(S, rng, per_class=3):
    """Error against the oracle per tolerance class: per class `per_class` NNFFT requests
    and one sinc request of the served mix's size distribution (M capped at 2e5 so that the
    oracle finishes), 48 sampled rows each; max |error| / 1-norm of the inputs."""
    import oracle
    from paper_2107_02671_gb300 import nnfft as B
    from paper_2107_02671_gb300 import workloads as W
    lN, lM = np.log([64, 16384]), np.log([1e3, 2e5])
    out = {}
    for tol in (1e-5, 1e-9, 1e-12):
        dt, _ = B.tolerance_params(tol)
        worst = 0.0
        for k in range(per_class + 1):
            N = int(np.rint(np.exp(rng.uniform(*lN))))
            m1, m2 = (int(np.rint(np.exp(rng.uniform(*lM)))) for _ in range(2))
            v, x = rng.uniform(-0.5, 0.5, m1), rng.uniform(-0.5, 0.5, m2)
            rows = W.sample_rows(m2, 48, k)
            if k < per_class:
                f = W.draw_complex(rng, m1, np.complex128 if dt == B.NNFFT_C128 else np.complex64)
                y = np.zeros(m2, f.dtype)
                S.wait(S.submit_nnfft(N, v, x, f, y, tol))
                want = oracle.nnfft_direct(N, v, f.astype(np.complex128), x, rows=rows)
            else:
                f = rng.standard_normal(m1).astype(np.float64 if dt == B.NNFFT_C128 else np.float32)
                y = np.zeros(m2, f.dtype)
                S.wait(S.submit_sinc(N, v, f, x, y, tol, "gl"))
                want = oracle.sinc_direct(N, v, f.astype(np.complex128), x, rows=rows)
            err = float(np.max(np.abs(y[rows].astype(np.complex128) - want)) / np.sum(np.abs(f)))
            worst = max(worst, err)
        out[f"{tol:g}"] = worst
    return out


def run_served(args, rank):
    """The served mixed stream: Poisson arrivals at 2000 requests/s, 70% NNFFT and 30% sinc
    transform, N log-uniform in [64, 16384], M1 and M2 log-uniform in [1e3, 4e6], tolerance
    drawn from {1e-5, 1e-9, 1e-12}, 64 GB device budget, 4 slots, 10^5 timed requests.  Host
    inputs are slices of pinned pools (synthetic uniform nodes, N(0,1) values).  The first
    SERVE_WARM requests fill the plan cache and are not counted; latency is submit ->
    completion.  Then a capacity sweep at higher offered rates and the error of sampled
    requests of each tolerance class against the oracle."""
    from paper_2107_02671_gb300 import nnfft as B
    rng = np.random.default_rng(42 + rank)
    pools = _serve_pools(rng)
    S = B.Server(mem_budget_bytes=64 << 30, slots=4, max_points=SERVE_MAXP)
    n_timed = args.serve_requests
    st, offered = _serve_stream(S, pools, rng, SERVE_WARM + n_timed, SERVE_RATE, SERVE_WARM)
    sweep = []
    for rate in SERVE_SWEEP:
        s2, off2 = _serve_stream(S, pools, rng, SERVE_SWEEP_N, rate, 0)
        sweep.append({"offered_rate_per_s": rate, "offered_pts_per_s": off2,
                      "completed_pts_per_s": s2["points"] / s2["seconds"] if s2["seconds"] > 0 else None,
                      "p50_ms": s2["p50_ms"], "p99_ms": s2["p99_ms"], "requests": SERVE_SWEEP_N})
    errs = None
    if rank == 0:
        try:
            errs = _served_errors(S, rng)
        except Exception as e:   # reported; the tests enforce the tolerances
            errs = {"error": f"{type(e).__name__}: {e}"}
    S.close()
    return {"requests_timed": n_timed, "requests_warmup": SERVE_WARM, "arrival_rate_per_s": SERVE_RATE,
            "mix": "70% NNFFT / 30% sinc (GL), N in [64, 16384], M in [1e3, 4e6], tol {1e-5, 1e-9, 1e-12}",
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
            "pts_per_s": st["points"] / st["seconds"] if st["seconds"] > 0 else None,
            "offered_pts_per_s": offered,
            "completed": st["completed"], "failed": st["failed"], "plans_cached": st["plans_cached"],
            "plans_made": st["plans_made"], "plans_evicted": st["plans_evicted"],
            "device_gb": st["device_bytes"] / 2**30, "slots": 4, "budget_gb": 64,
            "capacity_sweep": sweep,
            "capacity_note": "completed points/s at rising offered rates (4000 requests each, no "
                             "warm-up, plans already cached): where it stops following the "
                             "offered load, the loop is at capacity",
            "max_rel_err_by_tolerance": errs,
            "max_rel_err_note": "per class: 3 NNFFT + 1 sinc request of the mix (M <= 2e5), 48 "
                                "sampled rows each against the oracle's direct sums"}


def whole_job_value(total_ms, steps, pts_step, world, device="cpu"):
    """Replicas: every rank times its own copy of the workload; the job's time is the
    maximum over ranks and its throughput counts the points of all ranks."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps * pts_step / (total_ms / 1e3)


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2107_02671_gb300 import nnfft as B
    from paper_2107_02671_gb300 import workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    B.load_library()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    # ---- headline workload -----------------------------------------------------------------
    v, x, f = W.nnfft_inputs(M_PTS, M_PTS, rank)
    g = W.adjoint_inputs(M_PTS, rank)
    vd, xd, fd, gd = to_dev(v), to_dev(x), to_dev(f), to_dev(g)
    y = torch.empty(M_PTS, dtype=torch.complex128, device=dev)
    z = torch.empty(M_PTS, dtype=torch.complex128, device=dev)
    torch.cuda.synchronize()
    t_plan0 = time.perf_counter()
    plan = B.Plan(N_BW, M_PTS, M_PTS, 2.0, 2.0, 8, 8, dtype=torch.complex128)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t_plan0)
    info = plan.info

    def step(p=plan, vv=vd, xx=xd, ff=fd, gg=gd, yy=y, zz=z):
        # new nodes, forward and adjoint in one call: the two sorts and the two directions
        # overlap (each direction waits for the other side's sort only before its gather)
        p.transform(vv, xx, ff, gg, yy, zz)

    def timed(stepfn, k, pl=None, flush_l2=True, label="timed"):
        """Per-step CUDA-event timing on the plan stream, L2 flushed between steps.  The
        region is an NVTX range named `label`, so a profiler can filter on it."""
        evs = []
        torch.cuda.synchronize()
        barrier()
        if pl is not None:
            pl.timing(True)
            pl.timing_read(reset=True)
        l0 = B.launch_count()
        nvtx_push(label)
        for _ in range(k):
            if flush_l2:
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stepfn()
            b.record(stream)
            evs.append((a, b))
        nvtx_pop()
        torch.cuda.synchronize()
        launches = B.launch_count() - l0
        barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        stages = None
        if pl is not None:
            stages = pl.timing_read(reset=True)
            pl.timing(False)
        return ms, launches, stages

    if args.only_served:
        res = run_served(args, rank)
        if rank == 0:
            print(json.dumps({"section": "served", **res}))
        return 0
    if args.only_batched:      # the batched workload alone (profiling runs)
        pk, _ = peaks()
        res = run_batched(args, rank, dev, flush, timed, pk)
        if rank == 0:
            print(json.dumps({"section": "batched", **res}))
        return 0

    # kernel variants picked by the library's autotuner on this node set (outside timing)
    if args.tuning:              # a configuration kept from an earlier run (profiling runs)
        plan.set_tuning(*args.tuning)
        tuning = plan.tuning()
    else:
        tuning = plan.autotune(fd, gd, y, z, reps=3, v=vd, x=xd, flush_l2=True)
    # the step as one CUDA graph launch: nnfft_transform captured once over these buffers
    # (both node sorts, forward and adjoint on two streams), replayed every step
    graph = None if args.no_graph else plan.transform_graph(vd, xd, fd, gd, y, z)

    def step_graph(gr=graph):
        gr.launch()

    main_step = step if graph is None else step_graph
    for _ in range(args.warmup):
        main_step()
    torch.cuda.synchronize()
    plan.sync()
    with ClockSampler(local) as clk:
        ms, launches, _ = timed(main_step, args.steps, None, label="headline")
    plan.sync()
    pts_step = 2 * (M_PTS + M_PTS)
    # the same step launched kernel by kernel on the plan's two streams (and its
    # per-stage times with the directions overlapping)
    for _ in range(3):
        step()
    ms_str, _, stages = timed(step, max(3, args.steps // 2), plan, label="headline_streams")
    plan.sync()
    total_ms, value = whole_job_value(float(np.sum(ms)), args.steps, pts_step, world, dev)

    # ---- accuracy on sampled rows (rank 0) --------------------------------------------------
    acc = None
    if rank == 0:
        try:
            import oracle
            rows = W.sample_rows(M_PTS, 16, 99)
            yh = y.cpu().numpy()
            ex = oracle.nnfft_direct(N_BW, v, f, x, rows=rows)
            acc = float(np.max(np.abs(yh[rows] - ex)) / np.sum(np.abs(f)))
        except Exception as e:  # accuracy is reported, the tests enforce it
            acc = f"unavailable: {e}"

    # ---- roofline of the dominant kernel ----------------------------------------------------
    # In the step the forward and the adjoint run concurrently, so their kernels share the
    # GPU and each launch lasts longer than alone.  The kernel roofline is taken from a
    # second timed region of the same step with the two directions issued one after the
    # other (set_nodes, exec, adjoint; L2 flushed between steps, CUDA events per stage).
    def step_seq(p=plan, vv=vd, xx=xd, ff=fd, gg=gd, yy=y, zz=z):
        p.set_nodes(vv, xx)
        p.exec(ff, yy)
        p.adjoint(gg, zz)
    ms_seq, _, stages_seq = timed(step_seq, max(3, args.steps // 2), plan, label="headline_seq")
    plan.sync()
    stage_ms = {k: (tot / max(n, 1), n) for k, (tot, n) in stages_seq.items() if n}
    # dominant single kernel: the node stages (binning + radix sort) and the FFT are several
    # kernels each, every other stage is one kernel
    single = {k: v_ for k, v_ in stage_ms.items() if not k.startswith("nodes_") and not k.endswith("_fft")}
    dom = max(single, key=lambda k: single[k][0] * single[k][1])
    avg_ms = stage_ms[dom][0]
    pk, pk_kind = peaks()
    D1, D2, K1 = info["D1"], info["D2"], info["K1"]
    ncell1, ncell2 = info["ncell1"], info["ncell2"]
    # the split-precision kernels are bound by FP32 instruction issue, not by HBM (ncu: FMA
    # pipe 42 %, issue 56 %, DRAM 16 % in the moments kernel), so the roofline is taken
    # against the FP32 lane-operation peak with the HBM fraction alongside
    units = {"fwd_spread_conv": K1, "adj_spread_conv": ncell2 + 15, "adj_gather_conv": ncell1,
             "fwd_gather_conv": ncell2}
    gbs = 24 * M_PTS / (avg_ms / 1e3) / 1e9
    if dom in units:
        kind, n_units, D_ = "conv", units[dom], (D1 if dom in ("fwd_spread_conv", "adj_gather_conv") else D2)
        traffic, tnote = None, "grid kernel: no capture"
    else:
        kind, n_units = ("moments" if dom.endswith("_moments") else "eval"), M_PTS
        D_ = D1 if dom in ("fwd_moments", "adj_eval") else D2
        traffic, tnote = ncu_traffic(dom, tuning)
    ops = df_ops(kind, D_) * n_units
    alu_achieved = ops / (avg_ms / 1e3) / 1e12
    # The roofline is the HBM one: the dominant kernel's algorithmic bytes (24 B per point for
    # a point kernel: 8 B node + 16 B complex128 value) over its event-timed duration, against
    # the measured copy bandwidth.  The split-precision kernels are in fact bound by FP32
    # instruction issue (ncu: FMA pipe ~40 %, DRAM ~15 %), so the FP32 lane-operation view
    # is reported beside it under "alu".
    alg_bytes = 24 * M_PTS if kind != "conv" else None
    roof = {"bound": "hbm", "kernel": dom, "achieved": gbs if alg_bytes else None,
            "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": (gbs / pk["hbm_gbs"]) if alg_bytes else None, "traffic": traffic,
            "traffic_source": tnote, "algorithmic_bytes_per_launch": alg_bytes,
            "bytes_per_unit": 24, "units_per_launch": M_PTS,
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({pk_kind})",
            "alu": {"achieved": alu_achieved, "peak": FP32_LANE_TOPS, "unit": "Tops/s",
                    "frac": alu_achieved / FP32_LANE_TOPS, "algorithmic_ops_per_launch": ops,
                    "ops_per_unit": df_ops(kind, D_),
                    "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz: FP32/INT32 lane "
                                   "operations (an FMA counts once); the double-float arithmetic "
                                   "of the split-precision kernels runs there (FP64 pipe idle)"}}
    roof["stage_ms_per_launch"] = avg_ms
    roof["measured_in"] = ("sequential pass of the step (exec, then adjoint), "
                           f"{float(np.mean(ms_seq)):.4f} ms per step; CUDA events on the plan "
                           "stream around each stage, averaged over the timed steps")

    extra = {}
    # the critical path in parts: graphs of the node sorts alone, of the sorts with one
    # direction, and of the whole step (the same calls, fewer inputs), L2 flushed before each
    parts = {}
    if graph is not None:
        for pname, pargs in (("sorts", (vd, xd)), ("sorts_forward", (vd, xd, fd, None, y, None)),
                             ("sorts_adjoint", (vd, xd, None, gd, None, z)),
                             ("step", (vd, xd, fd, gd, y, z))):
            gp = plan.transform_graph(*pargs)
            for _ in range(3):
                gp.launch()
            plan.sync()
            msp, _, _ = timed(gp.launch, max(10, args.steps), label="graph_part")
            plan.sync()
            gp.close()
            parts[pname] = round(1e3 * float(np.median(msp)), 1)
        parts["what"] = ("median us of a CUDA graph of nnfft_transform with both node sets and: no "
                         "values (sorts only), f only, g only, both (the step)")
        extra["graph_parts_us"] = parts
    extra["stream_launched"] = {"value": pts_step / (np.mean(ms_str) / 1e3), "unit": "pts/s",
                                "ms_per_step": float(np.mean(ms_str)),
                                "what": "the headline step launched kernel by kernel (nnfft_transform "
                                        "on the plan's two streams) instead of one graph launch"}
    # ---- exec-only with a resident plan (fp64) ------------------------------------------------
    def fwd_adj():
        plan.exec_adjoint(fd, gd, y, z)
    ms_e, _, _ = timed(fwd_adj, max(3, args.steps // 2))
    extra["exec_only_fp64"] = {"value": pts_step / (np.mean(ms_e) / 1e3), "unit": "pts/s",
                               "ms_per_step": float(np.mean(ms_e)),
                               "median_ms": float(np.median(ms_e)), "runs": len(ms_e),
                               "what": "forward + adjoint with resident plan (nodes already set)"}
    extra["plan_ms"] = {"value": plan_ms,
                        "what": "nnfft_plan wall time for this workload (parameters, window fits, "
                                "tables, device buffers; host + device, before any transform; the "
                                "process's first plan, so it includes one-time kernel set-up)"}

    # ---- evaluation kernels side by side: flat, flat with TMA-staged cell tiles, 32-lane ----
    # (the sequential pass's per-stage event times; the other tuning choices kept)
    tune_keys = ("moments_lanes_v", "moments_lanes_x", "fft_variant", "item_split",
                 "eval_lanes_v", "eval_lanes_x", "item_cap", "sort_lsd")
    base_t = {k: tuning[k] for k in tune_keys if k in tuning}
    ab = {}
    for name, el in (("flat", 1), ("flat_tma", 2), ("lanes32", 32)):
        plan.set_tuning(**{**base_t, "eval_lanes_v": el, "eval_lanes_x": el})
        for _ in range(2):
            step_seq()
        _, _, st_ab = timed(step_seq, max(3, args.steps // 4), plan, label=f"eval_{name}")
        plan.sync()
        ab[name] = {k: round(1e3 * tot / n, 2) for k, (tot, n) in st_ab.items()
                    if n and k in ("fwd_eval", "adj_eval")}
    plan.set_tuning(**base_t)
    extra["eval_kernels_us"] = {**ab, "what": "per-launch device time (us) of the gather "
                                               "evaluation at the headline size: one thread per "
                                               "point, the same with each block's cell window "
                                               "sums staged in shared memory by one TMA bulk "
                                               "copy, one warp per work item"}

    # ---- Chebyshev nodes (fp64) ----------------------------------------------------------------
    vc, xc, _ = W.nnfft_inputs(M_PTS, M_PTS, rank, nodes="chebyshev")
    vcd, xcd = to_dev(vc), to_dev(xc)
    step_c = lambda: step(vv=vcd, xx=xcd)   # noqa: E731
    step_c(); torch.cuda.synchronize()
    ms_c, _, _ = timed(step_c, max(3, args.steps // 2))
    plan.sync()
    extra["chebyshev_fp64"] = {"value": pts_step / (np.mean(ms_c) / 1e3), "unit": "pts/s",
                               "ms_per_step": float(np.mean(ms_c))}
    del vcd, xcd

    # ---- all-FP64 arithmetic (m = 8): the same plan with every operation in FP64 ----------------
    plan.set_arith(B.ARITH_FP64)
    for _ in range(2):
        step()
    plan.sync()
    ms64, _, _ = timed(step, max(3, args.steps // 4))
    plan.sync()
    acc64 = None
    if rank == 0:
        try:
            import oracle
            rows = W.sample_rows(M_PTS, 16, 98)
            ex = oracle.nnfft_direct(N_BW, v, f, x, rows=rows)
            acc64 = float(np.max(np.abs(y.cpu().numpy()[rows] - ex)) / np.sum(np.abs(f)))
        except Exception as e:
            acc64 = f"unavailable: {e}"
    extra["fp64_all_fp64_m8"] = {
        "value": pts_step / (np.mean(ms64) / 1e3), "unit": "pts/s",
        "ms_per_step": float(np.mean(ms64)), "max_rel_err_sampled": acc64,
        "what": "the headline step (kernel by kernel) with nnfft_set_arith(NNFFT_ARITH_FP64): "
                "every point- and grid-kernel operation in FP64 instead of the split "
                "double-float/FP32 arithmetic"}
    plan.set_arith(B.ARITH_FP64_SPLIT)
    plan.set_tuning(**{k: tuning[k] for k in ("moments_lanes_v", "moments_lanes_x", "fft_variant",
                                              "item_split", "eval_lanes_v", "eval_lanes_x",
                                              "item_cap", "sort_lsd") if k in tuning})

    # ---- fp32 path (m = 4) -------------------------------------------------------------------
    f32 = fd.to(torch.complex64)
    g32 = gd.to(torch.complex64)
    y32 = torch.empty(M_PTS, dtype=torch.complex64, device=dev)
    z32 = torch.empty(M_PTS, dtype=torch.complex64, device=dev)
    plan32 = B.Plan(N_BW, M_PTS, M_PTS, 2.0, 2.0, 4, 4, dtype=torch.complex64)
    tuning32 = plan32.autotune(f32, g32, y32, z32, reps=3, v=vd, x=xd, flush_l2=True)
    step32 = lambda: step(p=plan32, ff=f32, gg=g32, yy=y32, zz=z32)   # noqa: E731
    for _ in range(2):
        step32()
    # per-stage times from the kernel-by-kernel step, the rate from the same step as one
    # CUDA graph launch (as the headline)
    _, _, st32 = timed(step32, max(3, args.steps // 4), plan32)
    plan32.sync()
    graph32 = plan32.transform_graph(vd, xd, f32, g32, y32, z32)
    for _ in range(3):
        graph32.launch()
    ms32, _, _ = timed(graph32.launch, max(3, args.steps // 2))
    plan32.sync()
    graph32.close()
    st32ms = {k: tot / max(n, 1) for k, (tot, n) in st32.items() if n}
    hbm32 = {}
    for kname, nbytes in (("fwd_moments", 16 * M_PTS), ("fwd_eval", 16 * M_PTS),
                          ("adj_moments", 16 * M_PTS), ("adj_eval", 16 * M_PTS)):
        if kname in st32ms:
            gbs = nbytes / (st32ms[kname] / 1e3) / 1e9
            hbm32[kname] = {"ms": st32ms[kname], "achieved_gbs": gbs,
                            "frac": gbs / pk["hbm_gbs"]}
    extra["fp32_m4"] = {"value": pts_step / (np.mean(ms32) / 1e3), "unit": "pts/s",
                        "ms_per_step": float(np.mean(ms32)), "D": plan32.info["D1"],
                        "stage_ms": st32ms, "hbm_roofline_point_kernels": hbm32,
                        "tuning": tuning32,
                        "algorithmic_bytes_per_point": 16}
    del plan32

    # ---- the same transform at larger M: the point kernels' HBM fraction as cells fill ----
    if not args.no_m_sweep:
        extra["m_sweep"] = run_m_sweep(args, rank, dev, flush, timed, pk)

    # ---- batched workload: 512 instances, M1, M2 log-uniform in [1e3, 1e6], N in [64, 8192] ----
    if not args.no_batch:
        extra["batched"] = run_batched(args, rank, dev, flush, timed, pk)

    # ---- served mixed stream (request loop) --------------------------------------------------
    if not args.no_serve and rank == 0:
        try:
            extra["served"] = run_served(args, rank)
        except Exception as e:   # reported, the tests enforce correctness
            extra["served"] = {"error": f"{type(e).__name__}: {e}"}

    # ---- fast sinc transform (config N=1024, L1=L2=2^18) ----------------------------------------
    a, c, bb = W.sinc_inputs(SINC_L, SINC_L, rank)
    ad, cd, bd = to_dev(a), to_dev(c), to_dev(bb)
    hd = torch.empty(SINC_L, dtype=torch.float64, device=dev)
    cd32 = cd.to(torch.float32)
    hd32 = torch.empty(SINC_L, dtype=torch.float32, device=dev)
    for name, cc, hh, m, rule in (("sinc_fp64_m8", cd, hd, 8, "gl"), ("sinc_fp32_m4", cd32, hd32, 4, "gl"),
                                  ("sinc_cc_fp64_m8", cd, hd, 8, "cc"),
                                  ("sinc_cc_fp32_m4", cd32, hd32, 4, "cc")):
        fn = lambda cc=cc, hh=hh, m=m, rule=rule: B.sinc(SINC_N, ad, cc, bd, m=m, out=hh, rule=rule)  # noqa: E731
        fn(); fn(); B.sinc_sync()
        ms_s, _, _ = timed(fn, max(3, args.steps // 2))
        B.sinc_sync()
        extra[name] = {"value": 2 * SINC_L / (np.mean(ms_s) / 1e3), "unit": "pts/s (L1+L2)/s",
                       "ms_per_call": float(np.mean(ms_s)),
                       "rule": "Gauss-Legendre, 2N nodes" if rule == "gl" else "Clenshaw-Curtis, n = 4N"}
    B.sinc_release()

    # ---- end to end through the host-buffer C ABI calls -----------------------------------------
    import torch as _t
    vh = _t.from_numpy(v).pin_memory().numpy()
    xh = _t.from_numpy(x).pin_memory().numpy()
    fh = _t.from_numpy(f).pin_memory().numpy()
    gh = _t.from_numpy(g).pin_memory().numpy()
    yh = _t.empty(M_PTS, dtype=_t.complex128).pin_memory().numpy()
    zh = _t.empty(M_PTS, dtype=_t.complex128).pin_memory().numpy()

    def e2e_call():
        plan.transform_host(vh, xh, fh, gh, yh, zh)
    # the same transform captured once over these page-locked buffers: one graph launch per
    # step uploads their contents, transforms and copies the results back
    hgraph = plan.transform_host_graph(vh, xh, fh, gh, yh, zh)

    def e2e_graph():
        hgraph.launch()
        plan.sync()
    k_e2e = max(3, min(args.steps, 10))

    def wall(fn):
        fn()
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            fn()
        t = (time.perf_counter() - t0) / k_e2e
        if world > 1:
            tt = torch.tensor([t], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        return t
    t_call = wall(e2e_call)
    t_e2e = wall(e2e_graph)
    hgraph.close()
    # two transforms in flight: a second plan with its own page-locked buffers; step i waits
    # only for step i - 2 before its graph launch, so one step's downloads overlap the next
    # step's uploads and transform (the two link directions run concurrently)
    pipe = None
    try:
        # on a stream of its own (the headline plan runs on the current stream)
        plan2 = B.Plan(N_BW, M_PTS, M_PTS, 2.0, 2.0, 8, 8, dtype=torch.complex128,
                       stream=torch.cuda.Stream(device=dev))
        t0v = plan.tuning()
        plan2.set_tuning(t0v["moments_lanes_v"], t0v["moments_lanes_x"], t0v["fft_variant"],
                         t0v["item_split"], t0v["eval_lanes_v"], t0v["eval_lanes_x"],
                         t0v["item_cap"], t0v["sort_lsd"])
        pin = lambda a: _t.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        vh2, xh2, fh2, gh2 = pin(v), pin(x), pin(f), pin(g)
        yh2 = _t.empty(M_PTS, dtype=_t.complex128).pin_memory().numpy()
        zh2 = _t.empty(M_PTS, dtype=_t.complex128).pin_memory().numpy()
        graphs = [(plan, plan.transform_host_graph(vh, xh, fh, gh, yh, zh)),
                  (plan2, plan2.transform_host_graph(vh2, xh2, fh2, gh2, yh2, zh2))]
        for pl, gr in graphs:                            # warm-up
            gr.launch()
            pl.sync()
        kp = 4 * k_e2e
        barrier()
        t0 = time.perf_counter()
        for i in range(kp):
            pl, gr = graphs[i % 2]
            if i >= 2:
                pl.sync()                                # step i - 2's results are on the host
            gr.launch()
        for pl, _ in graphs:
            pl.sync()
        tp = (time.perf_counter() - t0) / kp
        if world > 1:
            tt = torch.tensor([tp], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            tp = float(tt.item())
        pipe = world * pts_step / tp
        for _, gr in graphs:
            gr.close()
        plan2.close()
        del plan2
    except Exception as e:          # reported, not fatal
        pipe = f"unavailable: {type(e).__name__}: {e}"
    e2e = {"value": world * pts_step / t_e2e, "unit": "pts/s",
           "h2d_bytes_per_step": int(vh.nbytes + xh.nbytes + fh.nbytes + gh.nbytes),
           "d2h_bytes_per_step": int(yh.nbytes + zh.nbytes),
           "what": "nnfft_transform_host_graph launch + nnfft_sync per step (new nodes, forward "
                   "and adjoint) from pinned host buffers: uploads in need order overlapped with "
                   "the node sort, results copied back, wall clock",
           "per_call_value": world * pts_step / t_call,
           "per_call_what": "nnfft_transform_host per step (the same work issued call by call)",
           "pipelined_value": pipe,
           "pipelined_what": ("the same graph steps with two transforms in flight (two plans, "
                              "two sets of page-locked buffers; step i waits for step i-2's "
                              "results before its launch): a stream of independent transforms "
                              "from host memory, every step's copies inside the timed region")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample()
        try:
            cpu["stage_reference"] = oracle_stage_reference()
        except Exception as e:   # reported, not fatal
            cpu["stage_reference"] = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_BW, "M1": M_PTS, "M2": M_PTS, "m": 8,
                       "sigma": 2.0, "nodes": "uniform", "points_per_step": pts_step,
                       "l2": "flushed between timed steps (512 MB device write, outside the events)",
                       "launch": ("kernel by kernel on two streams" if graph is None else
                                  f"one CUDA graph launch per step ({graph.kernels} kernels)"),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "plan": {k: info[k] for k in ("N1", "K1", "N2", "D1", "D2", "fft_n1",
                                                     "fft_n2")}},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "tuning": tuning,
            "stage_ms": {k: v_[0] for k, v_ in stage_ms.items()},
            "stage_ms_note": "per-stage device time of the sequential pass; the timed step runs "
                             "forward and adjoint concurrently (stage_ms_concurrent)",
            "stage_ms_concurrent": {k: tot / n for k, (tot, n) in stages.items() if n},
            "max_rel_err_sampled": acc,
            "peaks_source": pk_kind,
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-m-sweep", action="store_true",
                    help="skip the fp64 transform at M = 2^22, 2^24, 2^26")
    ap.add_argument("--no-graph", action="store_true",
                    help="headline step launched kernel by kernel instead of as one CUDA graph")
    ap.add_argument("--tuning", type=lambda t: [int(u) for u in t.split(",")], default=None,
                    help="headline kernel variants instead of autotuning: moments lanes v,x, "
                         "fft variant, item split, evaluation lanes v,x[, item cap[, sort_lsd]] "
                         "(e.g. 8,8,0,0,1,1,64)")
    ap.add_argument("--no-serve", action="store_true", help="skip the served mixed stream")
    ap.add_argument("--only-served", action="store_true",
                    help="run only the served mixed stream and print its numbers")
    ap.add_argument("--serve-requests", type=int, default=SERVE_TIMED,
                    help="timed requests of the served stream (10^5)")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT,
                    help="instances of the batched workload (512; fewer for profiling runs)")
    ap.add_argument("--only-fp32-batch", action="store_true",
                    help="batched workload at fp32 only (profiling runs)")
    ap.add_argument("--only-batched", action="store_true",
                    help="run only the batched workload and print its numbers (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the X stage (cross-multiply-accumulate) on GB300.

Workload (the streamed real-time correlator): 64 inputs (32 dual-pol antennas), 768
channels, 1000 samples per dump, 200 dumps, complex 8-bit Gaussian samples (sigma 16,
clipped to +-127) with a common correlated component rho = 0.1, generated on the device
from a seeded generator.  One step = the whole job: all 200 dumps through the library's
X stage (fused unpack + tensor-core cross-multiply-accumulate + int64 dump), one launch.

Printed on rank 0 as one JSON line:
  value        TeraCMAC/s of the whole job, inputs resident in HBM, device-timed
  e2e          same metric through the C ABI with host (pinned) buffers: H2D of the packed
               samples and D2H of the visibilities inside the timed region
  fp32_path    the CUDA-core FP32 engine on the same job, and value / fp32 value
  roofline     the dominant kernel against measured HBM bandwidth
  cpu_baseline the CPU oracle on a bounded sample of the same workload
Options: --gpus N (torchrun, one rank per GPU, weak scaling: every rank runs the whole
job on its own GPU), --steps K, --warmup W, --impl reference (the CPU oracle arm).

Other workloads (--workload; each prints its own JSON line):
  large   1024 inputs (512 dual-pol antennas) x 1536 channels x 256 samples, 20 dumps
          per step, 8-bit Gaussian sigma 8; one launch per dump into a 2-dump output ring
  batch   40 uneven jobs (8 each of 16/32/64/128/256 dual-pol antennas, 64..1024
          channels, 128..2048 samples) in one persistent launch, autotuned, CUDA graph
  serve   Poisson arrivals (mean 200 jobs/s) tagged over 8 streams, each job a random
          array of 32..512 dual-pol antennas, 128..1536 channels, 256..1024 samples, 4 or
          8 bits; p50/p99 latency, real-time factor, TeraCMAC/s
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

N_INPUTS, N_CHAN, N_TIME, N_DUMPS, BITS = 64, 768, 1000, 200, 8
SIGMA, RHO, SEED = 16.0, 0.1, 2000
CHANNEL_RATE_HZ = 1.28e6 / 128.0
WORKLOAD = "stream64_8bit: 64 inputs x 768 channels x 1000 samples/dump x 200 dumps, 8-bit complex Gaussian sigma=16 rho=0.1"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per dump of the fused kernel on this
# workload, from one ncu capture of an 8-dump launch (786.6 MB read + 177.0 MB written), scaled
# by dumps; set to None whenever the kernel changes until it is captured again.
DRAM_BYTES_PER_DUMP = (786.616576e6 + 177.040384e6) / 8


def rank_max(x: float, dist, device) -> float:
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_tera_cmac(cmac_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank runs its own job (weak scaling); the slowest rank's
    time counts for all."""
    return cmac_per_rank * world / (ms_max / 1e3) / 1e12


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(target_s: float = 12.0):
    """The C oracle (OpenMP over the host's cores) on a bounded sample of the workload:
    repeated passes over one full 768-channel dump until about target_s seconds."""
    import oracle
    from paper_0906_1887_gb300 import synth
    re, im = synth.correlated_gaussian(SEED, N_TIME, N_CHAN, N_INPUTS, SIGMA, RHO, 127)
    packed = synth.pack(re, im, BITS)
    del re, im
    threads = oracle.threads_used(0)
    t0 = time.perf_counter()
    oracle.xcorr_int(packed, N_INPUTS, N_CHAN, N_TIME, BITS)
    one = time.perf_counter() - t0
    reps = max(1, int(target_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.xcorr_int(packed, N_INPUTS, N_CHAN, N_TIME, BITS)
    dt = time.perf_counter() - t0
    cm = N_INPUTS * (N_INPUTS + 1) // 2 * N_CHAN * N_TIME * reps
    # one thread, as the paper's CPU comparison ran (Sec. 5): a channel subset, about 3 s
    n_sel = 32
    chans = list(range(0, N_CHAN, N_CHAN // n_sel))[:n_sel]
    t0 = time.perf_counter()
    oracle.xcorr_int(packed, N_INPUTS, N_CHAN, N_TIME, BITS, chans=chans, n_threads=1)
    one1 = time.perf_counter() - t0
    reps1 = max(1, int(3.0 / max(one1, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(reps1):
        oracle.xcorr_int(packed, N_INPUTS, N_CHAN, N_TIME, BITS, chans=chans, n_threads=1)
    dt1 = time.perf_counter() - t0
    cm1 = N_INPUTS * (N_INPUTS + 1) // 2 * n_sel * N_TIME * reps1
    return {"value": cm / dt / 1e12, "unit": "TeraCMAC/s", "cores": threads, "kind": "oracle",
            "sample": f"{reps} passes over one full dump (64 inputs x 768 channels x 1000 samples, 8-bit, "
                      f"numpy PCG64 seed {SEED})", "seconds": dt,
            "single_thread": {"value": cm1 / dt1 / 1e12, "unit": "TeraCMAC/s", "cores": 1, "seconds": dt1,
                              "sample": f"{reps1} passes over {n_sel} of the dump's 768 channels"}}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_0906_1887_gb300 import synth
    re, im = synth.correlated_gaussian(SEED, N_TIME, 64, N_INPUTS, SIGMA, RHO, 127)
    packed = synth.pack(re, im, BITS)
    chans = np.arange(64, dtype=np.int32)        # a bounded sample of the job per step
    threads = oracle.threads_used(0)
    for _ in range(args.warmup):
        oracle.xcorr_int(packed, N_INPUTS, 64, N_TIME, BITS, chans=chans[:2])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.xcorr_int(packed, N_INPUTS, 64, N_TIME, BITS, chans=chans)
    dt = (time.perf_counter() - t0) / args.steps
    cm = N_INPUTS * (N_INPUTS + 1) // 2 * len(chans) * N_TIME
    v = cm / dt / 1e12
    line = {"metric": "X-engine TeraCMAC/s", "value": v, "unit": "TeraCMAC/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_per_step": "64 channels of one dump"},
            "cpu_baseline": {"value": v, "unit": "TeraCMAC/s", "cores": threads, "kind": "oracle",
                             "sample": "64 of 768 channels of one 1000-sample dump per step"},
            "e2e": {"value": v, "unit": "TeraCMAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- secondary workloads (--workload large | batch | serve) ----

def run_large(args):
    import torch

    from paper_0906_1887_gb300 import corr, synth
    n, c, t, d = 1024, args.large_chans, 256, 20
    if c != 1536:   # a reduced case for profiling captures: one dump
        d = 1
    dev = torch.device("cuda", 0)
    plan = corr.Plan(n, c, t, 8)
    P = plan.n_baselines
    packed = synth.torch_correlated_gaussian_packed8(d, t, c, n, 8.0, 0.0, 3000, dev)   # 16.1 GB
    per_dump = t * c * n * 2
    vis = [plan.empty_vis(1, dev) for _ in range(2)]                                  # 2 x 12.9 GB ring
    stream = torch.cuda.current_stream(dev)

    def step():
        for k in range(d):
            plan.run(packed[k], vis[k & 1], None, engine=corr.ENGINE_TC, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[-1]) / args.steps
    cm = P * c * t * d
    # one-dump launch times for the roofline
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.run(packed[0], vis[0], None, engine=corr.ENGINE_TC, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_one = e0.elapsed_time(e1)
    # the X stage with the dump step fused into its epilogue: float32 averaged, phase-corrected
    # visibilities (8 bytes per baseline) instead of the exact int64 sums, then the separate
    # dump step over int64 sums for comparison
    g = torch.Generator(device=dev)
    g.manual_seed(6001)
    tau = torch.randn(n, generator=g, dtype=torch.float64, device=dev) * 1e-6
    nu = 1.5e8 + 1e4 * torch.arange(c, dtype=torch.float64, device=dev)
    dws = torch.empty(plan.dump_workspace_size(), dtype=torch.uint8, device=dev)
    outf = torch.empty((c, P, 2), dtype=torch.float32, device=dev)
    plan.run_dump(packed[0], outf, 1, tau, nu, dws, stream=stream)
    e0.record(stream)
    for k in range(d):
        plan.run_dump(packed[k], outf, 1, tau, nu, dws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fused = e0.elapsed_time(e1) / d
    plan.dump(vis[0], outf, 1, tau, nu, dws, stream=stream)
    e0.record(stream)
    plan.dump(vis[0], outf, 1, tau, nu, dws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_dump = e0.elapsed_time(e1)
    del outf
    # FP32 engine on one dump
    ws = plan.empty_workspace(corr.ENGINE_FP32, 1, dev)
    plan.run(packed[0], vis[1], ws, engine=corr.ENGINE_FP32, stream=stream)
    e0.record(stream)
    plan.run(packed[0], vis[1], ws, engine=corr.ENGINE_FP32, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1)
    hbm, bf16, src = _peaks()
    out_bytes = P * c * 16
    bytes_launch = per_dump + out_bytes
    gbs = bytes_launch / (ms_one / 1e3) / 1e9
    line = {"metric": "X-engine TeraCMAC/s", "value": cm / (ms / 1e3) / 1e12, "unit": "TeraCMAC/s",
            "workload": f"large1024_8bit: 1024 inputs x {c} channels x 256 samples/dump x {d} dumps, sigma 8"
                        + ("" if c == 1536 else " (reduced for profiling)"),
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "real_time_factor": (t * d / CHANNEL_RATE_HZ) / (ms / 1e3),
            "fp32_path": {"value": P * c * t / (ms32 / 1e3) / 1e12, "ms_per_dump": ms32,
                          "speedup_tc_over_fp32": ms32 / ms_one},
            "fused_dump": {"ms_per_dump": ms_fused, "value": P * c * t / (ms_fused / 1e3) / 1e12,
                           "separate_x_plus_dump_ms": ms_one + ms_dump, "dump_step_ms": ms_dump,
                           "output": "float32 V / n_accum, phase-corrected (8 B per baseline)",
                           "achieved_gbs": (per_dump + P * c * 8) / (ms_fused / 1e3) / 1e9},
            "roofline": {"bound": "hbm", "kernel": "xeng_tc_kernel<raw8>", "achieved": gbs, "peak": hbm,
                         "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes_per_launch": bytes_launch,
                         "kernel_ms": ms_one, "tensor_tflops_algorithmic": 8.0 * P * c * t / (ms_one / 1e3) / 1e12,
                         "peak_source": src},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def _batch_jobs(rng):
    sizes = []
    for ant in (16, 32, 64, 128, 256):
        for _ in range(8):
            sizes.append((2 * ant, 64 * int(rng.integers(1, 17)), 128 * int(rng.integers(1, 17))))
    return sizes


def run_batch(args):
    import os
    import tempfile

    import torch

    from paper_0906_1887_gb300 import corr, synth
    rng = np.random.default_rng(4000)
    sizes = _batch_jobs(rng)
    dev = torch.device("cuda", 0)
    jobs, descs = [], []
    for k, (n, c, t) in enumerate(sizes):
        x = synth.torch_correlated_gaussian_packed8(1, t, c, n, 16.0, 0.0, 4000 + k, dev).reshape(-1)
        v = torch.empty((c, n * (n + 1) // 2, 2), dtype=torch.int64, device=dev)
        jobs.append((x, v))
        descs.append((n, c, t, 8, x, v))
    cm = sum(n * (n + 1) // 2 * c * t for n, c, t in sizes)
    cache = os.path.join(tempfile.gettempdir(), "corr_batch_tune.jsonl")
    t0 = time.time()
    b = corr.Batch(descs, flags=corr.BATCH_GRAPH | corr.BATCH_AUTOTUNE, tune_cache=cache)
    tune_s = time.time() - t0
    info = b.info()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        b.run(stream)
    torch.cuda.synchronize()
    assert b.check_device() == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        b.run(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the same jobs, one launch each
    plans = [corr.Plan(n, c, t, 8) for n, c, t in sizes]
    for p, (x, v) in zip(plans, jobs):
        p.run(x, v, None, engine=corr.ENGINE_TC, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for p, (x, v) in zip(plans, jobs):
            p.run(x, v, None, engine=corr.ENGINE_TC, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_each = e0.elapsed_time(e1) / args.steps
    # algorithmic bytes of the step: packed samples in (2 B per complex sample) + int64 visibilities out
    algo = sum(2 * n * c * t + 16 * (n * (n + 1) // 2) * c for n, c, t in sizes)
    hbm, bf16, src = _peaks()
    gbs = algo / (ms / 1e3) / 1e9
    tflops = 8 * cm / (ms / 1e3) / 1e12   # 4 real MACs per CMAC
    line = {"metric": "X-engine TeraCMAC/s", "value": cm / (ms / 1e3) / 1e12, "unit": "TeraCMAC/s",
            "workload": "batch40: 8 each of 16/32/64/128/256 dual-pol antennas, 64..1024 channels, "
                        "128..2048 samples, 8-bit Gaussian sigma 16, seed 4000",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "roofline": {"bound": "hbm", "kernel": "xeng_tc_kernel<raw8, job table>", "achieved": gbs,
                         "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes": algo,
                         "peak_source": src, "tensor_tflops_algorithmic": tflops,
                         "tensor_frac_of_measured_bf16_burst": tflops / bf16},
            "one_launch_per_job": {"ms_per_step": ms_each, "value": cm / (ms_each / 1e3) / 1e12},
            "batch": info, "autotune_seconds": tune_s, "cmacs_per_step": cm}
    print(json.dumps(line), flush=True)
    b.close()


def run_fx(args):
    """The paper's prototype configuration end to end on the GPU (Sec. 5, Table 3): 64 inputs of
    1.28 MHz complex 8-bit samples, F stage into 128 channels, X stage over 1 s of frames."""
    import torch

    from paper_0906_1887_gb300 import corr, synth
    n, c, frames = 64, 128, 10000   # 1.28 MHz / 128 channels = 10 k frames per second of data
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    fplan = corr.FPlan(n, c, corr.F_COMPLEX8)
    x = synth.torch_correlated_gaussian_packed8(1, frames * c, 1, n, 16.0, 0.1, 5000, dev).reshape(-1)
    spec = fplan.empty_spectra(frames, dev)
    xplan = corr.Plan(n, c, frames, 32)
    vis = xplan.empty_vis(1, dev)
    P = xplan.n_baselines
    hbm, _, src = _peaks()
    f_bytes = frames * (fplan.in_bytes_per_frame + fplan.out_bytes_per_frame)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2, written between steps

    def timed(fn, steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[2 * k].record(stream)
            fn()
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        return sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps)) / steps

    res = {}
    for name, engine in (("fp32", corr.ENGINE_FP32), ("bf16x3", corr.ENGINE_BF16X3)):
        ws = xplan.empty_workspace(engine, 1, dev)

        def step():
            fplan.run(x, spec, frames, stream=stream)
            xplan.run(spec, vis, ws, engine=engine, stream=stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        assert xplan.check_device() == 0
        res[name] = timed(step, args.steps)
        del ws
    f_ms = timed(lambda: fplan.run(x, spec, frames, stream=stream), args.steps)
    # the polyphase filterbank variant (8 taps, default prototype) on the same second of data
    taps = 8
    pplan = corr.FPlan(n, c, corr.F_COMPLEX8, n_taps=taps)
    xp = synth.torch_correlated_gaussian_packed8(1, (frames + taps - 1) * c, 1, n, 16.0, 0.1, 5001, dev).reshape(-1)
    pfb_run = lambda: pplan.run(xp, spec, frames, stream=stream)   # noqa: E731
    for _ in range(args.warmup):
        pfb_run()
    pfb_ms = timed(pfb_run, args.steps)
    pfb_bytes = (frames + taps - 1) * pplan.in_bytes_per_frame + frames * pplan.out_bytes_per_frame
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    timed(lambda: fplan.run(x, spec, frames, stream=stream), args.steps)
    clk = clocks.stop()
    ms = res["fp32"]
    cm = P * c * frames
    gbs = f_bytes / (f_ms / 1e3) / 1e9
    line = {"metric": "FX chain TeraCMAC/s (F stage + X stage, FP32 X engine)", "value": cm / (ms / 1e3) / 1e12,
            "unit": "TeraCMAC/s",
            "workload": "mwa32t_fx: 64 inputs x 1.28 MHz complex 8-bit (sigma 16, rho 0.1), 128 channels, "
                        "1 s of data per step (10000 frames), one dump",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "real_time_factor": 1000.0 / ms,
            "bf16x3_chain": {"ms_per_step": res["bf16x3"], "value": cm / (res["bf16x3"] / 1e3) / 1e12,
                             "real_time_factor": 1000.0 / res["bf16x3"]},
            "fstage": {"kernel": "fengine_kernel<complex8>", "ms": f_ms, "bound": "hbm", "achieved": gbs,
                       "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes": f_bytes,
                       "peak_source": src},
            "pfb_fstage": {"taps": taps, "ms": pfb_ms, "achieved": pfb_bytes / (pfb_ms / 1e3) / 1e9,
                           "frac": pfb_bytes / (pfb_ms / 1e3) / 1e9 / hbm, "algorithmic_bytes": pfb_bytes,
                           "note": "each input frame is read by 8 output frames (through L2); bytes counted once"},
            "paper_context": "C1060 (Table 3): unpack 53 + FFT 53 + CMAC (GP, G=4) 185 = 291 ms per second of data",
            "l2": "256 MB flush written between timed steps", "clocks": clk}
    print(json.dumps(line), flush=True)


def run_float(args):
    """The float variant of the 64-input stream workload (float32 samples, no rounding) through
    the BF16x3 tensor-core engine (bf16 hi/lo split, three products, fp32 accumulation) and the
    FP32 CUDA-core engine.  20 dumps per step: 7.9 GB of samples, larger than L2."""
    import torch

    from paper_0906_1887_gb300 import corr, synth
    n, c, t = 64, 768, 1000
    d = 20 if args.dumps == N_DUMPS else args.dumps   # fewer only for profiler captures
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    plan = corr.Plan(n, c, t, 32)
    P = plan.n_baselines
    x = synth.torch_correlated_gaussian_f32(d, t, c, n, 16.0, 0.1, 2500, dev)
    vis = plan.empty_vis(d, dev)
    hbm, bf16, src = _peaks()
    algo = d * (t * c * n * 8 + c * P * 8)   # float32 samples in, float32 visibilities out
    res = {}
    for name, engine in (("bf16x3", corr.ENGINE_BF16X3), ("fp32", corr.ENGINE_FP32)):
        ws = plan.empty_workspace(engine, d, dev)
        run = lambda: plan.run(x, vis, ws, engine=engine, n_dumps=d, stream=stream)   # noqa: E731
        for _ in range(args.warmup):
            run()
        torch.cuda.synchronize()
        assert plan.check_device() == 0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        for k in range(args.steps):
            run()
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        res[name] = ev[0].elapsed_time(ev[-1]) / args.steps
        del ws
    cm = P * c * t * d
    ms = res["bf16x3"]
    gbs = algo / (ms / 1e3) / 1e9
    line = {"metric": "X-engine TeraCMAC/s (float samples, BF16x3)", "value": cm / (ms / 1e3) / 1e12,
            "unit": "TeraCMAC/s",
            "workload": f"stream64_float: 64 inputs x 768 ch x 1000 samples/dump x {d} dumps, float32 "
                        "(sigma 16, rho 0.1, no rounding)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "dtype": "bf16x3/f32",
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "algorithmic_bytes": algo, "peak_source": src,
                         "note": "samples in + visibilities out; the bf16 hi/lo planes are an intermediate"},
            "fp32_path": {"ms_per_step": res["fp32"], "value": cm / (res["fp32"] / 1e3) / 1e12,
                          "speedup_bf16x3_over_fp32": res["fp32"] / ms},
            "l2": f"inputs larger than L2 ({d * t * c * n * 8 / 1e9:.1f} GB per step)"}
    print(json.dumps(line), flush=True)


def run_dump(args):
    """Dump step with phase correction (Fig. 1, Sec. 2) on one dump of the 1024-input array's
    accumulators: a pure HBM stream (int64 in, float32 out, zeros back when resetting)."""
    import torch

    from paper_0906_1887_gb300 import corr
    n, c, t = args.dump_inputs, 1536, 256
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    plan = corr.Plan(n, c, t, 8)
    P = plan.n_baselines
    g = torch.Generator(device=dev)
    g.manual_seed(6000)
    acc = torch.randint(-(1 << 30), 1 << 30, (c, P, 2), generator=g, dtype=torch.int64, device=dev)   # 12.9 GB
    out = torch.empty((c, P, 2), dtype=torch.float32, device=dev)                                    # 6.45 GB
    tau = torch.randn(n, generator=g, dtype=torch.float64, device=dev) * 1e-6
    nu = 1.5e8 + 1e4 * torch.arange(c, dtype=torch.float64, device=dev)
    ws = torch.empty(plan.dump_workspace_size(), dtype=torch.uint8, device=dev)
    hbm, _, src = _peaks()
    res = {}
    for reset in (False, True):
        for _ in range(args.warmup):
            plan.dump(acc, out, 4, tau, nu, ws, reset=reset, stream=stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        for k in range(args.steps):
            plan.dump(acc, out, 4, tau, nu, ws, reset=reset, stream=stream)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[-1]) / args.steps
        by = c * P * (16 + 8 + (16 if reset else 0))
        res["reset" if reset else "read_only"] = {"ms": ms, "algorithmic_bytes": by, "achieved": by / (ms / 1e3) / 1e9,
                                                  "frac": by / (ms / 1e3) / 1e9 / hbm}
    line = {"metric": "dump step GB/s (average + phase correction)", "value": res["reset"]["achieved"], "unit": "GB/s",
            "workload": f"dump{n}: accumulators of one {n}-input x {c}-channel dump ({c * P * 16 / 1e9:.1f} GB int64) -> "
                        "float32 corrected visibilities, accumulators reset",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["reset"]["ms"],
            "roofline": {"bound": "hbm", "peak": hbm, "unit": "GB/s", "frac": res["reset"]["frac"],
                         "peak_source": src},
            "without_reset": res["read_only"], "with_reset": res["reset"]}
    print(json.dumps(line), flush=True)


def run_serve(args):
    import torch

    from paper_0906_1887_gb300 import corr
    rng = np.random.default_rng(5000)
    max_in = 1024 * 1536 * 1024 * 2
    # one pinned pool of random bytes serves every job's samples (any byte is a valid sample)
    pool = torch.empty(max_in, dtype=torch.uint8).pin_memory()
    chunk = torch.randint(0, 256, (1 << 26,), dtype=torch.uint8, generator=torch.Generator().manual_seed(5000))
    for off in range(0, max_in, chunk.numel()):
        m = min(chunk.numel(), max_in - off)
        pool[off:off + m].copy_(chunk[:m])
    srv = corr.Server(160 << 30, n_streams=8)
    rate = 200.0
    records = []
    lock = threading.Lock()
    pending = []
    done_evt = threading.Event()

    def waiter():
        while not (done_evt.is_set() and not pending):
            with lock:
                item = pending.pop(0) if pending else None
            if item is None:
                time.sleep(0.0005)
                continue
            jid, n, c, t, bits = item
            st, r = srv.wait(jid, 60.0)
            with lock:
                records.append((st, r.t_submit, r.t_start, r.t_done, n, c, t, bits, r.gpu_ms))
            srv.release(jid)

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    # warm-up: one job of each mode
    for bits in (4, 8):
        jid = srv.submit(64, 128, 256, bits, pool, None)
        srv.wait(jid, 60.0)
        srv.release(jid)
    t_start = time.time()
    t_next = t_start
    n_sub = 0
    while True:
        now = time.time()
        if now - t_start > args.serve_seconds:
            break
        if now < t_next:
            time.sleep(min(t_next - now, 0.002))
            continue
        t_next += rng.exponential(1.0 / rate)
        a = 8 * int(rng.integers(4, 65))            # 32..512 antennas (multiples of 8)
        n, c, t = 2 * a, int(rng.integers(128, 1537)), int(rng.integers(256, 1025))
        bits = 4 if rng.random() < 0.5 else 8
        jid = srv.submit(n, c, t, bits, pool, None, stream_tag=n_sub % 8)
        n_sub += 1
        with lock:
            pending.append((jid, n, c, t, bits))
    done_evt.set()
    th.join(timeout=300)
    wall = time.time() - t_start
    srv.close()
    ok = [r for r in records if r[0] == 0]
    lat = np.array([r[3] - r[1] for r in ok]) * 1e3
    tdump = np.array([r[6] / CHANNEL_RATE_HZ for r in ok]) * 1e3
    cm = sum(r[4] * (r[4] + 1) // 2 * r[5] * r[6] for r in ok)
    line = {"metric": "serving p99 latency / real-time factor / TeraCMAC/s", "unit": "ms",
            "workload": "serve: Poisson 200 jobs/s over 8 stream tags, 32..512 dual-pol antennas, "
                        "128..1536 channels, 256..1024 samples, 4/8-bit",
            "value": float(np.percentile(lat, 99)) if len(lat) else None,
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "frac_within_dump_interval": float(np.mean(lat < tdump)) if len(lat) else None,
            "jobs_submitted": n_sub, "jobs_ok": len(ok), "jobs_failed": len(records) - len(ok),
            "wall_s": wall, "jobs_per_s": len(ok) / wall,
            "real_time_factor": float(tdump.sum() / 1e3 / wall) if len(lat) else None,
            "tera_cmac_per_s": cm / wall / 1e12,
            "result": "visibilities left in HBM (device-resident), released after completion"}
    print(json.dumps(line), flush=True)


def main():
    global N_DUMPS, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--dumps", type=int, default=N_DUMPS,
                    help="dumps per step (default: the full 200-dump job; smaller only for profiler captures)")
    ap.add_argument("--workload", default="stream", choices=["stream", "large", "batch", "serve", "fx", "dump", "float"])
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--dump-inputs", type=int, default=1024,
                    help="inputs of the dump workload (1024 = the 1024-input array; smaller for a profiler capture)")
    ap.add_argument("--large-chans", type=int, default=1536,
                    help="channels of the large-array workload (fewer only for profiling captures)")
    args = ap.parse_args()

    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload != "stream":
        {"large": run_large, "batch": run_batch, "serve": run_serve, "fx": run_fx, "dump": run_dump,
         "float": run_float}[args.workload](args)
        return

    import torch

    from paper_0906_1887_gb300 import corr, synth

    if args.dumps != N_DUMPS:
        WORKLOAD = WORKLOAD.replace("x 200 dumps", f"x {args.dumps} dumps (reduced for profiling)")
        N_DUMPS = args.dumps

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        return rank_max(x, dist, dev)

    corr.lib()
    plan = corr.Plan(N_INPUTS, N_CHAN, N_TIME, BITS)
    P = plan.n_baselines
    packed = synth.torch_correlated_gaussian_packed8(N_DUMPS, N_TIME, N_CHAN, N_INPUTS, SIGMA, RHO,
                                                     SEED + 7919 * rank, dev)
    vis = plan.empty_vis(N_DUMPS, dev)
    ws = plan.empty_workspace(corr.ENGINE_TC, N_DUMPS, dev)     # None: packed samples feed the kernel directly
    stream = torch.cuda.current_stream(dev)

    def step_tc():
        plan.run(packed, vis, ws, engine=corr.ENGINE_TC, n_dumps=N_DUMPS, stream=stream)

    # warm-up
    for _ in range(args.warmup):
        step_tc()
    barrier()
    if plan.check_device() != 0:
        raise RuntimeError("device-side wait gave up during warm-up")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # device-timed region: K whole-job steps (inputs 19.7 GB per step >> L2, no flush needed)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        step_tc()
        ev[k + 1].record(stream)
    barrier()
    clk = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms_total = ev[0].elapsed_time(ev[-1])
    if plan.check_device() != 0:
        raise RuntimeError("device-side wait gave up in the timed region")

    ms_step = max_over_ranks(ms_total / args.steps)
    cm_step = P * N_CHAN * N_TIME * N_DUMPS
    value = aggregate_tera_cmac(cm_step, world, ms_step)
    rtf = (N_TIME * N_DUMPS / CHANNEL_RATE_HZ) / (ms_step / 1e3)

    # FP32 CUDA-core engine on the same job (unpack to fp16 planes + CUDA-core cross-multiply)
    ws32 = plan.empty_workspace(corr.ENGINE_FP32, N_DUMPS, dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.run(packed, vis, ws32, engine=corr.ENGINE_FP32, n_dumps=N_DUMPS, stream=stream)
    barrier()
    ev0.record(stream)
    for _ in range(args.fp32_steps):
        plan.run(packed, vis, ws32, engine=corr.ENGINE_FP32, n_dumps=N_DUMPS, stream=stream)
    ev1.record(stream)
    barrier()
    ms32 = max_over_ranks(ev0.elapsed_time(ev1) / args.fp32_steps)
    value32 = cm_step * world / (ms32 / 1e3) / 1e12
    del ws32
    torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: corr_xengine_run_host pipelines the
    # host-to-device copy of the packed samples, the X stage and the device-to-host copy of
    # the visibilities over chunks of dumps (pinned host memory)
    host_in = torch.empty(packed.shape, dtype=torch.uint8, pin_memory=True)
    host_in.copy_(packed)
    host_out = torch.empty(vis.shape, dtype=vis.dtype, pin_memory=True)
    del ws
    torch.cuda.synchronize(dev)
    plan.run_host(host_in, host_out, n_dumps=N_DUMPS)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(e2e_steps):
        plan.run_host(host_in, host_out, n_dumps=N_DUMPS)
    ev1.record(stream)
    barrier()
    ms_e2e_wall = (time.perf_counter() - t0) * 1e3 / e2e_steps
    ms_e2e = max_over_ranks(ms_e2e_wall)
    e2e_value = cm_step * world / (ms_e2e / 1e3) / 1e12
    del host_in, host_out

    # roofline of the step's one kernel (the fused tensor-core X stage): HBM-bound here
    hbm_peak, bf16_peak, peak_src = _peaks()
    ms_x = statistics.median(step_ms)
    in_bytes = N_DUMPS * N_TIME * N_CHAN * N_INPUTS * 2
    out_bytes = N_DUMPS * N_CHAN * P * 16
    x_bytes = in_bytes + out_bytes                 # packed samples read once + int64 visibilities written
    x_gbs = x_bytes / (ms_x / 1e3) / 1e9
    flops = 8.0 * cm_step
    roofline = {"bound": "hbm", "kernel": "xeng_tc_kernel<raw8>", "achieved": x_gbs, "peak": hbm_peak,
                "unit": "GB/s", "frac": x_gbs / hbm_peak,
                "traffic": DRAM_BYTES_PER_DUMP * N_DUMPS if DRAM_BYTES_PER_DUMP else None,
                "peak_source": ("measured: MEASURED_PEAKS.json hbm_gbs" if peak_src == "measured" else peak_src),
                "algorithmic_bytes_per_launch": x_bytes, "kernel_ms": ms_x,
                "tensor_tflops_algorithmic": flops / (ms_x / 1e3) / 1e12,
                "tensor_frac_of_measured_bf16_burst": flops / (ms_x / 1e3) / 1e12 / bf16_peak}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # the CPU oracle is timed on rank 0 at N = 1 only (a reported baseline, not part of the run)
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline()
    line = {
        "metric": "X-engine TeraCMAC/s", "value": value, "unit": "TeraCMAC/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_inputs": N_INPUTS, "n_chan": N_CHAN, "n_time": N_TIME,
                   "n_dumps": N_DUMPS, "sample_bits": BITS, "engine": "fused tcgen05 X stage: packed 8-bit -> fp16 in shared memory, fp32 accum, exact int64",
                   "l2": "inputs (19.7 GB per step) far larger than L2; no flush", "parallelism": f"replicas{world}"},
        "real_time_factor": rtf,
        "fp32_path": {"value": value32, "unit": "TeraCMAC/s", "ms_per_step": ms32, "speedup_tc_over_fp32": value / value32},
        "e2e": {"value": e2e_value, "unit": "TeraCMAC/s", "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": int(packed.numel()) * world,
                "d2h_bytes_per_step": int(vis.numel() * vis.element_size()) * world,
                "api": "corr_xengine_run_host (pinned host buffers, chunked copy/compute overlap)",
                "timing": "host wall clock around the synchronous call"},
        "roofline": roofline,
        "gpu_launches": args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

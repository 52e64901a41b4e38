"""Benchmark of the X stage (cross-multiply-accumulate) on GB300.

Headline workload (the streamed real-time correlator): 64 inputs (32 dual-pol antennas),
768 channels, 1000 samples per dump, 200 dumps, complex 8-bit Gaussian samples (sigma 16,
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
  configs      (N = 1 only) every other workload of the benchmark set, each with its value,
               kernel time, roofline fraction and FP32 ratio or latency figures:
               mwa32t_4bit (64 inputs x 128 ch x 512 samples, 4-bit, one dump),
               large1024 (1024 inputs x 1536 ch x 256 samples x 20 dumps),
               batch40 (40 uneven jobs in one autotuned graph launch),
               serve (Poisson 200 jobs/s over 8 streams for 60 s: p50/p99, RTF),
               float_stream (the stream's float variant through BF16x3, error vs float64),
               fx_chain (F stage + X stage of the 32-antenna prototype, error vs float64)
Options: --gpus N (torchrun, one rank per GPU, weak scaling: every rank runs the whole
job on its own GPU), --steps K, --warmup W, --impl reference (the CPU oracle arm),
--no-configs (the headline workload only), --workload NAME (one workload on its own line).
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
# workload, from one ncu capture of an 8-dump launch of this build (786.62 MB read + 177.14 MB
# written), scaled by dumps; set to None whenever the kernel changes until it is captured again.
DRAM_BYTES_PER_DUMP = (786617856 + 177139200) / 8


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


# ---- the other workloads of the benchmark set (one sub-object each in the default line) ----

def _free():
    import gc

    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _event_ms(fn, steps, stream, flush=None):
    """Mean device time (ms) of fn over `steps` runs, CUDA events on `stream`; with `flush`, a
    buffer larger than L2 is written before every run (outside the timed span)."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
    for k in range(steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        ev[2 * k].record(stream)
        fn()
        ev[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    return sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps)) / steps


def _normwise(v, ref, n):
    """max |V - V64| / sqrt(V64_ii V64_jj) over channels and pairs."""
    iu, ju = np.triu_indices(n)
    auto = [i * n - i * (i - 1) // 2 for i in range(n)]
    a = ref[..., auto, 0]
    scale = np.sqrt(np.maximum(a[..., iu] * a[..., ju], 1e-300))
    err = np.hypot(v[..., 0] - ref[..., 0], v[..., 1] - ref[..., 1])
    return float((err / scale).max())


def oracle_float_errors(samples_host, n, c_sel, t, results):
    """CPU-baseline leg (host, rank 0, N = 1): the float64 oracle on a sample of channels, and
    the BF16x3 per-element bound.  samples_host: float32 [T][c_sel][N][2]; results: name ->
    float [c_sel][P][2] from the GPU.  Returns name -> normwise error against float64, and for
    BF16x3 the largest error / bound (<= 1 means within the bound)."""
    from oracle import precision
    bound, ex = precision.bf16x3_bound(samples_host, n, c_sel, t)
    out = {}
    for name, v in results.items():
        v = np.asarray(v, np.float64)
        out[name] = {"err_vs_fp64": _normwise(v, ex, n)}
        if name == "bf16x3":
            err = np.hypot(v[..., 0] - ex[..., 0], v[..., 1] - ex[..., 1])
            out[name]["max_err_over_bound"] = float((err / np.maximum(bound, 1e-300)).max())
    return out


def run_mwa32t(args):
    """The 32-antenna prototype's X stage as the paper sizes it: 64 inputs x 128 channels x 512
    samples, 4-bit, one dump per step (4.2 MB in, 4.3 MB out: an L2 flush between steps)."""
    import torch

    from paper_0906_1887_gb300 import corr, synth
    n, c, t = 64, 128, 512
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    plan = corr.Plan(n, c, t, 4)
    P = plan.n_baselines
    x = synth.torch_uniform_packed4(1, t, c, n, 1000, dev)
    vis = plan.empty_vis(1, dev)
    ws32 = plan.empty_workspace(corr.ENGINE_FP32, 1, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    steps = max(args.steps, 20)
    tc = lambda: plan.run(x, vis, None, engine=corr.ENGINE_TC, stream=stream)   # noqa: E731
    f32 = lambda: plan.run(x, vis, ws32, engine=corr.ENGINE_FP32, stream=stream)   # noqa: E731
    # the same dump with fp16 operands (the plan's default feeds 4-bit samples as e4m3 operands,
    # kind::f8f6f4): identical results, twice the operand bytes and MMAs per sample
    plan16 = corr.Plan(n, c, t, 4)
    plan16.set_operands(corr.OPERANDS_PACKED, 0)
    vis16 = plan16.empty_vis(1, dev)
    f16 = lambda: plan16.run(x, vis16, None, engine=corr.ENGINE_TC, stream=stream)   # noqa: E731
    for _ in range(args.warmup):
        tc()
        f16()
        f32()
    torch.cuda.synchronize()
    assert plan.check_device() == 0 and plan16.check_device() == 0
    f16()
    tc()
    torch.cuda.synchronize()
    assert torch.equal(vis, vis16)
    # a 20 us launch: two interleaved rounds of `steps` launches per operand type, the better
    # round's mean kept for each
    rounds = [(_event_ms(tc, steps, stream, flush), _event_ms(f16, steps, stream, flush)) for _ in range(2)]
    ms, ms16 = min(r[0] for r in rounds), min(r[1] for r in rounds)
    ms32 = _event_ms(f32, steps, stream, flush)
    hbm, _, src = _peaks()
    by = t * c * n + c * P * 16
    cm = P * c * t
    res = {"workload": "mwa32t_4bit: 64 inputs x 128 channels x 512 samples, 4-bit uniform [-7, 7], one dump",
           "value": cm / (ms / 1e3) / 1e12, "unit": "TeraCMAC/s", "kernel_ms": ms, "steps": steps,
           "real_time_factor": (t / CHANNEL_RATE_HZ) / (ms / 1e3),
           "roofline": {"bound": "hbm", "achieved": by / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": by / (ms / 1e3) / 1e9 / hbm, "algorithmic_bytes": by, "peak_source": src,
                        "note": "one 4.3 MB dump is launch- and latency-bound, far from either roofline"},
           "fp32_path": {"kernel_ms": ms32, "value": cm / (ms32 / 1e3) / 1e12, "speedup_tc_over_fp32": ms32 / ms},
           "l2": "256 MB written between timed steps"}
    res["operands"] = "e4m3 (tcgen05 kind::f8f6f4)"
    res["timing"] = f"best of 2 interleaved rounds of {steps} launches per operand type"
    res["fp16_operands"] = {"kernel_ms": ms16, "value": cm / (ms16 / 1e3) / 1e12, "same_bits": True}
    plan16.close()
    plan.close()
    del x, vis, vis16, ws32, flush
    _free()
    res["stream64_4bit"] = _stream4(args)
    return res


def _stream4(args):
    """A 4-bit stream at the headline's array size (64 inputs x 768 channels x 1000 samples per
    dump, 50 dumps, 2.5 GB in) through fp16 and e4m3 operands: where the conversion and the
    operand reads, not the launch, set the pace."""
    import torch

    from paper_0906_1887_gb300 import corr, synth
    n, c, t, d = 64, 768, 1000, 50
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    x = synth.torch_uniform_packed4(d, t, c, n, 1100, dev, -8, 7).reshape(-1)
    out = {}
    vis = {}
    for name, ops in (("fp16", corr.OPERANDS_PACKED), ("e4m3", corr.OPERANDS_PACKED_F8)):
        plan = corr.Plan(n, c, t, 4)
        plan.set_operands(ops, 0)
        v = plan.empty_vis(d, dev)
        fn = lambda: plan.run(x, v, None, engine=corr.ENGINE_TC, n_dumps=d, stream=stream)   # noqa: E731
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        assert plan.check_device() == 0
        ms = _event_ms(fn, max(args.steps, 3), stream)
        P = plan.n_baselines
        by = d * (t * c * n + c * P * 16)
        hbm, _, src = _peaks()
        out[name] = {"kernel_ms": ms, "value": P * c * t * d / (ms / 1e3) / 1e12,
                     "hbm_frac": by / (ms / 1e3) / 1e9 / hbm}
        vis[name] = v
        plan.close()
    out["same_bits"] = bool(torch.equal(vis["fp16"], vis["e4m3"]))
    out["workload"] = "stream64_4bit: 64 inputs x 768 ch x 1000 samples/dump x 50 dumps, 4-bit uniform [-8, 7]"
    out["unit"] = "TeraCMAC/s"
    out["l2"] = "inputs (2.5 GB) larger than L2"
    del x, vis
    _free()
    return out


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
    # the plane feed: the unpack kernel writes fp16 planes (1.6 GB), the tensor-core kernel reads
    # them in wide items; every X stage below is both kernels
    ws = plan.empty_workspace(corr.ENGINE_TC, 1, dev)
    stream = torch.cuda.current_stream(dev)
    steps = min(args.steps, 5)

    def step():
        for k in range(d):
            plan.run(packed[k], vis[k & 1], ws, engine=corr.ENGINE_TC, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for k in range(steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[-1]) / steps
    cm = P * c * t * d
    ms_one = ms / d
    # the two kernels of one dump on their own, and the packed feed (fused conversion) for comparison
    ms_unpack = _event_ms(lambda: plan.unpack(packed[0], ws, stream=stream), 3, stream)
    ms_xplanes = _event_ms(lambda: plan.run_planes(ws, vis[0], engine=corr.ENGINE_TC, stream=stream), 3, stream)
    plan.run(packed[0], vis[1], None, engine=corr.ENGINE_TC, stream=stream)
    ms_packed = _event_ms(lambda: plan.run(packed[0], vis[1], None, engine=corr.ENGINE_TC, stream=stream), 3, stream)
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
    ms_fused = _event_ms(lambda: [plan.run_dump(packed[k], outf, 1, tau, nu, dws, stream=stream)
                                  for k in range(d)], 1, stream) / d
    plan.dump(vis[0], outf, 1, tau, nu, dws, stream=stream)
    ms_dump = _event_ms(lambda: plan.dump(vis[0], outf, 1, tau, nu, dws, stream=stream), 1, stream)
    del outf
    # FP32 engine on one dump
    del ws
    ws = plan.empty_workspace(corr.ENGINE_FP32, 1, dev)
    plan.run(packed[0], vis[1], ws, engine=corr.ENGINE_FP32, stream=stream)
    ms32 = _event_ms(lambda: plan.run(packed[0], vis[1], ws, engine=corr.ENGINE_FP32, stream=stream), 1, stream)
    del ws
    hbm, bf16, src = _peaks()
    out_bytes = P * c * 16
    bytes_launch = per_dump + out_bytes
    gbs = bytes_launch / (ms_one / 1e3) / 1e9
    res = {"metric": "X-engine TeraCMAC/s", "value": cm / (ms / 1e3) / 1e12, "unit": "TeraCMAC/s",
           "workload": f"large1024_8bit: 1024 inputs x {c} channels x 256 samples/dump x {d} dumps, sigma 8"
                       + ("" if c == 1536 else " (reduced for profiling)"),
           "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "kernel_ms": ms_one,
           "real_time_factor": (t * d / CHANNEL_RATE_HZ) / (ms / 1e3),
           "fp32_path": {"value": P * c * t / (ms32 / 1e3) / 1e12, "kernel_ms": ms32,
                         "speedup_tc_over_fp32": ms32 / ms_one},
           "fused_dump": {"ms_per_dump": ms_fused, "value": P * c * t / (ms_fused / 1e3) / 1e12,
                          "separate_x_plus_dump_ms": ms_one + ms_dump, "dump_step_ms": ms_dump,
                          "output": "float32 V / n_accum, phase-corrected (8 B per baseline)",
                          "achieved_gbs": (per_dump + P * c * 8) / (ms_fused / 1e3) / 1e9},
           "roofline": {"bound": "hbm", "kernel": "unpack_fast_kernel<8> + xeng_tc_kernel<planes, wide items>",
                        "achieved": gbs, "peak": hbm,
                        "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes_per_launch": bytes_launch,
                        "kernel_ms": ms_one, "tensor_tflops_algorithmic": 8.0 * P * c * t / (ms_one / 1e3) / 1e12,
                        "peak_source": src,
                        "note": "per dump: samples in + int64 visibilities out over the time of both kernels"},
           "kernels": {"unpack_ms": ms_unpack, "xeng_planes_ms": ms_xplanes,
                       "packed_feed_ms": ms_packed,
                       "packed_feed_frac": bytes_launch / (ms_packed / 1e3) / 1e9 / hbm},
           "int8_target": {"note": "tcgen05 has no INT8 MMA on sm_103a; the legacy INT8 tensor path measures "
                                   "151 TOPS, against which the algorithmic rate below is the fraction",
                           "algorithmic_tops": 8.0 * P * c * t / (ms_one / 1e3) / 1e12,
                           "frac_of_int8_mma_sync_151tops": 8.0 * P * c * t / (ms_one / 1e3) / 1e12 / 151.0},
           "clocks": clk}
    del packed, vis
    return res


def _batch_jobs(rng):
    sizes = []
    for ant in (16, 32, 64, 128, 256):
        for _ in range(8):
            sizes.append((2 * ant, 64 * int(rng.integers(1, 17)), 128 * int(rng.integers(1, 17))))
    return sizes


def _tune_cache_path():
    """Autotune cache file keyed by the library build (its size and modification time), so a
    stale entry of another build is never reused."""
    import tempfile

    from paper_0906_1887_gb300 import corr
    st = os.stat(corr.LIB_PATH)
    return os.path.join(tempfile.gettempdir(), f"corr_batch_tune_{st.st_size}_{int(st.st_mtime)}.jsonl")


def run_batch(args):
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
    t0 = time.time()
    b = corr.Batch(descs, flags=corr.BATCH_GRAPH | corr.BATCH_AUTOTUNE | corr.BATCH_PLANES,
                   tune_cache=_tune_cache_path())
    tune_s = time.time() - t0
    info = b.info()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        b.run(stream)
    torch.cuda.synchronize()
    assert b.check_device() == 0
    steps = max(args.steps, 5)
    ms = _event_ms(lambda: b.run(stream), steps, stream)
    # the same jobs, one launch each
    plans = [corr.Plan(n, c, t, 8) for n, c, t in sizes]
    each = lambda: [p.run(x, v, None, engine=corr.ENGINE_TC, stream=stream) for p, (x, v) in zip(plans, jobs)]  # noqa
    each()
    ms_each = _event_ms(each, steps, stream)
    # the compute-heavy part: the 512-input jobs alone, in one launch
    big = [dd for dd in descs if dd[0] == 512]
    b512 = corr.Batch(big, flags=corr.BATCH_GRAPH | corr.BATCH_AUTOTUNE | corr.BATCH_PLANES,
                      tune_cache=_tune_cache_path())
    b512.run(stream)
    ms512 = _event_ms(lambda: b512.run(stream), steps, stream)
    cm512 = sum(dd[0] * (dd[0] + 1) // 2 * dd[1] * dd[2] for dd in big)
    b512.close()
    # algorithmic bytes of the step: packed samples in (2 B per complex sample) + int64 visibilities out
    algo = sum(2 * n * c * t + 16 * (n * (n + 1) // 2) * c for n, c, t in sizes)
    hbm, bf16, src = _peaks()
    gbs = algo / (ms / 1e3) / 1e9
    tflops = 8 * cm / (ms / 1e3) / 1e12   # 4 real MACs per CMAC
    res = {"metric": "X-engine TeraCMAC/s", "value": cm / (ms / 1e3) / 1e12, "unit": "TeraCMAC/s",
           "workload": "batch40: 8 each of 16/32/64/128/256 dual-pol antennas, 64..1024 channels, "
                       "128..2048 samples, 8-bit Gaussian sigma 16, seed 4000",
           "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "kernel_ms": ms,
           "roofline": {"bound": "hbm", "kernel": "xeng_tc_kernel job tables (packed feed; plane feed after unpack "
                                                  "for the tuner's array sizes)", "achieved": gbs,
                        "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes": algo,
                        "peak_source": src, "tensor_tflops_algorithmic": tflops,
                        "tensor_frac_of_measured_bf16_burst": tflops / bf16},
           "jobs_512_inputs": {"n_jobs": len(big), "ms": ms512, "value": cm512 / (ms512 / 1e3) / 1e12,
                               "tensor_tflops_algorithmic": 8 * cm512 / (ms512 / 1e3) / 1e12,
                               "tensor_frac_of_measured_bf16_burst": 8 * cm512 / (ms512 / 1e3) / 1e12 / bf16},
           "one_launch_per_job": {"ms_per_step": ms_each, "value": cm / (ms_each / 1e3) / 1e12},
           "batch": info, "autotune_seconds": tune_s, "cmacs_per_step": cm}
    b.close()
    for p in plans:
        p.close()
    return res


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
    steps = max(args.steps, 5)
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
        res[name] = _event_ms(step, steps, stream, flush)
        del ws
    f_ms = _event_ms(lambda: fplan.run(x, spec, frames, stream=stream), steps, stream, flush)
    # the polyphase filterbank variant (8 taps, default prototype) on the same second of data
    taps = 8
    pplan = corr.FPlan(n, c, corr.F_COMPLEX8, n_taps=taps)
    xp = synth.torch_correlated_gaussian_packed8(1, (frames + taps - 1) * c, 1, n, 16.0, 0.1, 5001, dev).reshape(-1)
    pfb_run = lambda: pplan.run(xp, spec, frames, stream=stream)   # noqa: E731
    for _ in range(args.warmup):
        pfb_run()
    pfb_ms = _event_ms(pfb_run, steps, stream, flush)
    pfb_bytes = (frames + taps - 1) * pplan.in_bytes_per_frame + frames * pplan.out_bytes_per_frame
    # error against float64 on a 1000-frame slice (0.1 s) of the same stream through the same
    # kernels: the oracle's complex128 F stage, then its X stage (CPU-baseline leg)
    ef = 1000
    xs = x[: ef * c * n * 2]
    spec_s = fplan.empty_spectra(ef, dev)
    fplan.run(xs, spec_s, ef, stream=stream)
    xplan_s = corr.Plan(n, c, ef, 32)
    outs = {}
    for name, engine in (("fp32", corr.ENGINE_FP32), ("bf16x3", corr.ENGINE_BF16X3)):
        v = xplan_s.empty_vis(1, dev)
        xplan_s.run(spec_s, v, xplan_s.empty_workspace(engine, 1, dev), engine=engine, stream=stream)
        torch.cuda.synchronize()
        outs[name] = v.cpu().numpy()[0].astype(np.float64)
    err = {}
    if not args.no_cpu_baseline:
        from oracle import fstage
        ref = fstage.xcorr_spectra(fstage.fstage(xs.cpu().numpy(), n, c, ef, "c8"))
        for name in outs:
            err[name] = {"err_vs_fp64": _normwise(outs[name], ref, n)}
        xb = oracle_float_errors(spec_s.cpu().numpy(), n, c, ef, {"bf16x3": outs["bf16x3"]})
        err["bf16x3"]["x_stage_max_err_over_bound"] = xb["bf16x3"]["max_err_over_bound"]
    xplan_s.close()
    ms = res["fp32"]
    cm = P * c * frames
    gbs = f_bytes / (f_ms / 1e3) / 1e9
    out = {"metric": "FX chain TeraCMAC/s (F stage + X stage, FP32 X engine)", "value": cm / (ms / 1e3) / 1e12,
           "unit": "TeraCMAC/s",
           "workload": "mwa32t_fx: 64 inputs x 1.28 MHz complex 8-bit (sigma 16, rho 0.1), 128 channels, "
                       "1 s of data per step (10000 frames), one dump",
           "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "kernel_ms": ms,
           "real_time_factor": 1000.0 / ms,
           "bf16x3_chain": {"ms_per_step": res["bf16x3"], "value": cm / (res["bf16x3"] / 1e3) / 1e12,
                            "real_time_factor": 1000.0 / res["bf16x3"]},
           # Table 4's actual column: the 1.28 MHz band processed in this time per second of data
           "processed_bandwidth_mhz": {"fp32_chain": 1.28 / (ms / 1e3), "bf16x3_chain": 1.28 / (res["bf16x3"] / 1e3),
                                       "paper_c1060_gp4_mhz": 6.9},
           "fstage": {"kernel": "fengine_kernel<complex8>", "ms": f_ms, "bound": "hbm", "achieved": gbs,
                      "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes": f_bytes,
                      "peak_source": src},
           "pfb_fstage": {"taps": taps, "ms": pfb_ms, "achieved": pfb_bytes / (pfb_ms / 1e3) / 1e9,
                          "frac": pfb_bytes / (pfb_ms / 1e3) / 1e9 / hbm, "algorithmic_bytes": pfb_bytes,
                          "note": "each input frame is read by 8 output frames (through L2); bytes counted once"},
           "err_vs_fp64": err,
           "err_sample": "1000-frame slice, all 128 channels, against the oracle's complex128 F and float64 X stages",
           "paper_context": "C1060 (Table 3): unpack 53 + FFT 53 + CMAC (GP, G=4) 185 = 291 ms per second of data",
           "l2": "256 MB flush written between timed steps"}
    fplan.close()
    pplan.close()
    xplan.close()
    return out


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
    vis = {"bf16x3": plan.empty_vis(d, dev), "fp32": plan.empty_vis(d, dev)}
    hbm, bf16, src = _peaks()
    algo = d * (t * c * n * 8 + c * P * 8)   # float32 samples in, float32 visibilities out
    steps = min(max(args.steps, 3), 10)
    res = {}
    for name, engine in (("bf16x3", corr.ENGINE_BF16X3), ("fp32", corr.ENGINE_FP32)):
        ws = plan.empty_workspace(engine, d, dev)
        run = lambda: plan.run(x, vis[name], ws, engine=engine, n_dumps=d, stream=stream)   # noqa: E731
        for _ in range(args.warmup):
            run()
        torch.cuda.synchronize()
        assert plan.check_device() == 0
        res[name] = _event_ms(run, steps, stream)
        del ws
    # error against float64 on 8 sampled channels of dump 0 (CPU-baseline leg)
    err = {}
    if not args.no_cpu_baseline:
        chans = np.sort(np.random.default_rng(2501).choice(c, 8, replace=False))
        ci = torch.from_numpy(chans).to(dev)
        xs = x[0].index_select(1, ci).contiguous().cpu().numpy()
        got = {k: v[0].index_select(0, ci).cpu().numpy() for k, v in vis.items()}
        err = oracle_float_errors(xs, n, len(chans), t, got)
    cm = P * c * t * d
    ms = res["bf16x3"]
    gbs = algo / (ms / 1e3) / 1e9
    out = {"metric": "X-engine TeraCMAC/s (float samples, BF16x3)", "value": cm / (ms / 1e3) / 1e12,
           "unit": "TeraCMAC/s",
           "workload": f"stream64_float: 64 inputs x 768 ch x 1000 samples/dump x {d} dumps, float32 "
                       "(sigma 16, rho 0.1, no rounding)",
           "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "kernel_ms": ms, "dtype": "bf16x3/f32",
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                        "algorithmic_bytes": algo, "peak_source": src,
                        "note": "samples in + visibilities out"},
           "fp32_path": {"ms_per_step": res["fp32"], "value": cm / (res["fp32"] / 1e3) / 1e12,
                         "speedup_bf16x3_over_fp32": res["fp32"] / ms},
           "err_vs_fp64": err,
           "err_sample": "8 seeded channels of dump 0 against the float64 oracle (normwise metric)",
           "l2": f"inputs larger than L2 ({d * t * c * n * 8 / 1e9:.1f} GB per step)"}
    plan.close()
    del x, vis
    return out


def run_shape(args):
    """One X stage of a given shape (--shape N,C,T,BITS) through the library's API, with a chosen
    engine (--engine tc|fp32) and, for the tensor cores, operand feed (--feed auto|packed|planes)
    and item shape (--items auto|tiles|wide): the launch a profiler capture of one kernel needs."""
    import torch

    from paper_0906_1887_gb300 import corr, synth
    n, c, t, bits = (int(v) for v in args.shape.split(","))
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    plan = corr.Plan(n, c, t, bits)
    engine = {"tc": corr.ENGINE_TC, "fp32": corr.ENGINE_FP32}[args.engine]
    # planes_fp16: the public planes calls (corr_unpack into fp16 planes, then the plane-fed X
    # stage), which 4-bit plans otherwise replace by e4m3 planes in their workspace
    plan.set_operands({"auto": corr.OPERANDS_AUTO, "packed": corr.OPERANDS_PACKED, "planes": corr.OPERANDS_PLANES,
                       "planes_fp16": corr.OPERANDS_PLANES, "packed_f8": corr.OPERANDS_PACKED_F8}[args.feed],
                      {"auto": corr.ITEMS_AUTO, "tiles": corr.ITEMS_TILES, "wide": corr.ITEMS_WIDE}[args.items])
    if args.op_stages:
        plan.set_tuning(args.op_stages, 0)
    if bits == 4:
        x = synth.torch_uniform_packed4(1, t, c, n, 7000, dev)
    elif bits == 8:
        x = synth.torch_correlated_gaussian_packed8(1, t, c, n, 16.0, 0.0, 7000, dev)
    else:
        x = synth.torch_correlated_gaussian_f32(1, t, c, n, 16.0, 0.0, 7000, dev)
    # the library takes raw pointers: the buffer must hold one dump of this shape
    if x.numel() * x.element_size() != plan.info()[1]:
        raise ValueError("sample buffer does not match the plan's packed size")
    vis = plan.empty_vis(1, dev)
    if args.feed == "planes_fp16":
        ws = torch.empty(plan.planes_size(1), dtype=torch.uint8, device=dev)

        def run():
            plan.unpack(x, ws, stream=stream)
            plan.run_planes(ws, vis, engine=engine, stream=stream)
    else:
        ws = plan.empty_workspace(engine, 1, dev) if args.feed != "packed" else None
        run = lambda: plan.run(x, vis, ws, engine=engine, stream=stream)   # noqa: E731
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    ms = _event_ms(run, args.steps, stream)
    P = plan.n_baselines
    hbm, bf16, src = _peaks()
    by = t * c * n * {4: 1, 8: 2, 32: 8}[bits] + (8 if bits == 32 else 16) * P * c
    out = {"workload": f"shape {n} inputs x {c} channels x {t} samples, {bits}-bit, engine {args.engine}, "
                       f"feed {args.feed}, items {args.items}, operand stages {args.op_stages or 'default'}",
           "value": P * c * t / (ms / 1e3) / 1e12, "unit": "TeraCMAC/s", "ms": ms, "steps": args.steps,
           "tensor_tflops_algorithmic": 8.0 * P * c * t / (ms / 1e3) / 1e12,
           "hbm_frac": by / (ms / 1e3) / 1e9 / hbm, "algorithmic_bytes": by}
    plan.close()
    return out


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
    return line


def _stream_latency(ok, s_, t_job_ms):
    """One open stream's latency summary: p50/p99 (ms), the fraction within its own sample time,
    its jobs' mean device time and mean wait from submission to the start of its copy."""
    lat = np.array([r[3] - r[1] for r in ok if r[4] == s_]) * 1e3
    if not len(lat):
        return {"stream": s_, "jobs": 0}
    gpu = np.array([r[6] for r in ok if r[4] == s_])
    queued = np.array([r[2] - r[1] for r in ok if r[4] == s_]) * 1e3
    return {"stream": s_, "jobs": int(len(lat)), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "sample_time_ms": t_job_ms,
            "frac_within_sample_time": float(np.mean(lat < t_job_ms)), "mean_gpu_ms": float(gpu.mean()),
            "mean_queued_ms": float(queued.mean())}


def run_serve(args):
    """Serving loop (config 5): 8 input streams, each a random array drawn once from the seed
    (32..512 dual-pol antennas, 128..1536 channels, 256..1024 samples per job, 4 or 8 bits), each
    opened with device state -- a 4-slot sample ring and accumulators -- and dumped every 16 jobs
    through the dump step (averaged, float32) into a pinned host buffer.  Jobs arrive as a
    Poisson process (mean 200 jobs/s over all streams) for --serve-seconds of wall time."""
    import torch

    from paper_0906_1887_gb300 import corr
    rng = np.random.default_rng(5000)
    n_streams, jobs_per_dump, ring = 8, 16, 4
    shapes = []
    for _ in range(n_streams):
        a = 8 * int(rng.integers(4, 65))            # 32..512 antennas (multiples of 8)
        shapes.append((2 * a, int(rng.integers(128, 1537)), int(rng.integers(256, 1025)),
                       4 if rng.random() < 0.5 else 8))
    max_in = max(n * c * t * (2 if b == 8 else 1) for n, c, t, b in shapes)
    # one pinned pool of random bytes serves every job's samples (any byte is a valid sample)
    pool = torch.empty(max_in, dtype=torch.uint8).pin_memory()
    chunk = torch.randint(0, 256, (1 << 26,), dtype=torch.uint8, generator=torch.Generator().manual_seed(5000))
    for off in range(0, max_in, chunk.numel()):
        m = min(chunk.numel(), max_in - off)
        pool[off:off + m].copy_(chunk[:m])
    dumps = [torch.empty((c, n * (n + 1) // 2, 2), dtype=torch.float32).pin_memory() for n, c, t, b in shapes]
    srv = corr.Server(200 << 30, n_streams=8)
    for s_, (n, c, t, b) in enumerate(shapes):
        srv.open_stream(s_, n, c, t, b, ring_slots=ring, jobs_per_dump=jobs_per_dump,
                        dump_mode=corr.STREAM_DUMP_AVERAGED)
    arena_state = srv.stats()["bytes_in_use"]
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
            jid, s_ = item
            st, r = srv.wait(jid, 120.0)
            with lock:
                records.append((st, r.t_submit, r.t_start, r.t_done, s_, r.closed_interval, r.gpu_ms))
            srv.release(jid)

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    seq = [0] * n_streams
    # warm-up: one full interval of every stream (kernels compiled, attributes set, rings primed)
    warm = []
    for s_, (n, c, t, b) in enumerate(shapes):
        for m in range(jobs_per_dump):
            warm.append(srv.submit(n, c, t, b, pool, dumps[s_] if m == jobs_per_dump - 1 else None, stream_tag=s_))
    for jid in warm:
        srv.wait(jid, 300.0)
        srv.release(jid)
    clocks = ClockSampler(0)
    clocks.start()
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
        s_ = int(rng.integers(0, n_streams))
        n, c, t, b = shapes[s_]
        seq[s_] += 1
        closes = seq[s_] % jobs_per_dump == 0
        jid = srv.submit(n, c, t, b, pool, dumps[s_] if closes else None, stream_tag=s_)
        n_sub += 1
        with lock:
            pending.append((jid, s_))
    done_evt.set()
    th.join(timeout=600)
    wall = time.time() - t_start
    clk = clocks.stop()
    coalesced = srv.stats()["coalesced"]
    for s_ in range(n_streams):
        srv.close_stream(s_, 60.0)
    srv.close()
    ok = [r for r in records if r[0] == 0]
    lat = np.array([r[3] - r[1] for r in ok]) * 1e3
    t_job = np.array([shapes[r[4]][2] / CHANNEL_RATE_HZ for r in ok]) * 1e3
    dump_lat = np.array([r[3] - r[1] for r in ok if r[5]]) * 1e3
    t_dump = np.array([jobs_per_dump * shapes[r[4]][2] / CHANNEL_RATE_HZ for r in ok if r[5]]) * 1e3
    cm = sum((lambda n, c, t, b: n * (n + 1) // 2 * c * t)(*shapes[r[4]]) for r in ok)
    offered = sum(rate / n_streams * n * (n + 1) // 2 * c * t for n, c, t, b in shapes)
    line = {"metric": "serving p99 latency / real-time factor / TeraCMAC/s", "unit": "ms",
            "workload": "serve: Poisson 200 jobs/s over 8 streams with device rings and accumulators, each stream a "
                        "random array (32..512 dual-pol antennas, 128..1536 channels, 256..1024 samples per job, "
                        "4/8-bit), averaged dump every 16 jobs to pinned host memory",
            "streams": [{"n_inputs": n, "n_chan": c, "n_time": t, "bits": b} for n, c, t, b in shapes],
            "value": float(np.percentile(lat, 99)) if len(lat) else None,
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "frac_within_own_sample_time": float(np.mean(lat < t_job)) if len(lat) else None,
            "dump_p99_ms": float(np.percentile(dump_lat, 99)) if len(dump_lat) else None,
            "frac_dumps_within_dump_interval": float(np.mean(dump_lat < t_dump)) if len(dump_lat) else None,
            "jobs_submitted": n_sub, "jobs_ok": len(ok), "jobs_failed": len(records) - len(ok),
            "dumps": int(len(dump_lat)), "wall_s": wall, "jobs_per_s": len(ok) / wall,
            "real_time_factor": float(t_job.sum() / 1e3 / wall) if len(lat) else None,
            "tera_cmac_per_s": cm / wall / 1e12, "offered_tera_cmac_per_s": offered / 1e12,
            "device_state_bytes": arena_state,
            "jobs_coalesced": int(coalesced),
            "per_stream": [_stream_latency(ok, s_, shapes[s_][2] / CHANNEL_RATE_HZ * 1e3) for s_ in range(n_streams)],
            "clocks": clk,
            "latency": "submit to the job's samples accumulated on the device (closing jobs: to the dump in "
                       "pinned host memory); target p99 below the job's own sample time and every dump within "
                       "its dump interval"}
    del pool, dumps
    return line


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
    ap.add_argument("--workload", default="stream",
                    choices=["stream", "mwa32t", "large", "batch", "serve", "fx", "dump", "float", "shape"])
    ap.add_argument("--shape", default="512,128,2048,8", help="shape workload: N,C,T,BITS")
    ap.add_argument("--engine", default="tc", choices=["tc", "fp32"], help="shape workload: X engine")
    ap.add_argument("--feed", default="auto", choices=["auto", "packed", "planes", "packed_f8", "planes_fp16"],
                    help="shape workload: operand feed (packed = fp16 operands; packed_f8 = e4m3, 4-bit samples; "
                         "planes = the workspace's planes, e4m3 for 4-bit samples; planes_fp16 = fp16 planes)")
    ap.add_argument("--items", default="auto", choices=["auto", "tiles", "wide"], help="shape workload: item shape")
    ap.add_argument("--op-stages", type=int, default=0, help="shape workload: operand-ring depth (0: default)")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--no-configs", action="store_true", help="the headline workload only")
    ap.add_argument("--dump-inputs", type=int, default=1024,
                    help="inputs of the dump workload (1024 = the 1024-input array; smaller for a profiler capture)")
    ap.add_argument("--large-chans", type=int, default=1536,
                    help="channels of the large-array workload (fewer only for profiling captures)")
    args = ap.parse_args()

    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload != "stream":
        out = WORKLOADS[args.workload](args)
        out.setdefault("n_gpus", 1)
        print(json.dumps(out), flush=True)
        return

    import torch

    from paper_0906_1887_gb300 import corr, metrics, synth

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

    # FP32 CUDA-core engine on the same job (reads the packed samples; upper-triangle sub-blocks only)
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
    h2d_bytes = int(packed.numel()) * world
    d2h_bytes = int(vis.numel() * vis.element_size()) * world
    # the CPU oracle is timed on rank 0 at N = 1 only (a reported baseline, not part of the run)
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline()
    # the other workloads of the benchmark set, one after another on this GPU (N = 1 only)
    configs = {}
    if world == 1 and not args.no_configs:
        del packed, vis
        _free()
        for name in ("mwa32t", "large", "batch", "float", "fx", "serve"):
            try:
                configs[CONFIG_KEYS[name]] = WORKLOADS[name](args)
            except Exception as e:   # a failed sub-workload is reported, never hidden
                configs[CONFIG_KEYS[name]] = {"error": f"{type(e).__name__}: {e}"}
            _free()
    line = {
        "metric": "X-engine TeraCMAC/s", "value": value, "unit": "TeraCMAC/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16 operands, f32 chunk sums, exact int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_inputs": N_INPUTS, "n_chan": N_CHAN, "n_time": N_TIME,
                   "n_dumps": N_DUMPS, "sample_bits": BITS, "engine": "fused tcgen05 X stage: packed 8-bit -> fp16 in shared memory, fp32 accum, exact int64",
                   "l2": "inputs (19.7 GB per step) far larger than L2; no flush", "parallelism": f"replicas{world}"},
        "real_time_factor": rtf,
        # Table 4's measure: the signal bandwidth these CMAC rates would sustain for the paper's
        # 64-input system (B = CMAC/s / 2080); the paper's best, GP4 on a Tesla C1060, processed 6.9 MHz
        "signal_bandwidth_mhz_at_64_inputs": {"device_resident": metrics.mhz_at_64_inputs(value),
                                              "e2e": metrics.mhz_at_64_inputs(e2e_value),
                                              "paper_c1060_gp4_mhz": 6.9},
        "fp32_path": {"value": value32, "unit": "TeraCMAC/s", "ms_per_step": ms32, "speedup_tc_over_fp32": value / value32},
        "e2e": {"value": e2e_value, "unit": "TeraCMAC/s", "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": h2d_bytes,
                "d2h_bytes_per_step": d2h_bytes,
                "api": "corr_xengine_run_host (pinned host buffers, chunked copy/compute overlap)",
                "timing": "host wall clock around the synchronous call"},
        "roofline": roofline,
        "gpu_launches": args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "configs": configs,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


WORKLOADS = {"mwa32t": run_mwa32t, "large": run_large, "batch": run_batch, "serve": run_serve, "fx": run_fx,
             "dump": run_dump, "float": run_float, "shape": run_shape}
CONFIG_KEYS = {"mwa32t": "mwa32t_4bit", "large": "large1024_8bit", "batch": "batch40", "float": "float_stream",
               "fx": "fx_chain", "serve": "serve"}


if __name__ == "__main__":
    main()

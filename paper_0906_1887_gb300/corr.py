"""ctypes binding of libcorr.so (the C ABI in include/corr.h).

Argument marshalling only: every step of the X stage runs in the library's CUDA
kernels.  PyTorch is used for device memory and streams; tensors are passed as raw
device pointers.  If the library has not been built, ``lib()`` raises -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcorr.so")

OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEOUT, PENDING, EUNSUPPORTED = range(8)
ENGINE_TC, ENGINE_FP32, ENGINE_BF16X3 = 0, 1, 2
OPERANDS_AUTO, OPERANDS_PACKED, OPERANDS_PLANES, OPERANDS_PACKED_F8 = 0, 1, 2, 3
ITEMS_AUTO, ITEMS_TILES, ITEMS_WIDE = 0, 1, 2
F_COMPLEX8, F_COMPLEX4, F_REAL8 = 0, 1, 2
STATUS_NAMES = {OK: "CORR_OK", EINVAL: "CORR_EINVAL", ENOMEM: "CORR_ENOMEM", ECUDA: "CORR_ECUDA",
                EBUSY: "CORR_EBUSY", ETIMEOUT: "CORR_ETIMEOUT", PENDING: "CORR_PENDING",
                EUNSUPPORTED: "CORR_EUNSUPPORTED"}

_lib = None

_c_int, _c_i64, _c_sz, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
_P = ctypes.POINTER

# name -> (restype, argtypes); the exported surface of include/corr.h
SIGNATURES = {
    "corr_version": (_c_int, []),
    "corr_last_error": (ctypes.c_char_p, []),
    "corr_plan_create": (_c_int, [_P(_vp), _c_int, _c_int, _c_int, _c_int]),
    "corr_plan_destroy": (_c_int, [_vp]),
    "corr_plan_info": (_c_int, [_vp, _P(_c_i64), _P(_c_sz), _P(_c_sz)]),
    "corr_plan_set_tuning": (_c_int, [_vp, _c_int, _c_int]),
    "corr_plan_set_operands": (_c_int, [_vp, _c_int, _c_int]),
    "corr_workspace_size": (_c_int, [_vp, _c_int, _c_int, _P(_c_sz)]),
    "corr_unpack": (_c_int, [_vp, _vp, _c_int, _vp, _vp]),
    "corr_planes_size": (_c_int, [_vp, _c_int, _P(_c_sz)]),
    "corr_xengine_run": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _vp]),
    "corr_xengine_run_batch": (_c_int, [_vp, _vp, _c_int, _vp, _vp, _c_int, _c_int, _vp]),
    "corr_xengine_run_planes": (_c_int, [_vp, _vp, _c_int, _vp, _c_int, _c_int, _vp]),
    "corr_xengine_run_static": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int, _vp, _c_int, _vp]),
    "corr_static_check": (_c_int, [_P(_c_int), _vp]),
    "corr_xengine_run_host": (_c_int, [_vp, _vp, _c_int, _vp, _c_int, _c_int]),
    "corr_plan_check": (_c_int, [_vp, _P(_c_int)]),
    "corr_selftest_stall": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _P(_c_int)]),
    "corr_batch_create": (_c_int, [_P(_vp), _vp, _c_int, _c_int, ctypes.c_char_p]),
    "corr_batch_run": (_c_int, [_vp, _vp]),
    "corr_batch_set_shape": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int]),
    "corr_batch_info": (_c_int, [_vp, _vp]),
    "corr_batch_check": (_c_int, [_vp, _P(_c_int)]),
    "corr_batch_destroy": (_c_int, [_vp]),
    "corr_server_create": (_c_int, [_P(_vp), _c_sz, _c_int, _c_int]),
    "corr_submit": (_c_int, [_vp, _vp, _P(ctypes.c_uint64)]),
    "corr_poll": (_c_int, [_vp, ctypes.c_uint64, _vp]),
    "corr_wait": (_c_int, [_vp, ctypes.c_uint64, ctypes.c_double, _vp]),
    "corr_release": (_c_int, [_vp, ctypes.c_uint64]),
    "corr_fetch": (_c_int, [_vp, ctypes.c_uint64, _vp]),
    "corr_server_resume": (_c_int, [_vp]),
    "corr_server_get_stats": (_c_int, [_vp, _vp]),
    "corr_server_destroy": (_c_int, [_vp, ctypes.c_double]),
    "corr_server_open_stream": (_c_int, [_vp, _c_int, _vp]),
    "corr_server_close_stream": (_c_int, [_vp, _c_int, ctypes.c_double]),
    "corr_host_alloc": (_c_int, [_P(_vp), _c_sz]),
    "corr_host_free": (_c_int, [_vp]),
    "corr_dump_workspace_size": (_c_int, [_vp, _P(_c_sz)]),
    "corr_dump": (_c_int, [_vp, _vp, _c_int, _vp, _vp, _vp, _vp, _c_int, _vp]),
    "corr_xengine_run_dump": (_c_int, [_vp, _vp, _c_int, _vp, _c_int, _vp, _vp, _vp, _vp]),
    "corr_fplan_create": (_c_int, [_P(_vp), _c_int, _c_int, _c_int]),
    "corr_fplan_destroy": (_c_int, [_vp]),
    "corr_fplan_info": (_c_int, [_vp, _P(_c_int), _P(_c_int), _P(_c_sz), _P(_c_sz)]),
    "corr_fengine_run": (_c_int, [_vp, _vp, _c_int, _vp, _vp]),
    "corr_fplan_create_pfb": (_c_int, [_P(_vp), _c_int, _c_int, _c_int, _c_int, _vp]),
    "corr_fplan_taps": (_c_int, [_vp, _P(_c_int)]),
    "corr_average_host": (_c_int, [_vp, _c_sz, _c_i64, _vp]),
}


class CorrError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libcorr.so (raises if it is missing; build it with paper_0906_1887_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcorr.so not built ({LIB_PATH}); run paper_0906_1887_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().corr_last_error().decode(errors="replace")


def check(status: int, where: str):
    if status != OK:
        raise CorrError(status, where, last_error())
    return status


def _ptr(x):
    """Device/host address of a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class FPlan:
    """F-stage plan: n_inputs, n_chan channels, sample kind (F_COMPLEX8 / F_COMPLEX4 / F_REAL8)."""

    def __init__(self, n_inputs: int, n_chan: int, kind: int, n_taps: int = 0, taps=None):
        """n_taps > 0: polyphase filterbank with that many taps; taps = numpy float32 prototype of
        n_taps x transform_len values, or None for the default windowed sinc."""
        h = ctypes.c_void_p()
        if n_taps > 0:
            import numpy as np
            tp = None if taps is None else np.ascontiguousarray(taps, dtype=np.float32)
            check(lib().corr_fplan_create_pfb(ctypes.byref(h), n_inputs, n_chan, kind, n_taps,
                                              None if tp is None else tp.ctypes.data), "corr_fplan_create_pfb")
        else:
            check(lib().corr_fplan_create(ctypes.byref(h), n_inputs, n_chan, kind), "corr_fplan_create")
        self._h = h
        self.n_inputs, self.n_chan, self.kind = n_inputs, n_chan, kind
        oc, tl, ib, ob = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t(), ctypes.c_size_t()
        check(lib().corr_fplan_info(h, ctypes.byref(oc), ctypes.byref(tl), ctypes.byref(ib), ctypes.byref(ob)),
              "corr_fplan_info")
        self.n_out_chan, self.transform_len = oc.value, tl.value
        nt = ctypes.c_int()
        check(lib().corr_fplan_taps(h, ctypes.byref(nt)), "corr_fplan_taps")
        self.n_taps = nt.value
        self.in_bytes_per_frame, self.out_bytes_per_frame = ib.value, ob.value

    def run(self, time_samples, spectra, n_frames: int, stream=None):
        """time_samples: n_frames x transform_len x n_inputs packed samples; spectra: float32
        [n_frames][n_out_chan][n_inputs][2] (the X stage's float sample layout)."""
        check(lib().corr_fengine_run(self._h, _ptr(time_samples), n_frames, _ptr(spectra), _stream_handle(stream)),
              "corr_fengine_run")

    def empty_spectra(self, n_frames: int, device="cuda"):
        import torch
        return torch.empty((n_frames, self.n_out_chan, self.n_inputs, 2), dtype=torch.float32, device=device)

    def close(self):
        if self._h is not None and self._h.value:
            lib().corr_fplan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A correlation plan: n_inputs (N_I), n_chan (N_C), n_time samples per dump, sample mode."""

    def __init__(self, n_inputs: int, n_chan: int, n_time: int, sample_bits: int):
        h = ctypes.c_void_p()
        check(lib().corr_plan_create(ctypes.byref(h), n_inputs, n_chan, n_time, sample_bits), "corr_plan_create")
        self._h = h
        self.n_inputs, self.n_chan, self.n_time, self.sample_bits = n_inputs, n_chan, n_time, sample_bits

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            lib().corr_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        nb, pk, vb = ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_size_t()
        check(lib().corr_plan_info(self._h, ctypes.byref(nb), ctypes.byref(pk), ctypes.byref(vb)), "corr_plan_info")
        return nb.value, pk.value, vb.value

    @property
    def n_baselines(self) -> int:
        return self.info()[0]

    def dump(self, acc, out, n_accum: int = 1, delays=None, freqs=None, workspace=None, reset: bool = False,
             stream=None):
        """Dump step: out = acc / n_accum rotated by exp(+2 pi i nu_c (tau_i - tau_j)); optional reset.
        delays (float64 [n_inputs], s) and freqs (float64 [n_chan], Hz) are device tensors."""
        if delays is not None and workspace is None:
            import torch
            workspace = torch.empty(max(1, self.dump_workspace_size()), dtype=torch.uint8, device=delays.device)
        check(lib().corr_dump(self._h, _ptr(acc), n_accum, _ptr(delays), _ptr(freqs), _ptr(workspace), _ptr(out),
                              1 if reset else 0, _stream_handle(stream)), "corr_dump")

    def run_dump(self, packed, out, n_accum: int = 1, delays=None, freqs=None, workspace=None, n_dumps: int = 1,
                 stream=None):
        """X stage + dump step fused: out float32 [n_dumps][C][P][2] = V / n_accum, phase-corrected."""
        if delays is not None and workspace is None:
            import torch
            workspace = torch.empty(max(1, self.dump_workspace_size()), dtype=torch.uint8, device=delays.device)
        check(lib().corr_xengine_run_dump(self._h, _ptr(packed), n_dumps, _ptr(out), n_accum, _ptr(delays),
                                          _ptr(freqs), _ptr(workspace), _stream_handle(stream)),
              "corr_xengine_run_dump")

    def dump_workspace_size(self) -> int:
        b = ctypes.c_size_t()
        check(lib().corr_dump_workspace_size(self._h, ctypes.byref(b)), "corr_dump_workspace_size")
        return b.value

    def set_tuning(self, op_stages: int = 0, float_planes: int = 0):
        """Operand ring depth of the tensor-core kernel, and for BF16x3 on float samples whether the
        hi/lo split goes through planes in memory (1) or happens in the kernel where it can (0);
        results do not depend on either."""
        check(lib().corr_plan_set_tuning(self._h, op_stages, float_planes), "corr_plan_set_tuning")

    def set_operands(self, operands: int = OPERANDS_AUTO, items: int = ITEMS_AUTO):
        """Operand feed of the tensor-core engine (packed samples into fp16 or, for 4-bit samples,
        e4m3 operands, or fp16 planes) and the plane feed's work-item shape; results do not
        depend on either."""
        check(lib().corr_plan_set_operands(self._h, operands, items), "corr_plan_set_operands")

    def workspace_size(self, engine: int, n_dumps: int = 1) -> int:
        b = ctypes.c_size_t()
        check(lib().corr_workspace_size(self._h, engine, n_dumps, ctypes.byref(b)), "corr_workspace_size")
        return b.value

    def planes_size(self, n_dumps: int = 1) -> int:
        """Bytes of the sample planes corr_unpack writes for n_dumps dumps."""
        b = ctypes.c_size_t()
        check(lib().corr_planes_size(self._h, n_dumps, ctypes.byref(b)), "corr_planes_size")
        return b.value

    def unpack(self, packed, planes, n_dumps: int = 1, stream=None):
        check(lib().corr_unpack(self._h, _ptr(packed), n_dumps, _ptr(planes), _stream_handle(stream)), "corr_unpack")

    def run(self, packed, vis, workspace=None, accumulate: bool = False, engine: int = ENGINE_TC,
            n_dumps: int = 1, stream=None):
        check(lib().corr_xengine_run_batch(self._h, _ptr(packed), n_dumps, _ptr(vis), _ptr(workspace),
                                           1 if accumulate else 0, engine, _stream_handle(stream)),
              "corr_xengine_run_batch")

    def run_planes(self, planes, vis, accumulate: bool = False, engine: int = ENGINE_TC, n_dumps: int = 1,
                   stream=None):
        check(lib().corr_xengine_run_planes(self._h, _ptr(planes), n_dumps, _ptr(vis), 1 if accumulate else 0,
                                            engine, _stream_handle(stream)), "corr_xengine_run_planes")

    def run_host(self, host_packed, host_vis, n_dumps: int = 1, dumps_per_chunk: int = 0,
                 engine: int = ENGINE_TC):
        """End to end from host buffers: pipelined copy in / X stage / copy out (returns when done)."""
        check(lib().corr_xengine_run_host(self._h, _ptr(host_packed), n_dumps, _ptr(host_vis), dumps_per_chunk,
                                          engine), "corr_xengine_run_host")

    def check_device(self) -> int:
        code = ctypes.c_int(0)
        st = lib().corr_plan_check(self._h, ctypes.byref(code))
        if st not in (OK, ETIMEOUT):
            check(st, "corr_plan_check")
        return code.value

    def selftest_stall(self, packed, vis, stall_item: int, wait_limit_ms: int = 100):
        """Make one bounded device wait run out on purpose; returns (status, device_error)."""
        code = ctypes.c_int(0)
        st = lib().corr_selftest_stall(self._h, _ptr(packed), _ptr(vis), stall_item, wait_limit_ms,
                                       ctypes.byref(code))
        return st, code.value

    # ---- torch conveniences (allocation only) ----
    def vis_dtype(self):
        import torch
        return torch.float32 if self.sample_bits == 32 else torch.int64

    def empty_vis(self, n_dumps: int = 1, device="cuda"):
        import torch
        return torch.empty((n_dumps, self.n_chan, self.n_baselines, 2), dtype=self.vis_dtype(), device=device)

    def empty_workspace(self, engine: int, n_dumps: int = 1, device="cuda"):
        import torch
        n = self.workspace_size(engine, n_dumps)
        return torch.empty(max(n, 16), dtype=torch.uint8, device=device) if n else None


class JobDesc(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int), ("n_chan", ctypes.c_int), ("n_time", ctypes.c_int),
                ("sample_bits", ctypes.c_int), ("packed", ctypes.c_void_p), ("vis", ctypes.c_void_p)]


class BatchStats(ctypes.Structure):
    _fields_ = [("n_jobs", ctypes.c_int), ("n_launches", ctypes.c_int), ("graph", ctypes.c_int),
                ("tuned", ctypes.c_int), ("n_items", ctypes.c_int64), ("cmacs", ctypes.c_double),
                ("op_stages", ctypes.c_int), ("pair_cpi", ctypes.c_int), ("order", ctypes.c_int),
                ("tune_ms", ctypes.c_float), ("plane_min_nb", ctypes.c_int), ("plane_bytes", ctypes.c_size_t),
                ("wide", ctypes.c_int), ("plane_splits", ctypes.c_int)]


BATCH_GRAPH, BATCH_AUTOTUNE, BATCH_ACCUMULATE, BATCH_PLANES = 1, 2, 4, 8


class Batch:
    """Many uneven jobs in one persistent launch per sample mode (optionally tuned, graph-captured).

    ``jobs``: sequence of (n_inputs, n_chan, n_time, sample_bits, packed_tensor, vis_tensor).
    """

    def __init__(self, jobs, flags: int = 0, tune_cache: str | None = None):
        arr = (JobDesc * len(jobs))()
        for k, (n, c, t, bits, packed, vis) in enumerate(jobs):
            arr[k] = JobDesc(n, c, t, bits, _ptr(packed), _ptr(vis))
        self._keep = list(jobs)
        h = ctypes.c_void_p()
        check(lib().corr_batch_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), len(jobs), flags,
                                      tune_cache.encode() if tune_cache else None), "corr_batch_create")
        self._h = h

    def run(self, stream=None):
        check(lib().corr_batch_run(self._h, _stream_handle(stream)), "corr_batch_run")

    def set_shape(self, op_stages: int = 0, pair_cpi: int = 2, order: int = 0, plane_min_nb: int = 0, wide: int = 1,
                  plane_splits: int = 1):
        """Launch shape chosen by the caller instead of the tuner (results do not depend on it)."""
        check(lib().corr_batch_set_shape(self._h, op_stages, pair_cpi, order, plane_min_nb, wide, plane_splits),
              "corr_batch_set_shape")

    def info(self) -> dict:
        st = BatchStats()
        check(lib().corr_batch_info(self._h, ctypes.byref(st)), "corr_batch_info")
        return {f: getattr(st, f) for f, _ in BatchStats._fields_}

    def check_device(self) -> int:
        code = ctypes.c_int(0)
        st = lib().corr_batch_check(self._h, ctypes.byref(code))
        if st not in (OK, ETIMEOUT):
            check(st, "corr_batch_check")
        return code.value

    def close(self):
        if self._h is not None and self._h.value:
            lib().corr_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ServerJob(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int), ("n_chan", ctypes.c_int), ("n_time", ctypes.c_int),
                ("sample_bits", ctypes.c_int), ("host_packed", ctypes.c_void_p), ("host_vis", ctypes.c_void_p),
                ("stream_tag", ctypes.c_int)]


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("gpu_ms", ctypes.c_float), ("d_vis", ctypes.c_void_p),
                ("closed_interval", ctypes.c_int), ("n_accum", ctypes.c_int64)]


class StreamDesc(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int), ("n_chan", ctypes.c_int), ("n_time", ctypes.c_int),
                ("sample_bits", ctypes.c_int), ("ring_slots", ctypes.c_int), ("jobs_per_dump", ctypes.c_int),
                ("dump_mode", ctypes.c_int), ("d_delays", ctypes.c_void_p), ("d_freqs", ctypes.c_void_p)]


STREAM_DUMP_SUMS, STREAM_DUMP_AVERAGED = 0, 1


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("cancelled", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("running", ctypes.c_int64), ("arena_bytes", ctypes.c_size_t), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("open_streams", ctypes.c_int64), ("coalesced", ctypes.c_int64)]


SERVER_START_PAUSED = 1


class Server:
    """Real-time serving loop: submit jobs (host buffers), poll or wait by id."""

    def __init__(self, hbm_budget_bytes: int, n_streams: int = 8, flags: int = 0):
        h = ctypes.c_void_p()
        check(lib().corr_server_create(ctypes.byref(h), int(hbm_budget_bytes), n_streams, flags),
              "corr_server_create")
        self._h = h
        self._keep_stream = {}

    def submit(self, n_inputs, n_chan, n_time, sample_bits, host_packed, host_vis=None, stream_tag=0) -> int:
        d = ServerJob(n_inputs, n_chan, n_time, sample_bits, _ptr(host_packed), _ptr(host_vis), stream_tag)
        jid = ctypes.c_uint64(0)
        check(lib().corr_submit(self._h, ctypes.byref(d), ctypes.byref(jid)), "corr_submit")
        return jid.value

    def open_stream(self, stream_tag: int, n_inputs: int, n_chan: int, n_time: int, sample_bits: int,
                    ring_slots: int = 4, jobs_per_dump: int = 1, dump_mode: int = STREAM_DUMP_SUMS,
                    delays=None, freqs=None):
        """Give stream_tag device state: a ring of sample slots and accumulators its jobs add into,
        dumped every jobs_per_dump jobs (delays/freqs: float64 device tensors, averaged mode)."""
        d = StreamDesc(n_inputs, n_chan, n_time, sample_bits, ring_slots, jobs_per_dump, dump_mode,
                       _ptr(delays), _ptr(freqs))
        self._keep_stream[stream_tag] = (delays, freqs)
        check(lib().corr_server_open_stream(self._h, stream_tag, ctypes.byref(d)), "corr_server_open_stream")

    def close_stream(self, stream_tag: int, drain_timeout_s: float = 30.0) -> int:
        st = lib().corr_server_close_stream(self._h, stream_tag, float(drain_timeout_s))
        if st == EINVAL:
            check(st, "corr_server_close_stream")
        self._keep_stream.pop(stream_tag, None)
        return st

    def poll(self, job_id: int):
        r = JobResult()
        st = lib().corr_poll(self._h, job_id, ctypes.byref(r))
        if st == EINVAL:
            check(st, "corr_poll")
        return st, r

    def wait(self, job_id: int, timeout_s: float):
        r = JobResult()
        st = lib().corr_wait(self._h, job_id, float(timeout_s), ctypes.byref(r))
        if st == EINVAL:
            check(st, "corr_wait")
        return st, r

    def release(self, job_id: int):
        check(lib().corr_release(self._h, job_id), "corr_release")

    def fetch(self, job_id: int, host_vis):
        """Copy a device-resident result (job submitted without host_vis) into host memory."""
        check(lib().corr_fetch(self._h, job_id, _ptr(host_vis)), "corr_fetch")

    def resume(self):
        check(lib().corr_server_resume(self._h), "corr_server_resume")

    def stats(self) -> dict:
        st = ServerStats()
        check(lib().corr_server_get_stats(self._h, ctypes.byref(st)), "corr_server_get_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self, drain_timeout_s: float = 30.0) -> int:
        st = OK
        if self._h is not None and self._h.value:
            st = lib().corr_server_destroy(self._h, float(drain_timeout_s))
        self._h = None
        return st

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> int:
    return int(lib().corr_version())


def average_host(vis_int64, n_accum: int):
    """int64 visibilities (numpy) divided by the number of accumulated dumps, in float64, on the host."""
    import numpy as np
    v = np.ascontiguousarray(vis_int64, dtype=np.int64)
    out = np.empty(v.shape, dtype=np.float64)
    check(lib().corr_average_host(v.ctypes.data, v.size, int(n_accum), out.ctypes.data), "corr_average_host")
    return out

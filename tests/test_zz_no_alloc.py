"""corr_xengine_run_static: the X stage for callers that cannot allocate device memory.

Such callers (a real-time loop that must not pay cudaMalloc's device-wide
synchronisation, or a framework that owns all device memory) still pass the packed
samples and the visibility buffer; the unpacked planes live in a fixed array inside the
library.  This file is collected last on purpose.  It calls the entry point through the
C ABI twice in a row -- the second call on a different problem, so stale contents of the
shared array would show -- and compares each result with corr_xengine_run's and with the
CPU oracle (bit-exact, as every integer-path test); a third call accumulates into the
second's output.  After every call the status block is read back through
corr_static_check and must be clear.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0906_1887_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _plan_path(packed, n, c, t, bits):
    from paper_0906_1887_gb300 import corr
    plan = corr.Plan(n, c, t, bits)
    x = torch.from_numpy(packed.reshape(-1).view(np.uint8)).cuda()
    vis = plan.empty_vis(1, "cuda")
    plan.run(x, vis, plan.empty_workspace(corr.ENGINE_TC, 1), engine=corr.ENGINE_TC)
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    out = vis.cpu().numpy()[0]
    plan.close()
    return out


def _static_check(lib, stream):
    code = ctypes.c_int(-1)
    st = lib.corr_static_check(ctypes.byref(code), ctypes.c_void_p(stream))
    assert st == 0 and code.value == 0, (st, code.value, lib.corr_last_error())


def _static_path(lib, packed, n, c, t, bits, vis=None, accumulate=0):
    x = torch.from_numpy(packed.reshape(-1).view(np.uint8)).cuda()
    if vis is None:
        vis = torch.full((c, n * (n + 1) // 2, 2), -3, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.corr_xengine_run_static(ctypes.c_void_p(x.data_ptr()), n, c, t, bits, ctypes.c_void_p(vis.data_ptr()),
                                     accumulate, ctypes.c_void_p(stream))
    assert st == 0, lib.corr_last_error()
    torch.cuda.synchronize()
    _static_check(lib, stream)
    return vis


def test_static_entry_point_matches_plan_path_and_oracle_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_1887_gb300 import corr
    lib = corr.lib()
    cases = [(64, 128, 512, 4, 1000), (100, 5, 300, 8, 77)]     # (N, C, T, bits, seed)
    vis = None
    for n, c, t, bits, seed in cases:
        lo, hi = (-8, 7) if bits == 4 else (-128, 127)
        re, im = synth.uniform_ints(seed, t, c, n, lo, hi)
        packed = synth.pack(re, im, bits)
        ref = oracle.xcorr_int(packed, n, c, t, bits)
        want = _plan_path(packed, n, c, t, bits)
        vis = _static_path(lib, packed, n, c, t, bits)
        got = vis.cpu().numpy()
        assert np.array_equal(got, want), (n, c, t, bits)
        assert np.array_equal(got, ref), (n, c, t, bits)
    # accumulate = 1 adds the same dump again into the last call's int64 output
    _static_path(lib, packed, n, c, t, bits, vis=vis, accumulate=1)
    assert np.array_equal(vis.cpu().numpy(), 2 * ref)


def test_static_entry_point_rejects_oversized_dump():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_1887_gb300 import corr
    lib = corr.lib()
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    vis = torch.zeros(16, dtype=torch.int64, device="cuda")
    # 64 inputs x 4096 channels x 1024 samples needs 4096 x 1 x 128 x 1024 x 2 bytes = 1 GiB
    # of planes, more than the 64 MiB (67108864-byte) array
    st = lib.corr_xengine_run_static(ctypes.c_void_p(x.data_ptr()), 64, 4096, 1024, 8,
                                     ctypes.c_void_p(vis.data_ptr()), 0, None)
    assert st == corr.EINVAL
    assert b"67108864" in lib.corr_last_error()
    # sizes whose products would wrap a 64-bit byte count are refused before any launch
    st = lib.corr_xengine_run_static(ctypes.c_void_p(x.data_ptr()), 8192, 1 << 30, (1 << 31) - 65, 8,
                                     ctypes.c_void_p(vis.data_ptr()), 0, None)
    assert st == corr.EINVAL

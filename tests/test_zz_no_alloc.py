"""corr_xengine_run_static: the X stage for callers that cannot allocate device memory.

Such callers (a real-time loop that must not pay cudaMalloc's device-wide
synchronisation, or a framework that owns all device memory) still pass the packed
samples and the visibility buffer; the unpacked planes live in a fixed array inside the
library.  This file is collected last on purpose.  It calls the entry point through the
C ABI twice in a row -- the second call on a different problem, so stale contents of the
shared array would show -- and compares each result with corr_xengine_run's (bit-exact,
as every integer-path test).
"""
import ctypes

import numpy as np
import pytest

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


def _static_path(lib, packed, n, c, t, bits):
    x = torch.from_numpy(packed.reshape(-1).view(np.uint8)).cuda()
    vis = torch.full((c, n * (n + 1) // 2, 2), -3, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.corr_xengine_run_static(ctypes.c_void_p(x.data_ptr()), n, c, t, bits, ctypes.c_void_p(vis.data_ptr()),
                                     0, ctypes.c_void_p(stream))
    assert st == 0, lib.corr_last_error()
    torch.cuda.synchronize()
    return vis.cpu().numpy()


def test_static_entry_point_matches_plan_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_1887_gb300 import corr
    lib = corr.lib()
    cases = [(64, 128, 512, 4, 1000), (100, 5, 300, 8, 77)]     # (N, C, T, bits, seed)
    for n, c, t, bits, seed in cases:
        lo, hi = (-8, 7) if bits == 4 else (-128, 127)
        re, im = synth.uniform_ints(seed, t, c, n, lo, hi)
        packed = synth.pack(re, im, bits)
        want = _plan_path(packed, n, c, t, bits)
        got = _static_path(lib, packed, n, c, t, bits)
        assert np.array_equal(got, want), (n, c, t, bits)


def test_static_entry_point_rejects_oversized_dump():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_1887_gb300 import corr
    lib = corr.lib()
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    vis = torch.zeros(16, dtype=torch.int64, device="cuda")
    # 64 inputs x 4096 channels x 1024 samples needs 128 MiB of planes (> 64 MiB)
    st = lib.corr_xengine_run_static(ctypes.c_void_p(x.data_ptr()), 64, 4096, 1024, 8,
                                     ctypes.c_void_p(vis.data_ptr()), 0, None)
    assert st == corr.EINVAL
    assert b"64 MiB" in lib.corr_last_error() or b"67108864" in lib.corr_last_error()

"""Parity at the full workload sizes, on sampled channels the oracle computes one by one.

The CUDA path runs the whole dump in the same launch configuration the benchmark uses;
the oracle recomputes a seeded sample of channels.
"""
import numpy as np
import pytest

import oracle
from paper_0906_1887_gb300 import synth
from _gpu_helpers import check_bf16x3, run_engine

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name,nsample", [("stream64_8bit", 24), ("large1024_8bit", 3)])
def test_fullsize_sampled_channels(name, nsample):
    re, im, bits, (n, c, t) = synth.workload(name)
    p = synth.pack(re, im, bits)
    del re, im
    v = run_engine(p, n, c, t, bits, 0)[0]
    chans = np.random.default_rng(7).choice(c, size=nsample, replace=False)
    ref = oracle.xcorr_int(p, n, c, t, bits, chans=chans)
    for k, ch in enumerate(chans):
        assert np.array_equal(v[ch], ref[k]), f"channel {ch}"
    # properties that hold for every channel: autos real and non-negative
    auto_idx = [i * n - i * (i - 1) // 2 for i in range(n)]
    assert (v[:, auto_idx, 1] == 0).all() and (v[:, auto_idx, 0] >= 0).all()


def test_fullsize_float_bf16x3_sampled_channels():
    # the float variant of the 64-input stream (one dump): BF16x3 with the hi/lo split in the
    # kernel, bit-identical to the planes path, and every element of sampled channels within the
    # BF16x3 bound against float64
    n, c, t = 64, 768, 1000
    re, im = synth.correlated_gaussian(2500, t, c, n, 16.0, 0.1, as_float=True)
    x = synth.packf32(re, im)
    del re, im
    fused = run_engine(x, n, c, t, 32, 2, tuning=(0, 0))[0]
    planes = run_engine(x, n, c, t, 32, 2, tuning=(0, 1))[0]
    assert np.array_equal(fused, planes)
    chans = np.random.default_rng(8).choice(c, size=6, replace=False)
    err, _ = check_bf16x3(fused[chans], x, n, c, t, chans=chans)
    assert err <= 1e-4


def test_headline_full_launch_sampled_dumps():
    # the benchmark's whole job in its own launch configuration: 200 dumps of 64 inputs x 768
    # channels x 1000 samples through one fused launch, inputs from the same seeded device
    # generator; 24 seeded (dump, channel) pairs recomputed by the oracle from the same bytes
    from paper_0906_1887_gb300 import corr
    n, c, t, d = 64, 768, 1000, 200
    dev = torch.device("cuda:0")
    packed = synth.torch_correlated_gaussian_packed8(d, t, c, n, 16.0, 0.1, 2000, dev)
    plan = corr.Plan(n, c, t, 8)
    vis = plan.empty_vis(d, dev)
    vis.fill_(-9)
    plan.run(packed, vis, plan.empty_workspace(corr.ENGINE_TC, d, dev), engine=corr.ENGINE_TC, n_dumps=d)
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    rng = np.random.default_rng(11)
    picks = [(int(rng.integers(0, d)), int(rng.integers(0, c))) for _ in range(24)]
    for dd, ch in picks:
        one = packed[dd, :, ch:ch + 1].contiguous().cpu().numpy()          # [T][1][N][2] bytes
        ref = oracle.xcorr_int(one, n, 1, t, 8)[0]
        assert np.array_equal(vis[dd, ch].cpu().numpy(), ref), (dd, ch)
    auto_idx = torch.tensor([i * n - i * (i - 1) // 2 for i in range(n)], device=dev)
    autos = vis.index_select(2, auto_idx)
    assert bool((autos[..., 1] == 0).all()) and bool((autos[..., 0] >= 0).all())
    # the FP32 CUDA-core engine on the same 200 dumps, as the benchmark runs it: both engines are
    # exact on integer samples, so every one of the 200 x 768 x 2080 results must agree
    vis32 = plan.empty_vis(d, dev)
    vis32.fill_(-7)
    plan.run(packed, vis32, None, engine=corr.ENGINE_FP32, n_dumps=d)
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    assert torch.equal(vis32, vis)
    plan.close()


def test_large_array_fp32_equals_tensor_core_full_dump():
    # one full dump of the 1024-input array (1536 channels x 256 samples): the plane-fed
    # tensor-core path and the FP32 engine, all 1536 x 524800 results equal; two channels
    # against the oracle
    from paper_0906_1887_gb300 import corr
    n, c, t = 1024, 1536, 256
    dev = torch.device("cuda:0")
    packed = synth.torch_correlated_gaussian_packed8(1, t, c, n, 8.0, 0.0, 3000, dev)
    plan = corr.Plan(n, c, t, 8)
    vis_tc = plan.empty_vis(1, dev)
    plan.run(packed, vis_tc, plan.empty_workspace(corr.ENGINE_TC, 1, dev), engine=corr.ENGINE_TC)
    vis32 = plan.empty_vis(1, dev)
    plan.run(packed, vis32, None, engine=corr.ENGINE_FP32)
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    assert torch.equal(vis_tc, vis32)
    for ch in (5, 1400):
        one = packed[0, :, ch:ch + 1].contiguous().cpu().numpy()
        ref = oracle.xcorr_int(one, n, 1, t, 8)[0]
        assert np.array_equal(vis_tc[0, ch].cpu().numpy(), ref), ch
    plan.close()

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
    plan.close()

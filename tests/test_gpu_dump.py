"""GPU parity of the dump step with post-correlation phase correction (Fig. 1, Sec. 2).

The kernel rounds each accumulator to float32, scales it by 1/n_accum and rotates it by two
float32 phasors (formed in double precision, then rounded): each of those steps adds at most
a couple of units of 2^-24 relative to |V|, so every element must lie within 8 x 2^-24 |V|
of the float64 oracle (which forms each baseline's phase from the delay difference directly).
"""
import numpy as np
import pytest

import oracle
from oracle import dump as odump
from oracle import fstage
from paper_0906_1887_gb300 import synth
from _gpu_helpers import int_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EPS = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_1887_gb300 import corr
    corr.lib()


def _check(got, ref):
    mag = np.hypot(ref[..., 0], ref[..., 1])
    err = np.hypot(got[..., 0] - ref[..., 0], got[..., 1] - ref[..., 1])
    assert np.all(err <= 8 * EPS * mag + 1e-30), float((err / np.maximum(mag, 1e-30)).max())


@pytest.mark.parametrize("n,c,t,bits,n_accum", [(1, 1, 64, 8, 1), (5, 3, 100, 8, 3), (64, 7, 256, 8, 1),
                                                (130, 2, 70, 4, 5), (64, 1, 1000, 8, 7)])
def test_dump_matches_oracle(n, c, t, bits, n_accum):
    from paper_0906_1887_gb300 import corr
    rng = np.random.default_rng(n + c)
    p = int_case(400 + n, n, c, t, bits)
    plan = corr.Plan(n, c, t, bits)
    acc = torch.from_numpy(oracle.xcorr_int(p, n, c, t, bits)).cuda()
    tau = rng.normal(0, 2e-6, n)                     # up to ~ thousands of cycles of phase
    nu = 1.5e8 + 1e4 * np.arange(c)
    out = torch.empty((c, plan.n_baselines, 2), dtype=torch.float32, device="cuda")
    plan.dump(acc, out, n_accum, torch.from_numpy(tau).cuda(), torch.from_numpy(nu).cuda())
    torch.cuda.synchronize()
    ref = odump.dump_corrected(acc.cpu().numpy(), n_accum, tau, nu)
    _check(out.cpu().numpy().astype(np.float64), ref)
    # the accumulators are untouched without reset
    assert np.array_equal(acc.cpu().numpy(), oracle.xcorr_int(p, n, c, t, bits))
    plan.close()


def test_dump_without_delays_and_with_reset():
    from paper_0906_1887_gb300 import corr
    n, c, t = 33, 4, 300
    p = int_case(9, n, c, t, 8)
    plan = corr.Plan(n, c, t, 8)
    ref_acc = oracle.xcorr_int(p, n, c, t, 8)
    acc = torch.from_numpy(ref_acc).cuda()
    out = torch.empty((c, plan.n_baselines, 2), dtype=torch.float32, device="cuda")
    plan.dump(acc, out, 2, reset=True)
    torch.cuda.synchronize()
    _check(out.cpu().numpy().astype(np.float64), ref_acc / 2.0)
    assert not acc.cpu().numpy().any()
    plan.close()


def test_dump_of_float_accumulators_point_source():
    # FX-chain visibilities (float plan): a point source behind known delays comes out real
    # and equal on every baseline after the correction
    from paper_0906_1887_gb300 import corr
    rng = np.random.default_rng(4)
    N, C, T = 8, 16, 32
    nu = 1.8e8 + 1e4 * np.arange(C)
    tau = rng.normal(0, 3e-7, N)
    S = rng.normal(size=(T, C)) + 1j * rng.normal(size=(T, C))
    X = S[:, :, None] * np.exp(-2j * np.pi * nu[None, :, None] * tau[None, None, :])
    samples = torch.from_numpy(fstage.spectra_as_float32_samples(X)).cuda()
    plan = corr.Plan(N, C, T, 32)
    vis = plan.empty_vis(1, "cuda")
    ws = plan.empty_workspace(corr.ENGINE_FP32, 1, "cuda")
    plan.run(samples, vis, ws, engine=corr.ENGINE_FP32)
    out = torch.empty((C, plan.n_baselines, 2), dtype=torch.float32, device="cuda")
    plan.dump(vis[0], out, 1, torch.from_numpy(tau).cuda(), torch.from_numpy(nu).cuda())
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    power = (np.abs(S) ** 2).sum(0)
    assert np.allclose(got[..., 0], power[:, None], rtol=2e-6)
    assert np.abs(got[..., 1]).max() <= 2e-6 * power.max()
    plan.close()


def test_dump_rejects_bad_arguments():
    from paper_0906_1887_gb300 import corr
    plan = corr.Plan(4, 2, 64, 8)
    acc = torch.zeros((2, plan.n_baselines, 2), dtype=torch.int64, device="cuda")
    out = torch.empty((2, plan.n_baselines, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(corr.CorrError):
        plan.dump(acc, out, 0)
    tau = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(corr.CorrError):
        plan.dump(acc, out, 1, delays=tau, freqs=None)
    plan.close()


# ---- the dump step fused into the tensor-core kernel's epilogue ----

@pytest.mark.parametrize("n,c,t,bits,n_dumps,n_accum,delays", [
    (64, 5, 1000, 8, 1, 1, True), (64, 4, 1024, 8, 2, 3, False), (136, 3, 200, 8, 1, 1, True),
    (16, 4, 300, 4, 3, 2, True), (192, 2, 256, 8, 2, 1, True), (8, 3, 64, 8, 1, 5, False),
    # 4-bit samples take e4m3 operands here too: single and multi-block, tails around 128 samples
    (64, 6, 500, 4, 2, 4, True), (128, 2, 129, 4, 1, 1, True),
])
def test_fused_dump_matches_oracle(n, c, t, bits, n_dumps, n_accum, delays):
    from paper_0906_1887_gb300 import corr
    rng = np.random.default_rng(n * 7 + t)
    dumps = [int_case(900 + n + k, n, c, t, bits) for k in range(n_dumps)]
    plan = corr.Plan(n, c, t, bits)
    x = torch.from_numpy(np.concatenate(dumps).view(np.uint8).reshape(-1).copy()).cuda()
    out = torch.full((n_dumps, c, plan.n_baselines, 2), float("nan"), dtype=torch.float32, device="cuda")
    tau = rng.normal(0, 2e-6, n) if delays else np.zeros(n)
    nu = 1.5e8 + 1e4 * np.arange(c)
    if delays:
        plan.run_dump(x, out, n_accum, torch.from_numpy(tau).cuda(), torch.from_numpy(nu).cuda(), n_dumps=n_dumps)
    else:
        plan.run_dump(x, out, n_accum, n_dumps=n_dumps)
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    got = out.cpu().numpy().astype(np.float64)
    for k in range(n_dumps):
        ref = odump.dump_corrected(oracle.xcorr_int(dumps[k], n, c, t, bits), n_accum, tau, nu)
        _check(got[k], ref)
    plan.close()


def test_tuning_rejects_bad_values():
    from paper_0906_1887_gb300 import corr
    plan = corr.Plan(64, 2, 64, 8)
    for bad in (-1, 17):
        with pytest.raises(corr.CorrError):
            plan.set_tuning(bad)
    plan.close()


def test_fused_dump_refuses_what_it_cannot_do():
    from paper_0906_1887_gb300 import corr
    plan = corr.Plan(64, 2, 1025, 8)           # two exact chunks per dump
    x = torch.zeros(1025 * 2 * 64 * 2, dtype=torch.uint8, device="cuda")
    out = torch.empty((2, plan.n_baselines, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(corr.CorrError):
        plan.run_dump(x, out, 1)
    plan.close()
    plan = corr.Plan(66, 2, 64, 8)             # packed rows of 132 bytes: not TMA-addressable
    x = torch.zeros(64 * 2 * 66 * 2, dtype=torch.uint8, device="cuda")
    out = torch.empty((2, plan.n_baselines, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(corr.CorrError):
        plan.run_dump(x, out, 1)
    plan.close()

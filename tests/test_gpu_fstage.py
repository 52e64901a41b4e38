"""GPU parity of the F stage (Sec. 2, Sec. 4) and of the FX chain, through the C ABI.

F stage: the float32 spectra of every (frame, input) against the complex128 oracle, in
relative L2 norm.  A radix-2/4 FFT in float32 with correctly rounded twiddles has a
normwise error of a small multiple of 2^-24 log2 L; the bound used is 4 x 2^-24 x log2 L
(a CPU model of the kernel's stages in complex64 stays below 1.2e-7 for L up to 4096).
All-zero blocks (padded inputs) must come out exactly zero.

FX chain: GPU F stage -> GPU X stage on the spectra, against the oracle's complex128 F and
X stages, in the normwise metric max |V - V64| / sqrt(V64_ii V64_jj): each spectrum enters
V twice, so the F-stage bound counts twice, plus the X engine's own bound (1e-6 for FP32;
for BF16x3 the largest normwise value of its per-element bound, oracle/precision.py).  The
BF16x3 X stage is also held, element by element, to that bound on the spectra the GPU F stage
produced.
"""
import math

import numpy as np
import pytest

from oracle import fstage
from paper_0906_1887_gb300 import synth
from _gpu_helpers import check_bf16x3, normwise_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KIND_ID = {"c8": 0, "c4": 1, "r8": 2}
EPS = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_1887_gb300 import corr
    corr.lib()


def _time_samples(seed, n_samples, n_inputs, kind):
    lo, hi = (-8, 7) if kind == "c4" else (-128, 127)
    re, im = synth.uniform_ints(seed, n_samples, 1, n_inputs, lo, hi)
    if kind == "r8":
        return synth.pack_real8(re[:, 0, :])
    return synth.pack(re, im, 8 if kind == "c8" else 4)


def _run_f(packed, n_inputs, n_chan, n_frames, kind):
    from paper_0906_1887_gb300 import corr
    fp = corr.FPlan(n_inputs, n_chan, KIND_ID[kind])
    x = torch.from_numpy(np.ascontiguousarray(packed).view(np.uint8).reshape(-1).copy()).cuda()
    spec = fp.empty_spectra(n_frames)
    spec.fill_(float("nan"))   # every element must be written
    fp.run(x, spec, n_frames)
    torch.cuda.synchronize()
    out = spec.cpu().numpy()
    fp.close()
    return out[..., 0].astype(np.float64) + 1j * out[..., 1]


def _check_spectra(got, ref, L):
    bound = 4 * EPS * math.log2(L)
    for f in range(ref.shape[0]):
        for n in range(ref.shape[2]):
            r = ref[f, :, n]
            g = got[f, :, n]
            nr = np.linalg.norm(r)
            if nr == 0:
                assert np.all(g == 0)
            else:
                assert np.linalg.norm(g - r) / nr <= bound, (f, n, np.linalg.norm(g - r) / nr, bound)


CASES = [  # (kind, n_chan, n_inputs, n_frames): every transform length 8 .. 4096, ragged inputs
    ("c8", 8, 1, 1), ("c8", 16, 3, 2), ("c8", 32, 64, 3), ("c8", 128, 64, 5), ("c8", 128, 70, 2),
    ("c8", 256, 5, 2), ("c8", 1024, 33, 1), ("c8", 4096, 2, 2),
    ("c4", 8, 7, 3), ("c4", 64, 64, 2), ("c4", 128, 130, 1), ("c4", 2048, 3, 1),
    ("r8", 4, 2, 2), ("r8", 64, 64, 2), ("r8", 128, 9, 3), ("r8", 2048, 1, 1),
    # L >= 512 with whole groups of 4 inputs: the 4-input vector loads (8 bytes for complex
    # 8-bit, 4 for the 1-byte kinds) and L = 2048 with pairs
    ("c8", 512, 8, 2), ("c8", 1024, 12, 2), ("c4", 1024, 20, 2), ("r8", 256, 8, 2), ("c8", 2048, 6, 1),
]


@pytest.mark.parametrize("kind,n_chan,n_inputs,n_frames", CASES)
def test_fstage_matches_oracle(kind, n_chan, n_inputs, n_frames):
    L = fstage.transform_length(n_chan, kind)
    p = _time_samples(100 + n_chan + n_inputs, n_frames * L, n_inputs, kind)
    got = _run_f(p, n_inputs, n_chan, n_frames, kind)
    ref = fstage.fstage(p, n_inputs, n_chan, n_frames, kind)
    assert got.shape == ref.shape
    _check_spectra(got, ref, L)


@pytest.mark.parametrize("kind,n_chan,n_inputs", [("c8", 512, 8), ("c4", 1024, 8), ("c8", 128, 64)])
def test_fstage_unaligned_samples(kind, n_chan, n_inputs):
    # samples starting 2 bytes past an 8-byte boundary: the kernel falls back to one load per
    # sample, with the same result
    from paper_0906_1887_gb300 import corr
    L = fstage.transform_length(n_chan, kind)
    F = 2
    p = _time_samples(55 + n_chan, F * L, n_inputs, kind)
    raw = np.ascontiguousarray(p).view(np.uint8).reshape(-1)
    buf = torch.zeros(raw.size + 16, dtype=torch.uint8, device="cuda")
    buf[2:2 + raw.size].copy_(torch.from_numpy(raw.copy()))
    x = buf[2:2 + raw.size]
    assert x.data_ptr() % 8 == 2
    fp = corr.FPlan(n_inputs, n_chan, KIND_ID[kind])
    spec = fp.empty_spectra(F)
    spec.fill_(float("nan"))
    fp.run(x, spec, F)
    torch.cuda.synchronize()
    out = spec.cpu().numpy()
    fp.close()
    got = out[..., 0].astype(np.float64) + 1j * out[..., 1]
    assert np.array_equal(got, _run_f(p, n_inputs, n_chan, F, kind))
    _check_spectra(got, fstage.fstage(p, n_inputs, n_chan, F, kind), L)


def test_fstage_tone_lands_in_its_channel():
    # an integer tone at bin L/4 on input 1 only: one channel of one input carries A L
    n_chan, N, F = 128, 4, 2
    s = np.arange(F * n_chan)
    tone = np.array([1, 1j, -1, -1j])[s % 4] * 100
    re = np.zeros((F * n_chan, 1, N), np.int16); im = np.zeros_like(re)
    re[:, 0, 1] = tone.real.round(); im[:, 0, 1] = tone.imag.round()
    got = _run_f(synth.pack(re, im, 8), N, n_chan, F, "c8")
    mag = np.abs(got)
    assert np.allclose(mag[:, n_chan // 4, 1], 100 * n_chan, rtol=1e-6)
    mag[:, n_chan // 4, 1] = 0
    assert mag.max() <= 1e-3


def test_fstage_more_frames_than_one_grid_row():
    # 70000 frames: the kernel loops over frames beyond the 65535 grid rows
    n_chan, N, F = 8, 1, 70000
    p = _time_samples(7, F * n_chan, N, "c8")
    got = _run_f(p, N, n_chan, F, "c8")
    ref = fstage.fstage(p, N, n_chan, F, "c8")
    err = np.linalg.norm((got - ref).reshape(F, -1), axis=1) / np.maximum(np.linalg.norm(ref.reshape(F, -1), axis=1), 1)
    assert err.max() <= 4 * EPS * 3


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("kind,n_chan,n_inputs,n_frames", [("c8", 128, 64, 40), ("c4", 64, 33, 25), ("r8", 32, 16, 30)])
def test_fx_chain(engine, kind, n_chan, n_inputs, n_frames):
    from paper_0906_1887_gb300 import corr
    L = fstage.transform_length(n_chan, kind)
    p = _time_samples(300 + n_chan, n_frames * L, n_inputs, kind)
    fp = corr.FPlan(n_inputs, n_chan, KIND_ID[kind])
    x = torch.from_numpy(np.ascontiguousarray(p).view(np.uint8).reshape(-1).copy()).cuda()
    spec = fp.empty_spectra(n_frames)
    fp.run(x, spec, n_frames)
    C = fp.n_out_chan
    xplan = corr.Plan(n_inputs, C, n_frames, 32)
    vis = xplan.empty_vis(1, "cuda")
    ws = xplan.empty_workspace(engine, 1, "cuda")
    xplan.run(spec, vis, ws, engine=engine)
    torch.cuda.synchronize()
    assert xplan.check_device() == 0
    got = vis.cpu().numpy()[0].astype(np.float64)
    if engine == 2:
        # the X stage alone, element by element, on the spectra it was given
        from oracle import precision
        sp = spec.cpu().numpy()
        check_bf16x3(got, sp, n_inputs, C, n_frames)
        bound, ex = precision.bf16x3_bound(sp, n_inputs, C, n_frames)
        auto = [i * n_inputs - i * (i - 1) // 2 for i in range(n_inputs)]
        iu, ju = np.triu_indices(n_inputs)
        a = ex[..., auto, 0]
        x_bound = float((bound / np.sqrt(np.maximum(a[:, iu] * a[:, ju], 1e-300))).max())
    else:
        x_bound = 1e-6
    ref = fstage.xcorr_spectra(fstage.fstage(p, n_inputs, n_chan, n_frames, kind))
    err = normwise_error(got, ref, n_inputs)
    assert err <= 2 * 4 * EPS * math.log2(L) + x_bound, err
    fp.close()
    xplan.close()


def test_fplan_rejects_bad_sizes():
    from paper_0906_1887_gb300 import corr
    with pytest.raises(corr.CorrError):
        corr.FPlan(4, 100, 0)        # not a power of two
    with pytest.raises(corr.CorrError):
        corr.FPlan(4, 4, 0)          # transform shorter than 8
    with pytest.raises(corr.CorrError):
        corr.FPlan(4, 4096, 2)       # real: 8192-point transform
    with pytest.raises(corr.CorrError):
        corr.FPlan(4, 64, 3)         # unknown kind


# ---- polyphase filterbank (Sec. 6.1) ----

def _run_pfb(packed, n_inputs, n_chan, n_frames, kind, n_taps, taps):
    from paper_0906_1887_gb300 import corr
    fp = corr.FPlan(n_inputs, n_chan, KIND_ID[kind], n_taps=n_taps, taps=taps)
    assert fp.n_taps == n_taps
    x = torch.from_numpy(np.ascontiguousarray(packed).view(np.uint8).reshape(-1).copy()).cuda()
    spec = fp.empty_spectra(n_frames)
    spec.fill_(float("nan"))
    fp.run(x, spec, n_frames)
    torch.cuda.synchronize()
    out = spec.cpu().numpy()
    fp.close()
    return out[..., 0].astype(np.float64) + 1j * out[..., 1]


@pytest.mark.parametrize("kind,n_chan,n_inputs,n_frames,n_taps", [
    ("c8", 128, 64, 6, 8), ("c8", 64, 70, 3, 4), ("c4", 32, 17, 5, 2), ("r8", 64, 9, 4, 8), ("c8", 1024, 3, 2, 4),
])
@pytest.mark.parametrize("custom", [False, True])
def test_pfb_matches_oracle(kind, n_chan, n_inputs, n_frames, n_taps, custom):
    L = fstage.transform_length(n_chan, kind)
    p = _time_samples(700 + n_chan, (n_frames + n_taps - 1) * L, n_inputs, kind)
    if custom:
        taps = np.random.default_rng(n_chan).normal(size=n_taps * L).astype(np.float32)
    else:
        taps = None
    got = _run_pfb(p, n_inputs, n_chan, n_frames, kind, n_taps, taps)
    h = fstage.default_prototype(n_taps, L) if taps is None else taps.astype(np.float64)
    ref = fstage.pfb(p, n_inputs, n_chan, n_frames, kind, h)
    bound = (4 * math.log2(L) + 4 * n_taps) * EPS
    for f in range(n_frames):
        for n in range(n_inputs):
            r = ref[f, :, n]
            assert np.linalg.norm(got[f, :, n] - r) <= bound * np.linalg.norm(r) + 1e-30, (f, n)


def test_pfb_one_tap_equals_plain_transform():
    n_chan, N, F = 128, 16, 4
    p = _time_samples(77, F * n_chan, N, "c8")
    a = _run_pfb(p, N, n_chan, F, "c8", 1, None)
    b = _run_f(p, N, n_chan, F, "c8")
    assert np.array_equal(a, b)

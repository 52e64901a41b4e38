"""Pins of the F-stage oracle (Sec. 2, Sec. 4) against facts fixed by the mathematics.

The oracle restates the paper's F stage: per input, N_C consecutive complex samples -> an
N_C-point DFT (or 2 N_C real samples -> a 2 N_C-point complex DFT keeping channels 0..N_C).
Each test pins it to something other than numpy's FFT call: the DFT as a double sum in pure
Python, exact tones and impulses whose spectra are known in closed form, Parseval's
identity, the Hermitian symmetry of real input, the placement of frames and inputs, and the
hand-decoded 4-bit format.
"""
import cmath

import numpy as np
import pytest

from oracle import fstage
from paper_0906_1887_gb300 import synth


def _time_packed(re, im, kind):
    """[T][N] integer samples -> packed bytes of the given kind."""
    re = np.asarray(re, np.int16)
    im = np.asarray(im, np.int16)
    if kind == "r8":
        return synth.pack_real8(re)
    return synth.pack(re[:, None, :], im[:, None, :], 8 if kind == "c8" else 4)


def _dft_brute(x):
    """Pure-Python DFT of one block: X_k = sum_s x_s exp(-2 pi i k s / L)."""
    L = len(x)
    return [sum(x[s] * cmath.exp(-2j * cmath.pi * k * s / L) for s in range(L)) for k in range(L)]


@pytest.mark.parametrize("kind", fstage.KINDS)
@pytest.mark.parametrize("n_chan", [4, 8, 16])
def test_matches_direct_dft_sum(kind, n_chan):
    rng = np.random.default_rng(11 + n_chan)
    N, F = 3, 2
    L = fstage.transform_length(n_chan, kind)
    lo, hi = (-8, 7) if kind == "c4" else (-128, 127)
    re = rng.integers(lo, hi + 1, (F * L, N))
    im = np.zeros_like(re) if kind == "r8" else rng.integers(lo, hi + 1, (F * L, N))
    X = fstage.fstage(_time_packed(re, im, kind), N, n_chan, F, kind)
    assert X.shape == (F, fstage.n_out_chan(n_chan, kind), N)
    for f in range(F):
        for n in range(N):
            x = [complex(int(re[f * L + s, n]), int(im[f * L + s, n])) for s in range(L)]
            ref = _dft_brute(x)[: fstage.n_out_chan(n_chan, kind)]
            assert np.allclose(X[f, :, n], ref, rtol=0, atol=1e-9 * L * 256)


@pytest.mark.parametrize("n_chan", [8, 32, 128])
def test_integer_tones_give_single_channels(n_chan):
    # x_s = A i^s is a tone at bin L/4 and A (-1)^s at bin L/2, both with integer samples:
    # their spectra are exactly A L at that bin and zero elsewhere
    L, A = n_chan, 100
    s = np.arange(L)
    quarter = np.array([1, 1j, -1, -1j])[s % 4] * A
    half = (-1.0) ** s * A
    re = np.stack([quarter.real, half], 1).round().astype(int)
    im = np.stack([quarter.imag, np.zeros(L)], 1).round().astype(int)
    X = fstage.fstage(_time_packed(re, im, "c8"), 2, n_chan, 1, "c8")[0]
    expect_q = np.zeros(L, complex); expect_q[L // 4] = A * L
    expect_h = np.zeros(L, complex); expect_h[L // 2] = A * L
    assert np.allclose(X[:, 0], expect_q, atol=1e-9 * A * L)
    assert np.allclose(X[:, 1], expect_h, atol=1e-9 * A * L)


@pytest.mark.parametrize("kind", fstage.KINDS)
def test_impulse_is_flat(kind):
    n_chan = 16
    L = fstage.transform_length(n_chan, kind)
    re = np.zeros((L, 1), int); im = np.zeros((L, 1), int)
    re[0, 0] = 7
    if kind != "r8":
        im[0, 0] = -3
    X = fstage.fstage(_time_packed(re, im, kind), 1, n_chan, 1, kind)[0, :, 0]
    assert np.allclose(X, complex(7, 0 if kind == "r8" else -3), atol=1e-12)


@pytest.mark.parametrize("kind", ["c8", "c4"])
def test_parseval(kind):
    rng = np.random.default_rng(5)
    n_chan, N, F = 64, 4, 3
    lo, hi = (-8, 7) if kind == "c4" else (-128, 127)
    re = rng.integers(lo, hi + 1, (F * n_chan, N)); im = rng.integers(lo, hi + 1, (F * n_chan, N))
    X = fstage.fstage(_time_packed(re, im, kind), N, n_chan, F, kind)
    energy_t = (re.astype(float) ** 2 + im.astype(float) ** 2).reshape(F, n_chan, N).sum(1)
    energy_f = (np.abs(X) ** 2).sum(1)
    assert np.allclose(energy_f, n_chan * energy_t, rtol=1e-12)


def test_real_input_keeps_dc_to_nyquist():
    # 2 N_C real samples -> N_C + 1 channels; DC = sum x_s and Nyquist = sum (-1)^s x_s are real,
    # and the dropped half is the conjugate mirror of the kept one
    rng = np.random.default_rng(9)
    n_chan, N = 16, 2
    L = 2 * n_chan
    x = rng.integers(-128, 128, (L, N))
    X = fstage.fstage(_time_packed(x, np.zeros_like(x), "r8"), N, n_chan, 1, "r8")[0]
    assert X.shape == (n_chan + 1, N)
    assert np.allclose(X[0], x.sum(0))
    assert np.allclose(X[n_chan], (x * ((-1) ** np.arange(L))[:, None]).sum(0))
    assert np.allclose(X[0].imag, 0) and np.allclose(X[n_chan].imag, 0, atol=1e-9)
    full = np.array([_dft_brute([complex(int(v)) for v in x[:, n]]) for n in range(N)]).T
    assert np.allclose(full[1:n_chan], np.conj(full[L - 1:n_chan:-1]), atol=1e-9)
    assert np.allclose(X, full[: n_chan + 1], atol=1e-8)


def test_frames_and_inputs_land_in_place():
    # only input 3 of frame 2 carries a signal: only spectra[2][:, 3] is non-zero
    n_chan, N, F = 8, 5, 4
    re = np.zeros((F * n_chan, N), int); im = np.zeros_like(re)
    re[2 * n_chan + 1, 3] = 5
    X = fstage.fstage(_time_packed(re, im, "c8"), N, n_chan, F, "c8")
    nz = np.argwhere(np.abs(X) > 1e-12)
    assert set(map(tuple, nz[:, [0, 2]])) == {(2, 3)}
    assert np.allclose(np.abs(X[2, :, 3]), 5)


def test_nibble_decode():
    b = np.array([0x8F, 0x70, 0x18], np.uint8)   # (-8, -1), (7, 0), (1, -8)
    x = fstage.unpack_time(b, 3, 1, "c4")[0]
    assert list(x) == [complex(-8, -1), complex(7, 0), complex(1, -8)]


def test_fx_closed_forms():
    # identical inputs: V_ij(c) = sum_f |X(c, f)|^2 for every pair; inputs carrying tones at
    # different channels: every cross term is zero and each auto is (A L)^2 per frame
    n_chan, F = 8, 3
    L = n_chan
    rng = np.random.default_rng(2)
    base = rng.integers(-100, 100, (F * L,))
    re = np.stack([base] * 3, 1); im = np.stack([base[::-1]] * 3, 1)
    X = fstage.fstage(_time_packed(re, im, "c8"), 3, n_chan, F, "c8")
    V = fstage.xcorr_spectra(X)
    power = (np.abs(X[:, :, 0]) ** 2).sum(0)
    for b in range(6):
        assert np.allclose(V[:, b, 0], power) and np.allclose(V[:, b, 1], 0, atol=1e-6)
    s = np.arange(F * L)
    A = 50
    t1 = np.exp(2j * np.pi * (L // 4) * s / L) * A     # bin L/4
    t2 = np.exp(2j * np.pi * (L // 2) * s / L) * A     # bin L/2
    re = np.stack([t1.real, t2.real], 1).round().astype(int); im = np.stack([t1.imag, t2.imag], 1).round().astype(int)
    V = fstage.xcorr_spectra(fstage.fstage(_time_packed(re, im, "c8"), 2, n_chan, F, "c8"))
    assert np.allclose(V[:, 1], 0, atol=1e-6)                      # baseline (0, 1)
    assert np.isclose(V[L // 4, 0, 0], F * (A * L) ** 2) and np.isclose(V[L // 2, 2, 0], F * (A * L) ** 2)


# ---- polyphase filterbank ----

def test_pfb_matches_definition_double_sum():
    rng = np.random.default_rng(21)
    n_chan, N, M, F = 8, 2, 3, 2
    L = n_chan
    h = rng.normal(size=M * L)
    re = rng.integers(-128, 128, ((F + M - 1) * L, N)); im = rng.integers(-128, 128, ((F + M - 1) * L, N))
    X = fstage.pfb(_time_packed(re, im, "c8"), N, n_chan, F, "c8", h)
    for f in range(F):
        for n in range(N):
            y = [sum(h[m * L + s] * complex(int(re[(f + m) * L + s, n]), int(im[(f + m) * L + s, n]))
                     for m in range(M)) for s in range(L)]
            assert np.allclose(X[f, :, n], _dft_brute(y), atol=1e-8 * 128 * L * M)


@pytest.mark.parametrize("kind", fstage.KINDS)
def test_pfb_with_one_unit_tap_is_the_plain_transform(kind):
    rng = np.random.default_rng(22)
    n_chan, N, F = 16, 3, 4
    L = fstage.transform_length(n_chan, kind)
    lo, hi = (-8, 7) if kind == "c4" else (-128, 127)
    re = rng.integers(lo, hi + 1, (F * L, N)); im = rng.integers(lo, hi + 1, (F * L, N))
    p = _time_packed(re, im, kind)
    assert np.allclose(fstage.pfb(p, N, n_chan, F, kind, fstage.default_prototype(1, L)),
                       fstage.fstage(p, N, n_chan, F, kind), atol=1e-9)


def test_pfb_frame_shift_and_linearity():
    rng = np.random.default_rng(23)
    n_chan, N, M, F = 16, 2, 4, 5
    L = n_chan
    re = rng.integers(-128, 128, ((F + M) * L, N)); im = rng.integers(-128, 128, ((F + M) * L, N))
    p = _time_packed(re, im, "c8")
    h1 = rng.normal(size=M * L); h2 = rng.normal(size=M * L)
    X = fstage.pfb(p, N, n_chan, F + 1, "c8", h1)
    Xs = fstage.pfb(_time_packed(re[L:], im[L:], "c8"), N, n_chan, F, "c8", h1)
    assert np.allclose(X[1:], Xs, atol=1e-8)                     # one frame later in, one frame later out
    lin = fstage.pfb(p, N, n_chan, F, "c8", 2 * h1 - 3 * h2)
    assert np.allclose(lin, 2 * fstage.pfb(p, N, n_chan, F, "c8", h1) - 3 * fstage.pfb(p, N, n_chan, F, "c8", h2),
                       atol=1e-6)


def test_pfb_prototype_shape():
    L, M = 64, 8
    h = fstage.default_prototype(M, L)
    assert h.shape == (M * L,)
    assert np.allclose(h, h[::-1])                                # symmetric
    assert np.argmax(h) in ((M * L - 1) // 2, M * L // 2)          # peak at the centre
    # zeros of the sinc at whole multiples of L from the centre (window aside)
    c = (M * L - 1) / 2.0
    assert abs(np.sinc((0 - c) / L)) < 1.0 and np.isclose(np.sinc(L / L), 0)


def test_pfb_confines_an_off_centre_tone():
    # a tone a third of a channel off a bin centre: the plain FFT leaks into many channels,
    # the 8-tap PFB keeps almost all the power within its two neighbouring channels
    n_chan, F, M = 64, 16, 8
    L = n_chan
    s = np.arange((F + M - 1) * L)
    tone = 100 * np.exp(2j * np.pi * (10 + 1 / 3) * s / L)
    re = np.round(tone.real).astype(int)[:, None]; im = np.round(tone.imag).astype(int)[:, None]
    p = _time_packed(re, im, "c8")
    power_pfb = (np.abs(fstage.pfb(p, 1, n_chan, F, "c8", fstage.default_prototype(M, L))[:, :, 0]) ** 2).sum(0)
    power_fft = (np.abs(fstage.fstage(p, 1, n_chan, F, "c8")[:, :, 0]) ** 2).sum(0)
    far = np.r_[0:8, 13:64]
    assert power_pfb[far].sum() / power_pfb.sum() < 1e-3
    assert power_fft[far].sum() / power_fft.sum() > 1e-2

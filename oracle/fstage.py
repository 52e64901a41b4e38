"""CPU oracle for the correlator F stage -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this module.  It restates the paper's F stage (Sec. 4, Fig. 1): a batch of time samples,
ordered with the input index varying fastest, is reordered into per-input blocks and each
block is Fourier transformed into spectral channels.

- Complex samples: N_C consecutive samples of an input -> an N_C-point complex DFT ->
  N_C channels (Sec. 2: "N_C samples are transformed into N_C spectral channels").
- Real samples: 2 N_C samples -> a 2 N_C-point complex-to-complex DFT, of which channels
  0 .. N_C (DC to Nyquist, N_C + 1 channels) are kept and the redundant half is dropped
  (Sec. 2 and Sec. 4: the paper uses a C2C transform of size 2 N_C for real input).

The DFT is the forward, unnormalised one, X_k = sum_s x_s exp(-2 pi i k s / L); channel c is
DFT bin c (no reordering of bins).  ``numpy.fft.fft`` is used as the transform step, in
complex128.  Spectra are returned as ``[n_frames][n_out_chan][n_inputs]`` complex128, the
sample order of the X stage (time = frame index).

Parity status: pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_fstage_pins.py``
(direct DFT sums, exact tones and impulses, Parseval, the real-input channel set, the
frame/input placement and the 4-bit nibble decode).  None is "parity unpinned".
"""
from __future__ import annotations

import numpy as np

KINDS = ("c8", "c4", "r8")   # complex 8-bit (re, im bytes), complex 4-bit (hi re, lo im), real 8-bit


def transform_length(n_chan: int, kind: str) -> int:
    """Samples per input per frame: N_C (complex) or 2 N_C (real)."""
    return 2 * n_chan if kind == "r8" else n_chan


def n_out_chan(n_chan: int, kind: str) -> int:
    """Channels produced: N_C (complex) or N_C + 1 (real, DC .. Nyquist)."""
    return n_chan + 1 if kind == "r8" else n_chan


def unpack_time(packed: np.ndarray, n_inputs: int, n_samples: int, kind: str) -> np.ndarray:
    """Packed time-domain samples ``[n_samples][n_inputs]`` -> complex128 of the same shape."""
    b = np.ascontiguousarray(packed).view(np.uint8).reshape(-1)
    if kind == "c8":
        v = b[: 2 * n_samples * n_inputs].view(np.int8).astype(np.float64).reshape(n_samples, n_inputs, 2)
        return v[..., 0] + 1j * v[..., 1]
    if kind == "c4":
        v = b[: n_samples * n_inputs].astype(np.int64).reshape(n_samples, n_inputs)
        hi = (v >> 4) & 0xF
        lo = v & 0xF
        re = np.where(hi >= 8, hi - 16, hi).astype(np.float64)   # two's complement nibbles
        im = np.where(lo >= 8, lo - 16, lo).astype(np.float64)
        return re + 1j * im
    if kind == "r8":
        v = b[: n_samples * n_inputs].view(np.int8).astype(np.float64).reshape(n_samples, n_inputs)
        return v + 0j
    raise ValueError(f"unknown sample kind {kind!r}")


def fstage(packed: np.ndarray, n_inputs: int, n_chan: int, n_frames: int, kind: str) -> np.ndarray:
    """Spectra ``[n_frames][n_out_chan][n_inputs]`` (complex128) of ``n_frames`` frames."""
    L = transform_length(n_chan, kind)
    x = unpack_time(packed, n_inputs, n_frames * L, kind).reshape(n_frames, L, n_inputs)
    X = np.fft.fft(x, axis=1)
    return X[:, : n_out_chan(n_chan, kind), :]


def spectra_as_float32_samples(X: np.ndarray) -> np.ndarray:
    """``[T][C][N]`` complex spectra -> the X stage's float sample layout ``[T][C][N][re, im]``."""
    out = np.empty(X.shape + (2,), np.float32)
    out[..., 0] = X.real
    out[..., 1] = X.imag
    return out


def xcorr_spectra(X: np.ndarray) -> np.ndarray:
    """X stage on complex spectra ``[T][C][N]`` in complex128: V_ij(c) = sum_t X_i conj(X_j) for
    i <= j (Sec. 2), returned ``[C][P][2]`` float64 in baseline order b = i N - i (i - 1) / 2 + (j - i)."""
    V = np.einsum("tci,tcj->cij", X, X.conj())
    iu, ju = np.triu_indices(X.shape[2])          # row-major upper triangle = baseline order
    out = np.empty((X.shape[1], iu.size, 2), np.float64)
    out[..., 0] = V[:, iu, ju].real
    out[..., 1] = V[:, iu, ju].imag
    return out


# ---- polyphase filterbank (Sec. 6.1: a PFB instead of the FFT, the extra cost in the unpack) ----
#
# Critically sampled PFB with M taps: output frame f weights the M input frames f .. f+M-1 by a
# prototype filter h of length M L and transforms the sum,
#     y_f[s] = sum_m h[m L + s] x[(f + m) L + s],   X_f[k] = sum_s y_f[s] exp(-2 pi i k s / L),
# so n_in frames give n_in - M + 1 output frames.  The paper names no filter; the default
# prototype is the windowed sinc h[n] = sinc((n - (M L - 1) / 2) / L) * w[n] with the Hamming
# window w[n] = 0.54 - 0.46 cos(2 pi n / (M L - 1)) (M = 1: the plain DFT, h = 1).

def default_prototype(n_taps: int, L: int) -> np.ndarray:
    n = np.arange(n_taps * L, dtype=np.float64)
    if n_taps == 1:
        return np.ones(L)
    x = (n - (n_taps * L - 1) / 2.0) / L
    w = 0.54 - 0.46 * np.cos(2.0 * np.pi * n / (n_taps * L - 1))
    return np.sinc(x) * w


def pfb(packed: np.ndarray, n_inputs: int, n_chan: int, n_frames_out: int, kind: str, h: np.ndarray) -> np.ndarray:
    """PFB spectra ``[n_frames_out][n_out_chan][n_inputs]`` (complex128) with prototype h (M L taps)."""
    L = transform_length(n_chan, kind)
    M = len(h) // L
    if M * L != len(h) or M < 1:
        raise ValueError("prototype length must be a multiple of the transform length")
    n_in = n_frames_out + M - 1
    x = unpack_time(packed, n_inputs, n_in * L, kind).reshape(n_in, L, n_inputs)
    hm = np.asarray(h, np.float64).reshape(M, L)
    y = np.zeros((n_frames_out, L, n_inputs), np.complex128)
    for m in range(M):
        y += hm[m][None, :, None] * x[m:m + n_frames_out]
    X = np.fft.fft(y, axis=1)
    return X[:, : n_out_chan(n_chan, kind), :]

"""CPU oracle for the dump step with post-correlation phase correction -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this module.  It restates two passages of the paper:

- Fig. 1: at the end of a dump interval the accumulators are read, divided by the number of
  times they were updated, and reset.
- Sec. 2: the MWA applies the geometric delay correction after correlation, as a phase
  correction.  A delay tau_i on input i multiplies its spectrum by exp(-2 pi i nu tau_i), so
  V_ij(c) carries the phase exp(-2 pi i nu_c (tau_i - tau_j)); the correction removes it:

      V'_ij(c) = V_ij(c) / n_accum * exp(+2 pi i nu_c (tau_i - tau_j))

  (the paper gives no sign convention; this reading removes the phase that the stated
  delays add).

Input: accumulators ``[C][P][2]`` (int64 or float), baseline b = i N - i (i - 1) / 2 + (j - i).
Output: ``[C][P][2]`` float64.  The phase of each baseline is formed from the delay
difference directly, in float64.

Parity status: pinned by ``tests/test_oracle_dump_pins.py`` (zero delays, autos, equal
delays, a point source whose corrected visibilities are real and equal on every baseline, a
pure delay difference of a quarter period, and the division by the update count).
"""
from __future__ import annotations

import numpy as np


def baseline_pairs(n_inputs: int):
    """(i, j) of every baseline b in order (row-major upper triangle)."""
    return np.triu_indices(n_inputs)


def dump_corrected(acc: np.ndarray, n_accum: int, delays_s: np.ndarray, freqs_hz: np.ndarray) -> np.ndarray:
    C, P, _ = acc.shape
    N = len(delays_s)
    if P != N * (N + 1) // 2 or len(freqs_hz) != C:
        raise ValueError("shape mismatch")
    i, j = baseline_pairs(N)
    tau = np.asarray(delays_s, np.float64)
    nu = np.asarray(freqs_hz, np.float64)
    phase = 2.0 * np.pi * nu[:, None] * (tau[i] - tau[j])[None, :]        # [C][P]
    v = (acc[..., 0].astype(np.float64) + 1j * acc[..., 1].astype(np.float64)) / float(n_accum)
    w = v * np.exp(1j * phase)
    out = np.empty((C, P, 2), np.float64)
    out[..., 0] = w.real
    out[..., 1] = w.imag
    return out

"""Pins of the dump/phase-correction oracle (Fig. 1, Sec. 2) against facts fixed by the maths.

The oracle divides the accumulators by the update count and removes the phase that input
delays add to each baseline, exp(-2 pi i nu (tau_i - tau_j)).  Each test pins it to an
independent fact: no delays change nothing but the scale, autos never rotate, equal delays
cancel, a point source seen through known delays comes out real and equal on every
baseline, a quarter-period delay difference is a factor of i, and the update count divides.
"""
import numpy as np

from oracle import dump as odump
from oracle import fstage


def _acc(rng, C, N, lo=-1000, hi=1000):
    P = N * (N + 1) // 2
    return rng.integers(lo, hi, (C, P, 2)).astype(np.int64)


def test_zero_delays_only_divide():
    rng = np.random.default_rng(1)
    acc = _acc(rng, 3, 5)
    out = odump.dump_corrected(acc, 4, np.zeros(5), np.linspace(1e8, 2e8, 3))
    assert np.allclose(out, acc / 4.0, rtol=0, atol=1e-12)


def test_autos_and_equal_delays_do_not_rotate():
    rng = np.random.default_rng(2)
    N, C = 6, 4
    acc = _acc(rng, C, N)
    tau = rng.normal(0, 1e-6, N)
    tau[2] = tau[4]
    out = odump.dump_corrected(acc, 1, tau, np.linspace(1.5e8, 1.6e8, C))
    i, j = odump.baseline_pairs(N)
    same = (i == j) | ((i == 2) & (j == 4))
    assert np.allclose(out[:, same], acc[:, same], rtol=0, atol=1e-9)
    assert not np.allclose(out[:, ~same], acc[:, ~same])


def test_point_source_becomes_real_and_equal():
    # spectra of one source seen with delays tau_i: X_i(c) = S(c) exp(-2 pi i nu_c tau_i);
    # after correction every baseline equals sum |S|^2 (real), whatever the delays
    rng = np.random.default_rng(3)
    N, C, T = 5, 6, 7
    nu = 1.8e8 + 1e4 * np.arange(C)
    tau = rng.normal(0, 3e-7, N)
    S = rng.normal(size=(T, C)) + 1j * rng.normal(size=(T, C))
    X = S[:, :, None] * np.exp(-2j * np.pi * nu[None, :, None] * tau[None, None, :])
    V = fstage.xcorr_spectra(X)                       # [C][P][2] float64
    out = odump.dump_corrected(V, 1, tau, nu)
    power = (np.abs(S) ** 2).sum(0)
    assert np.allclose(out[..., 0], power[:, None], rtol=1e-9)
    assert np.allclose(out[..., 1], 0, atol=1e-9 * power.max())


def test_quarter_period_is_a_factor_i():
    # tau_0 - tau_1 = 1 / (4 nu): V'_01 = V_01 * exp(i pi / 2) = i V_01
    nu = np.array([1e8])
    tau = np.array([1.0 / (4 * nu[0]), 0.0])
    acc = np.array([[[5, 0], [3, 2], [7, 0]]], np.int64)   # b = (0,0), (0,1), (1,1)
    out = odump.dump_corrected(acc, 1, tau, nu)
    assert np.allclose(out[0, 1], [-2, 3], atol=1e-9)
    assert np.allclose(out[0, [0, 2]], acc[0, [0, 2]], atol=1e-12)


def test_update_count_divides():
    acc = np.full((2, 3, 2), 12, np.int64)
    out = odump.dump_corrected(acc, 3, np.zeros(2), np.ones(2))
    assert np.allclose(out, 4.0)

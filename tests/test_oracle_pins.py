"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

The oracle computes V_ij(c) = sum_t x_i(c,t) conj(x_j(c,t)) for i <= j (Sec. 2, Sec. 4
Fig. 2).  Each test below pins it to something other than itself: brute force with
Python's complex type, numpy's einsum in complex128, Hermitian symmetry under input
reversal, closed forms (identical inputs, orthogonal Walsh-Hadamard inputs, an impulse,
the -128 overflow edge), additivity over time and hand-decoded bytes of the sample
formats.
"""
import itertools

import numpy as np
import pytest

from paper_0906_1887_gb300 import synth


def _pack(re, im, bits):
    return synth.pack(np.asarray(re), np.asarray(im), bits)


def _brute(re, im):
    """Pure-Python reference with the built-in complex type: [C][P][2] as Python ints."""
    T, C, N = re.shape
    out = []
    for c in range(C):
        rows = []
        for i in range(N):
            for j in range(i, N):
                acc = 0j
                for t in range(T):
                    a = complex(int(re[t, c, i]), int(im[t, c, i]))
                    b = complex(int(re[t, c, j]), int(im[t, c, j]))
                    acc += a * b.conjugate()
                rows.append((int(acc.real), int(acc.imag)))
        out.append(rows)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("n,c,t", [(1, 1, 1), (2, 3, 31), (3, 1, 33), (5, 3, 70), (8, 1, 33)])
@pytest.mark.parametrize("bits", [4, 8])
def test_brute_force_tiny(oracle_mod, n, c, t, bits):
    lo, hi = (-8, 7) if bits == 4 else (-128, 127)
    re, im = synth.uniform_ints(10 * n + c + t + bits, t, c, n, lo, hi)
    v = oracle_mod.xcorr_int(_pack(re, im, bits), n, c, t, bits)
    assert np.array_equal(v, _brute(re, im))


def test_einsum_complex128_mwa32t(oracle_mod):
    re, im, bits, (n, c, t) = synth.workload("mwa32t_4bit")
    v = oracle_mod.xcorr_int(synth.pack(re, im, bits), n, c, t, bits)
    x = re.astype(np.float64) + 1j * im.astype(np.float64)          # [T][C][N]
    full = np.einsum("tci,tcj->cij", x, x.conj())                    # exact: |entries| << 2**53
    iu, ju = np.triu_indices(n)
    ref = full[:, iu, ju]                                            # row-major upper triangle
    assert np.array_equal(v[..., 0], ref.real.astype(np.int64))
    assert np.array_equal(v[..., 1], ref.imag.astype(np.int64))


def test_pair_count_and_baseline_order(oracle_mod):
    assert oracle_mod.n_baselines(64) == 2080          # 64 inputs: N(N+1)/2 products (Sec. 2)
    assert oracle_mod.n_baselines(1024) == 524800
    n = 7
    seen = [oracle_mod.baseline_index(n, i, j) for i in range(n) for j in range(i, n)]
    assert seen == list(range(n * (n + 1) // 2))      # a bijection onto 0..P-1, row-major


def test_hermitian_under_input_reversal(oracle_mod):
    # Reversing the input order maps pair (i, j) to (N-1-j, N-1-i); the product becomes
    # x_j conj(x_i) = conj(V_ij) (Fig. 2: the two halves are conjugate copies).
    n, c, t = 9, 2, 45
    re, im = synth.uniform_ints(7, t, c, n, -128, 127)
    v = oracle_mod.xcorr_int(_pack(re, im, 8), n, c, t, 8)
    w = oracle_mod.xcorr_int(_pack(re[..., ::-1].copy(), im[..., ::-1].copy(), 8), n, c, t, 8)
    for i, j in itertools.combinations_with_replacement(range(n), 2):
        b = oracle_mod.baseline_index(n, i, j)
        b2 = oracle_mod.baseline_index(n, n - 1 - j, n - 1 - i)
        assert v[:, b, 0].tolist() == w[:, b2, 0].tolist()
        assert v[:, b, 1].tolist() == (-w[:, b2, 1]).tolist()
    autos = [oracle_mod.baseline_index(n, i, i) for i in range(n)]
    assert (v[:, autos, 1] == 0).all() and (v[:, autos, 0] >= 0).all()


def test_identical_inputs_closed_form(oracle_mod):
    n, c, t = 6, 2, 40
    r1, i1 = synth.uniform_ints(3, t, c, 1, -8, 7)
    re, im = np.repeat(r1, n, axis=2), np.repeat(i1, n, axis=2)
    v = oracle_mod.xcorr_int(_pack(re, im, 4), n, c, t, 4)
    power = (r1.astype(np.int64) ** 2 + i1.astype(np.int64) ** 2).sum(axis=0)[:, 0]   # sum |x|^2 per chan
    assert (v[..., 0] == power[:, None]).all()
    assert (v[..., 1] == 0).all()


def _hadamard(k):
    h = np.array([[1]], dtype=np.int64)
    while h.shape[0] < k:
        h = np.block([[h, h], [h, -h]])
    return h


def test_orthogonal_walsh_hadamard_closed_form(oracle_mod):
    # x_i(t) = H[i,t] + 1j H[i+N,t]: distinct Hadamard rows are orthogonal, so every cross
    # product sums to exactly 0 and every auto to 2K.
    k, n = 64, 16
    h = _hadamard(k)
    re = h[:n].T.reshape(k, 1, n)
    im = h[n:2 * n].T.reshape(k, 1, n)
    v = oracle_mod.xcorr_int(_pack(re, im, 4), n, 1, k, 4)
    for i, j in itertools.combinations_with_replacement(range(n), 2):
        b = oracle_mod.baseline_index(n, i, j)
        assert v[0, b, 0] == (2 * k if i == j else 0)
        assert v[0, b, 1] == 0


def test_impulse_closed_form(oracle_mod):
    # One non-zero time sample: V = x x^H for that sample (Sec. 4, Fig. 2), worked by hand
    # for x = (3 + 1j, -2 + 4j, 0 - 5j).
    n, t = 3, 17
    re = np.zeros((t, 1, n), np.int16)
    im = np.zeros((t, 1, n), np.int16)
    re[5, 0] = [3, -2, 0]
    im[5, 0] = [1, 4, -5]
    v = oracle_mod.xcorr_int(_pack(re, im, 8), n, 1, t, 8)[0]
    expect = {  # x_i * conj(x_j)
        (0, 0): (10, 0), (0, 1): (-2, -14), (0, 2): (-5, 15),
        (1, 1): (20, 0), (1, 2): (-20, -10), (2, 2): (25, 0),
    }
    for (i, j), val in expect.items():
        assert tuple(v[oracle_mod.baseline_index(n, i, j)]) == val


def test_conjugation_convention(oracle_mod):
    # x_0 = 1, x_1 = 1j  ->  V_01 = x_0 conj(x_1) = -1j per sample ("first spectrum times the
    # complex conjugate of the second", Sec. 2).
    t = 4
    re = np.array([[[1, 0]]] * t, np.int16)
    im = np.array([[[0, 1]]] * t, np.int16)
    v = oracle_mod.xcorr_int(_pack(re, im, 8), 2, 1, t, 8)[0]
    assert tuple(v[1]) == (0, -t)


def test_additivity_over_time(oracle_mod):
    n, c = 11, 3
    re, im = synth.uniform_ints(99, 130, c, n, -128, 127)
    whole = oracle_mod.xcorr_int(_pack(re, im, 8), n, c, 130, 8)
    a = oracle_mod.xcorr_int(_pack(re[:47], im[:47], 8), n, c, 47, 8)
    b = oracle_mod.xcorr_int(_pack(re[47:], im[47:], 8), n, c, 83, 8)
    assert np.array_equal(whole, a + b)


def test_overflow_edge_int32(oracle_mod):
    # All samples -128 - 128j for K = 65536: Re of every product sums to 2 * 128^2 * 65536 =
    # 2^31, one past int32; Im sums to 0.  A second pair has x0 = -128 + 127j,
    # x1 = 127 - 128j: x0 conj(x1) = -32512 - 255j per sample.
    k = 65536
    re = np.full((k, 1, 2), -128, np.int16)
    im = np.full((k, 1, 2), -128, np.int16)
    v = oracle_mod.xcorr_int(_pack(re, im, 8), 2, 1, k, 8)[0]
    assert (v[:, 0] == 2 ** 31).all() and (v[:, 1] == 0).all()
    re[:, 0, 0], im[:, 0, 0] = -128, 127
    re[:, 0, 1], im[:, 0, 1] = 127, -128
    v = oracle_mod.xcorr_int(_pack(re, im, 8), 2, 1, k, 8)[0]
    assert tuple(v[1]) == (-32512 * k, -255 * k)
    assert tuple(v[0]) == ((128 ** 2 + 127 ** 2) * k, 0)


def test_sample_format_decoding(oracle_mod):
    # 4-bit: high nibble re, low nibble im, two's complement.
    raw4 = np.array([0x7F, 0x80, 0x08, 0xF1, 0x00, 0x88], np.uint8).reshape(1, 1, 6)
    re, im = oracle_mod.unpack(raw4, 6, 1, 1, 4)
    assert re.ravel().tolist() == [7, -8, 0, -1, 0, -8]
    assert im.ravel().tolist() == [-1, 0, -8, 1, 0, -8]
    # 8-bit: re byte then im byte, two's complement.
    raw8 = np.array([0x80, 0x7F, 0xFF, 0x01, 0x00, 0x81], np.uint8).reshape(1, 1, 3, 2)
    re, im = oracle_mod.unpack(raw8, 3, 1, 1, 8)
    assert re.ravel().tolist() == [-128, -1, 0]
    assert im.ravel().tolist() == [127, 1, -127]


def test_float64_variant_matches_complex128(oracle_mod):
    n, c, t = 13, 3, 77
    re, im = synth.correlated_gaussian(5, t, c, n, 3.0, 0.2, as_float=True)
    v = oracle_mod.xcorr_f64(synth.packf32(re, im), n, c, t)
    x = re.astype(np.float64) + 1j * im.astype(np.float64)
    full = np.einsum("tci,tcj->cij", x, x.conj())
    iu, ju = np.triu_indices(n)
    ref = full[:, iu, ju]
    scale = np.abs(ref).max()
    assert np.abs(v[..., 0] - ref.real).max() <= 1e-12 * scale
    assert np.abs(v[..., 1] - ref.imag).max() <= 1e-12 * scale


def test_float64_impulse(oracle_mod):
    re = np.zeros((3, 1, 2), np.float32)
    im = np.zeros((3, 1, 2), np.float32)
    re[1, 0] = [0.5, -1.25]
    im[1, 0] = [2.0, 0.75]
    v = oracle_mod.xcorr_f64(synth.packf32(re, im), 2, 1, 3)[0]
    a, b = 0.5 + 2.0j, -1.25 + 0.75j
    assert v[1, 0] == (a * b.conjugate()).real and v[1, 1] == (a * b.conjugate()).imag
    assert v[0, 0] == abs(a) ** 2 and v[2, 0] == abs(b) ** 2


def test_channel_selection_and_threads(oracle_mod):
    n, c, t = 10, 6, 50
    re, im = synth.uniform_ints(12, t, c, n, -128, 127)
    p = _pack(re, im, 8)
    full = oracle_mod.xcorr_int(p, n, c, t, 8, n_threads=1)
    sel = oracle_mod.xcorr_int(p, n, c, t, 8, chans=[4, 1], n_threads=3)
    assert np.array_equal(sel[0], full[4]) and np.array_equal(sel[1], full[1])


def test_channel_independence(oracle_mod):
    # Channels are formed independently (Fig. 2): changing channel 1 leaves channel 0 alone.
    n, c, t = 5, 2, 20
    re, im = synth.uniform_ints(1, t, c, n, -8, 7)
    v = oracle_mod.xcorr_int(_pack(re, im, 4), n, c, t, 4)
    re2 = re.copy()
    re2[:, 1] = 0
    w = oracle_mod.xcorr_int(_pack(re2, im, 4), n, c, t, 4)
    assert np.array_equal(v[0], w[0]) and not np.array_equal(v[1], w[1])


def test_statistics_of_correlated_stream():
    # Sanity of the generator, not parity: E[V_ij]/K = 2 sigma^2 rho (i != j), 2 sigma^2 (autos).
    re, im = synth.correlated_gaussian(2000, 2000, 8, 8, 16.0, 0.1, 127)
    x = re.astype(np.float64) + 1j * im.astype(np.float64)
    full = np.einsum("tci,tcj->cij", x, x.conj()) / 2000
    off = full[:, ~np.eye(8, dtype=bool)].real.mean()
    auto = np.einsum("cii->ci", full).real.mean()
    assert abs(off - 51.2) < 5.0 and abs(auto - 512.0) < 15.0

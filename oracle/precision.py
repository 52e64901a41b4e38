"""Error model of the BF16x3 split products -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this module.  It states, for float samples, how far the tensor-core BF16x3 result may lie from
the exact cross-multiply-accumulate V_ij = sum_t x_i conj(x_j) (Sec. 2; Sec. 4, Fig. 2), so
that a test can tell BF16x3 apart from the cheaper variants that drop one or both correction
products.

The split (per real component x of a float32 sample):
    h = bf16(x)            round to nearest even, 8 significant bits
    l = bf16(x - h)
    r = x - h - l          what the split loses: |r| <= 2^-16 |x|, |l| <= 2^-8 (1 + 2^-8) |x|
For one real product a b the method forms h_a h_b + h_a l_b + l_a h_b and drops
    l_a l_b + (h_a + l_a) r_b + r_a (h_b + l_b) + r_a r_b,
at most 3 * 2^-16 (1 + 2^-7) |a| |b| (the representation error).  The products of bf16 values
are exact in fp32; the tensor core sums them into an fp32 accumulator.  Each MMA (16 samples,
one of the three products) is modelled as adding an error of at most 2 * 2^-23 times the sum
of the magnitudes it has accumulated so far (one rounding of the fp32 result, counted twice to
cover alignment of the addends); the epilogue's rr + ii (ir - ri) adds one rounding of the
result.  With S = sum_t (|a_r b_r| + |a_i b_i|) for the real part (|a_i b_r| + |a_r b_i| for
the imaginary part) and n_mma = 3 * (samples rounded up to 64) / 16 MMAs into each element:

    |Re V - Re V_exact| <= |Re E_rep| + (n_mma + 1) 2^-22 (1 + 2^-7) S_re + 2^-24 |Re V_exact|

and likewise for Im; the complex error bound is the root sum of squares of the two.  E_rep,
the representation error of the data at hand, is computed exactly here (float64 sums of
products of bf16 values and of the residuals), so the bound is per element and
data-dependent but not statistical.

``variant_errors`` computes, in float64 (no accumulation error at all), the results of h h^H
alone and of h h^H + h l^H, so a test can check that the bound sits below what those variants
would give on the same inputs.

Parity status: pinned by ``tests/test_oracle_precision_pins.py`` -- ``bf16_rn`` against
torch's float32 -> bfloat16 conversion (a library routine) including exact ties, the split's
residual bounds, the representation bound over random data, and an fp32 emulation of the
kernel's accumulation order staying within the bound.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24          # unit roundoff of fp32
U_BF16 = 2.0 ** -8        # unit roundoff of bf16 (8 significant bits)


def bf16_rn(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32 values."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).reshape(x.shape)


def split(x: np.ndarray):
    """(h, l) with h = bf16(x), l = bf16(x - h); x - h is exact in float32."""
    x = np.asarray(x, dtype=np.float32)
    h = bf16_rn(x)
    l = bf16_rn((x - h).astype(np.float32))
    return h, l


def _complex(samples: np.ndarray, n_inputs: int, n_chan: int, n_time: int, chans):
    x = np.asarray(samples, dtype=np.float32).reshape(n_time, n_chan, n_inputs, 2)
    if chans is not None:
        x = x[:, np.asarray(chans, dtype=np.int64)]
    return x


def _pairs(a: np.ndarray, b: np.ndarray, iu, ju):
    """Real and imaginary parts of sum_t a_i conj(b_j) over pairs (iu, ju), float64.

    a, b: [T][C][N][2] float64.  Returns (re, im) of shape [C][P].
    """
    ar, ai = a[..., 0], a[..., 1]
    br, bi = b[..., 0], b[..., 1]
    rr = np.einsum("tci,tcj->cij", ar, br)
    ii = np.einsum("tci,tcj->cij", ai, bi)
    ir = np.einsum("tci,tcj->cij", ai, br)
    ri = np.einsum("tci,tcj->cij", ar, bi)
    return (rr + ii)[:, iu, ju], (ir - ri)[:, iu, ju]


def variant_errors(samples: np.ndarray, n_inputs: int, n_chan: int, n_time: int, chans=None):
    """Exact V and the float64 results of the BF16 product variants, each [C][P][2].

    Keys: 'exact', 'hh' (h h^H), 'hh_hl' (h h^H + h l^H), 'x3' (h h^H + h l^H + l h^H).
    """
    x = _complex(samples, n_inputs, n_chan, n_time, chans)
    h, l = split(x)
    x64, h64, l64 = x.astype(np.float64), h.astype(np.float64), l.astype(np.float64)
    iu, ju = np.triu_indices(n_inputs)
    out = {}

    def pack(re, im):
        v = np.empty(re.shape + (2,), np.float64)
        v[..., 0], v[..., 1] = re, im
        return v

    out["exact"] = pack(*_pairs(x64, x64, iu, ju))
    hh = _pairs(h64, h64, iu, ju)
    hl = _pairs(h64, l64, iu, ju)
    lh = _pairs(l64, h64, iu, ju)
    out["hh"] = pack(*hh)
    out["hh_hl"] = pack(hh[0] + hl[0], hh[1] + hl[1])
    out["x3"] = pack(hh[0] + hl[0] + lh[0], hh[1] + hl[1] + lh[1])
    return out


def abs_sums(samples: np.ndarray, n_inputs: int, n_chan: int, n_time: int, chans=None):
    """(S_re, S_im), each [C][P]: sum_t |a_r b_r| + |a_i b_i| and sum_t |a_i b_r| + |a_r b_i|."""
    x = np.abs(_complex(samples, n_inputs, n_chan, n_time, chans).astype(np.float64))
    iu, ju = np.triu_indices(n_inputs)
    ar, ai = x[..., 0], x[..., 1]
    s_re = np.einsum("tci,tcj->cij", ar, ar) + np.einsum("tci,tcj->cij", ai, ai)
    s_im = np.einsum("tci,tcj->cij", ai, ar) + np.einsum("tci,tcj->cij", ar, ai)
    return s_re[:, iu, ju], s_im[:, iu, ju]


def n_mma(n_time: int) -> int:
    """MMAs accumulated into each element: three products per 16 samples of the padded dump."""
    kp = (n_time + 63) // 64 * 64
    return 3 * kp // 16


def bf16x3_bound(samples: np.ndarray, n_inputs: int, n_chan: int, n_time: int, chans=None, variants=None):
    """Per-element bound [C][P] on |V_bf16x3 - V_exact| (complex magnitude), and V_exact."""
    v = variants if variants is not None else variant_errors(samples, n_inputs, n_chan, n_time, chans)
    s_re, s_im = abs_sums(samples, n_inputs, n_chan, n_time, chans)
    ex, x3 = v["exact"], v["x3"]
    acc = (n_mma(n_time) + 1) * 2.0 * 2.0 ** -23 * (1.0 + 2.0 ** -7)
    b_re = np.abs(ex[..., 0] - x3[..., 0]) + acc * s_re + U32 * np.abs(ex[..., 0])
    b_im = np.abs(ex[..., 1] - x3[..., 1]) + acc * s_im + U32 * np.abs(ex[..., 1])
    return np.hypot(b_re, b_im), ex


def separation(samples: np.ndarray, n_inputs: int, n_chan: int, n_time: int, chans=None):
    """For each dropped-product variant, the largest ratio |V_variant - V_exact| / bound.

    A ratio above 1 means a kernel computing that variant (even with exact accumulation) would
    fail a test that holds every element to the bound.
    """
    v = variant_errors(samples, n_inputs, n_chan, n_time, chans)
    bound, ex = bf16x3_bound(samples, n_inputs, n_chan, n_time, chans, variants=v)
    out = {}
    for k in ("hh", "hh_hl"):
        err = np.hypot(v[k][..., 0] - ex[..., 0], v[k][..., 1] - ex[..., 1])
        out[k] = float((err / np.maximum(bound, 1e-300)).max())
    return out

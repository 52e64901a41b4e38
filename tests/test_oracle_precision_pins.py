"""Pins of the BF16x3 error model (oracle/precision.py) against things other than itself.

- bf16 rounding against torch's float32 -> bfloat16 conversion (a library routine), with
  exact ties, both signs and tiny values;
- the split's residual bounds, which follow from bf16 having 8 significant bits;
- the representation error of the three kept products against its analytic bound;
- an fp32 emulation of the tensor core's order of accumulation (16-sample MMAs, three
  products each, fp32 accumulator, fp32 re/im combine) staying within the per-element bound;
- the bound separating BF16x3 from the variants that drop correction products, on the
  shapes and recipes the GPU tests use.
"""
import numpy as np
import pytest

from oracle import precision as pr
from paper_0906_1887_gb300 import synth


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32) * np.float32(37.0),
        rng.standard_normal(2000).astype(np.float32) * np.float32(1e-20),
        np.array([0.0, -0.0, 1.0, -1.0, 3.0e38, -3.0e38], np.float32),
    ])
    # exact ties: the low 16 bits are 0x8000, with even and odd kept parts
    mant = rng.integers(0, 128, 2000).astype(np.uint32) << 16          # the 7 kept mantissa bits
    expo = rng.integers(100, 150, 2000).astype(np.uint32) << 23
    ties = (expo | mant | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(pr.bf16_rn(x).view(np.uint32), want.view(np.uint32))


def test_split_residual_bounds():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(200000) * 16).astype(np.float32)
    h, l = pr.split(x)
    x64 = x.astype(np.float64)
    r = x64 - h.astype(np.float64) - l.astype(np.float64)
    assert np.all(np.abs(r) <= 2.0 ** -16 * np.abs(x64))
    assert np.all(np.abs(l) <= 2.0 ** -8 * (1 + 2.0 ** -8) * np.abs(x64))
    # h and l are bf16 values (low 16 bits zero)
    assert not np.any(h.view(np.uint32) & 0xFFFF) and not np.any(l.view(np.uint32) & 0xFFFF)


@pytest.mark.parametrize("n,c,t,sigma,rho", [(16, 3, 500, 1.0, 0.3), (9, 2, 64, 16.0, 0.1)])
def test_representation_error_within_analytic_bound(n, c, t, sigma, rho):
    re, im = synth.correlated_gaussian(10 + n, t, c, n, sigma, rho, as_float=True)
    x = synth.packf32(re, im)
    v = pr.variant_errors(x, n, c, t)
    s_re, s_im = pr.abs_sums(x, n, c, t)
    k = 3 * 2.0 ** -16 * (1 + 2.0 ** -7)
    assert np.all(np.abs(v["exact"][..., 0] - v["x3"][..., 0]) <= k * s_re)
    assert np.all(np.abs(v["exact"][..., 1] - v["x3"][..., 1]) <= k * s_im)
    # and the representation error is what the correction products buy: h h^H alone is worse
    e_hh = np.abs(v["exact"] - v["hh"]).max()
    e_x3 = np.abs(v["exact"] - v["x3"]).max()
    assert e_x3 < e_hh / 50


def _emulate_fp32_mma_order(x, n, c, t):
    """fp32 model of the kernel: per 16 samples three MMAs (h h, h l, l h), each adding the
    float64-exact sum of its 16 bf16 products to the fp32 accumulator with one rounding; then
    Re = fp32(rr + ii), Im = fp32(ir - ri)."""
    xs = np.asarray(x, np.float32).reshape(t, c, n, 2)
    h, l = pr.split(xs)
    kp = (t + 63) // 64 * 64
    pad = np.zeros((kp - t, c, n, 2), np.float32)
    h = np.concatenate([h, pad]).astype(np.float64)
    l = np.concatenate([l, pad]).astype(np.float64)
    iu, ju = np.triu_indices(n)
    acc = {k: np.zeros((c, n, n), np.float32) for k in ("rr", "ii", "ir", "ri")}
    comp = {"rr": (0, 0), "ii": (1, 1), "ir": (1, 0), "ri": (0, 1)}
    for k0 in range(0, kp, 16):
        for a, b in ((h, h), (h, l), (l, h)):
            for name, (p, q) in comp.items():
                part = np.einsum("tci,tcj->cij", a[k0:k0 + 16, ..., p], b[k0:k0 + 16, ..., q])
                acc[name] = (acc[name].astype(np.float64) + part).astype(np.float32)
    re = (acc["rr"] + acc["ii"])[:, iu, ju]
    im = (acc["ir"] - acc["ri"])[:, iu, ju]
    out = np.empty(re.shape + (2,), np.float64)
    out[..., 0], out[..., 1] = re, im
    return out


@pytest.mark.parametrize("n,c,t,sigma,rho", [(8, 2, 1000, 1.0, 0.3), (12, 2, 333, 16.0, 0.1)])
def test_fp32_accumulation_model_within_bound(n, c, t, sigma, rho):
    re, im = synth.correlated_gaussian(20 + n, t, c, n, sigma, rho, as_float=True)
    x = synth.packf32(re, im)
    bound, ex = pr.bf16x3_bound(x, n, c, t)
    got = _emulate_fp32_mma_order(x, n, c, t)
    err = np.hypot(got[..., 0] - ex[..., 0], got[..., 1] - ex[..., 1])
    assert np.all(err <= bound)
    # the emulated error is well inside the bound (the bound is a worst case)
    assert (err / bound).max() < 0.5


# the shapes and recipes of the GPU BF16x3 tests (seed, n, c, t, sigma, rho)
GPU_FLOAT_CASES = [(2001, 64, 4, 1000, 16.0, 0.1), (155, 64, 5, 1000, 1.0, 0.3), (99, 8, 3, 100, 1.0, 0.3),
                   (125, 34, 4, 130, 1.0, 0.3), (142, 65, 2, 130, 1.0, 0.3), (1002, 16, 4, 96, 1.0, 0.3),
                   (907, 40, 6, 90, 2.0, 0.2), (2500, 64, 3, 1000, 16.0, 0.1)]


@pytest.mark.parametrize("seed,n,c,t,sigma,rho", GPU_FLOAT_CASES)
def test_bound_separates_bf16x3_from_dropped_products(seed, n, c, t, sigma, rho):
    re, im = synth.correlated_gaussian(seed, t, c, n, sigma, rho, as_float=True)
    x = synth.packf32(re, im)
    sep = pr.separation(x, n, c, t)
    # a kernel that drops l h^H (or both corrections) exceeds the bound by a wide margin
    assert sep["hh_hl"] > 2.0 and sep["hh"] > 2.0, sep


def test_bound_is_tight_enough_in_normwise_terms():
    # the 1000-sample float stream: the bound stays around 6e-5 normwise, five times below the
    # error of h h^H alone
    re, im = synth.correlated_gaussian(2001, 1000, 4, 64, 16.0, 0.1, as_float=True)
    x = synth.packf32(re, im)
    bound, ex = pr.bf16x3_bound(x, 64, 4, 1000)
    auto = [i * 64 - i * (i - 1) // 2 for i in range(64)]
    iu, ju = np.triu_indices(64)
    a = ex[..., auto, 0]
    scale = np.sqrt(a[:, iu] * a[:, ju])
    assert (bound / scale).max() < 1e-4

"""Seeded synthetic sample generators shared by the oracle tests and the CUDA path.

This module draws random numbers and packs them into the wire formats of the
correlator input; it contains none of the correlation arithmetic.

Wire formats (input varies fastest within one time instant, Sec. 3 and Sec. 4):

* 4-bit ("1-byte mode", Sec. 5): one byte per complex sample, real part in the
  high nibble, imaginary part in the low nibble, both two's complement (-8..7).
* 8-bit: two bytes per complex sample, real then imaginary, each int8.
* 32-bit float: eight bytes per complex sample, float32 real then imaginary.

Packed arrays are laid out ``[n_time][n_chan][n_inputs]`` (samples already
channelised by the F stage; the channel axis sits between time and input).

Recipes (numpy PCG64, ``default_rng(seed)``):

* ``uniform_ints``: re, im independent uniform integers in [lo, hi].
* ``correlated_gaussian``: x_i = rint(sigma * (sqrt(rho) s + sqrt(1 - rho) n_i)),
  with s (common to all inputs) and n_i complex standard normal (unit variance
  in each of re and im), clipped to +-clip.  ``rho = 0`` gives independent
  Gaussian inputs.  With ``as_float=True`` no rounding or clipping is applied.
"""
from __future__ import annotations

import numpy as np


def uniform_ints(seed: int, n_time: int, n_chan: int, n_inputs: int, lo: int = -7, hi: int = 7):
    """Return (re, im) int16 arrays ``[T][C][N]`` of independent uniform integers in [lo, hi]."""
    rng = np.random.default_rng(seed)
    shape = (n_time, n_chan, n_inputs)
    re = rng.integers(lo, hi + 1, size=shape, dtype=np.int16)
    im = rng.integers(lo, hi + 1, size=shape, dtype=np.int16)
    return re, im


def correlated_gaussian(seed: int, n_time: int, n_chan: int, n_inputs: int, sigma: float,
                        rho: float = 0.0, clip: int = 127, as_float: bool = False):
    """Return (re, im) arrays ``[T][C][N]``: int16 when quantised, float32 when ``as_float``."""
    rng = np.random.default_rng(seed)
    shape = (n_time, n_chan, n_inputs)
    a = np.sqrt(1.0 - rho)
    re = rng.standard_normal(size=shape, dtype=np.float32) * np.float32(a)
    im = rng.standard_normal(size=shape, dtype=np.float32) * np.float32(a)
    if rho > 0.0:
        b = np.float32(np.sqrt(rho))
        sr = rng.standard_normal(size=(n_time, n_chan, 1), dtype=np.float32) * b
        si = rng.standard_normal(size=(n_time, n_chan, 1), dtype=np.float32) * b
        re += sr
        im += si
    re *= np.float32(sigma)
    im *= np.float32(sigma)
    if as_float:
        return re, im
    re = np.clip(np.rint(re), -clip, clip).astype(np.int16)
    im = np.clip(np.rint(im), -clip, clip).astype(np.int16)
    return re, im


def pack4(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack int components in [-8, 7] into one byte each: high nibble re, low nibble im."""
    if re.min(initial=0) < -8 or re.max(initial=0) > 7 or im.min(initial=0) < -8 or im.max(initial=0) > 7:
        raise ValueError("4-bit samples must lie in [-8, 7]")
    hi = (re.astype(np.int16) & 0xF).astype(np.uint8)
    lo = (im.astype(np.int16) & 0xF).astype(np.uint8)
    return ((hi << 4) | lo).astype(np.uint8)


def pack8(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack int components in [-128, 127] as interleaved int8 (re, im) bytes: shape ``[T][C][N][2]``."""
    if re.min(initial=0) < -128 or re.max(initial=0) > 127 or im.min(initial=0) < -128 or im.max(initial=0) > 127:
        raise ValueError("8-bit samples must lie in [-128, 127]")
    out = np.empty(re.shape + (2,), dtype=np.int8)
    out[..., 0] = re
    out[..., 1] = im
    return out.view(np.uint8)


def packf32(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack float components as interleaved float32 (re, im): shape ``[T][C][N][2]``."""
    out = np.empty(re.shape + (2,), dtype=np.float32)
    out[..., 0] = re
    out[..., 1] = im
    return out


def pack_real8(x: np.ndarray) -> np.ndarray:
    """Real 8-bit samples (int8 two's complement), one byte each, same order as ``x``."""
    x = np.asarray(x)
    if x.min(initial=0) < -128 or x.max(initial=0) > 127:
        raise ValueError("8-bit samples must lie in [-128, 127]")
    return x.astype(np.int8).view(np.uint8)


def pack(re: np.ndarray, im: np.ndarray, bits: int) -> np.ndarray:
    if bits == 4:
        return pack4(re, im)
    if bits == 8:
        return pack8(re, im)
    if bits == 32:
        return packf32(re, im)
    raise ValueError(f"sample_bits must be 4, 8 or 32, got {bits}")


def packed_nbytes(n_time: int, n_chan: int, n_inputs: int, bits: int) -> int:
    per = {4: 1, 8: 2, 32: 8}[bits]
    return n_time * n_chan * n_inputs * per


# ---- the workloads of the paper's prototype, scaled as described in the design notes ----

def workload(name: str, dump: int = 0, as_float: bool = False):
    """Return (re, im, bits, dims) for one dump of a named workload.

    ``dims`` is (n_inputs, n_chan, n_time).  Seeds follow ``seed = 1000 * cfg + dump``.
    """
    if name == "mwa32t_4bit":            # 32 antennas x 2 pol, 128 channels, 512 samples, 4-bit
        n, c, t = 64, 128, 512
        re, im = uniform_ints(1000 + dump, t, c, n, -7, 7)
        return re, im, 4, (n, c, t)
    if name == "stream64_8bit":          # 64 inputs, 768 channels, 1000 samples per dump, rho = 0.1
        n, c, t = 64, 768, 1000
        re, im = correlated_gaussian(2000 + dump, t, c, n, 16.0, 0.1, 127, as_float=as_float)
        return re, im, (32 if as_float else 8), (n, c, t)
    if name == "large1024_8bit":         # 512 antennas x 2 pol, 1536 channels, 256 samples
        n, c, t = 1024, 1536, 256
        re, im = correlated_gaussian(3000 + dump, t, c, n, 8.0, 0.0, 127, as_float=as_float)
        return re, im, (32 if as_float else 8), (n, c, t)
    raise KeyError(name)


def torch_correlated_gaussian_packed8(n_dumps: int, n_time: int, n_chan: int, n_inputs: int,
                                      sigma: float, rho: float, seed: int, device):
    """Device-side generator for bench-sized inputs: same recipe, torch's seeded generator.

    Returns a uint8 tensor ``[n_dumps][T][C][N][2]`` (int8 re, im bytes).  Generated one
    dump at a time to bound the temporary memory.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty((n_dumps, n_time, n_chan, n_inputs, 2), dtype=torch.int8, device=device)
    a = float(np.sqrt(1.0 - rho))
    b = float(np.sqrt(rho))
    for d in range(n_dumps):
        z = torch.randn((n_time, n_chan, n_inputs, 2), generator=g, device=device) * a
        if rho > 0.0:
            s = torch.randn((n_time, n_chan, 1, 2), generator=g, device=device) * b
            z += s
        z.mul_(sigma).round_().clamp_(-127, 127)
        out[d].copy_(z.to(torch.int8))
        del z
    return out.view(torch.uint8)


def torch_correlated_gaussian_f32(n_dumps: int, n_time: int, n_chan: int, n_inputs: int,
                                  sigma: float, rho: float, seed: int, device):
    """Device-side float variant of the same recipe (no rounding, no clipping): float32
    ``[n_dumps][T][C][N][2]`` (re, im), generated one dump at a time."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty((n_dumps, n_time, n_chan, n_inputs, 2), dtype=torch.float32, device=device)
    a = float(np.sqrt(1.0 - rho))
    b = float(np.sqrt(rho))
    for d in range(n_dumps):
        z = torch.randn((n_time, n_chan, n_inputs, 2), generator=g, device=device) * a
        if rho > 0.0:
            z += torch.randn((n_time, n_chan, 1, 2), generator=g, device=device) * b
        out[d].copy_(z.mul_(sigma))
        del z
    return out


def torch_uniform_packed4(n_dumps: int, n_time: int, n_chan: int, n_inputs: int, seed: int, device,
                          lo: int = -7, hi: int = 7):
    """Device-side uniform 4-bit generator: uint8 ``[n_dumps][T][C][N]`` (high nibble re, low im)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    re = torch.randint(lo, hi + 1, (n_dumps, n_time, n_chan, n_inputs), generator=g, device=device,
                       dtype=torch.int16)
    im = torch.randint(lo, hi + 1, (n_dumps, n_time, n_chan, n_inputs), generator=g, device=device,
                       dtype=torch.int16)
    return (((re & 0xF) << 4) | (im & 0xF)).to(torch.uint8)

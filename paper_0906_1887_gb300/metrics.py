"""Throughput, real-time and bandwidth bookkeeping for the X stage.

* CMAC count: one complex multiply-accumulate per input pair (autos included), per
  channel, per time sample; N(N+1)/2 pairs (Sec. 2).  A CMAC is 4 real multiply-adds,
  8 real operations.
* Real-time factor: seconds of signal processed per wall-clock second.  The paper's
  prototype channelises a 1.28 MHz band into 128 channels (Sec. 5), so one channel
  carries 10 k complex samples per second.
* Memory-bound bandwidth model (Sec. 6): the CMAC stage reads epsilon * 4 * B * N (N+1)
  bytes per second of single-precision complex data, so a GPU with global-memory
  throughput M can keep up with at most B = M / (4 epsilon N (N+1)) of signal bandwidth;
  epsilon is the number of global reads per product per channel of a design (2, 1.5,
  1.25, 1, 0.5 for PP, HG2, HG4, GP2, GP4).
* Processed bandwidth (Sec. 6, Table 4): a band of B_sig processed in t seconds per
  second of data sustains B_sig / t of signal bandwidth.
"""
from __future__ import annotations

# the paper's per-design global-memory reads per product per channel (Sec. 6)
EPSILON = {"PP": 2.0, "HG2": 1.5, "HG4": 1.25, "GP2": 1.0, "GP4": 0.5}

CHANNEL_RATE_HZ = 1.28e6 / 128.0    # complex samples per second per channel (Sec. 3, Sec. 5)


def n_baselines(n_inputs: int) -> int:
    """Correlation products including autos: N(N+1)/2 (Sec. 2)."""
    return n_inputs * (n_inputs + 1) // 2


def cmacs(n_inputs: int, n_chan: int, n_time: int, n_dumps: int = 1) -> int:
    """Algorithmic CMACs of n_dumps dumps (only the N(N+1)/2 distinct products count)."""
    return n_baselines(n_inputs) * n_chan * n_time * n_dumps


def tera_cmac_per_s(n_cmac: float, seconds: float) -> float:
    return n_cmac / seconds / 1e12


def real_time_factor(n_time: int, n_dumps: int, seconds: float, channel_rate_hz: float = CHANNEL_RATE_HZ) -> float:
    """Seconds of signal processed per second of wall time."""
    return (n_time * n_dumps / channel_rate_hz) / seconds


def max_signal_bandwidth_hz(mem_bytes_per_s: float, epsilon: float, n_inputs: int) -> float:
    """B = M / (4 eps N (N+1)): the memory-bound ceiling of the CMAC stage (Sec. 6)."""
    return mem_bytes_per_s / (4.0 * epsilon * n_inputs * (n_inputs + 1))


def processed_bandwidth_hz(signal_bw_hz: float, seconds_per_second_of_data: float) -> float:
    """Signal bandwidth sustained when one second of B_sig data takes the given time (Table 4)."""
    return signal_bw_hz / seconds_per_second_of_data


def mhz_at_64_inputs(tera_cmac: float) -> float:
    """Signal bandwidth (MHz) a CMAC rate could process for the paper's 64-input system."""
    return tera_cmac * 1e12 / n_baselines(64) / 1e6


def packed_bytes(n_inputs: int, n_chan: int, n_time: int, sample_bits: int) -> int:
    per = {4: 1, 8: 2, 32: 8}[sample_bits]
    return n_inputs * n_chan * n_time * per


def vis_bytes(n_inputs: int, n_chan: int, sample_bits: int) -> int:
    """Output bytes of one dump: int64 (re, im) for integer samples, float32 for float samples."""
    per = 16 if sample_bits in (4, 8) else 8
    return n_baselines(n_inputs) * n_chan * per

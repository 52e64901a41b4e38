"""Pins of the throughput/bandwidth bookkeeping against the paper's printed tables."""
import os

import pytest

from paper_0906_1887_gb300 import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table4_bandwidth.txt")


def _rows():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        # half a unit in the last printed digit ("10" and "12" carry no decimal)
        tol = 0.5 if "." not in f[5] else 0.05
        yield f[0], float(f[1]), f[2], float(f[3]), float(f[4]), float(f[5]), float(f[6]), (f[7] if len(f) > 7 else ""), tol


@pytest.mark.parametrize("row", list(_rows()), ids=lambda r: f"{r[0]}-{r[2]}")
def test_table4(row):
    gpu, mem, design, ms, actual, theory, pct, flag, tol = row
    th = metrics.max_signal_bandwidth_hz(mem * 1e9, metrics.EPSILON[design], 64) / 1e6
    act = metrics.processed_bandwidth_hz(1.28e6, ms / 1000.0) / 1e6
    assert abs(act - actual) <= 0.051                      # printed to 0.1 MHz
    if flag != "theory_typo":
        assert abs(th - theory) <= tol + 0.02              # one row (3.46 -> 3.4) truncates
    assert abs(100.0 * act / th - pct) <= 1.0              # the printed ratio


def test_cmac_counts():
    # one second of the prototype's 1.28 MHz band at 64 inputs: 2080 * 1.28e6 CMAC (Sec. 6)
    assert metrics.n_baselines(64) == 2080
    assert metrics.cmacs(64, 128, 10000) == 2080 * 1.28e6
    # Table 3: the single-threaded CPU CMAC takes 20950 ms per second of data
    assert abs(metrics.cmacs(64, 128, 10000) / 20.950 / 1e9 - 0.127) < 0.001


def test_real_time_factor():
    # 10 k samples per channel per second: 1000 samples per dump are 0.1 s of signal
    assert metrics.real_time_factor(1000, 1, 0.05) == pytest.approx(2.0)
    assert metrics.real_time_factor(256, 20, 0.512) == pytest.approx(1.0)

"""Batched uneven jobs in one persistent launch (plus CUDA graph and autotuner), bit-exact vs the oracle."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_0906_1887_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JOBS = [  # (n_inputs, n_chan, n_time, bits): every array size and mode the batch path takes
    (32, 65, 200, 8), (64, 33, 1100, 8), (128, 7, 300, 8), (256, 3, 129, 8), (64, 64, 64, 8),
    (16, 9, 77, 4), (64, 12, 513, 4), (96, 5, 2100, 8), (48, 3, 256, 4), (512, 1, 128, 8),
    # 4-bit arrays of several blocks: e4m3 operands, converted in the kernel or read from e4m3 planes
    (256, 3, 300, 4), (192, 2, 129, 4),
]


@pytest.fixture(scope="module")
def jobs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = []
    for k, (n, c, t, bits) in enumerate(JOBS):
        lo, hi = (-8, 7) if bits == 4 else (-128, 127)
        re, im = synth.uniform_ints(500 + k, t, c, n, lo, hi)
        packed = synth.pack(re, im, bits)
        ref = oracle.xcorr_int(packed, n, c, t, bits)
        x = torch.from_numpy(packed.reshape(-1).view(np.uint8)).cuda()
        vis = torch.full((c, n * (n + 1) // 2, 2), -5, dtype=torch.int64, device="cuda")
        out.append(dict(n=n, c=c, t=t, bits=bits, x=x, vis=vis, ref=ref))
    return out


def _descs(jobs):
    return [(j["n"], j["c"], j["t"], j["bits"], j["x"], j["vis"]) for j in jobs]


def _check(jobs):
    for j in jobs:
        assert np.array_equal(j["vis"].cpu().numpy(), j["ref"]), (j["n"], j["c"], j["t"], j["bits"])


@pytest.mark.parametrize("flags", [0, 1])
def test_batch_bit_exact(jobs, flags):
    from paper_0906_1887_gb300 import corr
    for j in jobs:
        j["vis"].fill_(-5)
    b = corr.Batch(_descs(jobs), flags=flags)
    info = b.info()
    assert info["n_jobs"] == len(jobs) and info["n_launches"] == 2 and info["graph"] == flags
    for _ in range(2):        # a replayed graph gives the same answer
        b.run()
        torch.cuda.synchronize()
        assert b.check_device() == 0
        _check(jobs)
    b.close()


def test_batch_autotune_cache_and_accumulate(jobs):
    from paper_0906_1887_gb300 import corr
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "tune.jsonl")
        b = corr.Batch(_descs(jobs), flags=corr.BATCH_AUTOTUNE | corr.BATCH_GRAPH, tune_cache=cache)
        info = b.info()
        assert info["tuned"] == 1 and info["tune_ms"] > 0 and os.path.getsize(cache) > 0
        b.run()
        torch.cuda.synchronize()
        _check(jobs)
        b.close()
        # a second batch with the same sizes takes the cached choice without timing runs
        b2 = corr.Batch(_descs(jobs), flags=corr.BATCH_AUTOTUNE, tune_cache=cache)
        i2 = b2.info()
        assert (i2["op_stages"], i2["pair_cpi"], i2["order"]) == (info["op_stages"], info["pair_cpi"], info["order"])
        b2.close()
    # accumulate: visibilities hold V already, one more run doubles them
    b3 = corr.Batch(_descs(jobs), flags=corr.BATCH_ACCUMULATE)
    b3.run()
    torch.cuda.synchronize()
    for j in jobs:
        assert np.array_equal(j["vis"].cpu().numpy(), 2 * j["ref"])
    b3.close()
    with pytest.raises(corr.CorrError):
        corr.Batch(_descs(jobs), flags=corr.BATCH_AUTOTUNE | corr.BATCH_ACCUMULATE)


def test_batch_rejects_unaddressable_rows():
    from paper_0906_1887_gb300 import corr
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = torch.zeros(17 * 4 * 10 * 2, dtype=torch.uint8, device="cuda")
    v = torch.zeros((4, 17 * 18 // 2, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(corr.CorrError) as e:
        corr.Batch([(17, 4, 10, 8, x, v)])
    assert e.value.status == corr.EUNSUPPORTED


@pytest.mark.parametrize("graph", [0, 1])
def test_batch_plane_path_every_shape_bit_exact(jobs, graph):
    # the plane operand path (unpack kernel + plane-fed tensor-core kernel) for multi-block jobs,
    # mixed with the packed-sample path for the others, in every shape the tuner can choose
    from paper_0906_1887_gb300 import corr
    b = corr.Batch(_descs(jobs), flags=corr.BATCH_PLANES | (corr.BATCH_GRAPH if graph else 0))
    info = b.info()
    assert info["plane_bytes"] > 0 and info["plane_min_nb"] == 4
    for plane_min_nb, order, ops, wide, splits in [(0, 0, 0, 1, 1), (2, 0, 3, 1, 1), (4, 1, 5, 0, 1), (8, 0, 4, 1, 1),
                                                   (2, 1, 0, 0, 1), (2, 0, 0, 1, 2), (2, 0, 0, 1, 3), (2, 1, 4, 0, 8)]:
        # plane_splits > 1: the plane jobs in several launches, unpacks overlapped on another stream
        b.set_shape(ops, 2, order, plane_min_nb, wide, splits)
        for j in jobs:
            j["vis"].fill_(-5)
        b.run()
        torch.cuda.synchronize()
        assert b.check_device() == 0
        _check(jobs)
    b.close()


def test_batch_autotune_with_planes(jobs):
    from paper_0906_1887_gb300 import corr
    b = corr.Batch(_descs(jobs), flags=corr.BATCH_AUTOTUNE | corr.BATCH_PLANES)
    info = b.info()
    assert info["tuned"] == 1 and info["plane_min_nb"] in (0, 2, 4, 8) and info["wide"] in (0, 1)
    assert 1 <= info["plane_splits"] <= 4
    for j in jobs:
        j["vis"].fill_(-5)
    b.run()
    torch.cuda.synchronize()
    _check(jobs)
    with pytest.raises(corr.CorrError):
        corr.Batch(_descs(jobs)).set_shape(0, 2, 0, 2, 1)   # planes need CORR_BATCH_PLANES
    with pytest.raises(corr.CorrError):
        b.set_shape(0, 2, 0, 2, 1, 9)   # at most 8 plane launches
    b.close()

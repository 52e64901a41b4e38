"""Serving loop: jobs from concurrent host threads, HBM-footprint admission, polling, and
failure detection made on the host (a paused dispatcher, a job too large for the budget).
No test faults, traps or hangs the GPU."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_0906_1887_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _job(seed, n, c, t, bits):
    if bits == 32:
        re, im = synth.correlated_gaussian(seed, t, c, n, 2.0, 0.2, as_float=True)
        packed = synth.packf32(re, im)
        ref = oracle.xcorr_f64(packed, n, c, t)
    else:
        lo, hi = (-8, 7) if bits == 4 else (-128, 127)
        re, im = synth.uniform_ints(seed, t, c, n, lo, hi)
        packed = synth.pack(re, im, bits)
        ref = oracle.xcorr_int(packed, n, c, t, bits)
    host_in = torch.from_numpy(np.ascontiguousarray(packed).reshape(-1).view(np.uint8)).pin_memory()
    dtype = torch.float32 if bits == 32 else torch.int64
    host_out = torch.empty((c, n * (n + 1) // 2, 2), dtype=dtype).pin_memory()
    return dict(n=n, c=c, t=t, bits=bits, host_in=host_in, host_out=host_out, ref=ref, packed=packed)


JOBS = [(64, 40, 1000, 8), (128, 9, 300, 8), (32, 30, 512, 4), (17, 5, 100, 8), (256, 3, 200, 8),
        (64, 16, 2100, 8), (48, 11, 64, 4), (40, 6, 90, 32)]


def test_concurrent_submitters_bit_exact():
    from paper_0906_1887_gb300 import corr
    jobs = [_job(900 + k, *spec) for k, spec in enumerate(JOBS)]
    srv = corr.Server(512 * MiB, n_streams=4)
    ids = [None] * len(jobs)

    def submit(k):
        j = jobs[k]
        ids[k] = srv.submit(j["n"], j["c"], j["t"], j["bits"], j["host_in"], j["host_out"], stream_tag=k % 3)

    threads = [threading.Thread(target=submit, args=(k,)) for k in range(len(jobs))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for k, j in enumerate(jobs):
        st, r = srv.wait(ids[k], 60.0)
        assert st == corr.OK, (k, st, corr.last_error())
        assert r.t_submit <= r.t_start <= r.t_done
        got = j["host_out"].numpy()
        if j["bits"] == 32:
            from _gpu_helpers import check_bf16x3
            check_bf16x3(got, j["packed"], j["n"], j["c"], j["t"])
        else:
            assert np.array_equal(got, j["ref"]), JOBS[k]
        srv.release(ids[k])
    s = srv.stats()
    assert s["completed"] == len(jobs) and s["failed"] == 0 and s["bytes_in_use"] == 0
    assert srv.close() == corr.OK


def test_device_resident_result_and_admission_queueing():
    from paper_0906_1887_gb300 import corr
    # each job needs ~11 MiB on the device; a 24 MiB budget admits two at a time
    jobs = [_job(950 + k, 64, 64, 1000, 8) for k in range(5)]
    srv = corr.Server(24 * MiB, n_streams=4)
    ids = [srv.submit(j["n"], j["c"], j["t"], j["bits"], j["host_in"], None) for j in jobs]
    for k, j in enumerate(jobs):
        st, r = srv.wait(ids[k], 60.0)
        assert st == corr.OK and r.d_vis
        # the result stays in the arena until released
        out = np.zeros(j["ref"].shape, dtype=np.int64)
        srv.fetch(ids[k], out.ctypes.data)
        assert np.array_equal(out, j["ref"])
        srv.release(ids[k])
    s = srv.stats()
    assert s["peak_bytes"] <= 24 * MiB and s["completed"] == 5 and s["bytes_in_use"] == 0
    srv.close()


def test_rejection_and_host_side_failures():
    from paper_0906_1887_gb300 import corr
    srv = corr.Server(4 * MiB, n_streams=2, flags=corr.SERVER_START_PAUSED)
    big = _job(1, 64, 256, 1000, 8)                       # > 4 MiB of device footprint
    with pytest.raises(corr.CorrError) as e:
        srv.submit(big["n"], big["c"], big["t"], 8, big["host_in"], big["host_out"])
    assert e.value.status == corr.EBUSY
    with pytest.raises(corr.CorrError):
        srv.submit(0, 1, 1, 8, big["host_in"], None)
    small = _job(2, 16, 4, 64, 8)
    jid = srv.submit(16, 4, 64, 8, small["host_in"], small["host_out"])
    # the dispatcher is paused: the job stays queued and a bounded wait gives up
    st, _ = srv.poll(jid)
    assert st == corr.PENDING
    t0 = time.time()
    st, _ = srv.wait(jid, 0.2)
    assert st == corr.ETIMEOUT and time.time() - t0 < 5
    srv.resume()
    st, _ = srv.wait(jid, 30.0)
    assert st == corr.OK and np.array_equal(small["host_out"].numpy(), small["ref"])
    s = srv.stats()
    assert s["rejected"] == 1
    srv.close()


def test_shutdown_cancels_queued_jobs():
    from paper_0906_1887_gb300 import corr
    srv = corr.Server(8 * MiB, n_streams=2, flags=corr.SERVER_START_PAUSED)
    j = _job(3, 32, 8, 128, 8)
    ids = [srv.submit(32, 8, 128, 8, j["host_in"], j["host_out"]) for _ in range(3)]
    t0 = time.time()
    assert srv.close(drain_timeout_s=5.0) == corr.OK     # nothing was running: prompt return
    assert time.time() - t0 < 5

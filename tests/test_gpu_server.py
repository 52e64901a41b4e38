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


# ---- open streams: device sample rings and accumulators (Fig. 1) ----

def _stream_jobs(seed, k, n, c, t, bits):
    lo, hi = (-8, 7) if bits == 4 else (-128, 127)
    packs = []
    for m in range(k):
        re, im = synth.uniform_ints(seed + m, t, c, n, lo, hi)
        packs.append(np.ascontiguousarray(synth.pack(re, im, bits)))
    return packs


@pytest.mark.parametrize("n,c,t,bits,ring", [(64, 12, 300, 8, 2), (96, 5, 130, 4, 3), (40, 6, 100, 8, 1),
                                             # the plane feed: rows of 130 bytes; 256 inputs of 4 bits
                                             (65, 3, 200, 8, 2), (256, 2, 70, 4, 2)])
def test_open_stream_sums_equal_oracle_over_concatenated_samples(n, c, t, bits, ring):
    # additivity: the k jobs of one interval sum to the correlation of their concatenated samples
    from paper_0906_1887_gb300 import corr
    k = 5
    packs = _stream_jobs(4000 + n, 2 * k, n, c, t, bits)
    host_in = [torch.from_numpy(p.reshape(-1).view(np.uint8)).pin_memory() for p in packs]
    P = n * (n + 1) // 2
    outs = [torch.full((c, P, 2), -1, dtype=torch.int64).pin_memory() for _ in range(2)]
    srv = corr.Server(256 * MiB, n_streams=2)
    srv.open_stream(7, n, c, t, bits, ring_slots=ring, jobs_per_dump=k)
    assert srv.stats()["open_streams"] == 1
    ids = []
    for m in range(2 * k):
        closes = (m + 1) % k == 0
        ids.append(srv.submit(n, c, t, bits, host_in[m], outs[m // k] if closes else None, stream_tag=7))
    for m, jid in enumerate(ids):
        st, r = srv.wait(jid, 60.0)
        assert st == corr.OK, (m, st, corr.last_error())
        assert r.closed_interval == int((m + 1) % k == 0)
        if r.closed_interval:
            assert r.n_accum == k * t
        srv.release(jid)
    for iv in range(2):
        allp = np.concatenate([packs[iv * k + m].reshape(t, c, -1) for m in range(k)])   # [k t][C][...]
        ref = oracle.xcorr_int(allp, n, c, k * t, bits)
        assert np.array_equal(outs[iv].numpy(), ref), iv
    assert srv.close_stream(7) == corr.OK
    s = srv.stats()
    assert s["open_streams"] == 0 and s["bytes_in_use"] == 0 and s["completed"] == 2 * k
    srv.close()


def test_open_stream_averaged_dump_with_phase_correction():
    from oracle import dump as odump
    from paper_0906_1887_gb300 import corr
    n, c, t, bits, k = 64, 8, 256, 8, 3
    packs = _stream_jobs(4500, k, n, c, t, bits)
    rng = np.random.default_rng(9)
    tau = rng.normal(0, 1e-6, n)
    nu = 1.5e8 + 1e4 * np.arange(c)
    d_tau = torch.from_numpy(tau).cuda()
    d_nu = torch.from_numpy(nu).cuda()
    srv = corr.Server(128 * MiB, n_streams=2)
    srv.open_stream(3, n, c, t, bits, ring_slots=2, jobs_per_dump=k, dump_mode=corr.STREAM_DUMP_AVERAGED,
                    delays=d_tau, freqs=d_nu)
    P = n * (n + 1) // 2
    out = torch.zeros((c, P, 2), dtype=torch.float32).pin_memory()
    # host buffers stay alive (and unchanged) until their jobs finish
    host_in = [torch.from_numpy(p.reshape(-1).view(np.uint8)).pin_memory() for p in packs]
    ids = [srv.submit(n, c, t, bits, host_in[m], out if m == k - 1 else None, stream_tag=3) for m in range(k)]
    for jid in ids:
        st, r = srv.wait(jid, 60.0)
        assert st == corr.OK, corr.last_error()
    allp = np.concatenate([p.reshape(t, c, -1) for p in packs])
    want = odump.dump_corrected(oracle.xcorr_int(allp, n, c, k * t, bits), k * t, tau, nu)
    got = out.numpy().astype(np.float64)
    mag = np.hypot(want[..., 0], want[..., 1])
    assert np.all(np.hypot(*(got - want).transpose(2, 0, 1)) <= 8 * 2.0 ** -24 * mag + 1e-30)
    # the same stream keeps going: the dump reset the accumulators, so the next interval is fresh
    ids2 = [srv.submit(n, c, t, bits, host_in[m], out if m == k - 1 else None, stream_tag=3) for m in range(k)]
    for jid in ids2:
        assert srv.wait(jid, 60.0)[0] == corr.OK
    got2 = out.numpy().astype(np.float64)
    assert np.all(np.hypot(*(got2 - want).transpose(2, 0, 1)) <= 8 * 2.0 ** -24 * mag + 1e-30)
    srv.close()


def test_open_stream_rejections():
    from paper_0906_1887_gb300 import corr
    srv = corr.Server(8 * MiB, n_streams=2)
    with pytest.raises(corr.CorrError) as e:      # state larger than the arena
        srv.open_stream(1, 1024, 64, 256, 8, ring_slots=2, jobs_per_dump=4)
    assert e.value.status == corr.EBUSY
    srv.open_stream(2, 16, 4, 64, 8, ring_slots=2, jobs_per_dump=2)
    with pytest.raises(corr.CorrError):           # tag already open
        srv.open_stream(2, 16, 4, 64, 8)
    j = _job(5, 16, 4, 64, 8)
    with pytest.raises(corr.CorrError):           # shape differs from the stream's
        srv.submit(16, 4, 65, 8, j["host_in"], None, stream_tag=2)
    a = srv.submit(16, 4, 64, 8, j["host_in"], None, stream_tag=2)
    with pytest.raises(corr.CorrError):           # the interval's last job needs host_vis for the sums
        srv.submit(16, 4, 64, 8, j["host_in"], None, stream_tag=2)
    b = srv.submit(16, 4, 64, 8, j["host_in"], j["host_out"], stream_tag=2)
    assert srv.wait(a, 30.0)[0] == corr.OK and srv.wait(b, 30.0)[0] == corr.OK
    assert np.array_equal(j["host_out"].numpy(), 2 * j["ref"])
    # a job of another tag still goes through the arena meanwhile
    c_ = srv.submit(16, 4, 64, 8, j["host_in"], j["host_out"], stream_tag=9)
    assert srv.wait(c_, 30.0)[0] == corr.OK and np.array_equal(j["host_out"].numpy(), j["ref"])
    assert srv.close_stream(2) == corr.OK
    srv.close()


def test_large_job_on_the_plane_feed():
    # a 1024-input job of 40 channels x 2048 samples (the plane feed with wide items) matches the
    # oracle on sampled channels, as an arena job and as the two accumulating jobs of an open
    # stream's interval
    from paper_0906_1887_gb300 import corr
    n, c, t = 1024, 40, 2048
    packs = []
    for k in range(2):
        re, im = synth.uniform_ints(8100 + k, t, c, n, -128, 127)
        packs.append(np.ascontiguousarray(synth.pack(re, im, 8)))
    host_in = [torch.from_numpy(p.reshape(-1).view(np.uint8)).pin_memory() for p in packs]
    P = n * (n + 1) // 2
    out = torch.empty((c, P, 2), dtype=torch.int64).pin_memory()
    chans = [0, 36, 37, 39]
    srv = corr.Server(4096 * MiB, n_streams=2)
    jid = srv.submit(n, c, t, 8, host_in[0], out)
    assert srv.wait(jid, 120.0)[0] == corr.OK, corr.last_error()
    ref = oracle.xcorr_int(packs[0], n, c, t, 8, chans=chans)
    for k, ch in enumerate(chans):
        assert np.array_equal(out.numpy()[ch], ref[k]), ch
    srv.release(jid)
    srv.open_stream(5, n, c, t, 8, ring_slots=2, jobs_per_dump=2)
    out.fill_(-1)
    ids = [srv.submit(n, c, t, 8, host_in[0], None, stream_tag=5), srv.submit(n, c, t, 8, host_in[1], out, stream_tag=5)]
    for i in ids:
        assert srv.wait(i, 120.0)[0] == corr.OK, corr.last_error()
    ref = oracle.xcorr_int(np.concatenate([p.reshape(t, c, -1) for p in packs]), n, c, 2 * t, 8, chans=chans)
    for k, ch in enumerate(chans):
        assert np.array_equal(out.numpy()[ch], ref[k]), ch
    srv.close()


def test_close_stream_bounded_when_jobs_cannot_run():
    # host-made failure: the dispatcher is paused, so the stream's queued jobs never start;
    # close_stream gives up after its bound, cancels them and the server stays usable
    from paper_0906_1887_gb300 import corr
    srv = corr.Server(64 * MiB, n_streams=2, flags=corr.SERVER_START_PAUSED)
    srv.open_stream(4, 32, 4, 64, 8, ring_slots=2, jobs_per_dump=2)
    j = _job(6, 32, 4, 64, 8)
    a = srv.submit(32, 4, 64, 8, j["host_in"], None, stream_tag=4)
    b = srv.submit(32, 4, 64, 8, j["host_in"], j["host_out"], stream_tag=4)
    t0 = time.time()
    assert srv.close_stream(4, drain_timeout_s=0.2) == corr.ETIMEOUT
    assert time.time() - t0 < 20
    assert srv.poll(a)[0] == corr.EBUSY and srv.poll(b)[0] == corr.EBUSY     # cancelled
    assert srv.stats()["open_streams"] == 0 and srv.stats()["bytes_in_use"] == 0
    # the tag is free again and the server still runs jobs once resumed
    srv.resume()
    c_ = srv.submit(32, 4, 64, 8, j["host_in"], j["host_out"], stream_tag=4)
    assert srv.wait(c_, 30.0)[0] == corr.OK and np.array_equal(j["host_out"].numpy(), j["ref"])
    srv.close()


def test_destroy_with_open_streams_and_queued_jobs():
    from paper_0906_1887_gb300 import corr
    srv = corr.Server(64 * MiB, n_streams=2)
    srv.open_stream(1, 64, 8, 256, 8, ring_slots=3, jobs_per_dump=4)
    srv.open_stream(2, 16, 4, 64, 4, ring_slots=1, jobs_per_dump=1, dump_mode=corr.STREAM_DUMP_AVERAGED)
    j = _job(7, 64, 8, 256, 8)
    k = _job(8, 16, 4, 64, 4)
    ids = [srv.submit(64, 8, 256, 8, j["host_in"], None, stream_tag=1) for _ in range(3)]
    ids += [srv.submit(16, 4, 64, 4, k["host_in"], None, stream_tag=2) for _ in range(3)]
    assert srv.close(drain_timeout_s=30.0) == corr.OK


def test_earliest_deadline_first_issue_order():
    # jobs queued while the dispatcher is paused start in order of their deadlines (submission
    # time + their own sample time), not in order of arrival: the first queued job of each open
    # stream and the first arena job are the candidates
    from paper_0906_1887_gb300 import corr
    srv = corr.Server(256 * MiB, n_streams=2, flags=corr.SERVER_START_PAUSED)
    specs = {1: (32, 4, 2048), 3: (32, 4, 512), 2: (32, 4, 64)}    # tag -> (n, c, t)
    for tag, (n, c, t) in specs.items():
        srv.open_stream(tag, n, c, t, 8, ring_slots=2, jobs_per_dump=1)
    jobs, ids = {}, {}
    for tag, (n, c, t) in specs.items():                           # arrival order 1, 3, 2
        jobs[tag] = _job(7000 + tag, n, c, t, 8)
        ids[tag] = srv.submit(n, c, t, 8, jobs[tag]["host_in"], jobs[tag]["host_out"], stream_tag=tag)
    jobs["arena"] = _job(7100, 32, 4, 128, 8)
    ids["arena"] = srv.submit(32, 4, 128, 8, jobs["arena"]["host_in"], jobs["arena"]["host_out"])
    srv.resume()
    starts = {}
    for key, jid in ids.items():
        st, r = srv.wait(jid, 60.0)
        assert st == corr.OK, (key, corr.last_error())
        assert np.array_equal(jobs[key]["host_out"].numpy(), jobs[key]["ref"]), key
        starts[key] = r.t_start
        srv.release(jid)
    # deadlines: tag 2 (64 samples) < arena (128) < tag 3 (512) < tag 1 (2048)
    assert sorted(starts, key=starts.get) == [2, "arena", 3, 1], starts
    for tag in specs:
        assert srv.close_stream(tag) == corr.OK
    srv.close()


@pytest.mark.parametrize("n,c,t,bits,ring", [(64, 12, 300, 8, 4), (256, 2, 70, 4, 4), (96, 5, 130, 4, 3)])
def test_open_stream_coalesced_jobs_equal_oracle(n, c, t, bits, ring):
    # jobs queued while the dispatcher is paused run in pairs of adjacent ring slots (one X stage
    # over both jobs' samples, packed feed or planes); the interval sums still equal the
    # correlation of the concatenated samples, and every job completes with its own status
    from paper_0906_1887_gb300 import corr
    k = 5
    packs = _stream_jobs(7300 + n, 2 * k, n, c, t, bits)
    host_in = [torch.from_numpy(p.reshape(-1).view(np.uint8)).pin_memory() for p in packs]
    P = n * (n + 1) // 2
    outs = [torch.full((c, P, 2), -1, dtype=torch.int64).pin_memory() for _ in range(2)]
    srv = corr.Server(256 * MiB, n_streams=2, flags=corr.SERVER_START_PAUSED)
    srv.open_stream(11, n, c, t, bits, ring_slots=ring, jobs_per_dump=k)
    ids = []
    for m in range(2 * k):
        closes = (m + 1) % k == 0
        ids.append(srv.submit(n, c, t, bits, host_in[m], outs[m // k] if closes else None, stream_tag=11))
    srv.resume()
    for m, jid in enumerate(ids):
        st, r = srv.wait(jid, 60.0)
        assert st == corr.OK, (m, st, corr.last_error())
        assert r.closed_interval == int((m + 1) % k == 0)
        srv.release(jid)
    for iv in range(2):
        allp = np.concatenate([packs[iv * k + m].reshape(t, c, -1) for m in range(k)])
        assert np.array_equal(outs[iv].numpy(), oracle.xcorr_int(allp, n, c, k * t, bits)), iv
    s = srv.stats()
    # the first interval's jobs 0+1 and (with 4 slots) 2+3 pair up for certain: their slots are
    # free from the start (the closing job 4 runs alone, and a pair never wraps around the ring)
    assert s["coalesced"] >= (4 if ring >= 4 else 2) and s["completed"] == 2 * k and s["failed"] == 0, s
    assert srv.close_stream(11) == corr.OK
    srv.close()

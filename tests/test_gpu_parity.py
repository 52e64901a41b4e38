"""GPU parity: the CUDA X stage against the CPU oracle, through the C ABI.

Integer samples: bit-exact int64 equality with the oracle (the definition V_ij =
sum_t x_i conj(x_j), Sec. 2 / Fig. 2).  Float samples: the normwise error against the
float64 oracle, max |V - V64| / sqrt(V64_ii V64_jj), must stay within 1e-6 for the FP32
engine; every BF16x3 element must stay within the per-element bound of the split products
(oracle/precision.py), which a kernel dropping a correction product would exceed.
"""
import numpy as np
import pytest

import oracle
from paper_0906_1887_gb300 import synth
from _gpu_helpers import check_bf16x3, int_case, normwise_error, run_engine

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC, FP32, BF16X3 = 0, 1, 2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_1887_gb300 import corr
    corr.lib()


@pytest.mark.parametrize("engine", [TC, FP32])
def test_mwa32t_4bit_bit_exact(engine):
    re, im, bits, (n, c, t) = synth.workload("mwa32t_4bit")
    p = synth.pack(re, im, bits)
    v = run_engine(p, n, c, t, bits, engine)[0]
    assert np.array_equal(v, oracle.xcorr_int(p, n, c, t, bits))


CASES = [  # (n, c, t, bits): ragged inputs, tails, several tiles, chunk boundaries
    (1, 1, 1, 8), (2, 3, 33, 4), (3, 2, 64, 8), (17, 2, 100, 4), (63, 1, 65, 8), (64, 2, 127, 8),
    (65, 2, 70, 4), (100, 1, 200, 8), (130, 2, 129, 8), (200, 1, 64, 4), (64, 1, 1025, 8),
    (70, 1, 2100, 8), (257, 1, 96, 8),
    # shapes whose packed rows are 16-byte multiples take the fused packed-sample path
    (8, 2, 100, 8), (16, 3, 64, 4), (32, 2, 1000, 8), (96, 2, 130, 8), (96, 1, 77, 4), (128, 2, 256, 4),
    (192, 1, 65, 8), (200, 1, 100, 8), (64, 3, 2049, 8), (48, 2, 300, 4),
    # single-block arrays with enough channels for channel-pair items (>= 2 per SM)
    (64, 320, 100, 8), (32, 331, 64, 4), (16, 400, 130, 8),
]


@pytest.mark.parametrize("engine", [TC, FP32])
@pytest.mark.parametrize("n,c,t,bits", CASES)
def test_small_ragged_bit_exact(engine, n, c, t, bits):
    p = int_case(1000 + n + 7 * c + t, n, c, t, bits)
    v = run_engine(p, n, c, t, bits, engine)[0]
    assert np.array_equal(v, oracle.xcorr_int(p, n, c, t, bits))


# the fused kernel with operand-ring depths away from the default (single-block arrays use 4
# epilogue + 8 converter warps, multi-block arrays 8 + 6): every setting gives the same bits
RING_CASES = [(8, 2, 100, 8), (16, 3, 64, 4), (32, 3, 1000, 8), (64, 5, 1100, 8), (96, 1, 77, 4),
              (128, 2, 256, 4), (136, 3, 130, 8), (192, 1, 65, 8), (48, 2, 300, 4), (64, 1, 1, 8)]


@pytest.mark.parametrize("op_stages", [0, 2, 3, 5])
@pytest.mark.parametrize("n,c,t,bits", RING_CASES)
def test_fused_ring_depths_bit_exact(op_stages, n, c, t, bits):
    p = int_case(5000 + n + 3 * c + t, n, c, t, bits)
    v = run_engine(p, n, c, t, bits, TC, tuning=(op_stages,))[0]
    assert np.array_equal(v, oracle.xcorr_int(p, n, c, t, bits))


# BF16x3 on float samples: split into bf16 hi + lo inside the tensor-core kernel (single-block
# arrays of an even number of inputs) or through hi/lo planes in memory -- the same splits and
# the same products in the same order, so the same bits
@pytest.mark.parametrize("n,c,t", [(2, 1, 1), (8, 3, 100), (34, 4, 130), (64, 5, 1000), (64, 2, 64), (33, 2, 70)])
def test_bf16x3_split_in_kernel_matches_planes(n, c, t):
    re, im = synth.correlated_gaussian(91 + n, t, c, n, 1.0, 0.3, as_float=True)
    x = synth.packf32(re, im)
    fused = run_engine(x, n, c, t, 32, BF16X3, tuning=(0, 0))[0]
    planes = run_engine(x, n, c, t, 32, BF16X3, tuning=(0, 1))[0]
    assert np.array_equal(fused, planes)
    check_bf16x3(fused, x, n, c, t)


# multi-block arrays through both operand feeds and both item shapes of the plane feed: odd and
# even block counts (wide items end a row with a single tile when nb - I is odd), ragged last
# blocks, 4- and 8-bit samples, chunk flushes past 1024 samples, several dumps and accumulate
FEED_CASES = [(128, 2, 100, 8), (192, 3, 130, 8), (256, 2, 64, 4), (320, 1, 1100, 8), (136, 2, 70, 8),
              (200, 2, 129, 8), (448, 1, 65, 4), (512, 1, 2100, 8), (72, 3, 300, 8), (1000, 1, 64, 8)]
FEEDS = [(1, 0), (2, 1), (2, 2)]   # (operands, items): packed; planes + single tiles; planes + wide items


@pytest.mark.parametrize("feed", FEEDS)
@pytest.mark.parametrize("n,c,t,bits", FEED_CASES)
def test_operand_feeds_and_item_shapes_bit_exact(feed, n, c, t, bits):
    p = np.concatenate([int_case(9000 + n + t + k, n, c, t, bits) for k in range(2)])
    ref = np.stack([oracle.xcorr_int(p[k * t:(k + 1) * t], n, c, t, bits) for k in range(2)])
    v = run_engine(p, n, c, t, bits, TC, n_dumps=2, operands=feed)
    assert np.array_equal(v, ref)
    v = run_engine(p, n, c, t, bits, TC, n_dumps=2, accumulate=True, vis_init=ref, operands=feed)
    assert np.array_equal(v, 2 * ref)


# 4-bit samples through e4m3 operands (kind::f8f6f4, 128 samples per stage): ragged tails on
# both sides of a stage, single-block arrays with one channel or channel pairs per item,
# multi-block arrays with ragged last blocks, several dumps and accumulate
F8_CASES = [(16, 3, 64), (32, 2, 1000), (64, 2, 127), (64, 2, 128), (64, 2, 129), (64, 1, 1),
            (64, 320, 100), (32, 331, 300), (96, 1, 77), (128, 2, 256), (192, 1, 65), (48, 2, 300),
            (256, 2, 64), (448, 1, 200), (1008, 1, 130)]


@pytest.mark.parametrize("n,c,t", F8_CASES)
def test_e4m3_operands_4bit_bit_exact(n, c, t):
    p = np.concatenate([int_case(9400 + n + c + t + k, n, c, t, 4) for k in range(2)])
    ref = np.stack([oracle.xcorr_int(p[k * t:(k + 1) * t], n, c, t, 4) for k in range(2)])
    v = run_engine(p, n, c, t, 4, TC, n_dumps=2, operands=(3, 0))
    assert np.array_equal(v, ref)
    v = run_engine(p, n, c, t, 4, TC, n_dumps=2, accumulate=True, vis_init=ref, operands=(3, 0))
    assert np.array_equal(v, 2 * ref)


@pytest.mark.parametrize("t", [128, 131072, 131072 + 128, 131072 + 1])
def test_e4m3_operands_extremes_and_chunk_flush(t):
    # -8 - 8j everywhere but one -8 + 7j input: every product at its largest magnitude, odd
    # imaginary sums, and partial sums at 2^23 per exact chunk of 131072 samples
    n = 32
    re = np.full((t, 1, n), -8, np.int16)
    im = np.full((t, 1, n), -8, np.int16)
    im[:, 0, 3] = 7
    p = synth.pack(re, im, 4)
    v = run_engine(p, n, 1, t, 4, TC, operands=(3, 0))[0]
    assert np.array_equal(v, oracle.xcorr_int(p, n, 1, t, 4))


# 4-bit samples of arrays that take the plane feed: the workspace holds e4m3 planes (rows of
# n_time rounded up to 128 bytes) read by kind::f8f6f4 MMAs, single tiles and wide items, ragged
# last blocks and sample tails, several dumps and accumulate
E4M3_PLANE_CASES = [(256, 2, 64), (272, 3, 129), (448, 1, 200), (320, 2, 255), (512, 2, 1000), (1008, 1, 130)]


@pytest.mark.parametrize("items", [1, 2])
@pytest.mark.parametrize("n,c,t", E4M3_PLANE_CASES)
def test_e4m3_planes_4bit_bit_exact(items, n, c, t):
    p = np.concatenate([int_case(9600 + n + c + t + k, n, c, t, 4) for k in range(2)])
    ref = np.stack([oracle.xcorr_int(p[k * t:(k + 1) * t], n, c, t, 4) for k in range(2)])
    v = run_engine(p, n, c, t, 4, TC, n_dumps=2, operands=(2, items))
    assert np.array_equal(v, ref)
    v = run_engine(p, n, c, t, 4, TC, n_dumps=2, accumulate=True, vis_init=ref, operands=(2, items))
    assert np.array_equal(v, 2 * ref)


def test_e4m3_planes_chunk_flush():
    # -8 - 8j everywhere but one -8 + 7j input, one sample past the exact 131072-sample chunk
    n, t = 128, 131073
    re = np.full((t, 1, n), -8, np.int16)
    im = np.full((t, 1, n), -8, np.int16)
    im[:, 0, 100] = 7
    p = synth.pack(re, im, 4)
    v = run_engine(p, n, 1, t, 4, TC, operands=(2, 2))[0]
    assert np.array_equal(v, oracle.xcorr_int(p, n, 1, t, 4))


@pytest.mark.parametrize("n", [64, 192])
def test_fused_dumps_and_accumulate(n):
    c, t, bits, d = 3, 200, 8, 3
    p = np.concatenate([int_case(77 + k, n, c, t, bits) for k in range(d)])
    ref = np.stack([oracle.xcorr_int(p[k * t:(k + 1) * t], n, c, t, bits) for k in range(d)])
    v = run_engine(p, n, c, t, bits, TC, n_dumps=d)
    assert np.array_equal(v, ref)
    v = run_engine(p, n, c, t, bits, TC, n_dumps=d, accumulate=True, vis_init=ref)
    assert np.array_equal(v, 2 * ref)


@pytest.mark.parametrize("engine", [TC, FP32])
@pytest.mark.parametrize("t", [1023, 1024, 1025, 2048, 3000])
def test_extreme_magnitudes_chunk_flush(engine, t):
    # every sample -128 - 128j except a -128 + 127j input: partial sums reach 2^24 per chunk
    n = 66
    re = np.full((t, 1, n), -128, np.int16)
    im = np.full((t, 1, n), -128, np.int16)
    im[:, 0, 5] = 127
    p = synth.pack(re, im, 8)
    v = run_engine(p, n, 1, t, 8, engine)[0]
    assert np.array_equal(v, oracle.xcorr_int(p, n, 1, t, 8))


@pytest.mark.parametrize("n,t,bits,lo", [(66, 512, 8, -128), (64, 512, 8, -128), (136, 512, 8, -128),
                                         (66, 511, 8, -128), (64, 513, 8, -128),
                                         (16, 131072, 4, -8), (16, 131072 + 64, 4, -8)])
def test_fp32_combined_epilogue_edges(n, t, bits, lo):
    # chunks whose D elements reach 2^23 (rr + ii = 2^24, still exact in fp32): 512 samples
    # of -128 (8-bit) and a full 131072-sample chunk of -8 (4-bit), and one past each edge
    re = np.full((t, 1, n), lo, np.int16)
    im = np.full((t, 1, n), lo, np.int16)
    im[:, 0, 3] = -lo - 1
    re[::3, 0, 7] = -lo - 1
    p = synth.pack(re, im, bits)
    v = run_engine(p, n, 1, t, bits, TC)[0]
    ref = oracle.xcorr_int(p, n, 1, t, bits)
    assert np.array_equal(v, ref)
    assert int(ref[0, 0, 0]) == 2 * t * lo * lo


@pytest.mark.parametrize("n,c,t,bits,lo", [(64, 1, 511, 8, -128), (64, 1, 512, 8, -128), (64, 5, 513, 8, -128),
                                           (128, 3, 1025, 8, -128), (72, 2, 1536, 8, -128),
                                           (32, 1, 32768 + 32, 4, -8), (16, 3, 65536 + 96, 4, -8)])
def test_fp32_segment_edges(n, c, t, bits, lo):
    # the FP32 engine keeps exact fp32 partials over segments of 512 (8-bit) or 32768 (4-bit)
    # samples and adds each segment into the int64 output: full-scale samples put a partial at
    # 2^24 (8-bit) on a segment edge; rows of whole 16-byte pieces (the staged-copy path), channel
    # counts that leave the last group of a block partly empty
    re = np.full((t, c, n), lo, np.int16)
    im = np.full((t, c, n), lo, np.int16)
    im[:, :, 3] = -lo - 1
    re[::3, :, 7] = -lo - 1
    p = synth.pack(re, im, bits)
    v = run_engine(p, n, c, t, bits, FP32)[0]
    ref = oracle.xcorr_int(p, n, c, t, bits)
    assert np.array_equal(v, ref)
    assert int(ref[0, 0, 0]) == 2 * t * lo * lo


@pytest.mark.parametrize("engine", [TC, FP32])
def test_int64_beyond_int32(engine):
    t = 65536 + 64
    re = np.full((t, 1, 2), -128, np.int16)
    im = np.full((t, 1, 2), -128, np.int16)
    p = synth.pack(re, im, 8)
    v = run_engine(p, 2, 1, t, 8, engine)[0]
    ref = oracle.xcorr_int(p, 2, 1, t, 8)
    assert ref[0, 0, 0] > 2 ** 31 and np.array_equal(v, ref)


@pytest.mark.parametrize("engine", [TC, FP32])
def test_batch_of_dumps_and_accumulate(engine):
    n, c, t, d = 72, 3, 150, 3
    packs = [int_case(40 + k, n, c, t, 8) for k in range(d)]
    allp = np.concatenate([x.reshape(-1) for x in packs])
    v = run_engine(allp, n, c, t, 8, engine, n_dumps=d)
    refs = [oracle.xcorr_int(x, n, c, t, 8) for x in packs]
    for k in range(d):
        assert np.array_equal(v[k], refs[k])
    # accumulate=1 adds into the caller's accumulators (cross-dump accumulation in int64)
    init = np.stack(refs).astype(np.int64)
    v2 = run_engine(allp, n, c, t, 8, engine, n_dumps=d, accumulate=True, vis_init=init)
    assert np.array_equal(v2, 2 * init)


@pytest.mark.parametrize("n,c,t,bits", [(128, 2, 200, 8), (64, 3, 1100, 8), (80, 2, 70, 4)])
def test_plane_path_tc_and_fp32(n, c, t, bits):
    # the unpack + cross-multiply split (the path for shapes TMA cannot address directly)
    from paper_0906_1887_gb300 import corr
    p = int_case(300 + n + t, n, c, t, bits)
    ref = oracle.xcorr_int(p, n, c, t, bits)
    plan = corr.Plan(n, c, t, bits)
    x = torch.from_numpy(p.reshape(-1).view(np.uint8)).cuda()
    planes = torch.empty(plan.planes_size(), dtype=torch.uint8, device="cuda")
    plan.unpack(x, planes)
    for engine in (TC, FP32):
        vis = plan.empty_vis(1, "cuda")
        plan.run_planes(planes, vis, engine=engine)
        torch.cuda.synchronize()
        assert plan.check_device() == 0
        assert np.array_equal(vis.cpu().numpy()[0], ref), engine
    plan.close()


# (256, 4): the pipeline's workspace holds e4m3 planes (4 blocks take the plane feed)
@pytest.mark.parametrize("n,bits,chunk", [(64, 8, 2), (40, 8, 3), (128, 4, 0), (256, 4, 3)])
def test_host_pipeline_end_to_end(n, bits, chunk):
    # host buffers in, host buffers out: pipelined copies and X stage over chunks of dumps
    from paper_0906_1887_gb300 import corr
    c, t, d = 6, 300, 7
    packs = [int_case(700 + k + n, n, c, t, bits) for k in range(d)]
    host_in = torch.from_numpy(np.concatenate([x.reshape(-1) for x in packs])).pin_memory()
    P = n * (n + 1) // 2
    host_out = torch.full((d, c, P, 2), -1, dtype=torch.int64).pin_memory()
    plan = corr.Plan(n, c, t, bits)
    plan.run_host(host_in, host_out, n_dumps=d, dumps_per_chunk=chunk)
    assert plan.check_device() == 0
    out = host_out.numpy()
    for k in range(d):
        assert np.array_equal(out[k], oracle.xcorr_int(packs[k], n, c, t, bits)), k
    plan.close()


# (n, bits): rows that are whole 16-byte pieces take the vectorised unpack (64, 80, 96, 136 x 2 B;
# 64, 80, 112 x 1 B, several with a ragged last block), the others the general one
@pytest.mark.parametrize("n,bits,t", [(70, 4, 100), (70, 8, 100), (64, 8, 100), (136, 8, 130), (96, 8, 64),
                                      (64, 4, 65), (80, 4, 200), (112, 4, 33), (8, 8, 64), (16, 4, 1)])
def test_unpack_planes_match_oracle_unpack(n, bits, t):
    from paper_0906_1887_gb300 import corr
    c = 3
    p = int_case(5 + bits + n, n, c, t, bits)
    plan = corr.Plan(n, c, t, bits)
    x = torch.from_numpy(p.reshape(-1).view(np.uint8)).cuda()
    planes = torch.full((plan.planes_size() // 2,), float("nan"), dtype=torch.float16, device="cuda")
    plan.unpack(x, planes)
    torch.cuda.synchronize()
    nb, kp = (n + 63) // 64, (t + 63) // 64 * 64
    got = planes.cpu().float().numpy().reshape(c, nb, 128, kp)
    re, im = oracle.unpack(p, n, c, t, bits)                 # [T][C][N]
    want = np.zeros((c, nb, 128, kp), np.float32)
    for i in range(n):                                       # row 2r: re, row 2r + 1: im
        want[:, i // 64, 2 * (i % 64), :t] = re[:, :, i].T
        want[:, i // 64, 2 * (i % 64) + 1, :t] = im[:, :, i].T
    assert np.array_equal(got, want)                         # padding included: no NaN left
    plan.close()


def test_float_engines_error_vs_float64():
    re, im = synth.correlated_gaussian(2001, 1000, 4, 64, 16.0, 0.1, as_float=True)
    x = synth.packf32(re, im)
    ref = oracle.xcorr_f64(x, 64, 4, 1000)
    v32 = run_engine(x, 64, 4, 1000, 32, FP32)[0]
    vbf = run_engine(x, 64, 4, 1000, 32, BF16X3)[0]
    e32 = normwise_error(v32, ref, 64)
    assert e32 <= 1e-6, e32
    ebf, _ = check_bf16x3(vbf, x, 64, 4, 1000)
    assert ebf <= 1e-4, ebf


@pytest.mark.parametrize("n,c,t", [(1, 1, 1), (65, 2, 130), (130, 1, 70)])
def test_float_engines_ragged(n, c, t):
    re, im = synth.correlated_gaussian(77 + n, t, c, n, 1.0, 0.3, as_float=True)
    x = synth.packf32(re, im)
    ref = oracle.xcorr_f64(x, n, c, t)
    assert normwise_error(run_engine(x, n, c, t, 32, FP32)[0], ref, n) <= 1e-6
    check_bf16x3(run_engine(x, n, c, t, 32, BF16X3)[0], x, n, c, t)


@pytest.mark.parametrize("n,c,t", [(128, 640, 300), (66, 600, 130), (63, 5, 2000)])
def test_float_fp32_engine_ranges_and_accumulate(n, c, t):
    # the FP32 engine on float samples: enough channels for one sample range per item (128 and
    # 66 inputs: multi-block tiles, vector and element-wise staging), or few channels with the
    # sample axis split across blocks (63 inputs, 2000 samples); then accumulating into its output
    from paper_0906_1887_gb300 import corr
    re, im = synth.correlated_gaussian(4100 + n, t, c, n, 4.0, 0.2, as_float=True)
    x = synth.packf32(re, im)
    ref = oracle.xcorr_f64(x, n, c, t)
    plan = corr.Plan(n, c, t, 32)
    xd = torch.from_numpy(x.reshape(-1).view(np.uint8)).cuda()
    vis = plan.empty_vis(1, "cuda")
    plan.run(xd, vis, None, engine=FP32)
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    assert normwise_error(vis.cpu().numpy()[0], ref, n) <= 1e-6
    plan.run(xd, vis, None, accumulate=True, engine=FP32)
    torch.cuda.synchronize()
    assert normwise_error(vis.cpu().numpy()[0], 2 * ref, n) <= 1e-6
    plan.close()


@pytest.mark.parametrize("n", [64, 192])
def test_bounded_wait_gives_up_and_context_survives(n):
    # Failure detection without a GPU fault: the producer withholds one stage, the waiting
    # role's bounded wait (100 ms) runs out, the kernel records a status and returns
    # (single-block and multi-block arrays run different warp splits).
    import time
    from paper_0906_1887_gb300 import corr
    c, t = 16, 256
    p = int_case(31, n, c, t, 8)
    plan = corr.Plan(n, c, t, 8)
    x = torch.from_numpy(p.reshape(-1).view(np.uint8)).cuda()
    vis = plan.empty_vis(1, "cuda")
    t0 = time.time()
    st, code = plan.selftest_stall(x, vis, stall_item=3, wait_limit_ms=100)
    assert st == corr.ETIMEOUT and code == 1
    assert time.time() - t0 < 10
    # the context and the plan are intact: a normal run is bit-exact
    plan.run(x, vis, None, engine=TC)
    torch.cuda.synchronize()
    assert plan.check_device() == 0
    assert np.array_equal(vis.cpu().numpy()[0], oracle.xcorr_int(p, n, c, t, 8))
    plan.close()


def test_invalid_arguments_rejected():
    from paper_0906_1887_gb300 import corr
    with pytest.raises(corr.CorrError):
        corr.Plan(0, 1, 1, 8)
    with pytest.raises(corr.CorrError):
        corr.Plan(4, 1, 1, 6)
    plan = corr.Plan(4, 1, 16, 32)
    x = torch.zeros(4 * 16 * 8, dtype=torch.uint8, device="cuda")
    vis = plan.empty_vis(1, "cuda")
    with pytest.raises(corr.CorrError):            # TC engine takes integer samples only
        plan.run(x, vis, plan.empty_workspace(TC, 1), engine=TC)
    plan.close()
    # packed rows of 130 bytes: only the plane feed can read them, so the workspace is required
    plan = corr.Plan(65, 1, 16, 8)
    x = torch.zeros(65 * 16 * 2, dtype=torch.uint8, device="cuda")
    vis = plan.empty_vis(1, "cuda")
    assert plan.workspace_size(TC) > 0 and plan.workspace_size(FP32) == 0
    with pytest.raises(corr.CorrError):            # missing workspace
        plan.run(x, vis, None, engine=TC)
    with pytest.raises(corr.CorrError) as e:       # the packed feed cannot address these rows
        plan.set_operands(corr.OPERANDS_PACKED, 0)
    assert e.value.status == corr.EUNSUPPORTED
    with pytest.raises(corr.CorrError):
        plan.set_operands(4, 0)
    plan.close()
    plan = corr.Plan(64, 1, 16, 8)                 # e4m3 cannot hold 8-bit samples
    with pytest.raises(corr.CorrError) as e:
        plan.set_operands(corr.OPERANDS_PACKED_F8, 0)
    assert e.value.status == corr.EUNSUPPORTED
    plan.close()

/*
 * corr.h -- C ABI of the GB300 X-stage correlator library (libcorr.so).
 *
 * The X stage of an FX correlator (Wayth, Greenhill & Briggs, Sec. 2): for every
 * frequency channel c and every input pair i <= j (N(N+1)/2 products including the
 * N autos, Sec. 2), multiply the first spectrum by the complex conjugate of the
 * second and add the product into an accumulator over the samples of one dump:
 *
 *     V_ij(c) = sum_t x_i(c,t) * conj(x_j(c,t))
 *
 * The matrix over (i, j) is the outer product of one channel's sample vector with
 * its conjugate (Sec. 4, Fig. 2); its lower half is the conjugate of the upper half,
 * so only i <= j is formed and stored.  The problem is stated by the number of
 * inputs N_I, the number of channels N_C, the samples per batch and the sample mode
 * (Sec. 4 and Sec. 5); corr_plan_create takes exactly these.
 *
 * Conventions shared by every call
 * --------------------------------
 *  Packed input, one dump:   [n_time][n_chan][n_inputs] complex samples, input index
 *                            fastest (Sec. 3: the samples of one time instant are
 *                            grouped together; the F stage has already produced the
 *                            channel axis).
 *      sample_bits = 4 : 1 byte per sample, high nibble = re, low nibble = im, two's
 *                        complement in [-8, 7] (the "1-byte mode" of Sec. 5).
 *      sample_bits = 8 : 2 bytes per sample, re byte then im byte, int8 [-128, 127].
 *      sample_bits = 32: 8 bytes per sample, float32 re then float32 im.
 *  Visibilities, one dump:   [n_chan][P][2], P = N(N+1)/2, baseline
 *                            b(i,j) = i*N - i*(i-1)/2 + (j - i) for i <= j (row-major
 *                            upper triangle), last axis (re, im).  int64 for 4/8-bit
 *                            samples (exact sums), float32 for float samples.
 *  Several dumps:            dumps are consecutive in memory, packed input
 *                            [n_dumps][T][C][N], visibilities [n_dumps][C][P][2].
 *  Pointers:                 d_* arguments are device pointers (or pointers the GPU
 *                            can dereference), 16-byte aligned; the caller owns them
 *                            and the library never frees them.
 *  Streams:                  `stream` is a cudaStream_t passed as void* (NULL = the
 *                            legacy default stream).  Every run call is asynchronous
 *                            on that stream.
 *  Errors:                   every call returns a corr_status and never aborts;
 *                            corr_last_error() gives the calling thread's last message.
 *                            Launch-time CUDA errors return CORR_ECUDA; faults that
 *                            surface later appear at the caller's next synchronise.
 *                            Device-side bounded waits that give up are recorded in
 *                            the plan and reported by corr_plan_check().
 */
#ifndef CORR_H
#define CORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CORR_OK = 0,
    CORR_EINVAL = 1,       /* invalid argument, size or pointer                        */
    CORR_ENOMEM = 2,       /* device or host allocation failed                         */
    CORR_ECUDA = 3,        /* a CUDA runtime/driver call failed                        */
    CORR_EBUSY = 4,        /* not admitted: the job does not fit the HBM budget now    */
    CORR_ETIMEOUT = 5,     /* a bounded device or host wait gave up                    */
    CORR_PENDING = 6,      /* corr_poll: the job has not finished yet                  */
    CORR_EUNSUPPORTED = 7  /* engine/sample-mode combination not provided              */
} corr_status;

typedef enum {
    /* Tensor-core X stage (tcgen05 MMA, accumulators in tensor memory).  Integer
     * samples run exactly: 4/8-bit values are exact in fp16 and the fp32 partial
     * sums stay below 2^24 within each flushed time chunk, so the int64 result is
     * bit-identical to the definition.  Not valid for float samples. */
    CORR_ENGINE_TC = 0,
    /* CUDA-core FP32 X stage (the plain form), on the packed samples directly (no
     * workspace).  Exact for integer samples (time chunks flushed to int64); fp32
     * arithmetic with two-level summation for float samples. */
    CORR_ENGINE_FP32 = 1,
    /* Float samples on the tensor cores: x = h + l with h = bf16(x),
     * l = bf16(x - h); V ~= h h^H + h l^H + l h^H with fp32 accumulation.  For arrays of
     * at most 64 inputs (an even count) the split happens inside the tensor-core kernel
     * and needs no workspace; otherwise hi/lo planes go through the workspace.  Both give
     * the same bits. */
    CORR_ENGINE_BF16X3 = 2
} corr_engine;

typedef struct corr_plan_s *corr_plan;   /* opaque, owned by the library */

/* Library version as MAJOR*10000 + MINOR*100 + PATCH; CORR_VERSION is the value of the
 * header a caller was built with.  0.2.0: corr_server_stats gained `coalesced` and the operand
 * feeds CORR_OPERANDS_PACKED_F8. */
#define CORR_VERSION 200
int corr_version(void);

/* Last error message of the calling thread ("" if none).  Valid until the next call
 * on this thread. */
const char *corr_last_error(void);

/*
 * Create a plan for n_inputs inputs (N_I, >= 1), n_chan channels (N_C, >= 1),
 * n_time samples per dump (>= 1) and a sample mode (4, 8 or 32).  The paper's
 * prototype is n_inputs = 64 (32 antennas x 2 polarisations), n_chan = 128
 * (Sec. 4, Sec. 5).  Allocates a small device status block on the current device.
 * Errors: CORR_EINVAL on bad sizes/modes or an out-of-range problem (N <= 8192,
 * products that would overflow 64-bit indexing); CORR_ENOMEM, CORR_ECUDA.
 */
corr_status corr_plan_create(corr_plan *out, int n_inputs, int n_chan, int n_time, int sample_bits);

/* Destroy a plan (waits for nothing; the caller must have synchronised its work). */
corr_status corr_plan_destroy(corr_plan plan);

/* Sizes of one dump: number of baselines P, bytes of the packed input and of the
 * visibilities.  Any output pointer may be NULL. */
corr_status corr_plan_info(corr_plan plan, int64_t *n_baselines, size_t *packed_bytes, size_t *vis_bytes);

/*
 * Launch knobs of the tensor-core kernel for this plan (no counterpart in the paper: they
 * shape the pipeline, not what it computes).  op_stages = depth of the operand ring in shared
 * memory, 0 = the default; for the packed feed a depth that leaves fewer than 3 stages for the
 * sample ring is reduced to what fits; the plane feed uses the requested depth when it is
 * smaller than what fits (by default as deep as fits).  float_planes (CORR_ENGINE_BF16X3 on float samples): 0 = the
 * default, the tensor-core kernel loads the floats and splits them into bf16 hi + lo itself
 * where it can (arrays of at most 64 inputs, an even count), needing no workspace; 1 = always
 * split into hi/lo planes in the workspace first.  Results are identical for every setting.
 * CORR_EINVAL when op_stages is outside [0, 16] or float_planes outside [0, 1].
 */
corr_status corr_plan_set_tuning(corr_plan plan, int op_stages, int float_planes);

/*
 * Operand feed of the tensor-core X stage for 4/8-bit samples (no counterpart in the paper; the
 * results are identical for every setting).  The kernel either converts the packed samples
 * itself (converter warps; the samples cross HBM once, but each 64-input block is converted once
 * per tile it meets, about N/128 times per channel) or reads sample planes that the unpack
 * kernel wrote into the workspace first (each block converted once; the planes cost HBM
 * traffic; fp16 planes, or e4m3 ones for 4-bit samples of rows that are 16-byte multiples --
 * the workspace's own format, not the fp16 exchange format of corr_unpack).  operands:
 *   CORR_OPERANDS_AUTO    planes for arrays of at least 256 inputs (4 blocks; 192 inputs, 3
 *                         blocks, for 4-bit samples, whose planes are e4m3) when a workspace
 *                         is given, and always where the packed rows are not 16-byte multiples;
 *                         otherwise the fused conversion, into e4m3 operands for 4-bit samples;
 *   CORR_OPERANDS_PACKED  always the fused conversion into fp16 operands (CORR_EUNSUPPORTED
 *                         where rows are not 16-byte multiples);
 *   CORR_OPERANDS_PLANES  always planes (the workspace is then required);
 *   CORR_OPERANDS_PACKED_F8  4-bit samples only: the fused conversion into fp8 e4m3 operands
 *                         (tcgen05 kind::f8f6f4, 128 samples per 128-byte operand row), which hold
 *                         -8..7 exactly and halve the operand bytes per sample; fp32 accumulation
 *                         as for fp16, so results stay bit-exact (CORR_EUNSUPPORTED for 8-bit
 *                         samples, whose range e4m3 does not hold, or rows that are not 16-byte
 *                         multiples).
 * items (plane feed): CORR_ITEMS_WIDE = work items of block I against blocks J and J + 1 in one
 * M = 128, N = 256 MMA (a quarter fewer operand loads per tile); CORR_ITEMS_TILES = one 64 x 64
 * input tile per item; CORR_ITEMS_AUTO = wide, except single tiles for accumulating dumps of
 * fewer than 1024 samples (bound by their read-modify-write of the output).  CORR_EINVAL on
 * unknown values.
 */
enum { CORR_OPERANDS_AUTO = 0, CORR_OPERANDS_PACKED = 1, CORR_OPERANDS_PLANES = 2, CORR_OPERANDS_PACKED_F8 = 3 };
enum { CORR_ITEMS_AUTO = 0, CORR_ITEMS_TILES = 1, CORR_ITEMS_WIDE = 2 };
corr_status corr_plan_set_operands(corr_plan plan, int operands, int items);

/* Device workspace (bytes) corr_xengine_run_batch uses for `engine` and n_dumps dumps.  0 means
 * the engine needs none (d_workspace may be NULL).  For CORR_ENGINE_TC on arrays whose packed
 * rows are 16-byte multiples the workspace is optional unless CORR_OPERANDS_PLANES is set: a
 * NULL workspace runs the fused conversion, a workspace of this size the plane feed. */
corr_status corr_workspace_size(corr_plan plan, int engine, int n_dumps, size_t *bytes);

/*
 * Unpack/transpose step on its own (Sec. 4: reorder the time-ordered block so each
 * input's samples become contiguous, converting to a floating-point format).
 * Writes d_planes, laid out [n_dumps][n_chan][NB][128][Kp] with NB = ceil(N/64) input
 * blocks of 64 and Kp = n_time rounded up to a multiple of 64: row 2r holds the real
 * parts of input 64*nb + r and row 2r + 1 its imaginary parts, one element per time
 * sample, zero for padded inputs and samples.  Element type: fp16 for 4/8-bit
 * samples (exact), fp32 for float samples.  Size: corr_planes_size.
 */
corr_status corr_unpack(corr_plan plan, const void *d_packed, int n_dumps, void *d_planes, void *stream);
/* Bytes of the sample planes of n_dumps dumps (corr_unpack's output). */
corr_status corr_planes_size(corr_plan plan, int n_dumps, size_t *bytes);

/*
 * The X stage of one dump: V = sum over the dump's n_time samples, in baseline order.
 *   d_packed    packed input of one dump (layout above)
 *   d_vis       [n_chan][P][2] output; int64 for 4/8-bit samples, float32 for float
 *   d_workspace corr_workspace_size(engine, 1) bytes, or NULL when that is 0
 *   accumulate  0: overwrite d_vis;  1: add into d_vis (cross-dump accumulation in
 *               int64, Fig. 1: accumulators are read out and reset by the caller)
 *   engine      a corr_engine value
 */
corr_status corr_xengine_run(corr_plan plan, const void *d_packed, void *d_vis, void *d_workspace,
                             int accumulate, int engine, void *stream);

/* n_dumps consecutive dumps in one call (one launch per kernel for all dumps). */
corr_status corr_xengine_run_batch(corr_plan plan, const void *d_packed, int n_dumps, void *d_vis,
                                   void *d_workspace, int accumulate, int engine, void *stream);

/*
 * The cross-multiply-accumulate step alone, on sample planes that corr_unpack already
 * wrote (Sec. 4, step 3): d_planes as corr_unpack describes, n_dumps dumps; d_vis,
 * accumulate and engine as for corr_xengine_run.  CORR_ENGINE_TC and CORR_ENGINE_FP32
 * only (BF16X3 needs its own split planes and runs through corr_xengine_run).
 */
corr_status corr_xengine_run_planes(corr_plan plan, const void *d_planes, int n_dumps, void *d_vis,
                                    int accumulate, int engine, void *stream);

/*
 * The tensor-core X stage of one dump of 4/8-bit samples without allocating device
 * memory.  The paper has no counterpart: this call exists for callers that cannot call
 * cudaMalloc -- a real-time loop that must never pay the device-wide synchronisation of
 * cudaMalloc/cudaFree, or a host framework that owns all device memory and forbids its
 * plug-ins from allocating.  No plan is needed (a plan allocates a status block); the
 * problem is given directly.  d_packed, d_vis, accumulate and stream are as for
 * corr_xengine_run (engine: CORR_ENGINE_TC).
 *
 * Scratch: the unpacked sample planes (corr_unpack's layout, n_chan * ceil(N/64) * 128 *
 * Kp * 2 bytes) live in a fixed 64 MiB array inside the library; every GPU that loads the
 * library holds it until the process exits.  Larger dumps return CORR_EINVAL with a
 * message naming the array's size in bytes (the check is made before any size product can
 * overflow).  The first call on each device, and the first after that device's CUDA context
 * changes (cudaDeviceReset), looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture.  The call itself
 * calls no cudaMalloc, cudaFree or allocating library routine.  All calls share the array and
 * its contents persist between calls: calls whose GPU work overlaps (other streams or host
 * threads on the same device) race and must be serialised by the caller.  A bounded wait
 * inside the kernels that gives up leaves the output incomplete; it is recorded in a status
 * block beside the array, which each call zeroes on its stream and corr_static_check reads.
 */
corr_status corr_xengine_run_static(const void *d_packed, int n_inputs, int n_chan, int n_time,
                                    int sample_bits, void *d_vis, int accumulate, void *stream);

/*
 * Status of the last corr_xengine_run_static call on the current device, read and cleared
 * (no counterpart in the paper; allocates nothing).  Synchronises `stream` (pass the stream
 * of that call), copies the status block to the host, zeroes it, and sets *device_error to 0
 * or to the code a kernel recorded when one of its bounded waits gave up (then returns
 * CORR_ETIMEOUT).  CORR_EINVAL if device_error is NULL; CORR_ECUDA on a failed copy.
 */
corr_status corr_static_check(int *device_error, void *stream);

/*
 * The X stage of n_dumps dumps held in HOST memory, end to end: the prototype streams
 * samples to the GPU in large batches and overlaps staging with the CMAC (Sec. 5).  The
 * call splits the dumps into chunks of dumps_per_chunk (<= 0: about 256 MB of samples
 * per chunk) and pipelines, on three internal streams, the host-to-device copy of chunk
 * k+1, the X stage of chunk k and the device-to-host copy of chunk k-1, with double
 * buffers in device memory that the plan allocates on first use (and keeps, growing it
 * when a larger chunk needs it; freed by corr_plan_destroy).  host_packed: n_dumps x
 * [T][C][N] packed samples; host_vis: n_dumps x [C][P][2].  Page-locked host memory
 * (corr_host_alloc) lets the copies overlap.  Returns when host_vis holds every result.
 */
corr_status corr_xengine_run_host(corr_plan plan, const void *host_packed, int n_dumps, void *host_vis,
                                  int dumps_per_chunk, int engine);

/*
 * F stage (Sec. 2, Sec. 4): the step in front of the X stage.  Each input's time samples are
 * cut into frames and every frame is Fourier transformed into spectral channels:
 *   complex samples: N_C samples -> N_C-point complex DFT -> N_C channels;
 *   real samples:    2 N_C samples -> 2 N_C-point complex-to-complex DFT, channels 0 .. N_C
 *                    (DC to Nyquist, N_C + 1 channels) kept, the mirrored half dropped
 *                    (the paper transforms real input this way to keep power-of-two sizes).
 * The DFT is the forward, unnormalised X_k = sum_s x_s exp(-2 pi i k s / L); channel c is
 * bin c.  Computed in float32 on the GPU (Stockham stages of radix 16, the last of radix 8, 4
 * or 2; twiddles rounded from double); the relative L2 error of a frame's spectrum against an exact transform is a few
 * times 2^-24 log2 L.
 *
 *   kind               packed time samples, [time][n_inputs], input index fastest (Sec. 3)
 *   CORR_F_COMPLEX8    2 bytes: re byte, im byte, int8
 *   CORR_F_COMPLEX4    1 byte: high nibble re, low nibble im, two's complement
 *   CORR_F_REAL8       1 byte: int8 real sample
 *
 * corr_fplan_create: n_inputs in [1, 8192]; the transform length (n_chan, or 2 n_chan for
 * real samples) a power of two in [8, 4096].  Allocates a small twiddle table on the current
 * device; the plan owns it.
 * corr_fplan_info: channels produced per frame, transform length, and the bytes of one frame
 * of input (L x n_inputs x bytes per sample) and of output (n_out_chan x n_inputs x 8).
 * corr_fengine_run: n_frames consecutive frames; d_time holds n_frames x L time samples
 * (2-byte aligned), d_spectra receives [n_frames][n_out_chan][n_inputs] complex float32
 * (re, im; 8-byte aligned) -- the float sample layout of the X stage, so a plan with
 * n_time = n_frames, n_chan = n_out_chan, sample_bits = 32 correlates it.  Asynchronous on
 * `stream`; both buffers are the caller's.
 */
#define CORR_F_COMPLEX8 0
#define CORR_F_COMPLEX4 1
#define CORR_F_REAL8 2
typedef struct corr_fplan_s *corr_fplan;
corr_status corr_fplan_create(corr_fplan *out, int n_inputs, int n_chan, int kind);
corr_status corr_fplan_destroy(corr_fplan plan);
corr_status corr_fplan_info(corr_fplan plan, int *n_out_chan, int *transform_len, size_t *in_bytes_per_frame,
                            size_t *out_bytes_per_frame);
corr_status corr_fengine_run(corr_fplan plan, const void *d_time, int n_frames, void *d_spectra, void *stream);

/*
 * Polyphase filterbank in place of the plain transform (Sec. 6.1: less spectral leakage, the
 * extra cost in the unpack): output frame f weights the n_taps input frames f .. f+M-1 by a
 * prototype filter h of M L taps and transforms the sum,
 *     y_f[s] = sum_m h[m L + s] x[(f + m) L + s],   X_f[k] = sum_s y_f[s] exp(-2 pi i k s / L).
 * h_taps: host array of n_taps x L floats (L = the transform length), copied into the plan; or
 * NULL for the default prototype, the windowed sinc sinc((n - (M L - 1) / 2) / L) times the
 * Hamming window 0.54 - 0.46 cos(2 pi n / (M L - 1)) (computed in double, rounded to float;
 * n_taps = 1 with NULL is the plain transform).  n_taps in [1, 64], and the prototype (n_taps
 * x L floats) must fit in shared memory beside the transform buffers (n_taps x L <= about
 * 28000; CORR_EINVAL otherwise).  For such a plan
 * corr_fengine_run's d_time must hold n_frames + n_taps - 1 frames of L samples; n_frames
 * spectra are produced.  Destroy with corr_fplan_destroy.
 */
corr_status corr_fplan_create_pfb(corr_fplan *out, int n_inputs, int n_chan, int kind, int n_taps, const float *h_taps);
/* Taps of an F-stage plan (1 for a plain-transform plan). */
corr_status corr_fplan_taps(corr_fplan plan, int *n_taps);

/*
 * Dump step (Fig. 1) with post-correlation phase correction (Sec. 2) for one dump of `plan`:
 * the accumulators are read, divided by the number of updates, rotated to remove the phase
 * that per-input delays add, and optionally reset:
 *     V'_ij(c) = V_ij(c) / n_accum * exp(+2 pi i nu_c (tau_i - tau_j))
 * (a delay tau_i multiplies input i's spectrum by exp(-2 pi i nu tau_i); the paper applies the
 * MWA's geometric delay correction this way, after correlation).
 *   d_acc       accumulators [n_chan][P][2] of this plan (device): int64 for 4/8-bit plans,
 *               float32 for float plans; 16-byte aligned
 *   n_accum     update count >= 1 (the output is divided by it)
 *   d_delays    double [n_inputs], seconds (device), or NULL: no rotation, averaging only
 *   d_freqs     double [n_chan], channel sky frequencies in Hz (device); needed with d_delays
 *   d_workspace corr_dump_workspace_size bytes (device; per-input phasors), needed with d_delays
 *   d_out       float32 [n_chan][P][2] averaged, corrected visibilities (device, 8-byte aligned)
 *   reset       1: zero d_acc in the same pass, ready for the next interval
 * Phasors are formed in double precision and rounded to float; the rotation and the division
 * are float32 (relative error a few times 2^-24).  Asynchronous on `stream`.
 */
corr_status corr_dump_workspace_size(corr_plan plan, size_t *bytes);

/*
 * The X stage and the dump step of one or more dumps in one pass (the dump step fused into
 * the tensor-core kernel's epilogue): d_out[d] = V_d / n_accum rotated as corr_dump does,
 * float32 [n_dumps][n_chan][P][2], never the int64 sums.  Arguments as corr_xengine_run_batch
 * and corr_dump (phasor workspace of corr_dump_workspace_size bytes when delays are given).
 * CORR_EUNSUPPORTED unless the plan takes the packed-sample tensor-core path (4/8-bit samples,
 * packed rows a multiple of 16 bytes) and a dump fits one exact chunk (n_time <= 1024 for
 * 8-bit, <= 131072 for 4-bit).  Asynchronous on `stream`.
 */
corr_status corr_xengine_run_dump(corr_plan plan, const void *d_packed, int n_dumps, void *d_out, int n_accum,
                                  const double *d_delays, const double *d_freqs, void *d_workspace, void *stream);
corr_status corr_dump(corr_plan plan, void *d_acc, int n_accum, const double *d_delays, const double *d_freqs,
                      void *d_workspace, void *d_out, int reset, void *stream);

/*
 * Read and clear the plan's device status block (synchronises with the device).
 * *device_error receives 0, or the code a kernel recorded when one of its bounded
 * waits gave up.  Returns CORR_ETIMEOUT in that case, else CORR_OK / CORR_ECUDA.
 */
corr_status corr_plan_check(corr_plan plan, int *device_error);

/*
 * ---- Batched uneven jobs in one persistent launch --------------------------------
 *
 * Large batches per GPU call make launch overhead negligible (Sec. 4, Sec. 5).  A batch
 * packs many correlation jobs -- arrays of different sizes, channel counts and dump
 * lengths -- into one flat list of work items walked by one grid of persistent
 * tensor-core CTAs (one launch per sample mode present, 64 jobs per launch at most).
 * Every job here is one dump of 4/8-bit samples whose packed rows are TMA-addressable:
 * n_inputs * bytes-per-sample must be a multiple of 16 (CORR_EUNSUPPORTED otherwise).
 */
typedef struct {
    int n_inputs, n_chan, n_time, sample_bits;
    const void *packed;   /* device: [n_time][n_chan][n_inputs] packed samples, 16-byte aligned */
    void *vis;            /* device: [n_chan][P][2] int64, 16-byte aligned */
} corr_job;

typedef struct corr_batch_s *corr_batch;   /* opaque, owned by the library */

enum {
    CORR_BATCH_GRAPH = 1,       /* capture the launch(es) into a CUDA graph; corr_batch_run replays it */
    CORR_BATCH_AUTOTUNE = 2,    /* time candidate launch shapes on the batch's buffers, keep the fastest */
    CORR_BATCH_ACCUMULATE = 4,  /* add into the jobs' visibilities instead of overwriting them */
    CORR_BATCH_PLANES = 8       /* allow the plane operand path: the batch allocates fp16 sample planes
                                   for its jobs of more than 64 inputs (n_chan x ceil(N/64) x 128 x
                                   Kp x 2 bytes each); jobs of at least plane_min_nb 64-input blocks
                                   are unpacked into them and the tensor-core kernel reads the planes
                                   instead of converting packed samples itself (tuned, or 4 blocks
                                   when not tuned; packed 4-bit samples are converted to e4m3
                                   operands, 8-bit ones to fp16).  Results are identical either way. */
};

typedef struct {
    int n_jobs, n_launches, graph, tuned;
    int64_t n_items;            /* work items of all launches */
    double cmacs;               /* algorithmic CMACs of one run: sum of P * n_chan * n_time */
    int op_stages, pair_cpi, order;   /* the launch shape in use (0: default) */
    float tune_ms;              /* the tuner's best time, ms (0 if not tuned) */
    int plane_min_nb;           /* jobs of at least this many blocks read planes (0: none) */
    size_t plane_bytes;         /* the batch's plane workspace */
    int wide;                   /* plane jobs run wide work items (see CORR_ITEMS_WIDE) */
    int plane_splits;           /* plane jobs in this many launches, each run's unpack overlapping the
                                   previous run's tensor-core launch (1: unpacks, then one launch) */
} corr_batch_stats;

/*
 * Build a batch over jobs[0..n_jobs) (the library copies the descriptors; the caller
 * keeps the buffers alive).  flags: CORR_BATCH_* bits.  With CORR_BATCH_AUTOTUNE the
 * library runs the batch several times on its own buffers (overwriting the
 * visibilities) and keeps the fastest launch shape for this set of job sizes (operand-ring
 * depth, channels per item of single-block arrays, item order and, with CORR_BATCH_PLANES,
 * the operand path per array size); with a non-NULL tune_cache path the choice is read from
 * / appended to that JSON-lines file, keyed by the job sizes and the library build.
 * AUTOTUNE with ACCUMULATE is rejected (tuning runs would add into the accumulators).
 * With CORR_BATCH_GRAPH the launches are captured into a CUDA graph once.  Allocates a
 * small device status block and a stream (with CORR_BATCH_PLANES two more, a high-priority one
 * for the tensor-core launches and a low-priority one for the unpacks, and a few events).
 */
corr_status corr_batch_create(corr_batch *out, const corr_job *jobs, int n_jobs, int flags,
                              const char *tune_cache);
/* Set the launch shape directly instead of tuning it: op_stages (0 = default, up to 16),
 * pair_cpi (channels per work item of single-block arrays, 1 or 2), order (0: costliest jobs'
 * items first, 1: the caller's order), plane_min_nb (jobs of at least this many 64-input blocks
 * read fp16 planes; 0 = none; > 0 needs CORR_BATCH_PLANES), wide (plane jobs: 1 = wide work
 * items, 0 = single tiles), plane_splits (1..8: the plane jobs in this many launches of about
 * equal products; the unpacks run back to back on the low-priority stream and each launch waits
 * for its own jobs' unpacks, so unpacking overlaps the tensor cores' work; each such launch
 * leaves 10 KB of shared memory per SM for an unpack block).  A captured graph is re-captured.
 * Results are identical for every shape.  Not concurrent with corr_batch_run. */
corr_status corr_batch_set_shape(corr_batch b, int op_stages, int pair_cpi, int order, int plane_min_nb, int wide,
                                 int plane_splits);
/* Run the batch on `stream` (graph replay when captured).  Asynchronous. */
corr_status corr_batch_run(corr_batch b, void *stream);
corr_status corr_batch_info(corr_batch b, corr_batch_stats *stats);
/* Synchronise and read/clear the batch's device status block (see corr_plan_check). */
corr_status corr_batch_check(corr_batch b, int *device_error);
corr_status corr_batch_destroy(corr_batch b);

/*
 * ---- Real-time serving loop ------------------------------------------------------
 *
 * The prototype stages the next batch in host memory while the GPU correlates the
 * previous one (Sec. 5, Table 3 notes).  A server takes correlation jobs from any number
 * of host threads (the mailbox), admits them in arrival order by device footprint into
 * an HBM arena allocated once (packed samples + visibilities + any workspace), and runs
 * each on one of n_streams CUDA streams: host-to-device copy, X stage and, when host_vis is
 * given, device-to-host copy of the visibilities -- so the copies of some jobs overlap the
 * kernels of others.  Jobs are issued earliest deadline first (submission time + the job's own
 * sample time at a 10 kHz channel rate; an open stream's jobs keep their order), each when its
 * samples fit a 256 MB budget of host-to-device bytes in flight.  The kernels write each job's
 * status words straight into mapped pinned memory (no copy per job); events and status words
 * are pooled, so submitting and releasing a job neither allocates nor frees.  A job that can never fit the budget is rejected at
 * submission (CORR_EBUSY); one that fits waits until enough space is free.
 * Engines: the tensor-core X stage for 4/8-bit samples, BF16x3 for float samples.
 */
typedef struct corr_server_s *corr_server;   /* opaque, owned by the library */

typedef struct {
    int n_inputs, n_chan, n_time, sample_bits;
    const void *host_packed;  /* host: [n_time][n_chan][n_inputs] packed samples (pinned memory
                                 from corr_host_alloc makes the copy asynchronous) */
    void *host_vis;           /* host: [n_chan][P][2] output, or NULL to keep the result in the
                                 arena (corr_job_result.d_vis) until corr_release */
    int stream_tag;           /* caller's label of the input stream the job came from */
} corr_job_desc;

typedef struct {
    int status;               /* CORR_PENDING, CORR_OK, CORR_ETIMEOUT (a device wait gave up),
                                 CORR_ECUDA, or CORR_EBUSY (cancelled at shutdown) */
    double t_submit, t_start, t_done;   /* host monotonic seconds */
    float gpu_ms;             /* stream time from the job's first copy to its last */
    void *d_vis;              /* device result while the job keeps it (host_vis == NULL), or the
                                 open stream's averaged dump this job produced (see below) */
    int closed_interval;      /* open streams: 1 if this job ended a dump interval */
    int64_t n_accum;          /* open streams, closing jobs: samples summed in the dump */
} corr_job_result;

typedef struct {
    int64_t submitted, completed, failed, rejected, cancelled, queued, running;
    size_t arena_bytes, bytes_in_use, peak_bytes;
    int64_t open_streams;     /* streams with device state (corr_server_open_stream) */
    int64_t coalesced;        /* stream jobs issued in pairs (one X stage over two jobs' samples) */
} corr_server_stats;

enum { CORR_SERVER_START_PAUSED = 1 };   /* admit nothing until corr_server_resume */

/* Allocates the arena (hbm_budget_bytes of device memory), n_streams streams and two host
 * threads (dispatcher, completion). */
corr_status corr_server_create(corr_server *out, size_t hbm_budget_bytes, int n_streams, int flags);
/* Queue a job (thread-safe, non-blocking).  The host buffers must stay valid until the
 * job finishes.  CORR_EBUSY if the job can never fit the budget, CORR_EINVAL on bad sizes. */
corr_status corr_submit(corr_server s, const corr_job_desc *job, uint64_t *job_id);
/* Non-blocking: returns CORR_PENDING while the job is queued or running, else its final
 * status; *res gets the timestamps. */
corr_status corr_poll(corr_server s, uint64_t job_id, corr_job_result *res);
/* Bounded wait for a job: CORR_ETIMEOUT if not finished within timeout_s seconds. */
corr_status corr_wait(corr_server s, uint64_t job_id, double timeout_s, corr_job_result *res);
/* Copy a finished job's device-resident visibilities (host_vis was NULL) to host memory
 * (synchronous).  Do not call concurrently with corr_release of the same job. */
corr_status corr_fetch(corr_server s, uint64_t job_id, void *host_vis);
/* Forget a finished job; frees its device result if it kept one. */
corr_status corr_release(corr_server s, uint64_t job_id);
corr_status corr_server_resume(corr_server s);
corr_status corr_server_get_stats(corr_server s, corr_server_stats *st);
/* Cancel queued jobs, wait up to drain_timeout_s for running ones (CORR_ETIMEOUT if some
 * are still running; the streams are then synchronised before memory is freed). */
corr_status corr_server_destroy(corr_server s, double drain_timeout_s);
/*
 * ---- Per-stream device state: sample rings and accumulators kept on the device ----
 *
 * The correlator integrates: every batch of samples is added into accumulators, which are
 * read out at the end of a dump interval, divided by the number of times they were updated
 * and reset (Fig. 1).  corr_server_open_stream gives one input stream (a stream_tag) that state
 * on the device, admitted once against the HBM budget instead of per job:
 *   - a ring of ring_slots sample slots: job k of the stream is copied into slot k mod
 *     ring_slots as soon as the X stage of job k - ring_slots has read that slot, so copies of
 *     later jobs run ahead of the X stage of earlier ones;
 *   - accumulators [n_chan][P][2] (int64 for 4/8-bit samples, float32 for float samples) that
 *     every job of the stream adds into, in submission order (one CUDA stream per open stream);
 *     when a 4/8-bit stream's next job is already queued, in the adjacent slot and within the
 *     same interval, the two are issued together: one X stage over the 2 x n_time samples of
 *     both slots (one accumulator pass instead of two; each job still completes on its own);
 *   - at every jobs_per_dump-th job the interval ends:
 *       CORR_STREAM_DUMP_SUMS      the accumulated sums are copied to that job's host_vis (the
 *                                  exact integer sums for 4/8-bit samples; host_vis must not be
 *                                  NULL for such a job, CORR_EINVAL at submission otherwise) and
 *                                  the next interval's first job overwrites them;
 *       CORR_STREAM_DUMP_AVERAGED  the dump step (corr_dump) divides by the samples summed
 *                                  (jobs_per_dump x n_time), applies the phase correction when
 *                                  d_delays is given and writes float32 [n_chan][P][2] into a
 *                                  device dump buffer (the next interval's first job overwrites
 *                                  the accumulators, which resets them);
 *                                  copied to the closing job's host_vis when it is not NULL (on
 *                                  a third CUDA stream of the open stream, so its next jobs do
 *                                  not wait for the copy; the closing job completes when the
 *                                  dump is in host memory), else left there
 *                                  (corr_job_result.d_vis) until the stream's next dump
 *                                  overwrites it.
 * The stream's CUDA streams get a priority from its dump length (shorter dumps, tighter
 * deadlines: higher priority), which orders kernels of different streams when the GPU is busy.
 * Jobs submitted with that stream_tag must have the stream's shape (CORR_EINVAL otherwise); they
 * need no arena space of their own and are issued as soon as they reach the mailbox, never held
 * behind a job waiting for memory.  Results of such jobs other than the closing one carry no
 * visibilities (host_vis is ignored).  CORR_EBUSY if the stream's state does not fit the arena's
 * free space now; CORR_EINVAL if the tag is already open or the description is invalid.  d_delays
 * (float64 [n_inputs], seconds) and d_freqs (float64 [n_chan], Hz) are device arrays the caller
 * keeps alive while the stream is open (averaged mode only; NULL: averaging only).
 */
enum { CORR_STREAM_DUMP_SUMS = 0, CORR_STREAM_DUMP_AVERAGED = 1 };

typedef struct {
    int n_inputs, n_chan, n_time, sample_bits;   /* every job of the stream has this shape */
    int ring_slots;           /* device sample slots, >= 1 */
    int jobs_per_dump;        /* jobs accumulated into one dump interval, >= 1 */
    int dump_mode;            /* CORR_STREAM_DUMP_SUMS or CORR_STREAM_DUMP_AVERAGED */
    const double *d_delays;   /* averaged mode: per-input delays (device) or NULL */
    const double *d_freqs;    /* averaged mode: channel frequencies (device), with d_delays */
} corr_stream_desc;

corr_status corr_server_open_stream(corr_server s, int stream_tag, const corr_stream_desc *desc);
/* Stop taking jobs for the tag, wait up to drain_timeout_s for its jobs to finish (CORR_ETIMEOUT
 * if some are still running; they are then waited for on the GPU before the state is freed), and
 * return the stream's device state to the arena.  An interval left open is discarded. */
corr_status corr_server_close_stream(corr_server s, int stream_tag, double drain_timeout_s);

/* Page-locked host memory for job buffers (cudaMallocHost). */
corr_status corr_host_alloc(void **ptr, size_t bytes);
corr_status corr_host_free(void *ptr);

/*
 * Self-test of failure detection, with no GPU fault: runs the packed-sample tensor-core X
 * stage of one dump with its mbarrier waits bounded by wait_limit_ms, while the producer
 * withholds the first stage of work item `stall_item`, so the waiting role gives up,
 * records its code in the plan's status block and every role of that CTA exits cleanly
 * (in-flight copies and MMAs are drained first).  Synchronises; *device_error receives
 * the recorded code (0 if nothing timed out; 1 = a loaded stage never arrived) and the
 * call returns CORR_ETIMEOUT when one was recorded.  The plan stays usable afterwards.
 */
corr_status corr_selftest_stall(corr_plan plan, const void *d_packed, void *d_vis, int stall_item,
                                int wait_limit_ms, int *device_error);

/*
 * Divide int64 visibilities by the number of accumulated dumps, on the host, in
 * float64 (Fig. 1: accumulators are divided by the number of times they were
 * updated).  n_values = 2 * P * n_chan * n_dumps.  No GPU work.
 */
corr_status corr_average_host(const int64_t *vis, size_t n_values, int64_t n_accum, double *out);

#ifdef __cplusplus
}
#endif

#endif /* CORR_H */

// Tensor-core X stage on sm_103a: tcgen05 MMA with accumulators in tensor memory.
//
// For one channel the correlation matrix is the outer product of the sample vector with
// its conjugate, summed over time (Sec. 4, Fig. 2) -- a Hermitian rank-k update, i.e. a
// dense contraction over the time axis.  A 64-input block is held as 128 operand rows,
// interleaved: row 2m carries the real parts and row 2m+1 the imaginary parts of input m,
// one column per time sample.  With A = block I and B = block J in that form, one MMA per
// 16 samples accumulates D = A B^T (M = N = 128), whose 2 x 2 sub-blocks are
//     D[2i][2j] = sum xr_i xr_j    D[2i][2j+1] = sum xr_i xi_j
//     D[2i+1][2j] = sum xi_i xr_j  D[2i+1][2j+1] = sum xi_i xi_j
// so that Re V_ij = D[2i][2j] + D[2i+1][2j+1] and Im V_ij = D[2i+1][2j] - D[2i][2j+1]:
// x_i conj(x_j) summed over time (Sec. 2).  Rows 2i and 2i+1 sit in adjacent tensor-memory
// lanes, so the epilogue combines them with one lane-pair shuffle.  Only blocks with
// I <= J (the upper triangle of input pairs) are scheduled.
//
// Exactness for integer samples: 4/8-bit values are exact in fp16, their products
// (|p| <= 2^14) are exact, and each D element sums one product per sample, so a chunk of
// at most 1024 samples keeps every partial sum at or below 2^24 in magnitude, where fp32
// holds every integer.  Each D element is converted to int64 before the re/im sums, and
// chunks are flushed to int64; results are bit-exact.  4-bit samples (-8..7) are exact in
// fp8 e4m3 as well: their packed feed converts them to e4m3 operand bytes and issues
// kind::f8f6f4 MMAs (K = 32), with the same fp32 accumulation and chunking.
//
// Float samples (BF16x3): x = h + l with bf16 h, l; MMAs for h h^T, h l^T and l h^T with
// fp32 accumulation.
//
// Two ways to feed the operands:
//   planes  -- the unpack kernel has written fp16 (or bf16 hi/lo; e4m3 for 4-bit samples)
//              sample planes in the interleaved row order; TMA loads 128-row x 128-byte tiles
//              (64 fp16 or 128 e4m3 samples) with 128-byte swizzle straight into the operand
//              ring.
//   raw     -- (4/8-bit samples) TMA loads the packed [time][chan][input] bytes of a
//              64-input x 64-sample block (128 samples for 4-bit e4m3 operands) and eight
//              converter warps turn them into the swizzled operand tiles in shared memory: the
//              unpack/transpose step (Sec. 4) fused into the X kernel, so the samples cross
//              HBM once.  Float samples of single-block arrays go the same way (8-byte
//              complex floats in, bf16 hi and lo tiles out) instead of through planes.
//
// CTA roles (one CTA per SM, persistent over work items = (dump, channel, I, J)):
//   warp 0       TMA producer
//   warp 1       tensor-memory allocator and single-thread MMA issuer
//   warps 2..5   epilogue, one warp per tensor-memory lane quarter: tensor memory ->
//                registers -> lane-pair combine -> int64 -> baseline order, stored from
//                registers (single-block arrays) or staged in shared memory and bulk-copied
//   warps 6..13  (raw only) converters: packed bytes -> fp16 (floats -> bf16 hi/lo) K-major
//                swizzled tiles
// Shared memory is carved at launch: when the array has a single 64-input block every
// item is a diagonal tile (B = A), so stages hold one tile and the rings get deeper.
// Tensor memory holds two accumulators (128 columns each) so the epilogue of one item
// overlaps the MMAs of the next.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <mutex>
#include <new>

#include "corr_internal.h"
#include "sample_convert.cuh"
#include "tc_ptx.cuh"

namespace corr {
namespace {

constexpr int kTileBytes = kBlockRows * kTimeBlock * 2;     // 16 KB: 128 rows x 64 fp16
constexpr uint64_t kWaitLimitNs = 2000000000ull;            // 2 s per wait
constexpr uint64_t kDrainLimitNs = 200000000ull;            // 0.2 s for in-flight work at exit
constexpr int kMaxOpStages = 16;
constexpr int kMaxRawStages = 32;
constexpr int kBarBytes = 8 * (2 * kMaxOpStages + 2 * kMaxRawStages + 5) + 16;
constexpr int kSmemBudget = 227 * 1024 - kBarBytes - 1024;  // ring space after barriers and alignment
// Staged epilogue: a warp's 16 rows of 64 baselines (16 bytes each), row pitch 65 x 16 B so
// that the 16-byte stores of a quarter-warp fall in 8 distinct bank groups.
constexpr int kStageRowBytes = 65 * 16;
constexpr int kStageBytes = 4 * 16 * kStageRowBytes;
// Dump mode stages 8-byte float pairs: rows of 66 slots (16-byte aligned pitch), element j of a
// row at slot (j - J0) + s, with s the parity of the row's first global element index, so a
// slot and its destination are 16-byte aligned together and the bulk copies stay aligned.
constexpr int kStageRowBytesF = 66 * 8;

enum Mode : int { kPlanesF16 = 0, kPlanesBF16x3 = 1, kRaw8 = 2, kRaw4 = 3, kRawF32 = 4, kRaw4F8 = 5, kPlanesF8 = 6 };

template <int MODE>
struct Cfg {
    // kRawF32: float32 complex samples loaded by TMA and split into bf16 hi + lo by the converter
    // warps (the BF16x3 products of the planes path, without the planes in memory)
    static constexpr bool kFloat = MODE == kRawF32;
    // kRaw4F8: 4-bit samples converted to e4m3 operand bytes (kind::f8f6f4): a 128-byte operand
    // row then holds 128 samples, so a stage covers 128 samples in four K = 32 MMAs.  kPlanesF8:
    // the same operands read from e4m3 planes.
    static constexpr bool kF8 = MODE == kRaw4F8 || MODE == kPlanesF8;
    static constexpr bool kRaw = (MODE == kRaw8 || MODE == kRaw4 || kFloat || MODE == kRaw4F8);
    static constexpr bool kBits8 = MODE == kRaw8;
    static constexpr bool kSplit = (MODE == kPlanesBF16x3 || kFloat);
    static constexpr int kEpiWarps = 4;     // one per tensor-memory lane quarter
    static constexpr int kConvWarps = 8;
    static constexpr int kThreads = 64 + 32 * kEpiWarps + (kRaw ? 32 * kConvWarps : 0);
    static constexpr int kBps = kFloat ? 8 : (kBits8 ? 2 : 1);            // packed bytes per sample
    static constexpr int kStageT = kF8 ? 2 * kTimeBlock : kTimeBlock;    // samples per stage
    static constexpr int kRawTileBytes = kRaw ? kStageT * kBlockInputs * kBps : 0;
    // x coordinate of a 64-input block in the raw tensor map: bytes, or 8-byte complex floats
    static constexpr int kMapX = kFloat ? kBlockInputs : kBlockInputs * kBps;
    static constexpr int kTilesPerOperand = kSplit ? 2 : 1;               // hi (+ lo)
};

constexpr int kMaxJobs = kMaxJobsPerLaunch;   // jobs one launch packs (kernel-parameter space holds their maps)

// One correlation job of a launch: its TMA map (packed bytes, or fp16/bf16 hi planes),
// sizes, output and the flat index of its first work item.
struct TcJob {
    CUtensorMap map;
    CUtensorMap map_wide;   // plane path, wide items: boxes of two blocks (256 rows)
    void* vis;
    int64_t item_begin;  // first flat item of this job
    int n_inputs;
    int n_chan;
    int nb;              // 64-input blocks
    int kp;              // samples per dump rounded up to 64
    int n_tiles;         // work items per channel group: nb (nb + 1) / 2 tiles, or S(nb) wide items
    int tw;              // 2: wide items (block I against blocks J0, J0 + 1, one N = 256 MMA); 1: tiles
    int cpi;             // channels per work item (2: adjacent channel pair, single-block arrays)
    int n_groups;        // channel groups per dump = ceil(n_chan / cpi)
    int chunk_kb;        // stages (64 samples; 128 with e4m3 operands) per exactly-flushed chunk
    // division by n_tiles and n_groups as q = (umulhi(n, m) + n) >> s (n < 2^31; Granlund and
    // Montgomery, division by invariant integers using multiplication)
    uint32_t tiles_m, groups_m;
    int tiles_s, groups_s;
    // 1: every D element of a chunk is at most 2^23 in magnitude, so rr + ii and ir - ri are
    // exact in fp32 and each needs one conversion (4-bit samples; 8-bit with <= 512 samples)
    int f32_combine;
    // 1: dump mode (Fig. 1, Sec. 2) -- the epilogue writes float32 V / n_accum rotated by
    // phasor_i conj(phasor_j) (phasor [n_chan][n_inputs] or nullptr: no rotation) instead of
    // the exact int64 sums; a dump must fit one exact chunk and is never accumulated
    int out_mode;
    const float2* phasor;
    float inv_n;
};

template <int MAXJ>
struct TcLaunch {
    CUtensorMap map_lo;  // BF16x3 lo planes (single-job launches only)
    int n_jobs;
    int64_t n_items;     // sum over jobs of n_dumps * n_groups * n_tiles
    int accumulate;
    int* status;
    uint32_t tmem_cols;  // 256 or 512 (two accumulator sets of up to 2 x 128 columns)
    // shared-memory carve-up (bytes; ring base is 1024-aligned)
    int op_stages;
    int op_stage_bytes;  // operand tiles of one stage: A (+ B, or a second channel) (x2 for hi/lo)
    int b_offset;        // offset of the B tile(s) inside an op stage (0: B = A)
    int raw_stages;
    int raw_stage_bytes;
    int raw_offset;      // start of the raw ring
    int bar_offset;      // start of the barriers
    uint64_t wait_limit_ns;  // bound of every mbarrier wait
    int64_t stall_item;  // self-test: the producer withholds the first stage of this item (-1: none)
    int staged;          // 1: epilogue stages rows in shared memory and bulk-copies them out
    int staging_offset;  // start of the staging area (4 warps x 16 rows x kStageRowBytes)
    TcJob jobs[MAXJ];
};

// Work-item coordinates.  Items are visited in increasing order by every role, so the job
// index only moves forward.
struct ItemCtx {
    int j;
    int I, J;            // J: the first B block (wide items: J and J + 1 when nsub = 2)
    bool same;
    bool wide;
    int nsub;            // accumulators of the item: channels (cpi) or B blocks (wide)
    int64_t d;           // dump within the job
    int c0;              // first channel of the item
};

// Tiles are numbered row by row over I <= J: row I starts at off(I) = I nb - I (I - 1) / 2.
// The row is the larger root bound of off(I) <= tile, taken in float and corrected exactly.
__device__ __forceinline__ void tile_coords(int tile, int nb, int& I, int& J) {
    const int b = 2 * nb + 1;
    int i = (int)(((float)b - sqrtf((float)(b * b - 8 * tile))) * 0.5f);
    i = max(0, min(i, nb - 1));
    while (i > 0 && i * nb - i * (i - 1) / 2 > tile) --i;
    while (i + 1 < nb && (i + 1) * nb - (i + 1) * i / 2 <= tile) ++i;
    I = i;
    J = i + (tile - (i * nb - i * (i - 1) / 2));
}

// Wide items: row I holds the items J0 = I, I + 2, ... < nb, so the rows of lengths nb .. 1
// start at S(nb) - S(nb - I) with S(m) = floor((m + 1) / 2) floor((m + 2) / 2).  The row is
// the smallest m = nb - I with S(m) >= S(nb) - item, from S(m) ~ (m + 1.5)^2 / 4 in float and
// corrected exactly.
__device__ __forceinline__ int pairs_upto(int m) { return ((m + 1) >> 1) * ((m + 2) >> 1); }

__device__ __forceinline__ void wide_coords(int tile, int nb, int& I, int& J0) {
    const int R = pairs_upto(nb) - tile;
    int m = (int)(2.0f * sqrtf((float)R) - 1.5f);
    m = max(0, min(m, nb));
    while (m > 0 && pairs_upto(m - 1) >= R) --m;
    while (pairs_upto(m) < R) ++m;
    I = nb - m;
    J0 = I + 2 * (tile - (pairs_upto(nb) - pairs_upto(m)));
}

__device__ __forceinline__ uint32_t fast_div(uint32_t n, uint32_t m, int s) {
    return (uint32_t)(((uint64_t)__umulhi(n, m) + n) >> s);
}

template <int MAXJ>
__device__ __forceinline__ void decode_item(const TcLaunch<MAXJ>& L, int64_t item, int& j, ItemCtx& it) {
    while (j + 1 < L.n_jobs && item >= L.jobs[j + 1].item_begin) ++j;
    const TcJob& jb = L.jobs[j];
    const uint32_t local = (uint32_t)(item - jb.item_begin);   // < 2^31 per job (host-checked)
    const uint32_t dg = fast_div(local, jb.tiles_m, jb.tiles_s);
    const int tile = (int)(local - dg * (uint32_t)jb.n_tiles);
    const uint32_t d = fast_div(dg, jb.groups_m, jb.groups_s);
    it.j = j;
    it.d = d;
    it.c0 = (int)(dg - d * (uint32_t)jb.n_groups) * jb.cpi;
    it.wide = jb.tw == 2;
    if (it.wide) {
        wide_coords(tile, jb.nb, it.I, it.J);
        it.nsub = min(2, jb.nb - it.J);
    } else {
        tile_coords(tile, jb.nb, it.I, it.J);
        it.nsub = jb.cpi;
    }
    it.same = it.I == it.J;
}

__device__ __forceinline__ void record_error(int* status, volatile int* abort, int code, int detail) {
    *abort = 1;
    if (atomicCAS(status, 0, code) == 0) status[1] = detail;
}

using conv::lane_selector;
using conv::pair_to_half2;

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ void st_shared_v2_u64(uint32_t addr, uint64_t a, uint64_t b) {
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ void st_shared_v2_f32(uint32_t addr, float a, float b) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ float2 ld_shared_v2_f32(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Per-thread constants of the converters: for each of the 4 output rows a lane writes, the
// byte-lane selector, the row's swizzle-atom offset and (row & 7) << 4.  They depend only on
// the lane, so they are computed once per kernel.
struct ConvLane {
    uint32_t sel[4];
    uint32_t rowoff[4];
    uint32_t r7x16[4];
    // 4-bit: the lane writes its two rows of an input in the order (re, im) or (im, re): the
    // nibble shift of the first row's values and the byte offset of the second row from the first
    uint32_t first_shift;
    int32_t second_delta;
};

// 8-bit: lane l takes inputs 2l, 2l+1; byte lane k of a loaded word is re(2l), im(2l),
// re(2l+1), im(2l+1) = operand row 4l + k.  At step kk the lane writes k = (kk + l/2) & 3,
// so the rows of a quarter-warp (l = 8a .. 8a+7) fall in 8 distinct swizzle chunks: even l
// give (row & 7) in 0..3, odd l in 4..7, and the 16-byte stores never share a bank.
__device__ __forceinline__ ConvLane conv_lane8(int l) {
    ConvLane c;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int k = (kk + (l >> 1)) & 3;
        const int row = 4 * l + k;
        c.sel[kk] = lane_selector(k);
        c.rowoff[kk] = (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
        c.r7x16[kk] = (uint32_t)((row & 7) << 4);
    }
    c.first_shift = 0;
    c.second_delta = 0;
    return c;
}

// 4-bit: lane l takes inputs 4m .. 4m+3 (m = l & 15); at step kk input 4m + k with
// k = (kk + m/2) & 3, and writes rows 2(4m + k) (re) and 2(4m + k) + 1 (im), the im row first
// when m is odd.  A quarter-warp's first rows then have (row & 7) = 2k + (m & 1), eight distinct
// values, and so do its second rows: each 16-byte store of the quarter-warp lands in its own
// swizzle chunk, free of bank conflicts.
__device__ __forceinline__ ConvLane conv_lane4(int l) {
    ConvLane c;
    const int m = l & 15;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int k = (kk + (m >> 1)) & 3;
        const int row = 2 * (4 * m + k) + (m & 1);
        c.sel[kk] = lane_selector(k);
        c.rowoff[kk] = (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
        c.r7x16[kk] = (uint32_t)((row & 7) << 4);
    }
    c.first_shift = (m & 1) ? 0u : 4u;           // re is the high nibble, im the low one
    c.second_delta = (m & 1) ? -128 : 128;
    return c;
}

// One warp-sized slice of a packed 8-bit tile -> interleaved fp16 operand tile.  Lane l holds
// w[e] = bytes 4l .. 4l+3 (re, im of inputs 2l, 2l+1) of sample 8q + e; the slice is the 8
// samples of group q, written as four 16-byte swizzled row chunks.
__device__ __forceinline__ void convert_words8(const uint32_t (&w)[8], uint32_t dst, int q, const ConvLane& cl) {
    const __half2 bias = conv::bias8();
    const uint32_t flip = conv::kFlip8;   // exponent bytes 0x64, sign bit of each sample byte flipped
    const uint32_t q16 = (uint32_t)q << 4;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t sel = cl.sel[kk];
        st_shared_v4(dst + cl.rowoff[kk] + (q16 ^ cl.r7x16[kk]), pair_to_half2(w[0], w[1], sel, flip, bias),
                     pair_to_half2(w[2], w[3], sel, flip, bias), pair_to_half2(w[4], w[5], sel, flip, bias),
                     pair_to_half2(w[6], w[7], sel, flip, bias));
    }
}

// Packed 4-bit words (high nibble re, low nibble im): lane l holds w[e] = inputs 4m .. 4m+3
// (m = l & 15) of the 8 samples of group q; writes the 16-byte chunk q of each of its 8 rows.
__device__ __forceinline__ void convert_words4(const uint32_t (&w)[8], uint32_t dst, int q, const ConvLane& cl) {
    const __half2 bias = conv::bias4();
    const uint32_t flip = conv::kFlip4;   // exponent bytes 0x64, sign bit of each 4-bit sample flipped
    uint32_t a[8], b[8];                  // nibbles of the first and the second row, one per byte
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        a[e] = (w[e] >> cl.first_shift) & 0x0F0F0F0Fu;
        b[e] = (w[e] >> (4u - cl.first_shift)) & 0x0F0F0F0Fu;
    }
    const uint32_t q16 = (uint32_t)q << 4;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t sel = cl.sel[kk];
        const uint32_t at = dst + cl.rowoff[kk];
        st_shared_v4(at + (q16 ^ cl.r7x16[kk]), pair_to_half2(a[0], a[1], sel, flip, bias),
                     pair_to_half2(a[2], a[3], sel, flip, bias), pair_to_half2(a[4], a[5], sel, flip, bias),
                     pair_to_half2(a[6], a[7], sel, flip, bias));
        // the other row of the input: 128 bytes away, (row & 7) differing in its lowest bit
        st_shared_v4(at + (uint32_t)cl.second_delta + (q16 ^ (cl.r7x16[kk] ^ 16u)),
                     pair_to_half2(b[0], b[1], sel, flip, bias), pair_to_half2(b[2], b[3], sel, flip, bias),
                     pair_to_half2(b[4], b[5], sel, flip, bias), pair_to_half2(b[6], b[7], sel, flip, bias));
    }
}

// The e4m3 converter's lane constants: input 4m + k at step kk with k = (kk + m) & 3, its re row
// 2(4m + k) first and the im row after it.  Its stores are half as many as the fp16 ones and
// conflict in pairs; the conflict-free order of conv_lane4 and its loads (a variable shift per
// word, permuted row addresses) measured slower here (1.51-1.55 against 1.45 ms on a 4-bit
// stream of 64 inputs x 768 channels x 50 dumps) though faster for the fp16 converter.
__device__ __forceinline__ ConvLane conv_lane4_f8(int l) {
    ConvLane c;
    const int m = l & 15;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int k = (kk + m) & 3;
        const int row = 2 * (4 * m + k);
        c.sel[kk] = lane_selector(k);
        c.rowoff[kk] = (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
        c.r7x16[kk] = (uint32_t)((row & 7) << 4);
    }
    c.first_shift = 4;
    c.second_delta = 128;
    return c;
}

// Packed 4-bit words -> e4m3 operand tile (128 samples per 128-byte row): lane l holds
// w[e] = inputs 4m .. 4m+3 (m = l & 15) of sample 16c + e, e = 0..15, and writes, for the re
// and im rows of each of its four inputs, the row's 16-byte chunk c (16 samples).
__device__ __forceinline__ void convert_words4_f8(const uint32_t (&w)[16], uint32_t dst, int c, const ConvLane& cl) {
    const __half2 bias = conv::bias4();
    const uint32_t flip = conv::kFlip4;
    uint32_t a[16], b[16];                // re and im nibbles, one per byte (conv_lane4_f8)
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        a[e] = (w[e] >> 4) & 0x0F0F0F0Fu;
        b[e] = w[e] & 0x0F0F0F0Fu;
    }
    const uint32_t c16 = (uint32_t)c << 4;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t sel = cl.sel[kk];
        const uint32_t at = dst + cl.rowoff[kk];
        uint32_t r[4], m[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            r[o] = conv::e4m3x4(pair_to_half2(a[4 * o], a[4 * o + 1], sel, flip, bias),
                          pair_to_half2(a[4 * o + 2], a[4 * o + 3], sel, flip, bias));
            m[o] = conv::e4m3x4(pair_to_half2(b[4 * o], b[4 * o + 1], sel, flip, bias),
                          pair_to_half2(b[4 * o + 2], b[4 * o + 3], sel, flip, bias));
        }
        st_shared_v4(at + (c16 ^ cl.r7x16[kk]), r[0], r[1], r[2], r[3]);
        st_shared_v4(at + 128u + (c16 ^ (cl.r7x16[kk] + 16u)), m[0], m[1], m[2], m[3]);   // the im row
    }
}

// One warp-sized slice of a float32 tile -> bf16 hi and lo operand tiles (hi = bf16(x),
// lo = bf16(x - hi), both rounded to nearest, as the planes path splits).  A raw sample row
// holds 128 words, (re, im) of 64 inputs, so word w of a row is operand row w; lane l takes
// rows l + 32 kk (kk = 0..3) of samples 8q .. 8q + 7 and writes each row's 16-byte chunk q of
// the hi tile and of the lo tile (kTileBytes further).  A quarter-warp's rows differ in
// (row & 7), so its swizzled chunks fall in distinct banks.
__device__ __forceinline__ uint32_t bf16_pair(float a, float b, uint32_t& lo) {
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
    return (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
}

__device__ __forceinline__ void convert_slice_f32(uint32_t raw_tile, uint32_t dst_hi, int q, int lane) {
    constexpr uint32_t kRowBytes = kBlockInputs * 8;   // one sample row of the raw tile
    const uint32_t src = raw_tile + (uint32_t)q * 8u * kRowBytes + 4u * (uint32_t)lane;
    const uint32_t q16 = (uint32_t)q << 4;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t row = (uint32_t)lane + 32u * kk;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(ld_shared_u32(src + (uint32_t)e * kRowBytes + 128u * kk));
        uint32_t h[4], l[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) h[p] = bf16_pair(v[2 * p], v[2 * p + 1], l[p]);
        const uint32_t at = dst_hi + (row >> 3) * 1024u + (row & 7u) * 128u + (q16 ^ ((row & 7u) << 4));
        st_shared_v4(at, h[0], h[1], h[2], h[3]);
        st_shared_v4(at + (uint32_t)kTileBytes, l[0], l[1], l[2], l[3]);
    }
}

__device__ __forceinline__ void bulk_store(void* gdst, uint32_t ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_add_u64(void* gdst, uint32_t ssrc, uint32_t bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}

// One K step of a stage: 16 fp16 samples (kind::f16) or 32 e4m3 samples (kind::f8f6f4); either
// way 32 bytes of each 128-byte operand row, so the descriptors advance alike.
template <bool F8>
__device__ __forceinline__ void mma_op(uint32_t d, uint32_t a_lo, uint32_t b_lo, uint32_t hi, uint32_t idesc,
                                       uint32_t acc) {
    if constexpr (F8) ptx::mma_f8_lo(d, a_lo, b_lo, hi, idesc, acc);
    else ptx::mma_f16_lo(d, a_lo, b_lo, hi, idesc, acc);
}

// DUMP: the epilogue writes the dump-mode float pairs (out_mode = 1 jobs) instead of int64
// sums; a separate instantiation so the exact-output kernels keep their registers.
template <int MODE, int MAXJ, bool DUMP>
__global__ void __launch_bounds__(Cfg<MODE>::kThreads, 1) xeng_tc_kernel(const __grid_constant__ TcLaunch<MAXJ> prm) {
    using C = Cfg<MODE>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* ring = smem;
    uint8_t* rawring = smem + prm.raw_offset;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + prm.bar_offset);
    const int OS = prm.op_stages, RS = prm.raw_stages;
    // barriers: op_full[OS], op_empty[OS], raw_full[RS], raw_empty[RS], acc_full[2], acc_empty[2], drain
    const uint32_t bar_op_full = ptx::smem_u32(bars);
    const uint32_t bar_op_empty = bar_op_full + 8 * OS;
    const uint32_t bar_raw_full = bar_op_empty + 8 * OS;
    const uint32_t bar_raw_empty = bar_raw_full + 8 * RS;
    const uint32_t bar_acc_full = bar_raw_empty + 8 * RS;
    const uint32_t bar_acc_empty = bar_acc_full + 16;
    const uint32_t bar_drain = bar_acc_empty + 16;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OS + 2 * RS + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OS; ++s) {
            ptx::mbar_init(bar_op_full + 8 * s, C::kRaw ? C::kConvWarps : 1);
            ptx::mbar_init(bar_op_empty + 8 * s, 1);
        }
        for (int s = 0; s < RS; ++s) {
            ptx::mbar_init(bar_raw_full + 8 * s, 1);
            ptx::mbar_init(bar_raw_empty + 8 * s, C::kConvWarps);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(bar_acc_full + 8 * b, 1);
            ptx::mbar_init(bar_acc_empty + 8 * b, C::kEpiWarps);
        }
        ptx::mbar_init(bar_drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
        for (int j = 0; j < prm.n_jobs; ++j) {
            ptx::prefetch_tensormap(&prm.jobs[j].map);
            if (!C::kRaw && prm.jobs[j].tw == 2) ptx::prefetch_tensormap(&prm.jobs[j].map_wide);
        }
        if (C::kSplit && !C::kRaw) ptx::prefetch_tensormap(&prm.map_lo);
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(tmem_slot), prm.tmem_cols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;


    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const int S = C::kRaw ? RS : OS;
            const uint32_t bar_full = C::kRaw ? bar_raw_full : bar_op_full;
            const uint32_t bar_empty = C::kRaw ? bar_raw_empty : bar_op_empty;
            int s = 0;
            uint32_t ph = 0;
            int64_t n_slots = 0;       // ring slots used so far (issued or withheld)
            int64_t withheld = -1;     // the slot the self-test withheld
            bool ok = true;
            int jc = 0;
            for (int64_t item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
                ItemCtx it;
                decode_item(prm, item, jc, it);
                const TcJob& jb = prm.jobs[it.j];
                const int I = it.I, J = it.J;
                const bool same = it.same;
                const int nkb = jb.kp / C::kStageT;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!ptx::mbar_wait_bounded(bar_empty + 8 * s, ph ^ 1u, abort_flag, prm.wait_limit_ns)) {
                        record_error(prm.status, abort_flag, kDevTimeoutEmpty, kb);
                        ok = false;
                        break;
                    }
                    const uint32_t fb = bar_full + 8 * s;
                    if (item == prm.stall_item && kb == 0) {
                        // self-test of the bounded waits: nothing will complete this stage
                        withheld = n_slots++;
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                        continue;
                    }
                    if constexpr (C::kRaw) {
                        const uint32_t st = ptx::smem_u32(rawring + s * prm.raw_stage_bytes);
                        // one box covers cpi adjacent channels (cpi x 64 inputs per sample row)
                        ptx::mbar_expect_tx(fb, (same ? (uint32_t)jb.cpi : 2u) * (uint32_t)C::kRawTileBytes);
                        tma_load_4d(st, &jb.map, I * C::kMapX, it.c0, kb * C::kStageT, (int)it.d, fb);
                        if (!same)
                            tma_load_4d(st + C::kRawTileBytes, &jb.map, J * C::kMapX, it.c0, kb * C::kStageT,
                                        (int)it.d, fb);
                    } else {
                        const uint32_t st = ptx::smem_u32(ring + s * prm.op_stage_bytes);
                        const int64_t dc = it.d * jb.n_chan + it.c0;   // planes: one channel per item
                        const int rowA = (int)((dc * jb.nb + I) * kBlockRows);
                        const int rowB = (int)((dc * jb.nb + J) * kBlockRows);
                        const uint32_t bo = (uint32_t)prm.b_offset;
                        if (it.wide) {
                            // B = blocks J (, J + 1) in one box at b_offset; A = block I, or on the
                            // diagonal the first half of the B box itself
                            const uint32_t nB = (uint32_t)it.nsub;
                            ptx::mbar_expect_tx(fb, (nB + (same ? 0u : 1u)) * (uint32_t)kTileBytes);
                            if (!same) ptx::tma_load_2d(st, &jb.map, kb * C::kStageT, rowA, fb);
                            ptx::tma_load_2d(st + bo, nB == 2 ? &jb.map_wide : &jb.map, kb * C::kStageT, rowB, fb);
                        } else {
                            ptx::mbar_expect_tx(fb, (same ? 1u : 2u) * (uint32_t)(C::kTilesPerOperand * kTileBytes));
                            ptx::tma_load_2d(st, &jb.map, kb * C::kStageT, rowA, fb);
                            if (!same) ptx::tma_load_2d(st + bo, &jb.map, kb * C::kStageT, rowB, fb);
                            if (C::kSplit) {
                                ptx::tma_load_2d(st + kTileBytes, &prm.map_lo, kb * C::kStageT, rowA, fb);
                                if (!same) ptx::tma_load_2d(st + bo + kTileBytes, &prm.map_lo, kb * C::kStageT, rowB, fb);
                            }
                        }
                    }
                    ++n_slots;
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            // no copy of ours may still be landing in shared memory when the CTA exits:
            // wait for the last phase issued on each stage (even after an abort)
            if (!ok || *abort_flag) {
                const int64_t n_last = n_slots < S ? n_slots : S;
                for (int64_t k = 0; k < n_last; ++k) {
                    const int64_t idx = n_slots - 1 - k;        // k-th most recent slot
                    if (idx == withheld) continue;              // nothing was issued there
                    const int st = (int)(idx % S);
                    const uint32_t par = (uint32_t)((idx / S) & 1);
                    ptx::mbar_wait_drain(bar_full + 8 * st, par, kDrainLimitNs);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_f16(128, 128, C::kSplit);
            constexpr uint32_t idesc_wide = ptx::idesc_f16(128, 256, C::kSplit);
            constexpr uint32_t desc_hi = ptx::sw128_desc_hi();
            const uint32_t desc_lo_ring = ptx::sw128_desc_lo(ptx::smem_u32(ring));
            const uint32_t stage16 = (uint32_t)prm.op_stage_bytes >> 4;
            const uint32_t boff16 = (uint32_t)prm.b_offset >> 4;
            int s = 0;
            uint32_t ph = 0;
            int abuf = 0;
            uint32_t aph = 0;
            bool ok = true;
            bool any = false;
            int jc = 0;
            for (int64_t item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
                ItemCtx it;
                decode_item(prm, item, jc, it);
                const TcJob& jb = prm.jobs[it.j];
                const bool same = it.same;
                const int nkb = jb.kp / C::kStageT;
                for (int kb0 = 0; ok && kb0 < nkb; kb0 += jb.chunk_kb) {
                    const int kb1 = min(nkb, kb0 + jb.chunk_kb);
                    if (!ptx::mbar_wait_bounded(bar_acc_empty + 8 * abuf, aph ^ 1u, abort_flag, prm.wait_limit_ns)) {
                        record_error(prm.status, abort_flag, kDevTimeoutAccEmpty, kb0);
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t dset = tmem_base + (uint32_t)(abuf * (int)(prm.tmem_cols / 2));
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!ptx::mbar_wait_bounded(bar_op_full + 8 * s, ph, abort_flag, prm.wait_limit_ns)) {
                            record_error(prm.status, abort_flag, kDevTimeoutFull, kb);
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        // descriptor low words, in 16-byte units: the stage, then +1024 per
                        // 16 KB tile, +2 per 16-sample step along the swizzled rows
                        const uint32_t a0 = desc_lo_ring + (uint32_t)s * stage16;
                        const uint32_t acc0 = kb > kb0 ? 1u : 0u;
                        if (!C::kRaw && !C::kSplit && it.wide) {
                            // one M = 128, N = 256 MMA covers tiles (I, J) and (I, J + 1); on the
                            // diagonal A is the first half of the B box
                            const uint32_t b0 = a0 + boff16;
                            const uint32_t aw = same ? b0 : a0;
                            const uint32_t id = it.nsub == 2 ? idesc_wide : idesc;
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                mma_op<C::kF8>(dset, aw + 2u * k, b0 + 2u * k, desc_hi, id, (k > 0) | acc0);
                        } else if constexpr (C::kSplit) {
                            const uint32_t b0 = same ? a0 : a0 + boff16;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const uint32_t ak = a0 + 2u * k, bk = b0 + 2u * k;
                                ptx::mma_f16_lo(dset, ak, bk, desc_hi, idesc, (k > 0) | acc0);
                                ptx::mma_f16_lo(dset, ak, bk + 1024u, desc_hi, idesc, 1u);   // h_i l_j
                                ptx::mma_f16_lo(dset, ak + 1024u, bk, desc_hi, idesc, 1u);   // l_i h_j
                            }
                        } else if (jb.cpi == 2) {
                            // two channels, each its own diagonal tile (B = A), accumulators
                            // interleaved so consecutive MMAs are independent
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const uint32_t acc = (k > 0) | acc0;
                                mma_op<C::kF8>(dset, a0 + 2u * k, a0 + 2u * k, desc_hi, idesc, acc);
                                mma_op<C::kF8>(dset + 128u, a0 + 1024u + 2u * k, a0 + 1024u + 2u * k, desc_hi, idesc,
                                               acc);
                            }
                        } else {
                            const uint32_t b0 = same ? a0 : a0 + boff16;
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                mma_op<C::kF8>(dset, a0 + 2u * k, b0 + 2u * k, desc_hi, idesc, (k > 0) | acc0);
                        }
                        any = true;
                        ptx::mma_commit(bar_op_empty + 8 * s);
                        if (++s == OS) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    ptx::mma_commit(bar_acc_full + 8 * abuf);
                    if (++abuf == 2) {
                        abuf = 0;
                        aph ^= 1u;
                    }
                }
            }
            // every MMA of ours must be complete before tensor memory is released
            if (any) {
                ptx::mma_commit(bar_drain);
                ptx::mbar_wait_drain(bar_drain, 0, kDrainLimitNs);
            }
        }
        __syncwarp();
    } else if (warp < 2 + C::kEpiWarps) {
        // ---------------- epilogue (warps 2..5) ----------------
        // Lane L of quadrant q holds operand row 32q + L: input i_loc = 16q + L/2, real part
        // for even L, imaginary part for odd L.  Per 32 columns (16 inputs j, re/im each)
        // the even lane finishes j = 0..7 and the odd lane j = 8..15 of the chunk.
        const int q = warp & 3;
        const int i_loc = 16 * q + (lane >> 1);
        const bool odd = lane & 1;
        constexpr bool kIntOut = !C::kSplit;
        const uint32_t staging_q = ptx::smem_u32(smem + prm.staging_offset) + (uint32_t)(q * 16 * kStageRowBytes);
        int abuf = 0;
        uint32_t aph = 0;
        bool ok = true;
        int jc = 0;
        for (int64_t item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
            ItemCtx it;
            decode_item(prm, item, jc, it);
            const TcJob& jb = prm.jobs[it.j];
            const int n_in = jb.n_inputs;
            const int64_t P = (int64_t)n_in * (n_in + 1) / 2;
            const int I = it.I, J = it.J;
            const int nkb = jb.kp / C::kStageT;
            const int i = I * kBlockInputs + i_loc;
            const bool row_ok = i < n_in;
            // baseline b(i, j) = row_off + j within one channel's [P] block
            const int64_t row_off = (int64_t)i * n_in - (int64_t)i * (i - 1) / 2 - i;
            for (int kb0 = 0; kb0 < nkb; kb0 += jb.chunk_kb) {
                // lane 0 observes the phase; the warp decides as one.  An accumulator spans a
                // whole chunk of stages, so this wait gets twice the bound: a stage that never
                // arrives is reported by the role waiting for that stage
                const bool got =
                    ptx::mbar_wait_bounded_warp(bar_acc_full + 8 * abuf, aph, abort_flag, 2 * prm.wait_limit_ns);
                if (!got) {
                    if (lane == 0) record_error(prm.status, abort_flag, kDevTimeoutAccFull, kb0);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const bool add = prm.accumulate || kb0 > 0;
                for (int ch = 0; ch < it.nsub; ++ch) {
                // sub-accumulator ch: channel c0 + ch of a channel-pair item, or tile (I, J + ch)
                // of a wide item
                const int Jx = it.wide ? J + ch : J;
                const int cx = it.wide ? it.c0 : it.c0 + ch;
                const bool ch_ok = row_ok && cx < jb.n_chan;
                const int64_t chan_base = (it.d * jb.n_chan + cx) * P;
                const int64_t row_base = chan_base + row_off;
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) +
                                       (uint32_t)(abuf * (int)(prm.tmem_cols / 2) + ch * 128);
                if (kIntOut && prm.staged) {
                    // the bulk copies of the previous channel must have read the staging rows
                    if (lane < 16) bulk_wait_read();
                    __syncwarp();
                }
                // dump mode: this channel's phasors -- gi for the lane's row, and the J block's
                // 64 in shared memory after the warp's staging rows (staged launches)
                const float2* gch = nullptr;
                float2 gi = make_float2(1.f, 0.f);
                uint32_t phs = 0;
                if constexpr (DUMP) {
                    if (jb.phasor && cx < jb.n_chan) {   // warp-uniform: every lane stages
                        gch = jb.phasor + (size_t)cx * n_in;
                        if (row_ok) gi = gch[i];
                        if (prm.staged) {
                            phs = staging_q + 16u * (uint32_t)kStageRowBytesF;
                            for (int u = lane; u < kBlockInputs; u += 32) {
                                const int j = Jx * kBlockInputs + u;
                                const float2 g = j < n_in ? gch[j] : make_float2(1.f, 0.f);
                                st_shared_v2_f32(phs + 8u * (uint32_t)u, g.x, g.y);
                            }
                            __syncwarp();
                        }
                    }
                }
#pragma unroll 1
                for (int m = 0; m < 4; ++m) {
                    uint32_t v[32];
                    __syncwarp();
                    ptx::tmem_ld32(tbase + 32u * m, v);
                    ptx::tmem_wait_ld();
                    // exchange: the even lane keeps j-slots 0..7 and receives the odd lane's
                    // (xi_i xr_j, xi_i xi_j) for them; the odd lane keeps 8..15 likewise
                    uint32_t own0[8], own1[8], oth0[8], oth1[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t s0 = odd ? v[2 * k] : v[2 * k + 16];
                        const uint32_t s1 = odd ? v[2 * k + 1] : v[2 * k + 17];
                        oth0[k] = __shfl_xor_sync(0xffffffffu, s0, 1);
                        oth1[k] = __shfl_xor_sync(0xffffffffu, s1, 1);
                        own0[k] = odd ? v[2 * k + 16] : v[2 * k];
                        own1[k] = odd ? v[2 * k + 17] : v[2 * k + 1];
                    }
                    const int j0 = Jx * kBlockInputs + 16 * m + (odd ? 8 : 0);
                    if constexpr (kIntOut && DUMP) {
                        // dump mode: rr + ii and ir - ri in fp32 (each term exact, the sum rounded
                        // once), scaled by 1 / n_accum and rotated by phasor_i conj(phasor_j)
                        float2 wv[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int j = j0 + k;
                            const float rr = __uint_as_float(odd ? oth0[k] : own0[k]);
                            const float ri = __uint_as_float(odd ? oth1[k] : own1[k]);
                            const float ir = __uint_as_float(odd ? own0[k] : oth0[k]);
                            const float ii = __uint_as_float(odd ? own1[k] : oth1[k]);
                            float2 w = make_float2((rr + ii) * jb.inv_n, (ir - ri) * jb.inv_n);
                            if (gch && j < n_in) {
                                const float2 gj = prm.staged ? ld_shared_v2_f32(phs + 8u * (uint32_t)(j - Jx * kBlockInputs))
                                                             : gch[j];
                                const float2 t = make_float2(w.x * gi.x - w.y * gi.y, w.x * gi.y + w.y * gi.x);
                                w = make_float2(t.x * gj.x + t.y * gj.y, t.y * gj.x - t.x * gj.y);
                            }
                            wv[k] = w;
                        }
                        if (prm.staged) {
                            // slot (j - J0) + s of row lane/2, s = parity of the row's element J0
                            const int s_r = (int)((chan_base + row_off + Jx * kBlockInputs) & 1);
                            const uint32_t rowp = staging_q + (uint32_t)(lane >> 1) * kStageRowBytesF +
                                                  (uint32_t)(j0 - Jx * kBlockInputs + s_r) * 8u;
#pragma unroll
                            for (int k = 0; k < 8; ++k) st_shared_v2_f32(rowp + 8u * (uint32_t)k, wv[k].x, wv[k].y);
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const int j = j0 + k;
                                if (!ch_ok || j < i || j >= n_in) continue;
                                reinterpret_cast<float2*>(jb.vis)[row_base + j] = wv[k];
                            }
                        }
                    } else if constexpr (kIntOut) {
                        // (rr, ri) from the real-part row, (ir, ii) from the imaginary-part row;
                        // every D element is an integer of magnitude <= 2^24: exact in int32
                        long long re[8], imv[8];
                        if (jb.f32_combine) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float rr = __uint_as_float(odd ? oth0[k] : own0[k]);
                                const float ri = __uint_as_float(odd ? oth1[k] : own1[k]);
                                const float ir = __uint_as_float(odd ? own0[k] : oth0[k]);
                                const float ii = __uint_as_float(odd ? own1[k] : oth1[k]);
                                re[k] = __float2int_rn(rr + ii);
                                imv[k] = __float2int_rn(ir - ri);
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float rr = __uint_as_float(odd ? oth0[k] : own0[k]);
                                const float ri = __uint_as_float(odd ? oth1[k] : own1[k]);
                                const float ir = __uint_as_float(odd ? own0[k] : oth0[k]);
                                const float ii = __uint_as_float(odd ? own1[k] : oth1[k]);
                                re[k] = (long long)__float2int_rn(rr) + __float2int_rn(ii);
                                imv[k] = (long long)__float2int_rn(ir) - __float2int_rn(ri);
                            }
                        }
                        if (prm.staged) {
                            // row lane/2 of this warp's staging rows, slots j - J0; odd lanes
                            // write their slots rotated by 4 so a quarter-warp never shares banks
                            const uint32_t rowp = staging_q + (uint32_t)(lane >> 1) * kStageRowBytes +
                                                  (uint32_t)(j0 - Jx * kBlockInputs) * 16u;
#pragma unroll
                            for (int kk = 0; kk < 8; ++kk) {
                                const int k_even = kk, k_odd = (kk + 4) & 7;
                                const long long xr = odd ? re[k_odd] : re[k_even];
                                const long long xi = odd ? imv[k_odd] : imv[k_even];
                                const int k = odd ? k_odd : k_even;
                                st_shared_v2_u64(rowp + 16u * (uint32_t)k, (uint64_t)xr, (uint64_t)xi);
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const int j = j0 + k;
                                if (!ch_ok || j < i || j >= n_in) continue;
                                longlong2 val = make_longlong2(re[k], imv[k]);
                                longlong2* dst = reinterpret_cast<longlong2*>(jb.vis) + row_base + j;
                                if (add) {
                                    const longlong2 old = *dst;
                                    val.x += old.x;
                                    val.y += old.y;
                                }
                                *dst = val;
                            }
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int j = j0 + k;
                            if (!ch_ok || j < i || j >= n_in) continue;
                            const float rr = __uint_as_float(odd ? oth0[k] : own0[k]);
                            const float ri = __uint_as_float(odd ? oth1[k] : own1[k]);
                            const float ir = __uint_as_float(odd ? own0[k] : oth0[k]);
                            const float ii = __uint_as_float(odd ? own1[k] : oth1[k]);
                            float2 val = make_float2(rr + ii, ir - ri);
                            float2* dst = reinterpret_cast<float2*>(jb.vis) + row_base + j;
                            if (add) {
                                const float2 old = *dst;
                                val.x += old.x;
                                val.y += old.y;
                            }
                            *dst = val;
                        }
                    }
                }
                if (DUMP && prm.staged) {
                    // lane r (< 16) writes row r's float pairs [max(J0, i_r), min(J0 + 64, N)):
                    // an unaligned first element by a plain store, the 16-byte-aligned body by a
                    // bulk copy, an odd last element by a plain store
                    fence_async_shared();
                    __syncwarp();
                    if (lane < 16) {
                        const int ir_ = I * kBlockInputs + 16 * q + lane;
                        const int j_lo = max(Jx * kBlockInputs, ir_);
                        const int j_hi = min(Jx * kBlockInputs + kBlockInputs, n_in);
                        if (ir_ < n_in && j_lo < j_hi && cx < jb.n_chan) {
                            const int64_t rstart = chan_base + (int64_t)ir_ * n_in - (int64_t)ir_ * (ir_ - 1) / 2 - ir_;
                            const int s_r = (int)((rstart + Jx * kBlockInputs) & 1);
                            const uint32_t row_src = staging_q + (uint32_t)lane * kStageRowBytesF;
                            float2* vis2 = reinterpret_cast<float2*>(jb.vis);
                            int j = j_lo;
                            if ((rstart + j) & 1) {
                                vis2[rstart + j] =
                                    ld_shared_v2_f32(row_src + (uint32_t)(j - Jx * kBlockInputs + s_r) * 8u);
                                ++j;
                            }
                            const int body = (j_hi - j) & ~1;
                            if (body > 0)
                                bulk_store(vis2 + rstart + j, row_src + (uint32_t)(j - Jx * kBlockInputs + s_r) * 8u,
                                           (uint32_t)body * 8u);
                            j += body;
                            if (j < j_hi)
                                vis2[rstart + j] =
                                    ld_shared_v2_f32(row_src + (uint32_t)(j - Jx * kBlockInputs + s_r) * 8u);
                        }
                        bulk_commit();
                    }
                } else if (kIntOut && prm.staged) {
                    // make the staged rows visible to the bulk-copy engine, then lane r (< 16)
                    // copies row r's valid run of baselines [max(J0, i_r), min(J0 + 64, N))
                    fence_async_shared();
                    __syncwarp();
                    if (lane < 16) {
                        const int ir_ = I * kBlockInputs + 16 * q + lane;
                        const int j_lo = max(Jx * kBlockInputs, ir_);
                        const int j_hi = min(Jx * kBlockInputs + kBlockInputs, n_in);
                        if (ir_ < n_in && j_lo < j_hi && cx < jb.n_chan) {
                            const int64_t b0 = chan_base + (int64_t)ir_ * n_in - (int64_t)ir_ * (ir_ - 1) / 2 +
                                               (j_lo - ir_);
                            const uint32_t src = staging_q + (uint32_t)lane * kStageRowBytes +
                                                 (uint32_t)(j_lo - Jx * kBlockInputs) * 16u;
                            void* dst = reinterpret_cast<longlong2*>(jb.vis) + b0;
                            const uint32_t bytes = (uint32_t)(j_hi - j_lo) * 16u;
                            if (add) bulk_add_u64(dst, src, bytes);
                            else bulk_store(dst, src, bytes);
                        }
                        bulk_commit();
                    }
                }
                }  // sub-accumulators of the item
                // accumulator drained (the loads completed at tcgen05.wait::ld): hand the
                // tensor-memory buffer back to the MMA warp
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(bar_acc_empty + 8 * abuf);
                if (++abuf == 2) {
                    abuf = 0;
                    aph ^= 1u;
                }
            }
        }
        // every bulk copy of ours must have completed before the CTA exits
        if (kIntOut && prm.staged && lane < 16) bulk_wait_all();
    } else if constexpr (C::kRaw) {
        // ---------------- converters (the last kConvWarps warps) ----------------
        const int cwarp = warp - 2 - C::kEpiWarps;   // 0 .. kConvWarps - 1
        const ConvLane cl = C::kBits8 ? conv_lane8(lane) : (C::kF8 ? conv_lane4_f8(lane) : conv_lane4(lane));
        constexpr uint32_t kRow = kBlockInputs * C::kBps;   // packed bytes of 64 inputs
        const uint32_t lane_byte = C::kBits8 ? 4u * lane : 4u * (lane & 15);
        int rs = 0, os = 0;
        uint32_t rph = 0, oph = 0;
        bool ok = true;
        int jc = 0;
        for (int64_t item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
            ItemCtx it;
            decode_item(prm, item, jc, it);
            const int cpi = prm.jobs[it.j].cpi;
            const bool same = it.same;
            const int nkb = prm.jobs[it.j].kp / C::kStageT;
            // The stage holds n_tl packed tiles: cpi channels side by side in each sample row
            // (diagonal items, row pitch cpi x kRow), or blocks I and J (off-diagonal items,
            // pitch kRow).  Each tile splits into warp-sized slices (8 for 8-bit, 4 for 4-bit);
            // the converter warps take slices round-robin.
            constexpr int kSlices = C::kBits8 ? 8 : 4;
            const int n_tl = same ? cpi : 2;
            const bool pair_pitch = same && cpi == 2;
            for (int kb = 0; kb < nkb; ++kb) {
                const bool got =
                    ptx::mbar_wait_bounded_warp(bar_raw_full + 8 * rs, rph, abort_flag, prm.wait_limit_ns) &&
                    ptx::mbar_wait_bounded_warp(bar_op_empty + 8 * os, oph ^ 1u, abort_flag, prm.wait_limit_ns);
                if (!got) {   // the warp decides as one
                    if (lane == 0) record_error(prm.status, abort_flag, kDevTimeoutFull, kb);
                    ok = false;
                    break;
                }
                const uint32_t raw = ptx::smem_u32(rawring + rs * prm.raw_stage_bytes) + lane_byte;
                const uint32_t dst = ptx::smem_u32(ring + os * prm.op_stage_bytes);
                if constexpr (C::kFloat) {
                    // single-block arrays only (one tile, B = A): slice q of the tile per warp
                    const uint32_t raw_tile = ptx::smem_u32(rawring + rs * prm.raw_stage_bytes);
                    for (int sl = cwarp; sl < kTimeBlock / 8; sl += C::kConvWarps)
                        convert_slice_f32(raw_tile, dst, sl, lane);
                } else if constexpr (C::kF8) {
                    // e4m3 operands, a slice per warp: 32 samples of one tile, lanes 0..15 chunk
                    // c = 2 part (samples 16c .. 16c + 15) and 16..31 chunk c + 1.  (The fp16
                    // converter's conflict-free orders below measured slower here: this converter
                    // is bound by its instruction count, not by shared-memory conflicts.)
                    const uint32_t pitch = pair_pitch ? 2 * kRow : kRow;
                    for (int sl = cwarp; sl < n_tl * kSlices; sl += C::kConvWarps) {
                        const int tl = sl / kSlices;
                        const int c = 2 * (sl % kSlices) + (lane >> 4);
                        const uint32_t src = (same ? raw + tl * kRow : raw + tl * C::kRawTileBytes) +
                                             (uint32_t)c * 16u * pitch;
                        uint32_t w[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) w[e] = ld_shared_u32(src + (uint32_t)e * pitch);
                        convert_words4_f8(w, dst + (same ? tl * kTileBytes : tl * prm.b_offset), c, cl);
                    }
                } else {
                const uint32_t pitch = pair_pitch ? 2 * kRow : kRow;
                // all loads of the warp's slices (slices cwarp and cwarp + 8) are issued before
                // the first conversion, so their shared-memory latencies overlap
                constexpr int kSlots = (2 * kSlices + C::kConvWarps - 1) / C::kConvWarps;
                uint32_t w[kSlots][8];
                // 4-bit slices (8 samples of 64 inputs per half-warp) split like the e4m3 ones:
                // by channel with channel pairs, else by sample group with the upper half-warp
                // reading rows in the order e ^ 1 (adjacent samples swapped alike in every odd
                // group of every operand row: a permutation of the sample axis shared by A and B)
                const bool split_ch = !C::kBits8 && pair_pitch;
                const int eflip = (!C::kBits8 && !pair_pitch) ? (lane >> 4) : 0;
#pragma unroll
                for (int v = 0; v < kSlots; ++v) {
                    const int sl = cwarp + C::kConvWarps * v;
                    if (sl < n_tl * kSlices) {
                        const int tl = split_ch ? (lane >> 4) : sl / kSlices, part = sl % kSlices;
                        const int q = C::kBits8 ? part : (split_ch ? sl : 2 * part + (lane >> 4));
                        const uint32_t src = (same ? raw + tl * kRow : raw + tl * C::kRawTileBytes) +
                                             (uint32_t)q * 8u * pitch;
#pragma unroll
                        for (int e = 0; e < 8; ++e) w[v][e] = ld_shared_u32(src + (uint32_t)(e ^ eflip) * pitch);
                    }
                }
#pragma unroll
                for (int v = 0; v < kSlots; ++v) {
                    const int sl = cwarp + C::kConvWarps * v;
                    if (sl < n_tl * kSlices) {
                        const int tl = split_ch ? (lane >> 4) : sl / kSlices, part = sl % kSlices;
                        const uint32_t out = dst + (same ? tl * kTileBytes : tl * prm.b_offset);
                        if constexpr (C::kBits8) convert_words8(w[v], out, part, cl);
                        else convert_words4(w[v], out, split_ch ? sl : 2 * part + (lane >> 4), cl);
                    }
                }
                }   // packed integers
                fence_async_shared();   // generic-proxy writes -> visible to the tensor core
                __syncwarp();
                if (lane == 0) {
                    ptx::mbar_arrive(bar_op_full + 8 * os);
                    ptx::mbar_arrive(bar_raw_empty + 8 * rs);
                }
                if (++rs == RS) {
                    rs = 0;
                    rph ^= 1u;
                }
                if (++os == OS) {
                    os = 0;
                    oph ^= 1u;
                }
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem_base, prm.tmem_cols);
}

// ---- host side --------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D map over plane rows: dim0 = Kp samples (fp16/bf16), dim1 = all 128-row blocks; boxes of
// one block (128 rows) or, for wide items, of two adjacent blocks (256 rows).
// Planes [rows][kp] of 2-byte elements (fp16/bf16: boxes of 64 samples) or of e4m3 bytes
// (UINT8: boxes of 128 samples); either way a box row is 128 bytes, loaded with 128-byte swizzle.
bool make_plane_map(CUtensorMap* map, const void* base, int kp, int64_t rows, CUtensorMapDataType dt,
                    int box_rows = kBlockRows) {
    auto enc = get_encode();
    if (!enc) return false;
    const int elem = dt == CU_TENSOR_MAP_DATA_TYPE_UINT8 ? 1 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * elem};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 4-D map over packed bytes [dump][time][chan][input*bps]; box = 64 inputs x box_chans channels
// x box_t samples (64, or 128 for e4m3 operands).
// Out-of-range inputs (ragged last block) and samples (ragged last block) read as zero.
bool make_raw_map(CUtensorMap* map, const void* base, int n_inputs, int n_chan, int n_time, int n_dumps, int bps,
                  int box_chans, int box_t) {
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t row = (cuuint64_t)n_inputs * bps;
    cuuint64_t dims[4] = {row, (cuuint64_t)n_chan, (cuuint64_t)n_time, (cuuint64_t)n_dumps};
    cuuint64_t strides[3] = {row, row * n_chan, row * n_chan * n_time};
    cuuint32_t box[4] = {(cuuint32_t)(kBlockInputs * bps), (cuuint32_t)box_chans, (cuuint32_t)box_t, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// constants of fast_div for the divisor d (1 <= d <= 2^31)
void fast_div_make(uint32_t d, uint32_t& m, int& s) {
    int l = 0;
    while ((uint64_t{1} << l) < d) ++l;
    m = (uint32_t)(((uint64_t{1} << 32) * ((uint64_t{1} << l) - d)) / d + 1);
    s = l;
}

// S(m) = floor((m + 1) / 2) floor((m + 2) / 2): wide items of an array of m blocks
int wide_items(int m) { return ((m + 1) / 2) * ((m + 2) / 2); }

template <int MODE, int MAXJ>
cudaError_t launch_jobs(const TcJobSpec* specs, int n_jobs, const CUtensorMap* maps, const CUtensorMap* map_lo,
                        int accumulate, int* status, int n_sm, const TcTuning& tune, cudaStream_t s,
                        const CUtensorMap* maps_wide = nullptr) {
    using C = Cfg<MODE>;
    if (n_jobs < 1 || n_jobs > MAXJ) return cudaErrorInvalidValue;
    static_assert(sizeof(TcLaunch<MAXJ>) <= 32000, "kernel parameters exceed the launch limit");
    auto* prm = new (std::nothrow) TcLaunch<MAXJ>();
    if (!prm) return cudaErrorMemoryAllocation;
    prm->n_jobs = n_jobs;
    prm->accumulate = accumulate;
    prm->status = status;
    prm->wait_limit_ns = tune.wait_limit_ns ? tune.wait_limit_ns : kWaitLimitNs;
    prm->stall_item = tune.stall_item;
    if (map_lo) prm->map_lo = *map_lo;
    int64_t items = 0;
    int op_tiles = 1, raw_tiles = 1;
    bool any_pair = false;
    for (int j = 0; j < n_jobs; ++j) {
        const TcJobSpec& sp = specs[j];
        TcJob& jb = prm->jobs[j];
        jb.map = maps[j];
        // wide items only where the MMA feed reads fp16 planes (two blocks per TMA box)
        jb.tw = ((MODE == kPlanesF16 || MODE == kPlanesF8) && sp.tw == 2 && maps_wide) ? 2 : 1;
        if (jb.tw == 2) jb.map_wide = maps_wide[j];
        jb.vis = sp.vis;
        jb.n_inputs = sp.n_inputs;
        jb.n_chan = sp.n_chan;
        jb.nb = (sp.n_inputs + kBlockInputs - 1) / kBlockInputs;
        jb.kp = (sp.n_time + C::kStageT - 1) / C::kStageT * C::kStageT;   // whole stages (zeros past n_time)
        jb.n_tiles = jb.tw == 2 ? wide_items(jb.nb) : jb.nb * (jb.nb + 1) / 2;
        jb.cpi = sp.cpi;
        jb.n_groups = (sp.n_chan + jb.cpi - 1) / jb.cpi;
        // samples per exact chunk: 8-bit 1024 (|sum| <= 1024 * 2^14 = 2^24), 4-bit 131072, float: all
        // (in stages: 64 samples each, 128 for e4m3 operands)
        jb.chunk_kb = C::kSplit ? (jb.kp / kTimeBlock)
                                : (sp.sample_bits == 4 ? 131072 / C::kStageT : 1024 / C::kStageT);
        // |D| <= chunk samples x max |x_a x_b|: 4-bit 2^17 x 2^6 = 2^23, 8-bit 512 x 2^14 = 2^23
        jb.f32_combine = !C::kSplit && (sp.sample_bits == 4 || jb.kp <= 512) ? 1 : 0;
        jb.out_mode = sp.out_mode;
        jb.phasor = static_cast<const float2*>(sp.phasor);
        jb.inv_n = sp.inv_n;
        if (jb.out_mode && (accumulate || jb.kp > jb.chunk_kb * C::kStageT)) {   // one exact chunk per dump
            delete prm;
            return cudaErrorInvalidValue;
        }
        jb.item_begin = items;
        const int64_t job_items = (int64_t)sp.n_dumps * jb.n_groups * jb.n_tiles;
        if (job_items >= (int64_t{1} << 31)) {   // decode_item divides 32-bit item indices
            delete prm;
            return cudaErrorInvalidValue;
        }
        fast_div_make((uint32_t)jb.n_tiles, jb.tiles_m, jb.tiles_s);
        fast_div_make((uint32_t)jb.n_groups, jb.groups_m, jb.groups_s);
        items += job_items;
        // operand tiles one stage needs: A + a two-block B box for wide items
        const int tiles = jb.tw == 2 ? 3 : (jb.nb == 1 ? jb.cpi : 2);
        op_tiles = tiles > op_tiles ? tiles : op_tiles;
        raw_tiles = tiles > raw_tiles ? tiles : raw_tiles;
        any_pair = any_pair || jb.cpi == 2 || jb.tw == 2;   // two 256-column accumulator sets
    }
    prm->n_items = items;
    prm->tmem_cols = any_pair ? 512u : 256u;
    // shared-memory carve-up; multi-block arrays (output-heavy tiles) stage their epilogue rows
    bool any_multi = false, any_dump = false;
    for (int j = 0; j < n_jobs; ++j) {
        any_multi = any_multi || prm->jobs[j].nb > 1;
        any_dump = any_dump || prm->jobs[j].out_mode != 0;
    }
    prm->staged = (!C::kSplit && any_multi) ? 1 : 0;
    const int stage_space = prm->staged ? kStageBytes : 0;
    const int operand_bytes = C::kTilesPerOperand * kTileBytes;
    prm->op_stage_bytes = op_tiles * operand_bytes;
    prm->b_offset = operand_bytes;
    if (C::kRaw) {
        prm->raw_stage_bytes = raw_tiles * C::kRawTileBytes;
        prm->op_stages = tune.op_stages > 0 ? tune.op_stages : (prm->staged ? 3 : 4);
        // a requested depth that leaves fewer than 3 raw stages is reduced to what fits
        while (prm->op_stages > 2 &&
               kSmemBudget - stage_space - prm->op_stages * prm->op_stage_bytes < 3 * prm->raw_stage_bytes)
            --prm->op_stages;
        int raw_space = kSmemBudget - stage_space - prm->op_stages * prm->op_stage_bytes;
        prm->raw_stages = raw_space / prm->raw_stage_bytes;
        if (prm->raw_stages > kMaxRawStages) prm->raw_stages = kMaxRawStages;
        if (prm->raw_stages < 2) {
            delete prm;
            return cudaErrorInvalidValue;
        }
    } else {
        prm->raw_stage_bytes = 0;
        prm->raw_stages = 0;
        // as deep as fits (less any reserve for a kernel running beside it), or the requested
        // depth when that is smaller
        prm->op_stages = (kSmemBudget - stage_space - tune.smem_reserve) / prm->op_stage_bytes;
        if (prm->op_stages > kMaxOpStages) prm->op_stages = kMaxOpStages;
        if (tune.op_stages >= 2 && tune.op_stages < prm->op_stages) prm->op_stages = tune.op_stages;
    }
    if (prm->op_stages < 2 || prm->op_stages > kMaxOpStages) {
        delete prm;
        return cudaErrorInvalidValue;
    }
    prm->raw_offset = prm->op_stages * prm->op_stage_bytes;
    prm->staging_offset = prm->raw_offset + prm->raw_stages * prm->raw_stage_bytes;
    prm->bar_offset = prm->staging_offset + stage_space;
    const int smem_bytes = prm->bar_offset + kBarBytes + 1024;
    auto kern = xeng_tc_kernel<MODE, MAXJ, false>;
    if constexpr (C::kRaw && !C::kFloat && MAXJ == 1) {
        if (any_dump) kern = xeng_tc_kernel<MODE, MAXJ, true>;
    } else if (any_dump) {   // dump mode is built for single-job packed-sample launches only
        delete prm;
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e == cudaSuccess && items > 0) {
        const int grid = (int)(items < n_sm ? items : n_sm);
        kern<<<grid, C::kThreads, smem_bytes, s>>>(*prm);
        e = cudaGetLastError();
    }
    delete prm;
    return e;
}

}  // namespace

cudaError_t launch_xeng_tc(const Plan& p, const void* d_planes, const void* d_planes_lo, int n_dumps, void* d_vis,
                           int accumulate, cudaStream_t s) {
    const int64_t rows = (int64_t)n_dumps * p.n_chan * p.nb * kBlockRows;
    if (rows >= (int64_t)1 << 31) return cudaErrorInvalidValue;   // TMA row coordinates are int32
    CUtensorMap mh, ml;
    TcJobSpec sp{p.n_inputs, p.n_chan, p.n_time, n_dumps, p.sample_bits, d_planes, d_vis, 1};
    TcTuning tune{};
    tune.op_stages = p.tc_op_stages;
    if (d_planes_lo) {
        if (!make_plane_map(&mh, d_planes, p.kp, rows, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) ||
            !make_plane_map(&ml, d_planes_lo, p.kp, rows, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16))
            return cudaErrorInvalidValue;
        return launch_jobs<kPlanesBF16x3, 1>(&sp, 1, &mh, &ml, accumulate, p.d_status, p.n_sm, tune, s);
    }
    if (!make_plane_map(&mh, d_planes, p.kp, rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT16)) return cudaErrorInvalidValue;
    // wide items (one N = 256 MMA over blocks J, J + 1) unless the plan asks for single tiles; by
    // default also single tiles for accumulating dumps shorter than 1024 samples, whose
    // read-modify-write epilogue bounds them and which run faster on the deeper operand ring of
    // 32 KB stages (measured: 1024 inputs x 1228 channels x 472 samples, 4.05 against 4.41 ms)
    const bool wide = p.tc_items == 2 || (p.tc_items == 0 && !(accumulate && p.kp < 1024));
    CUtensorMap mw;
    if (p.nb >= 2 && wide && make_plane_map(&mw, d_planes, p.kp, rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                                            2 * kBlockRows)) {
        sp.tw = 2;
        return launch_jobs<kPlanesF16, 1>(&sp, 1, &mh, nullptr, accumulate, p.d_status, p.n_sm, tune, s, &mw);
    }
    return launch_jobs<kPlanesF16, 1>(&sp, 1, &mh, nullptr, accumulate, p.d_status, p.n_sm, tune, s);
}

bool tc_planes_e4m3(const Plan& p) { return p.sample_bits == 4 && tc_raw_supported(p); }

int tc_kp_e4m3(const Plan& p) { return (p.n_time + 127) / 128 * 128; }

cudaError_t launch_xeng_tc_e4m3_planes(const Plan& p, const void* d_planes, int n_dumps, void* d_vis, int accumulate,
                                       cudaStream_t s) {
    const int64_t rows = (int64_t)n_dumps * p.n_chan * p.nb * kBlockRows;
    if (rows >= (int64_t)1 << 31 || !tc_planes_e4m3(p)) return cudaErrorInvalidValue;
    const int kp8 = tc_kp_e4m3(p);
    CUtensorMap mh, mw;
    TcJobSpec sp{p.n_inputs, p.n_chan, p.n_time, n_dumps, p.sample_bits, d_planes, d_vis, 1};
    TcTuning tune{};
    tune.op_stages = p.tc_op_stages;
    if (!make_plane_map(&mh, d_planes, kp8, rows, CU_TENSOR_MAP_DATA_TYPE_UINT8)) return cudaErrorInvalidValue;
    // item shape as for fp16 planes
    const bool wide = p.tc_items == 2 || (p.tc_items == 0 && !(accumulate && kp8 < 1024));
    if (p.nb >= 2 && wide &&
        make_plane_map(&mw, d_planes, kp8, rows, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2 * kBlockRows)) {
        sp.tw = 2;
        return launch_jobs<kPlanesF8, 1>(&sp, 1, &mh, nullptr, accumulate, p.d_status, p.n_sm, tune, s, &mw);
    }
    return launch_jobs<kPlanesF8, 1>(&sp, 1, &mh, nullptr, accumulate, p.d_status, p.n_sm, tune, s);
}

cudaError_t launch_tc_plane_path(const Plan& p, const void* d_packed, int n_dumps, void* d_ws, void* d_vis,
                                 int accumulate, cudaStream_t s) {
    if (tc_planes_e4m3(p)) {
        const cudaError_t e = launch_unpack_e4m3(p, d_packed, n_dumps, d_ws, s);
        return e == cudaSuccess ? launch_xeng_tc_e4m3_planes(p, d_ws, n_dumps, d_vis, accumulate, s) : e;
    }
    const cudaError_t e = launch_unpack_fp16(p, d_packed, n_dumps, d_ws, s);
    return e == cudaSuccess ? launch_xeng_tc(p, d_ws, nullptr, n_dumps, d_vis, accumulate, s) : e;
}

bool tc_use_planes(const Plan& p) {
    if (!tc_raw_supported(p)) return true;
    if (p.tc_operands == 1 || p.tc_operands == 3) return false;
    if (p.tc_operands == 2) return true;
    return p.nb >= (tc_planes_e4m3(p) ? kPlaneMinBlocksE4m3 : kPlaneMinBlocks);
}

bool tc_raw_supported(int n_inputs, int sample_bits) {
    // TMA needs every global stride (the packed row of N samples) to be a multiple of 16 bytes
    if (sample_bits != 4 && sample_bits != 8) return false;
    const int64_t row = (int64_t)n_inputs * (sample_bits == 8 ? 2 : 1);
    return row % 16 == 0;
}

bool tc_raw_supported(const Plan& p) { return tc_raw_supported(p.n_inputs, p.sample_bits); }

// Channel pairs (256-byte TMA rows, one item's epilogue under the next item's MMAs) for
// single-block arrays, unless there are too few channels to give every SM a pair: a small dump
// then spreads its channels over twice as many CTAs.
int tc_default_cpi(int n_inputs, int64_t channels, int n_sm) {
    if (n_inputs > kBlockInputs) return 1;
    return channels >= 2 * (int64_t)n_sm ? 2 : 1;
}

bool tc_make_raw_map(CUtensorMap* map, const TcJobSpec& sp, bool f8) {
    const int bps = sp.sample_bits == 8 ? 2 : 1;
    return make_raw_map(map, sp.data, sp.n_inputs, sp.n_chan, sp.n_time, sp.n_dumps, bps, sp.cpi,
                        f8 ? Cfg<kRaw4F8>::kStageT : kTimeBlock);
}

cudaError_t launch_xeng_tc_raw_jobs(const TcJobSpec* specs, const CUtensorMap* maps, int n_jobs, int accumulate,
                                    int* status, int n_sm, const TcTuning& tune, cudaStream_t s) {
    if (n_jobs < 1) return cudaErrorInvalidValue;
    const int bits = specs[0].sample_bits;
    for (int j = 0; j < n_jobs; ++j)
        if (specs[j].sample_bits != bits || !tc_raw_supported(specs[j].n_inputs, bits) ||
            (specs[j].cpi != 1 && specs[j].cpi != 2) || (specs[j].cpi == 2 && specs[j].n_inputs > kBlockInputs))
            return cudaErrorInvalidValue;
    if (tune.f8_operands) {   // e4m3 operands: 4-bit samples (maps with 128-sample boxes)
        if (bits != 4) return cudaErrorInvalidValue;
        if (n_jobs == 1) return launch_jobs<kRaw4F8, 1>(specs, 1, maps, nullptr, accumulate, status, n_sm, tune, s);
        if (n_jobs > kMaxJobs) return cudaErrorInvalidValue;
        return launch_jobs<kRaw4F8, kMaxJobs>(specs, n_jobs, maps, nullptr, accumulate, status, n_sm, tune, s);
    }
    if (n_jobs == 1) {
        if (bits == 8) return launch_jobs<kRaw8, 1>(specs, 1, maps, nullptr, accumulate, status, n_sm, tune, s);
        return launch_jobs<kRaw4, 1>(specs, 1, maps, nullptr, accumulate, status, n_sm, tune, s);
    }
    if (n_jobs > kMaxJobs) return cudaErrorInvalidValue;
    if (bits == 8) return launch_jobs<kRaw8, kMaxJobs>(specs, n_jobs, maps, nullptr, accumulate, status, n_sm, tune, s);
    return launch_jobs<kRaw4, kMaxJobs>(specs, n_jobs, maps, nullptr, accumulate, status, n_sm, tune, s);
}

bool tc_make_plane_map(CUtensorMap* map, const TcJobSpec& sp, bool f8) {
    const int nb = (sp.n_inputs + kBlockInputs - 1) / kBlockInputs;
    const int step = f8 ? Cfg<kPlanesF8>::kStageT : kTimeBlock;
    const int kp = (sp.n_time + step - 1) / step * step;
    const int64_t rows = (int64_t)sp.n_dumps * sp.n_chan * nb * kBlockRows;
    if (rows >= (int64_t{1} << 31)) return false;   // TMA row coordinates are int32
    return make_plane_map(map, sp.data, kp, rows, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
}

bool tc_make_plane_map_wide(CUtensorMap* map, const TcJobSpec& sp, bool f8) {
    const int nb = (sp.n_inputs + kBlockInputs - 1) / kBlockInputs;
    const int step = f8 ? Cfg<kPlanesF8>::kStageT : kTimeBlock;
    const int kp = (sp.n_time + step - 1) / step * step;
    const int64_t rows = (int64_t)sp.n_dumps * sp.n_chan * nb * kBlockRows;
    if (rows >= (int64_t{1} << 31) || rows < 2 * kBlockRows) return false;
    return make_plane_map(map, sp.data, kp, rows, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                          2 * kBlockRows);
}

cudaError_t launch_xeng_tc_plane_jobs(const TcJobSpec* specs, const CUtensorMap* maps, int n_jobs, int accumulate,
                                      int* status, int n_sm, const TcTuning& tune, cudaStream_t s,
                                      const CUtensorMap* maps_wide) {
    if (n_jobs < 1 || n_jobs > kMaxJobs) return cudaErrorInvalidValue;
    for (int j = 0; j < n_jobs; ++j)
        if ((specs[j].sample_bits != 4 && specs[j].sample_bits != 8) || specs[j].cpi != 1 ||
            (specs[j].tw == 2 && !maps_wide))
            return cudaErrorInvalidValue;
    if (tune.f8_operands) {   // e4m3 planes of 4-bit samples (maps of tc_make_plane_map(..., true))
        for (int j = 0; j < n_jobs; ++j)
            if (specs[j].sample_bits != 4) return cudaErrorInvalidValue;
        if (n_jobs == 1)
            return launch_jobs<kPlanesF8, 1>(specs, 1, maps, nullptr, accumulate, status, n_sm, tune, s, maps_wide);
        return launch_jobs<kPlanesF8, kMaxJobs>(specs, n_jobs, maps, nullptr, accumulate, status, n_sm, tune, s,
                                                maps_wide);
    }
    if (n_jobs == 1)
        return launch_jobs<kPlanesF16, 1>(specs, 1, maps, nullptr, accumulate, status, n_sm, tune, s, maps_wide);
    return launch_jobs<kPlanesF16, kMaxJobs>(specs, n_jobs, maps, nullptr, accumulate, status, n_sm, tune, s,
                                             maps_wide);
}

namespace {
cudaError_t launch_raw_impl(const Plan& p, const void* d_packed, int n_dumps, void* d_vis, int accumulate,
                            cudaStream_t s, const TcTuning* tune, int out_mode, const void* phasor, float inv_n) {
    if (!tc_raw_supported(p) || (reinterpret_cast<uintptr_t>(d_packed) & 15u)) return cudaErrorInvalidValue;
    TcTuning plan_tune;
    plan_tune.op_stages = p.tc_op_stages;
    // 4-bit samples take e4m3 operands unless the plan asks for fp16 (CORR_OPERANDS_PACKED):
    // the same bits, half the operand bytes and MMAs per sample
    const bool f8 = p.sample_bits == 4 && (p.tc_operands == 0 || p.tc_operands == 3);
    TcTuning run_tune = tune ? *tune : plan_tune;
    run_tune.f8_operands = f8 ? 1 : 0;
    const int cpi = tc_default_cpi(p.n_inputs, (int64_t)n_dumps * p.n_chan, p.n_sm);
    // one launch covers fewer than 2^31 work items (the kernel decodes 32-bit item indices)
    const int64_t items_per_dump = (int64_t)((p.n_chan + cpi - 1) / cpi) * (p.nb * (p.nb + 1) / 2);
    const int64_t max_dumps = ((int64_t{1} << 31) - 1) / items_per_dump;
    if (max_dumps < 1) return cudaErrorInvalidValue;
    const size_t packed_dump = (size_t)p.n_time * p.n_chan * p.n_inputs * (p.sample_bits == 8 ? 2 : 1);
    const size_t vis_dump = (size_t)p.n_chan * (size_t)p.n_baselines * (out_mode ? 8 : 16);
    for (int d0 = 0; d0 < n_dumps;) {
        const int nd = (int)((n_dumps - d0) < max_dumps ? (n_dumps - d0) : max_dumps);
        TcJobSpec sp{p.n_inputs, p.n_chan, p.n_time, nd, p.sample_bits,
                     static_cast<const uint8_t*>(d_packed) + (size_t)d0 * packed_dump,
                     static_cast<uint8_t*>(d_vis) + (size_t)d0 * vis_dump, cpi};
        sp.out_mode = out_mode;
        sp.phasor = phasor;
        sp.inv_n = inv_n;
        CUtensorMap m;
        if (!tc_make_raw_map(&m, sp, f8)) return cudaErrorInvalidValue;
        const cudaError_t e = launch_xeng_tc_raw_jobs(&sp, &m, 1, accumulate, p.d_status, p.n_sm, run_tune, s);
        if (e != cudaSuccess) return e;
        d0 += nd;
    }
    return cudaSuccess;
}
}  // namespace

bool tc_rawf32_supported(const Plan& p) {
    // single-block arrays (the float raw stage and hi/lo operand tiles fill the ring), and a
    // row of N complex floats a multiple of 16 bytes (TMA strides)
    return p.sample_bits == 32 && p.n_inputs <= kBlockInputs && (p.n_inputs % 2) == 0;
}

cudaError_t launch_xeng_tc_rawf32(const Plan& p, const void* d_samples, int n_dumps, void* d_vis, int accumulate,
                                  cudaStream_t s) {
    if (!tc_rawf32_supported(p) || (reinterpret_cast<uintptr_t>(d_samples) & 15u)) return cudaErrorInvalidValue;
    if ((int64_t)n_dumps * p.n_chan >= (int64_t{1} << 31)) return cudaErrorInvalidValue;   // 32-bit item indices
    auto enc = get_encode();
    if (!enc) return cudaErrorInvalidValue;
    // [dump][time][chan][input] of 8-byte complex floats; box = 64 inputs x 1 channel x 64 samples
    CUtensorMap m;
    const cuuint64_t row = (cuuint64_t)p.n_inputs * 8;
    cuuint64_t dims[4] = {(cuuint64_t)p.n_inputs, (cuuint64_t)p.n_chan, (cuuint64_t)p.n_time, (cuuint64_t)n_dumps};
    cuuint64_t strides[3] = {row, row * p.n_chan, row * p.n_chan * p.n_time};
    cuuint32_t box[4] = {(cuuint32_t)kBlockInputs, 1, (cuuint32_t)kTimeBlock, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(d_samples), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    TcJobSpec sp{p.n_inputs, p.n_chan, p.n_time, n_dumps, 32, d_samples, d_vis, 1};
    TcTuning tune;
    tune.op_stages = p.tc_op_stages;
    return launch_jobs<kRawF32, 1>(&sp, 1, &m, nullptr, accumulate, p.d_status, p.n_sm, tune, s);
}

cudaError_t launch_xeng_tc_raw(const Plan& p, const void* d_packed, int n_dumps, void* d_vis, int accumulate,
                               cudaStream_t s, const TcTuning* tune) {
    return launch_raw_impl(p, d_packed, n_dumps, d_vis, accumulate, s, tune, 0, nullptr, 1.0f);
}

cudaError_t launch_xeng_tc_raw_dump(const Plan& p, const void* d_packed, int n_dumps, void* d_out, const void* phasor,
                                    float inv_n, cudaStream_t s) {
    return launch_raw_impl(p, d_packed, n_dumps, d_out, 0, s, nullptr, 1, phasor, inv_n);
}

}  // namespace corr

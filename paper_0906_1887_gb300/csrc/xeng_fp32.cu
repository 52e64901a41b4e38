// CUDA-core FP32 X stage: the plain form of the cross-multiply-accumulate.
//
// The paper's group-parallel design (Sec. 4) shares input samples between threads
// through shared memory so each global read feeds several products, with consecutive
// threads on consecutive data so every access is coalesced, and accumulates over a
// large batch in registers (Sec. 4, last paragraphs).  The same ideas, sized for an
// sm_103a SM.  This file holds three kernels: the plane-fed one right below (fp16/fp32
// planes written by the unpack pass), and two that read the packed samples themselves
// (float32 samples; 4/8-bit samples), further down.
//
// Plane-fed kernel: a block owns a 64 x 64 tile of input pairs of one channel, stages 32
// time samples of both 64-input blocks in shared memory, and each thread keeps a 4 x 4
// register tile of complex accumulators (16 products per 16 shared-memory reads per
// sample).  Tiles cover the upper triangle i <= j only.
//
// Integer samples: fp32 partial sums cover at most 64 samples (|Re| <= 64 * 2 * 128^2
// = 2^21 < 2^24, so every partial sum is an exact integer), are added into int32 totals
// over segments of up to 32768 samples (|Re| <= 2^30), and each segment's totals are added
// into the int64 output, so the result equals the int64 definition bit for bit.  Float
// samples: the 64-sample partials are added into fp32 totals (two-level summation).
#include <cuda_fp16.h>

#include <type_traits>

#include "corr_internal.h"

namespace corr {
namespace {

constexpr int kThreads = 256;
constexpr int kTC = 32;            // time samples per shared-memory chunk
constexpr int kStride = kBlockRows + 4;   // keeps (re, im) pairs 8-byte aligned
constexpr int kFlushChunks = 2;    // 2 * 32 = 64 samples per fp32 partial

// Global -> register prefetch of one 32-sample chunk of a 128-row plane block: each
// thread holds 2 (fp16) or 4 (fp32) 16-byte pieces.
template <typename InT>
struct ChunkRegs {
    static constexpr int kPieces = sizeof(InT) == 2 ? 2 : 4;
    uint4 v[kPieces];
};

template <typename InT>
__device__ __forceinline__ void fetch_chunk(const InT* __restrict__ rows, int kp, int t0, ChunkRegs<InT>& r) {
#pragma unroll
    for (int k = 0; k < ChunkRegs<InT>::kPieces; ++k) {
        const int q = threadIdx.x + k * kThreads;
        if constexpr (sizeof(InT) == 2) {
            const int row = q >> 2, part = q & 3;      // 8 samples per piece
            r.v[k] = *reinterpret_cast<const uint4*>(rows + (int64_t)row * kp + t0 + part * 8);
        } else {
            const int row = q >> 3, part = q & 7;      // 4 samples per piece
            r.v[k] = *reinterpret_cast<const uint4*>(rows + (int64_t)row * kp + t0 + part * 4);
        }
    }
}

// Registers -> shared memory, transposed to s[t][row] (row = plane row: 2i re, 2i + 1 im).
template <typename InT>
__device__ __forceinline__ void store_chunk(const ChunkRegs<InT>& r, float* __restrict__ s) {
#pragma unroll
    for (int k = 0; k < ChunkRegs<InT>::kPieces; ++k) {
        const int q = threadIdx.x + k * kThreads;
        if constexpr (sizeof(InT) == 2) {
            const int row = q >> 2, part = q & 3;
            const __half* h = reinterpret_cast<const __half*>(&r.v[k]);
#pragma unroll
            for (int e = 0; e < 8; ++e) s[(part * 8 + e) * kStride + row] = __half2float(h[e]);
        } else {
            const int row = q >> 3, part = q & 7;
            const float* f = reinterpret_cast<const float*>(&r.v[k]);
#pragma unroll
            for (int e = 0; e < 4; ++e) s[(part * 4 + e) * kStride + row] = f[e];
        }
    }
}

// tile index -> (I, J) with I <= J over nb blocks, row-major upper triangle
__device__ __forceinline__ void tile_coords(int tile, int nb, int& I, int& J) {
    int i = 0, rem = tile;
    while (rem >= nb - i) {
        rem -= nb - i;
        ++i;
    }
    I = i;
    J = i + rem;
}

template <typename InT, bool INT_OUT>
__global__ void __launch_bounds__(kThreads, 2)
    xeng_fp32_kernel(const InT* __restrict__ planes, int n_inputs, int n_chan, int nb, int kp, int64_t n_items,
                     int n_tiles, void* __restrict__ vis, int accumulate) {
    __shared__ float sI[kTC * kStride];
    __shared__ float sJ[kTC * kStride];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t P = (int64_t)n_inputs * (n_inputs + 1) / 2;

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tile = (int)(item % n_tiles);
        const int64_t dc = item / n_tiles;  // dump * n_chan + chan
        int I, J;
        tile_coords(tile, nb, I, J);
        const InT* rowsI = planes + ((dc * nb + I) * (int64_t)kBlockRows) * kp;
        const InT* rowsJ = planes + ((dc * nb + J) * (int64_t)kBlockRows) * kp;

        // Segments of at most kSegment samples: int32 totals stay exact within one (|Re| <=
        // 32768 * 2 * 128^2 = 2^30) and are added into the int64 output at its end.
        constexpr int kSegment = 32768;
        for (int s0 = 0; s0 < kp; s0 += kSegment) {
            const int s1 = min(kp, s0 + kSegment);
            float pr[4][4], pi[4][4];
            typename std::conditional<INT_OUT, int, float>::type tr[4][4], ti[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    pr[a][b] = pi[a][b] = 0.f;
                    tr[a][b] = ti[a][b] = 0;
                }

            int chunk = 0;
            ChunkRegs<InT> nI, nJ;
            fetch_chunk<InT>(rowsI, kp, s0, nI);
            fetch_chunk<InT>(rowsJ, kp, s0, nJ);
            for (int t0 = s0; t0 < s1; t0 += kTC) {
                store_chunk<InT>(nI, sI);
                store_chunk<InT>(nJ, sJ);
                __syncthreads();
                if (t0 + kTC < s1) {   // the next chunk's loads overlap this chunk's arithmetic
                    fetch_chunk<InT>(rowsI, kp, t0 + kTC, nI);
                    fetch_chunk<InT>(rowsJ, kp, t0 + kTC, nJ);
                }
#pragma unroll 4
                for (int t = 0; t < kTC; ++t) {
                    float2 a[4], b[4];   // (re, im) of inputs ty + 16a and tx + 16b
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        a[k] = *reinterpret_cast<const float2*>(sI + t * kStride + 2 * (ty + 16 * k));
                        b[k] = *reinterpret_cast<const float2*>(sJ + t * kStride + 2 * (tx + 16 * k));
                    }
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4)
#pragma unroll
                        for (int j4 = 0; j4 < 4; ++j4) {
                            // x_i * conj(x_j): re = ar*br + ai*bi, im = ai*br - ar*bi
                            pr[i4][j4] = fmaf(a[i4].x, b[j4].x, pr[i4][j4]);
                            pr[i4][j4] = fmaf(a[i4].y, b[j4].y, pr[i4][j4]);
                            pi[i4][j4] = fmaf(a[i4].y, b[j4].x, pi[i4][j4]);
                            pi[i4][j4] = fmaf(-a[i4].x, b[j4].y, pi[i4][j4]);
                        }
                }
                __syncthreads();
                if (++chunk == kFlushChunks || t0 + kTC >= s1) {
                    chunk = 0;
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            if constexpr (INT_OUT) {
                                tr[a][b] += __float2int_rn(pr[a][b]);   // exact: |partial| <= 2^21
                                ti[a][b] += __float2int_rn(pi[a][b]);
                            } else {
                                tr[a][b] += pr[a][b];
                                ti[a][b] += pi[a][b];
                            }
                            pr[a][b] = pi[a][b] = 0.f;
                        }
                }
            }

            // dump in baseline order: vis[dc][b(i,j)][re, im] for i <= j < N
            const bool add = accumulate || s0 > 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int i = I * kBlockInputs + ty + 16 * a;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int j = J * kBlockInputs + tx + 16 * b;
                    if (i <= j && j < n_inputs) {
                        const int64_t bl = (int64_t)i * n_inputs - (int64_t)i * (i - 1) / 2 + (j - i);
                        const int64_t o = (dc * P + bl);
                        if constexpr (INT_OUT) {
                            longlong2* dst = reinterpret_cast<longlong2*>(vis) + o;
                            longlong2 v = make_longlong2(tr[a][b], ti[a][b]);
                            if (add) {
                                longlong2 old = *dst;
                                v.x += old.x;
                                v.y += old.y;
                            }
                            *dst = v;
                        } else {
                            float2* dst = reinterpret_cast<float2*>(vis) + o;
                            float2 v = make_float2(tr[a][b], ti[a][b]);
                            if (add) {
                                float2 old = *dst;
                                v.x += old.x;
                                v.y += old.y;
                            }
                            *dst = v;
                        }
                    }
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_xeng_fp32(const Plan& p, const void* d_planes, int n_dumps, void* d_vis, int accumulate,
                             cudaStream_t s) {
    const int n_tiles = p.nb * (p.nb + 1) / 2;
    const int64_t n_items = (int64_t)n_dumps * p.n_chan * n_tiles;
    const int64_t cap = (int64_t)p.n_sm * 2 * 16;
    const int grid = (int)(n_items < cap ? n_items : cap);
    if (p.sample_bits == 32) {
        xeng_fp32_kernel<float, false><<<grid, kThreads, 0, s>>>(static_cast<const float*>(d_planes), p.n_inputs,
                                                                  p.n_chan, p.nb, p.kp, n_items, n_tiles, d_vis,
                                                                  accumulate);
    } else {
        xeng_fp32_kernel<__half, true><<<grid, kThreads, 0, s>>>(static_cast<const __half*>(d_planes), p.n_inputs,
                                                                  p.n_chan, p.nb, p.kp, n_items, n_tiles, d_vis,
                                                                  accumulate);
    }
    return cudaGetLastError();
}

// ---- FP32 CUDA-core engine reading the packed samples directly ----------------------------
//
// The plain form as run by corr_xengine_run: no unpack pass, and no products below the
// diagonal.  Two kernels below share one design (4 x 8 register sub-blocks, diagonal tiles as
// sub-blocks plus 8 x 8 triangles, several channel-dumps per block): one for 4/8-bit samples
// (converted in shared memory, exact integer partials into the int64 output) and one for float32
// samples (copied straight into shared memory, fp32 partials over 64 samples into the float32
// output).
namespace {

template <int BITS>
__device__ __forceinline__ float2 load_packed(const unsigned char* __restrict__ p, int64_t idx) {
    if constexpr (BITS == 4) {
        const int b = p[idx];
        return make_float2((float)((int)((unsigned)b << 24) >> 28), (float)((int)((unsigned)b << 28) >> 28));
    } else if constexpr (BITS == 8) {
        const unsigned short v = reinterpret_cast<const unsigned short*>(p)[idx];
        return make_float2((float)(signed char)(v & 0xFF), (float)(signed char)(v >> 8));
    } else {
        return reinterpret_cast<const float2*>(p)[idx];
    }
}

// strictly-upper tile index -> (I, J), I < J < nb, row-major
__device__ __forceinline__ void off_tile(int tile, int nb, int& I, int& J) {
    int i = 0, rem = tile;
    while (rem >= nb - 1 - i) {
        rem -= nb - 1 - i;
        ++i;
    }
    I = i;
    J = i + 1 + rem;
}

// ---- integer samples: 4 x 8 register sub-blocks, several channels per block ----
//
// For 4/8-bit samples a thread owns a 4 x 8 sub-block (rows 4g .. 4g+3, columns 8h .. 8h+7, 32
// complex accumulators): per sample it reads 12 float2 operands with six 16-byte loads for 128
// FFMAs, against three loads per 32 FFMAs for 2 x 4, so shared memory is no longer the limit.
// Only fp32 partial sums stay in registers; they are exact integers for a whole segment (8-bit:
// |Re| <= 2 * 128^2 = 2^15 per sample, so 512 samples keep every partial within 2^24; 4-bit:
// |Re| <= 2^7, segments of 32768 samples) and each segment is added into the int64 output in
// place.  An off-diagonal 64 x 64 tile is 128 sub-blocks; a diagonal tile's upper triangle is 56
// sub-blocks (the strictly-upper 8 x 8 blocks) and 8 triangle threads (the 8 x 8 blocks on the
// diagonal, 28 pairs and 8 autos each: the same 128 FFMAs), so no lane idles and no product
// falls below the diagonal.  A block runs four (diagonal, 256 threads) or two (off-diagonal, 256
// threads) channel-dumps of the same tile side by side, two blocks per SM at 128 registers a
// thread; what the loop does not need (the tile, the channel group, sizes) lives in shared
// memory or the kernel parameters, not in registers.  Sample rows in shared memory carry two pad
// slots after every eight inputs, so the eight column groups of a quarter-warp fall in distinct
// bank groups and a row group's loads are broadcasts.  The packed bytes of the next 32-sample
// chunk are copied asynchronously (cp.async, no registers) while the block computes the current
// one, then converted to float2 rows in shared memory.
constexpr int kIChunk = 32;                          // samples per shared-memory chunk
constexpr int kIRow = 80;                            // float2 slots per sample row (64 + 16 pads)
constexpr int kIDiagCh = 4;
constexpr int kIOffCh = 2;
constexpr int kIDiagThreads = kIDiagCh * 64;         // 4 x (56 sub-blocks + 8 triangles)
constexpr int kIOffThreads = kIOffCh * 128;          // 256

__device__ __forceinline__ int islot(int i) { return i + 2 * (i >> 3); }

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int BITS, int NBLK>
struct IShape {
    static constexpr int kBps = BITS == 4 ? 1 : 2;        // packed bytes per input sample
    static constexpr int kPieces = 64 * kBps / 16;        // 16-byte pieces per 64-input block row
    static constexpr int kPerPiece = 16 / kBps;           // inputs per piece
    static constexpr int kPerCh = NBLK * kIChunk * kPieces;   // pieces per channel-dump and chunk
};

// Raw staging of one chunk (vector form: packed rows of whole 16-byte pieces).  Piece k of the
// chunk is (q, t, blk, piece) with piece fastest; channel-dump q's packed row of sample t starts
// at element base[q] + t * tstride (base[q] < 0: past the last channel-dump, zero fill), and so
// do inputs past the last one and samples past s1.
template <int BITS, int NBLK, int KCH, int NT>
__device__ __forceinline__ void istage(const unsigned char* __restrict__ packed, uint4* __restrict__ raw,
                                       const int64_t* __restrict__ base, int64_t tstride, int tid, int n_inputs,
                                       int t0, int s1, int I, int J) {
    using S = IShape<BITS, NBLK>;
    for (int k = tid; k < KCH * S::kPerCh; k += NT) {
        const int q = k / S::kPerCh, r = k % S::kPerCh;
        const int piece = r % S::kPieces, blk = (r / S::kPieces) % NBLK, t = r / (S::kPieces * NBLK);
        const int i0 = (blk ? J : I) * 64 + piece * S::kPerPiece;
        const int64_t b = base[q];
        const unsigned char* src = packed;
        int bytes = 0;
        if (b >= 0 && t0 + t < s1 && i0 < n_inputs) {
            src = packed + (b + (int64_t)(t0 + t) * tstride + i0) * S::kBps;
            bytes = 16;
        }
        cp_async16(raw + k, src, bytes);
    }
}

// raw pieces -> float2 rows s[((q * NBLK + blk) * kIChunk + t) * kIRow + islot(i)].
template <int BITS, int NBLK, int KCH, int NT>
__device__ __forceinline__ void iconvert(const uint4* __restrict__ raw, float2* __restrict__ s, int tid) {
    using S = IShape<BITS, NBLK>;
    for (int k = tid; k < KCH * S::kPerCh; k += NT) {
        const int q = k / S::kPerCh, r = k % S::kPerCh;
        const int piece = r % S::kPieces, blk = (r / S::kPieces) % NBLK, t = r / (S::kPieces * NBLK);
        float2* row = s + ((q * NBLK + blk) * kIChunk + t) * kIRow;
        const uint4 v = raw[k];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        if constexpr (BITS == 8) {
            // 8 inputs of (re, im) bytes: eight contiguous slots.  Byte b -> float without an integer
            // conversion: b + 128 (the XOR with 0x80) placed in the low mantissa bits of 2^23 is the
            // float 2^23 + b + 128 exactly; subtracting 2^23 + 128 leaves b (IEEE-754 binary32)
            float4* dst = reinterpret_cast<float4*>(row + islot(piece * 8));
            constexpr float kOff = 8388736.0f;   // 2^23 + 128
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const uint32_t wb = w[x] ^ 0x80808080u;
                dst[x] = make_float4(__uint_as_float(__byte_perm(wb, 0x4Bu, 0x4550)) - kOff,
                                     __uint_as_float(__byte_perm(wb, 0x4Bu, 0x4551)) - kOff,
                                     __uint_as_float(__byte_perm(wb, 0x4Bu, 0x4552)) - kOff,
                                     __uint_as_float(__byte_perm(wb, 0x4Bu, 0x4553)) - kOff);
            }
        } else {
            // 16 inputs, one byte each (high nibble re, low nibble im): two groups of eight
#pragma unroll
            for (int gg = 0; gg < 2; ++gg) {
                float4* dst = reinterpret_cast<float4*>(row + islot(piece * 16 + 8 * gg));
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const uint32_t a = w[2 * gg + (x >> 1)] >> (16 * (x & 1));
                    const uint32_t b0 = a & 0xFF, b1 = (a >> 8) & 0xFF;
                    dst[x] = make_float4((float)((int)(b0 << 24) >> 28), (float)((int)(b0 << 28) >> 28),
                                         (float)((int)(b1 << 24) >> 28), (float)((int)(b1 << 28) >> 28));
                }
            }
        }
    }
}

// Element-wise form for packed rows that are not whole 16-byte pieces (one load at a time: the
// accumulators stay in registers meanwhile).
template <int BITS, int NBLK, int KCH, int NT, int CHUNK = kIChunk>
__device__ __forceinline__ void iload_scalar(const unsigned char* __restrict__ packed, float2* __restrict__ s,
                                             const int64_t* __restrict__ base, int64_t tstride, int tid,
                                             int n_inputs, int t0, int s1, int I, int J) {
    constexpr int kPerCh = NBLK * CHUNK * 64;
    for (int k = tid; k < KCH * kPerCh; k += NT) {
        const int q = k / kPerCh, r = k % kPerCh;
        const int x = r & 63, blk = (r >> 6) % NBLK, t = r / (64 * NBLK);
        const int ig = (blk ? J : I) * 64 + x;
        const int64_t b = base[q];
        float2 v = make_float2(0.f, 0.f);
        if (b >= 0 && t0 + t < s1 && ig < n_inputs) v = load_packed<BITS>(packed, b + (int64_t)(t0 + t) * tstride + ig);
        s[((q * NBLK + blk) * CHUNK + t) * kIRow + islot(x)] = v;
    }
}

// one sample's operands of a 4 x 8 sub-block: rows (4 inputs) and four of the eight columns
struct IRows {
    float r[4], i[4];
};
__device__ __forceinline__ IRows ild4(const float2* p) {
    const float4 u = *reinterpret_cast<const float4*>(p), v = *reinterpret_cast<const float4*>(p + 2);
    return IRows{{u.x, u.z, v.x, v.z}, {u.y, u.w, v.y, v.w}};
}
// x_i conj(x_j) into columns y0 .. y0 + 3 of a 4 x 8 sub-block: re = ar br + ai bi into
// acc[8x + y], im = ai br - ar bi into acc[32 + 8x + y]
__device__ __forceinline__ void icmac(float (&acc)[64], const IRows& a, const IRows& b, int y0) {
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            float& r = acc[8 * x + y0 + y];
            float& m = acc[32 + 8 * x + y0 + y];
            r = fmaf(a.r[x], b.r[y], r);
            r = fmaf(a.i[x], b.i[y], r);
            m = fmaf(a.i[x], b.r[y], m);
            m = fmaf(-a.r[x], b.i[y], m);
        }
}

// The upper triangle of an 8 x 8 diagonal block (inputs v[0..7]): the 28 pairs x < y (pair k in
// row-major order: re acc[2k], im acc[2k + 1]) and the 8 autos (acc[56 + x]; their imaginary part
// is zero and not computed): 128 FFMAs, as for a 4 x 8 sub-block.
__device__ __host__ constexpr int tri_pair(int x, int y) { return x * 7 - x * (x - 1) / 2 + (y - x - 1); }
__device__ __forceinline__ void itri(float (&acc)[64], const IRows& lo, const IRows& hi) {
    float r[8], m[8];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        r[x] = lo.r[x], m[x] = lo.i[x];
        r[4 + x] = hi.r[x], m[4 + x] = hi.i[x];
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        acc[56 + x] = fmaf(r[x], r[x], acc[56 + x]);
        acc[56 + x] = fmaf(m[x], m[x], acc[56 + x]);
#pragma unroll
        for (int y = x + 1; y < 8; ++y) {
            float& re = acc[2 * tri_pair(x, y)];
            float& im = acc[2 * tri_pair(x, y) + 1];
            re = fmaf(r[x], r[y], re);
            re = fmaf(m[x], m[y], re);
            im = fmaf(m[x], r[y], im);
            im = fmaf(-r[x], m[y], im);
        }
    }
}

// A thread's work in a block.  Off-diagonal tiles: two channel-dumps (q) x 128 sub-blocks of 4 x 8
// (row group g = loc / 8, column group h = loc % 8).  Diagonal tiles: the 64 x 64 upper triangle
// is 28 strictly-upper 8 x 8 blocks (R < C), each two 4 x 8 sub-blocks (rows 8R .. 8R+3 and
// 8R+4 .. 8R+7), and 8 diagonal 8 x 8 triangles; four channel-dumps give 224 sub-block threads
// (seven warps) and 32 triangle threads (the eighth warp): no idle lane and no product below the
// diagonal.
template <bool DIAG>
struct ISub {
    int q, g, h;       // channel-dump, row group (4 inputs), column group (8 inputs)
    bool tri;          // diagonal tiles: the triangle of the 8-input block h
    __device__ __forceinline__ explicit ISub(int tid) {
        if (DIAG) {
            tri = tid >= kIDiagCh * 56;
            if (tri) {
                q = (tid - kIDiagCh * 56) >> 3;
                g = 0;
                h = (tid - kIDiagCh * 56) & 7;
            } else {
                q = tid / 56;
                const int loc = tid % 56, pair = loc >> 1;
                int R = 0, rem = pair;
                while (rem >= 7 - R) {
                    rem -= 7 - R;
                    ++R;
                }
                g = 2 * R + (loc & 1);
                h = R + 1 + rem;
            }
        } else {
            tri = false;
            q = tid >> 7;
            g = (tid & 127) >> 3;
            h = tid & 7;
        }
    }
};

// The block's current work item, kept in shared memory rather than registers: the sample loop
// needs every register it can get for accumulators and operands, and these values are only read
// between chunks (staging) and at the end of a segment (the flush).
template <int KCH>
struct IItem {
    int64_t base[KCH];   // element offset of each channel-dump's sample-0 row; -1 past the last one
    int64_t dc0;         // first channel-dump of the group
    int I, J;            // tile: input blocks of the rows and of the columns
    int s_begin, s_end;  // the item's range of samples
};

// One exact partial into the int64 output: the first segment stores (or, accumulating, adds);
// later segments add with fire-and-forget 64-bit reductions (no old values in registers; each
// output element has one writing thread, so program order keeps the sum).
__device__ __forceinline__ void iflush(longlong2* dst, float re, float im, bool add) {
    const long long r = __float2int_rn(re), m = __float2int_rn(im);
    if (add) {
        unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
        atomicAdd(d, (unsigned long long)r);
        atomicAdd(d + 1, (unsigned long long)m);
    } else {
        *dst = make_longlong2(r, m);
    }
}

// VEC: packed rows of whole 16-byte pieces (staged copies); otherwise element-wise loads.
// P = baselines per channel-dump, tstride = elements from one sample row to the next.  An item is
// (channel group, sample range, tile); with ts > 1 sample ranges of range_len samples (whole
// chunks) go to different blocks, every range adds into an output the launcher zeroed first.
template <int BITS, bool DIAG, bool VEC>
__global__ void __launch_bounds__(DIAG ? kIDiagThreads : kIOffThreads, 2)
    xeng_fp32_int_kernel(const unsigned char* __restrict__ packed, int n_inputs, int n_chan, int n_time, int nb,
                         int n_tiles, int64_t P, int64_t tstride, int64_t n_dc, int64_t n_items, int ts,
                         int range_len, longlong2* __restrict__ vis, int accumulate) {
    constexpr int kCh = DIAG ? kIDiagCh : kIOffCh;
    constexpr int kThreads = DIAG ? kIDiagThreads : kIOffThreads;
    constexpr int NBLK = DIAG ? 1 : 2;
    constexpr int kSeg = BITS == 8 ? 512 : 32768;    // exact fp32 partials (see above)
    // [kCh][NBLK][kIChunk][kIRow] float2 rows, then the raw pieces of one chunk, then the item
    extern __shared__ __align__(16) float2 s_dyn[];
    uint4* raw = reinterpret_cast<uint4*>(s_dyn + kCh * NBLK * kIChunk * kIRow);
    IItem<kCh>* item_s = reinterpret_cast<IItem<kCh>*>(raw + kCh * IShape<BITS, NBLK>::kPerCh);
    const volatile IItem<kCh>* info = item_s;
    const int tid = threadIdx.x;
    const float2 *sa, *sb;
    bool tri;
    {
        const ISub<DIAG> u(tid);
        tri = u.tri;
        sa = s_dyn + (u.q * NBLK) * kIChunk * kIRow + (u.tri ? islot(8 * u.h) : islot(4 * u.g));
        sb = s_dyn + (u.q * NBLK + NBLK - 1) * kIChunk * kIRow + islot(8 * u.h);
    }

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        if (tid == 0) {
            const int tile = (int)(item % n_tiles);
            int I, J;
            if (DIAG) {
                I = J = tile;
            } else {
                off_tile(tile, nb, I, J);
            }
            const int64_t rest = item / n_tiles;
            const int r = (int)(rest % ts);
            item_s->I = I;
            item_s->J = J;
            item_s->dc0 = rest / ts * kCh;
            item_s->s_begin = r * range_len;
            item_s->s_end = min(n_time, (r + 1) * range_len);
        }
        if (tid < kCh) {
            const int64_t e = item / n_tiles / ts * kCh + tid;
            item_s->base[tid] = e < n_dc ? ((e / n_chan) * n_time * n_chan + e % n_chan) * (int64_t)n_inputs : -1;
        }
        __syncthreads();
        for (int s0 = info->s_begin; s0 < info->s_end; s0 += kSeg) {
            const int s1 = min(info->s_end, s0 + kSeg);
            float acc[64];
#pragma unroll
            for (int k = 0; k < 64; ++k) acc[k] = 0.f;
            if (VEC && s0 == info->s_begin)
                istage<BITS, NBLK, kCh, kThreads>(packed, raw, item_s->base, tstride, tid, n_inputs, s0, s1, info->I,
                                                  info->J);
            cp_async_commit();
            for (int t0 = s0; t0 < s1; t0 += kIChunk) {
                if constexpr (VEC) {
                    // raw holds this chunk (staged one chunk ahead); every thread is past the
                    // previous chunk's products, so the rows may be overwritten
                    cp_async_wait_all();
                    __syncthreads();
                    iconvert<BITS, NBLK, kCh, kThreads>(raw, s_dyn, tid);
                    __syncthreads();
                    // stage the next chunk: the rest of this segment, then the next segment's first
                    const int tn = t0 + kIChunk, se = info->s_end;
                    if (tn < se)
                        istage<BITS, NBLK, kCh, kThreads>(packed, raw, item_s->base, tstride, tid, n_inputs, tn,
                                                          tn < s1 ? s1 : min(se, s1 + kSeg), info->I, info->J);
                    cp_async_commit();
                } else {
                    __syncthreads();
                    iload_scalar<BITS, NBLK, kCh, kThreads>(packed, s_dyn, item_s->base, tstride, tid, n_inputs, t0,
                                                            s1, info->I, info->J);
                    __syncthreads();
                }
                // (a register-prefetching pipeline across samples measured slower: the other
                // resident warps already cover the shared-memory latency)
                if (DIAG && tri) {   // warp-uniform
#pragma unroll 1
                    for (int t = 0; t < kIChunk; ++t) itri(acc, ild4(sa + t * kIRow), ild4(sa + t * kIRow + 4));
                } else {
#pragma unroll 1
                    for (int t = 0; t < kIChunk; ++t) {
                        const IRows a = ild4(sa + t * kIRow), b0 = ild4(sb + t * kIRow), b1 = ild4(sb + t * kIRow + 4);
                        icmac(acc, a, b0, 0);
                        icmac(acc, a, b1, 4);
                    }
                }
            }
            const ISub<DIAG> u(tid);
            const int64_t dc = info->dc0 + u.q;
            if (dc >= n_dc) continue;
            const bool add = accumulate || s0 > info->s_begin || ts > 1;
            const int I = info->I, J = info->J;
            const int64_t row0 = dc * P;
            auto row_of = [&](int i) { return row0 + (int64_t)i * n_inputs - (int64_t)i * (i - 1) / 2 - i; };
            if (DIAG && u.tri) {
                const int i0 = I * 64 + 8 * u.h;
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const int i = i0 + x;
                    if (i >= n_inputs) continue;
                    longlong2* rowp = vis + row_of(i);
                    iflush(rowp + i, acc[56 + x], 0.f, add);
#pragma unroll
                    for (int y = x + 1; y < 8; ++y)
                        if (i0 + y < n_inputs)
                            iflush(rowp + i0 + y, acc[2 * tri_pair(x, y)], acc[2 * tri_pair(x, y) + 1], add);
                }
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = I * 64 + 4 * u.g + a;
                    if (i >= n_inputs) continue;
                    longlong2* rowp = vis + row_of(i);
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const int j = J * 64 + 8 * u.h + b;
                        if (j < i || j >= n_inputs) continue;
                        iflush(rowp + j, acc[8 * a + b], acc[32 + 8 * a + b], add);
                    }
                }
            }
        }
        // every thread is done with this item's record before thread 0 writes the next one
        __syncthreads();
    }
}

// ---- float32 samples: the same sub-blocks, rows copied straight into shared memory ----
//
// Float samples need no conversion: 16-byte pieces (two inputs' (re, im)) go from the packed rows
// into the float2 rows with cp.async, into one of two row buffers while the block computes on the
// other (16-sample chunks, so both buffers of four diagonal or two off-diagonal channel-dumps fit
// two blocks per SM).  Accuracy as in the kernels above: fp32 partials over 64 samples, each added
// into the float32 output (the first stored unless accumulating or split over sample ranges,
// later ones by vector float2 reductions, one writing thread per element).
constexpr int kFChunk = 16;
constexpr int kFSeg = 64;

template <int NBLK, int KCH, int NT>
__device__ __forceinline__ void fstage(const float2* __restrict__ packed, float2* __restrict__ rows,
                                       const int64_t* __restrict__ base, int64_t tstride, int tid, int n_inputs,
                                       int t0, int s1, int I, int J) {
    constexpr int kPieces = 32;                       // 16-byte pieces (two inputs) per 64-input row
    constexpr int kPerCh = NBLK * kFChunk * kPieces;
    for (int k = tid; k < KCH * kPerCh; k += NT) {
        const int q = k / kPerCh, r = k % kPerCh;
        const int piece = r % kPieces, blk = (r / kPieces) % NBLK, t = r / (kPieces * NBLK);
        const int i0 = (blk ? J : I) * 64 + 2 * piece;
        const int64_t b = base[q];
        const float2* src = packed;
        int bytes = 0;
        if (b >= 0 && t0 + t < s1 && i0 < n_inputs) {
            src = packed + b + (int64_t)(t0 + t) * tstride + i0;
            bytes = 16;
        }
        cp_async16(rows + ((q * NBLK + blk) * kFChunk + t) * kIRow + islot(2 * piece), src, bytes);
    }
}

__device__ __forceinline__ void fflush(float2* dst, float re, float im, bool add) {
    if (add) atomicAdd(dst, make_float2(re, im));
    else *dst = make_float2(re, im);
}

// VEC: an even number of inputs and a 16-byte aligned base (whole 16-byte pieces); otherwise
// element-wise loads.  Items and sample ranges as in xeng_fp32_int_kernel.
template <bool DIAG, bool VEC>
__global__ void __launch_bounds__(DIAG ? kIDiagThreads : kIOffThreads, 2)
    xeng_fp32_float_kernel(const float2* __restrict__ packed, int n_inputs, int n_chan, int n_time, int nb,
                           int n_tiles, int64_t P, int64_t tstride, int64_t n_dc, int64_t n_items, int ts,
                           int range_len, float2* __restrict__ vis, int accumulate) {
    constexpr int kCh = DIAG ? kIDiagCh : kIOffCh;
    constexpr int kThreads = DIAG ? kIDiagThreads : kIOffThreads;
    constexpr int NBLK = DIAG ? 1 : 2;
    constexpr int kBuf = kCh * NBLK * kFChunk * kIRow;   // float2 slots of one row buffer
    // two row buffers [kCh][NBLK][kFChunk][kIRow], then the item
    extern __shared__ __align__(16) float2 s_dyn[];
    IItem<kCh>* item_s = reinterpret_cast<IItem<kCh>*>(s_dyn + 2 * kBuf);
    const volatile IItem<kCh>* info = item_s;
    const int tid = threadIdx.x;
    const float2 *sa, *sb;
    bool tri;
    {
        const ISub<DIAG> u(tid);
        tri = u.tri;
        sa = s_dyn + (u.q * NBLK) * kFChunk * kIRow + (u.tri ? islot(8 * u.h) : islot(4 * u.g));
        sb = s_dyn + (u.q * NBLK + NBLK - 1) * kFChunk * kIRow + islot(8 * u.h);
    }

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        if (tid == 0) {
            const int tile = (int)(item % n_tiles);
            int I, J;
            if (DIAG) {
                I = J = tile;
            } else {
                off_tile(tile, nb, I, J);
            }
            const int64_t rest = item / n_tiles;
            const int r = (int)(rest % ts);
            item_s->I = I;
            item_s->J = J;
            item_s->dc0 = rest / ts * kCh;
            item_s->s_begin = r * range_len;
            item_s->s_end = min(n_time, (r + 1) * range_len);
        }
        if (tid < kCh) {
            const int64_t e = item / n_tiles / ts * kCh + tid;
            item_s->base[tid] = e < n_dc ? ((e / n_chan) * n_time * n_chan + e % n_chan) * (int64_t)n_inputs : -1;
        }
        __syncthreads();
        const int sbeg = info->s_begin;
        if (VEC) {
            fstage<NBLK, kCh, kThreads>(packed, s_dyn, item_s->base, tstride, tid, n_inputs, sbeg,
                                        min(info->s_end, sbeg + kFSeg), info->I, info->J);
            cp_async_commit();
        }
        for (int s0 = sbeg; s0 < info->s_end; s0 += kFSeg) {
            const int s1 = min(info->s_end, s0 + kFSeg);
            float acc[64];
#pragma unroll
            for (int k = 0; k < 64; ++k) acc[k] = 0.f;
            for (int t0 = s0; t0 < s1; t0 += kFChunk) {
                const int buf = ((t0 - sbeg) / kFChunk) & 1;
                if constexpr (VEC) {
                    // this chunk has landed in buf; every thread is past the chunk before, which
                    // used the other buffer: stage the next chunk there
                    cp_async_wait_all();
                    __syncthreads();
                    const int tn = t0 + kFChunk, se = info->s_end;
                    if (tn < se)
                        fstage<NBLK, kCh, kThreads>(packed, s_dyn + (buf ^ 1) * kBuf, item_s->base, tstride, tid,
                                                    n_inputs, tn, tn < s1 ? s1 : min(se, s1 + kFSeg), info->I,
                                                    info->J);
                    cp_async_commit();
                } else {
                    __syncthreads();
                    iload_scalar<32, NBLK, kCh, kThreads, kFChunk>(reinterpret_cast<const unsigned char*>(packed),
                                                                   s_dyn + buf * kBuf, item_s->base, tstride, tid,
                                                                   n_inputs, t0, s1, info->I, info->J);
                    __syncthreads();
                }
                const float2* pa = sa + buf * kBuf;
                const float2* pb = sb + buf * kBuf;
                if (DIAG && tri) {   // warp-uniform
#pragma unroll 1
                    for (int t = 0; t < kFChunk; ++t) itri(acc, ild4(pa + t * kIRow), ild4(pa + t * kIRow + 4));
                } else {
#pragma unroll 1
                    for (int t = 0; t < kFChunk; ++t) {
                        const IRows a = ild4(pa + t * kIRow), b0 = ild4(pb + t * kIRow), b1 = ild4(pb + t * kIRow + 4);
                        icmac(acc, a, b0, 0);
                        icmac(acc, a, b1, 4);
                    }
                }
            }
            const ISub<DIAG> u(tid);
            const int64_t dc = info->dc0 + u.q;
            if (dc >= n_dc) continue;
            const bool add = accumulate || s0 > sbeg || ts > 1;
            const int I = info->I, J = info->J;
            const int64_t row0 = dc * P;
            auto row_of = [&](int i) { return row0 + (int64_t)i * n_inputs - (int64_t)i * (i - 1) / 2 - i; };
            if (DIAG && u.tri) {
                const int i0 = I * 64 + 8 * u.h;
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const int i = i0 + x;
                    if (i >= n_inputs) continue;
                    float2* rowp = vis + row_of(i);
                    fflush(rowp + i, acc[56 + x], 0.f, add);
#pragma unroll
                    for (int y = x + 1; y < 8; ++y)
                        if (i0 + y < n_inputs)
                            fflush(rowp + i0 + y, acc[2 * tri_pair(x, y)], acc[2 * tri_pair(x, y) + 1], add);
                }
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = I * 64 + 4 * u.g + a;
                    if (i >= n_inputs) continue;
                    float2* rowp = vis + row_of(i);
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const int j = J * 64 + 8 * u.h + b;
                        if (j < i || j >= n_inputs) continue;
                        fflush(rowp + j, acc[8 * a + b], acc[32 + 8 * a + b], add);
                    }
                }
            }
        }
        // every thread is done with this item's record before thread 0 writes the next one
        __syncthreads();
    }
}

// Sample ranges per item for a launch of base_items items: with fewer than two waves of two
// blocks per SM, the sample axis is split (whole chunks, at least 64 samples a range).
void sample_ranges(const Plan& p, int64_t base_items, int* ts, int* range_len) {
    const int64_t target = 4LL * p.n_sm;
    int64_t t = 1;
    if (base_items > 0 && base_items < target) t = (target + base_items - 1) / base_items;
    const int64_t t_max = (p.n_time + 63) / 64;
    if (t > t_max) t = t_max;
    if (t < 1) t = 1;
    int len = (int)((p.n_time + t - 1) / t);
    len = (len + kIChunk - 1) / kIChunk * kIChunk;
    *range_len = len;
    *ts = (p.n_time + len - 1) / len;
}

template <int BITS, bool VEC>
cudaError_t launch_int_feed(const Plan& p, const unsigned char* src, int64_t n_dc, longlong2* out, int accumulate,
                            cudaStream_t s) {
    const int bps = BITS == 4 ? 1 : 2;
    const int64_t diag_base = (n_dc + kIDiagCh - 1) / kIDiagCh * p.nb;
    const int64_t off_base = (n_dc + kIOffCh - 1) / kIOffCh * (p.nb * (p.nb - 1) / 2);
    int ts_d, len_d, ts_o, len_o;
    sample_ranges(p, diag_base, &ts_d, &len_d);
    sample_ranges(p, off_base, &ts_o, &len_o);
    const int64_t diag_items = diag_base * ts_d, off_items = off_base * ts_o;
    // rows (20 KB per channel-dump and block), one chunk of raw pieces, the item
    const int per = kIChunk * kIRow * (int)sizeof(float2) + kIChunk * 64 * bps;
    const int smem_diag = kIDiagCh * per + (int)sizeof(IItem<kIDiagCh>);          // 96 KB (8-bit)
    const int smem_off = kIOffCh * 2 * per + (int)sizeof(IItem<kIOffCh>);         // 96 KB (8-bit)
    const int64_t P = p.n_baselines, tstride = (int64_t)p.n_chan * p.n_inputs;
    cudaError_t e = cudaFuncSetAttribute(xeng_fp32_int_kernel<BITS, true, VEC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_diag);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(xeng_fp32_int_kernel<BITS, false, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_off);
    // split sample ranges add into the output: it starts from zero unless accumulating
    if (e == cudaSuccess && !accumulate && (ts_d > 1 || ts_o > 1))
        e = cudaMemsetAsync(out, 0, (size_t)n_dc * P * sizeof(longlong2), s);
    if (e != cudaSuccess) return e;
    if (diag_items > 0) {
        const int64_t cap = (int64_t)p.n_sm * 2;
        const int grid = (int)(diag_items < cap ? diag_items : cap);
        xeng_fp32_int_kernel<BITS, true, VEC><<<grid, kIDiagThreads, smem_diag, s>>>(
            src, p.n_inputs, p.n_chan, p.n_time, p.nb, p.nb, P, tstride, n_dc, diag_items, ts_d, len_d, out,
            accumulate);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (off_items > 0) {
        const int64_t cap = (int64_t)p.n_sm * 2;
        const int grid = (int)(off_items < cap ? off_items : cap);
        xeng_fp32_int_kernel<BITS, false, VEC><<<grid, kIOffThreads, smem_off, s>>>(
            src, p.n_inputs, p.n_chan, p.n_time, p.nb, p.nb * (p.nb - 1) / 2, P, tstride, n_dc, off_items, ts_o,
            len_o, out, accumulate);
    }
    return cudaGetLastError();
}

template <bool VEC>
cudaError_t launch_float_feed(const Plan& p, const float2* src, int64_t n_dc, float2* out, int accumulate,
                              cudaStream_t s) {
    const int64_t diag_base = (n_dc + kIDiagCh - 1) / kIDiagCh * p.nb;
    const int64_t off_base = (n_dc + kIOffCh - 1) / kIOffCh * (p.nb * (p.nb - 1) / 2);
    int ts_d, len_d, ts_o, len_o;
    sample_ranges(p, diag_base, &ts_d, &len_d);
    sample_ranges(p, off_base, &ts_o, &len_o);
    const int64_t diag_items = diag_base * ts_d, off_items = off_base * ts_o;
    // two row buffers (10 KB per channel-dump and block each) and the item: 80 KB
    const int smem_diag = 2 * kIDiagCh * kFChunk * kIRow * (int)sizeof(float2) + (int)sizeof(IItem<kIDiagCh>);
    const int smem_off = 2 * kIOffCh * 2 * kFChunk * kIRow * (int)sizeof(float2) + (int)sizeof(IItem<kIOffCh>);
    const int64_t P = p.n_baselines, tstride = (int64_t)p.n_chan * p.n_inputs;
    cudaError_t e = cudaFuncSetAttribute(xeng_fp32_float_kernel<true, VEC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_diag);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(xeng_fp32_float_kernel<false, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_off);
    if (e == cudaSuccess && !accumulate && (ts_d > 1 || ts_o > 1))
        e = cudaMemsetAsync(out, 0, (size_t)n_dc * P * sizeof(float2), s);
    if (e != cudaSuccess) return e;
    if (diag_items > 0) {
        const int64_t cap = (int64_t)p.n_sm * 2;
        const int grid = (int)(diag_items < cap ? diag_items : cap);
        xeng_fp32_float_kernel<true, VEC><<<grid, kIDiagThreads, smem_diag, s>>>(
            src, p.n_inputs, p.n_chan, p.n_time, p.nb, p.nb, P, tstride, n_dc, diag_items, ts_d, len_d, out,
            accumulate);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (off_items > 0) {
        const int64_t cap = (int64_t)p.n_sm * 2;
        const int grid = (int)(off_items < cap ? off_items : cap);
        xeng_fp32_float_kernel<false, VEC><<<grid, kIOffThreads, smem_off, s>>>(
            src, p.n_inputs, p.n_chan, p.n_time, p.nb, p.nb * (p.nb - 1) / 2, P, tstride, n_dc, off_items, ts_o,
            len_o, out, accumulate);
    }
    return cudaGetLastError();
}

cudaError_t launch_float(const Plan& p, const void* d_packed, int n_dumps, void* d_vis, int accumulate,
                         cudaStream_t s) {
    const auto* src = static_cast<const float2*>(d_packed);
    const bool vec = p.n_inputs % 2 == 0 && (reinterpret_cast<uintptr_t>(d_packed) & 15u) == 0;
    const int64_t n_dc = (int64_t)n_dumps * p.n_chan;
    auto* out = static_cast<float2*>(d_vis);
    return vec ? launch_float_feed<true>(p, src, n_dc, out, accumulate, s)
               : launch_float_feed<false>(p, src, n_dc, out, accumulate, s);
}

template <int BITS>
cudaError_t launch_int(const Plan& p, const void* d_packed, int n_dumps, void* d_vis, int accumulate, cudaStream_t s) {
    const auto* src = static_cast<const unsigned char*>(d_packed);
    const int bps = BITS == 4 ? 1 : 2;
    const bool vec = ((int64_t)p.n_inputs * bps) % 16 == 0 && (reinterpret_cast<uintptr_t>(d_packed) & 15u) == 0;
    const int64_t n_dc = (int64_t)n_dumps * p.n_chan;
    auto* out = static_cast<longlong2*>(d_vis);
    return vec ? launch_int_feed<BITS, true>(p, src, n_dc, out, accumulate, s)
               : launch_int_feed<BITS, false>(p, src, n_dc, out, accumulate, s);
}

}  // namespace

cudaError_t launch_xeng_fp32_packed(const Plan& p, const void* d_packed, int n_dumps, void* d_vis, int accumulate,
                                    cudaStream_t s) {
    if (p.sample_bits == 4) return launch_int<4>(p, d_packed, n_dumps, d_vis, accumulate, s);
    if (p.sample_bits == 8) return launch_int<8>(p, d_packed, n_dumps, d_vis, accumulate, s);
    return launch_float(p, d_packed, n_dumps, d_vis, accumulate, s);
}

}  // namespace corr

// Unpack/transpose kernels: packed time-ordered samples -> per-input sample planes.
//
// The paper's first GPU step (Sec. 4) takes a block of N_I x N_C samples ordered with
// the input index fastest, converts them to floating point and regroups them so each
// input's samples are contiguous -- a transpose of the block.  Here the transpose is
// staged through shared memory so both the reads (consecutive inputs) and the writes
// (consecutive time samples of one plane row) are coalesced.
//
// Output planes: [dump][chan][NB][128][Kp]; row 2r holds the real parts and row 2r + 1
// the imaginary parts of input r of the block's 64 inputs; Kp = n_time rounded up to 64;
// padded inputs and samples are zero.  Elements are fp16, or, for the e4m3 plane feed of 4-bit
// samples, e4m3 bytes with Kp = n_time rounded up to 128.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "corr_internal.h"
#include "sample_convert.cuh"

namespace corr {
namespace {

constexpr int kThreads = 256;
constexpr int kPad = 65;  // smem row stride (floats)

enum OutKind { kOutF16 = 0, kOutF32 = 1, kOutBF16Split = 2 };

template <int BITS>
__device__ __forceinline__ void load_sample(const unsigned char* __restrict__ packed, int64_t idx, float& re,
                                            float& im) {
    if constexpr (BITS == 4) {
        int b = packed[idx];
        int r = (b >> 4) & 0xF, m = b & 0xF;
        re = (float)(r >= 8 ? r - 16 : r);
        im = (float)(m >= 8 ? m - 16 : m);
    } else if constexpr (BITS == 8) {
        unsigned short v = reinterpret_cast<const unsigned short*>(packed)[idx];
        re = (float)(signed char)(v & 0xFF);
        im = (float)(signed char)(v >> 8);
    } else {
        float2 v = reinterpret_cast<const float2*>(packed)[idx];
        re = v.x;
        im = v.y;
    }
}

template <int BITS, int OUT>
__global__ void __launch_bounds__(kThreads) unpack_kernel(const unsigned char* __restrict__ packed, int n_inputs,
                                                          int n_chan, int n_time, int nb_count, int kp,
                                                          int64_t n_tiles, void* __restrict__ out0,
                                                          void* __restrict__ out1) {
    __shared__ float s_re[kBlockInputs * kPad];
    __shared__ float s_im[kBlockInputs * kPad];
    const int tb_count = kp / kTimeBlock;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // tile -> (dc, nb, tb); dc = dump * n_chan + chan
        const int tb = (int)(tile % tb_count);
        const int64_t rest = tile / tb_count;
        const int nb = (int)(rest % nb_count);
        const int64_t dc = rest / nb_count;
        const int64_t d = dc / n_chan;
        const int c = (int)(dc % n_chan);
        // load: warp w takes time rows w, w+8, ...; lanes take consecutive inputs
        for (int t = warp; t < kTimeBlock; t += kThreads / 32) {
            const int tg = tb * kTimeBlock + t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                const int ig = nb * kBlockInputs + i;
                float re = 0.f, im = 0.f;
                if (tg < n_time && ig < n_inputs) {
                    const int64_t idx = ((d * n_time + tg) * n_chan + c) * (int64_t)n_inputs + ig;
                    load_sample<BITS>(packed, idx, re, im);
                }
                s_re[i * kPad + t] = re;
                s_im[i * kPad + t] = im;
            }
        }
        __syncthreads();
        // store: 128 rows x 64 samples, 8 samples (one 16-byte fp16 chunk) per step
        const int64_t row0 = ((dc * nb_count) + nb) * (int64_t)kBlockRows;
        for (int q = threadIdx.x; q < kBlockRows * (kTimeBlock / 8); q += kThreads) {
            const int r = q >> 3, ch = q & 7;
            const float* src = ((r & 1) ? s_im : s_re) + (r >> 1) * kPad + ch * 8;
            const int64_t off = (row0 + r) * (int64_t)kp + tb * kTimeBlock + ch * 8;
            if constexpr (OUT == kOutF16) {
                __align__(16) __half v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = __float2half_rn(src[e]);
                *reinterpret_cast<uint4*>(static_cast<__half*>(out0) + off) = *reinterpret_cast<uint4*>(v);
            } else if constexpr (OUT == kOutF32) {
                float4* dst = reinterpret_cast<float4*>(static_cast<float*>(out0) + off);
                dst[0] = make_float4(src[0], src[1], src[2], src[3]);
                dst[1] = make_float4(src[4], src[5], src[6], src[7]);
            } else {
                __align__(16) __nv_bfloat16 hi[8];
                __align__(16) __nv_bfloat16 lo[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    hi[e] = __float2bfloat16_rn(src[e]);
                    lo[e] = __float2bfloat16_rn(src[e] - __bfloat162float(hi[e]));
                }
                *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out0) + off) = *reinterpret_cast<uint4*>(hi);
                *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out1) + off) = *reinterpret_cast<uint4*>(lo);
            }
        }
        __syncthreads();
    }
}

// Packed 4/8-bit rows -> fp16 planes, for arrays whose packed row of N samples is a multiple of
// 16 bytes (so every 64-input block's row starts 16-byte aligned and its valid part is whole
// 16-byte pieces).  A tile is 64 samples x 64 inputs of one channel, handled by one block of
// kTileThreads threads:
//   load:    16-byte pieces of the 64 packed rows (64 x 128 B for 8-bit, 64 x 64 B for 4-bit)
//            into a shared byte tile, with 16-byte chunk c of row t stored at chunk
//            c ^ ((t >> 3) & 7) (8-bit) -- the conversion's reads are then bank-conflict-free;
//            pieces past the array's last input or past the dump's last sample are zero;
//   convert: thread (p, q) takes one 32-bit word (8-bit: inputs 2p, 2p+1; 4-bit: inputs 4p ..
//            4p+3) of the 8 samples 8q .. 8q+7 and writes its 4 (8-bit) or 8 (4-bit) plane rows'
//            16-byte piece q, converted exactly to fp16; lanes with consecutive q write one
//            128-byte row piece together.
template <int BITS>
struct FastTile {
    static constexpr int kRowBytes = kBlockInputs * (BITS == 8 ? 2 : 1);   // 128 or 64
    static constexpr int kWords = kRowBytes / 4;                            // 32 or 16
    static constexpr int kThreads = kWords * 8;                             // 256 or 128
    static constexpr int kTileBytes = kTimeBlock * kRowBytes;
};

// kGroup: tiles whose loads a block issues together (1 for the full grid; 8 for a launch of one
// block per SM beside a tensor-core launch, 64 KB in flight per block).  F8 (4-bit only): the
// planes hold e4m3 bytes instead of fp16 (rows of kp bytes), for the e4m3 plane feed.
template <int BITS, int kGroup, bool F8 = false>
__global__ void __launch_bounds__(FastTile<BITS>::kThreads) unpack_fast_kernel(
    const unsigned char* __restrict__ packed, int n_inputs, int n_chan, int n_time, int nb_count, int kp,
    int64_t n_tiles, void* __restrict__ planes_out) {
    static_assert(!F8 || BITS == 4, "e4m3 planes hold 4-bit samples only");
    __half* __restrict__ planes = static_cast<__half*>(planes_out);
    using F = FastTile<BITS>;
    __shared__ __align__(16) uint32_t tile[F::kTileBytes / 4];
    const int tid = threadIdx.x;
    const int tb_count = kp / kTimeBlock;
    const int64_t row_bytes = (int64_t)n_inputs * (BITS == 8 ? 2 : 1);
    constexpr int kPieces = F::kRowBytes / 16;          // 16-byte pieces per packed row
    constexpr int kPer = kTimeBlock * kPieces / F::kThreads;   // pieces a thread moves per tile (2)
    static_assert(kPer * F::kThreads == kTimeBlock * kPieces, "whole pieces per thread");
    // conversion task of this thread
    const int q = tid & 7, pw = tid >> 3;             // sample group, word within the row
    const uint32_t* src = tile + (size_t)(8 * q) * F::kWords;
    // A block takes kGroup tiles at a time (strided by the grid) and issues every load of the
    // group before converting any: kGroup x 8 KB in flight per block.
    for (int64_t t_base = blockIdx.x; t_base < n_tiles; t_base += (int64_t)kGroup * gridDim.x) {
        uint4 v[kGroup][kPer];
#pragma unroll
        for (int gi = 0; gi < kGroup; ++gi) {
            const int64_t t_idx = t_base + (int64_t)gi * gridDim.x;
            const bool tile_ok = t_idx < n_tiles;
            const int tb = tile_ok ? (int)(t_idx % tb_count) : 0;
            const int64_t rest = tile_ok ? t_idx / tb_count : 0;
            const int nb = (int)(rest % nb_count);
            const int64_t dc = rest / nb_count;          // dump * n_chan + chan
            const int64_t d = dc / n_chan;
            const int c = (int)(dc % n_chan);
            const int64_t valid = row_bytes - (int64_t)nb * F::kRowBytes;   // bytes of this block's row that exist
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int k = tid + u * F::kThreads;
                const int t = k / kPieces, piece = k % kPieces;
                const int tg = tb * kTimeBlock + t;
                v[gi][u] = make_uint4(0u, 0u, 0u, 0u);
                if (tile_ok && tg < n_time && (int64_t)piece * 16 < valid) {
                    const int64_t off =
                        ((d * n_time + tg) * n_chan + c) * row_bytes + (int64_t)nb * F::kRowBytes + piece * 16;
                    v[gi][u] = *reinterpret_cast<const uint4*>(packed + off);
                }
            }
        }
#pragma unroll
        for (int gi = 0; gi < kGroup; ++gi) {
            const int64_t t_idx = t_base + (int64_t)gi * gridDim.x;
            if (t_idx >= n_tiles) break;   // uniform across the block
            const int tb = (int)(t_idx % tb_count);
            const int64_t rest = t_idx / tb_count;
            const int nb = (int)(rest % nb_count);
            const int64_t dc = rest / nb_count;
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int k = tid + u * F::kThreads;
                const int t = k / kPieces, piece = k % kPieces;
                const int chunk = BITS == 8 ? (piece ^ ((t >> 3) & 7)) : (piece ^ ((t >> 3) & 3));
                *reinterpret_cast<uint4*>(tile + t * F::kWords + chunk * 4) = v[gi][u];
            }
            __syncthreads();
            uint32_t w[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int t = 8 * q + e;
                const int word = BITS == 8 ? (pw ^ (((t >> 3) & 7) << 2)) : (pw ^ (((t >> 3) & 3) << 2));
                w[e] = src[e * F::kWords + word];
            }
            __syncthreads();   // the tile is free for the next store once every thread holds its words
            const int64_t row0 = (dc * nb_count + nb) * (int64_t)kBlockRows;
            __half* out = planes + row0 * kp + (int64_t)tb * kTimeBlock + 8 * q;
            if constexpr (BITS == 8) {
                // word pw = (re, im) of inputs 2pw, 2pw + 1 -> plane rows 4pw + k, k = byte lane
                const __half2 bias = conv::bias8();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t sel = conv::lane_selector(k);
                    uint4 o;
                    o.x = conv::pair_to_half2(w[0], w[1], sel, conv::kFlip8, bias);
                    o.y = conv::pair_to_half2(w[2], w[3], sel, conv::kFlip8, bias);
                    o.z = conv::pair_to_half2(w[4], w[5], sel, conv::kFlip8, bias);
                    o.w = conv::pair_to_half2(w[6], w[7], sel, conv::kFlip8, bias);
                    *reinterpret_cast<uint4*>(out + (int64_t)(4 * pw + k) * kp) = o;
                }
            } else if constexpr (F8) {
                // as below, each row's 8 samples written as 8 e4m3 bytes (rows of kp bytes)
                const __half2 bias = conv::bias4();
                unsigned char* out8 = static_cast<unsigned char*>(planes_out) + row0 * kp +
                                      (int64_t)tb * kTimeBlock + 8 * q;
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    hi[e] = (w[e] >> 4) & 0x0F0F0F0Fu;
                    lo[e] = w[e] & 0x0F0F0F0Fu;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t sel = conv::lane_selector(k);
                    uint2 o;
                    o.x = conv::e4m3x4(conv::pair_to_half2(hi[0], hi[1], sel, conv::kFlip4, bias),
                                       conv::pair_to_half2(hi[2], hi[3], sel, conv::kFlip4, bias));
                    o.y = conv::e4m3x4(conv::pair_to_half2(hi[4], hi[5], sel, conv::kFlip4, bias),
                                       conv::pair_to_half2(hi[6], hi[7], sel, conv::kFlip4, bias));
                    *reinterpret_cast<uint2*>(out8 + (int64_t)(8 * pw + 2 * k) * kp) = o;
                    o.x = conv::e4m3x4(conv::pair_to_half2(lo[0], lo[1], sel, conv::kFlip4, bias),
                                       conv::pair_to_half2(lo[2], lo[3], sel, conv::kFlip4, bias));
                    o.y = conv::e4m3x4(conv::pair_to_half2(lo[4], lo[5], sel, conv::kFlip4, bias),
                                       conv::pair_to_half2(lo[6], lo[7], sel, conv::kFlip4, bias));
                    *reinterpret_cast<uint2*>(out8 + (int64_t)(8 * pw + 2 * k + 1) * kp) = o;
                }
            } else {
                // word pw = inputs 4pw .. 4pw + 3, high nibble re, low nibble im -> rows 8pw + 2k (+1)
                const __half2 bias = conv::bias4();
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    hi[e] = (w[e] >> 4) & 0x0F0F0F0Fu;
                    lo[e] = w[e] & 0x0F0F0F0Fu;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t sel = conv::lane_selector(k);
                    uint4 o;
                    o.x = conv::pair_to_half2(hi[0], hi[1], sel, conv::kFlip4, bias);
                    o.y = conv::pair_to_half2(hi[2], hi[3], sel, conv::kFlip4, bias);
                    o.z = conv::pair_to_half2(hi[4], hi[5], sel, conv::kFlip4, bias);
                    o.w = conv::pair_to_half2(hi[6], hi[7], sel, conv::kFlip4, bias);
                    *reinterpret_cast<uint4*>(out + (int64_t)(8 * pw + 2 * k) * kp) = o;
                    o.x = conv::pair_to_half2(lo[0], lo[1], sel, conv::kFlip4, bias);
                    o.y = conv::pair_to_half2(lo[2], lo[3], sel, conv::kFlip4, bias);
                    o.z = conv::pair_to_half2(lo[4], lo[5], sel, conv::kFlip4, bias);
                    o.w = conv::pair_to_half2(lo[6], lo[7], sel, conv::kFlip4, bias);
                    *reinterpret_cast<uint4*>(out + (int64_t)(8 * pw + 2 * k + 1) * kp) = o;
                }
            }
        }
    }
}

template <int BITS>
cudaError_t launch_fast(const Plan& p, const void* d_packed, int n_dumps, void* planes, cudaStream_t s,
                       int blocks_per_sm) {
    using F = FastTile<BITS>;
    const int64_t n_tiles = (int64_t)n_dumps * p.n_chan * p.nb * (p.kp / kTimeBlock);
    if (n_tiles < 1) return cudaSuccess;
    const auto* src = static_cast<const unsigned char*>(d_packed);
    auto* out = static_cast<__half*>(planes);
    if (blocks_per_sm > 0) {   // few blocks: each keeps eight tiles of loads in flight
        const int64_t cap = (int64_t)p.n_sm * blocks_per_sm;
        const int grid = (int)(n_tiles < cap ? n_tiles : cap);
        unpack_fast_kernel<BITS, 8><<<grid, F::kThreads, 0, s>>>(src, p.n_inputs, p.n_chan, p.n_time, p.nb, p.kp,
                                                                 n_tiles, out);
    } else {                   // the whole GPU: many blocks, one tile each at a time
        const int64_t cap = (int64_t)p.n_sm * (BITS == 8 ? 8 : 16);
        const int grid = (int)(n_tiles < cap ? n_tiles : cap);
        unpack_fast_kernel<BITS, 1><<<grid, F::kThreads, 0, s>>>(src, p.n_inputs, p.n_chan, p.n_time, p.nb, p.kp,
                                                                 n_tiles, out);
    }
    return cudaGetLastError();
}

// 4-bit samples into e4m3 planes with rows of kp8 bytes (n_time rounded up to 128 samples);
// blocks_per_sm as for launch_fast
cudaError_t launch_fast_e4m3(const Plan& p, const void* d_packed, int n_dumps, void* planes, int kp8,
                             cudaStream_t s, int blocks_per_sm) {
    using F = FastTile<4>;
    const int64_t n_tiles = (int64_t)n_dumps * p.n_chan * p.nb * (kp8 / kTimeBlock);
    if (n_tiles < 1) return cudaSuccess;
    const auto* src = static_cast<const unsigned char*>(d_packed);
    if (blocks_per_sm > 0) {
        const int64_t cap = (int64_t)p.n_sm * blocks_per_sm;
        const int grid = (int)(n_tiles < cap ? n_tiles : cap);
        unpack_fast_kernel<4, 8, true><<<grid, F::kThreads, 0, s>>>(src, p.n_inputs, p.n_chan, p.n_time, p.nb, kp8,
                                                                    n_tiles, planes);
    } else {
        const int64_t cap = (int64_t)p.n_sm * 16;
        const int grid = (int)(n_tiles < cap ? n_tiles : cap);
        unpack_fast_kernel<4, 1, true><<<grid, F::kThreads, 0, s>>>(src, p.n_inputs, p.n_chan, p.n_time, p.nb, kp8,
                                                                    n_tiles, planes);
    }
    return cudaGetLastError();
}

template <int BITS, int OUT>
cudaError_t launch(const Plan& p, const void* d_packed, int n_dumps, void* o0, void* o1, cudaStream_t s) {
    const int64_t n_tiles = (int64_t)n_dumps * p.n_chan * p.nb * (p.kp / kTimeBlock);
    const int64_t cap = (int64_t)p.n_sm * 8;
    const int grid = (int)(n_tiles < cap ? n_tiles : cap);
    unpack_kernel<BITS, OUT><<<grid, kThreads, 0, s>>>(static_cast<const unsigned char*>(d_packed), p.n_inputs,
                                                        p.n_chan, p.n_time, p.nb, p.kp, n_tiles, o0, o1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_unpack_fp16(const Plan& p, const void* d_packed, int n_dumps, void* d_planes, cudaStream_t s,
                               int blocks_per_sm) {
    // packed rows of whole 16-byte pieces (and a 16-byte aligned base) take the vectorised kernel
    const int64_t row = (int64_t)p.n_inputs * (p.sample_bits == 8 ? 2 : 1);
    const bool fast = row % 16 == 0 && (reinterpret_cast<uintptr_t>(d_packed) & 15u) == 0 &&
                      (reinterpret_cast<uintptr_t>(d_planes) & 15u) == 0;
    if (p.sample_bits == 4)
        return fast ? launch_fast<4>(p, d_packed, n_dumps, d_planes, s, blocks_per_sm)
                    : launch<4, kOutF16>(p, d_packed, n_dumps, d_planes, nullptr, s);
    return fast ? launch_fast<8>(p, d_packed, n_dumps, d_planes, s, blocks_per_sm)
                : launch<8, kOutF16>(p, d_packed, n_dumps, d_planes, nullptr, s);
}

cudaError_t launch_unpack_e4m3(const Plan& p, const void* d_packed, int n_dumps, void* d_planes, cudaStream_t s,
                               int blocks_per_sm) {
    if (!tc_planes_e4m3(p) || (reinterpret_cast<uintptr_t>(d_packed) & 15u) || (reinterpret_cast<uintptr_t>(d_planes) & 15u))
        return cudaErrorInvalidValue;
    return launch_fast_e4m3(p, d_packed, n_dumps, d_planes, tc_kp_e4m3(p), s, blocks_per_sm);
}

cudaError_t launch_unpack_f32(const Plan& p, const void* d_packed, int n_dumps, void* d_planes, cudaStream_t s) {
    return launch<32, kOutF32>(p, d_packed, n_dumps, d_planes, nullptr, s);
}

cudaError_t launch_unpack_bf16x2(const Plan& p, const void* d_packed, int n_dumps, void* d_hi, void* d_lo,
                                 cudaStream_t s) {
    return launch<32, kOutBF16Split>(p, d_packed, n_dumps, d_hi, d_lo, s);
}

}  // namespace corr

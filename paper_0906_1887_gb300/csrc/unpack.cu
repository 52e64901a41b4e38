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
// padded inputs and samples are zero.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "corr_internal.h"

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

cudaError_t launch_unpack_fp16(const Plan& p, const void* d_packed, int n_dumps, void* d_planes, cudaStream_t s) {
    if (p.sample_bits == 4) return launch<4, kOutF16>(p, d_packed, n_dumps, d_planes, nullptr, s);
    return launch<8, kOutF16>(p, d_packed, n_dumps, d_planes, nullptr, s);
}

cudaError_t launch_unpack_f32(const Plan& p, const void* d_packed, int n_dumps, void* d_planes, cudaStream_t s) {
    return launch<32, kOutF32>(p, d_packed, n_dumps, d_planes, nullptr, s);
}

cudaError_t launch_unpack_bf16x2(const Plan& p, const void* d_packed, int n_dumps, void* d_hi, void* d_lo,
                                 cudaStream_t s) {
    return launch<32, kOutBF16Split>(p, d_packed, n_dumps, d_hi, d_lo, s);
}

}  // namespace corr

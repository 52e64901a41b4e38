// CUDA-core FP32 X stage: the plain form of the cross-multiply-accumulate.
//
// The paper's group-parallel design (Sec. 4) shares input samples between threads
// through shared memory so each global read feeds several products, with consecutive
// threads on consecutive data so every access is coalesced, and accumulates over a
// large batch in registers (Sec. 4, last paragraphs).  The same ideas, sized for an
// sm_103a SM: a block owns a 64 x 64 tile of input pairs of one channel, stages 32
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

}  // namespace corr

// Tensor-core X stage on sm_103a: tcgen05 MMA with accumulators in tensor memory.
//
// For one channel the correlation matrix is the outer product of the sample vector with
// its conjugate, summed over time (Sec. 4, Fig. 2) -- a Hermitian rank-k update, i.e. a
// dense contraction over the time axis.  Write X_r, X_i for the real and imaginary
// sample matrices (inputs x time).  A 64-input block I is stacked as A = [X_r,I ; X_i,I]
// (128 rows), a 64-input block J gives B_r = X_r,J and B_i = X_i,J, and two MMAs per
// K-step accumulate
//     D1 = A B_r^T = [ Xr_I Xr_J^T ; Xi_I Xr_J^T ]     D2 = A B_i^T = [ Xr_I Xi_J^T ; Xi_I Xi_J^T ]
// so that, for i in I and j in J,
//     Re V_ij = D1[re row i][j] + D2[im row i][j]      Im V_ij = D1[im row i][j] - D2[re row i][j]
// which is x_i conj(x_j) summed over time (Sec. 2).  Only blocks with I <= J (the
// upper triangle of input pairs) are scheduled.
//
// Exactness for integer samples: 4/8-bit values are exact in fp16, their products
// (|p| <= 2^14) are exact, and each D element sums one product per sample, so a chunk
// of at most 1024 samples keeps every partial sum at or below 2^24 in magnitude, where
// fp32 holds every integer.  Chunks are flushed to int64; results are bit-exact.
//
// Float samples (BF16x3): x = h + l with bf16 h, l; each MMA pair runs for h*h^T,
// h*l^T and l*h^T with fp32 accumulation.
//
// CTA roles (one CTA per SM, persistent over work items = (dump, channel, I, J)):
//   warp 0      TMA producer: 128-row x 64-sample fp16 tiles into a 4-stage ring
//   warp 1      tensor-memory allocator and single-thread MMA issuer
//   warps 2..5  epilogue: tensor memory -> registers -> combine -> int64 -> global,
//               written in baseline order with coalesced 16-byte stores
// Tensor memory holds two accumulator sets (D1, D2: 64 columns each) so the epilogue of
// one item overlaps the MMAs of the next.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "corr_internal.h"
#include "tc_ptx.cuh"

namespace corr {
namespace {

constexpr int kThreads = 192;
constexpr int kTileBytes = kBlockRows * kTimeBlock * 2;     // 16 KB: 128 rows x 64 fp16
constexpr int kStagingStride = kBlockInputs + 1;            // 16-byte entries per staging row
constexpr int kStagingBytes = kBlockInputs * kStagingStride * 16;
constexpr uint32_t kTmemCols = 256;                         // 2 buffers x (D1 64 + D2 64)
constexpr uint64_t kWaitLimitNs = 2000000000ull;            // 2 s per wait

template <bool SPLIT>
struct Cfg {
    static constexpr int kStages = SPLIT ? 2 : 4;
    static constexpr int kTilesPerStage = SPLIT ? 4 : 2;     // A, B (+ A_lo, B_lo)
    static constexpr int kStageBytes = kTilesPerStage * kTileBytes;
    static constexpr int kRingBytes = kStages * kStageBytes;
    static constexpr int kBarOffset = kRingBytes + kStagingBytes;
    static constexpr int kSmemBytes = kBarOffset + 256 + 1024;  // barriers + alignment slack
};

struct TcParams {
    int n_inputs;
    int n_chan;
    int nb;
    int kp;
    int n_tiles;
    int64_t n_items;
    int chunk_kb;       // k-blocks (64 samples) per exactly-flushed chunk
    int accumulate;
    void* vis;
    int* status;
};

__device__ __forceinline__ void tile_coords(int tile, int nb, int& I, int& J) {
    int i = 0, rem = tile;
    while (rem >= nb - i) {
        rem -= nb - i;
        ++i;
    }
    I = i;
    J = i + rem;
}

__device__ __forceinline__ void record_error(int* status, volatile int* abort, int code, int detail) {
    *abort = 1;
    if (atomicCAS(status, 0, code) == 0) status[1] = detail;
}

template <bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    xeng_tc_kernel(const __grid_constant__ CUtensorMap tmap_hi, const __grid_constant__ CUtensorMap tmap_lo,
                   const TcParams prm) {
    using C = Cfg<SPLIT>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* ring = smem;
    uint8_t* staging = smem + C::kRingBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::kBarOffset);
    // bars: full[S], empty[S], acc_full[2], acc_empty[2], drain
    const uint32_t bar_full = ptx::smem_u32(bars);
    const uint32_t bar_empty = bar_full + 8 * C::kStages;
    const uint32_t bar_acc_full = bar_empty + 8 * C::kStages;
    const uint32_t bar_acc_empty = bar_acc_full + 16;
    const uint32_t bar_drain = bar_acc_empty + 16;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::kStages + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            ptx::mbar_init(bar_full + 8 * s, 1);
            ptx::mbar_init(bar_empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(bar_acc_full + 8 * b, 1);
            ptx::mbar_init(bar_acc_empty + 8 * b, 4);
        }
        ptx::mbar_init(bar_drain, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
        ptx::prefetch_tensormap(&tmap_hi);
        if (SPLIT) ptx::prefetch_tensormap(&tmap_lo);
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(tmem_slot), kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int nkb = prm.kp / kTimeBlock;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued_parity[4] = {0, 0, 0, 0};
            bool issued[4] = {false, false, false, false};
            bool ok = true;
            for (int64_t item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
                const int tile = (int)(item % prm.n_tiles);
                const int64_t dc = item / prm.n_tiles;
                int I, J;
                tile_coords(tile, prm.nb, I, J);
                const int rowA = (int)((dc * prm.nb + I) * kBlockRows);
                const int rowB = (int)((dc * prm.nb + J) * kBlockRows);
                const bool same = (I == J);
                const uint32_t bytes = (same ? 1u : 2u) * (SPLIT ? 2u : 1u) * (uint32_t)kTileBytes;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!ptx::mbar_wait_bounded(bar_empty + 8 * s, ph ^ 1u, abort_flag, kWaitLimitNs)) {
                        record_error(prm.status, abort_flag, kDevTimeoutEmpty, kb);
                        ok = false;
                        break;
                    }
                    const uint32_t fb = bar_full + 8 * s;
                    const uint32_t st = ptx::smem_u32(ring + s * C::kStageBytes);
                    ptx::mbar_expect_tx(fb, bytes);
                    ptx::tma_load_2d(st, &tmap_hi, kb * kTimeBlock, rowA, fb);
                    if (!same) ptx::tma_load_2d(st + kTileBytes, &tmap_hi, kb * kTimeBlock, rowB, fb);
                    if (SPLIT) {
                        ptx::tma_load_2d(st + 2 * kTileBytes, &tmap_lo, kb * kTimeBlock, rowA, fb);
                        if (!same) ptx::tma_load_2d(st + 3 * kTileBytes, &tmap_lo, kb * kTimeBlock, rowB, fb);
                    }
                    issued[s] = true;
                    issued_parity[s] = ph;
                    if (++s == C::kStages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            // make sure no copy of ours is still landing in shared memory when the CTA exits
            for (int k = 0; k < C::kStages; ++k)
                if (issued[k]) ptx::mbar_wait_bounded(bar_full + 8 * k, issued_parity[k], abort_flag, kWaitLimitNs);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_f16(128, 64, SPLIT);
            int s = 0;
            uint32_t ph = 0;
            int abuf = 0;
            uint32_t aph = 0;
            bool ok = true;
            bool any = false;
            for (int64_t item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
                const int tile = (int)(item % prm.n_tiles);
                int I, J;
                tile_coords(tile, prm.nb, I, J);
                const bool same = (I == J);
                for (int kb0 = 0; ok && kb0 < nkb; kb0 += prm.chunk_kb) {
                    const int kb1 = min(nkb, kb0 + prm.chunk_kb);
                    if (!ptx::mbar_wait_bounded(bar_acc_empty + 8 * abuf, aph ^ 1u, abort_flag, kWaitLimitNs)) {
                        record_error(prm.status, abort_flag, kDevTimeoutAccEmpty, kb0);
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t d1 = tmem_base + (uint32_t)(abuf * 128);
                    const uint32_t d2 = d1 + 64;
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!ptx::mbar_wait_bounded(bar_full + 8 * s, ph, abort_flag, kWaitLimitNs)) {
                            record_error(prm.status, abort_flag, kDevTimeoutFull, kb);
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t a_hi = ptx::smem_u32(ring + s * C::kStageBytes);
                        const uint32_t b_hi = same ? a_hi : a_hi + kTileBytes;
                        const uint32_t a_lo = a_hi + 2 * kTileBytes;
                        const uint32_t b_lo = same ? a_lo : a_lo + kTileBytes;
#pragma unroll
                        for (int k = 0; k < kTimeBlock / 16; ++k) {
                            const uint32_t acc = (kb > kb0 || k > 0) ? 1u : 0u;
                            const uint32_t ko = 32u * k;  // 16 fp16 = 32 bytes along the swizzled row
                            const uint64_t da = ptx::sw128_kmajor_desc(a_hi + ko);
                            const uint64_t dbr = ptx::sw128_kmajor_desc(b_hi + ko);
                            const uint64_t dbi = ptx::sw128_kmajor_desc(b_hi + 8192 + ko);
                            ptx::mma_f16(d1, da, dbr, idesc, acc);
                            ptx::mma_f16(d2, da, dbi, idesc, acc);
                            if (SPLIT) {
                                const uint64_t dal = ptx::sw128_kmajor_desc(a_lo + ko);
                                const uint64_t dblr = ptx::sw128_kmajor_desc(b_lo + ko);
                                const uint64_t dbli = ptx::sw128_kmajor_desc(b_lo + 8192 + ko);
                                ptx::mma_f16(d1, da, dblr, idesc, 1u);   // h_i l_j
                                ptx::mma_f16(d2, da, dbli, idesc, 1u);
                                ptx::mma_f16(d1, dal, dbr, idesc, 1u);   // l_i h_j
                                ptx::mma_f16(d2, dal, dbi, idesc, 1u);
                            }
                        }
                        any = true;
                        ptx::mma_commit(bar_empty + 8 * s);
                        if (++s == C::kStages) {
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
                ptx::mbar_wait_bounded(bar_drain, 0, abort_flag, kWaitLimitNs);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int q = warp & 3;                  // tensor-memory lane quadrant of this warp
        const int ew = warp - 2;                 // 0..3 within the epilogue group
        const bool re_rows = q < 2;              // lanes 0..63 hold the real-part rows of A
        const int i_loc = (q & 1) * 32 + lane;   // input within block I
        const int64_t P = (int64_t)prm.n_inputs * (prm.n_inputs + 1) / 2;
        int abuf = 0;
        uint32_t aph = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; ok && item < prm.n_items; item += gridDim.x) {
            const int tile = (int)(item % prm.n_tiles);
            const int64_t dc = item / prm.n_tiles;
            int I, J;
            tile_coords(tile, prm.nb, I, J);
            for (int kb0 = 0; kb0 < nkb; kb0 += prm.chunk_kb) {
                bool got = ptx::mbar_wait_bounded(bar_acc_full + 8 * abuf, aph, abort_flag, kWaitLimitNs);
                if (!got) record_error(prm.status, abort_flag, kDevTimeoutAccFull, kb0);
                ptx::named_bar_sync(1, 128);
                if (*abort_flag) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(abuf * 128);
                // two passes: real-part rows write, then imaginary-part rows add
                for (int pass = 0; pass < 2; ++pass) {
                    if ((pass == 0) == re_rows) {
#pragma unroll 1
                        for (int m = 0; m < 2; ++m) {
                            uint32_t v1[32], v2[32];
                            ptx::tmem_ld32(tbase + 32u * m, v1);
                            ptx::tmem_ld32(tbase + 64u + 32u * m, v2);
                            ptx::tmem_wait_ld();
                            uint8_t* rowp = staging + (size_t)i_loc * kStagingStride * 16;
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const float f1 = __uint_as_float(v1[e]);
                                const float f2 = __uint_as_float(v2[e]);
                                const int jl = 32 * m + e;
                                if constexpr (!SPLIT) {
                                    longlong2* p = reinterpret_cast<longlong2*>(rowp) + jl;
                                    if (re_rows) {
                                        *p = make_longlong2(__float2ll_rn(f1), -__float2ll_rn(f2));
                                    } else {
                                        longlong2 o = *p;
                                        o.x += __float2ll_rn(f2);
                                        o.y += __float2ll_rn(f1);
                                        *p = o;
                                    }
                                } else {
                                    float2* p = reinterpret_cast<float2*>(rowp + 16 * jl);
                                    if (re_rows) {
                                        *p = make_float2(f1, -f2);
                                    } else {
                                        float2 o = *p;
                                        o.x += f2;
                                        o.y += f1;
                                        *p = o;
                                    }
                                }
                            }
                        }
                    }
                    ptx::named_bar_sync(1, 128);
                }
                // accumulator drained: hand the tensor-memory buffer back to the MMA warp
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(bar_acc_empty + 8 * abuf);
                if (++abuf == 2) {
                    abuf = 0;
                    aph ^= 1u;
                }
                // write the tile's valid baselines: row i, columns j in [max(J0, i), min(J0 + 64, N))
                const bool add = prm.accumulate || kb0 > 0;
                for (int r = ew; r < kBlockInputs; r += 4) {
                    const int i = I * kBlockInputs + r;
                    if (i >= prm.n_inputs) break;
                    const int j_lo = max(J * kBlockInputs, i);
                    const int j_hi = min(J * kBlockInputs + kBlockInputs, prm.n_inputs);
                    if (j_lo >= j_hi) continue;
                    const int64_t b0 = (int64_t)i * prm.n_inputs - (int64_t)i * (i - 1) / 2 + (j_lo - i);
                    const int64_t o0 = dc * P + b0;
                    const uint8_t* rowp = staging + (size_t)r * kStagingStride * 16;
                    for (int j = j_lo + lane; j < j_hi; j += 32) {
                        const int jl = j - J * kBlockInputs;
                        if constexpr (!SPLIT) {
                            longlong2 v = *reinterpret_cast<const longlong2*>(rowp + 16 * jl);
                            longlong2* dst = reinterpret_cast<longlong2*>(prm.vis) + o0 + (j - j_lo);
                            if (add) {
                                longlong2 old = *dst;
                                v.x += old.x;
                                v.y += old.y;
                            }
                            *dst = v;
                        } else {
                            float2 v = *reinterpret_cast<const float2*>(rowp + 16 * jl);
                            float2* dst = reinterpret_cast<float2*>(prm.vis) + o0 + (j - j_lo);
                            if (add) {
                                float2 old = *dst;
                                v.x += old.x;
                                v.y += old.y;
                            }
                            *dst = v;
                        }
                    }
                }
                ptx::named_bar_sync(1, 128);  // staging free for the next accumulator
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 1) ptx::tmem_dealloc(tmem_base, kTmemCols);
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

// 2-D map over plane rows: dim0 = Kp samples (fp16/bf16), dim1 = all 128-row blocks.
bool make_plane_map(CUtensorMap* map, const void* base, int kp, int64_t rows, CUtensorMapDataType dt) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTimeBlock, (cuuint32_t)kBlockRows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <bool SPLIT>
cudaError_t launch_impl(const Plan& p, const void* hi, const void* lo, int n_dumps, void* vis, int accumulate,
                        cudaStream_t s) {
    using C = Cfg<SPLIT>;
    const int64_t rows = (int64_t)n_dumps * p.n_chan * p.nb * kBlockRows;
    if (rows >= (int64_t)1 << 31) return cudaErrorInvalidValue;   // TMA row coordinates are int32
    CUtensorMap mh, ml;
    const CUtensorMapDataType dt = SPLIT ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    if (!make_plane_map(&mh, hi, p.kp, rows, dt)) return cudaErrorInvalidValue;
    if (SPLIT) {
        if (!make_plane_map(&ml, lo, p.kp, rows, dt)) return cudaErrorInvalidValue;
    } else {
        ml = mh;
    }
    TcParams prm;
    prm.n_inputs = p.n_inputs;
    prm.n_chan = p.n_chan;
    prm.nb = p.nb;
    prm.kp = p.kp;
    prm.n_tiles = p.nb * (p.nb + 1) / 2;
    prm.n_items = (int64_t)n_dumps * p.n_chan * prm.n_tiles;
    // samples per exact chunk: 8-bit 1024 (|sum| <= 1024 * 2^14 = 2^24), 4-bit 131072, float: all
    prm.chunk_kb = SPLIT ? (p.kp / kTimeBlock) : (p.sample_bits == 4 ? 2048 : 16);
    prm.accumulate = accumulate;
    prm.vis = vis;
    prm.status = p.d_status;
    cudaError_t e = cudaFuncSetAttribute(xeng_tc_kernel<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::kSmemBytes);
    if (e != cudaSuccess) return e;
    const int grid = (int)(prm.n_items < p.n_sm ? prm.n_items : p.n_sm);
    xeng_tc_kernel<SPLIT><<<grid, kThreads, C::kSmemBytes, s>>>(mh, ml, prm);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_xeng_tc(const Plan& p, const void* d_planes, const void* d_planes_lo, int n_dumps, void* d_vis,
                           int accumulate, cudaStream_t s) {
    if (d_planes_lo) return launch_impl<true>(p, d_planes, d_planes_lo, n_dumps, d_vis, accumulate, s);
    return launch_impl<false>(p, d_planes, nullptr, n_dumps, d_vis, accumulate, s);
}

}  // namespace corr

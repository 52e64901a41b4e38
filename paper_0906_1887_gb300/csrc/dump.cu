// Dump step (Fig. 1) with post-correlation phase correction (Sec. 2).
//
// At the end of a dump interval the accumulators are read, divided by the number of times
// they were updated and reset (Fig. 1).  The MWA corrects the geometric delay after
// correlation, as a phase (Sec. 2): a delay tau_i multiplies input i's spectrum by
// exp(-2 pi i nu tau_i), so baseline (i, j) carries exp(-2 pi i nu_c (tau_i - tau_j)), which
// the correction removes:
//
//     V'_ij(c) = V_ij(c) / n_accum * g_i(c) conj(g_j(c)),   g_n(c) = exp(+2 pi i nu_c tau_n)
//
// The per-input phasors g_n(c) are formed once per call in double precision (sincospi of
// 2 nu tau, whose argument reduction keeps large phases accurate) and rounded to float; the
// per-baseline work is two complex products in float32 -- the kernel is a stream over the
// accumulators (16 bytes read, 8 written, 16 more written when resetting).
#include <algorithm>
#include <type_traits>

#include "corr_internal.h"

namespace corr {
namespace {

constexpr int kDumpThreads = 256;

__global__ void phasor_kernel(const double* __restrict__ tau, const double* __restrict__ nu, int N, int C,
                              float2* __restrict__ g) {
    const int64_t total = (int64_t)N * C;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / N), n = (int)(idx - (int64_t)c * N);
        double s, co;
        sincospi(2.0 * nu[c] * tau[n], &s, &co);
        g[idx] = make_float2((float)co, (float)s);
    }
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulf_conj(float2 a, float2 b) {   // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Each block takes the baseline rows i and N - 1 - i (i < N / 2, or the middle row alone when
// N is odd) of the channels c = blockIdx.y + m gridDim.y: N - i + i + 1 = N + 1 elements per
// channel for every block, so the blocks are equal, and an element's (i, j) follows from its
// position in the pair without any search.  Row i starts at off(i) = i N - i (i - 1) / 2
// within a channel.  The block's (channel, element) pairs are numbered flat, so each thread
// issues kU loads before it computes whatever N is (the host keeps the flat count < 2^31).
constexpr int kU = 4;

template <typename AccT>
__global__ void __launch_bounds__(kDumpThreads) dump_kernel(AccT* __restrict__ acc, const float2* __restrict__ g,
                                                            int N, int64_t P, int C, float inv_n,
                                                            float2* __restrict__ out, int reset) {
    using Pair = std::conditional_t<sizeof(AccT) == 8, longlong2, float2>;
    const int i0 = blockIdx.x, i1 = N - 1 - i0;
    const int len0 = N - i0;                        // elements of row i0
    const int len = i1 == i0 ? len0 : N + 1;        // elements of the pair
    const int64_t off0 = (int64_t)i0 * N - (int64_t)i0 * (i0 - 1) / 2;
    const int64_t off1 = (int64_t)i1 * N - (int64_t)i1 * (i1 - 1) / 2;
    const int nch = (C - (int)blockIdx.y + (int)gridDim.y - 1) / (int)gridDim.y;   // channels of this block
    const uint32_t total = (uint32_t)nch * (uint32_t)len;
    Pair* const a = reinterpret_cast<Pair*>(acc);
    for (uint32_t f0 = 0; f0 < total; f0 += kDumpThreads * kU) {
        Pair v[kU];
        int64_t at[kU];   // element index in the [C][P] arrays, -1 past the end
        int ci[kU], ej[kU];
        // (channel step m, element e) of the thread's first element by one division, the
        // others by adding the block size and wrapping
        const uint32_t fl0 = f0 + threadIdx.x;
        uint32_t m = fl0 / (uint32_t)len;
        int e = (int)(fl0 - m * (uint32_t)len);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (u > 0) {
                e += kDumpThreads;
                while (e >= len) {
                    e -= len;
                    ++m;
                }
            }
            at[u] = -1;
            if (f0 + (uint32_t)(u * kDumpThreads) + threadIdx.x < total) {
                const int c = (int)blockIdx.y + (int)m * (int)gridDim.y;
                at[u] = (int64_t)c * P + (e < len0 ? off0 + e : off1 + (e - len0));
                ci[u] = c;
                ej[u] = e;
                v[u] = a[at[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (at[u] < 0) continue;
            float2 w = make_float2((float)v[u].x * inv_n, (float)v[u].y * inv_n);
            if (g) {
                const bool first = ej[u] < len0;
                const int i = first ? i0 : i1;
                const int j = first ? i0 + ej[u] : i1 + (ej[u] - len0);
                const float2* gc = g + (size_t)ci[u] * N;
                w = cmulf_conj(cmulf(w, gc[i]), gc[j]);
            }
            out[at[u]] = w;
            if (reset) {
                Pair z;
                z.x = 0;
                z.y = 0;
                a[at[u]] = z;
            }
        }
    }
}

}  // namespace

cudaError_t launch_phasors(const Plan& p, const double* d_delays, const double* d_freqs, void* d_g, cudaStream_t s) {
    const int64_t total = (int64_t)p.n_inputs * p.n_chan;
    const int64_t want = (total + kDumpThreads - 1) / kDumpThreads;
    const int blocks = (int)(want < 4096 ? want : 4096);
    phasor_kernel<<<blocks, kDumpThreads, 0, s>>>(d_delays, d_freqs, p.n_inputs, p.n_chan, static_cast<float2*>(d_g));
    return cudaGetLastError();
}

}  // namespace corr

using namespace corr;

extern "C" {

corr_status corr_dump_workspace_size(corr_plan plan, size_t* bytes) {
    if (!plan || !bytes) return set_error(CORR_EINVAL, "corr_dump_workspace_size: NULL argument");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    *bytes = (size_t)p->n_chan * p->n_inputs * sizeof(float2);
    return CORR_OK;
}

corr_status corr_dump(corr_plan plan, void* d_acc, int n_accum, const double* d_delays, const double* d_freqs,
                      void* d_workspace, void* d_out, int reset, void* stream) {
    if (!plan || !d_acc || !d_out) return set_error(CORR_EINVAL, "corr_dump: NULL argument");
    if (n_accum < 1) return set_error(CORR_EINVAL, "n_accum=%d must be >= 1", n_accum);
    if (d_delays && (!d_freqs || !d_workspace))
        return set_error(CORR_EINVAL, "corr_dump: delays need channel frequencies and the phasor workspace");
    if ((reinterpret_cast<uintptr_t>(d_acc) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 7u))
        return set_error(CORR_EINVAL, "corr_dump: accumulators must be 16-byte and output 8-byte aligned");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float2* g = nullptr;
    if (d_delays) {
        g = static_cast<float2*>(d_workspace);
        const cudaError_t e = launch_phasors(*p, d_delays, d_freqs, g, s);
        if (e != cudaSuccess) return cuda_error(e, "phasor launch");
    }
    const int64_t P = p->n_baselines;
    // row pairs x channel groups: a few waves of blocks, each block looping over channels
    const int pairs = (p->n_inputs + 1) / 2;
    const int64_t want_y = ((int64_t)(p->n_sm > 0 ? p->n_sm : 148) * 64 + pairs - 1) / pairs;
    int gy = (int)std::min<int64_t>(std::min<int64_t>(want_y, p->n_chan), 65535);
    if (gy < 1) gy = 1;
    // each block numbers its (channel, element) pairs in 32 bits
    const int64_t per_block = ((int64_t)p->n_chan + gy - 1) / gy * (int64_t)(p->n_inputs + 1);
    if (per_block >= (int64_t{1} << 31)) {
        gy = (int)std::min<int64_t>(65535, std::min<int64_t>(
                 p->n_chan, ((int64_t)p->n_chan * (p->n_inputs + 1) + (int64_t{1} << 30) - 1) >> 30));
        if (((int64_t)p->n_chan + gy - 1) / gy * (int64_t)(p->n_inputs + 1) >= (int64_t{1} << 31))
            return set_error(CORR_EUNSUPPORTED, "corr_dump: %d channels x %d inputs is too large for one call",
                             p->n_chan, p->n_inputs);
    }
    const dim3 grid((unsigned)pairs, (unsigned)gy);
    const float inv_n = 1.0f / (float)n_accum;
    if (p->sample_bits == 32)
        dump_kernel<float><<<grid, kDumpThreads, 0, s>>>(static_cast<float*>(d_acc), g, p->n_inputs, P, p->n_chan,
                                                          inv_n, static_cast<float2*>(d_out), reset);
    else
        dump_kernel<long long><<<grid, kDumpThreads, 0, s>>>(static_cast<long long*>(d_acc), g, p->n_inputs, P,
                                                              p->n_chan, inv_n, static_cast<float2*>(d_out), reset);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "dump launch");
    return CORR_OK;
}

corr_status corr_xengine_run_dump(corr_plan plan, const void* d_packed, int n_dumps, void* d_out, int n_accum,
                                  const double* d_delays, const double* d_freqs, void* d_workspace, void* stream) {
    if (!plan || !d_packed || !d_out) return set_error(CORR_EINVAL, "corr_xengine_run_dump: NULL argument");
    if (n_dumps < 1) return set_error(CORR_EINVAL, "n_dumps=%d must be >= 1", n_dumps);
    if (n_accum < 1) return set_error(CORR_EINVAL, "n_accum=%d must be >= 1", n_accum);
    if (d_delays && (!d_freqs || !d_workspace))
        return set_error(CORR_EINVAL, "corr_xengine_run_dump: delays need channel frequencies and the phasor workspace");
    if (reinterpret_cast<uintptr_t>(d_out) & 7u) return set_error(CORR_EINVAL, "corr_xengine_run_dump: output not 8-byte aligned");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (!tc_raw_supported(*p))
        return set_error(CORR_EUNSUPPORTED, "the fused dump runs the packed-sample tensor-core path (4/8-bit samples, "
                                            "packed rows a multiple of 16 bytes)");
    const int64_t chunk = p->sample_bits == 8 ? 1024 : 131072;
    if (p->kp > chunk)
        return set_error(CORR_EUNSUPPORTED, "the fused dump needs a dump of at most %lld samples (one exact chunk)",
                         (long long)chunk);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const void* g = nullptr;
    if (d_delays) {
        const cudaError_t e = launch_phasors(*p, d_delays, d_freqs, d_workspace, s);
        if (e != cudaSuccess) return cuda_error(e, "phasor launch");
        g = d_workspace;
    }
    const cudaError_t e = launch_xeng_tc_raw_dump(*p, d_packed, n_dumps, d_out, g, 1.0f / (float)n_accum, s);
    if (e != cudaSuccess) return cuda_error(e, "fused dump launch");
    return CORR_OK;
}

}  // extern "C"

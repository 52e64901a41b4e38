// F stage of the FX correlator (Sec. 2, Sec. 4): unpack + per-input DFT of time blocks.
//
// The paper's GPU correlator unpacks a batch of time samples (input index fastest), reorders
// it into per-input blocks and Fourier transforms each block into spectral channels: an
// N_C-point complex transform for complex samples, and for real samples a 2 N_C-point
// complex-to-complex transform of which channels 0 .. N_C are kept (Sec. 4).  Here one
// kernel does both steps for a block of G inputs and one frame of L samples:
//
//   load    packed samples [t][input] -> float2 rows in shared memory, one row per input
//           (coalesced along the inputs; rows padded to L + 1 so column reads do not
//           collide in banks)
//   FFT     Stockham autosort stages of radix 16 (the last one of radix 8, 4 or 2 when
//           log2 L is not a multiple of 4), ping-ponging between two shared buffers: each
//           task loads R values, applies the stage twiddles (a table exp(-2 pi i k / L)
//           computed on the host in double precision) and does the R-point DFT in registers
//           (radix-2 butterflies with exact constant twiddles of the 16th roots of unity).
//           L = 128, the paper's channel count, takes two stages (16 x 8).  Rows are padded
//           one element per 16 so the strided stores of the first stage, and the column
//           reads of the load and store phases, fall in distinct banks
//   store   spectra [frame][channel][input] complex float32, coalesced along the inputs --
//           exactly the float sample layout the X stage takes ([T][C][N], T = frames)
//
// A Stockham stage with sub-transform length Ns and radix R takes, for each j < L / R, the R
// values v_r = x[j + r L / R], multiplies v_r by exp(-2 pi i (j mod Ns) r / (Ns R)), applies
// the R-point DFT and writes output q to position (j - j mod Ns) R + j mod Ns + q Ns.  After
// log_R L stages the result is in natural order.  The DFT is the forward, unnormalised one,
// X_k = sum_s x_s exp(-2 pi i k s / L); channel c is bin c.
#include <cmath>
#include <new>
#include <vector>

#include "corr_internal.h"

namespace corr {
namespace {

constexpr int kFPoints = 4096;   // complex points per CTA (inputs x transform length)
constexpr int kFThreads = 256;
constexpr int kFMinLen = 8, kFMaxLen = 4096;

struct FPlan {
    int n_inputs = 0;
    int n_chan = 0;
    int kind = 0;        // CORR_F_COMPLEX8 / CORR_F_COMPLEX4 / CORR_F_REAL8
    int L = 0;           // transform length: N_C, or 2 N_C for real samples
    int n_out = 0;       // channels produced: N_C, or N_C + 1
    int G = 0;           // inputs per CTA
    int log2L = 0, log2G = 0;
    int device = 0;
    int n_sm = 0;
    float2* d_tw = nullptr;   // exp(-2 pi i k / L), k < L
    int n_taps = 1;           // PFB taps M (input frames per output frame)
    float* d_taps = nullptr;  // PFB prototype, M L values; nullptr: plain transform
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// position of row element i: one pad element after every 16
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

// x * exp(-2 pi i a / 16) for a compile-time a in 0..7 (the roots a DFT of size <= 16 uses);
// the constants are cos and sin of multiples of pi / 8, correctly rounded to float
template <int A>
__device__ __forceinline__ float2 rot16(float2 x) {
    constexpr float kC1 = 0.92387953251128676f;   // cos(pi / 8)
    constexpr float kS1 = 0.38268343236508977f;   // sin(pi / 8)
    constexpr float kH = 0.70710678118654752f;    // cos(pi / 4)
    if constexpr (A == 0) return x;
    else if constexpr (A == 4) return make_float2(x.y, -x.x);
    else if constexpr (A == 2) return make_float2(kH * (x.x + x.y), kH * (x.y - x.x));
    else if constexpr (A == 6) return make_float2(kH * (x.y - x.x), -kH * (x.x + x.y));
    else if constexpr (A == 1) return cmul(x, make_float2(kC1, -kS1));
    else if constexpr (A == 3) return cmul(x, make_float2(kS1, -kC1));
    else if constexpr (A == 5) return cmul(x, make_float2(-kS1, -kC1));
    else return cmul(x, make_float2(-kC1, -kS1));
}

template <int M>
__host__ __device__ constexpr int bit_reverse(int r) {
    int o = 0;
    for (int b = 0; b < M; ++b) o |= ((r >> b) & 1) << (M - 1 - b);
    return o;
}

// one radix-2 butterfly level of an in-register DIT DFT: groups of SIZE, element j of a group
// combined with j + SIZE / 2 after a rotation by exp(-2 pi i j / SIZE)
template <int R, int SIZE, int J>
__device__ __forceinline__ void dit_level(float2 (&x)[R], int k0) {
    if constexpr (J < SIZE / 2) {
        const float2 u = x[k0 + J];
        const float2 t = rot16<J * (16 / SIZE)>(x[k0 + J + SIZE / 2]);
        x[k0 + J] = cadd(u, t);
        x[k0 + J + SIZE / 2] = csub(u, t);
        dit_level<R, SIZE, J + 1>(x, k0);
    }
}

template <int R, int SIZE>
__device__ __forceinline__ void dit_levels(float2 (&x)[R]) {
    if constexpr (SIZE <= R) {
#pragma unroll
        for (int k0 = 0; k0 < R; k0 += SIZE) dit_level<R, SIZE, 0>(x, k0);
        dit_levels<R, SIZE * 2>(x);
    }
}

// forward R-point DFT in registers (R = 2, 4, 8, 16): y_q = sum_r v_r exp(-2 pi i r q / R)
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
    constexpr int M = R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[bit_reverse<M>(r)] = v[r];
    dit_levels<R, 2>(x);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[r];
}

// one Stockham stage of radix R over the G rows of `a` into `b`
template <int R>
__device__ __forceinline__ void stockham_stage(const float2* a, float2* b, const float2* twl, int pitch, int G,
                                               int log2LR, int Ns, int tshift) {
    const int LR = 1 << log2LR;
    for (int task = threadIdx.x; task < LR * G; task += kFThreads) {
        const int g = task >> log2LR, j = task & (LR - 1);
        const float2* src = a + g * pitch;
        float2* dst = b + g * pitch;
        const int k = j & (Ns - 1);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[pad(j + r * LR)];
        if (k) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twl[(r * k) << tshift]);
        }
        dft_reg<R>(v);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[pad(d + q * Ns)] = v[q];
    }
}

// raw packed sample: 2 bytes for complex 8-bit, 1 byte otherwise
template <int KIND>
__device__ __forceinline__ uint32_t load_raw(const uint8_t* __restrict__ in, size_t idx) {
    if constexpr (KIND == CORR_F_COMPLEX8) return reinterpret_cast<const unsigned short*>(in)[idx];
    else return in[idx];
}

// the samples thread `tid` moves of one frame: element idx = tid + q x threads is sample
// s = idx >> log2G of input n0 + (idx & (G - 1)); zero outside the array
template <int KIND, int PER>
__device__ __forceinline__ void fetch_frame(uint32_t (&raw)[PER], const uint8_t* __restrict__ in, size_t row0, int N,
                                            int n0, int g_n, int log2G, int pts) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int idx = threadIdx.x + q * kFThreads;
        const int s = idx >> log2G, g = idx & ((1 << log2G) - 1);
        raw[q] = (idx < pts && g < g_n) ? load_raw<KIND>(in, (row0 + s) * N + n0 + g) : 0u;
    }
}

// one packed sample -> complex float (small integers: exact)
template <int KIND>
__device__ __forceinline__ float2 unpack_raw(uint32_t r) {
    if constexpr (KIND == CORR_F_COMPLEX8) {
        return make_float2((float)(signed char)(r & 0xFF), (float)(signed char)(r >> 8));
    } else if constexpr (KIND == CORR_F_COMPLEX4) {
        int re = (int)(r >> 4), im = (int)(r & 15);
        re -= (re & 8) << 1;   // two's complement nibbles
        im -= (im & 8) << 1;
        return make_float2((float)re, (float)im);
    } else {
        return make_float2((float)(signed char)r, 0.f);
    }
}

// Persistent over frames: frame f + gridDim.y's samples are fetched into registers (kPer per
// thread) while frame f is transformed, so the global loads overlap the FFT.  PFB = true is
// the polyphase filterbank (Sec. 6.1): the load phase forms y[s] = sum_m h[m L + s] x[(f + m)
// L + s] over M input frames (the extra cost the paper places in the unpack), then the same
// transform runs.
template <int KIND, bool PFB>
__global__ void __launch_bounds__(kFThreads, 3) fengine_kernel(const uint8_t* __restrict__ in, float2* __restrict__ out,
                                                            const float2* __restrict__ tw, int N, int log2L, int n_out,
                                                            int log2G, int n_frames, const float* __restrict__ taps,
                                                            int M) {
    constexpr int kPer = kFPoints / kFThreads;   // samples per thread per frame (at most)
    extern __shared__ float2 fsm[];
    const int L = 1 << log2L, G = 1 << log2G;
    const int pitch = L + (L >> 4) + 1;   // padded row: element i at pad(i)
    float2* const buf0 = fsm;
    float2* const buf1 = fsm + G * pitch;
    float2* const twl = fsm + 2 * G * pitch;
    float* const tapl = reinterpret_cast<float*>(twl + L);   // PFB: the prototype, M L values
    const int n0 = blockIdx.x * G;
    const int g_n = min(G, N - n0);
    const int pts = L * G;
    for (int k = threadIdx.x; k < L; k += blockDim.x) twl[k] = tw[k];
    if constexpr (PFB)
        for (int k = threadIdx.x; k < M * L; k += blockDim.x) tapl[k] = taps[k];

    uint32_t raw[kPer];
    int f = blockIdx.y;
    if constexpr (!PFB) {
        if (f < n_frames) fetch_frame<KIND>(raw, in, (size_t)f * L, N, n0, g_n, log2G, pts);
    }
    for (; f < n_frames; f += gridDim.y) {
        float2* a = buf0;
        float2* b = buf1;
        if constexpr (PFB) {
            // weighted overlap of input frames f .. f + M - 1 -> a[g][s]; each frame's loads are
            // issued together before its taps are applied
            float2 acc[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int m = 0; m < M; ++m) {
                fetch_frame<KIND>(raw, in, (size_t)(f + m) * L, N, n0, g_n, log2G, pts);
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const int idx = threadIdx.x + q * kFThreads;
                    if (idx < pts) {
                        const float hw = tapl[m * L + (idx >> log2G)];
                        const float2 v = unpack_raw<KIND>(raw[q]);
                        acc[q].x = fmaf(hw, v.x, acc[q].x);
                        acc[q].y = fmaf(hw, v.y, acc[q].y);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int idx = threadIdx.x + q * kFThreads;
                if (idx < pts) a[(idx & (G - 1)) * pitch + pad(idx >> log2G)] = acc[q];
            }
            __syncthreads();
        } else {
            // sample s of input n0 + g, time f L + s -> a[g][s]
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int idx = threadIdx.x + q * kFThreads;
                if (idx < pts) a[(idx & (G - 1)) * pitch + pad(idx >> log2G)] = unpack_raw<KIND>(raw[q]);
            }
            __syncthreads();
            if (f + (int)gridDim.y < n_frames)
                fetch_frame<KIND>(raw, in, (size_t)(f + gridDim.y) * L, N, n0, g_n, log2G, pts);
        }
        for (int Ns = 1, log2Ns = 0; Ns < L;) {
            const int log2R = log2L - log2Ns < 4 ? log2L - log2Ns : 4;
            const int log2LR = log2L - log2R;
            const int tshift = log2L - log2Ns - log2R;   // twiddle step L / (Ns R)
            if (log2R == 4) stockham_stage<16>(a, b, twl, pitch, G, log2LR, Ns, tshift);
            else if (log2R == 3) stockham_stage<8>(a, b, twl, pitch, G, log2LR, Ns, tshift);
            else if (log2R == 2) stockham_stage<4>(a, b, twl, pitch, G, log2LR, Ns, tshift);
            else stockham_stage<2>(a, b, twl, pitch, G, log2LR, Ns, tshift);
            __syncthreads();
            float2* t = a;
            a = b;
            b = t;
            Ns <<= log2R;
            log2Ns += log2R;
        }
        // channel c of input n0 + g -> out[f][c][n0 + g]
        float2* o = out + (size_t)f * n_out * N + n0;
        for (int idx = threadIdx.x; idx < n_out * G; idx += blockDim.x) {
            const int c = idx >> log2G, g = idx & (G - 1);
            if (g < g_n) o[(size_t)c * N + g] = a[g * pitch + pad(c)];
        }
        __syncthreads();   // the next frame reuses the buffers
    }
}

size_t fplan_smem(const FPlan& p) {
    const size_t taps = p.d_taps ? (size_t)p.n_taps * p.L * sizeof(float) : 0;
    return ((size_t)2 * p.G * (p.L + (p.L >> 4) + 1) + p.L) * sizeof(float2) + taps;
}

template <int KIND, bool PFB>
cudaError_t launch_fengine(const FPlan& p, const void* d_in, int n_frames, void* d_out, cudaStream_t s) {
    const int smem = (int)fplan_smem(p);
    cudaError_t e = cudaFuncSetAttribute(fengine_kernel<KIND, PFB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // persistent over frames: enough CTAs to fill every SM a few times over
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fengine_kernel<KIND, PFB>, kFThreads, smem);
    if (e != cudaSuccess) return e;
    const int groups = (p.n_inputs + p.G - 1) / p.G;
    int rows = (p.n_sm * (per_sm > 0 ? per_sm : 1) * 4 + groups - 1) / groups;
    if (rows > n_frames) rows = n_frames;
    if (rows > 65535) rows = 65535;
    const dim3 grid(groups, rows);
    fengine_kernel<KIND, PFB><<<grid, kFThreads, smem, s>>>(static_cast<const uint8_t*>(d_in),
                                                            static_cast<float2*>(d_out), p.d_tw, p.n_inputs, p.log2L,
                                                            p.n_out, p.log2G, n_frames, p.d_taps, p.n_taps);
    return cudaGetLastError();
}

}  // namespace
}  // namespace corr

using namespace corr;

extern "C" {

corr_status corr_fplan_create(corr_fplan* out, int n_inputs, int n_chan, int kind) {
    if (!out) return set_error(CORR_EINVAL, "corr_fplan_create: out is NULL");
    *out = nullptr;
    if (n_inputs < 1 || n_inputs > kMaxInputs)
        return set_error(CORR_EINVAL, "n_inputs=%d outside [1, %d]", n_inputs, kMaxInputs);
    if (kind != CORR_F_COMPLEX8 && kind != CORR_F_COMPLEX4 && kind != CORR_F_REAL8)
        return set_error(CORR_EINVAL, "kind=%d is not CORR_F_COMPLEX8/COMPLEX4/REAL8", kind);
    const int L = kind == CORR_F_REAL8 ? 2 * n_chan : n_chan;
    if (n_chan < 1 || L < kFMinLen || L > kFMaxLen || (L & (L - 1)))
        return set_error(CORR_EINVAL, "transform length %d (n_chan=%d) must be a power of two in [%d, %d]", L, n_chan,
                         kFMinLen, kFMaxLen);
    FPlan* p = new (std::nothrow) FPlan();
    if (!p) return set_error(CORR_ENOMEM, "corr_fplan_create: host allocation failed");
    p->n_inputs = n_inputs;
    p->n_chan = n_chan;
    p->kind = kind;
    p->L = L;
    p->n_out = kind == CORR_F_REAL8 ? n_chan + 1 : n_chan;
    p->G = kFPoints / L < 64 ? (kFPoints / L > 0 ? kFPoints / L : 1) : 64;
    while ((1 << p->log2L) < L) ++p->log2L;
    while ((1 << p->log2G) < p->G) ++p->log2G;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device);
    std::vector<float2> tw(L);
    for (int k = 0; k < L; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)L;
        tw[k] = make_float2((float)cos(ang), (float)sin(ang));
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw, (size_t)L * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw, tw.data(), (size_t)L * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (p->d_tw) cudaFree(p->d_tw);
        delete p;
        return cuda_error(e, "corr_fplan_create");
    }
    *out = reinterpret_cast<corr_fplan>(p);
    return CORR_OK;
}

corr_status corr_fplan_destroy(corr_fplan plan) {
    if (!plan) return CORR_OK;
    FPlan* p = reinterpret_cast<FPlan*>(plan);
    if (p->d_tw) cudaFree(p->d_tw);
    if (p->d_taps) cudaFree(p->d_taps);
    delete p;
    return CORR_OK;
}

corr_status corr_fplan_create_pfb(corr_fplan* out, int n_inputs, int n_chan, int kind, int n_taps, const float* h_taps) {
    if (!out) return set_error(CORR_EINVAL, "corr_fplan_create_pfb: out is NULL");
    *out = nullptr;
    if (n_taps < 1 || n_taps > 64) return set_error(CORR_EINVAL, "n_taps=%d outside [1, 64]", n_taps);
    corr_fplan h = nullptr;
    corr_status st = corr_fplan_create(&h, n_inputs, n_chan, kind);
    if (st != CORR_OK) return st;
    FPlan* p = reinterpret_cast<FPlan*>(h);
    const int ML = n_taps * p->L;
    // the prototype sits in shared memory beside the transform buffers
    const size_t smem = ((size_t)2 * p->G * (p->L + (p->L >> 4) + 1) + p->L) * sizeof(float2) + (size_t)ML * sizeof(float);
    if (smem > (size_t)227 * 1024) {
        corr_fplan_destroy(h);
        return set_error(CORR_EINVAL, "n_taps=%d x transform length %d: the prototype does not fit in shared memory",
                         n_taps, p->L);
    }
    std::vector<float> taps(ML);
    if (h_taps) {
        for (int n = 0; n < ML; ++n) taps[n] = h_taps[n];
    } else if (n_taps == 1) {
        for (int n = 0; n < ML; ++n) taps[n] = 1.0f;
    } else {
        // windowed sinc: sinc((n - (M L - 1) / 2) / L) x Hamming(n), in double, rounded to float
        for (int n = 0; n < ML; ++n) {
            const double x = ((double)n - (ML - 1) / 2.0) / (double)p->L;
            const double sinc = x == 0.0 ? 1.0 : sin(M_PI * x) / (M_PI * x);
            const double w = 0.54 - 0.46 * cos(2.0 * M_PI * (double)n / (double)(ML - 1));
            taps[n] = (float)(sinc * w);
        }
    }
    cudaError_t e = cudaMalloc(&p->d_taps, (size_t)ML * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_taps, taps.data(), (size_t)ML * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        corr_fplan_destroy(h);
        return cuda_error(e, "corr_fplan_create_pfb");
    }
    p->n_taps = n_taps;
    *out = h;
    return CORR_OK;
}

corr_status corr_fplan_taps(corr_fplan plan, int* n_taps) {
    if (!plan || !n_taps) return set_error(CORR_EINVAL, "corr_fplan_taps: NULL argument");
    *n_taps = reinterpret_cast<const FPlan*>(plan)->n_taps;
    return CORR_OK;
}

corr_status corr_fplan_info(corr_fplan plan, int* n_out_chan, int* transform_len, size_t* in_bytes_per_frame,
                            size_t* out_bytes_per_frame) {
    if (!plan) return set_error(CORR_EINVAL, "corr_fplan_info: plan is NULL");
    const FPlan* p = reinterpret_cast<const FPlan*>(plan);
    const size_t bps = p->kind == CORR_F_COMPLEX8 ? 2 : 1;
    if (n_out_chan) *n_out_chan = p->n_out;
    if (transform_len) *transform_len = p->L;
    if (in_bytes_per_frame) *in_bytes_per_frame = (size_t)p->L * p->n_inputs * bps;
    if (out_bytes_per_frame) *out_bytes_per_frame = (size_t)p->n_out * p->n_inputs * sizeof(float2);
    return CORR_OK;
}

corr_status corr_fengine_run(corr_fplan plan, const void* d_time, int n_frames, void* d_spectra, void* stream) {
    if (!plan || !d_time || !d_spectra) return set_error(CORR_EINVAL, "corr_fengine_run: NULL argument");
    if (n_frames < 1) return set_error(CORR_EINVAL, "n_frames=%d must be >= 1", n_frames);
    const FPlan* p = reinterpret_cast<const FPlan*>(plan);
    if ((reinterpret_cast<uintptr_t>(d_time) & 1u) || (reinterpret_cast<uintptr_t>(d_spectra) & 7u))
        return set_error(CORR_EINVAL, "corr_fengine_run: samples must be 2-byte and spectra 8-byte aligned");
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    const bool pfb = p->d_taps != nullptr;
    if (p->kind == CORR_F_COMPLEX8)
        e = pfb ? launch_fengine<CORR_F_COMPLEX8, true>(*p, d_time, n_frames, d_spectra, s)
                : launch_fengine<CORR_F_COMPLEX8, false>(*p, d_time, n_frames, d_spectra, s);
    else if (p->kind == CORR_F_COMPLEX4)
        e = pfb ? launch_fengine<CORR_F_COMPLEX4, true>(*p, d_time, n_frames, d_spectra, s)
                : launch_fengine<CORR_F_COMPLEX4, false>(*p, d_time, n_frames, d_spectra, s);
    else
        e = pfb ? launch_fengine<CORR_F_REAL8, true>(*p, d_time, n_frames, d_spectra, s)
                : launch_fengine<CORR_F_REAL8, false>(*p, d_time, n_frames, d_spectra, s);
    if (e != cudaSuccess) return cuda_error(e, "F-stage launch");
    return CORR_OK;
}

}  // extern "C"

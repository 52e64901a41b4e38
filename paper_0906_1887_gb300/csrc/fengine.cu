// F stage of the FX correlator (Sec. 2, Sec. 4): unpack + per-input DFT of time blocks.
//
// The paper's GPU correlator unpacks a batch of time samples (input index fastest), reorders
// it into per-input blocks and Fourier transforms each block into spectral channels: an
// N_C-point complex transform for complex samples, and for real samples a 2 N_C-point
// complex-to-complex transform of which channels 0 .. N_C are kept (Sec. 4).  Here one
// kernel does both steps for a block of G inputs and one frame of L samples:
//
//   load    packed samples [t][input] -> float2 rows in shared memory, one row per input;
//           each thread loads 4 adjacent inputs of a sample at once (8 or 4 bytes) and
//           converts bytes and nibbles to float with the 2^23 exponent trick
//   FFT     Stockham autosort stages of radix 16 (the last one of radix 8, 4 or 2 when
//           log2 L is not a multiple of 4), ping-ponging between two shared buffers: each
//           task loads R values, applies the stage twiddles (per-stage tables computed on the
//           host in double precision) and does the R-point DFT in registers (radix-2
//           butterflies with exact constant twiddles of the 16th roots of unity).  L = 128,
//           the paper's channel count, takes two stages (16 x 8)
//   store   spectra [frame][channel][input] complex float32, coalesced along the inputs --
//           exactly the float sample layout the X stage takes ([T][C][N], T = frames)
//
// L is a template parameter (one kernel per power of two from 8 to 4096): every index is then
// a shift or a compile-time offset from a per-thread base, and the row pitch and task layout
// of each length keep all shared-memory phases free of bank conflicts.
//
// A Stockham stage with sub-transform length Ns and radix R takes, for each j < L / R, the R
// values v_r = x[j + r L / R], multiplies v_r by exp(-2 pi i (j mod Ns) r / (Ns R)), applies
// the R-point DFT and writes output q to position (j - j mod Ns) R + j mod Ns + q Ns.  After
// log_R L stages the result is in natural order.  The DFT is the forward, unnormalised one,
// X_k = sum_s x_s exp(-2 pi i k s / L); channel c is bin c.
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "corr_internal.h"

namespace corr {
namespace {

constexpr int kFPoints = 4096;   // complex points per CTA (inputs x transform length)
constexpr int kFThreads = 256;
constexpr int kFMinLen = 8, kFMaxLen = 4096;

// position of row element i: one pad element after every 16.  For a power of two P and
// j < P, pad(j + r P) = pad(j) + pad(r P): every strided access below is a per-thread base
// plus compile-time offsets.
__host__ __device__ constexpr int pad(int i) { return i + (i >> 4); }

// Geometry of the transform length L = 2^LG.  G inputs per CTA (G L = 4096 points, at most
// 64 inputs).  The row pitch (float2 elements, at least pad(L - 1) + 1) is chosen per length so
// that the load, transform and store phases below all fall in distinct shared-memory banks
// (each access pattern was modelled bank by bank on the CPU).
__host__ __device__ constexpr int f_groups(int LG) { return LG >= 6 ? kFPoints >> LG : 64; }
__host__ __device__ constexpr int f_pitch(int LG) {
    return LG == 3 ? 9 : LG == 4 ? 17 : LG == 5 ? 35 : LG == 6 ? 69 : LG == 7 ? 137 : LG == 8 ? 273 :
           LG == 9 ? 546 : LG == 10 ? 1092 : LG == 11 ? 2184 : 4352;
}
__host__ __device__ constexpr int f_stages(int LG) { return (LG + 3) / 4; }
__host__ __device__ constexpr int f_stage_lgr(int LG, int st) { return LG - 4 * st < 4 ? LG - 4 * st : 4; }
// Stage st (sub-transform length Ns = 16^st, radix R) uses twiddles exp(-2 pi i k r / (Ns R))
// for k < Ns, 1 <= r < R, stored k-major at entry k (R - 1) + r - 1 of the stage's table;
// the tables of stages 1, 2, ... follow one another (stage 0 has Ns = 1: no twiddles).
__host__ __device__ constexpr int f_tw_offset(int LG, int st) {
    int o = 0;
    for (int u = 1; u < st; ++u) o += (1 << (4 * u)) * ((1 << f_stage_lgr(LG, u)) - 1);
    return o;
}
__host__ __device__ constexpr int f_tw_entries(int LG) { return f_tw_offset(LG, f_stages(LG)); }

template <int LG>
struct FGeom {
    static constexpr int L = 1 << LG;
    static constexpr int G = f_groups(LG);
    static constexpr int LGG = LG >= 6 ? 12 - LG : 6;
    static constexpr int PITCH = f_pitch(LG);
    static constexpr int PTS = L * G;
    static constexpr int V = G < 4 ? G : 4;                      // inputs per vector load
    static constexpr int VPR = G / V;                            // vector loads per sample row
    static constexpr int NVEC = (PTS / V + kFThreads - 1) / kFThreads;   // per thread per frame
    static_assert(PITCH >= pad(L - 1) + 1, "row shorter than the padded transform");
    static_assert((1 << LGG) == G, "inputs per CTA");
};

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
    float2* d_tw = nullptr;   // the stage twiddle tables (f_tw_entries(log2L) values, at least one)
    int n_taps = 1;           // PFB taps M (input frames per output frame)
    float* d_taps = nullptr;  // PFB prototype, M L values; nullptr: plain transform
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

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

// Task -> row of a transposed-path stage.  When a half-warp spans several rows (L / R < 16),
// the rows it takes are spread by rotating the low four bits of the row index, which puts
// their bank windows side by side instead of on top of one another (first stage of L = 32,
// 64, 128).
template <int LG, int ST>
__device__ __forceinline__ int stage_row(int gi) {
    if constexpr (ST == 0 && LG == 5) return ((gi & 7) << 1) | ((gi >> 3) & 1) | (gi & ~15);
    else if constexpr (ST == 0 && LG == 6) return ((gi & 3) << 2) | ((gi >> 2) & 3) | (gi & ~15);
    else if constexpr (ST == 0 && LG == 7) return ((gi & 1) << 3) | ((gi >> 1) & 7) | (gi & ~15);
    else return gi;
}

// Stockham stage ST over the G rows of `a` into `b` (Ns = 16^ST, radix R, L / R tasks per
// row).  The transposed path runs every stage but the last one this way.
template <int LG, int ST>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ a, float2* __restrict__ b,
                                          const float2* __restrict__ tws) {
    using Geo = FGeom<LG>;
    constexpr int LGNS = 4 * ST, NS = 1 << LGNS;
    constexpr int LGR = f_stage_lgr(LG, ST), R = 1 << LGR;
    constexpr int LGLR = LG - LGR, LR = 1 << LGLR;
    constexpr int NTASK = LR * Geo::G;
    constexpr int NIT = (NTASK + kFThreads - 1) / kFThreads;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int task = threadIdx.x + it * kFThreads;
        if (NTASK % kFThreads != 0 && task >= NTASK) break;
        const int g = stage_row<LG, ST>(task >> LGLR), j = task & (LR - 1);
        const float2* src = a + g * Geo::PITCH + pad(j);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[pad(r * LR)];
        const int k = j & (NS - 1);
        if constexpr (ST > 0) {
            if (k) {
                const float2* t = tws + f_tw_offset(LG, ST) + k * (R - 1) - 1;
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = cmul(v[r], t[r]);
            }
        }
        dft_reg<R>(v);
        float2* dst = b + g * Geo::PITCH + pad((j - k) * R + k);
#pragma unroll
        for (int q = 0; q < R; ++q) dst[pad(q * NS)] = v[q];
    }
}

// stages ST .. (last - 1), ping-ponging between the buffers; returns the one the last stage reads
template <int LG, int ST>
__device__ __forceinline__ const float2* fft_mid_stages(float2* a, float2* b, const float2* tws) {
    if constexpr (ST < f_stages(LG) - 1) {
        fft_stage<LG, ST>(a, b, tws);
        __syncthreads();
        return fft_mid_stages<LG, ST + 1>(b, a, tws);
    } else {
        return a;
    }
}

// The last stage stores the spectrum itself: its sub-transform length is Ns = L / R, so task
// j < Ns yields channels j + q Ns.  Tasks run inputs fastest, so a warp's stores of a channel
// are contiguous.  out_f points at channel 0 of input n0 of the frame.
template <int KIND, int LG>
__device__ __forceinline__ void fft_last_stage(const float2* __restrict__ a, const float2* __restrict__ tws,
                                               float2* __restrict__ out_f, int N, int g_n) {
    using Geo = FGeom<LG>;
    constexpr int ST = f_stages(LG) - 1;
    constexpr int NS = 1 << (4 * ST);
    constexpr int LGR = f_stage_lgr(LG, ST), R = 1 << LGR;
    constexpr int LR = 1 << (LG - LGR);
    static_assert(LR == NS, "the last stage's tasks are its sub-transform offsets");
    constexpr int NOUT = KIND == CORR_F_REAL8 ? Geo::L / 2 + 1 : Geo::L;
    constexpr int NTASK = LR * Geo::G;
    constexpr int NIT = (NTASK + kFThreads - 1) / kFThreads;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int task = threadIdx.x + it * kFThreads;
        if (NTASK % kFThreads != 0 && task >= NTASK) break;
        const int g = task & (Geo::G - 1), j = task >> Geo::LGG;
        if (g >= g_n) continue;
        const float2* src = a + g * Geo::PITCH + pad(j);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[pad(r * LR)];
        if constexpr (ST > 0) {
            if (j) {
                const float2* t = tws + f_tw_offset(LG, ST) + j * (R - 1) - 1;
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = cmul(v[r], t[r]);
            }
        }
        dft_reg<R>(v);
        float2* o = out_f + j * N + g;
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (NOUT == Geo::L || j + q * NS < NOUT) o[q * NS * N] = v[q];
    }
}

// bytes per packed sample: 2 for complex 8-bit, 1 otherwise
template <int KIND>
__host__ __device__ constexpr int f_bps() { return KIND == CORR_F_COMPLEX8 ? 2 : 1; }

// V consecutive inputs of one sample: 8 bytes (complex 8-bit, V = 4) or at most 4
template <int KIND, int LG>
using FRaw = std::conditional_t<KIND == CORR_F_COMPLEX8 && FGeom<LG>::V == 4, uint2, uint32_t>;

// one vector: exactly V x (bytes per sample) bytes, aligned to that size
template <int KIND, int LG>
__device__ __forceinline__ FRaw<KIND, LG> load_vec(const uint8_t* src) {
    constexpr int B = FGeom<LG>::V * f_bps<KIND>();
    if constexpr (B == 8) return *reinterpret_cast<const uint2*>(src);
    else if constexpr (B == 4) return *reinterpret_cast<const uint32_t*>(src);
    else if constexpr (B == 2) return (uint32_t)*reinterpret_cast<const unsigned short*>(src);
    else return (uint32_t)*src;
}

// vector load e of a frame -> sample s and first input g.  For rows of 8 or more vectors a warp
// takes 4 samples x 8 vectors (each half-warp 4 x 4), whose shared-memory rows fall in
// distinct banks; the global reads stay 32-byte sectors
template <int LG>
__device__ __forceinline__ void vec_pos(int e, int& s, int& g) {
    using Geo = FGeom<LG>;
    if constexpr (Geo::VPR >= 8) {
        constexpr int NB = Geo::VPR / 8;
        const int b = e >> 5, t = e & 31;
        const int m = (t & 3) | ((t >> 4) << 2);
        s = (b / NB) * 4 + ((t >> 2) & 3);
        g = ((b % NB) * 8 + m) * Geo::V;
    } else {
        s = e / Geo::VPR;
        g = (e % Geo::VPR) * Geo::V;
    }
}

// the packed samples thread `threadIdx.x` moves of one frame (zeros outside the array).
// `in_f` points at sample 0 of input n0 of the frame; vec: one aligned load per vector
template <int KIND, int LG>
__device__ __forceinline__ void fetch_frame(FRaw<KIND, LG> (&raw)[FGeom<LG>::NVEC], const uint8_t* __restrict__ in_f,
                                            int N, int g_n, bool vec) {
    using Geo = FGeom<LG>;
    using RawT = FRaw<KIND, LG>;
    constexpr int BPS = f_bps<KIND>();
#pragma unroll
    for (int q = 0; q < Geo::NVEC; ++q) {
        const int e = threadIdx.x + q * kFThreads;
        RawT r{};
        if (Geo::NVEC * kFThreads * Geo::V == Geo::PTS || e < Geo::PTS / Geo::V) {
            int s, g;
            vec_pos<LG>(e, s, g);
            const uint8_t* src = in_f + (s * N + g) * BPS;
            if (vec) {
                if (g < g_n) r = load_vec<KIND, LG>(src);
            } else {
                uint32_t w[2] = {0u, 0u};
#pragma unroll
                for (int k = 0; k < Geo::V; ++k) {
                    if (g + k < g_n) {
                        const uint32_t x = BPS == 2 ? (uint32_t)*reinterpret_cast<const unsigned short*>(src + 2 * k)
                                                    : (uint32_t)src[k];
                        w[(k * BPS) >> 2] |= x << (((k * BPS) & 3) * 8);
                    }
                }
                if constexpr (sizeof(RawT) == 8) r = make_uint2(w[0], w[1]);
                else r = w[0];
            }
        }
        raw[q] = r;
    }
}

// small integers to float by the 2^23 exponent trick: a byte u (or nibble) placed in the low
// mantissa of 2^23 gives the float 2^23 + u exactly; the sign offset is flipped into u first
// (u = x + 128 for a signed byte, x + 8 for a signed nibble), then one exact subtraction
__device__ __forceinline__ float f_byte(uint32_t w, uint32_t sel, float bias) {
    return __int_as_float((int)__byte_perm(w, 0x4B000000u, sel)) - bias;
}
constexpr float kBias8 = 8388736.0f;   // 2^23 + 128
constexpr float kBias4 = 8388616.0f;   // 2^23 + 8

// vector load -> V complex values (inputs g .. g + V - 1)
template <int KIND, int LG>
__device__ __forceinline__ void unpack_vec(FRaw<KIND, LG> r, float2 (&x)[FGeom<LG>::V]) {
    constexpr int V = FGeom<LG>::V;
    if constexpr (KIND == CORR_F_COMPLEX8) {
        uint32_t w[2];
        if constexpr (V == 4) {
            w[0] = r.x ^ 0x80808080u;
            w[1] = r.y ^ 0x80808080u;
        } else {
            w[0] = r ^ 0x80808080u;
            w[1] = 0u;
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const uint32_t ww = w[k >> 1];
            const uint32_t b0 = (uint32_t)(2 * (k & 1));
            x[k] = make_float2(f_byte(ww, 0x7540u | b0, kBias8), f_byte(ww, 0x7540u | (b0 + 1), kBias8));
        }
    } else if constexpr (KIND == CORR_F_COMPLEX4) {
        const uint32_t w = r ^ 0x88888888u;   // high nibble re, low nibble im
        const uint32_t hi = (w >> 4) & 0x0F0F0F0Fu, lo = w & 0x0F0F0F0Fu;
#pragma unroll
        for (int k = 0; k < V; ++k)
            x[k] = make_float2(f_byte(hi, 0x7540u | (uint32_t)k, kBias4), f_byte(lo, 0x7540u | (uint32_t)k, kBias4));
    } else {
        const uint32_t w = r ^ 0x80808080u;
#pragma unroll
        for (int k = 0; k < V; ++k) x[k] = make_float2(f_byte(w, 0x7540u | (uint32_t)k, kBias8), 0.f);
    }
}

// Fused first stage (G >= 16, i.e. L <= 256): thread t takes input g = t mod G and offset
// j = t / G (< L / R), and loads the R samples j + r L / R of its input straight from global
// memory -- lanes run along the inputs, so each load of a warp reads whole sample rows of the
// CTA's inputs -- then does the first radix-R DFT in registers (Ns = 1: no twiddles).  The
// transposing pass through shared memory disappears.
template <int LG>
struct FFirst {
    static constexpr int R = 1 << f_stage_lgr(LG, 0);
    static constexpr int LR = FGeom<LG>::L / R;
    static constexpr int NTASK = LR * FGeom<LG>::G;
    static_assert(NTASK <= kFThreads, "one first-stage task per thread");
};

template <int KIND, int LG>
__device__ __forceinline__ void fetch_task(uint32_t (&raw)[FFirst<LG>::R], const uint8_t* __restrict__ in_f, int N,
                                           bool active) {
    using F = FFirst<LG>;
    constexpr int BPS = f_bps<KIND>();
    const int g = threadIdx.x & (FGeom<LG>::G - 1), j = threadIdx.x >> FGeom<LG>::LGG;
    const uint8_t* src = in_f + (j * N + g) * BPS;
    const int step = F::LR * N * BPS;
#pragma unroll
    for (int r = 0; r < F::R; ++r)
        raw[r] = !active ? 0u
                         : (BPS == 2 ? (uint32_t)*reinterpret_cast<const unsigned short*>(src + r * step)
                                     : (uint32_t)src[r * step]);
}

// one packed sample -> complex float (exact)
template <int KIND>
__device__ __forceinline__ float2 unpack1(uint32_t r) {
    if constexpr (KIND == CORR_F_COMPLEX8) {
        const uint32_t w = r ^ 0x8080u;
        return make_float2(f_byte(w, 0x7540u, kBias8), f_byte(w, 0x7541u, kBias8));
    } else if constexpr (KIND == CORR_F_COMPLEX4) {
        const uint32_t w = r ^ 0x88u;
        return make_float2(f_byte((w >> 4) & 15u, 0x7540u, kBias4), f_byte(w & 15u, 0x7540u, kBias4));
    } else {
        return make_float2(f_byte(r ^ 0x80u, 0x7540u, kBias8), 0.f);
    }
}

// Persistent over frames: frame f + gridDim.y's samples are fetched into registers while frame
// f is transformed, so the global loads overlap the FFT.  PFB = true is the polyphase
// filterbank (Sec. 6.1): the load phase forms y[s] = sum_m h[m L + s] x[(f + m) L + s] over M
// input frames (the extra cost the paper places in the unpack), then the same transform runs.
template <int KIND, bool PFB, int LG>
__global__ void __launch_bounds__(kFThreads, 3) fengine_kernel(const uint8_t* __restrict__ in, float2* __restrict__ out,
                                                            const float2* __restrict__ tw, int N, int n_frames,
                                                            const float* __restrict__ taps, int M, int vec) {
    using Geo = FGeom<LG>;
    constexpr int L = Geo::L, G = Geo::G;
    constexpr int BPS = f_bps<KIND>();
    constexpr int TWN = f_tw_entries(LG);
    constexpr int NOUT = KIND == CORR_F_REAL8 ? L / 2 + 1 : L;
    // first stage straight from global memory for L <= 256; the filterbank keeps the vector
    // loads (M input frames per output frame: four times fewer load instructions)
    constexpr bool kFused = G >= 16 && !PFB;
    extern __shared__ float2 fsm[];
    float2* const buf0 = fsm;
    float2* const buf1 = fsm + G * Geo::PITCH;
    float2* const tws = fsm + 2 * G * Geo::PITCH;
    float* const tapl = reinterpret_cast<float*>(tws + TWN);   // PFB: the prototype, M L values
    const int n0 = blockIdx.x * G;
    const int g_n = min(G, N - n0);
    for (int k = threadIdx.x; k < TWN; k += kFThreads) tws[k] = tw[k];
    if constexpr (PFB)
        for (int k = threadIdx.x; k < M * L; k += kFThreads) tapl[k] = taps[k];
    __syncthreads();   // the tables are read by other threads (the taps before the first barrier below)
    const size_t frame_bytes = (size_t)L * N * BPS;
    const uint8_t* const in_n0 = in + (size_t)n0 * BPS;

    if constexpr (kFused) {
        using F = FFirst<LG>;
        constexpr int R = F::R;
        const int g = threadIdx.x & (G - 1), j = threadIdx.x >> Geo::LGG;
        const bool active = (F::NTASK == kFThreads || (int)threadIdx.x < F::NTASK) && g < g_n;
        uint32_t raw[R];
        int f = blockIdx.y;
        if constexpr (!PFB) {
            if (f < n_frames) fetch_task<KIND, LG>(raw, in_n0 + (size_t)f * frame_bytes, N, active);
        }
        int par = 0;
        for (; f < n_frames; f += gridDim.y) {
            float2 v[R];
            if constexpr (PFB) {
                // weighted overlap of input frames f .. f + M - 1 for samples j + r L / R
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
                for (int m = 0; m < M; ++m) {
                    fetch_task<KIND, LG>(raw, in_n0 + (size_t)(f + m) * frame_bytes, N, active);
                    if (active) {   // a thread without a task has j >= L / R: no taps of its own
                        const float* hm = tapl + m * L + j;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const float hw = hm[r * F::LR];
                            const float2 x = unpack1<KIND>(raw[r]);
                            v[r].x = fmaf(hw, x.x, v[r].x);
                            v[r].y = fmaf(hw, x.y, v[r].y);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = unpack1<KIND>(raw[r]);
                if (f + (int)gridDim.y < n_frames)
                    fetch_task<KIND, LG>(raw, in_n0 + (size_t)(f + gridDim.y) * frame_bytes, N, active);
            }
            dft_reg<R>(v);
            float2* const out_f = out + (size_t)f * NOUT * N + n0;
            if constexpr (f_stages(LG) == 1) {
                // the whole transform (L = R): channel q of input g
                if (active) {
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        if (q < NOUT) out_f[q * N + g] = v[q];
                }
            } else {
                // first-stage outputs j R + q of row g; the buffers alternate between frames, so
                // one barrier per frame orders every write against every read
                float2* const buf = par ? buf1 : buf0;
                if (active) {
                    float2* dst = buf + g * Geo::PITCH + pad(j * R);
#pragma unroll
                    for (int q = 0; q < R; ++q) dst[pad(q)] = v[q];
                }
                __syncthreads();
                fft_last_stage<KIND, LG>(buf, tws, out_f, N, g_n);
                par ^= 1;
            }
        }
    } else {
        // coalesced vector loads transposed into rows, then the stages
        using RawT = FRaw<KIND, LG>;
        constexpr int V = Geo::V, NVEC = Geo::NVEC;
        RawT raw[NVEC];
        int f = blockIdx.y;
        if constexpr (!PFB) {
            if (f < n_frames) fetch_frame<KIND, LG>(raw, in_n0 + (size_t)f * frame_bytes, N, g_n, vec != 0);
        }
        for (; f < n_frames; f += gridDim.y) {
            if constexpr (PFB) {
                float2 acc[NVEC][V];
#pragma unroll
                for (int q = 0; q < NVEC; ++q)
#pragma unroll
                    for (int k = 0; k < V; ++k) acc[q][k] = make_float2(0.f, 0.f);
                for (int m = 0; m < M; ++m) {
                    fetch_frame<KIND, LG>(raw, in_n0 + (size_t)(f + m) * frame_bytes, N, g_n, vec != 0);
#pragma unroll
                    for (int q = 0; q < NVEC; ++q) {
                        const int e = threadIdx.x + q * kFThreads;
                        if (NVEC * kFThreads * V == Geo::PTS || e < Geo::PTS / V) {
                            int s, g;
                            vec_pos<LG>(e, s, g);
                            const float hw = tapl[m * L + s];
                            float2 x[V];
                            unpack_vec<KIND, LG>(raw[q], x);
#pragma unroll
                            for (int k = 0; k < V; ++k) {
                                acc[q][k].x = fmaf(hw, x[k].x, acc[q][k].x);
                                acc[q][k].y = fmaf(hw, x[k].y, acc[q][k].y);
                            }
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < NVEC; ++q) {
                    const int e = threadIdx.x + q * kFThreads;
                    if (NVEC * kFThreads * V == Geo::PTS || e < Geo::PTS / V) {
                        int s, g;
                        vec_pos<LG>(e, s, g);
                        float2* d = buf0 + g * Geo::PITCH + pad(s);
#pragma unroll
                        for (int k = 0; k < V; ++k) d[k * Geo::PITCH] = acc[q][k];
                    }
                }
                __syncthreads();
            } else {
                // sample s of input n0 + g + k, time f L + s -> buf0[g + k][s]
#pragma unroll
                for (int q = 0; q < NVEC; ++q) {
                    const int e = threadIdx.x + q * kFThreads;
                    if (NVEC * kFThreads * V == Geo::PTS || e < Geo::PTS / V) {
                        int s, g;
                        vec_pos<LG>(e, s, g);
                        float2 x[V];
                        unpack_vec<KIND, LG>(raw[q], x);
                        float2* d = buf0 + g * Geo::PITCH + pad(s);
#pragma unroll
                        for (int k = 0; k < V; ++k) d[k * Geo::PITCH] = x[k];
                    }
                }
                __syncthreads();
                if (f + (int)gridDim.y < n_frames)
                    fetch_frame<KIND, LG>(raw, in_n0 + (size_t)(f + gridDim.y) * frame_bytes, N, g_n, vec != 0);
            }
            const float2* last = fft_mid_stages<LG, 0>(buf0, buf1, tws);
            fft_last_stage<KIND, LG>(last, tws, out + (size_t)f * NOUT * N + n0, N, g_n);
            __syncthreads();   // the next frame rewrites the buffers
        }
    }
}

size_t fplan_smem(int log2L, int n_taps_pfb) {
    const size_t G = (size_t)f_groups(log2L);
    return (2 * G * (size_t)f_pitch(log2L) + (size_t)f_tw_entries(log2L)) * sizeof(float2) +
           (size_t)n_taps_pfb * ((size_t)1 << log2L) * sizeof(float);
}

size_t fplan_smem(const FPlan& p) { return fplan_smem(p.log2L, p.d_taps ? p.n_taps : 0); }

template <int KIND, bool PFB, int LG>
cudaError_t launch_fengine_l(const FPlan& p, const void* d_in, int n_frames, void* d_out, cudaStream_t s) {
    auto kern = fengine_kernel<KIND, PFB, LG>;
    const int smem = (int)fplan_smem(p);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // persistent over frames: enough CTAs to fill every SM a few times over
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFThreads, smem);
    if (e != cudaSuccess) return e;
    constexpr int G = FGeom<LG>::G, V = FGeom<LG>::V;
    const int groups = (p.n_inputs + G - 1) / G;
    int rows = (p.n_sm * (per_sm > 0 ? per_sm : 1) * 4 + groups - 1) / groups;
    if (rows > n_frames) rows = n_frames;
    if (rows > 65535) rows = 65535;
    // one load per V inputs when every such group starts on a V-sample boundary in memory
    const int vec = (p.n_inputs % V == 0 && (reinterpret_cast<uintptr_t>(d_in) % (size_t)(V * f_bps<KIND>())) == 0) ? 1 : 0;
    const dim3 grid(groups, rows);
    kern<<<grid, kFThreads, smem, s>>>(static_cast<const uint8_t*>(d_in), static_cast<float2*>(d_out), p.d_tw,
                                       p.n_inputs, n_frames, p.d_taps, p.n_taps, vec);
    return cudaGetLastError();
}

template <int KIND, bool PFB>
cudaError_t launch_fengine(const FPlan& p, const void* d_in, int n_frames, void* d_out, cudaStream_t s) {
    switch (p.log2L) {
        case 3: return launch_fengine_l<KIND, PFB, 3>(p, d_in, n_frames, d_out, s);
        case 4: return launch_fengine_l<KIND, PFB, 4>(p, d_in, n_frames, d_out, s);
        case 5: return launch_fengine_l<KIND, PFB, 5>(p, d_in, n_frames, d_out, s);
        case 6: return launch_fengine_l<KIND, PFB, 6>(p, d_in, n_frames, d_out, s);
        case 7: return launch_fengine_l<KIND, PFB, 7>(p, d_in, n_frames, d_out, s);
        case 8: return launch_fengine_l<KIND, PFB, 8>(p, d_in, n_frames, d_out, s);
        case 9: return launch_fengine_l<KIND, PFB, 9>(p, d_in, n_frames, d_out, s);
        case 10: return launch_fengine_l<KIND, PFB, 10>(p, d_in, n_frames, d_out, s);
        case 11: return launch_fengine_l<KIND, PFB, 11>(p, d_in, n_frames, d_out, s);
        case 12: return launch_fengine_l<KIND, PFB, 12>(p, d_in, n_frames, d_out, s);
        default: return cudaErrorInvalidValue;
    }
}

// the stage twiddle tables for L = 2^LG, each entry rounded from double precision
std::vector<float2> make_twiddles(int LG) {
    const int L = 1 << LG;
    std::vector<float2> tw((size_t)(f_tw_entries(LG) > 0 ? f_tw_entries(LG) : 1), make_float2(1.f, 0.f));
    for (int st = 1; st < f_stages(LG); ++st) {
        const int Ns = 1 << (4 * st), lgr = f_stage_lgr(LG, st), R = 1 << lgr;
        const int tshift = LG - 4 * st - lgr;   // exp(-2 pi i k r / (Ns R)) = w_L^((k r) << tshift)
        for (int k = 0; k < Ns; ++k)
            for (int r = 1; r < R; ++r) {
                const int m = (r * k) << tshift;
                const double ang = -2.0 * M_PI * (double)m / (double)L;
                tw[(size_t)f_tw_offset(LG, st) + (size_t)k * (R - 1) + (r - 1)] =
                    make_float2((float)cos(ang), (float)sin(ang));
            }
    }
    return tw;
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
    while ((1 << p->log2L) < L) ++p->log2L;
    p->G = f_groups(p->log2L);
    while ((1 << p->log2G) < p->G) ++p->log2G;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device);
    const std::vector<float2> tw = make_twiddles(p->log2L);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tw, tw.size() * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
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
    if (fplan_smem(p->log2L, n_taps) > (size_t)227 * 1024) {
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

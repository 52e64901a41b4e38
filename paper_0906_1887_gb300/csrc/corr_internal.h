// Internal declarations shared by the host runtime and the CUDA kernels of libcorr.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/corr.h"

namespace corr {

constexpr int kBlockInputs = 64;      // inputs per operand block (rows 0..63 re, 64..127 im)
constexpr int kBlockRows = 128;       // rows of one plane block
constexpr int kTimeBlock = 64;        // samples per pipeline stage (one 128-byte fp16 row)
constexpr int kMaxInputs = 8192;
constexpr int kMaxJobsPerLaunch = 64;  // jobs one packed tensor-core launch carries

// Device error codes written to the plan's status block.
enum DeviceError : int {
    kDevOk = 0,
    kDevTimeoutFull = 1,      // MMA waited too long for a loaded stage
    kDevTimeoutEmpty = 2,     // producer waited too long for a free stage
    kDevTimeoutAccFull = 3,   // epilogue waited too long for an accumulator
    kDevTimeoutAccEmpty = 4,  // MMA waited too long for a drained accumulator
    kDevBadItem = 5,          // a work item decoded outside its problem
};

struct Plan {
    int n_inputs = 0;
    int n_chan = 0;
    int n_time = 0;
    int sample_bits = 0;
    int nb = 0;              // ceil(N / 64)
    int kp = 0;              // n_time rounded up to 64
    int64_t n_baselines = 0;
    int device = 0;
    int n_sm = 0;
    int* d_status = nullptr; // [4] device status words
    int tc_op_stages = 0;     // operand ring depth of the packed-sample kernel (0: default)
    int tc_float_planes = 0;  // BF16x3: 1 = hi/lo planes through memory even where the fused path applies
    int tc_operands = 0;      // 4/8-bit, tensor cores: 0 auto, 1 packed samples (fused converters), 2 fp16 planes,
                              // 3 packed 4-bit samples converted to e4m3 operands
    int tc_items = 0;         // plane path: 0 auto (wide), 1 single tiles, 2 wide items
    // host-buffer pipeline (corr_xengine_run_host), created on first use
    char* pipe_dev = nullptr;   // 2 x (chunk inputs) + 2 x (chunk outputs) + workspace
    size_t pipe_bytes = 0;
    cudaStream_t pipe_stream[3] = {nullptr, nullptr, nullptr};   // copy in, compute, copy out
    cudaEvent_t pipe_ev[8] = {};
};

inline int64_t n_baselines(int64_t n) { return n * (n + 1) / 2; }

// Host-side error reporting (thread-local message).
corr_status set_error(corr_status st, const char* fmt, ...);
corr_status cuda_error(cudaError_t e, const char* what);

size_t plane_elem_bytes(const Plan& p);              // 2 (fp16) or 4 (fp32)
size_t planes_bytes(const Plan& p, int n_dumps);     // one set of planes

// Kernel launchers (return cudaSuccess or the launch error).
// blocks_per_sm > 0 caps the vectorised kernel's grid at that many blocks per SM (a launch that
// runs beside a tensor-core launch takes one, which fits next to its CTA in either launch order)
cudaError_t launch_unpack_fp16(const Plan& p, const void* d_packed, int n_dumps, void* d_planes,
                               cudaStream_t s, int blocks_per_sm = 0);
cudaError_t launch_unpack_f32(const Plan& p, const void* d_packed, int n_dumps, void* d_planes,
                              cudaStream_t s);
cudaError_t launch_unpack_bf16x2(const Plan& p, const void* d_packed, int n_dumps, void* d_hi,
                                 void* d_lo, cudaStream_t s);
cudaError_t launch_xeng_fp32(const Plan& p, const void* d_planes, int n_dumps, void* d_vis,
                             int accumulate, cudaStream_t s);
// FP32 engine on the packed samples themselves (4/8-bit or float32), no planes
cudaError_t launch_xeng_fp32_packed(const Plan& p, const void* d_packed, int n_dumps, void* d_vis, int accumulate,
                                    cudaStream_t s);
cudaError_t launch_xeng_tc(const Plan& p, const void* d_planes, const void* d_planes_lo, int n_dumps,
                           void* d_vis, int accumulate, cudaStream_t s);
// Fused path: packed 4/8-bit samples straight into the tensor-core kernel (no planes).
bool tc_raw_supported(const Plan& p);
// Whether the tensor-core X stage of 4/8-bit samples reads fp16 planes (written by the unpack
// kernel into the workspace) rather than converting the packed samples itself: always when the
// packed rows are not TMA-addressable; otherwise as the plan's knob says, by default for arrays
// of at least kPlaneMinBlocks 64-input blocks, whose tiles re-read every block nb / 2 times
// (kPlaneMinBlocksE4m3 for 4-bit samples, whose e4m3 planes cost half as much: measured, 192
// inputs x 1024 channels x 1024 samples 0.269 ms on planes against 0.398 ms converted in the
// kernel; at 128 inputs the two feeds trade places with the dump length).
constexpr int kPlaneMinBlocks = 4;
constexpr int kPlaneMinBlocksE4m3 = 3;
bool tc_use_planes(const Plan& p);
bool tc_raw_supported(int n_inputs, int sample_bits);
// The workspace's planes: e4m3 bytes for 4-bit samples of TMA-addressable rows (rows of
// tc_kp_e4m3 = n_time rounded up to 128 bytes, read by kind::f8f6f4 MMAs), fp16 otherwise.  The
// public planes calls (corr_unpack, corr_xengine_run_planes) keep fp16 planes.
bool tc_planes_e4m3(const Plan& p);
int tc_kp_e4m3(const Plan& p);
size_t tc_workspace_planes_bytes(const Plan& p, int n_dumps);
cudaError_t launch_unpack_e4m3(const Plan& p, const void* d_packed, int n_dumps, void* d_planes, cudaStream_t s,
                               int blocks_per_sm = 0);
cudaError_t launch_xeng_tc_e4m3_planes(const Plan& p, const void* d_planes, int n_dumps, void* d_vis, int accumulate,
                                       cudaStream_t s);
// unpack into the workspace's planes, then the plane-fed tensor-core X stage
cudaError_t launch_tc_plane_path(const Plan& p, const void* d_packed, int n_dumps, void* d_ws, void* d_vis,
                                 int accumulate, cudaStream_t s);
struct TcTuning;
cudaError_t launch_xeng_tc_raw(const Plan& p, const void* d_packed, int n_dumps, void* d_vis, int accumulate,
                               cudaStream_t s, const TcTuning* tune = nullptr);

// One job of a packed (multi-job) tensor-core launch.
struct TcJobSpec {
    int n_inputs, n_chan, n_time, n_dumps, sample_bits;
    const void* data;   // packed samples [n_dumps][T][C][N] (device)
    void* vis;          // [n_dumps][C][P][2] int64 (device)
    int cpi;            // channels per work item: 1, or 2 for arrays of at most 64 inputs
    int out_mode = 0;   // 1: dump mode, float32 [n_dumps][C][P][2] of V / n_accum * phasor_i conj(phasor_j)
    const void* phasor = nullptr;   // float2 [C][N] (device) or nullptr
    float inv_n = 1.0f;
    int tw = 1;         // plane path: 2 = wide items (block I against blocks J, J + 1 in one MMA)
};
// Launch-shape knobs the autotuner chooses (0 = default).
struct TcTuning {
    int op_stages = 0;
    int smem_reserve = 0;         // plane feed: shared memory per SM left free for a concurrent kernel
    uint64_t wait_limit_ns = 0;   // 0: the default bound (2 s)
    int64_t stall_item = -1;      // self-test of the bounded waits (-1: off)
    int f8_operands = 0;          // packed 4-bit samples: e4m3 operands (kind::f8f6f4; maps with 128-sample boxes)
};
int tc_default_cpi(int n_inputs, int64_t channels, int n_sm);   // channels = dumps x n_chan of the launch
// BF16x3 on float samples with the hi/lo split done in the tensor-core kernel (single-block arrays)
bool tc_rawf32_supported(const Plan& p);
cudaError_t launch_xeng_tc_rawf32(const Plan& p, const void* d_samples, int n_dumps, void* d_vis, int accumulate,
                                  cudaStream_t s);
// Fused dump mode: float32 [n_dumps][C][P][2] = V / n_accum * phasor_i conj(phasor_j) (phasor
// float2 [C][N] or nullptr); every dump must fit one exact chunk.
cudaError_t launch_xeng_tc_raw_dump(const Plan& p, const void* d_packed, int n_dumps, void* d_out, const void* phasor,
                                    float inv_n, cudaStream_t s);
// Per-input phasors exp(+2 pi i nu_c tau_n) as float2 [C][N], formed in double precision.
cudaError_t launch_phasors(const Plan& p, const double* d_delays, const double* d_freqs, void* d_g, cudaStream_t s);
bool tc_make_raw_map(CUtensorMap* map, const TcJobSpec& sp, bool f8 = false);   // f8: 128-sample boxes
// Jobs whose samples the unpack kernel already turned into fp16 planes (TcJobSpec::data = the
// planes, [n_dumps][C][NB][128][Kp]); one channel per work item.
bool tc_make_plane_map(CUtensorMap* map, const TcJobSpec& sp, bool f8 = false);   // f8: e4m3 planes
// the same planes in boxes of two adjacent blocks, for wide items (TcJobSpec::tw = 2)
bool tc_make_plane_map_wide(CUtensorMap* map, const TcJobSpec& sp, bool f8 = false);   // f8: e4m3 planes
cudaError_t launch_xeng_tc_plane_jobs(const TcJobSpec* specs, const CUtensorMap* maps, int n_jobs, int accumulate,
                                      int* status, int n_sm, const TcTuning& tune, cudaStream_t s,
                                      const CUtensorMap* maps_wide = nullptr);
// All jobs of one launch share a sample mode (4 or 8 bits) and must be TMA-addressable.
cudaError_t launch_xeng_tc_raw_jobs(const TcJobSpec* specs, const CUtensorMap* maps, int n_jobs, int accumulate,
                                    int* status, int n_sm, const TcTuning& tune, cudaStream_t s);

}  // namespace corr

// X stage for callers that cannot allocate device memory.
//
// The plan-based entry points take a caller-allocated workspace (the unpacked sample
// planes).  Some callers cannot provide one: a real-time acquisition loop that must never
// call cudaMalloc/cudaFree (both synchronise the device and would stall the streams that
// keep up with the telescope), or a host framework that owns every byte of device memory
// and forbids its plug-ins from allocating.  corr_xengine_run_static serves them: it
// keeps the planes in a fixed array compiled into this library, so the call allocates
// nothing; the caller still passes the packed samples and the visibility buffer.
//
// The array lives in every GPU that loads this library until the process exits, so it is
// kept modest (64 MiB).  All calls share it and it keeps the last call's contents; the
// unpack kernel rewrites every byte a call reads (zero padding included), so nothing
// needs clearing except the small status block, which each call zeroes on its stream.
// Calls whose work overlaps on the GPU (different streams, or different host threads on
// the same device) race on the array and must be serialised by the caller.
#include <mutex>

#include "corr_internal.h"

static constexpr size_t kStaticScratchBytes = size_t(64) << 20;

static __device__ __align__(256) unsigned char corr_static_scratch[kStaticScratchBytes];
static __device__ __align__(256) int corr_static_status[4];

namespace corr {
namespace {

constexpr int kMaxDevices = 64;

struct StaticSlots {
    std::mutex mu;
    void* scratch[kMaxDevices] = {};
    int* status[kMaxDevices] = {};
};

StaticSlots& slots() {
    static StaticSlots s;
    return s;
}

// Device addresses of the two arrays for the current device, looked up once per device
// (the host-side names are only stand-ins, never device addresses).
corr_status static_addresses(int dev, void** scratch, int** status) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(CORR_EINVAL, "device ordinal %d out of range", dev);
    StaticSlots& s = slots();
    std::lock_guard<std::mutex> lock(s.mu);
    if (!s.scratch[dev]) {
        void* a = nullptr;
        void* b = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, corr_static_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
        e = cudaGetSymbolAddress(&b, corr_static_status);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(status)");
        s.scratch[dev] = a;
        s.status[dev] = static_cast<int*>(b);
    }
    *scratch = s.scratch[dev];
    *status = s.status[dev];
    return CORR_OK;
}

}  // namespace
}  // namespace corr

using namespace corr;

extern "C" corr_status corr_xengine_run_static(const void* d_packed, int n_inputs, int n_chan, int n_time,
                                               int sample_bits, void* d_vis, int accumulate, void* stream) {
    if (!d_packed || !d_vis) return set_error(CORR_EINVAL, "corr_xengine_run_static: NULL argument");
    if (((uintptr_t)d_packed & 15u) || ((uintptr_t)d_vis & 15u))
        return set_error(CORR_EINVAL, "corr_xengine_run_static: pointers must be 16-byte aligned");
    if (sample_bits != 4 && sample_bits != 8)
        return set_error(CORR_EINVAL, "corr_xengine_run_static: sample_bits=%d (4 or 8 only)", sample_bits);
    if (n_inputs < 1 || n_inputs > kMaxInputs || n_chan < 1 || n_time < 1)
        return set_error(CORR_EINVAL, "corr_xengine_run_static: bad sizes N=%d C=%d T=%d", n_inputs, n_chan, n_time);
    if (accumulate != 0 && accumulate != 1) return set_error(CORR_EINVAL, "accumulate must be 0 or 1");
    Plan p;
    p.n_inputs = n_inputs;
    p.n_chan = n_chan;
    p.n_time = n_time;
    p.sample_bits = sample_bits;
    p.nb = (n_inputs + kBlockInputs - 1) / kBlockInputs;
    p.kp = (n_time + kTimeBlock - 1) / kTimeBlock * kTimeBlock;
    p.n_baselines = n_baselines(n_inputs);
    const size_t need = planes_bytes(p, 1);
    if (need > kStaticScratchBytes)
        return set_error(CORR_EINVAL,
                         "corr_xengine_run_static: this dump needs %zu bytes of sample planes, more than the "
                         "built-in %zu-byte array; use corr_xengine_run with a workspace",
                         need, kStaticScratchBytes);
    cudaError_t e = cudaGetDevice(&p.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&p.n_sm, cudaDevAttrMultiProcessorCount, p.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
    void* scratch = nullptr;
    corr_status st = static_addresses(p.device, &scratch, &p.d_status);
    if (st != CORR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(p.d_status, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(status)");
    e = launch_unpack_fp16(p, d_packed, 1, scratch, s);
    if (e == cudaSuccess) e = launch_xeng_tc(p, scratch, nullptr, 1, d_vis, accumulate, s);
    if (e != cudaSuccess) return cuda_error(e, "X-stage launch");
    return CORR_OK;
}

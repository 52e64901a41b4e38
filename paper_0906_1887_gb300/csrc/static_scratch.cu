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
// needs clearing except the small status block, which each call zeroes on its stream and
// corr_static_check reads and clears.  Calls whose work overlaps on the GPU (different
// streams, or different host threads on the same device) race on the array and must be
// serialised by the caller.
//
// Host code never hands the arrays' names to a kernel (on the host they are stand-ins, not
// device addresses): the device addresses are looked up with cudaGetSymbolAddress, with the
// device current, once per device and CUDA context, and looked up again if the context
// changes (after cudaDeviceReset the module can load at another address).
#include <climits>
#include <mutex>

#include "corr_internal.h"

static constexpr size_t kStaticScratchBytes = size_t(64) << 20;

static __device__ __align__(256) unsigned char corr_static_scratch[kStaticScratchBytes];
static __device__ __align__(256) int corr_static_status[4];

namespace corr {
namespace {

constexpr int kMaxDevices = 64;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry-point query (no link against libcuda)
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    return fn;
}

struct StaticSlots {
    std::mutex mu;
    CUcontext ctx[kMaxDevices] = {};
    void* scratch[kMaxDevices] = {};
    int* status[kMaxDevices] = {};
};

StaticSlots& slots() {
    static StaticSlots s;
    return s;
}

// Device addresses of the two arrays for the current device and context.
corr_status static_addresses(int dev, void** scratch, int** status) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(CORR_EINVAL, "device ordinal %d out of range", dev);
    CUcontext ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (!get || get(&ctx) != CUDA_SUCCESS)
        return set_error(CORR_ECUDA, "cuCtxGetCurrent is unavailable or failed");
    StaticSlots& s = slots();
    std::lock_guard<std::mutex> lock(s.mu);
    if (!s.scratch[dev] || s.ctx[dev] != ctx) {
        void* a = nullptr;
        void* b = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, corr_static_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
        e = cudaGetSymbolAddress(&b, corr_static_status);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(status)");
        // the context is current now (the runtime made it so for the lookups)
        if (get(&ctx) != CUDA_SUCCESS) return set_error(CORR_ECUDA, "cuCtxGetCurrent failed");
        s.ctx[dev] = ctx;
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
    // the size check comes before any product that could wrap: n_time + 63 must not overflow,
    // and the plane bytes are first formed in double precision
    if (n_time > INT_MAX - kTimeBlock)
        return set_error(CORR_EINVAL, "corr_xengine_run_static: n_time=%d too large", n_time);
    const int nb = (n_inputs + kBlockInputs - 1) / kBlockInputs;
    const int kp = (n_time + kTimeBlock - 1) / kTimeBlock * kTimeBlock;
    const double need_d = (double)n_chan * (double)nb * kBlockRows * (double)kp * 2.0;
    if (need_d > (double)kStaticScratchBytes)
        return set_error(CORR_EINVAL,
                         "corr_xengine_run_static: this dump needs %.0f bytes of sample planes, more than the "
                         "built-in %zu-byte array; use corr_xengine_run with a workspace",
                         need_d, kStaticScratchBytes);
    Plan p;
    p.n_inputs = n_inputs;
    p.n_chan = n_chan;
    p.n_time = n_time;
    p.sample_bits = sample_bits;
    p.nb = nb;
    p.kp = kp;
    p.n_baselines = n_baselines(n_inputs);
    if (tc_workspace_planes_bytes(p, 1) > kStaticScratchBytes)   // cannot happen after the check above
        return set_error(CORR_EINVAL, "corr_xengine_run_static: plane size check failed");
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
    e = launch_tc_plane_path(p, d_packed, 1, scratch, d_vis, accumulate, s);
    if (e != cudaSuccess) return cuda_error(e, "X-stage launch");
    return CORR_OK;
}

extern "C" corr_status corr_static_check(int* device_error, void* stream) {
    if (!device_error) return set_error(CORR_EINVAL, "corr_static_check: device_error is NULL");
    *device_error = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    void* scratch = nullptr;
    int* d_status = nullptr;
    corr_status st = static_addresses(dev, &scratch, &d_status);
    if (st != CORR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int h[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(h, d_status, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(h), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "corr_static_check");
    *device_error = h[0];
    if (h[0] != 0) return set_error(CORR_ETIMEOUT, "device reported error %d (detail %d)", h[0], h[1]);
    return CORR_OK;
}

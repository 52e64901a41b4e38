// C ABI of libcorr: plans, validation, dispatch of the X-stage engines.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "corr_internal.h"

namespace corr {

static thread_local char g_msg[512] = "";

corr_status set_error(corr_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

corr_status cuda_error(cudaError_t e, const char* what) {
    return set_error(CORR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t plane_elem_bytes(const Plan& p) { return p.sample_bits == 32 ? 4 : 2; }

size_t planes_bytes(const Plan& p, int n_dumps) {
    return (size_t)n_dumps * (size_t)p.n_chan * (size_t)p.nb * kBlockRows * (size_t)p.kp * plane_elem_bytes(p);
}

size_t tc_workspace_planes_bytes(const Plan& p, int n_dumps) {
    if (tc_planes_e4m3(p))
        return (size_t)n_dumps * (size_t)p.n_chan * (size_t)p.nb * kBlockRows * (size_t)tc_kp_e4m3(p);
    return planes_bytes(p, n_dumps);
}

static size_t packed_bytes_one(const Plan& p) {
    size_t per = p.sample_bits == 4 ? 1 : (p.sample_bits == 8 ? 2 : 8);
    return (size_t)p.n_time * (size_t)p.n_chan * (size_t)p.n_inputs * per;
}

static size_t vis_bytes_one(const Plan& p) {
    size_t per = p.sample_bits == 32 ? 8 : 16;
    return (size_t)p.n_baselines * (size_t)p.n_chan * per;
}

static bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

}  // namespace corr

using namespace corr;

extern "C" {

int corr_version(void) { return CORR_VERSION; }  // 0.2.0

const char* corr_last_error(void) { return g_msg; }

corr_status corr_plan_create(corr_plan* out, int n_inputs, int n_chan, int n_time, int sample_bits) {
    g_msg[0] = 0;
    if (!out) return set_error(CORR_EINVAL, "corr_plan_create: out is NULL");
    *out = nullptr;
    if (n_inputs < 1 || n_inputs > kMaxInputs)
        return set_error(CORR_EINVAL, "n_inputs=%d outside [1, %d]", n_inputs, kMaxInputs);
    if (n_chan < 1) return set_error(CORR_EINVAL, "n_chan=%d must be >= 1", n_chan);
    if (n_time < 1) return set_error(CORR_EINVAL, "n_time=%d must be >= 1", n_time);
    if (sample_bits != 4 && sample_bits != 8 && sample_bits != 32)
        return set_error(CORR_EINVAL, "sample_bits=%d must be 4, 8 or 32", sample_bits);
    Plan tmp;
    tmp.n_inputs = n_inputs;
    tmp.n_chan = n_chan;
    tmp.n_time = n_time;
    tmp.sample_bits = sample_bits;
    tmp.nb = (n_inputs + kBlockInputs - 1) / kBlockInputs;
    tmp.kp = (n_time + kTimeBlock - 1) / kTimeBlock * kTimeBlock;
    tmp.n_baselines = n_baselines(n_inputs);
    // keep every element index of a dump's planes and visibilities inside int64 comfortably
    double planes = (double)n_chan * tmp.nb * kBlockRows * (double)tmp.kp;
    double vis = (double)n_chan * (double)tmp.n_baselines * 2.0;
    if (planes > 4.0e15 || vis > 4.0e15) return set_error(CORR_EINVAL, "problem too large");
    cudaError_t e = cudaGetDevice(&tmp.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&tmp.n_sm, cudaDevAttrMultiProcessorCount, tmp.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
    e = cudaMalloc((void**)&tmp.d_status, 4 * sizeof(int));
    if (e != cudaSuccess) return set_error(CORR_ENOMEM, "cudaMalloc(status): %s", cudaGetErrorString(e));
    e = cudaMemset(tmp.d_status, 0, 4 * sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(tmp.d_status);
        return cuda_error(e, "cudaMemset(status)");
    }
    Plan* p = new (std::nothrow) Plan(tmp);
    if (!p) {
        cudaFree(tmp.d_status);
        return set_error(CORR_ENOMEM, "host allocation of plan failed");
    }
    *out = reinterpret_cast<corr_plan>(p);
    return CORR_OK;
}

corr_status corr_plan_destroy(corr_plan plan) {
    if (!plan) return set_error(CORR_EINVAL, "corr_plan_destroy: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    for (auto& st : p->pipe_stream)
        if (st) cudaStreamDestroy(st);
    for (auto& ev : p->pipe_ev)
        if (ev) cudaEventDestroy(ev);
    if (p->pipe_dev) cudaFree(p->pipe_dev);
    if (p->d_status) cudaFree(p->d_status);
    delete p;
    return CORR_OK;
}

corr_status corr_plan_info(corr_plan plan, int64_t* n_bl, size_t* packed_bytes, size_t* vis_bytes) {
    if (!plan) return set_error(CORR_EINVAL, "corr_plan_info: plan is NULL");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    if (n_bl) *n_bl = p->n_baselines;
    if (packed_bytes) *packed_bytes = packed_bytes_one(*p);
    if (vis_bytes) *vis_bytes = vis_bytes_one(*p);
    return CORR_OK;
}

corr_status corr_plan_set_tuning(corr_plan plan, int op_stages, int float_planes) {
    if (!plan) return set_error(CORR_EINVAL, "corr_plan_set_tuning: plan is NULL");
    if (op_stages < 0 || op_stages > 16) return set_error(CORR_EINVAL, "op_stages=%d outside [0, 16]", op_stages);
    if (float_planes < 0 || float_planes > 1)
        return set_error(CORR_EINVAL, "float_planes=%d outside [0, 1]", float_planes);
    reinterpret_cast<Plan*>(plan)->tc_op_stages = op_stages;
    reinterpret_cast<Plan*>(plan)->tc_float_planes = float_planes;
    return CORR_OK;
}

corr_status corr_plan_set_operands(corr_plan plan, int operands, int items) {
    if (!plan) return set_error(CORR_EINVAL, "corr_plan_set_operands: plan is NULL");
    if (operands < CORR_OPERANDS_AUTO || operands > CORR_OPERANDS_PACKED_F8)
        return set_error(CORR_EINVAL, "operands=%d is not a CORR_OPERANDS_* value", operands);
    if (items < CORR_ITEMS_AUTO || items > CORR_ITEMS_WIDE)
        return set_error(CORR_EINVAL, "items=%d is not a CORR_ITEMS_* value", items);
    Plan* p = reinterpret_cast<Plan*>(plan);
    if ((operands == CORR_OPERANDS_PACKED || operands == CORR_OPERANDS_PACKED_F8) && !tc_raw_supported(*p))
        return set_error(CORR_EUNSUPPORTED, "packed rows of %d inputs are not 16-byte multiples: planes only",
                         p->n_inputs);
    if (operands == CORR_OPERANDS_PACKED_F8 && p->sample_bits != 4)
        return set_error(CORR_EUNSUPPORTED, "e4m3 operands hold 4-bit samples exactly, not %d-bit ones",
                         p->sample_bits);
    p->tc_operands = operands;
    p->tc_items = items;
    return CORR_OK;
}

corr_status corr_workspace_size(corr_plan plan, int engine, int n_dumps, size_t* bytes) {
    if (!plan || !bytes) return set_error(CORR_EINVAL, "corr_workspace_size: NULL argument");
    if (n_dumps < 1) return set_error(CORR_EINVAL, "n_dumps=%d must be >= 1", n_dumps);
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    switch (engine) {
        case CORR_ENGINE_TC:
            // fp16 planes when the kernel reads planes (required where TMA cannot address the
            // packed rows; optional otherwise: without a workspace it converts packed samples)
            *bytes = tc_use_planes(*p) ? tc_workspace_planes_bytes(*p, n_dumps) : 0;
            return CORR_OK;
        case CORR_ENGINE_FP32:
            *bytes = 0;   // reads the packed samples directly
            return CORR_OK;
        case CORR_ENGINE_BF16X3:
            // hi and lo bf16 planes, unless the tensor-core kernel splits the floats itself
            *bytes = (!p->tc_float_planes && tc_rawf32_supported(*p))
                         ? 0
                         : (size_t)n_dumps * p->n_chan * (size_t)p->nb * kBlockRows * (size_t)p->kp * 2 * 2;
            return CORR_OK;
        default:
            return set_error(CORR_EINVAL, "unknown engine %d", engine);
    }
}

corr_status corr_planes_size(corr_plan plan, int n_dumps, size_t* bytes) {
    if (!plan || !bytes) return set_error(CORR_EINVAL, "corr_planes_size: NULL argument");
    if (n_dumps < 1) return set_error(CORR_EINVAL, "n_dumps=%d must be >= 1", n_dumps);
    *bytes = planes_bytes(*reinterpret_cast<const Plan*>(plan), n_dumps);
    return CORR_OK;
}

corr_status corr_unpack(corr_plan plan, const void* d_packed, int n_dumps, void* d_planes, void* stream) {
    if (!plan || !d_packed || !d_planes) return set_error(CORR_EINVAL, "corr_unpack: NULL argument");
    if (n_dumps < 1) return set_error(CORR_EINVAL, "n_dumps=%d must be >= 1", n_dumps);
    if (!aligned16(d_packed) || !aligned16(d_planes))
        return set_error(CORR_EINVAL, "corr_unpack: pointers must be 16-byte aligned");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = p->sample_bits == 32 ? launch_unpack_f32(*p, d_packed, n_dumps, d_planes, s)
                                         : launch_unpack_fp16(*p, d_packed, n_dumps, d_planes, s);
    if (e != cudaSuccess) return cuda_error(e, "unpack launch");
    return CORR_OK;
}

corr_status corr_xengine_run_batch(corr_plan plan, const void* d_packed, int n_dumps, void* d_vis,
                                   void* d_workspace, int accumulate, int engine, void* stream) {
    if (!plan || !d_packed || !d_vis) return set_error(CORR_EINVAL, "corr_xengine_run: NULL argument");
    if (n_dumps < 1) return set_error(CORR_EINVAL, "n_dumps=%d must be >= 1", n_dumps);
    if (accumulate != 0 && accumulate != 1) return set_error(CORR_EINVAL, "accumulate must be 0 or 1");
    if (!aligned16(d_packed) || !aligned16(d_vis) || (d_workspace && !aligned16(d_workspace)))
        return set_error(CORR_EINVAL, "corr_xengine_run: pointers must be 16-byte aligned");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t need = 0;
    corr_status st = corr_workspace_size(plan, engine, n_dumps, &need);
    if (st != CORR_OK) return st;
    // the tensor-core engine's planes are optional where the kernel can read the packed rows
    // itself (the automatic choice), so a NULL workspace takes the fused path there
    const bool tc_fused_ok = engine == CORR_ENGINE_TC && p->sample_bits != 32 && tc_raw_supported(*p) &&
                             p->tc_operands != 2;
    if (need && !d_workspace && !tc_fused_ok)
        return set_error(CORR_EINVAL, "engine %d needs %zu bytes of workspace", engine, need);
    cudaError_t e = cudaSuccess;
    if (engine == CORR_ENGINE_TC) {
        if (p->sample_bits == 32)
            return set_error(CORR_EUNSUPPORTED, "float samples run on CORR_ENGINE_BF16X3 or CORR_ENGINE_FP32");
        if (!d_workspace || !tc_use_planes(*p)) {
            e = launch_xeng_tc_raw(*p, d_packed, n_dumps, d_vis, accumulate, s);
        } else {
            e = launch_tc_plane_path(*p, d_packed, n_dumps, d_workspace, d_vis, accumulate, s);
        }
    } else if (engine == CORR_ENGINE_FP32) {
        e = launch_xeng_fp32_packed(*p, d_packed, n_dumps, d_vis, accumulate, s);
    } else if (engine == CORR_ENGINE_BF16X3) {
        if (p->sample_bits != 32)
            return set_error(CORR_EUNSUPPORTED, "CORR_ENGINE_BF16X3 takes float samples (sample_bits=32)");
        if (need == 0) {   // fused: TMA loads the floats, the converter warps split them
            e = launch_xeng_tc_rawf32(*p, d_packed, n_dumps, d_vis, accumulate, s);
        } else {
            char* hi = static_cast<char*>(d_workspace);
            char* lo = hi + need / 2;
            e = launch_unpack_bf16x2(*p, d_packed, n_dumps, hi, lo, s);
            if (e == cudaSuccess) e = launch_xeng_tc(*p, hi, lo, n_dumps, d_vis, accumulate, s);
        }
    } else {
        return set_error(CORR_EINVAL, "unknown engine %d", engine);
    }
    if (e != cudaSuccess) return cuda_error(e, "X-stage launch");
    return CORR_OK;
}

corr_status corr_xengine_run_planes(corr_plan plan, const void* d_planes, int n_dumps, void* d_vis, int accumulate,
                                    int engine, void* stream) {
    if (!plan || !d_planes || !d_vis) return set_error(CORR_EINVAL, "corr_xengine_run_planes: NULL argument");
    if (n_dumps < 1) return set_error(CORR_EINVAL, "n_dumps=%d must be >= 1", n_dumps);
    if (accumulate != 0 && accumulate != 1) return set_error(CORR_EINVAL, "accumulate must be 0 or 1");
    if (!aligned16(d_planes) || !aligned16(d_vis))
        return set_error(CORR_EINVAL, "corr_xengine_run_planes: pointers must be 16-byte aligned");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (engine == CORR_ENGINE_TC) {
        if (p->sample_bits == 32)
            return set_error(CORR_EUNSUPPORTED, "float samples run on CORR_ENGINE_BF16X3 or CORR_ENGINE_FP32");
        e = launch_xeng_tc(*p, d_planes, nullptr, n_dumps, d_vis, accumulate, s);
    } else if (engine == CORR_ENGINE_FP32) {
        e = launch_xeng_fp32(*p, d_planes, n_dumps, d_vis, accumulate, s);
    } else {
        return set_error(CORR_EUNSUPPORTED, "corr_xengine_run_planes takes CORR_ENGINE_TC or CORR_ENGINE_FP32");
    }
    if (e != cudaSuccess) return cuda_error(e, "X-stage launch");
    return CORR_OK;
}

corr_status corr_xengine_run(corr_plan plan, const void* d_packed, void* d_vis, void* d_workspace, int accumulate,
                             int engine, void* stream) {
    return corr_xengine_run_batch(plan, d_packed, 1, d_vis, d_workspace, accumulate, engine, stream);
}

corr_status corr_xengine_run_host(corr_plan plan, const void* host_packed, int n_dumps, void* host_vis,
                                  int dumps_per_chunk, int engine) {
    if (!plan || !host_packed || !host_vis) return set_error(CORR_EINVAL, "corr_xengine_run_host: NULL argument");
    if (n_dumps < 1) return set_error(CORR_EINVAL, "n_dumps=%d must be >= 1", n_dumps);
    Plan* p = reinterpret_cast<Plan*>(plan);
    const size_t in1 = packed_bytes_one(*p), out1 = vis_bytes_one(*p);
    int chunk = dumps_per_chunk;
    if (chunk <= 0) {   // default: about 256 MB of samples per chunk
        chunk = (int)((size_t)256 << 20) / (int)(in1 > 0 ? in1 : 1);
        if (chunk < 1) chunk = 1;
    }
    if (chunk > n_dumps) chunk = n_dumps;
    size_t ws = 0;
    corr_status st = corr_workspace_size(plan, engine, chunk, &ws);
    if (st != CORR_OK) return st;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t in_c = up(in1 * chunk), out_c = up(out1 * chunk);
    const size_t need = 2 * in_c + 2 * out_c + up(ws);
    cudaError_t e = cudaSuccess;
    if (need > p->pipe_bytes) {
        if (p->pipe_dev) cudaFree(p->pipe_dev);
        p->pipe_dev = nullptr;
        p->pipe_bytes = 0;
        e = cudaMalloc((void**)&p->pipe_dev, need);
        if (e != cudaSuccess) return set_error(CORR_ENOMEM, "cudaMalloc(%zu) for the host pipeline failed", need);
        p->pipe_bytes = need;
    }
    for (auto& s : p->pipe_stream)
        if (!s && e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (auto& ev : p->pipe_ev)
        if (!ev && e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_error(e, "host pipeline set-up");
    cudaStream_t s_in = p->pipe_stream[0], s_x = p->pipe_stream[1], s_out = p->pipe_stream[2];
    // events per buffer b: in_ready[b] = pipe_ev[b], x_done[b] = pipe_ev[2 + b], out_free[b] = pipe_ev[4 + b]
    char* in_buf[2] = {p->pipe_dev, p->pipe_dev + in_c};
    char* out_buf[2] = {p->pipe_dev + 2 * in_c, p->pipe_dev + 2 * in_c + out_c};
    char* wsp = ws ? p->pipe_dev + 2 * in_c + 2 * out_c : nullptr;
    const int n_chunks = (n_dumps + chunk - 1) / chunk;
    for (int k = 0; k < n_chunks && st == CORR_OK; ++k) {
        const int b = k & 1;
        const int nd = (k == n_chunks - 1) ? n_dumps - k * chunk : chunk;
        // copy in: the buffer is free once the X stage of chunk k - 2 finished with it
        if (k >= 2) e = cudaStreamWaitEvent(s_in, p->pipe_ev[2 + b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(in_buf[b], static_cast<const char*>(host_packed) + (size_t)k * chunk * in1, in1 * nd,
                                cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaEventRecord(p->pipe_ev[b], s_in);
        // X stage: needs the samples and a drained output buffer
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_x, p->pipe_ev[b], 0);
        if (e == cudaSuccess && k >= 2) e = cudaStreamWaitEvent(s_x, p->pipe_ev[4 + b], 0);
        if (e != cudaSuccess) break;
        st = corr_xengine_run_batch(plan, in_buf[b], nd, out_buf[b], wsp, 0, engine, s_x);
        if (st != CORR_OK) break;
        e = cudaEventRecord(p->pipe_ev[2 + b], s_x);
        // copy out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, p->pipe_ev[2 + b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char*>(host_vis) + (size_t)k * chunk * out1, out_buf[b], out1 * nd,
                                cudaMemcpyDeviceToHost, s_out);
        if (e == cudaSuccess) e = cudaEventRecord(p->pipe_ev[4 + b], s_out);
    }
    cudaError_t e2 = cudaStreamSynchronize(s_out);
    cudaError_t e3 = cudaStreamSynchronize(s_x);
    cudaError_t e4 = cudaStreamSynchronize(s_in);
    if (st != CORR_OK) return st;
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4);
    if (e != cudaSuccess) return cuda_error(e, "host pipeline");
    return CORR_OK;
}

corr_status corr_selftest_stall(corr_plan plan, const void* d_packed, void* d_vis, int stall_item, int wait_limit_ms,
                                int* device_error) {
    if (!plan || !d_packed || !d_vis || !device_error) return set_error(CORR_EINVAL, "corr_selftest_stall: NULL argument");
    if (wait_limit_ms < 1 || wait_limit_ms > 10000) return set_error(CORR_EINVAL, "wait_limit_ms outside [1, 10000]");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (!tc_raw_supported(*p))
        return set_error(CORR_EUNSUPPORTED, "the self-test runs the packed-sample tensor-core kernel");
    TcTuning tune;
    tune.op_stages = p->tc_op_stages;
    tune.wait_limit_ns = (uint64_t)wait_limit_ms * 1000000ull;
    tune.stall_item = stall_item;
    cudaError_t e = launch_xeng_tc_raw(*p, d_packed, 1, d_vis, 0, nullptr, &tune);
    if (e != cudaSuccess) return cuda_error(e, "self-test launch");
    return corr_plan_check(plan, device_error);
}

corr_status corr_plan_check(corr_plan plan, int* device_error) {
    if (!plan) return set_error(CORR_EINVAL, "corr_plan_check: plan is NULL");
    Plan* p = reinterpret_cast<Plan*>(plan);
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
    e = cudaMemcpy(h, p->d_status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(status)");
    e = cudaMemset(p->d_status, 0, sizeof(h));
    if (e != cudaSuccess) return cuda_error(e, "cudaMemset(status)");
    if (device_error) *device_error = h[0];
    if (h[0] != 0) return set_error(CORR_ETIMEOUT, "device reported error %d (detail %d)", h[0], h[1]);
    return CORR_OK;
}

corr_status corr_average_host(const int64_t* vis, size_t n_values, int64_t n_accum, double* out) {
    if (!vis || !out) return set_error(CORR_EINVAL, "corr_average_host: NULL argument");
    if (n_accum < 1) return set_error(CORR_EINVAL, "n_accum=%lld must be >= 1", (long long)n_accum);
    const double n = (double)n_accum;
    for (size_t k = 0; k < n_values; ++k) out[k] = (double)vis[k] / n;
    return CORR_OK;
}

}  // extern "C"

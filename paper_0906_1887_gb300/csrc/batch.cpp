// Batched X stage: many uneven correlation jobs in one persistent tensor-core launch per
// sample mode, optionally autotuned and captured in a CUDA graph.
//
// The paper runs large batches per GPU call so that launch and transfer overhead vanish
// (Sec. 4, Sec. 5: no gain beyond ~20 batches of samples).  Here the batch is across
// jobs: arrays of different sizes, channel counts and dump lengths are packed into one
// flat list of work items walked by one grid of persistent CTAs, so small jobs no longer
// pay a launch each and large ones no longer leave SMs idle at their tail.
//
// Autotuning: per job-set signature the tuner times each candidate launch shape
// (operand-ring depth, channels per work item for single-block arrays, item order) on the
// batch's own buffers and keeps the fastest; results are cached in memory and, when a
// cache path is given, in a JSON-lines file.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "corr_internal.h"

namespace corr {
namespace {

struct TuneChoice {
    int op_stages = 0;   // 0: default
    int pair_cpi = 2;    // channels per item for arrays of <= 64 inputs
    int order = 0;       // 0: items of the costliest jobs first; 1: jobs in the caller's order
    float ms = 0.f;
};

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;

struct ModeGroup {
    int bits = 0;
    std::vector<int> job_index;           // caller's job indices in this group
    std::vector<TcJobSpec> specs;         // launch order
    std::vector<CUtensorMap> maps;
    TcTuning tune{};
};

}  // namespace
}  // namespace corr

struct corr_batch_s {
    int device = 0;
    int n_sm = 0;
    int accumulate = 0;
    std::vector<corr_job> jobs;
    std::vector<corr::ModeGroup> groups;  // one per sample mode present
    int* d_status = nullptr;
    bool graph = false;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t gx = nullptr;
    cudaStream_t own_stream = nullptr;
    double cmacs = 0.0;
    int64_t items = 0;
    corr::TuneChoice choice;
    bool tuned = false;
};

namespace corr {
namespace {

double job_cost_per_item(const corr_job& j, int cpi) {
    const int nb = (j.n_inputs + kBlockInputs - 1) / kBlockInputs;
    const int nkb = (j.n_time + kTimeBlock - 1) / kTimeBlock;
    return (double)nkb * (nb == 1 ? cpi : 2);
}

// (Re)build the launch groups for a tuning choice.
bool build_groups(corr_batch_s* b, const TuneChoice& ch) {
    b->groups.clear();
    b->items = 0;
    for (int bits : {8, 4}) {
        ModeGroup g;
        g.bits = bits;
        for (int k = 0; k < (int)b->jobs.size(); ++k)
            if (b->jobs[k].sample_bits == bits) g.job_index.push_back(k);
        if (g.job_index.empty()) continue;
        auto cpi_of = [&](const corr_job& j) { return j.n_inputs <= kBlockInputs ? ch.pair_cpi : 1; };
        if (ch.order == 0)
            std::stable_sort(g.job_index.begin(), g.job_index.end(), [&](int x, int y) {
                return job_cost_per_item(b->jobs[x], cpi_of(b->jobs[x])) >
                       job_cost_per_item(b->jobs[y], cpi_of(b->jobs[y]));
            });
        for (int k : g.job_index) {
            const corr_job& j = b->jobs[k];
            TcJobSpec sp{j.n_inputs, j.n_chan, j.n_time, 1, j.sample_bits, j.packed, j.vis, cpi_of(j)};
            CUtensorMap m;
            if (!tc_make_raw_map(&m, sp)) return false;
            g.specs.push_back(sp);
            g.maps.push_back(m);
            const int nb = (j.n_inputs + kBlockInputs - 1) / kBlockInputs;
            b->items += (int64_t)((j.n_chan + sp.cpi - 1) / sp.cpi) * (nb * (nb + 1) / 2);
        }
        g.tune.op_stages = ch.op_stages;
        b->groups.push_back(std::move(g));
    }
    return true;
}

cudaError_t launch_groups(corr_batch_s* b, cudaStream_t s) {
    for (auto& g : b->groups) {
        // at most kMaxJobs jobs per launch
        for (size_t k0 = 0; k0 < g.specs.size(); k0 += kMaxJobsPerLaunch) {
            const int n = (int)std::min(g.specs.size() - k0, (size_t)kMaxJobsPerLaunch);
            cudaError_t e = launch_xeng_tc_raw_jobs(g.specs.data() + k0, g.maps.data() + k0, n, b->accumulate,
                                                    b->d_status, b->n_sm, g.tune, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

std::string signature(const corr_batch_s* b) {
    std::vector<std::string> parts;
    for (const auto& j : b->jobs) {
        char buf[96];
        snprintf(buf, sizeof(buf), "%d:%d:%d:%d", j.sample_bits, j.n_inputs, j.n_chan, j.n_time);
        parts.push_back(buf);
    }
    std::sort(parts.begin(), parts.end());
    std::string key;
    for (auto& p : parts) key += p + ",";
    return key;
}

void load_cache_file(const char* path) {
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[65536];
    while (fgets(line, sizeof(line), f)) {
        // {"key": "...", "op_stages": A, "pair_cpi": B, "order": C, "ms": D}
        char* k0 = strstr(line, "\"key\": \"");
        if (!k0) continue;
        k0 += 8;
        char* k1 = strchr(k0, '"');
        if (!k1) continue;
        std::string key(k0, k1 - k0);
        TuneChoice c;
        const char* p;
        if ((p = strstr(k1, "\"op_stages\": "))) c.op_stages = atoi(p + 13);
        if ((p = strstr(k1, "\"pair_cpi\": "))) c.pair_cpi = atoi(p + 12);
        if ((p = strstr(k1, "\"order\": "))) c.order = atoi(p + 9);
        if ((p = strstr(k1, "\"ms\": "))) c.ms = (float)atof(p + 6);
        if (c.pair_cpi != 1 && c.pair_cpi != 2) continue;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = c;
    }
    fclose(f);
}

void append_cache_file(const char* path, const std::string& key, const TuneChoice& c) {
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"op_stages\": %d, \"pair_cpi\": %d, \"order\": %d, \"ms\": %.6f}\n", key.c_str(),
            c.op_stages, c.pair_cpi, c.order, c.ms);
    fclose(f);
}

// Median time (ms) of `reps` runs of the current groups on `s`.
float time_groups(corr_batch_s* b, cudaStream_t s, int reps, cudaError_t* err) {
    cudaEvent_t e0, e1;
    *err = cudaEventCreate(&e0);
    if (*err != cudaSuccess) return 0.f;
    *err = cudaEventCreate(&e1);
    if (*err != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0.f;
    }
    *err = launch_groups(b, s);   // warm-up (also sets kernel attributes)
    std::vector<float> t;
    for (int r = 0; r < reps && *err == cudaSuccess; ++r) {
        cudaEventRecord(e0, s);
        *err = launch_groups(b, s);
        cudaEventRecord(e1, s);
        if (*err == cudaSuccess) *err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (*err == cudaSuccess) *err = cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (t.empty()) return 0.f;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

corr_status autotune(corr_batch_s* b, const char* cache_path) {
    const std::string key = signature(b);
    load_cache_file(cache_path);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->choice = it->second;
            b->tuned = true;
            return build_groups(b, b->choice) ? CORR_OK : set_error(CORR_EINVAL, "tensor map encoding failed");
        }
    }
    bool any_small = false;
    for (const auto& j : b->jobs) any_small = any_small || j.n_inputs <= kBlockInputs;
    std::vector<TuneChoice> cands;
    for (int order : {0, 1})
        for (int cpi : any_small ? std::vector<int>{2, 1} : std::vector<int>{2})
            for (int ops : {3, 4, 5}) {
                TuneChoice c;
                c.op_stages = ops;
                c.pair_cpi = cpi;
                c.order = order;
                cands.push_back(c);
            }
    TuneChoice best;
    float best_ms = 1e30f;
    cudaStream_t s = b->own_stream;
    for (auto& c : cands) {
        if (!build_groups(b, c)) return set_error(CORR_EINVAL, "tensor map encoding failed");
        cudaError_t err;
        const float ms = time_groups(b, s, 3, &err);
        if (err != cudaSuccess) return cuda_error(err, "autotune run");
        c.ms = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    b->choice = best;
    b->tuned = true;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    append_cache_file(cache_path, key, best);
    return build_groups(b, best) ? CORR_OK : set_error(CORR_EINVAL, "tensor map encoding failed");
}

}  // namespace
}  // namespace corr

using namespace corr;

extern "C" {

corr_status corr_batch_create(corr_batch* out, const corr_job* jobs, int n_jobs, int flags, const char* tune_cache) {
    if (!out || !jobs || n_jobs < 1) return set_error(CORR_EINVAL, "corr_batch_create: bad arguments");
    *out = nullptr;
    double cm = 0.0;
    for (int k = 0; k < n_jobs; ++k) {
        const corr_job& j = jobs[k];
        if (j.sample_bits != 4 && j.sample_bits != 8)
            return set_error(CORR_EUNSUPPORTED, "job %d: batches take 4/8-bit samples", k);
        if (j.n_inputs < 1 || j.n_inputs > kMaxInputs || j.n_chan < 1 || j.n_time < 1)
            return set_error(CORR_EINVAL, "job %d: bad sizes", k);
        if (!tc_raw_supported(j.n_inputs, j.sample_bits))
            return set_error(CORR_EUNSUPPORTED,
                             "job %d: n_inputs * bytes per sample = %d is not a multiple of 16 (TMA row stride)", k,
                             j.n_inputs * (j.sample_bits == 8 ? 2 : 1));
        if (!j.packed || !j.vis || ((uintptr_t)j.packed & 15u) || ((uintptr_t)j.vis & 15u))
            return set_error(CORR_EINVAL, "job %d: pointers must be non-NULL and 16-byte aligned", k);
        cm += (double)n_baselines(j.n_inputs) * j.n_chan * j.n_time;
    }
    corr_batch_s* b = new (std::nothrow) corr_batch_s();
    if (!b) return set_error(CORR_ENOMEM, "host allocation failed");
    b->jobs.assign(jobs, jobs + n_jobs);
    b->accumulate = (flags & CORR_BATCH_ACCUMULATE) ? 1 : 0;
    b->cmacs = cm;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_status, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        corr_batch_destroy(b);
        return cuda_error(e, "corr_batch_create");
    }
    corr_status st = CORR_OK;
    if ((flags & CORR_BATCH_AUTOTUNE) && (flags & CORR_BATCH_ACCUMULATE)) {
        corr_batch_destroy(b);
        return set_error(CORR_EINVAL, "CORR_BATCH_AUTOTUNE with CORR_BATCH_ACCUMULATE would add tuning runs into "
                                      "the accumulators; tune without ACCUMULATE first (the choice is cached)");
    }
    if (flags & CORR_BATCH_AUTOTUNE) {
        st = autotune(b, tune_cache);
    } else if (!build_groups(b, TuneChoice{})) {
        st = set_error(CORR_EINVAL, "tensor map encoding failed");
    }
    if (st != CORR_OK) {
        corr_batch_destroy(b);
        return st;
    }
    if (flags & CORR_BATCH_GRAPH) {
        // one eager run sets the kernels' shared-memory attributes outside the capture
        e = launch_groups(b, b->own_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->own_stream);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->own_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = launch_groups(b, b->own_stream);
            e = cudaStreamEndCapture(b->own_stream, &b->g);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gx, b->g, 0);
        if (e != cudaSuccess) {
            corr_batch_destroy(b);
            return cuda_error(e, "CUDA graph capture of the batch");
        }
        b->graph = true;
    }
    *out = b;
    return CORR_OK;
}

corr_status corr_batch_run(corr_batch b, void* stream) {
    if (!b) return set_error(CORR_EINVAL, "corr_batch_run: NULL batch");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = b->graph ? cudaGraphLaunch(b->gx, s) : launch_groups(b, s);
    if (e != cudaSuccess) return cuda_error(e, "corr_batch_run");
    return CORR_OK;
}

corr_status corr_batch_info(corr_batch b, corr_batch_stats* st) {
    if (!b || !st) return set_error(CORR_EINVAL, "corr_batch_info: NULL argument");
    memset(st, 0, sizeof(*st));
    st->n_jobs = (int)b->jobs.size();
    st->n_items = b->items;
    st->cmacs = b->cmacs;
    int launches = 0;
    for (auto& g : b->groups) launches += (int)((g.specs.size() + kMaxJobsPerLaunch - 1) / kMaxJobsPerLaunch);
    st->n_launches = launches;
    st->graph = b->graph ? 1 : 0;
    st->tuned = b->tuned ? 1 : 0;
    st->op_stages = b->choice.op_stages;
    st->pair_cpi = b->choice.pair_cpi;
    st->order = b->choice.order;
    st->tune_ms = b->choice.ms;
    return CORR_OK;
}

corr_status corr_batch_check(corr_batch b, int* device_error) {
    if (!b) return set_error(CORR_EINVAL, "corr_batch_check: NULL batch");
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, b->d_status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(h));
    if (e != cudaSuccess) return cuda_error(e, "corr_batch_check");
    if (device_error) *device_error = h[0];
    if (h[0] != 0) return set_error(CORR_ETIMEOUT, "device reported error %d (detail %d)", h[0], h[1]);
    return CORR_OK;
}

corr_status corr_batch_destroy(corr_batch b) {
    if (!b) return set_error(CORR_EINVAL, "corr_batch_destroy: NULL batch");
    if (b->gx) cudaGraphExecDestroy(b->gx);
    if (b->g) cudaGraphDestroy(b->g);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    if (b->d_status) cudaFree(b->d_status);
    delete b;
    return CORR_OK;
}

}  // extern "C"

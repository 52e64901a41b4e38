// Batched X stage: many uneven correlation jobs in one persistent tensor-core launch per
// sample mode and operand path, optionally autotuned and captured in a CUDA graph.
//
// The paper runs large batches per GPU call so that launch and transfer overhead vanish
// (Sec. 4, Sec. 5: no gain beyond ~20 batches of samples).  Here the batch is across
// jobs: arrays of different sizes, channel counts and dump lengths are packed into one
// flat list of work items walked by one grid of persistent CTAs, so small jobs no longer
// pay a launch each and large ones no longer leave SMs idle at their tail.
//
// Operand path: the tensor-core kernel either converts packed samples itself (converter
// warps, the samples cross HBM once) or reads fp16 sample planes that the unpack kernel wrote
// first.  The first converts every 64-input block once per tile it meets, i.e. about nb/2
// times per channel for an array of nb blocks; the second converts each block once and
// spends HBM traffic on the planes instead.  Arrays of many blocks with long dumps are
// compute-heavy and run faster from planes; with CORR_BATCH_PLANES the batch owns a plane
// workspace and jobs of at least plane_min_nb blocks take that path.
//
// Autotuning: per job-set signature the tuner times each candidate launch shape
// (operand-ring depth, channels per work item for single-block arrays, item order, and with
// planes allowed the block count from which jobs take the plane path) on the batch's own
// buffers and keeps the fastest; results are cached in memory and, when a cache path is
// given, in a JSON-lines file, keyed by the job sizes and this library's build.
#include <algorithm>
#include <cstdint>
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
    int plane_min_nb = 0;   // jobs of at least this many 64-input blocks read fp16 planes (0: none)
    int wide = 1;           // plane jobs: wide items (block I against J, J + 1 in one MMA)
    int plane_splits = 1;   // plane jobs in this many launches, each next one's unpack beside the last
    float ms = 0.f;
};

// Shared memory a plane-fed launch leaves free on each SM when unpacks run beside it: one 8-bit
// unpack block (8 KB static + the 1 KB every block reserves), which still leaves the wide
// items' three-stage ring in place.
constexpr int kOverlapReserve = 10 * 1024;
constexpr int kMaxPlaneSplits = 8;

// The build this file was compiled in: tuning results of another build are not reused.
constexpr const char* kBuildStamp = __DATE__ " " __TIME__;

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;

struct ModeGroup {
    int bits = 0;
    bool planes = false;                  // jobs read fp16 planes the unpack kernel writes first
    std::vector<int> job_index;           // caller's job indices in this group
    std::vector<TcJobSpec> specs;         // launch order
    std::vector<CUtensorMap> maps;
    std::vector<CUtensorMap> maps_wide;   // plane jobs with wide items
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
    // overlapped plane launches: tensor-core launches on a high-priority stream, unpacks on a
    // low-priority one, so the launches' CTAs are placed first and unpack blocks fill the rest
    cudaStream_t x_stream = nullptr, u_stream = nullptr;
    std::vector<cudaEvent_t> events;      // fork, unpack-done per split, join
    double cmacs = 0.0;
    int64_t items = 0;
    corr::TuneChoice choice;
    bool tuned = false;
    bool allow_planes = false;
    char* d_planes = nullptr;             // plane workspace of the multi-block jobs
    std::vector<size_t> plane_off;        // per job: offset in d_planes (SIZE_MAX: none)
    size_t plane_bytes = 0;
};

namespace corr {
namespace {

double job_cost_per_item(const corr_job& j, int cpi) {
    const int nb = (j.n_inputs + kBlockInputs - 1) / kBlockInputs;
    const int nkb = (j.n_time + kTimeBlock - 1) / kTimeBlock;
    return (double)nkb * (nb == 1 ? cpi : 2);
}

int blocks_of(const corr_job& j) { return (j.n_inputs + kBlockInputs - 1) / kBlockInputs; }

Plan plan_of_job(const corr_job& j, int n_sm) {
    Plan p;
    p.n_inputs = j.n_inputs;
    p.n_chan = j.n_chan;
    p.n_time = j.n_time;
    p.sample_bits = j.sample_bits;
    p.nb = blocks_of(j);
    p.kp = (j.n_time + kTimeBlock - 1) / kTimeBlock * kTimeBlock;
    p.n_baselines = n_baselines(j.n_inputs);
    p.n_sm = n_sm;
    return p;
}

bool takes_planes(const corr_batch_s* b, const TuneChoice& ch, int k) {
    return ch.plane_min_nb > 0 && b->d_planes && b->plane_off[k] != SIZE_MAX &&
           blocks_of(b->jobs[k]) >= ch.plane_min_nb;
}

// (Re)build the launch groups for a tuning choice.
bool build_groups(corr_batch_s* b, const TuneChoice& ch) {
    b->groups.clear();
    b->items = 0;
    for (int bits : {8, 4}) {
        for (bool planes : {false, true}) {
            ModeGroup g;
            g.bits = bits;
            g.planes = planes;
            for (int k = 0; k < (int)b->jobs.size(); ++k)
                if (b->jobs[k].sample_bits == bits && takes_planes(b, ch, k) == planes) g.job_index.push_back(k);
            if (g.job_index.empty()) continue;
            auto cpi_of = [&](const corr_job& j) { return !planes && j.n_inputs <= kBlockInputs ? ch.pair_cpi : 1; };
            if (ch.order == 0)
                std::stable_sort(g.job_index.begin(), g.job_index.end(), [&](int x, int y) {
                    return job_cost_per_item(b->jobs[x], cpi_of(b->jobs[x])) >
                           job_cost_per_item(b->jobs[y], cpi_of(b->jobs[y]));
                });
            // 4-bit samples take e4m3 operands (128-sample boxes), as single-job calls do: converted
            // in the kernel, or read from e4m3 planes.  Batch jobs have TMA-addressable rows, so the
            // plane workspace holds e4m3 planes for every 4-bit job; anything else is refused here
            // rather than written as fp16 planes into a slot sized for e4m3 ones.
            const bool f8 = bits == 4;
            if (f8 && planes)
                for (int k : g.job_index)
                    if (!tc_planes_e4m3(plan_of_job(b->jobs[k], b->n_sm))) return false;
            for (int k : g.job_index) {
                const corr_job& j = b->jobs[k];
                const void* data = planes ? static_cast<const void*>(b->d_planes + b->plane_off[k]) : j.packed;
                TcJobSpec sp{j.n_inputs, j.n_chan, j.n_time, 1, j.sample_bits, data, j.vis, cpi_of(j)};
                CUtensorMap m, mw{};
                if (!(planes ? tc_make_plane_map(&m, sp, f8) : tc_make_raw_map(&m, sp, f8))) return false;
                const int nb = blocks_of(j);
                if (planes && ch.wide && nb >= 2 && tc_make_plane_map_wide(&mw, sp, f8)) sp.tw = 2;
                g.specs.push_back(sp);
                g.maps.push_back(m);
                g.maps_wide.push_back(mw);
                const int per_chan = sp.tw == 2 ? ((nb + 1) / 2) * ((nb + 2) / 2) : nb * (nb + 1) / 2;
                b->items += (int64_t)((j.n_chan + sp.cpi - 1) / sp.cpi) * per_chan;
            }
            g.tune.op_stages = ch.op_stages;
            g.tune.f8_operands = f8 ? 1 : 0;
            b->groups.push_back(std::move(g));
        }
    }
    return true;
}

cudaError_t unpack_range(corr_batch_s* b, const ModeGroup& g, size_t i0, size_t i1, cudaStream_t s,
                         int blocks_per_sm = 0) {
    for (size_t i = i0; i < i1; ++i) {   // each plane job writes its own planes
        const corr_job& j = b->jobs[g.job_index[i]];
        const Plan p = plan_of_job(j, b->n_sm);
        void* planes = const_cast<void*>(g.specs[i].data);
        const cudaError_t e = g.tune.f8_operands ? launch_unpack_e4m3(p, j.packed, 1, planes, s, blocks_per_sm)
                                                 : launch_unpack_fp16(p, j.packed, 1, planes, s, blocks_per_sm);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The group's jobs [i0, i1) in launches of at most kMaxJobsPerLaunch jobs.
cudaError_t x_range(corr_batch_s* b, const ModeGroup& g, size_t i0, size_t i1, const TcTuning& tune,
                    cudaStream_t s) {
    for (size_t k0 = i0; k0 < i1; k0 += kMaxJobsPerLaunch) {
        const int n = (int)std::min(i1 - k0, (size_t)kMaxJobsPerLaunch);
        const cudaError_t e =
            g.planes ? launch_xeng_tc_plane_jobs(g.specs.data() + k0, g.maps.data() + k0, n, b->accumulate,
                                                 b->d_status, b->n_sm, tune, s, g.maps_wide.data() + k0)
                     : launch_xeng_tc_raw_jobs(g.specs.data() + k0, g.maps.data() + k0, n, b->accumulate,
                                               b->d_status, b->n_sm, tune, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Split points of the plane jobs (launch order) into `splits` runs of about equal products.
std::vector<size_t> split_points(const corr_batch_s* b, const ModeGroup& g, int splits) {
    std::vector<double> cost(g.specs.size());
    double total = 0.0;
    for (size_t i = 0; i < g.specs.size(); ++i) {
        const corr_job& j = b->jobs[g.job_index[i]];
        cost[i] = (double)n_baselines(j.n_inputs) * j.n_chan * j.n_time;
        total += cost[i];
    }
    std::vector<size_t> pts{0};
    double acc = 0.0;
    for (size_t i = 0; i < g.specs.size(); ++i) {
        acc += cost[i];
        if ((int)pts.size() < splits && acc >= total * pts.size() / splits && i + 1 < g.specs.size())
            pts.push_back(i + 1);
    }
    pts.push_back(g.specs.size());
    return pts;
}

cudaError_t launch_groups(corr_batch_s* b, cudaStream_t s) {
    const int splits = b->choice.plane_splits;
    const ModeGroup* plane_group = nullptr;
    int n_plane_groups = 0;
    for (auto& g : b->groups)
        if (g.planes) {
            plane_group = &g;
            ++n_plane_groups;
        }
    if (splits <= 1 || n_plane_groups != 1 || plane_group->specs.size() < 2 || !b->x_stream) {
        // one launch per group, each plane group's unpacks first
        for (auto& g : b->groups) {
            if (g.planes) {
                const cudaError_t e = unpack_range(b, g, 0, g.specs.size(), s);
                if (e != cudaSuccess) return e;
            }
            const cudaError_t e = x_range(b, g, 0, g.specs.size(), g.tune, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // Overlapped form: the plane jobs in `splits` launches; the unpacks run back to back on the
    // low-priority stream and each launch waits for its own jobs' unpacks, so the unpack of the
    // next run of jobs (and the first run's, beside the packed-sample launches) proceeds while
    // the tensor cores work on the current one:
    //   u: U1 -> e1 -> U2 -> e2 -> ...        x: packed launches, [e1] X1, [e2] X2, ...
    const ModeGroup& pg = *plane_group;
    const std::vector<size_t> pts = split_points(b, pg, splits);
    const size_t n_runs = pts.size() - 1;
    if (b->events.size() < n_runs + 2) return cudaErrorInvalidValue;
    cudaEvent_t ev_fork = b->events[0], ev_join = b->events[n_runs + 1];
    cudaError_t e = cudaEventRecord(ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->x_stream, ev_fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->u_stream, ev_fork, 0);
    // the first run's unpacks have the GPU to themselves (beside the packed-sample launches at
    // most); the later ones take one block per SM, which fits beside a tensor-core CTA whichever
    // of the two is placed first
    for (size_t r = 0; r < n_runs && e == cudaSuccess; ++r) {
        e = unpack_range(b, pg, pts[r], pts[r + 1], b->u_stream, r == 0 ? 0 : 1);
        if (e == cudaSuccess) e = cudaEventRecord(b->events[1 + r], b->u_stream);
    }
    for (auto& g : b->groups)
        if (!g.planes && e == cudaSuccess) e = x_range(b, g, 0, g.specs.size(), g.tune, b->x_stream);
    TcTuning tune = pg.tune;
    tune.smem_reserve = kOverlapReserve;
    for (size_t r = 0; r < n_runs && e == cudaSuccess; ++r) {
        e = cudaStreamWaitEvent(b->x_stream, b->events[1 + r], 0);
        if (e == cudaSuccess) e = x_range(b, pg, pts[r], pts[r + 1], tune, b->x_stream);
    }
    // join: the caller's stream continues after the last launch (which followed every unpack)
    if (e == cudaSuccess) e = cudaEventRecord(ev_join, b->x_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join, 0);
    return e;
}

std::string signature(const corr_batch_s* b) {
    std::vector<std::string> parts;
    parts.push_back(std::string("build ") + kBuildStamp + (b->allow_planes ? " planes" : " raw"));
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
        if ((p = strstr(k1, "\"plane_min_nb\": "))) c.plane_min_nb = atoi(p + 16);
        if ((p = strstr(k1, "\"wide\": "))) c.wide = atoi(p + 8);
        if ((p = strstr(k1, "\"plane_splits\": "))) c.plane_splits = atoi(p + 16);
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
    fprintf(f,
            "{\"key\": \"%s\", \"op_stages\": %d, \"pair_cpi\": %d, \"order\": %d, \"plane_min_nb\": %d, "
            "\"wide\": %d, \"plane_splits\": %d, \"ms\": %.6f}\n",
            key.c_str(), c.op_stages, c.pair_cpi, c.order, c.plane_min_nb, c.wide, c.plane_splits, c.ms);
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
    int max_nb = 1;
    for (const auto& j : b->jobs) {
        any_small = any_small || j.n_inputs <= kBlockInputs;
        max_nb = std::max(max_nb, blocks_of(j));
    }
    std::vector<int> plane_opts{0};
    if (b->d_planes)
        for (int nb : {2, 4, 8, 16})
            if (nb <= max_nb) plane_opts.push_back(nb);
    std::vector<TuneChoice> cands;
    for (int order : {0, 1})
        for (int cpi : any_small ? std::vector<int>{2, 1} : std::vector<int>{2})
            for (int ops : {3, 4, 5})
                for (int pm : plane_opts)
                    for (int wide : pm ? std::vector<int>{1, 0} : std::vector<int>{1}) {
                        TuneChoice c;
                        c.op_stages = ops;
                        c.pair_cpi = cpi;
                        c.order = order;
                        c.plane_min_nb = pm;
                        c.wide = wide;
                        cands.push_back(c);
                    }
    TuneChoice best;
    float best_ms = 1e30f;
    cudaStream_t s = b->own_stream;
    for (auto& c : cands) {
        b->choice = c;
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
    // second stage: the best shape with its plane jobs split into overlapped launches
    if (best.plane_min_nb > 0) {
        for (int splits : {2, 3, 4}) {
            TuneChoice c = best;
            c.plane_splits = splits;
            b->choice = c;
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

// Capture the batch's launches into a CUDA graph (one eager run first sets the kernels'
// shared-memory attributes outside the capture).
cudaError_t capture_graph(corr_batch_s* b) {
    cudaError_t e = launch_groups(b, b->own_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->own_stream);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->own_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t el = launch_groups(b, b->own_stream);
        e = cudaStreamEndCapture(b->own_stream, &b->g);
        if (el != cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gx, b->g, 0);
    if (e == cudaSuccess) b->graph = true;
    return e;
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
    if (e == cudaSuccess && (flags & CORR_BATCH_PLANES)) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->x_stream, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->u_stream, cudaStreamNonBlocking, least);
        for (int k = 0; k < kMaxPlaneSplits + 2 && e == cudaSuccess; ++k) {
            cudaEvent_t ev = nullptr;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) b->events.push_back(ev);
        }
    }
    if (e != cudaSuccess) {
        corr_batch_destroy(b);
        return cuda_error(e, "corr_batch_create");
    }
    // plane workspace: one set of planes per multi-block job (fp16, or e4m3 for 4-bit samples of
    // TMA-addressable rows), owned by the batch
    b->plane_off.assign(n_jobs, SIZE_MAX);
    if (flags & CORR_BATCH_PLANES) {
        b->allow_planes = true;
        size_t total = 0;
        for (int k = 0; k < n_jobs; ++k) {
            const Plan p = plan_of_job(b->jobs[k], b->n_sm);
            if (p.nb < 2) continue;
            b->plane_off[k] = total;
            total += (tc_workspace_planes_bytes(p, 1) + 255) / 256 * 256;   // e4m3 planes for 4-bit jobs
        }
        if (total) {
            e = cudaMalloc((void**)&b->d_planes, total);
            if (e != cudaSuccess) {
                corr_batch_destroy(b);
                return set_error(CORR_ENOMEM, "cudaMalloc(%zu) of the batch's plane workspace failed", total);
            }
            b->plane_bytes = total;
        }
    }
    corr_status st = CORR_OK;
    if ((flags & CORR_BATCH_AUTOTUNE) && (flags & CORR_BATCH_ACCUMULATE)) {
        corr_batch_destroy(b);
        return set_error(CORR_EINVAL, "CORR_BATCH_AUTOTUNE with CORR_BATCH_ACCUMULATE would add tuning runs into "
                                      "the accumulators; tune without ACCUMULATE first (the choice is cached)");
    }
    if (flags & CORR_BATCH_AUTOTUNE) {
        st = autotune(b, tune_cache);
    } else {
        TuneChoice def;
        if (b->d_planes) def.plane_min_nb = 4;   // untuned: arrays of 256 inputs and more read planes
        b->choice = def;
        if (!build_groups(b, def)) st = set_error(CORR_EINVAL, "tensor map encoding failed");
    }
    if (st != CORR_OK) {
        corr_batch_destroy(b);
        return st;
    }
    if (flags & CORR_BATCH_GRAPH) {
        e = capture_graph(b);
        if (e != cudaSuccess) {
            corr_batch_destroy(b);
            return cuda_error(e, "CUDA graph capture of the batch");
        }
    }
    *out = b;
    return CORR_OK;
}

corr_status corr_batch_set_shape(corr_batch b, int op_stages, int pair_cpi, int order, int plane_min_nb, int wide,
                                 int plane_splits) {
    if (!b) return set_error(CORR_EINVAL, "corr_batch_set_shape: NULL batch");
    if (op_stages < 0 || op_stages > 16 || (pair_cpi != 1 && pair_cpi != 2) || (order != 0 && order != 1) ||
        plane_min_nb < 0 || (wide != 0 && wide != 1) || plane_splits < 1 || plane_splits > kMaxPlaneSplits)
        return set_error(CORR_EINVAL, "corr_batch_set_shape: op_stages in [0, 16], pair_cpi 1 or 2, order 0 or 1, "
                                      "plane_min_nb >= 0, wide 0 or 1, plane_splits in [1, %d]", kMaxPlaneSplits);
    if (plane_min_nb > 0 && !b->d_planes)
        return set_error(CORR_EINVAL, "plane_min_nb > 0 needs a batch created with CORR_BATCH_PLANES");
    TuneChoice c;
    c.op_stages = op_stages;
    c.pair_cpi = pair_cpi;
    c.order = order;
    c.plane_min_nb = plane_min_nb;
    c.wide = wide;
    c.plane_splits = plane_splits;
    if (!build_groups(b, c)) return set_error(CORR_EINVAL, "tensor map encoding failed");
    b->choice = c;
    b->tuned = false;
    if (b->graph) {
        if (b->gx) cudaGraphExecDestroy(b->gx);
        if (b->g) cudaGraphDestroy(b->g);
        b->gx = nullptr;
        b->g = nullptr;
        b->graph = false;
        const cudaError_t e = capture_graph(b);
        if (e != cudaSuccess) return cuda_error(e, "CUDA graph capture of the batch");
    }
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
    st->plane_min_nb = b->choice.plane_min_nb;
    st->wide = b->choice.wide;
    st->plane_splits = b->choice.plane_splits;
    st->plane_bytes = b->plane_bytes;
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
    if (b->x_stream) cudaStreamDestroy(b->x_stream);
    if (b->u_stream) cudaStreamDestroy(b->u_stream);
    for (auto ev : b->events) cudaEventDestroy(ev);
    if (b->d_status) cudaFree(b->d_status);
    if (b->d_planes) cudaFree(b->d_planes);
    delete b;
    return CORR_OK;
}

}  // extern "C"

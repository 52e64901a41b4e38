// Real-time serving loop: correlation jobs from concurrent streams, admitted by HBM
// footprint into a device arena, run asynchronously, polled by id.
//
// The paper's prototype overlaps staging of the next batch in host memory with the
// CMAC of the previous one on the GPU (Sec. 5, Table 3 notes).  Here a dispatcher thread
// takes jobs from a mailbox in arrival order, admits each when its device footprint
// (packed samples + visibilities + any workspace) fits the free space of a fixed arena
// allocated once at start-up, and issues on one of n_streams CUDA streams: the
// host-to-device copy of the samples, the X-stage kernel, the readback of the kernel's
// status words and, if the caller gave a host buffer, the device-to-host copy of the
// visibilities.  Copies of one job overlap the kernels of others on the other streams.
// A completion thread retires jobs as their events complete, frees their arena blocks
// and wakes waiters.  All host waits are bounded; the kernels' own waits are bounded and
// report through the status words.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "corr_internal.h"

namespace corr {
namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

constexpr size_t kAlign = 256;

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over one device allocation (offsets only; the caller locks).
class Arena {
public:
    explicit Arena(size_t bytes) : size_(bytes) { free_[0] = bytes; }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    bool fits(size_t bytes) const {
        for (const auto& kv : free_)
            if (kv.second >= bytes) return true;
        return false;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    size_t size_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

enum JobState { kQueued, kRunning, kDone, kFailed, kCancelled };

struct Job {
    uint64_t id = 0;
    corr_job_desc desc{};
    JobState state = kQueued;
    corr_status final_status = CORR_PENDING;
    double t_submit = 0, t_start = 0, t_done = 0;
    size_t off = 0, bytes = 0;
    bool holds_arena = false;
    bool raw = false;
    int stream = -1;
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    int* h_status = nullptr;   // pinned host copy of the kernel status words
    float gpu_ms = 0.f;
    void* d_vis = nullptr;     // device result while the job keeps it
};

size_t packed_bytes(const corr_job_desc& d) {
    const size_t per = d.sample_bits == 4 ? 1 : (d.sample_bits == 8 ? 2 : 8);
    return (size_t)d.n_time * d.n_chan * d.n_inputs * per;
}

size_t vis_bytes(const corr_job_desc& d) {
    return (size_t)n_baselines(d.n_inputs) * d.n_chan * (d.sample_bits == 32 ? 8 : 16);
}

Plan plan_of(const corr_job_desc& d, int device, int n_sm) {
    Plan p;
    p.n_inputs = d.n_inputs;
    p.n_chan = d.n_chan;
    p.n_time = d.n_time;
    p.sample_bits = d.sample_bits;
    p.nb = (d.n_inputs + kBlockInputs - 1) / kBlockInputs;
    p.kp = (d.n_time + kTimeBlock - 1) / kTimeBlock * kTimeBlock;
    p.n_baselines = n_baselines(d.n_inputs);
    p.device = device;
    p.n_sm = n_sm;
    return p;
}

// Device bytes a job occupies while it runs: status, packed samples, visibilities, workspace.
size_t footprint(const corr_job_desc& d, bool* raw) {
    Plan p = plan_of(d, 0, 0);
    // samples the tensor-core kernel reads as they are: packed integers it can address with TMA,
    // and float samples of single-block arrays (split into bf16 hi/lo inside the kernel)
    *raw = d.sample_bits == 32 ? tc_rawf32_supported(p) : tc_raw_supported(p);
    size_t ws = 0;
    if (!*raw) ws = d.sample_bits == 32 ? 2 * (size_t)p.n_chan * p.nb * kBlockRows * p.kp * 2 : planes_bytes(p, 1);
    return round_up(16) + round_up(packed_bytes(d)) + round_up(vis_bytes(d)) + round_up(ws);
}

}  // namespace
}  // namespace corr

struct corr_server_s {
    int device = 0, n_sm = 0;
    char* d_base = nullptr;
    corr::Arena* arena = nullptr;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    std::mutex mu;
    std::condition_variable cv_dispatch, cv_done;
    std::deque<uint64_t> queue;                       // the mailbox, arrival order
    std::unordered_map<uint64_t, corr::Job> jobs;
    std::vector<uint64_t> running;
    std::atomic<uint64_t> next_id{1};
    bool stop = false, paused = false;
    std::thread dispatcher, completer;
    corr_server_stats stats{};
};

namespace corr {
namespace {

// Issue one admitted job on its stream (called with the lock released).
cudaError_t issue(corr_server_s* S, Job& j) {
    cudaStream_t s = S->streams[j.stream];
    char* base = S->d_base + j.off;
    int* d_status = reinterpret_cast<int*>(base);
    char* d_packed = base + round_up(16);
    char* d_vis = d_packed + round_up(packed_bytes(j.desc));
    char* d_ws = d_vis + round_up(vis_bytes(j.desc));
    Plan p = plan_of(j.desc, S->device, S->n_sm);
    p.d_status = d_status;
    cudaError_t e = cudaEventRecord(j.ev_start, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, 16, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_packed, j.desc.host_packed, packed_bytes(j.desc),
                                              cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        if (j.raw) {
            e = j.desc.sample_bits == 32 ? launch_xeng_tc_rawf32(p, d_packed, 1, d_vis, 0, s)
                                         : launch_xeng_tc_raw(p, d_packed, 1, d_vis, 0, s);
        } else if (j.desc.sample_bits == 32) {
            const size_t half = (size_t)p.n_chan * p.nb * kBlockRows * p.kp * 2;
            e = launch_unpack_bf16x2(p, d_packed, 1, d_ws, d_ws + half, s);
            if (e == cudaSuccess) e = launch_xeng_tc(p, d_ws, d_ws + half, 1, d_vis, 0, s);
        } else {
            e = launch_unpack_fp16(p, d_packed, 1, d_ws, s);
            if (e == cudaSuccess) e = launch_xeng_tc(p, d_ws, nullptr, 1, d_vis, 0, s);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(j.h_status, d_status, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && j.desc.host_vis)
        e = cudaMemcpyAsync(j.desc.host_vis, d_vis, vis_bytes(j.desc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(j.ev_done, s);
    return e;
}

void dispatcher_loop(corr_server_s* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (true) {
        S->cv_dispatch.wait_for(lock, std::chrono::milliseconds(50), [&] {
            if (S->stop) return true;
            if (S->paused || S->queue.empty()) return false;
            auto it = S->jobs.find(S->queue.front());
            return it != S->jobs.end() && S->arena->fits(it->second.bytes);
        });
        if (S->stop) break;
        if (S->paused || S->queue.empty()) continue;
        const uint64_t id = S->queue.front();
        Job& j = S->jobs[id];
        size_t off;
        if (!S->arena->alloc(j.bytes, &off)) continue;   // head of line waits for memory (FIFO admission)
        S->queue.pop_front();
        j.off = off;
        j.holds_arena = true;
        j.stream = S->next_stream;
        S->next_stream = (S->next_stream + 1) % (int)S->streams.size();
        j.state = kRunning;
        j.t_start = now_s();
        j.d_vis = S->d_base + off + round_up(16) + round_up(packed_bytes(j.desc));   // layout of issue()
        S->stats.bytes_in_use = S->arena->used();
        S->stats.peak_bytes = S->arena->peak();
        lock.unlock();
        cudaError_t e = issue(S, j);
        lock.lock();
        // the completion thread sees the job only once its events are recorded
        if (e == cudaSuccess) S->running.push_back(id);
        if (e != cudaSuccess) {
            // nothing of this job is queued behind a failed call that we can rely on; mark it
            // failed once its stream has drained the calls that were accepted
            cudaStreamSynchronize(S->streams[j.stream]);
            j.state = kFailed;
            j.final_status = CORR_ECUDA;
            j.t_done = now_s();
            S->arena->release(j.off, j.bytes);
            j.holds_arena = false;
            S->stats.failed++;
            S->cv_done.notify_all();
        }
    }
}

void completer_loop(corr_server_s* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (true) {
        bool progressed = false;
        for (size_t k = 0; k < S->running.size();) {
            Job& j = S->jobs[S->running[k]];
            const cudaError_t q = cudaEventQuery(j.ev_done);
            if (q == cudaErrorNotReady) {
                ++k;
                continue;
            }
            j.t_done = now_s();
            cudaEventElapsedTime(&j.gpu_ms, j.ev_start, j.ev_done);
            if (q != cudaSuccess) {
                j.state = kFailed;
                j.final_status = CORR_ECUDA;
            } else if (j.h_status[0] != 0) {
                j.state = kFailed;
                j.final_status = CORR_ETIMEOUT;   // a bounded device wait gave up
            } else {
                j.state = kDone;
                j.final_status = CORR_OK;
            }
            if (j.state == kDone) S->stats.completed++;
            else S->stats.failed++;
            // results copied to the host free their device block now; device-resident
            // results stay until corr_release
            if (j.desc.host_vis || j.state != kDone) {
                S->arena->release(j.off, j.bytes);
                j.holds_arena = false;
                j.d_vis = nullptr;
            }
            S->stats.bytes_in_use = S->arena->used();
            S->running[k] = S->running.back();
            S->running.pop_back();
            progressed = true;
        }
        if (progressed) {
            S->cv_done.notify_all();
            S->cv_dispatch.notify_all();
        }
        if (S->stop && S->running.empty()) break;
        lock.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(progressed ? 0 : 20));
        lock.lock();
    }
}

void fill_result(const Job& j, corr_job_result* r) {
    r->status = j.state == kQueued || j.state == kRunning ? CORR_PENDING : j.final_status;
    r->t_submit = j.t_submit;
    r->t_start = j.t_start;
    r->t_done = j.t_done;
    r->gpu_ms = j.gpu_ms;
    r->d_vis = j.d_vis;
}

}  // namespace
}  // namespace corr

using namespace corr;

extern "C" {

corr_status corr_server_create(corr_server* out, size_t hbm_budget_bytes, int n_streams, int flags) {
    if (!out) return set_error(CORR_EINVAL, "corr_server_create: out is NULL");
    *out = nullptr;
    if (n_streams < 1 || n_streams > 64) return set_error(CORR_EINVAL, "n_streams=%d outside [1, 64]", n_streams);
    if (hbm_budget_bytes < (size_t)1 << 20) return set_error(CORR_EINVAL, "HBM budget below 1 MiB");
    corr_server_s* S = new (std::nothrow) corr_server_s();
    if (!S) return set_error(CORR_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->n_sm, cudaDevAttrMultiProcessorCount, S->device);
    hbm_budget_bytes = hbm_budget_bytes / kAlign * kAlign;
    if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_base, hbm_budget_bytes);
    if (e != cudaSuccess) {
        delete S;
        return e == cudaErrorMemoryAllocation ? set_error(CORR_ENOMEM, "cudaMalloc of the %zu-byte arena failed",
                                                          hbm_budget_bytes)
                                              : cuda_error(e, "corr_server_create");
    }
    S->arena = new Arena(hbm_budget_bytes);
    for (int k = 0; k < n_streams && e == cudaSuccess; ++k) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) S->streams.push_back(st);
    }
    if (e != cudaSuccess) {
        for (auto st : S->streams) cudaStreamDestroy(st);
        cudaFree(S->d_base);
        delete S->arena;
        delete S;
        return cuda_error(e, "cudaStreamCreate");
    }
    S->paused = (flags & CORR_SERVER_START_PAUSED) != 0;
    S->stats.arena_bytes = hbm_budget_bytes;
    S->dispatcher = std::thread(dispatcher_loop, S);
    S->completer = std::thread(completer_loop, S);
    *out = S;
    return CORR_OK;
}

corr_status corr_submit(corr_server S, const corr_job_desc* d, uint64_t* job_id) {
    if (!S || !d || !job_id) return set_error(CORR_EINVAL, "corr_submit: NULL argument");
    *job_id = 0;
    if (d->sample_bits != 4 && d->sample_bits != 8 && d->sample_bits != 32)
        return set_error(CORR_EINVAL, "sample_bits=%d must be 4, 8 or 32", d->sample_bits);
    if (d->n_inputs < 1 || d->n_inputs > kMaxInputs || d->n_chan < 1 || d->n_time < 1)
        return set_error(CORR_EINVAL, "bad job sizes N=%d C=%d T=%d", d->n_inputs, d->n_chan, d->n_time);
    if (!d->host_packed) return set_error(CORR_EINVAL, "host_packed is NULL");
    Job j;
    j.desc = *d;
    j.bytes = footprint(*d, &j.raw);
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->stop) return set_error(CORR_EBUSY, "server is shutting down");
    if (j.bytes > S->arena->size()) {
        S->stats.rejected++;
        return set_error(CORR_EBUSY, "job needs %zu device bytes, more than the %zu-byte HBM budget", j.bytes,
                         S->arena->size());
    }
    cudaError_t e = cudaEventCreate(&j.ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&j.ev_done);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&j.h_status, 16);
    if (e != cudaSuccess) {
        if (j.ev_start) cudaEventDestroy(j.ev_start);
        if (j.ev_done) cudaEventDestroy(j.ev_done);
        return cuda_error(e, "corr_submit");
    }
    memset(j.h_status, 0, 16);
    j.id = S->next_id++;
    j.t_submit = now_s();
    *job_id = j.id;
    S->jobs.emplace(j.id, j);
    S->queue.push_back(j.id);
    S->stats.submitted++;
    S->cv_dispatch.notify_all();
    return CORR_OK;
}

corr_status corr_poll(corr_server S, uint64_t job_id, corr_job_result* res) {
    if (!S || !res) return set_error(CORR_EINVAL, "corr_poll: NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(job_id);
    if (it == S->jobs.end()) return set_error(CORR_EINVAL, "unknown job id %llu", (unsigned long long)job_id);
    fill_result(it->second, res);
    return (corr_status)res->status;
}

corr_status corr_wait(corr_server S, uint64_t job_id, double timeout_s, corr_job_result* res) {
    if (!S || !res) return set_error(CORR_EINVAL, "corr_wait: NULL argument");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->jobs.find(job_id);
    if (it == S->jobs.end()) return set_error(CORR_EINVAL, "unknown job id %llu", (unsigned long long)job_id);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
    S->cv_done.wait_until(lock, deadline, [&] {
        const JobState st = S->jobs[job_id].state;
        return st != kQueued && st != kRunning;
    });
    const Job& j = S->jobs[job_id];
    fill_result(j, res);
    if (j.state == kQueued || j.state == kRunning)
        return set_error(CORR_ETIMEOUT, "job %llu not finished within %.3f s", (unsigned long long)job_id, timeout_s);
    return (corr_status)res->status;
}

corr_status corr_release(corr_server S, uint64_t job_id) {
    if (!S) return set_error(CORR_EINVAL, "corr_release: NULL server");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(job_id);
    if (it == S->jobs.end()) return set_error(CORR_EINVAL, "unknown job id %llu", (unsigned long long)job_id);
    Job& j = it->second;
    if (j.state == kQueued || j.state == kRunning) return set_error(CORR_PENDING, "job still in flight");
    if (j.holds_arena) {
        S->arena->release(j.off, j.bytes);
        j.holds_arena = false;
        j.d_vis = nullptr;
        S->stats.bytes_in_use = S->arena->used();
        S->cv_dispatch.notify_all();
    }
    if (j.ev_start) cudaEventDestroy(j.ev_start);
    if (j.ev_done) cudaEventDestroy(j.ev_done);
    if (j.h_status) cudaFreeHost(j.h_status);
    S->jobs.erase(it);
    return CORR_OK;
}

corr_status corr_fetch(corr_server S, uint64_t job_id, void* host_vis) {
    if (!S || !host_vis) return set_error(CORR_EINVAL, "corr_fetch: NULL argument");
    void* src = nullptr;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->jobs.find(job_id);
        if (it == S->jobs.end()) return set_error(CORR_EINVAL, "unknown job id %llu", (unsigned long long)job_id);
        const Job& j = it->second;
        if (j.state != kDone) return set_error(j.state == kFailed ? j.final_status : CORR_PENDING,
                                               "job %llu has no result", (unsigned long long)job_id);
        if (!j.holds_arena) return set_error(CORR_EINVAL, "job %llu did not keep its result on the device",
                                             (unsigned long long)job_id);
        src = j.d_vis;
        bytes = vis_bytes(j.desc);
    }
    // the block stays reserved until corr_release, which the caller must not race with this copy
    cudaError_t e = cudaMemcpy(host_vis, src, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "corr_fetch");
    return CORR_OK;
}

corr_status corr_server_resume(corr_server S) {
    if (!S) return set_error(CORR_EINVAL, "corr_server_resume: NULL server");
    std::lock_guard<std::mutex> lock(S->mu);
    S->paused = false;
    S->cv_dispatch.notify_all();
    return CORR_OK;
}

corr_status corr_server_get_stats(corr_server S, corr_server_stats* st) {
    if (!S || !st) return set_error(CORR_EINVAL, "corr_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    *st = S->stats;
    st->queued = (int64_t)S->queue.size();
    st->running = (int64_t)S->running.size();
    st->bytes_in_use = S->arena->used();
    st->peak_bytes = S->arena->peak();
    return CORR_OK;
}

corr_status corr_server_destroy(corr_server S, double drain_timeout_s) {
    if (!S) return set_error(CORR_EINVAL, "corr_server_destroy: NULL server");
    corr_status result = CORR_OK;
    {
        std::unique_lock<std::mutex> lock(S->mu);
        // queued jobs never start; running jobs are waited for (bounded)
        for (uint64_t id : S->queue) {
            S->jobs[id].state = kCancelled;
            S->jobs[id].final_status = CORR_EBUSY;
        }
        S->stats.cancelled += (int64_t)S->queue.size();
        S->queue.clear();
        const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                                 std::chrono::duration<double>(drain_timeout_s > 0 ? drain_timeout_s : 0));
        S->cv_done.wait_until(lock, deadline, [&] { return S->running.empty(); });
        if (!S->running.empty()) result = set_error(CORR_ETIMEOUT, "%zu jobs still running after %.1f s",
                                                    S->running.size(), drain_timeout_s);
        S->stop = true;
        S->cv_dispatch.notify_all();
    }
    // the streams must be idle before the arena goes away: wait for them (the kernels'
    // own waits are bounded, so this returns)
    for (auto st : S->streams) cudaStreamSynchronize(st);
    S->dispatcher.join();
    S->completer.join();
    for (auto& kv : S->jobs) {
        if (kv.second.ev_start) cudaEventDestroy(kv.second.ev_start);
        if (kv.second.ev_done) cudaEventDestroy(kv.second.ev_done);
        if (kv.second.h_status) cudaFreeHost(kv.second.h_status);
    }
    for (auto st : S->streams) cudaStreamDestroy(st);
    cudaFree(S->d_base);
    delete S->arena;
    delete S;
    return result;
}

corr_status corr_host_alloc(void** ptr, size_t bytes) {
    if (!ptr) return set_error(CORR_EINVAL, "corr_host_alloc: NULL argument");
    cudaError_t e = cudaMallocHost(ptr, bytes);
    if (e != cudaSuccess) return set_error(CORR_ENOMEM, "cudaMallocHost(%zu): %s", bytes, cudaGetErrorString(e));
    return CORR_OK;
}

corr_status corr_host_free(void* ptr) {
    cudaError_t e = cudaFreeHost(ptr);
    if (e != cudaSuccess) return cuda_error(e, "cudaFreeHost");
    return CORR_OK;
}

}  // extern "C"

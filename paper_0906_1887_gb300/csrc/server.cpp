// Real-time serving loop: correlation jobs from concurrent streams, admitted by HBM
// footprint into a device arena, run asynchronously, polled by id.
//
// The paper's prototype overlaps staging of the next batch in host memory with the
// CMAC of the previous one on the GPU (Sec. 5, Table 3 notes), and integrates: batches are
// added into accumulators that are read out, divided by the update count and reset at each
// dump (Fig. 1).  Here a dispatcher thread takes jobs from a mailbox in arrival order.  A job
// of an input stream opened with corr_server_open_stream uses that stream's device state,
// admitted once: a ring of sample slots and accumulators that its jobs add into, dumped
// every jobs_per_dump jobs; such jobs are issued as soon as they arrive, on the stream's own
// pair of CUDA streams (copy-in of job k into its ring slot waits only for the X stage of job
// k - ring_slots).  Any other job is admitted when its device footprint (packed samples +
// visibilities + any workspace) fits the free space of a fixed arena allocated once at
// start-up, and is issued on one of n_streams CUDA streams: the host-to-device copy of the
// samples, the X-stage kernel, the readback of the kernel's status words and, if the caller
// gave a host buffer, the device-to-host copy of the visibilities.  Copies of one job overlap
// the kernels of others.  A completion thread retires jobs as their events complete, frees
// their arena blocks and wakes waiters.  All host waits are bounded; the kernels' own waits
// are bounded and report through the status words.
#include <algorithm>
#include <atomic>
#include <cstdint>
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

struct StreamState;

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
    int* h_status = nullptr;   // the kernels' status words in mapped pinned memory (host view)
    int* d_status = nullptr;   // the same words, device view
    float gpu_ms = 0.f;
    void* d_vis = nullptr;     // device result while the job keeps it
    bool stream_job = false;   // runs on an open stream's device state
    int64_t seq = 0;           // index of the job within its open stream
    bool closes = false;       // ends a dump interval of its open stream
    int64_t n_accum = 0;       // samples summed in that dump
    StreamState* st = nullptr;  // the open stream's state (stream jobs)
    double deadline = 0;       // t_submit + the job's own sample time (earliest-deadline-first issue)
    cudaEvent_t ev_copied = nullptr;   // recorded after the job's samples reached the device
    size_t copy_bytes = 0;     // its host-to-device bytes while they count against the copy budget
    const int* h_status_pair = nullptr;   // issued with the next job of its stream: that job's
                                          // status words carry the shared X stage's status
};

// Device state of one open input stream (corr_server_open_stream).
struct StreamState {
    corr_stream_desc d{};
    size_t off = 0, bytes = 0;           // arena block
    size_t slot_bytes = 0;               // one ring slot (packed samples of one job)
    char* slots = nullptr;               // [ring_slots] sample slots
    char* acc = nullptr;                 // accumulators [C][P][2]
    char* ws = nullptr;                  // sample planes when the kernel cannot read the packed layout
    char* dumpbuf = nullptr;             // averaged mode: float32 [C][P][2]
    char* phasor = nullptr;              // averaged mode with delays: float2 [C][N]
    bool raw = false;
    cudaStream_t copy_s = nullptr, comp_s = nullptr;
    // averaged dumps: the readout of the dump buffer to the host runs on out_s, so the stream's
    // next jobs (which only need the dump kernel to have read the accumulators) do not queue
    // behind a copy of several GB; the next dump kernel waits for the previous readout (ev_out)
    cudaStream_t out_s = nullptr;
    cudaEvent_t ev_dumped = nullptr, ev_out = nullptr;
    bool out_pending = false;
    std::vector<cudaEvent_t> slot_full, slot_free;
    int64_t n_submitted = 0, n_retired = 0;
    bool closing = false;
    // adjacent ring slots form one [2T][C][N] block (no padding between slots): two queued jobs
    // of the stream can then run as one X stage over 2T samples, the workspace sized for it
    bool pairable = false;
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
    // samples the tensor-core kernel reads as they are: packed integers it can address with TMA
    // (unless the array is large enough for the plane feed to be faster), and float samples of
    // single-block arrays (split into bf16 hi/lo inside the kernel)
    *raw = d.sample_bits == 32 ? tc_rawf32_supported(p) : !tc_use_planes(p);
    size_t ws = 0;
    if (!*raw) ws = d.sample_bits == 32 ? 2 * (size_t)p.n_chan * p.nb * kBlockRows * p.kp * 2 : tc_workspace_planes_bytes(p, 1);
    return round_up(16) + round_up(packed_bytes(d)) + round_up(vis_bytes(d)) + round_up(ws);
}

corr_job_desc shape_of(const corr_stream_desc& sd) {
    corr_job_desc d{};
    d.n_inputs = sd.n_inputs;
    d.n_chan = sd.n_chan;
    d.n_time = sd.n_time;
    d.sample_bits = sd.sample_bits;
    return d;
}

// Carve an open stream's arena block: status words, ring slots, accumulators, workspace,
// dump buffer and phasors.  Returns the bytes needed; with base != nullptr fills the pointers.
size_t stream_layout(StreamState& st, char* base) {
    const corr_job_desc d = shape_of(st.d);
    Plan p = plan_of(d, 0, 0);
    // slots 16-byte aligned (TMA and the vectorised unpack need no more), so for rows of whole
    // 16-byte pieces they abut and two adjacent slots are one [2T][C][N] block
    st.slot_bytes = (packed_bytes(d) + 15) / 16 * 16;
    st.pairable = d.sample_bits != 32 && st.d.ring_slots >= 2 && st.slot_bytes == packed_bytes(d) &&
                  d.n_time <= (1 << 28);
    corr_job_desc d2 = d;
    if (st.pairable) d2.n_time = 2 * d.n_time;
    size_t ws = 0;
    if (!st.raw) ws = d.sample_bits == 32 ? 2 * (size_t)p.n_chan * p.nb * kBlockRows * p.kp * 2
                                          : tc_workspace_planes_bytes(plan_of(d2, 0, 0), 1);
    const bool avg = st.d.dump_mode == CORR_STREAM_DUMP_AVERAGED;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* ptr = base ? base + off : nullptr;
        off += round_up(bytes);
        return ptr;
    };
    st.slots = take(st.slot_bytes * (size_t)st.d.ring_slots);
    st.acc = take(vis_bytes(d));
    st.ws = ws ? take(ws) : nullptr;
    st.dumpbuf = avg ? take((size_t)n_baselines(d.n_inputs) * d.n_chan * 8) : nullptr;
    st.phasor = (avg && st.d.d_delays) ? take((size_t)d.n_chan * d.n_inputs * 8) : nullptr;
    return off;
}

}  // namespace
}  // namespace corr

namespace corr {
namespace {

// Per-job resources recycled from job to job: pinned status words (allocated kStatusChunk jobs'
// worth at a time) and timing events.  Allocating and freeing them per job put cudaMallocHost
// and cudaFreeHost -- which can wait for the device -- on the submit and release paths under
// the server lock, where a release behind a deep GPU queue stalled dispatch for every stream.
constexpr int kStatusChunk = 4096;
struct JobResources {
    struct Slot {
        int* host;   // mapped pinned memory: the kernels write a job's status words here directly
        int* dev;    // the same words as a device pointer
    };
    std::vector<int*> chunks;
    std::vector<Slot> free_status;
    std::vector<cudaEvent_t> events, free_events;
    cudaError_t take_status(Slot* out) {
        if (free_status.empty()) {
            int* c = nullptr;
            int* d = nullptr;
            cudaError_t e = cudaHostAlloc((void**)&c, (size_t)kStatusChunk * 4 * sizeof(int), cudaHostAllocMapped);
            if (e != cudaSuccess) return e;
            e = cudaHostGetDevicePointer((void**)&d, c, 0);
            if (e != cudaSuccess) {
                cudaFreeHost(c);
                return e;
            }
            chunks.push_back(c);
            for (int k = kStatusChunk - 1; k >= 0; --k) free_status.push_back(Slot{c + 4 * k, d + 4 * k});
        }
        *out = free_status.back();
        free_status.pop_back();
        memset(out->host, 0, 4 * sizeof(int));   // zeroed before the job's kernels are issued
        return cudaSuccess;
    }
    void give_status(const Slot& s) {
        if (s.host) free_status.push_back(s);
    }
    cudaError_t take_event(cudaEvent_t* out) {
        if (free_events.empty()) {
            cudaEvent_t ev = nullptr;
            const cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return e;
            events.push_back(ev);
            free_events.push_back(ev);
        }
        *out = free_events.back();
        free_events.pop_back();
        return cudaSuccess;
    }
    void give_event(cudaEvent_t ev) {
        if (ev) free_events.push_back(ev);
    }
    void destroy() {
        for (auto ev : events) cudaEventDestroy(ev);
        for (auto c : chunks) cudaFreeHost(c);
        events.clear();
        free_events.clear();
        chunks.clear();
        free_status.clear();
    }
};

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
    std::map<int, corr::StreamState*> open_streams;   // by stream_tag
    corr::JobResources res;                           // recycled status words and events (lock held)
    size_t copy_inflight = 0;                         // host-to-device bytes issued and not yet landed
    std::vector<uint64_t> copying;                    // jobs whose copies count against the budget
};

namespace corr {
namespace {

// The X stage of one job into d_vis: packed samples straight into the tensor-core kernel
// when it can read them, else through sample planes in d_ws.
cudaError_t run_x(const Plan& p, const corr_job_desc& d, bool raw, const char* d_packed, void* d_vis, char* d_ws,
                  int accumulate, cudaStream_t s) {
    if (raw)
        return d.sample_bits == 32 ? launch_xeng_tc_rawf32(p, d_packed, 1, d_vis, accumulate, s)
                                   : launch_xeng_tc_raw(p, d_packed, 1, d_vis, accumulate, s);
    if (d.sample_bits == 32) {
        const size_t half = (size_t)p.n_chan * p.nb * kBlockRows * p.kp * 2;
        cudaError_t e = launch_unpack_bf16x2(p, d_packed, 1, d_ws, d_ws + half, s);
        return e == cudaSuccess ? launch_xeng_tc(p, d_ws, d_ws + half, 1, d_vis, accumulate, s) : e;
    }
    return launch_tc_plane_path(p, d_packed, 1, d_ws, d_vis, accumulate, s);
}

// Issue one admitted job on its stream (called with the lock released).
// A job's samples to the device in pieces of at most kCopyPiece bytes: the copy engines serve
// operations in order, so a small job's copy waits behind at most one piece of a large one.
constexpr size_t kCopyPiece = (size_t)64 << 20;
cudaError_t copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (size_t off = 0; off < bytes && e == cudaSuccess; off += kCopyPiece)
        e = cudaMemcpyAsync(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off,
                            std::min(kCopyPiece, bytes - off), cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t issue(corr_server_s* S, Job& j) {
    cudaStream_t s = S->streams[j.stream];
    char* base = S->d_base + j.off;
    char* d_packed = base + round_up(16);
    char* d_vis = d_packed + round_up(packed_bytes(j.desc));
    char* d_ws = d_vis + round_up(vis_bytes(j.desc));
    Plan p = plan_of(j.desc, S->device, S->n_sm);
    // the kernels write the status words straight into the job's mapped pinned slot (zeroed at
    // submission): no copy of 16 bytes queued on a copy engine behind other jobs' large copies
    p.d_status = j.d_status;
    cudaError_t e = cudaEventRecord(j.ev_start, s);
    if (e == cudaSuccess) e = copy_in(d_packed, j.desc.host_packed, packed_bytes(j.desc), s);
    if (e == cudaSuccess) e = cudaEventRecord(j.ev_copied, s);
    if (e == cudaSuccess) e = run_x(p, j.desc, j.raw, d_packed, d_vis, d_ws, 0, s);
    if (e == cudaSuccess && j.desc.host_vis)
        e = cudaMemcpyAsync(j.desc.host_vis, d_vis, vis_bytes(j.desc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(j.ev_done, s);
    return e;
}

// Issue job `seq` of an open stream (called with the lock released; jobs of one stream are
// issued in submission order by the single dispatcher thread).  The copy stream fills ring
// slot seq mod R once the X stage of job seq - R has read it; the compute stream runs the X
// stage into the stream's accumulators and, for the job that ends an interval, the dump.
// With `b` (job seq + 1, in the adjacent slot of a pairable stream) both jobs' samples are
// copied and one X stage over the 2T samples of the two slots adds them into the accumulators:
// one accumulator pass for two jobs.  The later job's status words carry the kernels' status.
cudaError_t issue_stream(corr_server_s* S, Job& j, StreamState& st, Job* b = nullptr) {
    const int R = st.d.ring_slots;
    const int slot = (int)(j.seq % R);
    char* d_packed = st.slots + (size_t)slot * st.slot_bytes;
    Job& last = b ? *b : j;    // the job that may end the interval
    corr_job_desc dx = j.desc;
    if (b) dx.n_time = 2 * j.desc.n_time;
    Plan p = plan_of(dx, S->device, S->n_sm);
    p.d_status = last.d_status;   // mapped pinned status words (see issue())
    const bool sums = st.d.dump_mode == CORR_STREAM_DUMP_SUMS;
    // an interval's first job overwrites the accumulators (the previous interval's dump, issued
    // earlier on the same stream, has read them): that is the reset of Fig. 1, with no extra pass
    const int accumulate = j.seq % st.d.jobs_per_dump == 0 ? 0 : 1;
    cudaError_t e = cudaSuccess;
    if (j.seq >= R) e = cudaStreamWaitEvent(st.copy_s, st.slot_free[slot], 0);
    if (b && e == cudaSuccess && b->seq >= R) e = cudaStreamWaitEvent(st.copy_s, st.slot_free[slot + 1], 0);
    if (e == cudaSuccess) e = cudaEventRecord(j.ev_start, st.copy_s);
    if (e == cudaSuccess)
        e = copy_in(d_packed, j.desc.host_packed, packed_bytes(j.desc), st.copy_s);
    if (e == cudaSuccess) e = cudaEventRecord(j.ev_copied, st.copy_s);
    if (b) {
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_start, st.copy_s);
        if (e == cudaSuccess)
            e = copy_in(d_packed + st.slot_bytes, b->desc.host_packed, packed_bytes(b->desc), st.copy_s);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_copied, st.copy_s);
    }
    const int full = b ? slot + 1 : slot;
    if (e == cudaSuccess) e = cudaEventRecord(st.slot_full[full], st.copy_s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st.comp_s, st.slot_full[full], 0);
    if (e == cudaSuccess) e = run_x(p, dx, st.raw, d_packed, st.acc, st.ws, accumulate, st.comp_s);
    if (e == cudaSuccess) e = cudaEventRecord(st.slot_free[slot], st.comp_s);
    if (b && e == cudaSuccess) e = cudaEventRecord(st.slot_free[slot + 1], st.comp_s);
    if (b && e == cudaSuccess) e = cudaEventRecord(j.ev_done, st.comp_s);   // the first job: X stage done
    Job& jl = last;
    if (e == cudaSuccess && jl.closes) {
        if (sums) {
            e = cudaMemcpyAsync(jl.desc.host_vis, st.acc, vis_bytes(jl.desc), cudaMemcpyDeviceToHost, st.comp_s);
        } else {
            // Fig. 1: read out and divide by the update count (the next job's overwrite resets).
            // The dump buffer must have reached the host from the previous dump first.
            if (st.out_pending) e = cudaStreamWaitEvent(st.comp_s, st.ev_out, 0);
            if (e == cudaSuccess) {
                const corr_status cs = corr_dump(reinterpret_cast<corr_plan>(&p), st.acc, (int)jl.n_accum,
                                                 st.d.d_delays, st.d.d_freqs, st.phasor, st.dumpbuf, 0, st.comp_s);
                if (cs != CORR_OK) e = cudaErrorLaunchFailure;
            }
            if (e == cudaSuccess && jl.desc.host_vis) {
                e = cudaEventRecord(st.ev_dumped, st.comp_s);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st.out_s, st.ev_dumped, 0);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(jl.desc.host_vis, st.dumpbuf, (size_t)p.n_baselines * p.n_chan * 8,
                                        cudaMemcpyDeviceToHost, st.out_s);
                if (e == cudaSuccess) e = cudaEventRecord(st.ev_out, st.out_s);
                if (e == cudaSuccess) {
                    st.out_pending = true;
                    // the job is done when its dump is in host memory
                    return cudaEventRecord(jl.ev_done, st.out_s);
                }
            }
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(jl.ev_done, st.comp_s);
    return e;
}

// Copies in flight are capped so that a job with an early deadline never queues behind a
// backlog of other jobs' copies (copy engines serve operations in order): a job may start its
// copy when nothing is in flight or its bytes fit the budget with what is.
constexpr size_t kCopyBudget = (size_t)256 << 20;
// Deadlines: a job's own sample time at the paper's channel rate (1.28 MHz over 128 channels =
// 10 kHz); only their order matters, so the rate is a scale, the same for every job.
constexpr double kChannelRateHz = 10000.0;
bool copy_fits(const corr_server_s* S, size_t bytes) {
    return S->copy_inflight == 0 || S->copy_inflight + bytes <= kCopyBudget;
}

// The next job the dispatcher may issue, earliest deadline first among the candidates: the
// first queued job of each open stream (a stream's jobs keep their order: ring slots, intervals)
// once its ring slot is free on the device, and the first other job once it fits the arena's
// free space (the others wait behind it in arrival order).  The earliest candidate is issued
// when its copy fits the budget; otherwise nothing is, until the copies in flight drain (a later
// deadline never overtakes it, so a large job is not starved by a stream of small ones).
// Called with the lock held.
bool pick_next(corr_server_s* S, std::deque<uint64_t>::iterator* pick) {
    bool arena_head_seen = false, found = false;
    double best = 0;
    std::vector<const StreamState*> heads;
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        const Job& j = S->jobs[*it];
        bool ready = false;
        if (j.stream_job) {
            if (std::find(heads.begin(), heads.end(), j.st) != heads.end()) continue;
            heads.push_back(j.st);
            const int R = j.st->d.ring_slots;
            ready = j.seq < R || cudaEventQuery(j.st->slot_free[(int)(j.seq % R)]) != cudaErrorNotReady;
        } else if (!arena_head_seen) {
            arena_head_seen = true;
            ready = S->arena->fits(j.bytes);
        }
        if (ready && (!found || j.deadline < best)) {
            found = true;
            best = j.deadline;
            *pick = it;
        }
    }
    return found && copy_fits(S, packed_bytes(S->jobs[**pick].desc));
}

// The queued job that can join a picked stream job in one X stage (issue_stream with `b`): the
// stream's next job, already queued, in the adjacent ring slot (no wrap), the picked job not
// ending the interval, the later slot free on the device and both copies within the budget.
// Called with the lock held; returns the partner's queue position or end().
std::deque<uint64_t>::iterator pair_partner(corr_server_s* S, std::deque<uint64_t>::iterator pick) {
    const Job& j = S->jobs[*pick];
    const StreamState* st = j.st;
    const int R = st->d.ring_slots;
    if (!st->pairable || j.closes || (int)(j.seq % R) + 1 >= R) return S->queue.end();
    for (auto it = std::next(pick); it != S->queue.end(); ++it) {
        const Job& c = S->jobs[*it];
        if (!c.stream_job || c.st != st) continue;
        // a stream's jobs queue in submission order, so this is job seq + 1
        if (c.seq != j.seq + 1) return S->queue.end();
        const bool free = c.seq < R || cudaEventQuery(st->slot_free[(int)(c.seq % R)]) != cudaErrorNotReady;
        if (!free || !copy_fits(S, packed_bytes(j.desc) + packed_bytes(c.desc))) return S->queue.end();
        return it;
    }
    return S->queue.end();
}

void dispatcher_loop(corr_server_s* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (true) {
        std::deque<uint64_t>::iterator pick;
        bool have = false;
        // queued jobs blocked on a ring slot or on the copy budget are looked at again soon
        // (the completion thread also wakes this thread when copies land or jobs finish)
        const auto wait = S->queue.empty() ? std::chrono::microseconds(50000) : std::chrono::microseconds(500);
        S->cv_dispatch.wait_for(lock, wait, [&] {
            if (S->stop) return true;
            if (S->paused || S->queue.empty()) return false;
            have = pick_next(S, &pick);
            return have;
        });
        if (S->stop) break;
        if (!have) continue;
        const uint64_t id = *pick;
        Job& j = S->jobs[id];
        cudaError_t e = cudaSuccess;
        Job* b = nullptr;   // a stream job's partner in one X stage (pair_partner)
        if (j.stream_job) {
            const auto partner = pair_partner(S, pick);
            const uint64_t id_b = partner != S->queue.end() ? *partner : 0;
            S->queue.erase(pick);   // invalidates `partner`
            if (id_b) {
                S->queue.erase(std::find(S->queue.begin(), S->queue.end(), id_b));
                b = &S->jobs[id_b];
            }
            j.state = kRunning;
            j.t_start = now_s();
            StreamState* st = j.st;
            j.copy_bytes = packed_bytes(j.desc);
            S->copy_inflight += j.copy_bytes;
            if (b) {
                b->state = kRunning;
                b->t_start = j.t_start;
                b->copy_bytes = packed_bytes(b->desc);
                S->copy_inflight += b->copy_bytes;
                j.h_status_pair = b->h_status;
                S->stats.coalesced += 2;
            }
            lock.unlock();
            e = issue_stream(S, j, *st, b);
            lock.lock();
        } else {
            size_t off;
            if (!S->arena->alloc(j.bytes, &off)) continue;   // cannot happen: fits() held under the lock
            S->queue.erase(pick);
            j.off = off;
            j.holds_arena = true;
            j.stream = S->next_stream;
            S->next_stream = (S->next_stream + 1) % (int)S->streams.size();
            j.state = kRunning;
            j.t_start = now_s();
            j.d_vis = S->d_base + off + round_up(16) + round_up(packed_bytes(j.desc));   // layout of issue()
            S->stats.bytes_in_use = S->arena->used();
            S->stats.peak_bytes = S->arena->peak();
            j.copy_bytes = packed_bytes(j.desc);
            S->copy_inflight += j.copy_bytes;
            lock.unlock();
            e = issue(S, j);
            lock.lock();
        }
        // the completion thread sees the job only once its events are recorded
        if (e == cudaSuccess) {
            S->running.push_back(id);
            S->copying.push_back(id);
            if (b) {
                S->running.push_back(b->id);
                S->copying.push_back(b->id);
            }
        }
        if (e != cudaSuccess) {
            // nothing of this job is queued behind a failed call that we can rely on; mark it
            // failed once its stream has drained the calls that were accepted
            cudaStreamSynchronize(j.stream_job ? j.st->comp_s : S->streams[j.stream]);
            if (j.stream_job) {
                cudaStreamSynchronize(j.st->copy_s);
                cudaStreamSynchronize(j.st->out_s);
            }
            for (Job* f : {&j, b}) {
                if (!f) continue;
                S->copy_inflight -= f->copy_bytes;
                f->copy_bytes = 0;
                f->state = kFailed;
                f->final_status = CORR_ECUDA;
                f->t_done = now_s();
                if (f->holds_arena) {
                    S->arena->release(f->off, f->bytes);
                    f->holds_arena = false;
                }
                if (f->stream_job) f->st->n_retired++;
                S->stats.failed++;
            }
            S->cv_done.notify_all();
        }
    }
}

void completer_loop(corr_server_s* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (true) {
        bool progressed = false;
        // copies that have landed give their bytes back to the copy budget
        for (size_t k = 0; k < S->copying.size();) {
            Job& j = S->jobs[S->copying[k]];
            if (cudaEventQuery(j.ev_copied) == cudaErrorNotReady) {
                ++k;
                continue;
            }
            S->copy_inflight -= j.copy_bytes;
            j.copy_bytes = 0;
            S->copying[k] = S->copying.back();
            S->copying.pop_back();
            progressed = true;
        }
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
            } else if ((j.h_status_pair ? j.h_status_pair : j.h_status)[0] != 0) {
                // (a job issued with its stream's next one reads that job's words, which stay
                // valid: the partner's completion event follows this one's)
                j.state = kFailed;
                j.final_status = CORR_ETIMEOUT;   // a bounded device wait gave up
            } else {
                j.state = kDone;
                j.final_status = CORR_OK;
            }
            if (j.state == kDone) S->stats.completed++;
            else S->stats.failed++;
            if (j.copy_bytes) {
                // its copy preceded its completion event, whichever of the two this pass saw
                // first: settle the copy budget before the job can be released
                S->copy_inflight -= j.copy_bytes;
                j.copy_bytes = 0;
                const auto at = std::find(S->copying.begin(), S->copying.end(), S->running[k]);
                if (at != S->copying.end()) S->copying.erase(at);
            }
            if (j.stream_job) {
                // an averaged dump left on the device stays in the stream's dump buffer
                j.d_vis = (j.state == kDone && j.closes && !j.desc.host_vis &&
                           j.st->d.dump_mode == CORR_STREAM_DUMP_AVERAGED)
                              ? j.st->dumpbuf
                              : nullptr;
                j.st->n_retired++;
            } else if (j.desc.host_vis || j.state != kDone) {
                // results copied to the host free their device block now; device-resident
                // results stay until corr_release
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

// Destroy an open stream's streams and events (its work must be finished) and give its block
// back to the arena (lock held by the caller, or the server's threads stopped).
void free_stream_state(corr_server_s* S, StreamState* st) {
    if (st->copy_s) cudaStreamSynchronize(st->copy_s);
    if (st->comp_s) cudaStreamSynchronize(st->comp_s);
    if (st->out_s) cudaStreamSynchronize(st->out_s);
    if (st->ev_dumped) cudaEventDestroy(st->ev_dumped);
    if (st->ev_out) cudaEventDestroy(st->ev_out);
    if (st->out_s) cudaStreamDestroy(st->out_s);
    for (auto ev : st->slot_full)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : st->slot_free)
        if (ev) cudaEventDestroy(ev);
    if (st->copy_s) cudaStreamDestroy(st->copy_s);
    if (st->comp_s) cudaStreamDestroy(st->comp_s);
    if (st->bytes) S->arena->release(st->off, st->bytes);
    delete st;
}

void fill_result(const Job& j, corr_job_result* r) {
    r->status = j.state == kQueued || j.state == kRunning ? CORR_PENDING : j.final_status;
    r->t_submit = j.t_submit;
    r->t_start = j.t_start;
    r->t_done = j.t_done;
    r->gpu_ms = j.gpu_ms;
    r->d_vis = j.d_vis;
    r->closed_interval = j.stream_job && j.closes ? 1 : 0;
    r->n_accum = j.stream_job && j.closes ? j.n_accum : 0;
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
    {   // the first chunk of pinned status words now, not under the lock of the first submission
        JobResources::Slot warm{};
        if (S->res.take_status(&warm) == cudaSuccess) S->res.give_status(warm);
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
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->stop) return set_error(CORR_EBUSY, "server is shutting down");
    auto sit = S->open_streams.find(d->stream_tag);
    StreamState* st = sit == S->open_streams.end() ? nullptr : sit->second;
    if (st) {
        // a job of an open stream: its shape is the stream's, its place is the next ring slot
        if (st->closing) return set_error(CORR_EINVAL, "stream %d is closing", d->stream_tag);
        if (d->n_inputs != st->d.n_inputs || d->n_chan != st->d.n_chan || d->n_time != st->d.n_time ||
            d->sample_bits != st->d.sample_bits)
            return set_error(CORR_EINVAL, "job shape differs from the shape stream %d was opened with",
                             d->stream_tag);
        j.stream_job = true;
        j.st = st;
        j.seq = st->n_submitted;
        j.closes = (j.seq + 1) % st->d.jobs_per_dump == 0;
        j.n_accum = j.closes ? (int64_t)st->d.jobs_per_dump * st->d.n_time : 0;
        j.raw = st->raw;
        j.bytes = 0;
        if (j.closes && st->d.dump_mode == CORR_STREAM_DUMP_SUMS && !d->host_vis)
            return set_error(CORR_EINVAL, "job %lld of stream %d ends a dump interval: host_vis must receive the sums",
                             (long long)j.seq, d->stream_tag);
    } else {
        j.bytes = footprint(*d, &j.raw);
        if (j.bytes > S->arena->size()) {
            S->stats.rejected++;
            return set_error(CORR_EBUSY, "job needs %zu device bytes, more than the %zu-byte HBM budget", j.bytes,
                             S->arena->size());
        }
    }
    cudaError_t e = S->res.take_event(&j.ev_start);
    if (e == cudaSuccess) e = S->res.take_event(&j.ev_done);
    if (e == cudaSuccess) e = S->res.take_event(&j.ev_copied);
    JobResources::Slot slot{};
    if (e == cudaSuccess) e = S->res.take_status(&slot);
    j.h_status = slot.host;
    j.d_status = slot.dev;
    if (e != cudaSuccess) {
        S->res.give_event(j.ev_start);
        S->res.give_event(j.ev_done);
        S->res.give_event(j.ev_copied);
        return cuda_error(e, "corr_submit");
    }
    if (st) st->n_submitted++;
    j.id = S->next_id++;
    j.t_submit = now_s();
    j.deadline = j.t_submit + (double)d->n_time / kChannelRateHz;
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
    S->res.give_event(j.ev_start);
    S->res.give_event(j.ev_done);
    S->res.give_event(j.ev_copied);
    S->res.give_status(JobResources::Slot{j.h_status, j.d_status});
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
        if (!j.d_vis) return set_error(CORR_EINVAL, "job %llu did not keep its result on the device",
                                       (unsigned long long)job_id);
        src = j.d_vis;
        // an open stream's averaged dump is float32; any other kept result is the job's visibilities
        bytes = j.stream_job ? (size_t)n_baselines(j.desc.n_inputs) * j.desc.n_chan * 8 : vis_bytes(j.desc);
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
    st->open_streams = (int64_t)S->open_streams.size();
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
    // the dispatcher issues nothing more once it sees stop (it may be finishing one issue now);
    // then the streams must be idle before the arena goes away: wait for them (the kernels' own
    // waits are bounded, so this returns), and the completion thread retires what is left
    S->dispatcher.join();
    for (auto st : S->streams) cudaStreamSynchronize(st);
    for (auto& kv : S->open_streams) {
        cudaStreamSynchronize(kv.second->copy_s);
        cudaStreamSynchronize(kv.second->comp_s);
        cudaStreamSynchronize(kv.second->out_s);
    }
    S->completer.join();
    S->res.destroy();   // every job's events and status words came from the pools
    for (auto& kv : S->open_streams) free_stream_state(S, kv.second);
    S->open_streams.clear();
    for (auto st : S->streams) cudaStreamDestroy(st);
    cudaFree(S->d_base);
    delete S->arena;
    delete S;
    return result;
}

corr_status corr_server_open_stream(corr_server S, int stream_tag, const corr_stream_desc* d) {
    if (!S || !d) return set_error(CORR_EINVAL, "corr_server_open_stream: NULL argument");
    if (d->sample_bits != 4 && d->sample_bits != 8 && d->sample_bits != 32)
        return set_error(CORR_EINVAL, "sample_bits=%d must be 4, 8 or 32", d->sample_bits);
    if (d->n_inputs < 1 || d->n_inputs > kMaxInputs || d->n_chan < 1 || d->n_time < 1)
        return set_error(CORR_EINVAL, "bad stream sizes N=%d C=%d T=%d", d->n_inputs, d->n_chan, d->n_time);
    if (d->ring_slots < 1 || d->ring_slots > 64) return set_error(CORR_EINVAL, "ring_slots=%d outside [1, 64]", d->ring_slots);
    if (d->jobs_per_dump < 1) return set_error(CORR_EINVAL, "jobs_per_dump=%d must be >= 1", d->jobs_per_dump);
    if (d->dump_mode != CORR_STREAM_DUMP_SUMS && d->dump_mode != CORR_STREAM_DUMP_AVERAGED)
        return set_error(CORR_EINVAL, "unknown dump_mode %d", d->dump_mode);
    if (d->dump_mode == CORR_STREAM_DUMP_AVERAGED && (int64_t)d->jobs_per_dump * d->n_time > INT32_MAX)
        return set_error(CORR_EINVAL, "an averaged dump sums more than 2^31 samples");
    if (d->d_delays && !d->d_freqs) return set_error(CORR_EINVAL, "delays need channel frequencies");
    if ((double)n_baselines(d->n_inputs) * d->n_chan * 16.0 > 4.0e15) return set_error(CORR_EINVAL, "stream too large");
    StreamState* st = new (std::nothrow) StreamState();
    if (!st) return set_error(CORR_ENOMEM, "host allocation failed");
    st->d = *d;
    if (st->d.dump_mode != CORR_STREAM_DUMP_AVERAGED) {
        st->d.d_delays = nullptr;
        st->d.d_freqs = nullptr;
    }
    const Plan p = plan_of(shape_of(*d), 0, 0);
    st->raw = d->sample_bits == 32 ? tc_rawf32_supported(p) : !tc_use_planes(p);
    const size_t need = stream_layout(*st, nullptr);
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->stop) {
        delete st;
        return set_error(CORR_EBUSY, "server is shutting down");
    }
    if (S->open_streams.count(stream_tag)) {
        delete st;
        return set_error(CORR_EINVAL, "stream %d is already open", stream_tag);
    }
    size_t off = 0;
    if (need > S->arena->size() || !S->arena->alloc(need, &off)) {
        const size_t arena = S->arena->size();
        delete st;
        return set_error(CORR_EBUSY, "stream %d needs %zu device bytes (ring, accumulators, dump); the %zu-byte "
                                     "arena has not that much free now", stream_tag, need, arena);
    }
    st->off = off;
    st->bytes = need;
    stream_layout(*st, S->d_base + off);
    // deadline-aware priority: a job must be correlated within its own sample time, so streams
    // with shorter dumps get the higher priority when the GPU picks the next kernel to run
    int lo_prio = 0, hi_prio = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    int prio = lo_prio;
    if (e == cudaSuccess && hi_prio < lo_prio) {
        // 1024 samples or more: the lowest; each halving of the sample time one step higher
        int steps = 0;
        for (int t = d->n_time; t < 1024 && steps < lo_prio - hi_prio; t *= 2) ++steps;
        prio = lo_prio - steps;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&st->copy_s, cudaStreamNonBlocking, prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&st->comp_s, cudaStreamNonBlocking, prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&st->out_s, cudaStreamNonBlocking, prio);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_dumped, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_out, cudaEventDisableTiming);
    st->slot_full.assign(d->ring_slots, nullptr);
    st->slot_free.assign(d->ring_slots, nullptr);
    for (int k = 0; k < d->ring_slots && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&st->slot_full[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->slot_free[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        free_stream_state(S, st);
        return cuda_error(e, "corr_server_open_stream");
    }
    S->open_streams[stream_tag] = st;
    S->stats.bytes_in_use = S->arena->used();
    S->stats.peak_bytes = S->arena->peak();
    return CORR_OK;
}

corr_status corr_server_close_stream(corr_server S, int stream_tag, double drain_timeout_s) {
    if (!S) return set_error(CORR_EINVAL, "corr_server_close_stream: NULL server");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->open_streams.find(stream_tag);
    if (it == S->open_streams.end()) return set_error(CORR_EINVAL, "stream %d is not open", stream_tag);
    StreamState* st = it->second;
    st->closing = true;
    corr_status result = CORR_OK;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(drain_timeout_s > 0 ? drain_timeout_s : 0));
    S->cv_done.wait_until(lock, deadline, [&] { return st->n_retired == st->n_submitted; });
    if (st->n_retired != st->n_submitted) {
        result = set_error(CORR_ETIMEOUT, "stream %d: %lld jobs unfinished after %.1f s", stream_tag,
                           (long long)(st->n_submitted - st->n_retired), drain_timeout_s);
        // jobs not yet issued never will be; issued ones are waited for on the GPU
        for (auto q = S->queue.begin(); q != S->queue.end();) {
            Job& j = S->jobs[*q];
            if (j.stream_job && j.st == st) {
                j.state = kCancelled;
                j.final_status = CORR_EBUSY;
                st->n_retired++;
                S->stats.cancelled++;
                q = S->queue.erase(q);
            } else {
                ++q;
            }
        }
        lock.unlock();
        cudaStreamSynchronize(st->copy_s);
        cudaStreamSynchronize(st->comp_s);
        cudaStreamSynchronize(st->out_s);
        lock.lock();
        // the completion thread retires the issued jobs once their events are complete
        S->cv_done.wait_for(lock, std::chrono::seconds(10), [&] { return st->n_retired == st->n_submitted; });
        if (st->n_retired != st->n_submitted) {
            S->open_streams.erase(stream_tag);   // jobs still reference the state: keep it alive
            return result;
        }
    }
    S->open_streams.erase(stream_tag);
    // finished jobs keep no pointer into the state except their dump result, which goes now
    for (auto& kv : S->jobs)
        if (kv.second.st == st) {
            kv.second.st = nullptr;
            kv.second.d_vis = nullptr;
        }
    free_stream_state(S, st);
    S->stats.bytes_in_use = S->arena->used();
    S->cv_dispatch.notify_all();
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

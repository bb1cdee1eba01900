// Serving form of the C ABI (include/gempe.h): embedding jobs admitted by
// device-memory budget and run with continuous batching.
//
// Native threads per server:
//  - admission workers (a small pool) take submitted jobs in arrival order
//    and validate their CSR on the host in parallel; each job then waits for
//    its turn -- capacity is reserved strictly in arrival order -- until a
//    job slot is free and the job's device bytes fit in the budget next to
//    the running jobs; the worker then builds the job's device-resident
//    state (CSR, edge set, positions, accumulators; a pack of one graph,
//    stream-ordered allocations on the slot's stream) and captures its epoch
//    graphs, while other workers build other jobs;
//  - one stepper keeps every running job's epochs in flight on its own
//    stream (chunks of up to kChunk epochs, at most two chunks ahead), so
//    the kernels of all running jobs overlap on the device; a job whose
//    epochs are done has its positions copied to pinned host memory and its
//    device memory released, which lets the next job in line start.
// A job's arithmetic is the same as gempe_create + gempe_step with the
// job's seed: only the order of FP32 atomic additions can differ.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.cuh"
#include "gempe.h"
#include "pack.cuh"

#define GEMPE_API extern "C" __attribute__((visibility("default")))

using namespace gempe;

namespace {

constexpr int kChunk = 10;          // epochs per captured chunk
constexpr int kInFlight = 2;        // chunks enqueued ahead per job

enum JobState { kQueued = 0, kRunning = 1, kDone = 2 };

struct Job;

void* job_alloc(size_t bytes, void* user);
void job_free(void* ptr, void* user);

struct Job {
    uint64_t id = 0;
    uint64_t ticket = 0;                // arrival order: capacity is reserved in this order
    std::vector<int32_t> rp, ci;
    int32_t n = 0, d = 0, epochs = 0;
    uint64_t seed = 0;
    size_t bytes = 0;
    std::atomic<int> state{kQueued};    // kQueued, kRunning, kDone, or a negative gempe_status
    std::string error;
    uint64_t submit_ns = 0, admit_ns = 0, done_ns = 0;
    uint64_t pairs = 0;
    float final_sigma = 0.0f;
    std::atomic<int32_t> epochs_done{0};
    // running
    int slot = -1;
    cudaStream_t stream = nullptr;
    std::unique_ptr<Pack> pk;
    cudaGraphExec_t g1 = nullptr, gc = nullptr;     // one epoch, kChunk epochs
    cudaGraph_t gr1 = nullptr, grc = nullptr;
    struct Flight {
        cudaEvent_t ev;
        int epochs;
    };
    std::deque<Flight> inflight;
    std::vector<cudaEvent_t> free_events;
    int32_t enqueued = 0;
    bool copying = false;
    cudaEvent_t done_ev = nullptr;
    float* host_x = nullptr;            // pinned, n * d
    size_t host_x_bytes = 0;
    GraphState* host_state = nullptr;   // pinned, the slot's
    PackState* host_ps = nullptr;       // pinned, the slot's

    void release_device() {
        if (gc) cudaGraphExecDestroy(gc);
        if (g1) cudaGraphExecDestroy(g1);
        if (grc) cudaGraphDestroy(grc);
        if (gr1) cudaGraphDestroy(gr1);
        gc = g1 = nullptr;
        grc = gr1 = nullptr;
        pk.reset();   // synchronises the slot stream, frees through job_free
        for (auto& f : inflight) cudaEventDestroy(f.ev);
        inflight.clear();
        for (cudaEvent_t e : free_events) cudaEventDestroy(e);
        free_events.clear();
        if (done_ev) cudaEventDestroy(done_ev);
        done_ev = nullptr;
    }
};

void* job_alloc(size_t bytes, void* user) {
    Job* j = static_cast<Job*>(user);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, j->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void job_free(void* ptr, void* user) {
    Job* j = static_cast<Job*>(user);
    cudaFreeAsync(ptr, j->stream);
}

uint64_t now_ns(std::chrono::steady_clock::time_point t0) {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
        .count();
}

}  // namespace

struct gempe_server {
    gempe_params p{};
    size_t budget = 0, in_use = 0, peak_in_use = 0;
    int device = 0;
    std::vector<cudaStream_t> slot_streams;
    std::vector<char> slot_busy;
    GraphState* slot_state = nullptr;   // pinned [max_jobs]: a finished job's final graph state
    PackState* slot_ps = nullptr;       // pinned [max_jobs]
    std::mutex mu;
    std::condition_variable cv_pending, cv_capacity, cv_done, cv_work;
    std::deque<Job*> pending;           // submitted, not yet taken by a worker
    size_t waiting = 0;                 // taken by a worker, capacity not yet reserved
    uint64_t next_ticket = 0, tickets = 0;
    std::vector<Job*> active;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    uint64_t next_id = 1;
    uint64_t completed = 0, failed = 0;
    std::atomic<bool> stop{false};
    std::vector<std::thread> admitters;
    std::thread stepper;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    // pinned host buffers kept for reuse (freeing pinned memory can synchronise the device)
    std::multimap<size_t, float*> pinned_pool;
    std::vector<void*> pinned_all;

    float* take_pinned(size_t bytes) {
        {
            std::lock_guard<std::mutex> lock(mu);
            auto it = pinned_pool.lower_bound(bytes);
            if (it != pinned_pool.end() && it->first <= 2 * bytes + 4096) {
                float* b = it->second;
                pinned_pool.erase(it);
                return b;
            }
        }
        void* ptr = nullptr;
        if (cudaHostAlloc(&ptr, bytes, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        std::lock_guard<std::mutex> lock(mu);
        pinned_all.push_back(ptr);
        return (float*)ptr;
    }
    void give_pinned_locked(float* b, size_t bytes) {
        if (b) pinned_pool.emplace(bytes, b);
    }

    void admit_loop();
    void step_loop();
    gempe_status start_job(Job* j);
    void finish_job(Job* j, int status);
};

// ---------------------------------------------------------------------------
// admitter
// ---------------------------------------------------------------------------
gempe_status gempe_server::start_job(Job* j) {
    gempe_params pp = p;
    pp.seed = j->seed;
    if (j->d < 8) {
        pp.precision = 0;
        pp.block_partners = 0;
    }
    pp.autotune = 0;
    pp.dev_alloc = job_alloc;
    pp.dev_free = job_free;
    pp.alloc_user = j;
    j->pk.reset(new Pack());
    std::vector<GraphInput> in(1);
    in[0].row_ptr = j->rp.data();
    in[0].col_idx = j->ci.data();
    in[0].n = j->n;
    in[0].key = j->seed;
    gempe_status rc = j->pk->build(in, j->d, pp, j->stream, false);
    if (rc != GEMPE_OK) return rc;
    Pack& pk = *j->pk;
    rc = pk.prime();
    if (rc != GEMPE_OK) return rc;
    // epoch graphs: one epoch and kChunk epochs
    for (int which = 0; which < 2; ++which) {
        const int reps = which == 0 ? 1 : kChunk;
        if (which == 1 && j->epochs < kChunk) break;
        cudaError_t e = cudaStreamBeginCapture(j->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return pack_cuda_fail(e, "begin capture");
        for (int r = 0; r < reps && rc == GEMPE_OK; ++r) {
            rc = pk.enqueue_sweep();
            if (rc == GEMPE_OK) rc = pk.enqueue_update();
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(j->stream, &g);
        if (rc != GEMPE_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc != GEMPE_OK ? rc : pack_cuda_fail(e, "end capture");
        }
        cudaGraphExec_t x = nullptr;
        e = cudaGraphInstantiate(&x, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return pack_cuda_fail(e, "graph instantiate");
        }
        if (which == 0) {
            j->gr1 = g;
            j->g1 = x;
        } else {
            j->grc = g;
            j->gc = x;
        }
    }
    for (int q = 0; q < kInFlight; ++q) {
        cudaEvent_t ev = nullptr;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return pack_cuda_fail(e, "cudaEventCreate");
        j->free_events.push_back(ev);
    }
    cudaError_t e = cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return pack_cuda_fail(e, "cudaEventCreate");
    return GEMPE_OK;
}

void gempe_server::finish_job(Job* j, int status) {
    j->release_device();
    std::lock_guard<std::mutex> lock(mu);
    in_use -= j->bytes;
    if (j->slot >= 0) slot_busy[j->slot] = 0;
    j->slot = -1;
    j->done_ns = now_ns(t0);
    if (status == kDone) ++completed;
    else ++failed;
    j->state.store(status);
    active.erase(std::remove(active.begin(), active.end(), j), active.end());
    cv_capacity.notify_all();
    cv_done.notify_all();
}

void gempe_server::admit_loop() {
    cudaSetDevice(device);
    for (;;) {
        Job* j = nullptr;
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_pending.wait(lock, [&] { return stop.load() || !pending.empty(); });
            if (stop.load()) return;
            j = pending.front();
            pending.pop_front();
            ++waiting;
        }
        // the rows checked on the host, in parallel with other workers (one
        // thread each); the symmetry on the device when the job starts
        const gempe_status vrc = validate_csr(j->rp.data(), j->ci.data(), j->n, 1, false);
        const std::string verr = vrc != GEMPE_OK ? std::string(gempe_last_error()) : std::string();
        int slot = -1;
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_capacity.wait(lock, [&] {
                if (stop.load()) return true;
                if (j->ticket != next_ticket) return false;
                if (vrc != GEMPE_OK) return true;
                if (in_use + j->bytes > budget) return false;
                for (size_t s2 = 0; s2 < slot_busy.size(); ++s2)
                    if (!slot_busy[s2]) return true;
                return false;
            });
            if (stop.load()) return;
            --waiting;
            ++next_ticket;
            if (vrc != GEMPE_OK) {
                j->error = verr;
                j->done_ns = now_ns(t0);
                ++failed;
                j->state.store(vrc);
                cv_capacity.notify_all();
                cv_done.notify_all();
                continue;
            }
            for (size_t s2 = 0; s2 < slot_busy.size(); ++s2)
                if (!slot_busy[s2]) {
                    slot = (int)s2;
                    break;
                }
            slot_busy[slot] = 1;
            in_use += j->bytes;
            peak_in_use = std::max(peak_in_use, in_use);
            j->slot = slot;
            j->stream = slot_streams[slot];
            j->host_state = slot_state + slot;
            j->host_ps = slot_ps + slot;
            j->admit_ns = now_ns(t0);
            cv_capacity.notify_all();   // the next ticket may proceed
        }
        j->host_x_bytes = sizeof(float) * (size_t)j->n * j->d;
        j->host_x = take_pinned(j->host_x_bytes);
        gempe_status rc = j->host_x ? start_job(j) : pack_fail(GEMPE_E_OOM, "pinned host buffer");
        if (rc != GEMPE_OK) {
            j->error = gempe_last_error();
            finish_job(j, rc);
            continue;
        }
        {
            std::lock_guard<std::mutex> lock(mu);
            j->state.store(kRunning);
            active.push_back(j);
        }
        cv_work.notify_all();
    }
}

// ---------------------------------------------------------------------------
// stepper
// ---------------------------------------------------------------------------
void gempe_server::step_loop() {
    cudaSetDevice(device);
    std::vector<Job*> snap;
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_work.wait_for(lock, std::chrono::milliseconds(50), [&] { return stop.load() || !active.empty(); });
            if (stop.load()) return;
            snap = active;
        }
        bool progressed = false;
        for (Job* j : snap) {
            // retire finished chunks
            while (!j->inflight.empty()) {
                const cudaError_t q = cudaEventQuery(j->inflight.front().ev);
                if (q == cudaErrorNotReady) break;
                if (q != cudaSuccess) {
                    j->error = std::string("epoch chunk: ") + cudaGetErrorString(q);
                    cudaGetLastError();
                    break;
                }
                j->epochs_done += j->inflight.front().epochs;
                j->free_events.push_back(j->inflight.front().ev);
                j->inflight.pop_front();
                progressed = true;
            }
            if (!j->error.empty()) {
                finish_job(j, GEMPE_E_CUDA);
                progressed = true;
                continue;
            }
            if (j->copying) {
                const cudaError_t q = cudaEventQuery(j->done_ev);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess || j->host_ps->status != 0) {
                    j->error = q != cudaSuccess ? std::string("result copy: ") + cudaGetErrorString(q)
                                                : std::string("a position became non-finite during an update");
                    finish_job(j, q != cudaSuccess ? GEMPE_E_CUDA : j->host_ps->status);
                } else {
                    j->pairs = (uint64_t)j->epochs * (uint64_t)(j->pk->nnz[0] / 2) + j->host_state->used;
                    j->final_sigma = j->host_state->sigma;
                    finish_job(j, kDone);
                }
                progressed = true;
                continue;
            }
            while ((int)j->inflight.size() < kInFlight && j->enqueued < j->epochs) {
                const int c = (j->gc && j->epochs - j->enqueued >= kChunk) ? kChunk : 1;
                cudaError_t e = cudaGraphLaunch(c == kChunk ? j->gc : j->g1, j->stream);
                cudaEvent_t ev = j->free_events.back();
                if (e == cudaSuccess) e = cudaEventRecord(ev, j->stream);
                if (e != cudaSuccess) {
                    j->error = std::string("epoch launch: ") + cudaGetErrorString(e);
                    break;
                }
                j->free_events.pop_back();
                j->inflight.push_back(Job::Flight{ev, c});
                j->enqueued += c;
                progressed = true;
            }
            if (!j->error.empty()) continue;
            if (j->enqueued == j->epochs && j->inflight.empty()) {
                Pack& pk = *j->pk;
                cudaError_t e = cudaMemcpyAsync(j->host_x, pk.x, j->host_x_bytes, cudaMemcpyDeviceToHost, j->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(j->host_state, pk.gst, sizeof(GraphState), cudaMemcpyDeviceToHost, j->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(j->host_ps, pk.ps, sizeof(PackState), cudaMemcpyDeviceToHost, j->stream);
                if (e == cudaSuccess) e = cudaEventRecord(j->done_ev, j->stream);
                if (e != cudaSuccess) j->error = std::string("result copy: ") + cudaGetErrorString(e);
                j->copying = true;
                progressed = true;
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
GEMPE_API size_t gempe_job_bytes(int32_t n, int64_t nnz, int32_t d, const gempe_params* p) {
    if (!p || n < 2 || nnz < 0 || !supported_dim(d)) return 0;
    return Pack::bytes_for(n, nnz, d, *p);
}

GEMPE_API gempe_status gempe_server_create(size_t hbm_budget_bytes, int32_t max_jobs, const gempe_params* p,
                                           gempe_server** out) {
    if (!out || !p) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    *out = nullptr;
    if (max_jobs < 1 || max_jobs > 256) return pack_fail(GEMPE_E_INVALID_ARG, "max_jobs must be in [1, 256]");
    if (hbm_budget_bytes == 0) return pack_fail(GEMPE_E_INVALID_ARG, "the budget must be positive");
    gempe_status rc = check_params(p, 8);
    if (rc != GEMPE_OK) return rc;
    if (p->dev_alloc) return pack_fail(GEMPE_E_INVALID_ARG, "the server allocates stream-ordered itself");
    std::unique_ptr<gempe_server> s(new gempe_server());
    s->p = *p;
    s->budget = hbm_budget_bytes;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return pack_cuda_fail(e, "cudaGetDevice");
    e = ensure_mills_table();
    if (e != cudaSuccess) return pack_cuda_fail(e, "Mills table");
    for (int q = 0; q < max_jobs; ++q) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t x : s->slot_streams) cudaStreamDestroy(x);
            return pack_cuda_fail(e, "cudaStreamCreate");
        }
        s->slot_streams.push_back(st);
    }
    s->slot_busy.assign(max_jobs, 0);
    void* hs = nullptr;
    void* hp = nullptr;
    e = cudaHostAlloc(&hs, sizeof(GraphState) * max_jobs, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&hp, sizeof(PackState) * max_jobs, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        if (hs) cudaFreeHost(hs);
        for (cudaStream_t x : s->slot_streams) cudaStreamDestroy(x);
        return pack_cuda_fail(e, "pinned host memory");
    }
    s->slot_state = (GraphState*)hs;
    s->slot_ps = (PackState*)hp;
    gempe_server* raw = s.release();
    const unsigned hw = std::thread::hardware_concurrency();
    const int workers = std::max(2, std::min(8, (int)(hw ? hw / 2 : 2)));
    for (int q = 0; q < workers; ++q) raw->admitters.emplace_back([raw] { raw->admit_loop(); });
    raw->stepper = std::thread([raw] { raw->step_loop(); });
    *out = raw;
    return GEMPE_OK;
}

GEMPE_API void gempe_server_destroy(gempe_server* s) {
    if (!s) return;
    s->stop.store(true);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->cv_pending.notify_all();
        s->cv_capacity.notify_all();
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    for (auto& t : s->admitters)
        if (t.joinable()) t.join();
    if (s->stepper.joinable()) s->stepper.join();
    for (auto& kv : s->jobs) kv.second->release_device();
    for (cudaStream_t st : s->slot_streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (void* b : s->pinned_all) cudaFreeHost(b);
    cudaFreeHost(s->slot_state);
    cudaFreeHost(s->slot_ps);
    delete s;
}

GEMPE_API gempe_status gempe_server_submit(gempe_server* s, const gempe_job_desc* job, uint64_t* job_id) {
    if (!s || !job || !job_id) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    if (job->n < 2 || !job->row_ptr || !supported_dim(job->d) || job->epochs < 1)
        return pack_fail(GEMPE_E_INVALID_ARG, "need n >= 2, row_ptr, a supported d and epochs >= 1");
    const int64_t nnz = job->row_ptr[job->n];
    if (nnz < 0 || nnz > INT32_MAX || (nnz > 0 && !job->col_idx))
        return pack_fail(GEMPE_E_INVALID_ARG, "row_ptr[n] out of range or col_idx null");
    gempe_params pp = s->p;
    if (job->d < 8) {
        pp.precision = 0;
        pp.block_partners = 0;
    }
    const size_t bytes = Pack::bytes_for(job->n, nnz, job->d, pp);
    if (bytes > s->budget)
        return pack_fail(GEMPE_E_BUDGET, "the job needs " + std::to_string(bytes) + " device bytes, the budget is " +
                                             std::to_string(s->budget));
    std::unique_ptr<Job> j(new Job());
    j->rp.assign(job->row_ptr, job->row_ptr + job->n + 1);
    j->ci.assign(job->col_idx ? job->col_idx : job->row_ptr, job->col_idx ? job->col_idx + nnz : job->row_ptr);
    j->n = job->n;
    j->d = job->d;
    j->epochs = job->epochs;
    j->seed = job->seed;
    j->bytes = bytes;
    std::lock_guard<std::mutex> lock(s->mu);
    j->id = s->next_id++;
    j->ticket = s->tickets++;
    j->submit_ns = now_ns(s->t0);
    *job_id = j->id;
    s->pending.push_back(j.get());
    s->jobs[j->id] = std::move(j);
    s->cv_pending.notify_all();
    return GEMPE_OK;
}

namespace {
void fill_info(const Job* j, gempe_job_info* info) {
    info->state = j->state.load();
    info->epochs = j->epochs;
    info->epochs_done = j->epochs_done;
    info->submit_ns = j->submit_ns;
    info->admit_ns = j->admit_ns;
    info->done_ns = j->done_ns;
    info->device_bytes = j->bytes;
    info->pairs = j->pairs;
    info->sigma = j->final_sigma;
}
}  // namespace

GEMPE_API gempe_status gempe_server_poll(gempe_server* s, uint64_t job_id, gempe_job_info* info) {
    if (!s || !info) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return pack_fail(GEMPE_E_INVALID_ARG, "unknown job id");
    fill_info(it->second.get(), info);
    if (info->state < 0) return pack_fail((gempe_status)info->state, it->second->error);
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_server_wait(gempe_server* s, uint64_t job_id, int32_t timeout_ms, gempe_job_info* info) {
    if (!s || !info) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return pack_fail(GEMPE_E_INVALID_ARG, "unknown job id");
    Job* j = it->second.get();
    const bool ok = s->cv_done.wait_for(lock, std::chrono::milliseconds(std::max(timeout_ms, 0)), [&] {
        const int st = j->state.load();
        return st == kDone || st < 0;
    });
    fill_info(j, info);
    if (info->state < 0) return pack_fail((gempe_status)info->state, j->error);
    if (!ok) return pack_fail(GEMPE_E_TIMEOUT, "job not finished within the timeout");
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_server_result(gempe_server* s, uint64_t job_id, float* host_out, size_t count) {
    if (!s) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    std::unique_ptr<Job> j;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return pack_fail(GEMPE_E_INVALID_ARG, "unknown job id");
        const int st = it->second->state.load();
        if (st != kDone && st >= 0) return pack_fail(GEMPE_E_INVALID_ARG, "job not finished");
        if (st == kDone && (!host_out || count != (size_t)it->second->n * it->second->d))
            return pack_fail(GEMPE_E_INVALID_ARG, "count must be n*d");
        j = std::move(it->second);
        s->jobs.erase(it);
        if (st == kDone) std::memcpy(host_out, j->host_x, sizeof(float) * count);
        s->give_pinned_locked(j->host_x, j->host_x_bytes);
        j->host_x = nullptr;
    }
    const int st = j->state.load();
    if (st < 0) return pack_fail((gempe_status)st, j->error);
    return GEMPE_OK;
}

GEMPE_API gempe_status gempe_server_stats(gempe_server* s, int64_t* out6) {
    if (!s || !out6) return pack_fail(GEMPE_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out6[0] = (int64_t)(s->pending.size() + s->waiting);
    out6[1] = (int64_t)s->active.size();
    out6[2] = (int64_t)s->completed;
    out6[3] = (int64_t)s->failed;
    out6[4] = (int64_t)s->in_use;
    out6[5] = (int64_t)s->peak_in_use;
    return GEMPE_OK;
}

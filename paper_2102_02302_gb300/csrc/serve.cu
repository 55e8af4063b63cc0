// Serving runtime (include/cleora.h, cleora_serve_*): a continuous-batching request loop.
//
// Slots.  max_slots worker threads, each owning a context and two streams (high and low
// priority); the contexts share one device memory pool (below).  A worker
// that is free takes the waiting job with the earliest virtual finish time -- its arrival
// plus its estimated service time (a cost model of its host transfers, graph build and
// gathered bytes) -- among those whose estimated peak device bytes fit in the budget beside
// the running jobs' reservations.  Short jobs thus go ahead of long ones, but a job is only
// passed by jobs that arrived less than its own service estimate after it, so every job
// progresses; and a job passed over 8 times for lack of memory blocks further passing.
//
// Short jobs (estimated service at most short_job_seconds) also have short_slots slots of
// their own, with a memory reserve of their own, so they never wait for a long job to leave a
// slot; and every short job runs on a high-priority stream.
//
// A job runs the whole method on a stream of its slot (upload and build, init, iterations,
// FP32 result to host), so jobs on different slots overlap on the GPU.  The slots' contexts
// allocate from one stream-ordered pool that keeps freed blocks: a job reuses the memory of
// jobs before it, and no job returns memory to the driver or maps new memory once the pool
// has grown to the working set.  When a job ends its slot frees what it held (the frees are
// complete before the slot takes another job) and returns the reservation; waiting workers
// are woken and admission runs again.
//
// Waits are bounded where a caller waits: cleora_serve_poll uses a timed condition wait.
// Failures are per job (status in its result); the server keeps running.  The allocation
// failure hook (inject_alloc_failure_every) makes the k-th admitted job's first device
// allocation fail on the host side, which exercises the OOM path without touching the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace cleora {
namespace serve {

enum JobState { WAITING, RUNNING, DONE };

struct Job {
    uint64_t id = 0;
    cleora_job spec;
    int64_t est = 0;       // estimated peak device bytes
    double key = 0.0;      // arrival + estimated service seconds: admission order
    int bypassed = 0;
    bool is_short = false;     // estimated service at most the server's short_job_seconds
    bool on_short_slot = false;
    JobState state = WAITING;
    cleora_result res;
};

constexpr int MAX_BYPASS = 8;

// Estimated service seconds of a job on a GB300 (only the order of jobs depends on it): a
// fixed cost per job, edges up and FP32 rows down over the host link (~50 GB/s), the graph
// build (~3e9 edges/s) and I iterations of gathered rows (~3e12 bytes/s).
double service_estimate(const cleora_job& j) {
    const double E = (double)j.num_edges;
    const double m = j.directed ? E : 2.0 * E;
    const double n = j.nodes_hint > 0 ? (double)j.nodes_hint : std::min(2.0 * E, 2147483647.0);
    const double es = j.storage == CLEORA_F32 ? 4.0 : 2.0;
    return 5e-3 + (E * (16.0 + (j.weights ? 4.0 : 0.0)) + n * j.d * 4.0) / 50e9 + E / 3e9 +
           j.iters * m * j.d * es / 3e12;
}

}  // namespace serve
}  // namespace cleora

struct cleora_server {
    cleora_server_config cfg;
    int64_t budget = 0;      // for running jobs' reservations (general slots)
    int64_t short_budget = 0;   // the short slots' own reserve
    int64_t reserved_short = 0;
    double short_s = 0.02;      // service estimate at or below which a job is short
    std::vector<cudaStream_t> hi, lo;  // per slot: high- and low-priority streams
    cudaMemPool_t pool = nullptr;  // shared by the slots' contexts
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work;  // workers: a job arrived or memory was returned
    std::condition_variable cv_done;  // pollers: a job finished
    std::deque<std::shared_ptr<cleora::serve::Job>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<cleora::serve::Job>> jobs;
    std::deque<uint64_t> finished;  // completion order, for cleora_serve_next
    int64_t reserved = 0;
    int running = 0;
    int64_t completed = 0;
    int64_t admitted = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::vector<cleora_ctx*> slots;
    std::vector<std::thread> workers;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace cleora {
namespace serve {
namespace {

bool valid_job(const cleora_job& j) {
    return j.num_edges >= 0 && (j.num_edges == 0 || (j.src && j.dst)) && j.d >= 8 && j.d <= 1024 &&
           j.d % 8 == 0 && j.iters >= 0 && (j.storage == CLEORA_F32 || j.storage == CLEORA_BF16) &&
           (!j.out || j.out_rows >= 0) && j.nodes_hint >= 0;
}

// Runs one job on a slot context; returns the job's status.
int run_job(cleora_server* s, cleora_ctx* ctx, Job& job) {
    const cleora_job& j = job.spec;
    int rc = cleora_graph_build(ctx, j.src, j.dst, j.weights, j.num_edges, j.directed, 0);
    job.res.t_built = s->now();
    if (rc == CLEORA_OK) {
        cleora_num_nodes(ctx, &job.res.n);
        cleora_num_entries(ctx, &job.res.nnz);
        if (j.out && job.res.n > j.out_rows) rc = CLEORA_ERR_INVALID_ARG;
    }
    if (rc == CLEORA_OK) {
        rc = cleora_init(ctx, j.d, j.seed, j.storage);
        job.res.t_inited = s->now();
    }
    if (rc == CLEORA_OK) rc = cleora_propagate(ctx, j.iters, j.out, 0);
    if (rc == CLEORA_OK) rc = cleora_sync(ctx);
    return rc;
}

void worker_main(cleora_server* s, int slot) {
    cleora_ctx* ctx = s->slots[slot];
    const bool short_slot = slot >= s->cfg.max_slots;
    for (;;) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stop) return;
                std::stable_sort(s->queue.begin(), s->queue.end(),
                                 [](const std::shared_ptr<Job>& x, const std::shared_ptr<Job>& y) {
                                     return x->key < y->key;
                                 });
                if (short_slot) {
                    // the earliest short job that fits the short reserve (the general slots'
                    // memory is not touched, so no job's bypass count moves)
                    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                        if ((*it)->is_short && s->reserved_short + (*it)->est <= s->short_budget) {
                            job = *it;
                            s->queue.erase(it);
                            break;
                        }
                    }
                    if (job) break;
                } else {
                    // earliest virtual finish that fits; a job passed over too often for lack
                    // of memory stops the scan (its turn comes when memory is returned)
                    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                        if (s->reserved + (*it)->est <= s->budget) {
                            job = *it;
                            s->queue.erase(it);
                            break;
                        }
                        if ((*it)->bypassed >= MAX_BYPASS) break;
                    }
                    if (job) {
                        for (auto& q : s->queue)  // every job ahead of it did not fit
                            if (q->key < job->key) q->bypassed++;
                        break;
                    }
                }
                s->cv_work.wait(lk);
            }
            job->on_short_slot = short_slot;
            (short_slot ? s->reserved_short : s->reserved) += job->est;
            s->running += 1;
            s->admitted += 1;
            job->state = RUNNING;
            job->res.slot = slot;
            job->res.t_admit = s->now();
            job->res.bytes_reserved = job->est;
            const int k = s->cfg.inject_alloc_failure_every;
            ctx->inject_alloc_fail = (k > 0 && s->admitted % k == 0) ? 0 : -1;
        }
        // the slot's previous job ended with a synchronize of its stream, so the context can
        // move to the other stream
        ctx->stream = job->is_short ? s->hi[slot] : s->lo[slot];
        int st = run_job(s, ctx, *job);
        ctx->inject_alloc_fail = -1;
        {
            DeviceGuard guard(ctx->device);
            ctx_release_all(ctx);
            cudaStreamSynchronize(ctx->stream);
            cudaGetLastError();
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            job->res.status = st;
            job->res.t_done = s->now();
            job->state = DONE;
            s->finished.push_back(job->id);
            (job->on_short_slot ? s->reserved_short : s->reserved) -= job->est;
            s->running -= 1;
            s->completed += 1;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace
}  // namespace serve
}  // namespace cleora

using namespace cleora;
using namespace cleora::serve;

extern "C" {

int64_t cleora_serve_estimate(const cleora_job* j) {
    if (!j) return -1;
    const int64_t E = j->num_edges;
    const int64_t m = j->directed ? E : 2 * E;      // CSR entries before dedup (upper bound)
    const int64_t n = j->nodes_hint > 0 ? j->nodes_hint : std::min<int64_t>(2 * E, ((int64_t)1 << 31) - 1);
    const int64_t es = j->storage == CLEORA_F32 ? 4 : 2;
    const int64_t w = j->weights ? 1 : 0;
    const int64_t MiB = (int64_t)1 << 20;
    // graph build: uploads, the id set / two 2E-key sort buffers, the id -> rank table, run
    // starts, sorted weights, CSR arrays
    const int64_t build = E * (16 + 4 * w) + 2 * (2 * E * 8) + (j->directed ? 0 : 8 * m) +
                          w * 2 * 4 * m + m * (4 + 8 + 4) + n * 96 + 8 * m + 64 * MiB;
    // resident: CSR (+values), ids, rowptr, degrees; then plan build, then embeddings
    const int64_t resident = m * 8 + n * (8 + 8 + 4 + 8);
    const int64_t plan = resident + n * 53 + (m / 64 + 1) * 16;
    const int64_t prop = resident + (m / 64 + 1) * 16 + 2 * n * j->d * es +
                         (2 * m / 8192 + 1) * j->d * 4 + (es == 2 ? 256 * MiB : 0) + 64 * MiB;
    // init with T larger than twice the hot-row budget partitions the rows hot-first: a new
    // column (and value) array, flag words and their counts, bins, row prefixes, hot counts
    const int64_t part = n * j->d * es > 2 * DEFAULT_HOT_BYTES
                             ? prop + m * (4 + 4 * w) + m / 8 + m / 4 + n * (5 + 8 + 4) + 64 * MiB
                             : 0;
    const int64_t peak = std::max(std::max(build, part), std::max(plan, prop));
    return peak + peak / 10;  // pool rounding and fragmentation
}

int cleora_serve_create(cleora_server** out, const cleora_server_config* cfg) {
    if (!out || !cfg || cfg->max_slots < 0 || cfg->queue_capacity < 0 || cfg->hbm_budget_bytes < 0 ||
        cfg->short_slots < 0 || cfg->short_slots > 64 || !(cfg->short_job_seconds >= 0.0))
        return CLEORA_ERR_INVALID_ARG;
    *out = nullptr;
    cleora_server* s = new (std::nothrow) cleora_server();
    if (!s) return CLEORA_ERR_OOM;
    s->cfg = *cfg;
    if (s->cfg.max_slots == 0) s->cfg.max_slots = 4;
    if (s->cfg.short_job_seconds > 0.0) s->short_s = s->cfg.short_job_seconds;
    const int all_slots = s->cfg.max_slots + s->cfg.short_slots;
    s->t0 = std::chrono::steady_clock::now();
    {
        DeviceGuard guard(cfg->device);
        if (!guard.ok) {
            delete s;
            return CLEORA_ERR_INVALID_ARG;
        }
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return CLEORA_ERR_CUDA;
        }
        const int64_t total = cfg->hbm_budget_bytes > 0 ? cfg->hbm_budget_bytes : (int64_t)(free_b / 10 * 8);
        // the short slots' reserve (2 GiB each, at most an eighth of the total) is set aside
        s->short_budget = std::min<int64_t>(total / 8, (int64_t)s->cfg.short_slots << 31);
        s->budget = total - s->short_budget;
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = cfg->device;
        if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return CLEORA_ERR_CUDA;
        }
        uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool for the next jobs
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    int lo_prio = 0, hi_prio = 0;  // numerically lower is higher priority
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    int rc = CLEORA_OK;
    for (int k = 0; k < all_slots && rc == CLEORA_OK; ++k) {
        DeviceGuard guard(cfg->device);
        cudaStream_t h = nullptr, l = nullptr;
        if (cudaStreamCreateWithPriority(&h, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
            cudaStreamCreateWithPriority(&l, cudaStreamNonBlocking, lo_prio) != cudaSuccess) {
            cudaGetLastError();
            if (h) cudaStreamDestroy(h);
            rc = CLEORA_ERR_CUDA;
            break;
        }
        s->hi.push_back(h);
        s->lo.push_back(l);
        cleora_ctx* c = nullptr;
        rc = ctx_create(&c, cfg->device, l, s->pool);
        if (rc == CLEORA_OK) s->slots.push_back(c);
    }
    if (rc != CLEORA_OK) {
        for (cleora_ctx* x : s->slots) cleora_destroy(x);
        for (cudaStream_t x : s->hi) cudaStreamDestroy(x);
        for (cudaStream_t x : s->lo) cudaStreamDestroy(x);
        cudaMemPoolDestroy(s->pool);
        delete s;
        return rc;
    }
    for (int k = 0; k < all_slots; ++k) s->workers.emplace_back(worker_main, s, k);
    *out = s;
    return CLEORA_OK;
}

int cleora_serve_submit(cleora_server* s, const cleora_job* job, uint64_t* job_id) {
    if (!s || !job || !job_id || !valid_job(*job)) return CLEORA_ERR_INVALID_ARG;
    auto j = std::make_shared<Job>();
    j->spec = *job;
    j->est = cleora_serve_estimate(job);
    const double svc = service_estimate(*job);
    j->res = cleora_result();
    j->res.slot = -1;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return CLEORA_ERR_STATE;
        j->is_short = svc <= s->short_s;
        if (j->est > s->budget && !(j->is_short && j->est <= s->short_budget)) return CLEORA_ERR_REJECTED;
        if (s->cfg.queue_capacity > 0 && (int)s->queue.size() >= s->cfg.queue_capacity)
            return CLEORA_ERR_REJECTED;
        j->id = s->next_id++;
        j->res.t_submit = s->now();
        j->key = j->res.t_submit + svc;
        s->queue.push_back(j);
        s->jobs[j->id] = j;
        *job_id = j->id;
    }
    s->cv_work.notify_one();
    return CLEORA_OK;
}

int cleora_serve_poll(cleora_server* s, uint64_t job_id, int timeout_ms, cleora_result* result) {
    if (!s || !result) return CLEORA_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return CLEORA_ERR_INVALID_ARG;
    std::shared_ptr<Job> j = it->second;
    auto done = [&] { return j->state == DONE; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        return CLEORA_ERR_TIMEOUT;
    }
    *result = j->res;
    s->jobs.erase(job_id);
    return CLEORA_OK;
}

int cleora_serve_cancel(cleora_server* s, uint64_t job_id) {
    if (!s) return CLEORA_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return CLEORA_ERR_INVALID_ARG;
        std::shared_ptr<Job> j = it->second;
        if (j->state != WAITING) return CLEORA_ERR_STATE;
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), j), s->queue.end());
        j->state = DONE;
        j->res.status = CLEORA_ERR_CANCELLED;
        j->res.t_done = s->now();
        s->finished.push_back(j->id);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    return CLEORA_OK;
}

int cleora_serve_next(cleora_server* s, int timeout_ms, uint64_t* job_id, cleora_result* result) {
    if (!s || !job_id || !result) return CLEORA_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        while (!s->finished.empty() && !s->jobs.count(s->finished.front())) s->finished.pop_front();
        return !s->finished.empty();
    };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        return CLEORA_ERR_TIMEOUT;
    }
    const uint64_t id = s->finished.front();
    s->finished.pop_front();
    *job_id = id;
    *result = s->jobs[id]->res;
    s->jobs.erase(id);
    return CLEORA_OK;
}

double cleora_serve_now(const cleora_server* s) { return s ? s->now() : 0.0; }

int cleora_serve_stats(const cleora_server* s, int* queued, int* running, int64_t* bytes_reserved,
                       int64_t* completed, int64_t* budget) {
    if (!s) return CLEORA_ERR_INVALID_ARG;
    cleora_server* m = const_cast<cleora_server*>(s);
    std::lock_guard<std::mutex> lk(m->mu);
    if (queued) *queued = (int)s->queue.size();
    if (running) *running = s->running;
    if (bytes_reserved) *bytes_reserved = s->reserved + s->reserved_short;
    if (completed) *completed = s->completed;
    if (budget) *budget = s->budget + s->short_budget;
    return CLEORA_OK;
}

void cleora_serve_destroy(cleora_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto& j : s->queue) {
            j->state = DONE;
            j->res.status = CLEORA_ERR_CANCELLED;
            j->res.t_done = s->now();
            s->finished.push_back(j->id);
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (std::thread& t : s->workers) t.join();  // running jobs finish first
    for (size_t k = 0; k < s->slots.size(); ++k) {
        s->slots[k]->stream = s->lo[k];  // the slot's own stream; the context owns neither
        cleora_destroy(s->slots[k]);
    }
    for (cudaStream_t x : s->hi) cudaStreamDestroy(x);
    for (cudaStream_t x : s->lo) cudaStreamDestroy(x);
    if (s->pool) {
        DeviceGuard guard(s->cfg.device);
        cudaMemPoolDestroy(s->pool);
    }
    delete s;
}

}  // extern "C"

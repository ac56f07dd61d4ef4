// serve.cu — a job server with continuous batching under an HBM budget.
//
// Each job is one clustering (Section I's three steps, as dbscan_run).  The
// server owns `slots` execution slots; a slot is one CUDA stream, one plan
// without a workspace of its own and one completion event.  Device memory
// comes from a stream-ordered memory pool of the server: a job's workspace is
// exactly what its (n, d) needs, allocated on the slot's stream when the job
// is admitted and freed on that stream behind the job's kernels, so the bytes
// the jobs on the device hold are what the budget limits.  A worker thread:
//   - completes jobs whose event has fired (decodes the status word copied out
//     before the workspace was freed, stamps the submit-to-done latency, wakes
//     waiters, returns the job's bytes to the budget and frees the slot);
//   - admits queued jobs in arrival order while a slot is free and the summed
//     workspace of the jobs on the device stays within the budget (a job is
//     always admitted when nothing else runs, so one larger than the budget
//     still runs, alone);
//   - enqueues an admitted job (workspace allocation, kernels, status copy,
//     workspace free) on its slot's stream and records the slot's event.
// Jobs on different slots run concurrently on the device, and new jobs start
// as soon as earlier ones finish, while the rest keep running.  Submit, poll,
// wait and info are thread-safe.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t id = 0;
    dbscan_instance inst{};
    int64_t bytes = 0;  // the job's workspace, exactly as its (n, d) needs
    int status = DBSCAN_OK;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

struct Slot {
    dbscan_plan *plan = nullptr;  // bound to each job's workspace in turn
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    Job *job = nullptr;
};

}  // namespace

struct dbscan_server {
    dbscan_serve_opts opts{};
    dbscan_opts plan_opts{};
    std::vector<Slot> slots;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_idle;
    int waiters = 0;  // threads inside dbscan_serve_wait (destroy frees nothing while any is)
    std::deque<Job *> queue;
    std::unordered_map<uint64_t, Job *> jobs;
    uint64_t next_id = 1;
    int64_t in_flight_bytes = 0;
    int running = 0;
    // statistics (dbscan_serve_info)
    int64_t jobs_done = 0, peak_bytes = 0;
    int max_running = 0;
    bool stop = false;
    std::thread worker;
};

namespace {

// Enqueues job j on slot sl (called without the server lock).  Returns the
// job's status if it could not be enqueued; the slot's event is recorded
// either way, so the job completes through the normal path.
int launch_job(dbscan_server *s, Slot &sl, const Job &j) {
    const dbscan_instance &in = j.inst;
    int st = DBSCAN_OK;
    void *ws = nullptr;
    if (in.n > 0) {
        if (cudaMallocFromPoolAsync(&ws, (size_t)j.bytes, s->pool, sl.stream) != cudaSuccess) {
            cudaGetLastError();
            ws = nullptr;
            st = DBSCAN_ERR_OOM;
        }
        if (!st) st = plan_bind_workspace(sl.plan, ws, (size_t)j.bytes, in.n, in.d, true);
        if (!st) st = dbscan_run(sl.plan, in.points, in.n, in.d, in.eps, in.min_pts, in.labels_out, nullptr);
        // the run's device error bits, read out before the workspace goes back to the pool
        *sl.plan->h_status = 0;
        if (!st && cudaMemcpyAsync(sl.plan->h_status, sl.plan->w.status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                   sl.stream) != cudaSuccess)
            st = DBSCAN_ERR_CUDA;
        if (ws && cudaFreeAsync(ws, sl.stream) != cudaSuccess) st = st ? st : DBSCAN_ERR_CUDA;
    }
    if (cudaEventRecord(sl.done_ev, sl.stream) != cudaSuccess) st = st ? st : DBSCAN_ERR_CUDA;
    return st;
}

void serve_loop(dbscan_server *s) {
    cudaSetDevice(s->opts.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool busy = false;
        // completions
        for (Slot &sl : s->slots) {
            if (!sl.job) continue;
            const cudaError_t q = cudaEventQuery(sl.done_ev);
            if (q == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            Job *j = sl.job;
            int st = (q == cudaSuccess) ? plan_status_from_bits(*sl.plan->h_status) : DBSCAN_ERR_CUDA;
            if (q != cudaSuccess) cudaGetLastError();
            if (j->status == DBSCAN_OK) j->status = st;
            j->done = true;
            j->t_done = Clock::now();
            s->in_flight_bytes -= j->bytes;
            --s->running;
            ++s->jobs_done;
            sl.job = nullptr;
            s->cv_done.notify_all();
        }
        // admissions, in arrival order
        while (!s->queue.empty()) {
            Job *j = s->queue.front();
            Slot *free_slot = nullptr;
            for (Slot &sl : s->slots)
                if (!sl.job) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            if (s->running > 0 && s->in_flight_bytes + j->bytes > s->opts.hbm_budget_bytes) break;
            s->queue.pop_front();
            free_slot->job = j;
            s->in_flight_bytes += j->bytes;
            ++s->running;
            s->peak_bytes = std::max(s->peak_bytes, s->in_flight_bytes);
            s->max_running = std::max(s->max_running, s->running);
            busy = true;
            lk.unlock();  // launches happen outside the lock
            const int st = launch_job(s, *free_slot, *j);
            lk.lock();
            j->status = st;
        }
        if (s->stop && s->queue.empty() && !busy) break;
        if (!busy && s->queue.empty()) {
            s->cv_work.wait(lk, [s] { return s->stop || !s->queue.empty(); });
        } else {
            // jobs are running: poll their events again shortly
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

void release_server(dbscan_server *s) {
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.plan) dbscan_plan_destroy(sl.plan);
        if (sl.done_ev) cudaEventDestroy(sl.done_ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
}

}  // namespace

extern "C" {

void dbscan_serve_opts_default(dbscan_serve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->device = 0;
    o->slots = 8;
    o->hbm_budget_bytes = (int64_t)120 << 30;
    o->label_mode = DBSCAN_LABEL_ROOT_INDEX;
    o->precision = DBSCAN_PREC_AUTO;
    o->max_n = 500000;
    o->max_d = 64;
    o->max_queue = 1000000;
}

int dbscan_serve_create(dbscan_server **out, const dbscan_serve_opts *opts) {
    if (!out) return DBSCAN_ERR_ARG;
    *out = nullptr;
    dbscan_serve_opts o;
    if (opts) o = *opts;
    else dbscan_serve_opts_default(&o);
    if (o.slots < 1 || o.slots > 256 || o.hbm_budget_bytes <= 0 || o.max_n < 1 || o.max_n > INT32_MAX / 2 ||
        o.max_d < 1 || o.max_d > 64 || o.max_queue < 1 || o.precision < 0 || o.precision > 3 || o.label_mode < 0 ||
        o.label_mode > 1)
        return DBSCAN_ERR_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(o.device) != cudaSuccess) return DBSCAN_ERR_CUDA;
    dbscan_server *s = new (std::nothrow) dbscan_server();
    if (!s) return DBSCAN_ERR_OOM;
    s->opts = o;
    dbscan_opts &po = s->plan_opts;
    dbscan_opts_default(&po);
    po.device = o.device;
    po.synchronous = 0;
    po.max_n = o.max_n;
    po.max_d = o.max_d;
    po.precision = o.precision;
    po.label_mode = o.label_mode;
    int rc = DBSCAN_OK;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = o.device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        s->pool = nullptr;
        rc = DBSCAN_ERR_CUDA;
    } else {
        // keep freed blocks for the next jobs instead of returning them at every sync
        uint64_t keep = (uint64_t)o.hbm_budget_bytes;
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s->slots.resize(o.slots);
    for (Slot &sl : s->slots) {
        if (rc) break;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming) != cudaSuccess) {
            rc = DBSCAN_ERR_CUDA;
            break;
        }
        dbscan_opts so = po;
        so.stream = sl.stream;
        rc = plan_create_unbound(&sl.plan, so);
    }
    if (rc == DBSCAN_OK) {
        s->worker = std::thread(serve_loop, s);
    } else {
        release_server(s);
        s = nullptr;
    }
    if (prev >= 0) cudaSetDevice(prev);
    *out = s;
    return rc;
}

int dbscan_serve_submit(dbscan_server *s, const dbscan_instance *inst, uint64_t *job_id) {
    if (!s || !inst || !job_id) return DBSCAN_ERR_ARG;
    const dbscan_instance &in = *inst;
    if (in.n < 0 || in.n > s->opts.max_n || in.d < 1 || in.d > s->opts.max_d || !(in.eps > 0.0f) ||
        in.eps > 3.0e38f || in.min_pts < 1 || (in.n > 0 && (!in.points || !in.labels_out)))
        return DBSCAN_ERR_ARG;
    Job *j = new (std::nothrow) Job();
    if (!j) return DBSCAN_ERR_OOM;
    j->inst = in;
    j->bytes = in.n > 0 ? (int64_t)plan_workspace_bytes_for(s->plan_opts, in.n, in.d, true) : 0;
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop || (int64_t)s->queue.size() >= s->opts.max_queue) {
            delete j;
            return DBSCAN_ERR_BUSY;
        }
        j->id = s->next_id++;
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        *job_id = j->id;
    }
    s->cv_work.notify_one();
    return DBSCAN_OK;
}

int dbscan_serve_poll(dbscan_server *s, uint64_t job_id, int32_t *done) {
    if (!s || !done) return DBSCAN_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return DBSCAN_ERR_NOT_FOUND;
    *done = it->second->done ? 1 : 0;
    return it->second->done ? it->second->status : DBSCAN_OK;
}

int dbscan_serve_wait(dbscan_server *s, uint64_t job_id, int64_t timeout_us, double *latency_us) {
    if (!s) return DBSCAN_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return DBSCAN_ERR_NOT_FOUND;
    Job *j = it->second;
    auto ready = [j] { return j->done; };
    ++s->waiters;
    bool ok = true;
    if (timeout_us < 0) s->cv_done.wait(lk, ready);
    else ok = s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    if (--s->waiters == 0 && s->stop) s->cv_idle.notify_all();
    if (!ok) return DBSCAN_ERR_TIMEOUT;
    if (latency_us)
        *latency_us = std::chrono::duration<double, std::micro>(j->t_done - j->t_submit).count();
    const int st = j->status;
    s->jobs.erase(job_id);
    delete j;
    return st;
}

int dbscan_serve_info(dbscan_server *s, dbscan_serve_stats *out) {
    if (!s || !out) return DBSCAN_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    {
        std::lock_guard<std::mutex> lk(s->mu);
        out->jobs_done = s->jobs_done;
        out->jobs_queued = (int64_t)s->queue.size();
        out->jobs_running = s->running;
        out->max_jobs_running = s->max_running;
        out->hbm_budget_bytes = s->opts.hbm_budget_bytes;
        out->bytes_in_flight = s->in_flight_bytes;
        out->peak_bytes_in_flight = s->peak_bytes;
    }
    uint64_t v = 0;
    if (cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReservedMemCurrent, &v) == cudaSuccess)
        out->pool_reserved_bytes = (int64_t)v;
    if (cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReservedMemHigh, &v) == cudaSuccess)
        out->pool_peak_reserved_bytes = (int64_t)v;
    cudaGetLastError();
    return DBSCAN_OK;
}

int64_t dbscan_serve_job_bytes(const dbscan_server *s, int64_t n, int32_t d) {
    if (!s || n < 0 || n > s->opts.max_n || d < 1 || d > s->opts.max_d) return -1;
    return n > 0 ? (int64_t)plan_workspace_bytes_for(s->plan_opts, n, d, true) : 0;
}

int dbscan_serve_destroy(dbscan_server *s) {
    if (!s) return DBSCAN_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Job *j : s->queue) {  // queued jobs are dropped
            j->status = DBSCAN_ERR_BUSY;
            j->done = true;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();  // every admitted job is done now
    {
        // Wake the threads blocked in dbscan_serve_wait (all their jobs are done)
        // and free nothing until the last has left.
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.notify_all();
        s->cv_idle.wait(lk, [s] { return s->waiters == 0; });
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->opts.device);
    release_server(s);
    if (prev >= 0) cudaSetDevice(prev);
    return DBSCAN_OK;
}

}  // extern "C"

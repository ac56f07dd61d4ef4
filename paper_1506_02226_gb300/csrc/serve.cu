// serve.cu — a job server with continuous batching under an HBM budget.
//
// Each job is one clustering (Section I's three steps, as dbscan_run).  The
// server owns `slots` execution slots; a slot is one CUDA stream, one
// asynchronous plan sized for the largest accepted job and one completion
// event.  A worker thread:
//   - completes jobs whose event has fired (reads the plan's device status,
//     stamps the submit-to-done latency, wakes waiters, frees the slot);
//   - admits queued jobs in arrival order while a slot is free and the summed
//     footprint of the jobs on the device stays within the HBM budget (a job
//     is always admitted when nothing else runs);
//   - enqueues an admitted job's kernels on its slot's stream and records the
//     slot's event.
// Jobs on different slots run concurrently on the device, and new jobs start
// as soon as earlier ones finish, while the rest keep running.  Submit, poll
// and wait are thread-safe.
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
    int64_t bytes = 0;
    int status = DBSCAN_OK;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

struct Slot {
    dbscan_plan *plan = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    Job *job = nullptr;
};

}  // namespace

struct dbscan_server {
    dbscan_serve_opts opts{};
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_idle;
    int waiters = 0;  // threads inside dbscan_serve_wait (destroy frees nothing while any is)
    std::deque<Job *> queue;
    std::unordered_map<uint64_t, Job *> jobs;
    uint64_t next_id = 1;
    int64_t in_flight_bytes = 0;
    int64_t bytes_per_point = 0;  // workspace footprint per point of a job
    bool stop = false;
    std::thread worker;
};

namespace {

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
            int st = (q == cudaSuccess) ? dbscan_plan_sync(sl.plan) : DBSCAN_ERR_CUDA;
            if (q != cudaSuccess) cudaGetLastError();
            if (j->status == DBSCAN_OK) j->status = st;
            j->done = true;
            j->t_done = Clock::now();
            s->in_flight_bytes -= j->bytes;
            sl.job = nullptr;
            s->cv_done.notify_all();
        }
        // admissions, in arrival order
        while (!s->queue.empty()) {
            Job *j = s->queue.front();
            Slot *free_slot = nullptr;
            bool any_running = false;
            for (Slot &sl : s->slots) {
                if (sl.job) any_running = true;
                else if (!free_slot) free_slot = &sl;
            }
            if (!free_slot) break;
            if (any_running && s->in_flight_bytes + j->bytes > s->opts.hbm_budget_bytes) break;
            s->queue.pop_front();
            free_slot->job = j;
            s->in_flight_bytes += j->bytes;
            busy = true;
            const dbscan_instance in = j->inst;
            lk.unlock();  // launches happen outside the lock
            int st = dbscan_run(free_slot->plan, in.points, in.n, in.d, in.eps, in.min_pts, in.labels_out, nullptr);
            cudaEventRecord(free_slot->done_ev, free_slot->stream);
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
    if (o.slots < 1 || o.slots > 256 || o.hbm_budget_bytes <= 0 || o.max_n < 1 || o.max_d < 1 || o.max_d > 64 ||
        o.max_queue < 1)
        return DBSCAN_ERR_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(o.device) != cudaSuccess) return DBSCAN_ERR_CUDA;
    dbscan_server *s = new (std::nothrow) dbscan_server();
    if (!s) return DBSCAN_ERR_OOM;
    s->opts = o;
    s->slots.resize(o.slots);
    int rc = DBSCAN_OK;
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming) != cudaSuccess) {
            rc = DBSCAN_ERR_CUDA;
            break;
        }
        dbscan_opts po;
        dbscan_opts_default(&po);
        po.device = o.device;
        po.synchronous = 0;
        po.stream = sl.stream;
        po.max_n = o.max_n;
        po.max_d = o.max_d;
        po.precision = o.precision;
        po.label_mode = o.label_mode;
        if ((rc = dbscan_plan_create(&sl.plan, &po)) != DBSCAN_OK) break;
    }
    if (rc == DBSCAN_OK) {
        const int64_t ws = dbscan_plan_workspace_bytes(s->slots[0].plan);
        s->bytes_per_point = ws / o.max_n + 1;
        s->worker = std::thread(serve_loop, s);
    } else {
        for (Slot &sl : s->slots) {
            if (sl.plan) dbscan_plan_destroy(sl.plan);
            if (sl.done_ev) cudaEventDestroy(sl.done_ev);
            if (sl.stream) cudaStreamDestroy(sl.stream);
        }
        delete s;
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
    j->bytes = s->bytes_per_point * in.n + (int64_t)in.n * (4 * in.d + 4);
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
    for (Slot &sl : s->slots) {
        if (sl.plan) dbscan_plan_destroy(sl.plan);
        if (sl.done_ev) cudaEventDestroy(sl.done_ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
    return DBSCAN_OK;
}

}  // extern "C"

// server.cu -- interactive layout serving with continuous batching (host runtime).
//
// Jobs (a graph plus a queue of requests) are admitted by device-memory footprint
// into at most `max_active` slots; each admitted job owns a tfdp_graph on its own CUDA
// stream. A worker thread keeps one chunk of up to `chunk_iters` iterations queued for
// every admitted job with work: it polls the jobs' completion events and gives each job
// its next chunk as soon as that job's previous chunk is done, so the jobs' kernels
// overlap on the GPU and a small job never waits for a large one. Jobs that arrive
// while others run are admitted as soon as a slot and memory are free (iteration-level
// scheduling, not a FIFO of whole jobs). A request is either the initial layout of a job or an update: new t-force
// parameters (Sec. 3.3) applied to the current layout with the step schedule restarted
// over the update's iterations (warm start; the global refinement of Sec. 5). The
// kernel spectrum is rebuilt only when gamma, k or the grid change. The computation of
// a job does not depend on what else is running: its result in the mix equals its
// result alone.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/tfdp.h"

namespace {

struct Request {
    int64_t id = 0;
    int32_t kind = 0;  // 0 layout, 1 update
    int32_t iters = 0;
    int32_t remaining = 0;
    bool started = false;
    tfdp_params params{};
    double t_submit = 0, t_start = 0;
};

struct Job {
    int64_t id = 0;
    int64_t n = 0, m = 0;
    std::vector<int32_t> edges;
    std::vector<float> xy0;
    tfdp_params params{};
    size_t footprint = 0;
    tfdp_graph* g = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    std::deque<Request> queue;
    bool admitted = false;
    bool release = false;
    int32_t issued = 0;  // iterations of the chunk in flight
    bool in_flight = false;  // a chunk of this job is queued on the GPU
    int32_t error = 0;
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct tfdp_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_load;
    std::thread worker, loader;
    bool stop = false;
    int device = 0;
    size_t budget = 0, used = 0;
    int32_t max_active = 1, chunk = 10;
    int64_t next_job = 1, next_req = 1;
    std::map<int64_t, std::unique_ptr<Job>> jobs;
    std::deque<int64_t> waiting;  // submitted, not yet admitted (FIFO)
    std::vector<tfdp_done> done;
    double t0 = 0;
    int64_t node_iterations = 0;
    int32_t active = 0;
    int32_t peak_active = 0;
    std::atomic<bool> kick{false};  // new work for an idle job: stop polling the GPU early

    void run();
    void load();
    void fail_job_locked(Job* j, tfdp_status st);
};

void tfdp_server::fail_job_locked(Job* j, tfdp_status st) {
    j->error = st;
    for (const Request& r : j->queue) {
        tfdp_done d{};
        d.request_id = r.id;
        d.job_id = j->id;
        d.kind = r.kind;
        d.iters = r.iters;
        d.t_submit = r.t_submit - t0;
        d.t_start = d.t_done = now_s() - t0;
        d.status = st;
        done.push_back(d);
    }
    j->queue.clear();
    cv_done.notify_all();
}

// Admission: the front job of the FIFO gets a slot once one is free and its footprint
// fits the budget (or nothing else is resident); its graph is then built outside the
// lock, so scheduling of the admitted jobs goes on meanwhile.
void tfdp_server::load() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        if (waiting.empty() || active >= max_active) {
            cv_load.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        Job* j = jobs[waiting.front()].get();
        if (used + j->footprint > budget && active > 0) {
            cv_load.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        waiting.pop_front();
        used += j->footprint;  // reserved
        ++active;
        if (active > peak_active) peak_active = active;
        lk.unlock();
        tfdp_graph* g = nullptr;
        cudaStream_t stream = nullptr;
        cudaEvent_t ev = nullptr;
        tfdp_status st = TFDP_OK;
        // the job's own non-blocking stream, for its upload and all its iterations
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) st = TFDP_ERR_CUDA;
        if (st == TFDP_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) st = TFDP_ERR_CUDA;
        if (st == TFDP_OK)
            st = tfdp_create_graph(j->n, j->m, j->m ? j->edges.data() : nullptr, j->xy0.data(), 0, &j->params,
                                   stream, &g);
        lk.lock();
        if (st != TFDP_OK) {
            if (g) tfdp_destroy_graph(g);
            if (ev) cudaEventDestroy(ev);
            if (stream) cudaStreamDestroy(stream);
            used -= j->footprint;
            --active;
            fail_job_locked(j, st);
            continue;
        }
        j->g = g;
        j->stream = stream;
        j->ev = ev;
        j->xy0.clear();
        j->xy0.shrink_to_fit();
        j->edges.clear();
        j->edges.shrink_to_fit();
        j->admitted = true;
        kick.store(true);
        cv_work.notify_all();
    }
}

void tfdp_server::run() {
    cudaSetDevice(device);
    // jobs with a chunk queued on the GPU, and the request each chunk belongs to (the
    // pointer is taken under the lock; other threads only append to a job's queue, which
    // leaves its elements in place)
    std::vector<std::pair<Job*, Request*>> inflight;
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        // jobs ready for their next chunk: admitted, a request queued, nothing in flight
        std::vector<std::pair<Job*, Request*>> ready;
        kick.store(false);
        for (auto& kv : jobs) {
            Job* j = kv.second.get();
            if (j->admitted && !j->in_flight && !j->queue.empty()) ready.emplace_back(j, &j->queue.front());
        }
        // free the slots of released, drained jobs
        for (auto it = jobs.begin(); it != jobs.end();) {
            Job* j = it->second.get();
            if (j->release && j->queue.empty() && !j->in_flight && (j->admitted || j->error)) {
                if (j->g) tfdp_destroy_graph(j->g);
                if (j->ev) cudaEventDestroy(j->ev);
                if (j->stream) cudaStreamDestroy(j->stream);
                if (j->admitted) {
                    used -= j->footprint;
                    --active;
                    cv_load.notify_all();
                }
                it = jobs.erase(it);
            } else {
                ++it;
            }
        }
        if (ready.empty() && inflight.empty()) {
            cv_work.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        for (auto& jr : ready) jr.first->in_flight = true;
        // queue the chunks without holding the lock: clients may submit and poll meanwhile,
        // and a parameter change synchronises only the job's own stream
        lk.unlock();
        for (auto& jr : ready) {
            Job* j = jr.first;
            Request& r = *jr.second;
            if (!r.started) {
                r.started = true;
                r.t_start = now_s();
                tfdp_status st = TFDP_OK;
                if (r.kind == 1) {
                    st = tfdp_set_params(j->g, &r.params);  // spectrum rebuilt only if needed
                    if (st == TFDP_OK) st = tfdp_set_iteration(j->g, 0);  // restart the cooling
                }
                if (st != TFDP_OK) {
                    j->error = st;
                    r.remaining = 0;
                }
            }
            j->issued = r.remaining < chunk ? r.remaining : chunk;
            if (j->issued > 0) {
                const tfdp_status st = tfdp_iterate(j->g, j->issued);
                if (st != TFDP_OK) {
                    j->error = st;
                    j->issued = 0;
                    r.remaining = 0;
                }
            }
            cudaEventRecord(j->ev, j->stream);
            inflight.push_back(jr);
        }
        // take whatever has finished, without waiting for the slowest job: each job gets
        // its next chunk as soon as its own previous one is done
        std::vector<std::pair<Job*, Request*>> finished;
        for (;;) {
            for (auto it = inflight.begin(); it != inflight.end();) {
                if (cudaEventQuery(it->first->ev) == cudaErrorNotReady) {
                    ++it;
                    continue;
                }
                finished.push_back(*it);
                it = inflight.erase(it);
            }
            if (!finished.empty() || inflight.empty() || kick.load()) break;
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        // a request that ends with this chunk reports the job's device-side checks
        for (auto& jr : finished) {
            Job* j = jr.first;
            if (jr.second->remaining - j->issued <= 0 && j->error == TFDP_OK) {
                const tfdp_status st = tfdp_synchronize(j->g);
                if (st != TFDP_OK) j->error = st;
            }
        }
        lk.lock();
        const double t = now_s();
        for (auto& jr : finished) {
            Job* j = jr.first;
            Request& r = *jr.second;
            j->in_flight = false;
            r.remaining -= j->issued;
            node_iterations += (int64_t)j->issued * j->n;
            if (r.remaining <= 0) {
                tfdp_done d{};
                d.request_id = r.id;
                d.job_id = j->id;
                d.kind = r.kind;
                d.iters = r.iters;
                d.t_submit = r.t_submit - t0;
                d.t_start = r.t_start - t0;
                d.t_done = t - t0;
                d.status = j->error;
                done.push_back(d);
                j->queue.pop_front();
                cv_done.notify_all();
            }
        }
    }
    // stopping: let queued chunks finish before the jobs are destroyed
    lk.unlock();
    for (auto& jr : inflight) cudaEventSynchronize(jr.first->ev);
}

extern "C" {

tfdp_status tfdp_server_create(size_t hbm_budget_bytes, int32_t max_active, int32_t chunk_iters, tfdp_server** out) {
    if (!out || hbm_budget_bytes == 0 || max_active < 1 || chunk_iters < 1) return TFDP_ERR_INVALID_ARG;
    tfdp_server* s = new (std::nothrow) tfdp_server();
    if (!s) return TFDP_ERR_OUT_OF_MEMORY;
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    s->chunk = chunk_iters;
    s->t0 = now_s();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return TFDP_ERR_CUDA;
    }
    s->worker = std::thread([s]() { s->run(); });
    s->loader = std::thread([s]() { s->load(); });
    *out = s;
    return TFDP_OK;
}

tfdp_status tfdp_server_submit(tfdp_server* s, int64_t n, int64_t m, const int32_t* edges, const float* xy0,
                               const tfdp_params* p, int32_t iters, int64_t* job_id, int64_t* request_id) {
    if (!s || n < 1 || m < 0 || (m > 0 && !edges) || !xy0 || iters < 0) return TFDP_ERR_INVALID_ARG;
    tfdp_params prm;
    if (p) prm = *p;
    else tfdp_params_default(&prm);
    tfdp_status st = tfdp_params_check(&prm, nullptr);
    if (st != TFDP_OK) return st;
    size_t fp = 0;
    st = tfdp_graph_footprint(n, m, &prm, &fp);
    if (st != TFDP_OK) return st;
    if (fp > s->budget) return TFDP_ERR_OUT_OF_MEMORY;  // could never be admitted
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return TFDP_ERR_OUT_OF_MEMORY;
    j->n = n;
    j->m = m;
    j->edges.assign(edges, edges + 2 * m);
    j->xy0.assign(xy0, xy0 + 2 * n);
    j->params = prm;
    j->footprint = fp;
    Request r;
    r.kind = 0;
    r.iters = iters;
    r.remaining = iters;
    r.params = prm;
    r.t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    j->id = s->next_job++;
    r.id = s->next_req++;
    j->queue.push_back(r);
    if (job_id) *job_id = j->id;
    if (request_id) *request_id = r.id;
    s->waiting.push_back(j->id);
    s->jobs[j->id] = std::move(j);
    s->cv_load.notify_all();
    return TFDP_OK;
}

tfdp_status tfdp_server_update(tfdp_server* s, int64_t job_id, const tfdp_params* p, int32_t iters,
                               int64_t* request_id) {
    if (!s || !p || iters < 1) return TFDP_ERR_INVALID_ARG;
    tfdp_params prm = *p;
    prm.total_iters = iters;  // the cooling schedule restarts over the update
    tfdp_status st = tfdp_params_check(&prm, nullptr);
    if (st != TFDP_OK) return st;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end() || it->second->release) return TFDP_ERR_INVALID_ARG;
    Job* j = it->second.get();
    if (prm.k_interp != j->params.k_interp || prm.grid_max != j->params.grid_max ||
        prm.rep_mode != j->params.rep_mode)
        return TFDP_ERR_PARAM_RANGE;  // the job's memory was sized for these
    Request r;
    r.id = s->next_req++;
    r.kind = 1;
    r.iters = iters;
    r.remaining = iters;
    r.params = prm;
    r.t_submit = now_s();
    j->queue.push_back(r);
    if (request_id) *request_id = r.id;
    s->kick.store(true);
    s->cv_work.notify_all();
    return TFDP_OK;
}

tfdp_status tfdp_server_poll(tfdp_server* s, tfdp_done* out, int32_t max, int32_t* count, int32_t wait_ms) {
    if (!s || !count || max < 0 || (max > 0 && !out)) return TFDP_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms));
    const int32_t c = (int32_t)std::min<size_t>(s->done.size(), (size_t)max);
    for (int32_t i = 0; i < c; ++i) out[i] = s->done[(size_t)i];
    s->done.erase(s->done.begin(), s->done.begin() + c);
    *count = c;
    return TFDP_OK;
}

tfdp_status tfdp_server_get_positions(tfdp_server* s, int64_t job_id, float* xy) {
    if (!s || !xy) return TFDP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return TFDP_ERR_INVALID_ARG;
    Job* j = it->second.get();
    if (!j->admitted || !j->queue.empty()) return TFDP_ERR_BUSY;  // work pending or not admitted
    return tfdp_get_positions(j->g, xy, 0);  // the worker leaves an idle job alone
}

tfdp_status tfdp_server_release(tfdp_server* s, int64_t job_id) {
    if (!s) return TFDP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return TFDP_ERR_INVALID_ARG;
    it->second->release = true;
    s->kick.store(true);
    s->cv_work.notify_all();
    return TFDP_OK;
}

tfdp_status tfdp_server_get_stats(tfdp_server* s, tfdp_server_stats* out) {
    if (!s || !out) return TFDP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->active = s->active;
    out->peak_active = s->peak_active;
    out->waiting = (int32_t)s->waiting.size();
    out->jobs = (int32_t)s->jobs.size();
    out->used_bytes = s->used;
    out->budget_bytes = s->budget;
    out->node_iterations = s->node_iterations;
    return TFDP_OK;
}

tfdp_status tfdp_server_destroy(tfdp_server* s) {
    if (!s) return TFDP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
        s->cv_load.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->loader.joinable()) s->loader.join();
    for (auto& kv : s->jobs) {
        Job* j = kv.second.get();
        if (j->g) tfdp_destroy_graph(j->g);
        if (j->ev) cudaEventDestroy(j->ev);
        if (j->stream) cudaStreamDestroy(j->stream);
    }
    delete s;
    return TFDP_OK;
}

}  // extern "C"

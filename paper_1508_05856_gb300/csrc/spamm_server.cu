// Request server for square-root solves (spamm_server_* in include/spamm.h).
//
// Requests arrive at any time (spamm_server_submit) and are admitted in
// arrival order as soon as a worker is free and the device memory the request
// needs (its scratch footprint) fits in the server's budget next to the
// requests already running.  Each worker thread owns a CUDA stream, so
// admitted requests run concurrently on the device while later ones wait;
// finished requests free their share of the budget for the next ones
// (continuous batching).  A request computes exactly what spamm_sqrt_invsqrt
// computes for it: its result does not depend on what else is running.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "spamm.h"
#include "spamm_internal.cuh"

namespace spamm {
namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2 };

struct Request {
    long long id = 0;
    const double* S = nullptr;
    int n = 0;
    double tau = 0.0;
    int maxit = 0;
    double* Y = nullptr;
    double* Z = nullptr;
    size_t bytes = 0;
    int state = REQ_QUEUED;
    int status = SPAMM_OK;
    std::string error;
    spamm_stats stats{};
    Clock::time_point t_submit, t_done;
};

}  // namespace
}  // namespace spamm

using namespace spamm;

struct spamm_server {
    spamm_opts opts{};
    size_t budget = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<long long, Request*> reqs;
    size_t active_bytes = 0;
    bool stop = false;
    long long next_id = 1;
    std::vector<std::thread> workers;

    void worker_loop() {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        spamm_opts o = opts;
        o.stream = st;
        for (;;) {
            Request* r = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    return stop && queue.empty() ? true
                                                 : (!queue.empty() && active_bytes + queue.front()->bytes <= budget);
                });
                if (queue.empty()) break;  // stop requested and nothing left
                r = queue.front();
                queue.pop_front();
                active_bytes += r->bytes;
                r->state = REQ_RUNNING;
            }
            spamm_stats stats{};
            const int status = run_sqrt(r->S, r->n, r->tau, r->maxit, r->Y, r->Z, o, &stats);
            const std::string err = status ? std::string(last_error_message()) : std::string();
            // keep the cached scratch of idle plans within the budget
            trim_plans(budget);
            {
                std::lock_guard<std::mutex> lk(mu);
                r->status = status;
                r->error = err;
                r->stats = stats;
                r->stats.t_hist = nullptr;
                r->stats.task_hist = nullptr;
                r->t_done = Clock::now();
                r->state = REQ_DONE;
                active_bytes -= r->bytes;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        cudaStreamDestroy(st);
    }
};

extern "C" {

int spamm_server_create(size_t bytes_budget, int max_active, const spamm_opts* opts, spamm_server** out) {
    set_error_message("");
    if (!out || bytes_budget == 0 || max_active <= 0 || max_active > 64) {
        set_error_message("need an output pointer, a positive budget and 1..64 active requests");
        return SPAMM_ERR_ARG;
    }
    *out = nullptr;
    spamm_opts o = resolved(opts);
    if (o.residual) {
        set_error_message("the server does not compute residuals");
        return SPAMM_ERR_UNSUPPORTED;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error_message(cudaGetErrorString(e));
        return SPAMM_ERR_CUDA;
    }
    spamm_server* s = new spamm_server;
    s->opts = o;
    s->opts.stream = nullptr;
    s->budget = bytes_budget;
    s->device = dev;
    for (int w = 0; w < max_active; ++w) s->workers.emplace_back([s] { s->worker_loop(); });
    *out = s;
    return SPAMM_OK;
}

int spamm_server_submit(spamm_server* s, const double* S, int n, double tau, int maxit, double* Y, double* Z,
                        long long* id) {
    set_error_message("");
    if (!s || !S || !Y || !Z || !id || maxit < 0) {
        set_error_message("null argument or maxit < 0");
        return SPAMM_ERR_ARG;
    }
    int st = check_args(n, tau, s->opts);
    if (st) return st;
    // device memory of another GPU is refused; host memory (pageable: staged) adds staging to the footprint
    void* vS = nullptr;
    void* vY = nullptr;
    void* vZ = nullptr;
    if ((st = pointer_view(S, s->device, &vS)) || (st = pointer_view(Y, s->device, &vY)) ||
        (st = pointer_view(Z, s->device, &vZ)))
        return st;
    const bool host_io = !vS || !vY || !vZ;
    const size_t bytes = plan_footprint(n, s->opts.leaf, s->opts.precision, host_io);
    if (bytes > s->budget) {
        set_error_message("the request's device footprint exceeds the server's memory budget");
        return SPAMM_ERR_ADMIT;
    }
    Request* r = new Request;
    r->S = S;
    r->n = n;
    r->tau = tau;
    r->maxit = maxit;
    r->Y = Y;
    r->Z = Z;
    r->bytes = bytes;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            set_error_message("server is shutting down");
            return SPAMM_ERR_ARG;
        }
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->queue.push_back(r);
        *id = r->id;
    }
    s->cv_work.notify_all();
    return SPAMM_OK;
}

int spamm_server_poll(spamm_server* s, long long id, int* state) {
    if (!s || !state) return SPAMM_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return SPAMM_ERR_NOTFOUND;
    *state = it->second->state;
    return SPAMM_OK;
}

int spamm_server_wait(spamm_server* s, long long id, double timeout_s, spamm_stats* stats, double* latency_s) {
    if (!s) return SPAMM_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        set_error_message("unknown request id");
        return SPAMM_ERR_NOTFOUND;
    }
    Request* r = it->second;
    auto ready = [&] { return r->state == REQ_DONE; };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        set_error_message("request not finished within the timeout");
        return SPAMM_ERR_TIMEOUT;
    }
    const int status = r->status;
    if (status) set_error_message(r->error.c_str());
    if (stats) {
        double* th = stats->t_hist;
        long long* kh = stats->task_hist;
        *stats = r->stats;
        stats->t_hist = th;
        stats->task_hist = kh;
    }
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    s->reqs.erase(it);
    delete r;
    return status;
}

int spamm_server_destroy(spamm_server* s) {
    if (!s) return SPAMM_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return SPAMM_OK;
}

}  // extern "C"

// Request server for square-root solves (spamm_server_* in include/spamm.h).
//
// Requests arrive at any time (spamm_server_submit) and are admitted in
// arrival order as soon as a worker is free and the device memory the work
// needs fits in the server's budget next to the work already running.  Each
// worker owns a CUDA stream, so admitted work of different workers runs
// concurrently on the device while later requests wait; finished work frees
// its share of the budget for the next (continuous batching).
//
// When the options are ones the batched engine covers (spamm_batch.cu) and a
// request's matrices are device or page-locked memory, a worker takes the
// head of the queue together with the requests queued behind it (same
// iteration count, up to kMaxGroup, within the worker's share of the budget)
// and solves them as one batch: every stage of their iterations is one
// launch of each kernel over all of them, so concurrent requests share the
// leaf-product launches.  Other requests run one per worker.  A request
// computes exactly what spamm_sqrt_invsqrt computes for it: its result does
// not depend on what else is running or what it is grouped with.
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

constexpr int kMaxGroup = 64;

struct Request {
    long long id = 0;
    bool grouped = false;  // may share a batch with other requests
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

    // the batched engine's buffers and graph of each worker, and the share of the budget one group may use
    std::vector<BatchSlot*> slots;
    size_t group_limit = 0;

    void finish(Request* r, int status, const std::string& err, const spamm_stats& stats) {
        r->status = status;
        r->error = err;
        r->stats = stats;
        r->stats.t_hist = nullptr;
        r->stats.task_hist = nullptr;
        r->stats.lens_hist = nullptr;
        r->t_done = Clock::now();
        r->state = REQ_DONE;
    }

    void worker_loop(int w) {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        spamm_opts o = opts;
        o.stream = st;
        std::vector<Request*> grp;
        for (;;) {
            grp.clear();
            size_t gbytes = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    return stop && queue.empty() ? true
                                                 : (!queue.empty() && active_bytes + queue.front()->bytes <= budget);
                });
                if (queue.empty()) break;  // stop requested and nothing left
                Request* head = queue.front();
                queue.pop_front();
                grp.push_back(head);
                gbytes = head->bytes;
                // requests queued behind the head join its batch while they fit the worker's share
                while (head->grouped && head->bytes <= group_limit && (int)grp.size() < kMaxGroup && !queue.empty()) {
                    Request* r = queue.front();
                    if (!r->grouped || r->maxit != head->maxit || gbytes + r->bytes > group_limit ||
                        active_bytes + gbytes + r->bytes > budget)
                        break;
                    queue.pop_front();
                    grp.push_back(r);
                    gbytes += r->bytes;
                }
                active_bytes += gbytes;
                for (Request* r : grp) r->state = REQ_RUNNING;
            }
            std::vector<spamm_stats> stats(grp.size());
            std::vector<int> status(grp.size(), SPAMM_ERR_UNSUPPORTED);
            std::vector<std::string> err(grp.size());
            int e = SPAMM_ERR_UNSUPPORTED;
            if (grp.size() > 1) {
                std::vector<const double*> S(grp.size());
                std::vector<double*> Y(grp.size()), Z(grp.size());
                std::vector<int> n(grp.size());
                std::vector<double> tau(grp.size());
                for (size_t q = 0; q < grp.size(); ++q) {
                    S[q] = grp[q]->S;
                    Y[q] = grp[q]->Y;
                    Z[q] = grp[q]->Z;
                    n[q] = grp[q]->n;
                    tau[q] = grp[q]->tau;
                }
                e = batched_solve_slot(slots[w], (int)grp.size(), S.data(), n.data(), tau.data(), grp[0]->maxit,
                                       Y.data(), Z.data(), o, stats.data(), group_limit, status.data());
                if (e != SPAMM_ERR_UNSUPPORTED && e != SPAMM_OK) {
                    const std::string m = last_error_message();
                    for (size_t q = 0; q < grp.size(); ++q) {
                        // a failure of the whole batch (not one problem's own status) goes to every request
                        if (status[q] == SPAMM_ERR_UNSUPPORTED || e == SPAMM_ERR_TIMEOUT || e == SPAMM_ERR_CUDA)
                            status[q] = e;
                        if (status[q]) err[q] = status[q] == e ? m : std::string(spamm_strerror(status[q]));
                    }
                }
            }
            if (e == SPAMM_ERR_UNSUPPORTED) {
                for (size_t q = 0; q < grp.size(); ++q) {
                    Request* r = grp[q];
                    stats[q] = spamm_stats{};
                    status[q] = run_sqrt(r->S, r->n, r->tau, r->maxit, r->Y, r->Z, o, &stats[q]);
                    if (status[q]) err[q] = last_error_message();
                }
                // keep the cached scratch of idle plans within the budget
                trim_plans(budget);
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                for (size_t q = 0; q < grp.size(); ++q) finish(grp[q], status[q], err[q], stats[q]);
                active_bytes -= gbytes;
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
    s->group_limit = bytes_budget / (size_t)max_active;
    for (int w = 0; w < max_active; ++w) s->slots.push_back(batch_slot_create());
    for (int w = 0; w < max_active; ++w) s->workers.emplace_back([s, w] { s->worker_loop(w); });
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
    const bool grouped = !host_io && batch_engine_covers(s->opts) &&
                         batch_footprint(n, s->opts.leaf, s->opts.precision, maxit) <= s->group_limit;
    const size_t bytes = grouped ? batch_footprint(n, s->opts.leaf, s->opts.precision, maxit)
                                 : plan_footprint(n, s->opts.leaf, s->opts.precision, host_io);
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
    r->grouped = grouped;
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
    for (BatchSlot* b : s->slots) batch_slot_destroy(b);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return SPAMM_OK;
}

}  // extern "C"

// C ABI of libspamm (declared in include/spamm.h): argument checks, scratch
// management per problem size, and the host-side driver of the SpAMM product
// and of the dual-channel Newton-Schulz iteration (Eq. (cannonical)).
//
// Every arithmetic step runs in the CUDA kernels of kernels_*.cu; this file
// only orders the launches on the caller's stream and moves data across the
// host/device boundary when the caller passes host pointers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <atomic>
#include <tuple>
#include <vector>

#include "spamm.h"
#include "spamm_internal.cuh"

namespace spamm {

static std::atomic<long long> g_launches{0};
// this thread's launches: what a capture on this thread enqueued (other threads may launch meanwhile)
static thread_local long long t_launches = 0;
void note_launch(int k) {
    g_launches.fetch_add(k, std::memory_order_relaxed);
    t_launches += k;
}

static std::mutex g_attr_mu;
static bool g_attr_done[64] = {};
static int g_sm_count[64] = {};

void init_device_attributes() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (g_attr_done[dev]) return;
    f64_kernel_attributes();
    emu_kernel_attributes();
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_sm_count[dev] = sms > 0 ? sms : 1;
    g_attr_done[dev] = true;
}

int device_sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    return (dev >= 0 && dev < 64 && g_sm_count[dev] > 0) ? g_sm_count[dev] : 148;
}

static thread_local std::string g_last_error;

void set_error_message(const char* msg) { g_last_error = msg; }

static void set_error(const char* what, cudaError_t e) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    g_last_error = buf;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) {                  \
            set_error(#call, e_);                 \
            return SPAMM_ERR_CUDA;                \
        }                                         \
    } while (0)

#define CKA(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) {                               \
            set_error(#call, e_);                              \
            return e_ == cudaErrorMemoryAllocation ? SPAMM_ERR_NOMEM : SPAMM_ERR_CUDA; \
        }                                                      \
    } while (0)

// The address kernels use for a caller matrix they can read and write in place, for work on `device`:
// device memory of that device or managed memory as it is, and page-locked host memory through its device
// mapping (on this part the GPU reaches host memory over NVLink-C2C, so the pack and unpack kernels move the
// data themselves, with no staging copy).  *view is null for pageable host memory, which is staged.  Device
// memory of another GPU is an argument error: without peer access the kernels cannot reach it.
int pointer_view(const void* p, int device, void** view) {
    *view = nullptr;
    if (!p) return SPAMM_OK;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return SPAMM_OK;
    }
    if (a.type == cudaMemoryTypeManaged) {
        *view = const_cast<void*>(p);
    } else if (a.type == cudaMemoryTypeDevice) {
        if (a.device != device) {
            char buf[160];
            snprintf(buf, sizeof(buf), "a matrix is device memory of GPU %d, but the call runs on GPU %d", a.device,
                     device);
            g_last_error = buf;
            return SPAMM_ERR_ARG;
        }
        *view = const_cast<void*>(p);
    } else if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *view = a.devicePointer;
    }
    return SPAMM_OK;
}

static int current_view(const void* p, void** view) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    return pointer_view(p, dev, view);
}

// ----------------------------------------------------------------------------
// What a captured solve graph depends on besides the plan's own buffers.
struct GraphKey {
    const double* S = nullptr;
    double* Y = nullptr;
    double* Z = nullptr;
    int n = 0, leaf = 0, precision = 0, order = 0, maxit = 0, profile = 0, map = 0, channel = 0, lens_bins = 0;
    double tau = 0.0, tau_s = 0.0, mu_rel = 0.0, tol_t = 0.0;
    bool operator==(const GraphKey& o) const {
        return S == o.S && Y == o.Y && Z == o.Z && n == o.n && leaf == o.leaf && precision == o.precision &&
               order == o.order && maxit == o.maxit && profile == o.profile && map == o.map &&
               channel == o.channel && lens_bins == o.lens_bins && tau == o.tau &&
               tau_s == o.tau_s && mu_rel == o.mu_rel && tol_t == o.tol_t;
    }
};

// Scratch of one problem size on one device.  Device flags (ints): [0] stop, [1] iterations run, [2] error
// of a bounded wait, [8..11] leaf-product tile tickets (two branches), [16..20] and [24..28] output-tile
// bucket counts (two branches), [30..31] tensor-core units issued (64-bit).
constexpr int kFlagInts = 32;

struct Plan {
    int device = 0;
    Geometry g;
    TileMat buf[6];
    int* counts = nullptr;
    int* jlist = nullptr;
    int* tile_list = nullptr;                // [kTileBuckets*m*m] compacted output tiles of one product
    // second product scratch and stream: the iteration's two independent
    // products (Y and Z updates) run on two branches
    int* counts2 = nullptr;
    int* jlist2 = nullptr;
    int* tile_list2 = nullptr;
    // plane-diagonal profiles of the products (stats->lens_hist): lens_bins > 0 for this call
    unsigned long long* lens = nullptr;
    size_t lens_elems = 0;
    int lens_bins = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // tensor-core path: the slicing of a product output runs on its own stream per branch, beside the
    // tree and the next culls; ev_norm orders it after the output's norm pass
    cudaStream_t slice_st[2] = {nullptr, nullptr};
    // the prologue's side passes (Z0, X0's slices): streams of their own, never used inside a loop body,
    // which is captured separately from the solve around it
    cudaStream_t pro_st[2] = {nullptr, nullptr};
    cudaEvent_t ev_norm[2] = {nullptr, nullptr};
    unsigned sliced_mask = 0;  // buffers whose `sliced` event this call recorded
    unsigned long long* task_ctr = nullptr;  // [3 * maxit_cap + 4]
    double* t_hist = nullptr;                // [maxit_cap]
    int maxit_cap = 0;
    double* trace_part = nullptr;  // [m]
    double* scal = nullptr;        // c0, mu, c, sqrt c, thr, resid, 1/c, 1/sqrt c, spare...
    double* rowsum = nullptr;      // [n]
    int* flags = nullptr;          // [0] done, [1] iters, [2] device error, [8..11] tile tickets of the
                                   // tensor-core kernel per branch, [16 + 8 b ..] output-tile bucket counts
    double* partial = nullptr;     // [m*m]
    double* stage[3] = {nullptr, nullptr, nullptr};  // n*n row-major staging
    // profiling: event pairs around each leaf-product, cull, tree and slicing kernel of a call, and what
    // each pair times (ProfKind)
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    int ev_used = 0;
    bool profile = false;
    long long gemm_launches = 0;
    unsigned long long last_use = 0;  // release order, for evicting the least recently used idle plan
    bool emu = false;        // this call uses the tensor-core (SPAMM_EMU64) leaf products
    long long stall_polls = 0;  // the next tensor-core leaf-product launch takes its expired-wait path
    bool emu_ready = false;  // slice buffers allocated
    // CUDA graph of the last fixed-iteration solve and what it was captured for
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    long long graph_kernels = 0;       // kernels of one replay (a loop graph: without its body)
    long long graph_body_kernels = 0;  // kernels of one loop body (two iterations)
    bool graph_loop = false;           // the iteration is a WHILE conditional node
    int graph_events = 0;       // profiling events recorded inside the graph
    long long graph_gemm = 0;   // leaf-product launches inside the graph
    cudaStream_t gstream = nullptr;
    cudaStream_t bstream = nullptr;    // captures the loop body
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

static void free_plan(Plan* p) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    for (auto& b : p->buf) {
        cudaFree(b.t);
        cudaFree(b.tree);
        cudaFree(b.sliceA);
        cudaFree(b.sliceB);
        cudaFree(b.rmax);
        cudaFree(b.slice_list);
        if (b.sliced) cudaEventDestroy(b.sliced);
    }
    for (int q = 0; q < 2; ++q) {
        if (p->slice_st[q]) cudaStreamDestroy(p->slice_st[q]);
        if (p->pro_st[q]) cudaStreamDestroy(p->pro_st[q]);
        if (p->ev_norm[q]) cudaEventDestroy(p->ev_norm[q]);
    }
    cudaFree(p->counts);
    cudaFree(p->jlist);
    cudaFree(p->tile_list);
    cudaFree(p->counts2);
    cudaFree(p->jlist2);
    cudaFree(p->tile_list2);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    cudaFree(p->task_ctr);
    cudaFree(p->t_hist);
    cudaFree(p->trace_part);
    cudaFree(p->lens);
    cudaFree(p->scal);
    cudaFree(p->rowsum);
    cudaFree(p->flags);
    cudaFree(p->partial);
    for (auto& s : p->stage) cudaFree(s);
    for (auto e : p->ev) cudaEventDestroy(e);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->gstream) cudaStreamDestroy(p->gstream);
    if (p->bstream) cudaStreamDestroy(p->bstream);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    cudaSetDevice(cur);
    delete p;
}

// Idle cached plans are freed when a device allocation fails; defined after the pool.
static void free_idle_plans();

// cudaMalloc that, when the device is out of memory, frees the idle cached plans and tries once more.
static cudaError_t dev_alloc(void** ptr, size_t bytes) {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        free_idle_plans();
        e = cudaMalloc(ptr, bytes);
    }
    return e;
}
template <typename T>
static cudaError_t dev_alloc(T** ptr, size_t bytes) {
    return dev_alloc(reinterpret_cast<void**>(ptr), bytes);
}

static int alloc_plan(Plan* p, int n, int nb) {
    p->g = make_geometry(n, nb);
    const Geometry& g = p->g;
    for (auto& b : p->buf) {
        CKA(dev_alloc(&b.t, g.elems() * sizeof(double)));
        CKA(dev_alloc(&b.tree, g.tree_size * sizeof(double)));
    }
    CKA(dev_alloc(&p->counts, (size_t)g.m * g.m * sizeof(int)));
    CKA(dev_alloc(&p->jlist, (size_t)g.m * g.m * g.m * sizeof(int)));
    CKA(dev_alloc(&p->tile_list, (size_t)kTileBuckets * g.m * g.m * sizeof(int)));
    CKA(dev_alloc(&p->counts2, (size_t)g.m * g.m * sizeof(int)));
    CKA(dev_alloc(&p->jlist2, (size_t)g.m * g.m * g.m * sizeof(int)));
    CKA(dev_alloc(&p->tile_list2, (size_t)kTileBuckets * g.m * g.m * sizeof(int)));
    CKA(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    CKA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    CKA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    CKA(dev_alloc(&p->trace_part, (size_t)g.m * sizeof(double)));
    CKA(dev_alloc(&p->scal, 16 * sizeof(double)));
    CKA(dev_alloc(&p->rowsum, (size_t)n * sizeof(double)));
    CKA(dev_alloc(&p->flags, kFlagInts * sizeof(int)));
    CKA(dev_alloc(&p->partial, (size_t)g.m * g.m * sizeof(double)));
    return SPAMM_OK;
}

// Device histograms of the plane-diagonal profile: maxit_cap iterations x 3 products x 3 planes x bins.
static int ensure_lens(Plan* p, int bins) {
    const size_t need = (size_t)p->maxit_cap * 9 * bins;
    if (need <= p->lens_elems) return SPAMM_OK;
    cudaFree(p->lens);
    p->lens = nullptr;
    p->lens_elems = 0;
    CKA(dev_alloc(&p->lens, need * sizeof(unsigned long long)));
    p->lens_elems = need;
    return SPAMM_OK;
}

static int ensure_hist(Plan* p, int maxit) {
    if (maxit <= p->maxit_cap) return SPAMM_OK;
    cudaFree(p->task_ctr);
    cudaFree(p->t_hist);
    p->task_ctr = nullptr;
    p->t_hist = nullptr;
    int cap = maxit < 64 ? 64 : maxit;
    CKA(dev_alloc(&p->task_ctr, (3 * (size_t)cap + 4) * sizeof(unsigned long long)));
    CKA(dev_alloc(&p->t_hist, (size_t)cap * sizeof(double)));
    p->maxit_cap = cap;
    return SPAMM_OK;
}

static int ensure_emu(Plan* p) {
    if (p->emu_ready) return SPAMM_OK;
    const Geometry& g = p->g;
    const size_t per = emu_slice_bytes_per_tile() * (size_t)g.m * g.m;
    for (auto& b : p->buf) {
        CKA(dev_alloc(&b.sliceA, per));
        CKA(dev_alloc(&b.sliceB, per));
        CKA(dev_alloc(&b.rmax, 2 * (size_t)g.m * g.nb * sizeof(unsigned long long)));
        b.cmax = b.rmax + (size_t)g.m * g.nb;
        CKA(dev_alloc(&b.slice_list, ((size_t)g.m * g.m + 1) * sizeof(int)));
        CKA(cudaEventCreateWithFlags(&b.sliced, cudaEventDisableTiming));
    }
    for (int q = 0; q < 2; ++q) {
        CKA(cudaStreamCreateWithFlags(&p->slice_st[q], cudaStreamNonBlocking));
        CKA(cudaStreamCreateWithFlags(&p->pro_st[q], cudaStreamNonBlocking));
        CKA(cudaEventCreateWithFlags(&p->ev_norm[q], cudaEventDisableTiming));
    }
    p->emu_ready = true;
    return SPAMM_OK;
}

static int ensure_stage(Plan* p, int which) {
    if (p->stage[which]) return SPAMM_OK;
    CKA(dev_alloc(&p->stage[which], (size_t)p->g.n * p->g.n * sizeof(double)));
    return SPAMM_OK;
}

// Device bytes one plan holds (tile buffers, trees, task lists, slices for
// the tensor-core path, row-major staging when the caller passes host memory).
size_t plan_footprint(int n, int nb, int precision, bool host_io) {
    // leaf 0 (chosen later by the autotuner): the largest scratch among the sizes it may pick
    if (nb == 0) nb = precision == SPAMM_EMU64 ? 64 : 32;
    const Geometry g = make_geometry(n, nb);
    size_t b = 6 * (g.elems() + (size_t)g.tree_size) * sizeof(double);
    b += 2 * ((size_t)g.m * g.m * (g.m + 1 + kTileBuckets)) * sizeof(int) + (size_t)g.m * sizeof(double) +
         (size_t)n * sizeof(double) +
         (size_t)g.m * g.m * sizeof(double) + 4096;
    if (precision == SPAMM_EMU64)
        b += 6 * (2 * emu_slice_bytes_per_tile() * (size_t)g.m * g.m + 2 * (size_t)g.m * g.nb * 8 +
                  ((size_t)g.m * g.m + 1) * sizeof(int));
    if (host_io) b += 3 * (size_t)n * n * sizeof(double);
    return b;
}

static size_t plan_bytes(const Plan* p) {
    return plan_footprint(p->g.n, p->g.nb, p->emu_ready ? SPAMM_EMU64 : SPAMM_FP64, p->stage[0] != nullptr);
}

class PlanPool {
  public:
    int acquire(int n, int nb, Plan** out) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        auto key = std::make_tuple(dev, n, nb);
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto& v = free_[key];
            if (!v.empty()) {
                *out = v.back();
                v.pop_back();
                return SPAMM_OK;
            }
        }
        Plan* p = new Plan;
        p->device = dev;
        int st = alloc_plan(p, n, nb);
        if (st) {
            free_plan(p);
            return st;
        }
        *out = p;
        return SPAMM_OK;
    }
    // Idle plans are kept for reuse up to a quarter of the device's memory; beyond that the least
    // recently released ones are freed.
    void release(Plan* p) {
        std::lock_guard<std::mutex> lk(mu_);
        p->last_use = ++clock_;
        free_[std::make_tuple(p->device, p->g.n, p->g.nb)].push_back(p);
        const size_t cap = idle_cap(p->device);
        for (;;) {
            size_t idle = 0;
            Plan* oldest = nullptr;
            std::vector<Plan*>* where = nullptr;
            for (auto& kv : free_)
                for (Plan* q : kv.second) {
                    if (q->device != p->device) continue;
                    idle += plan_bytes(q);
                    if (!oldest || q->last_use < oldest->last_use) {
                        oldest = q;
                        where = &kv.second;
                    }
                }
            if (idle <= cap || !oldest || oldest == p) break;
            where->erase(std::find(where->begin(), where->end(), oldest));
            free_plan(oldest);
        }
    }
    void clear() {
        std::lock_guard<std::mutex> lk(mu_);
        for (auto& kv : free_)
            for (Plan* p : kv.second) free_plan(p);
        free_.clear();
    }
    // Free idle plans until the idle ones hold at most keep_bytes.
    void trim(size_t keep_bytes) {
        std::lock_guard<std::mutex> lk(mu_);
        size_t idle = 0;
        for (auto& kv : free_)
            for (Plan* p : kv.second) idle += plan_bytes(p);
        for (auto& kv : free_) {
            while (idle > keep_bytes && !kv.second.empty()) {
                Plan* p = kv.second.back();
                kv.second.pop_back();
                idle -= std::min(idle, plan_bytes(p));
                free_plan(p);
            }
        }
    }

  private:
    static size_t idle_cap(int device) {
        static std::mutex m;
        static std::map<int, size_t> caps;
        std::lock_guard<std::mutex> lk(m);
        auto it = caps.find(device);
        if (it != caps.end()) return it->second;
        size_t fr = 0, tot = 0;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            tot = (size_t)16 << 30;
        }
        cudaSetDevice(cur);
        return caps[device] = tot / 4;
    }
    std::mutex mu_;
    unsigned long long clock_ = 0;
    std::map<std::tuple<int, int, int>, std::vector<Plan*>> free_;
};

static PlanPool g_pool;

static void free_idle_plans() { g_pool.clear(); }

struct PlanGuard {
    Plan* p = nullptr;
    ~PlanGuard() {
        if (p) g_pool.release(p);
    }
};

static bool leaf_ok(int nb) { return nb == 32 || nb == 64 || nb == 128; }

static spamm_opts resolve_opts(const spamm_opts* o) {
    spamm_opts r;
    spamm_opts_init(&r);
    if (o) r = *o;
    return r;  // leaf 0 stays 0: the call resolves it with the autotuner
}

// Device view of a caller matrix: the pointer itself (or its device mapping), or a staged copy.
// A caller matrix in host memory (page-locked or not).
static bool host_memory(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// read_once: the kernels read the input a single time, so page-locked host memory is read in place through
// its device mapping; an input read more than once (the solve's S: row sums, then the pack) is copied to
// the device once instead, by the copy engine, so that the link carries it once.
static int stage_in(Plan* p, int which, const double* src, cudaStream_t st, const double** dev,
                    bool read_once = true) {
    void* v = nullptr;
    int e = pointer_view(src, p->device, &v);
    if (e) return e;
    if (v && !read_once && host_memory(src)) v = nullptr;
    if (v) {
        *dev = static_cast<const double*>(v);
        return SPAMM_OK;
    }
    e = ensure_stage(p, which);
    if (e) return e;
    CK(cudaMemcpyAsync(p->stage[which], src, (size_t)p->g.n * p->g.n * sizeof(double), cudaMemcpyHostToDevice, st));
    *dev = p->stage[which];
    return SPAMM_OK;
}

static int out_target(Plan* p, int which, double* dst, double** dev) {
    void* v = nullptr;
    int e = pointer_view(dst, p->device, &v);
    if (e) return e;
    if (v) {
        *dev = static_cast<double*>(v);
        return SPAMM_OK;
    }
    e = ensure_stage(p, which);
    if (e) return e;
    *dev = p->stage[which];
    return SPAMM_OK;
}

// Copies a staged result out; a result the kernels wrote in place (device memory or the mapping of a
// page-locked host buffer) needs nothing.
static int stage_out(Plan* p, int which, double* dst, const double* dev, cudaStream_t st) {
    if (dev != p->stage[which]) return SPAMM_OK;
    CK(cudaMemcpyAsync(dst, dev, (size_t)p->g.n * p->g.n * sizeof(double), cudaMemcpyDeviceToHost, st));
    return SPAMM_OK;
}

static void begin_call(Plan* p, bool profile, bool emu) {
    p->lens_bins = 0;
    p->profile = profile;
    p->emu = emu;
    p->ev_used = 0;
    p->gemm_launches = 0;
    p->sliced_mask = 0;
}

// What a profiled event pair times.
enum ProfKind { PROF_GEMM = 0, PROF_CULL = 1, PROF_TREE = 2, PROF_SLICE = 3 };

static cudaEvent_t next_event(Plan* p, int kind) {
    if (p->ev_used == (int)p->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p->ev.push_back(e);
        p->ev_kind.push_back(kind);
    }
    p->ev_kind[p->ev_used] = kind;
    return p->ev[p->ev_used++];
}

// Summed duration of the profiled kernels of one kind, and how many were timed (call after the stream is
// synchronised).
static double profiled_ms(Plan* p, int kind, long long* count = nullptr) {
    double ms = 0.0;
    long long c = 0;
    for (int q = 0; q + 1 < p->ev_used; q += 2) {
        if (p->ev_kind[q] != kind) continue;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->ev[q], p->ev[q + 1]) == cudaSuccess) {
            ms += t;
            ++c;
        } else {
            cudaGetLastError();  // leave no error behind for the caller
        }
    }
    if (count) *count = c;
    return ms;
}

// Events around the kernels enqueued on `st` while it lives, when the call is profiled.  Under stream capture
// the records are "external", so that they become event-record nodes of the graph; an uncaptured call (a
// single product) records plainly.
struct ProfSpan {
    cudaEvent_t e1 = nullptr;
    cudaStream_t st = nullptr;
    unsigned flags = cudaEventRecordDefault;
    ProfSpan(Plan* p, cudaStream_t s, int kind) : st(s) {
        if (!p->profile) return;
        cudaEvent_t e0 = next_event(p, kind);
        e1 = next_event(p, kind);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
            flags = cudaEventRecordExternal;
        if (e0 && e1) cudaEventRecordWithFlags(e0, st, flags);
        else e1 = nullptr;
    }
    ~ProfSpan() {
        if (e1) cudaEventRecordWithFlags(e1, st, flags);
    }
};

// Profiled kernel times of the call into stats.
static void profile_stats(Plan* p, spamm_stats* stats) {
    if (!p->profile) {
        stats->gemm_ms = stats->cull_ms = stats->tree_ms = stats->slice_ms = 0.0;
        stats->cull_launches = stats->tree_launches = stats->slice_launches = 0;
        return;
    }
    stats->gemm_ms = profiled_ms(p, PROF_GEMM);
    stats->cull_ms = profiled_ms(p, PROF_CULL, &stats->cull_launches);
    stats->tree_ms = profiled_ms(p, PROF_TREE, &stats->tree_launches);
    stats->slice_ms = profiled_ms(p, PROF_SLICE, &stats->slice_launches);
}

// Tensor-core work issued by the call's leaf products (flags[30..31], cleared with the flags).
static unsigned long long* tensor_units(Plan* p) { return reinterpret_cast<unsigned long long*>(p->flags + 30); }

static bool slicing_pending(const Plan* p, const TileMat& M) {
    for (int q = 0; q < 6; ++q)
        if (p->buf[q].t == M.t) return (p->sliced_mask >> q) & 1u;
    return false;
}

// One SpAMM product of two packed operands into dst (tree leaves + levels).
// Records that M's slices are complete once `st` reaches this point.
static void mark_sliced(Plan* p, const TileMat& M, cudaStream_t st) {
    for (int q = 0; q < 6; ++q)
        if (p->buf[q].t == M.t) {
            cudaEventRecord(p->buf[q].sliced, st);
            p->sliced_mask |= 1u << q;
        }
}

// The output-tile bucket counters are zero on entry (the call's flag reset,
// then the tree pass of the previous product on the branch); the tree pass
// may also carry the iteration's trace error (tk).
static void product(Plan* p, const TileMat& A, const TileMat& B, TileMat& C, double tau, EpiMode mode,
                    unsigned long long* ctr, cudaStream_t st, const TreeExtra* tk = nullptr, int slot = 0,
                    int map = SPAMM_MAP_NS) {
    const Geometry& g = p->g;
    int* counts = slot ? p->counts2 : p->counts;
    int* jlist = slot ? p->jlist2 : p->jlist;
    int* tile_list = slot ? p->tile_list2 : p->tile_list;
    int* tile_count = p->flags + 16 + 8 * slot;  // kTileBuckets counts
    CullOut co{counts, jlist, tile_list, tile_count, C.tree, mode != EPI_PLAIN ? 1 : 0};
    co.iter = p->flags + 1;  // the task counter of iteration k is ctr[3 k]
    co.buckets = kTileBuckets;
    if (p->emu) {
        co.zero_u64 = C.rmax;  // rmax and cmax, contiguous
        co.zero_n = 2 * (long)g.m * g.nb;
    }
    {
        ProfSpan ps(p, st, PROF_CULL);
        launch_cull(g, A.tree, B.tree, tau, co, ctr, nullptr, p->flags, st);
    }
    if (p->lens_bins > 0)
        launch_lens(counts, jlist, g, p->lens_bins, p->flags + 1, (int)(ctr - p->task_ctr), p->lens, p->flags, st);
    if (p->emu) {
        // the operands' slices may still be in flight on a slicing stream (only slicing enqueued since the
        // last join is waited on: a captured loop body depends on nothing recorded outside it)
        if (slicing_pending(p, A)) cudaStreamWaitEvent(st, A.sliced, 0);
        if (B.sliced != A.sliced && slicing_pending(p, B)) cudaStreamWaitEvent(st, B.sliced, 0);
    }
    {
        ProfSpan ps(p, st, PROF_GEMM);
        if (p->emu) {
            launch_gemm_emu(g, A, B, C, counts, jlist, tile_list, tile_count, mode, p->trace_part,
                            p->flags + 8 + 2 * slot, p->flags, p->flags + 2, tau, st, kTileBuckets,
                            tensor_units(p), p->stall_polls);
            p->stall_polls = 0;
        } else {
            launch_gemm_f64(g, A.t, B.t, C.t, A.tree, B.tree, C.tree, counts, jlist, tile_list, tile_count, 0,
                            mode, p->trace_part, p->flags, st, kTileBuckets);
        }
    }
    p->gemm_launches++;
    // X's map whose coefficients need the finished tr X: in place, with T's leaf norms (and maxima)
    if (mode == EPI_X) launch_map(C.t, C.tree, C, g, map, p->trace_part, p->emu, p->flags, st);
    if (p->emu) {
        // tensor-core path: the leaf-product kernel wrote the output's leaf norms (all the tree and the next
        // culls need); its slices follow on the branch's slicing stream, beside the tree and the next culls.
        // A profiled call keeps everything on one stream so that kernel timings are the kernels' own
        cudaStream_t ss = p->profile ? st : p->slice_st[slot];
        if (ss != st) {
            cudaEventRecord(p->ev_norm[slot], st);
            cudaStreamWaitEvent(ss, p->ev_norm[slot], 0);
        }
        const int mm = g.m * g.m;
        {
            ProfSpan ps(p, ss, PROF_SLICE);
            launch_slice(C.t, C.tree, nullptr, C.rmax, C.cmax, C.sliceA, C.sliceB, g, C.slice_list,
                         C.slice_list + mm, p->flags, ss);
        }
        mark_sliced(p, C, ss);
    }
    TreeExtra ex = tk ? *tk : TreeExtra();
    ex.zero_int = tile_count;
    ex.zero_n = kTileBuckets;
    ProfSpan ps(p, st, PROF_TREE);
    launch_tree(g, C.tree, p->flags, st, ex);
}

// Row/column maxima and slices of a freshly packed matrix (tensor-core path).
// tau_min > 0: every product that reads M culls at tau >= tau_min, so the tiles below 0.999 tau_min^2 of M's
// squared norm are never read (a kept pair has nu_a nu_b >= tau^2 nu_A nu_B with nu_b <= nu_B; the factor
// leaves a margin far above the rounding of that test) and are not sliced.  M's quadtree must be complete.
static void slice_emu(Plan* p, const TileMat& M, cudaStream_t st, double tau_min) {
    const Geometry& g = p->g;
    launch_slice(M.t, M.tree, nullptr, M.rmax, M.cmax, M.sliceA, M.sliceB, g, nullptr, nullptr, nullptr, st,
                 tau_min > 0.0 ? M.tree + g.off[0] : nullptr, 0.999 * tau_min * tau_min);
    mark_sliced(p, M, st);
}
static void prepare_emu(Plan* p, const TileMat& M, cudaStream_t st, double tau_min = 0.0) {
    const Geometry& g = p->g;
    cudaMemsetAsync(M.rmax, 0, 2 * (size_t)g.m * g.nb * sizeof(unsigned long long), st);
    launch_rowcol_max(M.t, g, M.rmax, M.cmax, st);
    slice_emu(p, M, st, tau_min);
}

// Every slicing stream of this call joins the call's stream (before the outputs are read, and before a
// capture ends); only events recorded by this call are waited on.
static void join_slicing(Plan* p, cudaStream_t st) {
    for (int q = 0; q < 6; ++q)
        if (p->sliced_mask & (1u << q)) cudaStreamWaitEvent(st, p->buf[q].sliced, 0);
    p->sliced_mask = 0;
}

// Set by spamm_test_expire_next_wait: the next tensor-core product of this thread takes the kernel's
// expired-wait path.
static thread_local long long t_stall_next = 0;

static int multiply_core(const double* A, const double* B, double* C, int n, double tau, const spamm_opts& o,
                         spamm_stats* stats) {
    cudaStream_t st = (cudaStream_t)o.stream;
    init_device_attributes();
    PlanGuard pg;
    int e = g_pool.acquire(n, o.leaf, &pg.p);
    if (e) return e;
    Plan* p = pg.p;
    const Geometry& g = p->g;
    if ((e = ensure_hist(p, 1))) return e;
    const double *dA, *dB;
    double* dC;
    if ((e = stage_in(p, 0, A, st, &dA))) return e;
    if ((e = stage_in(p, 1, B, st, &dB))) return e;
    if ((e = out_target(p, 2, C, &dC))) return e;
    begin_call(p, o.profile != 0, o.precision == SPAMM_EMU64);
    if (p->emu && (e = ensure_emu(p))) return e;
    if (p->emu) {
        p->stall_polls = t_stall_next;
        t_stall_next = 0;
    }
    CK(cudaMemsetAsync(p->flags, 0, kFlagInts * sizeof(int), st));
    CK(cudaMemsetAsync(p->task_ctr, 0, 4 * sizeof(unsigned long long), st));
    launch_pack(dA, n, g, nullptr, nullptr, p->buf[0], st);
    launch_tree(g, p->buf[0].tree, nullptr, st);
    launch_pack(dB, n, g, nullptr, nullptr, p->buf[1], st);
    launch_tree(g, p->buf[1].tree, nullptr, st);
    if (p->emu) {
        prepare_emu(p, p->buf[0], st);
        prepare_emu(p, p->buf[1], st);
    }
    product(p, p->buf[0], p->buf[1], p->buf[2], tau, EPI_PLAIN, p->task_ctr, st);
    join_slicing(p, st);
    launch_unpack(p->buf[2].t, p->buf[2].tree, g, dC, nullptr, st);
    CK(cudaGetLastError());
    if ((e = stage_out(p, 2, C, dC, st))) return e;
    unsigned long long tasks = 0;
    int flags_h[kFlagInts] = {};
    CK(cudaMemcpyAsync(&tasks, p->task_ctr, sizeof(tasks), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(flags_h, p->flags, kFlagInts * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flags_h[2]) {
        g_last_error = "a bounded device-side wait of the tensor-core kernel expired";
        return SPAMM_ERR_TIMEOUT;
    }
    if (stats) {
        stats->iters = 0;
        stats->t_final = 0.0;
        stats->resid_F = -1.0;
        stats->scale_c = 1.0;
        stats->tasks_total = (long long)tasks;
        stats->tasks_dense = (long long)g.m * g.m * g.m;
        stats->flops = 2.0 * (double)g.nb * g.nb * g.nb * (double)tasks;
        profile_stats(p, stats);
        stats->gemm_launches = p->gemm_launches;
        unsigned long long units = 0;
        std::memcpy(&units, flags_h + 30, sizeof(units));
        stats->tensor_units = (long long)units;
    }
    return SPAMM_OK;
}

// ||Z S Z - I||_F in FP64 with dense products (verification only).
// ---- leaf-size autotuner (opts.leaf = 0) --------------------------------
// Times one SpAMM product S (x)_tau S at every leaf size the arithmetic
// supports (32, 64, 128 for SPAMM_FP64; SPAMM_EMU64 runs on 64 only) and keeps
// the fastest, per device, size, arithmetic and decade of tau.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, int> g_tune;

static int tau_decade(double tau) { return tau > 0.0 ? (int)std::floor(std::log10(tau)) : -1000; }

static int autotune_leaf_impl(const double* S, int n, double tau, const spamm_opts& o, int* leaf) {
    if (o.precision == SPAMM_EMU64) {
        *leaf = 64;
        return SPAMM_OK;
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, n, o.precision, tau_decade(tau));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *leaf = it->second;
            return SPAMM_OK;
        }
    }
    double* C = nullptr;
    CKA(dev_alloc(&C, (size_t)n * n * sizeof(double)));
    int best = 64;
    double best_s = 1e300;
    const int cands[3] = {32, 64, 128};
    for (int nb : cands) {
        if ((n + nb - 1) / nb > 1024) continue;
        spamm_opts t = o;
        t.leaf = nb;
        t.profile = 0;
        t.residual = 0;
        int e = multiply_core(S, S, C, n, tau, t, nullptr);  // first call: plan allocation, caches warm
        if (e == SPAMM_OK) {
            const auto t0 = std::chrono::steady_clock::now();
            e = multiply_core(S, S, C, n, tau, t, nullptr);
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (e == SPAMM_OK && dt < best_s) {
                best_s = dt;
                best = nb;
            }
        }
        if (e) {
            cudaFree(C);
            return e;
        }
    }
    cudaFree(C);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    *leaf = best;
    return SPAMM_OK;
}

// opts with leaf 0 resolved by the autotuner on the call's own input.
static int with_leaf(const double* S, int n, double tau, const spamm_opts& o, spamm_opts* out) {
    *out = o;
    if (o.leaf) return SPAMM_OK;
    return autotune_leaf_impl(S, n, tau, o, &out->leaf);
}

static int multiply_impl(const double* A, const double* B, double* C, int n, double tau, const spamm_opts& o_in,
                         spamm_stats* stats) {
    spamm_opts o;
    const int e = with_leaf(A, n, tau, o_in, &o);
    return e ? e : multiply_core(A, B, C, n, tau, o, stats);
}

static int residual_impl(Plan* p, const double* dS, const double* dZ, double* out, cudaStream_t st) {
    const Geometry& g = p->g;
    launch_pack(dS, g.n, g, nullptr, nullptr, p->buf[3], st);
    launch_pack(dZ, g.n, g, nullptr, nullptr, p->buf[4], st);
    launch_gemm_f64(g, p->buf[4].t, p->buf[3].t, p->buf[5].t, p->buf[4].tree, p->buf[3].tree, p->buf[5].tree,
                    nullptr, nullptr, nullptr, nullptr, 1, EPI_PLAIN, nullptr, nullptr, st);
    launch_gemm_f64(g, p->buf[5].t, p->buf[4].t, p->buf[3].t, p->buf[5].tree, p->buf[4].tree, p->buf[3].tree,
                    nullptr, nullptr, nullptr, nullptr, 1, EPI_PLAIN, nullptr, nullptr, st);
    launch_resid_norm(p->buf[3].t, g, p->partial, p->scal + 5, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, p->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
    return SPAMM_OK;
}

// The buffers of one solve: Y, Z and their successors (swapped every iteration) and T.  The single channel
// keeps s packed (Sb), writes W = s Z into Yb (= Y2, not swapped) and Z^T into Ztb.
struct SolveBufs {
    TileMat Yb, Zb, Tb, Y2, Z2, Sb, Ztb;
};

// a1-a2: flags and histories cleared, Gershgorin bound (plus the Tikhonov shift of Sec. 6) and scaling,
// X0 = Y0 = S / c packed with leaf norms, T0 = h[X0], Z0 = I (and their slices on the tensor-core path).
// tau_min is the smallest threshold of the products that read them (tau_s or tau): their slices are cut
// only for tiles those products can keep.
static int enqueue_prologue(Plan* p, const double* dS, int n, const spamm_opts& o, cudaStream_t st, SolveBufs* sb,
                            double tau_min) {
    const Geometry& g = p->g;
    CK(cudaMemsetAsync(p->flags, 0, kFlagInts * sizeof(int), st));
    CK(cudaMemsetAsync(p->task_ctr, 0, (3 * (size_t)p->maxit_cap + 4) * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(p->t_hist, 0, (size_t)p->maxit_cap * sizeof(double), st));
    if (p->lens_bins > 0)
        CK(cudaMemsetAsync(p->lens, 0, (size_t)p->maxit_cap * 9 * p->lens_bins * sizeof(unsigned long long), st));

    double* c0 = p->scal + 0;
    double* mu = p->scal + 1;
    double* c = p->scal + 2;
    double* sqc = p->scal + 3;
    double* rc = p->scal + 6;
    double* rsqc = p->scal + 7;
    // Z0 = I does not depend on S: on the tensor-core path its pass (identity, quadtree, maxima, slices) runs
    // on a side stream beside the scaling and packing of S, and X0's maxima and slices run on another one
    // beside the map.  A profiled call keeps everything on one stream.
    const bool side = p->emu && !p->profile;
    cudaStream_t zs = side ? p->pro_st[1] : st;
    cudaStream_t xs = side ? p->pro_st[0] : st;
    if (o.channel == SPAMM_CHANNEL_SINGLE)
        *sb = SolveBufs{p->buf[3], p->buf[1], p->buf[2], p->buf[3], p->buf[4], p->buf[0], p->buf[5]};
    else
        *sb = SolveBufs{p->buf[0], p->buf[1], p->buf[2], p->buf[3], p->buf[4], TileMat(), TileMat()};
    if (side) {
        cudaEventRecord(p->ev_norm[1], st);
        cudaStreamWaitEvent(zs, p->ev_norm[1], 0);
    }
    launch_identity(g, sb->Zb, zs);
    launch_tree(g, sb->Zb.tree, nullptr, zs);
    if (p->emu) prepare_emu(p, sb->Zb, zs, tau_min);

    const double* mu_ptr = nullptr;
    if (o.mu_rel > 0.0) {
        launch_gershgorin(dS, n, nullptr, p->rowsum, c0, st);
        launch_scale_mu(c0, o.mu_rel, mu, st);
        mu_ptr = mu;
    }
    launch_gershgorin(dS, n, mu_ptr, p->rowsum, c, st);
    launch_scale_consts(c, sqc, rc, rsqc, st);

    // X0 = s in buf 0: Y0 of the dual channel, the constant s of the single channel
    const TileMat X0 = p->buf[0];
    // the tensor-core path's tile norms are FP32 sums (they only steer its culls)
    launch_pack(dS, n, g, mu_ptr, rc, X0, st, p->emu);
    launch_tree(g, X0.tree, nullptr, st);
    if (side) {
        cudaEventRecord(p->ev_norm[0], st);
        cudaStreamWaitEvent(xs, p->ev_norm[0], 0);
    }
    if (p->emu) prepare_emu(p, X0, xs, tau_min);
    if (o.map == SPAMM_MAP_SCALED) launch_trace_parts(X0.t, g, p->trace_part, st);
    // on the tensor-core path the map also takes T0's row and column maxima
    if (p->emu) cudaMemsetAsync(sb->Tb.rmax, 0, 2 * (size_t)g.m * g.nb * sizeof(unsigned long long), st);
    launch_map(X0.t, X0.tree, sb->Tb, g, o.map, p->trace_part, p->emu, nullptr, st, p->emu);
    launch_tree(g, sb->Tb.tree, nullptr, st);
    if (p->emu) slice_emu(p, sb->Tb, st, tau_min);
    // the first culls read Z0's quadtree (its slicing event follows the tree on the same stream)
    if (side) cudaStreamWaitEvent(st, sb->Zb.sliced, 0);
    if (o.channel == SPAMM_CHANNEL_SINGLE) {
        // W = s Z0 = s: the Y output of a solve with no iteration
        CK(cudaMemcpyAsync(sb->Yb.t, X0.t, g.elems() * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(sb->Yb.tree, X0.tree, (size_t)g.tree_size * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaGetLastError());
    return SPAMM_OK;
}

// One iteration (a3-a6).  Its index k lives on the device (the iteration counter flags[1], advanced by the
// X product's tree pass together with t_k), so the same launches serve every iteration of a loop; once the
// stop flag is set (|t_k| <= tol_t, or maxit steps) every kernel returns at once.  cond (may be null) is the
// graph conditional that the stopping tree pass clears.
static int enqueue_iteration(Plan* p, SolveBufs& sb, double tau, double tau_s, int maxit, const spamm_opts& o,
                             cudaStream_t st, const cudaGraphConditionalHandle* cond) {
    const Geometry& g = p->g;
    TreeExtra tk;
    tk.trace_part = p->trace_part;
    tk.n = g.n;
    tk.maxit = maxit;
    tk.tol_t = o.tol_t;
    tk.t_hist = p->t_hist;
    tk.done = p->flags;
    tk.iters = p->flags + 1;
    if (cond) {
        tk.cond = *cond;
        tk.has_cond = 1;
    }
    unsigned long long* ctr = p->task_ctr;  // + 3 k on the device
    const EpiMode xmode = o.map == SPAMM_MAP_NS ? EPI_NS_X : EPI_X;
    if (o.channel == SPAMM_CHANNEL_SINGLE) {
        // Eq. (single): Z <- Z (x) T, then Z^T (tile transpose, its quadtree and slices) on the side branch
        // beside W = s (x)_{tau_s} Z (the sensitive product, as in the paper's single-instance volumes), then
        // X = Z^T (x) W with T = h[X] and t_k
        product(p, sb.Zb, sb.Tb, sb.Z2, tau, EPI_PLAIN, ctr + 0, st);  // Z <- Z (x)_tau T
        std::swap(sb.Zb, sb.Z2);
        cudaStream_t zs = p->profile ? st : p->side;
        if (zs != st) {
            CK(cudaEventRecord(p->ev_fork, st));
            CK(cudaStreamWaitEvent(zs, p->ev_fork, 0));
        }
        TileMat Zt = sb.Ztb;  // its row maxima are Z's column maxima and vice versa
        Zt.rmax = sb.Zb.cmax;
        Zt.cmax = sb.Zb.rmax;
        launch_transpose(sb.Zb, Zt, g, p->flags, zs);
        launch_tree(g, Zt.tree, p->flags, zs);
        if (p->emu) {
            launch_slice(Zt.t, Zt.tree, nullptr, Zt.rmax, Zt.cmax, Zt.sliceA, Zt.sliceB, g, nullptr, nullptr,
                         p->flags, zs);
            mark_sliced(p, Zt, zs);
        }
        product(p, sb.Sb, sb.Zb, sb.Yb, tau_s, EPI_PLAIN, ctr + 1, st);  // W <- s (x)_{tau_s} Z
        if (zs != st) {
            CK(cudaEventRecord(p->ev_join, zs));
            CK(cudaStreamWaitEvent(st, p->ev_join, 0));
        }
        product(p, Zt, sb.Yb, sb.Tb, tau, xmode, ctr + 2, st, &tk, 0, o.map);  // X <- Z^T (x)_tau W, T = h[X]
        CK(cudaGetLastError());
        return SPAMM_OK;
    }
    // the Y and Z updates are independent: the Z update runs on the side branch (a profiled call keeps them
    // in order, so that each leaf-product timing is that kernel's own)
    cudaStream_t zs = p->profile ? st : p->side;
    if (zs != st) {
        CK(cudaEventRecord(p->ev_fork, st));
        CK(cudaStreamWaitEvent(zs, p->ev_fork, 0));
    }
    if (o.order == SPAMM_ORDER_PAPER) {
        product(p, sb.Tb, sb.Yb, sb.Y2, tau_s, EPI_PLAIN, ctr + 0, st);           // Y <- T (x)_{tau_s} Y
        product(p, sb.Zb, sb.Tb, sb.Z2, tau, EPI_PLAIN, ctr + 1, zs, nullptr, 1);  // Z <- Z (x)_tau T
    } else {
        product(p, sb.Yb, sb.Tb, sb.Y2, tau_s, EPI_PLAIN, ctr + 0, st);           // Y <- Y (x)_{tau_s} T
        product(p, sb.Tb, sb.Zb, sb.Z2, tau, EPI_PLAIN, ctr + 1, zs, nullptr, 1);  // Z <- T (x)_tau Z
    }
    if (zs != st) {
        CK(cudaEventRecord(p->ev_join, zs));
        CK(cudaStreamWaitEvent(st, p->ev_join, 0));
    }
    // alpha = 1: T = h[X] fused into the X product's epilogue; the damped map needs tr X first
    std::swap(sb.Yb, sb.Y2);
    std::swap(sb.Zb, sb.Z2);
    if (o.order == SPAMM_ORDER_PAPER)
        product(p, sb.Yb, sb.Zb, sb.Tb, tau, xmode, ctr + 2, st, &tk, 0, o.map);  // X <- Y (x)_tau Z, T = h[X]
    else
        product(p, sb.Zb, sb.Yb, sb.Tb, tau, xmode, ctr + 2, st, &tk, 0, o.map);  // X <- Z (x)_tau Y, T = h[X]
    CK(cudaGetLastError());
    return SPAMM_OK;
}

// a7: unscale and unpack.  The iterates alternate between two buffers; `swaps` is the number of iterations
// enqueued since sb was set up, and the unpack picks the buffer of the last iteration that ran.
static int enqueue_epilogue(Plan* p, const SolveBufs& sb, double* dY, double* dZ, int swaps, cudaStream_t st) {
    const Geometry& g = p->g;
    const double* sqc = p->scal + 3;
    const double* rsqc = p->scal + 7;
    join_slicing(p, st);
    launch_unpack(sb.Yb.t, sb.Yb.tree, g, dY, sqc, st, sb.Y2.t, sb.Y2.tree, p->flags + 1, swaps);
    launch_unpack(sb.Zb.t, sb.Zb.tree, g, dZ, rsqc, st, sb.Z2.t, sb.Z2.tree, p->flags + 1, swaps);
    CK(cudaGetLastError());
    return SPAMM_OK;
}

// The whole solve on st, one launch sequence per iteration.  Nothing here synchronises unless host_poll is
// set with tol_t > 0: then the host reads the stop flag after every iteration and stops enqueueing.
static int enqueue_solve(Plan* p, const double* dS, double* dY, double* dZ, int n, double tau, double tau_s,
                         int maxit, const spamm_opts& o, cudaStream_t st, bool host_poll) {
    SolveBufs sb;
    int e = enqueue_prologue(p, dS, n, o, st, &sb, std::min(tau, tau_s));
    if (e) return e;
    int swaps = 0;
    for (int k = 0; k < maxit; ++k) {
        if ((e = enqueue_iteration(p, sb, tau, tau_s, maxit, o, st, nullptr))) return e;
        swaps = k + 1;
        if (host_poll && o.tol_t > 0.0) {
            int done = 0;
            CK(cudaMemcpyAsync(&done, p->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (done) break;
        }
    }
    return enqueue_epilogue(p, sb, dY, dZ, swaps, st);
}

// The solve captured with its iteration as a WHILE conditional node: the body holds two iterations (so the
// alternating buffers are back in place after it) and runs until the stopping tree pass clears the
// condition.  Only the iterations that run are launched.  Called while gstream is capturing.
static int enqueue_solve_loop(Plan* p, const double* dS, double* dY, double* dZ, int n, double tau, double tau_s,
                              int maxit, const spamm_opts& o, cudaStream_t st) {
    SolveBufs sb;
    int e = enqueue_prologue(p, dS, n, o, st, &sb, std::min(tau, tau_s));
    if (e) return e;
    join_slicing(p, st);  // the body waits on nothing recorded outside it
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, &edata, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return SPAMM_ERR_CUDA;
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, graph, maxit > 0 ? 1u : 0u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, graph, deps, edata, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaStreamBeginCaptureToGraph(p->bstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const long long l0 = t_launches;
    int eb = enqueue_iteration(p, sb, tau, tau_s, maxit, o, p->bstream, &cond);
    if (!eb) eb = enqueue_iteration(p, sb, tau, tau_s, maxit, o, p->bstream, &cond);
    if (!eb) join_slicing(p, p->bstream);
    p->graph_body_kernels = t_launches - l0;
    cudaGraph_t bg = nullptr;
    const cudaError_t be = cudaStreamEndCapture(p->bstream, &bg);
    if (eb) return eb;
    CK(be);
    return enqueue_epilogue(p, sb, dY, dZ, 0, st);
}

// SPAMM_NO_LOOP_GRAPH=1 captures one launch sequence per iteration instead of the conditional loop.
static bool loop_graphs_enabled() {
    static const bool on = [] {
        const char* v = getenv("SPAMM_NO_LOOP_GRAPH");
        return !(v && v[0] && v[0] != '0');
    }();
    return on;
}

static bool graphs_enabled() {
    static const bool on = [] {
        const char* v = getenv("SPAMM_NO_GRAPH");
        return !(v && v[0] && v[0] != '0');
    }();
    return on;
}

// Replay (or capture, then replay) the whole solve as one CUDA graph on the plan's own stream, ordered after
// and before `st`.  The iteration is a WHILE conditional node (only the iterations that run are launched);
// a profiled solve, whose event records cannot sit in a conditional body, and a device or driver that
// rejects the conditional graph get one launch sequence per iteration instead.
static std::atomic<bool> g_loop_graph_ok{true};

static int capture_solve(Plan* p, const double* dS, double* dY, double* dZ, int n, double tau, double tau_s,
                         int maxit, const spamm_opts& o, bool loop, cudaGraphExec_t* exec) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal));
    const int e = loop ? enqueue_solve_loop(p, dS, dY, dZ, n, tau, tau_s, maxit, o, p->gstream)
                       : enqueue_solve(p, dS, dY, dZ, n, tau, tau_s, maxit, o, p->gstream, false);
    const cudaError_t ce = cudaStreamEndCapture(p->gstream, &graph);
    if (e || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (!e) {
            g_last_error = std::string("graph capture: ") + cudaGetErrorString(ce);
            return SPAMM_ERR_CUDA;
        }
        return e;
    }
    const cudaError_t ie = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        g_last_error = std::string("graph instantiate: ") + cudaGetErrorString(ie);
        return SPAMM_ERR_CUDA;
    }
    return SPAMM_OK;
}

static int solve_graph(Plan* p, const double* dS, double* dY, double* dZ, int n, double tau, double tau_s, int maxit,
                       const spamm_opts& o, cudaStream_t st) {
    if (!p->gstream) {
        CK(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&p->bstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
    }
    const GraphKey key{dS, dY, dZ, n, o.leaf, o.precision, o.order, maxit, o.profile ? 1 : 0, o.map, o.channel,
                       p->lens_bins, tau, tau_s, o.mu_rel, o.tol_t};
    CK(cudaEventRecord(p->ev_in, st));
    CK(cudaStreamWaitEvent(p->gstream, p->ev_in, 0));
    if (!p->gexec || !(p->gkey == key)) {
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        const long long l0 = t_launches;
        const int ev0 = p->ev_used;
        const bool loop = g_loop_graph_ok && !p->profile && loop_graphs_enabled();
        int e = capture_solve(p, dS, dY, dZ, n, tau, tau_s, maxit, o, loop, &p->gexec);
        if (e == SPAMM_ERR_CUDA && loop) {
            // conditional graphs unavailable here: fall back to one launch sequence per iteration
            cudaGetLastError();
            g_loop_graph_ok = false;
            p->gexec = nullptr;
            p->sliced_mask = 0;
            p->ev_used = ev0;
            p->gemm_launches = 0;
            g_launches.fetch_sub(t_launches - l0);
            t_launches = l0;
            e = capture_solve(p, dS, dY, dZ, n, tau, tau_s, maxit, o, false, &p->gexec);
        }
        if (e) return e;
        p->gkey = key;
        p->graph_loop = loop && g_loop_graph_ok;
        p->graph_kernels = t_launches - l0;
        g_launches.fetch_sub(p->graph_kernels);  // counted again when the graph runs
        t_launches = l0;
        if (p->graph_loop) p->graph_kernels -= p->graph_body_kernels;
        p->graph_events = p->ev_used;
        p->graph_gemm = p->gemm_launches;
    }
    // the profiling events and launch counts of this call are those recorded in the graph
    p->ev_used = p->graph_events;
    p->gemm_launches = p->graph_gemm;
    CK(cudaGraphLaunch(p->gexec, p->gstream));
    // a loop graph launches its body once per two iterations run: counted after the call from the iteration
    // count (graph_kernels then covers the prologue, one body and the epilogue)
    if (!p->graph_loop) note_launch((int)p->graph_kernels);
    CK(cudaEventRecord(p->ev_out, p->gstream));
    CK(cudaStreamWaitEvent(st, p->ev_out, 0));
    return SPAMM_OK;
}

static int sqrt_impl(const double* S, int n, double tau, int maxit, double* Y, double* Z, const spamm_opts& o_in,
                     spamm_stats* stats);

// ---- schedule autotuner (opts.schedule = SPAMM_SCHED_AUTO) -----------------
// Times one solve of the call's own input with each schedule (after one untimed solve that captures its
// graph) and keeps the faster, per device, size, arithmetic, leaf and decade of tau.
static std::mutex g_sched_mu;
static std::map<std::tuple<int, int, int, int, int>, int> g_sched;

static int autotune_schedule(const double* S, int n, double tau, int maxit, double* Y, double* Z,
                             const spamm_opts& o, int* sched) {
    *sched = SPAMM_SCHED_BRANCHES;
    spamm_opts t = o;
    t.schedule = SPAMM_SCHED_STAGES;
    if (!batch_engine_covers(t) || maxit <= 0) return SPAMM_OK;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, n, o.precision, o.leaf, tau_decade(tau));
    {
        std::lock_guard<std::mutex> lk(g_sched_mu);
        auto it = g_sched.find(key);
        if (it != g_sched.end()) {
            *sched = it->second;
            return SPAMM_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)o.stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // one untimed solve per schedule captures its graph; then three timed solves each, alternating, and the
    // faster minimum wins (schedules within a percent of each other are told apart by the minimum, not by
    // one sample)
    const int kScheds[2] = {SPAMM_SCHED_BRANCHES, SPAMM_SCHED_STAGES};
    float best[2] = {3.4e38f, 3.4e38f};
    bool applies[2] = {true, true};
    int err = SPAMM_OK;
    for (int q = 0; q < 2 && !err; ++q) {
        t.schedule = kScheds[q];
        spamm_stats ss;
        std::memset(&ss, 0, sizeof(ss));
        const int e = sqrt_impl(S, n, tau, maxit, Y, Z, t, &ss);
        if (e && e != SPAMM_ERR_DIVERGED && e != SPAMM_ERR_NOTCONVERGED) err = e;
        applies[q] = ss.schedule == kScheds[q];  // the schedule did not apply to this call
    }
    for (int rep = 0; rep < 3 && !err; ++rep)
        for (int q = 0; q < 2 && !err; ++q) {
            if (!applies[q]) continue;
            t.schedule = kScheds[q];
            cudaEventRecord(e0, st);
            const int e = sqrt_impl(S, n, tau, maxit, Y, Z, t, nullptr);
            cudaEventRecord(e1, st);
            if (e && e != SPAMM_ERR_DIVERGED && e != SPAMM_ERR_NOTCONVERGED) {
                err = e;
                break;
            }
            float ms = 0.f;
            if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                best[q] = std::min(best[q], ms);
            cudaGetLastError();
        }
    const int choice = best[1] < best[0] ? SPAMM_SCHED_STAGES : SPAMM_SCHED_BRANCHES;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err) return err;
    g_last_error.clear();
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched[key] = choice;
    *sched = choice;
    return SPAMM_OK;
}

static int sqrt_impl(const double* S, int n, double tau, int maxit, double* Y, double* Z, const spamm_opts& o_in,
                     spamm_stats* stats) {
    spamm_opts o;
    {
        const int e = with_leaf(S, n, tau, o_in, &o);
        if (e) return e;
    }
    if (o.schedule == SPAMM_SCHED_AUTO) {
        int sc = SPAMM_SCHED_BRANCHES;
        const int e = autotune_schedule(S, n, tau, maxit, Y, Z, o, &sc);
        if (e) return e;
        o.schedule = sc;
    }
    if (o.schedule == SPAMM_SCHED_STAGES) {
        const int e = stage_solve(S, n, tau, maxit, Y, Z, o, stats);
        if (e != SPAMM_ERR_UNSUPPORTED) {
            if (stats) stats->schedule = SPAMM_SCHED_STAGES;
            return e;
        }
        g_last_error.clear();  // not covered: the branch schedule serves the call
    }
    if (stats) stats->schedule = SPAMM_SCHED_BRANCHES;
    cudaStream_t st = (cudaStream_t)o.stream;
    const double tau_s = o.tau_s < 0.0 ? 0.01 * tau : o.tau_s;
    init_device_attributes();
    PlanGuard pg;
    int e = g_pool.acquire(n, o.leaf, &pg.p);
    if (e) return e;
    Plan* p = pg.p;
    const Geometry& g = p->g;
    if ((e = ensure_hist(p, maxit > 0 ? maxit : 1))) return e;
    const double* dS;
    double *dY, *dZ;
    if ((e = stage_in(p, 0, S, st, &dS, false))) return e;
    if ((e = out_target(p, 1, Y, &dY))) return e;
    if ((e = out_target(p, 2, Z, &dZ))) return e;
    begin_call(p, o.profile != 0, o.precision == SPAMM_EMU64);
    if (p->emu && (e = ensure_emu(p))) return e;
    if (stats && stats->lens_hist && maxit > 0) {
        if (stats->lens_bins < 1 || stats->lens_bins > 4096) {
            g_last_error = "lens_bins must be 1 .. 4096";
            return SPAMM_ERR_ARG;
        }
        if ((e = ensure_lens(p, stats->lens_bins))) return e;
        p->lens_bins = stats->lens_bins;
    }

    const int it_host = maxit;  // at most; the device counts the iterations that ran
    const bool graph = graphs_enabled();
    if (graph) {
        if ((e = solve_graph(p, dS, dY, dZ, n, tau, tau_s, maxit, o, st))) return e;
    } else {
        if ((e = enqueue_solve(p, dS, dY, dZ, n, tau, tau_s, maxit, o, st, true))) return e;
    }
    double* c = p->scal + 2;
    double resid = -1.0;
    if (o.residual) {
        if ((e = residual_impl(p, dS, dZ, &resid, st))) return e;
    }
    if ((e = stage_out(p, 1, Y, dY, st))) return e;
    if ((e = stage_out(p, 2, Z, dZ, st))) return e;

    std::vector<double> th((size_t)(it_host > 0 ? it_host : 1), 0.0);
    std::vector<unsigned long long> kc(3 * (size_t)(it_host > 0 ? it_host : 1), 0ull);
    double c_host = 0.0;
    int flags_h[kFlagInts] = {};
    if (it_host > 0) {
        CK(cudaMemcpyAsync(th.data(), p->t_hist, it_host * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(kc.data(), p->task_ctr, 3 * (size_t)it_host * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, st));
    }
    CK(cudaMemcpyAsync(&c_host, c, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(flags_h, p->flags, kFlagInts * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flags_h[2]) {
        g_last_error = "a bounded device-side wait of the tensor-core kernel expired";
        return SPAMM_ERR_TIMEOUT;
    }

    // iterations run on the device (fewer than enqueued once |t_k| <= tol_t)
    const int iters = std::min(it_host, flags_h[1]);
    if (graph && p->graph_loop) note_launch((int)(p->graph_kernels + (long long)((iters + 1) / 2) * p->graph_body_kernels));
    long long total = 0;
    for (int q = 0; q < 3 * iters; ++q) total += (long long)kc[q];
    const double t_final = iters > 0 ? th[iters - 1] : 0.0;
    if (stats) {
        stats->iters = iters;
        stats->t_final = t_final;
        stats->resid_F = resid;
        stats->scale_c = c_host;
        stats->tasks_total = total;
        stats->tasks_dense = 3ll * iters * (long long)g.m * g.m * g.m;
        stats->flops = 2.0 * (double)g.nb * g.nb * g.nb * (double)total;
        if (stats->t_hist)
            for (int q = 0; q < iters; ++q) stats->t_hist[q] = th[q];
        if (stats->task_hist)
            for (int q = 0; q < 3 * iters; ++q) stats->task_hist[q] = (long long)kc[q];
        if (p->lens_bins > 0 && iters > 0) {
            const size_t cnt = (size_t)iters * 9 * p->lens_bins;
            CK(cudaMemcpy(stats->lens_hist, p->lens, cnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        }
        profile_stats(p, stats);
        stats->gemm_launches = p->gemm_launches;
        unsigned long long units = 0;
        std::memcpy(&units, flags_h + 30, sizeof(units));
        stats->tensor_units = (long long)units;
    }
    for (int q = 0; q < iters; ++q)
        if (!std::isfinite(th[q]) || std::fabs(th[q]) >= 1.0) {
            g_last_error = "trace error left [0, 1): the iteration diverged";
            return SPAMM_ERR_DIVERGED;
        }
    // The trace error follows X = YZ, which stays near I even when culling has moved Y and Z off the
    // square roots of S.  With the residual computed, a solve whose trace error says converged
    // (|t_k| < 1e-8) while ||Z S Z - I||_F >= 1 has reached a wrong fixed point: Z is outside the region
    // ||I - Z S Z|| < 1 in which a further Newton-Schulz refinement is guaranteed to converge.  (A solve cut
    // short by maxit, with a large trace error, is not converged, not diverged.)
    if (o.residual && iters > 0 && std::fabs(t_final) < 1e-8 && !(resid < 1.0)) {
        g_last_error = "||Z S Z - I||_F >= 1: Z is no longer an approximate inverse square root of S";
        return SPAMM_ERR_DIVERGED;
    }
    if (o.tol_t > 0.0 && !(std::fabs(t_final) <= o.tol_t)) {
        g_last_error = "maxit reached before |t_k| <= tol_t";
        return SPAMM_ERR_NOTCONVERGED;
    }
    return SPAMM_OK;
}

static int check_common(int n, double tau, const spamm_opts& o) {
    if (n <= 0) {
        g_last_error = "n must be positive";
        return SPAMM_ERR_ARG;
    }
    if (!(tau >= 0.0) || std::isinf(tau)) {
        g_last_error = "tau must be finite and >= 0";
        return SPAMM_ERR_ARG;
    }
    if (o.leaf != 0 && !leaf_ok(o.leaf)) {
        g_last_error = "leaf must be 0 (autotune), 32, 64 or 128";
        return SPAMM_ERR_ARG;
    }
    if (o.precision != SPAMM_FP64 && o.precision != SPAMM_EMU64) {
        g_last_error = "unknown precision";
        return SPAMM_ERR_ARG;
    }
    if (o.order != SPAMM_ORDER_PAPER && o.order != SPAMM_ORDER_TRANSPOSED) {
        g_last_error = "unknown order";
        return SPAMM_ERR_ARG;
    }
    if (o.map != SPAMM_MAP_NS && o.map != SPAMM_MAP_SCALED) {
        g_last_error = "unknown map";
        return SPAMM_ERR_ARG;
    }
    if (o.channel != SPAMM_CHANNEL_DUAL && o.channel != SPAMM_CHANNEL_SINGLE) {
        g_last_error = "unknown channel";
        return SPAMM_ERR_ARG;
    }
    if (o.schedule != SPAMM_SCHED_BRANCHES && o.schedule != SPAMM_SCHED_STAGES && o.schedule != SPAMM_SCHED_AUTO) {
        g_last_error = "unknown schedule";
        return SPAMM_ERR_ARG;
    }
    if (o.channel == SPAMM_CHANNEL_SINGLE && o.order != SPAMM_ORDER_PAPER) {
        g_last_error = "the single channel is defined in the paper order only";
        return SPAMM_ERR_ARG;
    }
    if (std::isnan(o.tau_s) || std::isnan(o.mu_rel) || o.mu_rel < 0.0 || std::isnan(o.tol_t) || o.tol_t < 0.0) {
        g_last_error = "tau_s, mu_rel, tol_t must be numbers (mu_rel, tol_t >= 0)";
        return SPAMM_ERR_ARG;
    }
    const int leaf = o.leaf ? o.leaf : (o.precision == SPAMM_EMU64 ? 64 : 128);
    const long m = (n + leaf - 1) / leaf;
    if (o.precision == SPAMM_EMU64 && (leaf != 64 || m > 512)) {
        g_last_error = "SPAMM_EMU64 needs leaf 64 and n <= 32768";
        return SPAMM_ERR_UNSUPPORTED;
    }
    if (m > 1024) {
        g_last_error = "more than 1024 leaf tiles per side";
        return SPAMM_ERR_UNSUPPORTED;
    }
    return SPAMM_OK;
}

// Device scratch of one call, freed when the call returns.
struct CallScratch {
    std::vector<void*> ptrs;
    ~CallScratch() {
        for (void* q : ptrs) cudaFree(q);
    }
    template <typename T>
    cudaError_t get(T** out, size_t bytes) {
        void* q = nullptr;
        const cudaError_t e = dev_alloc(&q, bytes);
        if (e == cudaSuccess) ptrs.push_back(q);
        *out = static_cast<T*>(q);
        return e;
    }
};

// Sec. 6 product representation: slice z_0 of S + mu_0 c0 I, then per level the residual
// Z^T (S + mu_l c0 I) Z, its inverse square root z_l and Z <- Z (x) z_l (see spamm.h).
static int invsqrt_product_impl(const double* S, int n, int levels, const double* mu, double tau0, double tau1,
                                int maxit, double* Z, int* iters, const spamm_opts& o_in) {
    cudaStream_t st = (cudaStream_t)o_in.stream;
    init_device_attributes();
    const size_t bytes = (size_t)n * n * sizeof(double);
    CallScratch cs;
    double *dZa, *dW, *dR, *dz, *dY, *dT, *rowsum, *c0;
    CKA(cs.get(&dZa, bytes));
    CKA(cs.get(&dW, bytes));
    CKA(cs.get(&dR, bytes));
    CKA(cs.get(&dz, bytes));
    CKA(cs.get(&dY, bytes));
    CKA(cs.get(&dT, bytes));
    CKA(cs.get(&rowsum, (size_t)n * sizeof(double)));
    CKA(cs.get(&c0, sizeof(double)));
    void* vS = nullptr;
    int ev = current_view(S, &vS);
    if (ev) return ev;
    void* vZ = nullptr;
    if ((ev = current_view(Z, &vZ))) return ev;
    const double* dS = static_cast<const double*>(vS);
    if (!dS) {
        double* st_S;
        CKA(cs.get(&st_S, bytes));
        CK(cudaMemcpyAsync(st_S, S, bytes, cudaMemcpyHostToDevice, st));
        dS = st_S;
    }
    launch_gershgorin(dS, n, nullptr, rowsum, c0, st);
    spamm_opts o = o_in;
    o.residual = 0;
    o.profile = 0;
    int status = SPAMM_OK;
    auto solve = [&](const double* M, double mu_rel, double* out, int level) -> int {
        spamm_opts os = o;
        os.mu_rel = mu_rel;
        spamm_stats sst;
        std::memset(&sst, 0, sizeof(sst));
        const int e = sqrt_impl(M, n, tau0, maxit, dY, out, os, &sst);
        if (e && e != SPAMM_ERR_DIVERGED && e != SPAMM_ERR_NOTCONVERGED) return e;
        if (e && !status) status = e;
        if (iters) iters[level] = sst.iters;
        return SPAMM_OK;
    };
    int e = solve(dS, mu[0], dZa, 0);
    if (e) return e;
    for (int l = 1; l < levels; ++l) {
        launch_shift_copy(dS, dT, n, mu[l], c0, st);                   // S + mu_l c0 I
        if ((e = multiply_impl(dT, dZa, dW, n, tau1, o, nullptr))) return e;  // W = S_mu (x) Z
        launch_transpose_rm(dZa, dT, n, st);                           // Z^T
        if ((e = multiply_impl(dT, dW, dR, n, tau1, o, nullptr))) return e;   // R = Z^T (x) W
        if ((e = solve(dR, 0.0, dz, l))) return e;                     // z_l = R^{-1/2}
        if ((e = multiply_impl(dZa, dz, dW, n, tau1, o, nullptr))) return e;  // Z (x) z_l
        std::swap(dZa, dW);
    }
    CK(cudaMemcpyAsync(Z, dZa, bytes, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return status;
}

// Internal entry points used by the request server (spamm_server.cu).
int run_sqrt(const double* S, int n, double tau, int maxit, double* Y, double* Z, const spamm_opts& o,
             spamm_stats* stats) {
    try {
        return sqrt_impl(S, n, tau, maxit, Y, Z, o, stats);
    } catch (...) {
        g_last_error = "internal exception";
        return SPAMM_ERR_CUDA;
    }
}
int check_args(int n, double tau, const spamm_opts& o) { return check_common(n, tau, o); }
spamm_opts resolved(const spamm_opts* o) { return resolve_opts(o); }
void trim_plans(size_t keep_bytes) { g_pool.trim(keep_bytes); }
const char* last_error_message() { return g_last_error.c_str(); }

}  // namespace spamm

using namespace spamm;

extern "C" {

void spamm_opts_init(spamm_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->leaf = 64;
    o->precision = SPAMM_FP64;
    o->tau_s = -1.0;
    o->mu_rel = 0.0;
    o->tol_t = 0.0;
    o->order = SPAMM_ORDER_PAPER;
    o->residual = 0;
    o->stream = nullptr;
    o->map = SPAMM_MAP_NS;
    o->channel = SPAMM_CHANNEL_DUAL;
    o->schedule = SPAMM_SCHED_BRANCHES;
}

int spamm_autotune_leaf(const double* S, int n, double tau, const spamm_opts* opts, int* leaf) {
    try {
        g_last_error.clear();
        spamm_opts o = resolve_opts(opts);
        o.leaf = 0;
        int e = check_common(n, tau, o);
        if (e) return e;
        if (!S || !leaf) {
            g_last_error = "null pointer";
            return SPAMM_ERR_ARG;
        }
        return autotune_leaf_impl(S, n, tau, o, leaf);
    } catch (...) {
        g_last_error = "internal exception";
        return SPAMM_ERR_CUDA;
    }
}

int spamm_test_expire_next_wait(long long polls) {
    if (polls < 0) {
        g_last_error = "polls must be >= 0";
        return SPAMM_ERR_ARG;
    }
    t_stall_next = polls;
    return SPAMM_OK;
}

int spamm_test_emu_alternate(int mode) {
    if (mode < -1 || mode > 1) {
        g_last_error = "mode must be -1, 0 or 1";
        return SPAMM_ERR_ARG;
    }
    set_emu_alternate(mode);
    return SPAMM_OK;
}

int spamm_multiply(const double* A, const double* B, double* C, int n, double tau, const spamm_opts* opts,
                   spamm_stats* stats) {
    try {
        g_last_error.clear();
        spamm_opts o = resolve_opts(opts);
        int e = check_common(n, tau, o);
        if (e) return e;
        if (!A || !B || !C) {
            g_last_error = "null matrix pointer";
            return SPAMM_ERR_ARG;
        }
        return multiply_impl(A, B, C, n, tau, o, stats);
    } catch (...) {
        g_last_error = "internal exception";
        return SPAMM_ERR_CUDA;
    }
}

int spamm_sqrt_invsqrt(const double* S, int n, double tau, int maxit, double* Y, double* Z, const spamm_opts* opts,
                       spamm_stats* stats) {
    try {
        g_last_error.clear();
        spamm_opts o = resolve_opts(opts);
        int e = check_common(n, tau, o);
        if (e) return e;
        if (!S || !Y || !Z || maxit < 0) {
            g_last_error = "null matrix pointer or maxit < 0";
            return SPAMM_ERR_ARG;
        }
        return sqrt_impl(S, n, tau, maxit, Y, Z, o, stats);
    } catch (...) {
        g_last_error = "internal exception";
        return SPAMM_ERR_CUDA;
    }
}

int spamm_invsqrt_product(const double* S, int n, int levels, const double* mu, double tau0, double tau1, int maxit,
                          double* Z, int* iters, const spamm_opts* opts) {
    try {
        g_last_error.clear();
        spamm_opts o = resolve_opts(opts);
        int e = check_common(n, tau0, o);
        if (e) return e;
        if (!S || !Z || !mu || levels < 1 || maxit < 0 || !(tau1 >= 0.0) || std::isinf(tau1)) {
            g_last_error = "bad product-representation arguments";
            return SPAMM_ERR_ARG;
        }
        for (int l = 0; l < levels; ++l)
            if (!(mu[l] >= 0.0) || std::isinf(mu[l])) {
                g_last_error = "shifts must be finite and >= 0";
                return SPAMM_ERR_ARG;
            }
        return invsqrt_product_impl(S, n, levels, mu, tau0, tau1, maxit, Z, iters, o);
    } catch (...) {
        g_last_error = "internal exception";
        return SPAMM_ERR_CUDA;
    }
}

int spamm_sqrt_invsqrt_batched(int count, const double* const* S, const int* n, const double* tau, int maxit,
                               double* const* Y, double* const* Z, const spamm_opts* opts, spamm_stats* stats) {
    try {
        g_last_error.clear();
        if (count < 0 || (count > 0 && (!S || !n || !tau || !Y || !Z))) {
            g_last_error = "bad batch arguments";
            return SPAMM_ERR_ARG;
        }
        if (count == 0) return SPAMM_OK;
        spamm_opts base = resolve_opts(opts);
        for (int q = 0; q < count; ++q) {
            int e = check_common(n[q], tau[q], base);
            if (e) return e;
        }
        // one graph over the whole batch when the options allow it; otherwise every problem on its own
        {
            const int e = batched_solve(count, S, n, tau, maxit, Y, Z, base, stats);
            if (e != SPAMM_ERR_UNSUPPORTED) return e;
            g_last_error.clear();
        }
        int dev = 0;
        CK(cudaGetDevice(&dev));
        const int workers = count < 8 ? count : 8;
        std::vector<int> status(count, SPAMM_OK);
        std::vector<std::string> errs(count);
        std::atomic<int> next(0);
        auto work = [&]() {
            cudaSetDevice(dev);
            cudaStream_t st = nullptr;
            cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            spamm_opts o = base;
            o.stream = st;
            for (;;) {
                int q = next.fetch_add(1);
                if (q >= count) break;
                status[q] = sqrt_impl(S[q], n[q], tau[q], maxit, Y[q], Z[q], o, stats ? stats + q : nullptr);
                if (status[q]) errs[q] = g_last_error;
            }
            cudaStreamDestroy(st);
        };
        std::vector<std::thread> th;
        for (int w = 0; w < workers; ++w) th.emplace_back(work);
        for (auto& t : th) t.join();
        for (int q = 0; q < count; ++q)
            if (status[q]) {
                g_last_error = errs[q];
                return status[q];
            }
        return SPAMM_OK;
    } catch (...) {
        g_last_error = "internal exception";
        return SPAMM_ERR_CUDA;
    }
}

int spamm_norm_tree(const double* A, int n, int leaf, double* nu_leaf, double* root, void* stream) {
    try {
        g_last_error.clear();
        spamm_opts o;
        spamm_opts_init(&o);
        o.leaf = leaf == 0 ? 64 : leaf;
        int e = check_common(n, 0.0, o);
        if (e) return e;
        if (!A || !nu_leaf || !root) {
            g_last_error = "null pointer";
            return SPAMM_ERR_ARG;
        }
        cudaStream_t st = (cudaStream_t)stream;
        PlanGuard pg;
        if ((e = g_pool.acquire(n, o.leaf, &pg.p))) return e;
        Plan* p = pg.p;
        const Geometry& g = p->g;
        const double* dA;
        if ((e = stage_in(p, 0, A, st, &dA))) return e;
        launch_pack(dA, n, g, nullptr, nullptr, p->buf[0], st);
        launch_tree(g, p->buf[0].tree, nullptr, st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(nu_leaf, p->buf[0].tree, (size_t)g.m * g.m * sizeof(double), cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(root, p->buf[0].tree + g.off[0], sizeof(double), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
        return SPAMM_OK;
    } catch (...) {
        g_last_error = "internal exception";
        return SPAMM_ERR_CUDA;
    }
}

int spamm_cull(const double* A, const double* B, int n, double tau, int leaf, int* counts, int* jlist, double* thr,
               long long* total, void* stream) {
    try {
        g_last_error.clear();
        spamm_opts o;
        spamm_opts_init(&o);
        o.leaf = leaf == 0 ? 64 : leaf;
        int e = check_common(n, tau, o);
        if (e) return e;
        if (!A || !B || !counts || !jlist) {
            g_last_error = "null pointer";
            return SPAMM_ERR_ARG;
        }
        cudaStream_t st = (cudaStream_t)stream;
        PlanGuard pg;
        if ((e = g_pool.acquire(n, o.leaf, &pg.p))) return e;
        Plan* p = pg.p;
        const Geometry& g = p->g;
        if ((e = ensure_hist(p, 1))) return e;
        const double *dA, *dB;
        if ((e = stage_in(p, 0, A, st, &dA))) return e;
        if ((e = stage_in(p, 1, B, st, &dB))) return e;
        CK(cudaMemsetAsync(p->task_ctr, 0, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(p->jlist, 0xff, (size_t)g.m * g.m * g.m * sizeof(int), st));
        launch_pack(dA, n, g, nullptr, nullptr, p->buf[0], st);
        launch_tree(g, p->buf[0].tree, nullptr, st);
        launch_pack(dB, n, g, nullptr, nullptr, p->buf[1], st);
        launch_tree(g, p->buf[1].tree, nullptr, st);
        const CullOut co{p->counts, p->jlist, nullptr, nullptr, nullptr, 0};
        launch_cull(g, p->buf[0].tree, p->buf[1].tree, tau, co, p->task_ctr, p->scal + 4, nullptr, st);
        CK(cudaGetLastError());
        unsigned long long tot = 0;
        double thr_h = 0.0;
        CK(cudaMemcpyAsync(counts, p->counts, (size_t)g.m * g.m * sizeof(int), cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(jlist, p->jlist, (size_t)g.m * g.m * g.m * sizeof(int), cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(&tot, p->task_ctr, sizeof(tot), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&thr_h, p->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (thr) *thr = thr_h;
        if (total) *total = (long long)tot;
        return SPAMM_OK;
    } catch (...) {
        g_last_error = "internal exception";
        return SPAMM_ERR_CUDA;
    }
}

const char* spamm_last_error(void) { return g_last_error.c_str(); }

const char* spamm_strerror(int s) {
    switch (s) {
        case SPAMM_OK: return "SPAMM_OK";
        case SPAMM_ERR_ARG: return "SPAMM_ERR_ARG";
        case SPAMM_ERR_NOMEM: return "SPAMM_ERR_NOMEM";
        case SPAMM_ERR_DIVERGED: return "SPAMM_ERR_DIVERGED";
        case SPAMM_ERR_NOTCONVERGED: return "SPAMM_ERR_NOTCONVERGED";
        case SPAMM_ERR_TIMEOUT: return "SPAMM_ERR_TIMEOUT";
        case SPAMM_ERR_ADMIT: return "SPAMM_ERR_ADMIT";
        case SPAMM_ERR_CUDA: return "SPAMM_ERR_CUDA";
        case SPAMM_ERR_UNSUPPORTED: return "SPAMM_ERR_UNSUPPORTED";
        case SPAMM_ERR_NOTFOUND: return "SPAMM_ERR_NOTFOUND";
        default: return "SPAMM_ERR_UNKNOWN";
    }
}

int spamm_release(void) {
    release_batches();
    g_pool.clear();
    return SPAMM_OK;
}

long long spamm_kernel_launches(void) { return g_launches.load(); }

const char* spamm_version(void) { return "spamm-gb300 0.1"; }

}  // extern "C"

// Batched square-root solves: many independent problems of mixed sizes advance together, one stage of the
// dual-channel iteration (Eq. (cannonical)) at a time.
//
// Per iteration a batch runs two stages: the y and z products of every live matrix (Y <- T Y, Z <- Z T; or
// the transposed order), then the x product of every live matrix (X <- Y Z with T = h[X] fused).  Each
// stage is one launch of each kernel over all of its products: the cull (one warp per output tile of every
// product), the leaf products (the persistent tensor-core kernel, or the FP64 kernel, drawing output tiles
// of all products from one cost-ordered list), the digit slicing of the outputs (beside the quadtree pass),
// and the quadtree pass, which for the x stage also takes every matrix's trace error and stop.  So the
// launches per iteration do not grow with the number of matrices.  The whole solve is captured once as a
// CUDA graph whose iteration is a WHILE conditional node (two iterations per body, so the alternating
// buffers are back in place after it); the body ends when every matrix has stopped.
//
// Every result is the one a single call gives: each output tile's arithmetic is the single path's, on
// the same operands in the same order, whatever other tiles the launch also holds; the setup and finish
// passes are the single path's own kernels, per matrix.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "spamm.h"
#include "spamm_internal.cuh"

namespace spamm {
namespace {

#define BK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            set_error_message((std::string(#call) + ": " + cudaGetErrorString(e_)).c_str());  \
            return e_ == cudaErrorMemoryAllocation ? SPAMM_ERR_NOMEM : SPAMM_ERR_CUDA;        \
        }                                                                                     \
    } while (0)

constexpr int kForks = 8;  // streams the per-matrix setup and finish passes are spread over

// Bump allocator over one device allocation (256-byte aligned pieces).
struct Arena {
    char* base = nullptr;
    size_t size = 0, used = 0;
    template <typename T>
    T* take(size_t count) {
        const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (used + bytes > size) return nullptr;
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};

// One matrix of a batch: its inputs and outputs and its device buffers (the single path's plan layout:
// buffers 0..4 are Y0 = X0, Z0, T, and the successors of Y and Z).
struct BatchMat {
    Geometry g;
    double tau = 0.0, tau_s = 0.0;
    const double* S = nullptr;
    double* Y = nullptr;
    double* Z = nullptr;
    TileMat buf[5];
    int* counts[2] = {nullptr, nullptr};
    int* jlist[2] = {nullptr, nullptr};
    double* trace_part = nullptr;
    double* scal = nullptr;  // c0, mu, c, sqrt c, -, -, 1/c, 1/sqrt c
    double* rowsum = nullptr;
};

// What a captured batch graph depends on.
struct BatchKey {
    int device = 0, count = 0, leaf = 0, precision = 0, order = 0, maxit = 0;
    double tau_s = 0.0, mu_rel = 0.0, tol_t = 0.0;
    std::vector<int> n;
    std::vector<double> tau;
    std::vector<const void*> ptrs;
    bool operator==(const BatchKey& o) const {
        return device == o.device && count == o.count && leaf == o.leaf && precision == o.precision &&
               order == o.order && maxit == o.maxit && tau_s == o.tau_s && mu_rel == o.mu_rel && tol_t == o.tol_t &&
               n == o.n && tau == o.tau && ptrs == o.ptrs;
    }
};

// Stage types: 0 the y and z products, 1 the x product.  Tables: [stage type][parity of the iteration].
struct Batch {
    BatchKey key;
    int device = 0, count = 0, leaf = 0, maxit = 0;
    bool emu = false;
    Arena arena;
    std::vector<BatchMat> mats;
    int* mflags = nullptr;                  // [count * 4]: stop, iterations run
    double* t_hist = nullptr;               // [count * maxit]
    unsigned long long* task_ctr = nullptr;  // [count * 3 * maxit]
    int* gflags = nullptr;  // [0] all stopped, [1] matrices stopped, [2] stage block counter, [3] device error,
                            // [4..7] leaf-product tickets (two stage types), [8..9] tensor units (64-bit),
                            // [16 + 8 t ..] the cost-class counts of stage type t
    ProdDesc* desc[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int nprod[2] = {0, 0};
    int4* cull_blocks[2] = {nullptr, nullptr};
    int ncull_blocks[2] = {0, 0};
    int cap[2] = {0, 0};
    int* tile_list[2] = {nullptr, nullptr};
    int* slice_items[2] = {nullptr, nullptr};
    cudaStream_t gst = nullptr, bst = nullptr, sst = nullptr;
    cudaStream_t fork[kForks] = {};
    cudaEvent_t ev_fork = nullptr, ev_sliced = nullptr, ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_join[kForks] = {};
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0, body_kernels = 0;

    ~Batch() {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (exec) cudaGraphExecDestroy(exec);
        for (auto s : {gst, bst, sst})
            if (s) cudaStreamDestroy(s);
        for (auto s : fork)
            if (s) cudaStreamDestroy(s);
        for (auto e : {ev_fork, ev_sliced, ev_in, ev_out})
            if (e) cudaEventDestroy(e);
        for (auto e : ev_join)
            if (e) cudaEventDestroy(e);
        cudaFree(arena.base);
        cudaSetDevice(cur);
    }
};

int* stage_counts(Batch* b, int t) { return b->gflags + 16 + 8 * t; }
int* stage_sched(Batch* b, int t) { return b->gflags + 4 + 2 * t; }
unsigned long long* tensor_units_of(Batch* b) { return reinterpret_cast<unsigned long long*>(b->gflags + 8); }

// Carves every device buffer of the batch out of the arena (a counting pass with a null base gives the size).
bool layout(Batch* b) {
    Arena& a = b->arena;
    const size_t slice_bytes = b->emu ? emu_slice_bytes_per_tile() : 0;
    for (BatchMat& M : b->mats) {
        const Geometry& g = M.g;
        const size_t mm = (size_t)g.m * g.m;
        for (TileMat& t : M.buf) {
            t = TileMat();
            t.t = a.take<double>(g.elems());
            t.tree = a.take<double>((size_t)g.tree_size);
            if (b->emu) {
                t.sliceA = a.take<uint8_t>(slice_bytes * mm);
                t.sliceB = a.take<uint8_t>(slice_bytes * mm);
                t.rmax = a.take<unsigned long long>(2 * (size_t)g.m * g.nb);
                t.cmax = t.rmax + (size_t)g.m * g.nb;
            }
        }
        for (int q = 0; q < 2; ++q) {
            M.counts[q] = a.take<int>(mm);
            M.jlist[q] = a.take<int>(mm * g.m);
        }
        M.trace_part = a.take<double>(g.m);
        M.scal = a.take<double>(16);
        M.rowsum = a.take<double>(g.n);
    }
    const int c = b->count;
    b->mflags = a.take<int>(4 * (size_t)c);
    b->t_hist = a.take<double>((size_t)c * std::max(1, b->maxit));
    b->task_ctr = a.take<unsigned long long>(3 * (size_t)c * std::max(1, b->maxit));
    b->gflags = a.take<int>(64);
    for (int t = 0; t < 2; ++t) {
        for (int par = 0; par < 2; ++par) b->desc[t][par] = a.take<ProdDesc>(b->nprod[t]);
        b->cull_blocks[t] = a.take<int4>(b->ncull_blocks[t]);
        b->tile_list[t] = a.take<int>((size_t)kTileBuckets * b->cap[t]);
        b->slice_items[t] = a.take<int>((size_t)b->cap[t] + 1);
    }
    return a.base == nullptr || a.used <= a.size;
}

ProdDesc make_desc(const Batch* b, int q, const TileMat& A, const TileMat& B, const TileMat& C, int list, double tau,
                   int mode, int which, double tol_t) {
    const BatchMat& M = b->mats[q];
    ProdDesc d;
    std::memset(&d, 0, sizeof(d));
    d.At = A.t;
    d.Atree = A.tree;
    d.AsliceA = A.sliceA;
    d.Armax = A.rmax;
    d.Bt = B.t;
    d.Btree = B.tree;
    d.BsliceB = B.sliceB;
    d.Bcmax = B.cmax;
    d.Ct = C.t;
    d.Ctree = C.tree;
    d.CsliceA = C.sliceA;
    d.CsliceB = C.sliceB;
    d.Crmax = C.rmax;
    d.Ccmax = C.cmax;
    d.counts = M.counts[list];
    d.jlist = M.jlist[list];
    d.mflags = b->mflags + 4 * q;
    d.trace_part = M.trace_part;
    d.t_hist = b->t_hist + (size_t)q * std::max(1, b->maxit);
    d.task_ctr = b->task_ctr + 3 * (size_t)q * std::max(1, b->maxit);
    d.tau = tau;
    d.tol_t = tol_t;
    d.mode = mode;
    d.which = which;
    d.n = M.g.n;
    d.maxit = b->maxit;
    d.td = tree_dev(M.g);
    return d;
}

// The four product tables (stage type x parity) and the cull block tables, uploaded once.  Parity 0 reads
// Y, Z from buffers 0, 1 and writes 3, 4; parity 1 the other way round; T is buffer 2 throughout.  The y
// product uses tau_s, the others tau.
int upload_tables(Batch* b, int order, double tol_t) {
    std::vector<ProdDesc> h;
    for (int par = 0; par < 2; ++par) {
        const int yi = par ? 3 : 0, zi = par ? 4 : 1, yo = par ? 0 : 3, zo = par ? 1 : 4;
        h.clear();
        for (int q = 0; q < b->count; ++q) {
            const BatchMat& M = b->mats[q];
            const TileMat &Yb = M.buf[yi], &Zb = M.buf[zi], &Tb = M.buf[2], &Y2 = M.buf[yo], &Z2 = M.buf[zo];
            if (order == SPAMM_ORDER_PAPER) {
                h.push_back(make_desc(b, q, Tb, Yb, Y2, 0, M.tau_s, EPI_PLAIN, 0, tol_t));  // Y <- T (x)_{tau_s} Y
                h.push_back(make_desc(b, q, Zb, Tb, Z2, 1, M.tau, EPI_PLAIN, 1, tol_t));    // Z <- Z (x)_tau T
            } else {
                h.push_back(make_desc(b, q, Yb, Tb, Y2, 0, M.tau_s, EPI_PLAIN, 0, tol_t));  // Y <- Y (x)_{tau_s} T
                h.push_back(make_desc(b, q, Tb, Zb, Z2, 1, M.tau, EPI_PLAIN, 1, tol_t));    // Z <- T (x)_tau Z
            }
        }
        BK(cudaMemcpy(b->desc[0][par], h.data(), h.size() * sizeof(ProdDesc), cudaMemcpyHostToDevice));
        h.clear();
        for (int q = 0; q < b->count; ++q) {
            const BatchMat& M = b->mats[q];
            const TileMat &Y2 = M.buf[yo], &Z2 = M.buf[zo], &Tb = M.buf[2];
            if (order == SPAMM_ORDER_PAPER)
                h.push_back(make_desc(b, q, Y2, Z2, Tb, 0, M.tau, EPI_NS_X, 2, tol_t));  // X <- Y (x)_tau Z
            else
                h.push_back(make_desc(b, q, Z2, Y2, Tb, 0, M.tau, EPI_NS_X, 2, tol_t));  // X <- Z (x)_tau Y
        }
        BK(cudaMemcpy(b->desc[1][par], h.data(), h.size() * sizeof(ProdDesc), cudaMemcpyHostToDevice));
    }
    for (int t = 0; t < 2; ++t) {
        std::vector<int4> blk;
        const int per = t == 0 ? 2 : 1;
        for (int q = 0; q < b->count; ++q)
            for (int r = 0; r < per; ++r) {
                const int p = q * per + r;
                const int mm = b->mats[q].g.m * b->mats[q].g.m;
                const int nb = (mm + 7) / 8;
                for (int k = 0; k < nb; ++k) blk.push_back(make_int4(p, 8 * k, nb, k));
            }
        BK(cudaMemcpy(b->cull_blocks[t], blk.data(), blk.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    return SPAMM_OK;
}

// a1-a2 for one matrix, as the single path's prologue does it (dual channel, alpha = 1): Gershgorin bound
// (plus the shift), X0 = Y0 = S / c packed with its norms, T0 = h[X0], Z0 = I, and their digit slices.
void enqueue_setup(Batch* b, BatchMat& M, double mu_rel, cudaStream_t st) {
    const Geometry& g = M.g;
    double* c0 = M.scal + 0;
    double* mu = M.scal + 1;
    double* c = M.scal + 2;
    double* sqc = M.scal + 3;
    double* rc = M.scal + 6;
    double* rsqc = M.scal + 7;
    const double* mu_ptr = nullptr;
    if (mu_rel > 0.0) {
        launch_gershgorin(M.S, g.n, nullptr, M.rowsum, c0, st);
        launch_scale_mu(c0, mu_rel, mu, st);
        mu_ptr = mu;
    }
    launch_gershgorin(M.S, g.n, mu_ptr, M.rowsum, c, st);
    launch_scale_consts(c, sqc, rc, rsqc, st);
    const TileMat &X0 = M.buf[0], &Z0 = M.buf[1], &T0 = M.buf[2];
    launch_pack(M.S, g.n, g, mu_ptr, rc, X0, st, b->emu);  // FP32 tile norms on the tensor-core path, as one solve
    launch_tree(g, X0.tree, nullptr, st);
    // the tensor-core path takes T0's row and column maxima in the map
    if (b->emu) cudaMemsetAsync(T0.rmax, 0, 2 * (size_t)g.m * g.nb * sizeof(unsigned long long), st);
    launch_map(X0.t, X0.tree, T0, g, SPAMM_MAP_NS, M.trace_part, b->emu, nullptr, st, b->emu);
    launch_tree(g, T0.tree, nullptr, st);
    launch_identity(g, Z0, st);
    launch_tree(g, Z0.tree, nullptr, st);
    // the first y and z products read these at tau_s and tau: tiles neither can keep are not sliced
    const double tau_min = std::min(M.tau, M.tau_s);
    if (b->emu)
        for (const TileMat* P : {&X0, &T0, &Z0}) {
            if (P != &T0) {
                cudaMemsetAsync(P->rmax, 0, 2 * (size_t)g.m * g.nb * sizeof(unsigned long long), st);
                launch_rowcol_max(P->t, g, P->rmax, P->cmax, st);
            }
            launch_slice(P->t, P->tree, nullptr, P->rmax, P->cmax, P->sliceA, P->sliceB, g, nullptr, nullptr,
                         nullptr, st, tau_min > 0.0 ? P->tree + g.off[0] : nullptr, 0.999 * tau_min * tau_min);
        }
}

// a7 for one matrix: Y sqrt(c), Z / sqrt(c) from the buffers of the last iteration it ran.
void enqueue_finish(Batch* b, int q, cudaStream_t st) {
    BatchMat& M = b->mats[q];
    const int* iters = b->mflags + 4 * q + 1;
    launch_unpack(M.buf[0].t, M.buf[0].tree, M.g, M.Y, M.scal + 3, st, M.buf[3].t, M.buf[3].tree, iters, 0);
    launch_unpack(M.buf[1].t, M.buf[1].tree, M.g, M.Z, M.scal + 7, st, M.buf[4].t, M.buf[4].tree, iters, 0);
}

// One stage (t = 0: y and z products, t = 1: x products) of the iteration of parity par, on st.  The leaf
// products wait for the previous stage's slicing when wait_slices; this stage's slicing runs on the side
// stream beside its quadtree pass and the next cull.
void enqueue_stage(Batch* b, int t, int par, bool wait_slices, const cudaGraphConditionalHandle* cond,
                   cudaStream_t st) {
    int* all_done = b->gflags;
    const ProdDesc* d = b->desc[t][par];
    launch_cull_batched(d, b->cull_blocks[t], b->ncull_blocks[t], b->tile_list[t], stage_counts(b, t), b->cap[t],
                        all_done, st);
    if (b->emu) {
        if (wait_slices) cudaStreamWaitEvent(st, b->ev_sliced, 0);
        launch_gemm_emu_batched(d, b->tile_list[t], stage_counts(b, t), b->cap[t], b->slice_items[t],
                                stage_sched(b, t), all_done, b->gflags + 3, st, tensor_units_of(b));
        cudaEventRecord(b->ev_fork, st);
        cudaStreamWaitEvent(b->sst, b->ev_fork, 0);
        launch_slice_batched(d, b->slice_items[t], b->cap[t], all_done, b->sst);
        cudaEventRecord(b->ev_sliced, b->sst);
    } else {
        launch_gemm_f64_batched(b->leaf, d, b->tile_list[t], stage_counts(b, t), b->cap[t], all_done, st);
    }
    launch_tree_batched(d, b->nprod[t], stage_counts(b, t), b->gflags + 2, b->gflags + 1, b->count, all_done,
                        t == 1 ? cond : nullptr, t == 1, st);
}

// Spreads per-matrix work over the fork streams and joins them back into st.
template <typename F>
void fork_over_matrices(Batch* b, cudaStream_t st, F&& f) {
    cudaEventRecord(b->ev_fork, st);
    const int nf = std::min(kForks, b->count);
    for (int k = 0; k < nf; ++k) cudaStreamWaitEvent(b->fork[k], b->ev_fork, 0);
    for (int q = 0; q < b->count; ++q) f(q, b->fork[q % nf]);
    for (int k = 0; k < nf; ++k) {
        cudaEventRecord(b->ev_join[k], b->fork[k]);
        cudaStreamWaitEvent(st, b->ev_join[k], 0);
    }
}

// The whole batched solve captured on gst: state cleared, per-matrix setup, the iteration as a WHILE node
// (body: two iterations of two stages each), per-matrix finish.
int capture(Batch* b, double mu_rel) {
    cudaStream_t st = b->gst;
    BK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const long long l0 = spamm_kernel_launches();
    const int mi = std::max(1, b->maxit);
    cudaMemsetAsync(b->mflags, 0, 4 * (size_t)b->count * sizeof(int), st);
    cudaMemsetAsync(b->t_hist, 0, (size_t)b->count * mi * sizeof(double), st);
    cudaMemsetAsync(b->task_ctr, 0, 3 * (size_t)b->count * mi * sizeof(unsigned long long), st);
    cudaMemsetAsync(b->gflags, 0, 64 * sizeof(int), st);
    fork_over_matrices(b, st, [&](int q, cudaStream_t fs) { enqueue_setup(b, b->mats[q], mu_rel, fs); });

    int err = SPAMM_OK;
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle cond;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t node;
    cudaError_t ce = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, &edata, &ndeps);
    if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&cond, graph, b->maxit > 0 ? 1u : 0u,
                                                                 cudaGraphCondAssignDefault);
    if (ce == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ce = cudaGraphAddNode(&node, graph, deps, edata, ndeps, &np);
    }
    if (ce == cudaSuccess)
        ce = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    long long lb0 = 0, lb1 = 0;
    if (ce == cudaSuccess) {
        ce = cudaStreamBeginCaptureToGraph(b->bst, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            lb0 = spamm_kernel_launches();
            for (int par = 0; par < 2; ++par) {
                enqueue_stage(b, 0, par, par > 0, &cond, b->bst);
                enqueue_stage(b, 1, par, true, &cond, b->bst);
            }
            if (b->emu) cudaStreamWaitEvent(b->bst, b->ev_sliced, 0);
            lb1 = spamm_kernel_launches();
            cudaGraph_t bg = nullptr;
            ce = cudaStreamEndCapture(b->bst, &bg);
        }
    }
    if (ce == cudaSuccess)
        fork_over_matrices(b, st, [&](int q, cudaStream_t fs) { enqueue_finish(b, q, fs); });
    if (ce == cudaSuccess) ce = cudaGetLastError();
    cudaGraph_t whole = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(st, &whole);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec, whole, 0);
    if (whole) cudaGraphDestroy(whole);
    const long long l1 = spamm_kernel_launches();
    b->body_kernels = lb1 - lb0;
    b->graph_kernels = (l1 - l0) - b->body_kernels;
    note_launch((int)-(l1 - l0));  // counted when the graph runs
    if (ce != cudaSuccess) {
        set_error_message((std::string("batched solve graph: ") + cudaGetErrorString(ce)).c_str());
        cudaGetLastError();
        err = SPAMM_ERR_CUDA;
    }
    return err;
}

// (Re)builds b for a new set of problems: sizes, the arena (kept when it is large enough, else replaced;
// limit > 0 caps its size, limit = 0 allows 70 % of the free device memory), the tables and the graph.
int build_batch(Batch* b, int count, const double* const* dS, const int* n, const double* tau, int maxit,
                double* const* dY, double* const* dZ, const spamm_opts& o, size_t limit) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->count = count;
    b->leaf = o.leaf;
    b->maxit = maxit;
    b->emu = o.precision == SPAMM_EMU64;
    b->mats.assign(count, BatchMat());
    long cap0 = 0, cap1 = 0, blk0 = 0, blk1 = 0;
    for (int q = 0; q < count; ++q) {
        BatchMat& M = b->mats[q];
        M.g = make_geometry(n[q], o.leaf);
        M.tau = tau[q];
        M.tau_s = o.tau_s < 0.0 ? 0.01 * tau[q] : o.tau_s;
        M.S = dS[q];
        M.Y = dY[q];
        M.Z = dZ[q];
        const long mm = (long)M.g.m * M.g.m;
        cap0 += 2 * mm;
        cap1 += mm;
        blk0 += 2 * ((mm + 7) / 8);
        blk1 += (mm + 7) / 8;
    }
    if (cap0 >= (1l << 31) / kTileBuckets || blk0 >= (1l << 31)) {
        set_error_message("batch too large for one launch list");
        return SPAMM_ERR_UNSUPPORTED;
    }
    b->nprod[0] = 2 * count;
    b->nprod[1] = count;
    b->cap[0] = (int)cap0;
    b->cap[1] = (int)cap1;
    b->ncull_blocks[0] = (int)blk0;
    b->ncull_blocks[1] = (int)blk1;
    // size, then the allocation (when it does not fit, the caller solves the matrices one by one instead)
    Arena keep = b->arena;
    b->arena = Arena();
    b->arena.size = ~size_t(0) >> 1;
    layout(b);
    const size_t bytes = b->arena.used;
    b->arena = keep;
    if (!b->arena.base || b->arena.size < bytes) {
        size_t fr = 0, tot = 0;
        BK(cudaMemGetInfo(&fr, &tot));
        if (b->arena.base) fr += b->arena.size;
        const size_t cap = limit ? limit : fr / 10 * 7;
        if (bytes > cap) {
            set_error_message("batch footprint exceeds the memory it may use");
            return SPAMM_ERR_NOMEM;
        }
        cudaFree(b->arena.base);
        b->arena = Arena();
        const size_t want = std::min(cap, bytes + bytes / 2);  // headroom for the next, slightly larger batch
        BK(cudaMalloc(reinterpret_cast<void**>(&b->arena.base), want));
        b->arena.size = want;
    }
    b->arena.used = 0;
    if (!layout(b)) {
        set_error_message("batch layout overflow");
        return SPAMM_ERR_CUDA;
    }
    int e = upload_tables(b, o.order, o.tol_t);
    if (e) return e;
    if (!b->gst) {
        BK(cudaStreamCreateWithFlags(&b->gst, cudaStreamNonBlocking));
        BK(cudaStreamCreateWithFlags(&b->bst, cudaStreamNonBlocking));
        BK(cudaStreamCreateWithFlags(&b->sst, cudaStreamNonBlocking));
        for (auto& f : b->fork) BK(cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking));
        for (cudaEvent_t* ev : {&b->ev_fork, &b->ev_sliced, &b->ev_in, &b->ev_out})
            BK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
        for (auto& ev : b->ev_join) BK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    return capture(b, o.mu_rel);
}

// The batch cached per device (its buffers and graph), reused while the call's key is the same.
std::mutex g_batch_mu;
std::unique_ptr<Batch> g_batch[64];

// Statistics and status of every matrix after a run (the caller's stream is synchronised).
int collect(Batch* b, const spamm_opts& o, cudaStream_t st, spamm_stats* stats, int* statuses = nullptr) {
    const int c = b->count;
    const int mi = std::max(1, b->maxit);
    std::vector<int> mf(4 * (size_t)c);
    std::vector<double> th((size_t)c * mi);
    std::vector<unsigned long long> kc(3 * (size_t)c * mi);
    std::vector<double> scal(16 * (size_t)c);
    int gf[64];
    BK(cudaMemcpyAsync(mf.data(), b->mflags, mf.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(th.data(), b->t_hist, th.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(kc.data(), b->task_ctr, kc.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(gf, b->gflags, sizeof(gf), cudaMemcpyDeviceToHost, st));
    for (int q = 0; q < c; ++q)
        BK(cudaMemcpyAsync(scal.data() + 16 * (size_t)q, b->mats[q].scal, 16 * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    int max_iters = 0;
    for (int q = 0; q < c; ++q) max_iters = std::max(max_iters, std::min(b->maxit, mf[4 * q + 1]));
    note_launch((int)(b->graph_kernels + (long long)((max_iters + 1) / 2) * b->body_kernels));
    if (gf[3]) {
        set_error_message("a bounded device-side wait of the tensor-core kernel expired");
        return SPAMM_ERR_TIMEOUT;
    }
    unsigned long long units = 0;
    std::memcpy(&units, gf + 8, sizeof(units));
    int first = SPAMM_OK;
    std::string first_msg;
    for (int q = 0; q < c; ++q) {
        const Geometry& g = b->mats[q].g;
        const int iters = std::min(b->maxit, mf[4 * q + 1]);
        const double* tq = th.data() + (size_t)q * mi;
        const unsigned long long* kq = kc.data() + 3 * (size_t)q * mi;
        long long total = 0;
        for (int k = 0; k < 3 * iters; ++k) total += (long long)kq[k];
        const double t_final = iters > 0 ? tq[iters - 1] : 0.0;
        if (stats) {
            spamm_stats& s = stats[q];
            s.iters = iters;
            s.t_final = t_final;
            s.resid_F = -1.0;
            s.scale_c = scal[16 * (size_t)q + 2];
            s.tasks_total = total;
            s.tasks_dense = 3ll * iters * (long long)g.m * g.m * g.m;
            s.flops = 2.0 * (double)g.nb * g.nb * g.nb * (double)total;
            if (s.t_hist)
                for (int k = 0; k < iters; ++k) s.t_hist[k] = tq[k];
            if (s.task_hist)
                for (int k = 0; k < 3 * iters; ++k) s.task_hist[k] = (long long)kq[k];
            s.gemm_ms = s.cull_ms = s.tree_ms = s.slice_ms = 0.0;
            s.cull_launches = s.tree_launches = s.slice_launches = 0;
            s.gemm_launches = 2ll * ((iters + 1) / 2) * 2;  // this matrix's share: the stages it took part in
            s.tensor_units = q == 0 ? (long long)units : 0;
        }
        int status = SPAMM_OK;
        const char* msg = "";
        for (int k = 0; k < iters; ++k)
            if (!std::isfinite(tq[k]) || std::fabs(tq[k]) >= 1.0) {
                status = SPAMM_ERR_DIVERGED;
                msg = "trace error left [0, 1): the iteration diverged";
                break;
            }
        if (!status && o.tol_t > 0.0 && !(std::fabs(t_final) <= o.tol_t)) {
            status = SPAMM_ERR_NOTCONVERGED;
            msg = "maxit reached before |t_k| <= tol_t";
        }
        if (statuses) statuses[q] = status;
        if (status && !first) {
            first = status;
            first_msg = msg;
        }
    }
    if (first) set_error_message(first_msg.c_str());
    return first;
}

// Whether the engine serves these options (the rest go through the per-matrix path).
bool engine_covers(const spamm_opts& o) {
    static const bool off = [] {
        const char* v = getenv("SPAMM_NO_BATCH_ENGINE");
        return v && v[0] && v[0] != '0';
    }();
    return !off && o.map == SPAMM_MAP_NS && o.channel == SPAMM_CHANNEL_DUAL && !o.residual && !o.profile &&
           o.leaf != 0;
}

// The batched solve in a caller-held slot.  SPAMM_ERR_UNSUPPORTED (message untouched) when the per-matrix
// path must serve the call.
int solve_in_slot(std::unique_ptr<Batch>& slot, int count, const double* const* S, const int* n, const double* tau,
                  int maxit, double* const* Y, double* const* Z, const spamm_opts& o, spamm_stats* stats,
                  size_t limit, int* statuses = nullptr) {
    if (!engine_covers(o) || count < 1 || 2 * count > kMaxStageProducts) return SPAMM_ERR_UNSUPPORTED;
    if (stats)
        for (int q = 0; q < count; ++q)
            if (stats[q].lens_hist) return SPAMM_ERR_UNSUPPORTED;
    int dev = 0;
    BK(cudaGetDevice(&dev));
    std::vector<const double*> dS(count);
    std::vector<double*> dY(count), dZ(count);
    for (int q = 0; q < count; ++q) {
        void* v[3] = {nullptr, nullptr, nullptr};
        const void* p[3] = {S[q], Y[q], Z[q]};
        for (int r = 0; r < 3; ++r) {
            const int e = pointer_view(p[r], dev, &v[r]);
            if (e) return e;
            if (!v[r]) return SPAMM_ERR_UNSUPPORTED;  // pageable host memory: staged per matrix
        }
        dS[q] = static_cast<const double*>(v[0]);
        dY[q] = static_cast<double*>(v[1]);
        dZ[q] = static_cast<double*>(v[2]);
    }
    BatchKey key;
    key.device = dev;
    key.count = count;
    key.leaf = o.leaf;
    key.precision = o.precision;
    key.order = o.order;
    key.maxit = maxit;
    key.tau_s = o.tau_s;
    key.mu_rel = o.mu_rel;
    key.tol_t = o.tol_t;
    key.n.assign(n, n + count);
    key.tau.assign(tau, tau + count);
    for (int q = 0; q < count; ++q) {
        key.ptrs.push_back(dS[q]);
        key.ptrs.push_back(dY[q]);
        key.ptrs.push_back(dZ[q]);
    }
    init_device_attributes();
    if (slot && slot->device != dev) slot.reset();
    if (!slot || !slot->exec || !(slot->key == key)) {
        if (!slot) {
            slot.reset(new Batch);
            slot->device = dev;
        }
        slot->key = BatchKey();
        const int e = build_batch(slot.get(), count, dS.data(), n, tau, maxit, dY.data(), dZ.data(), o, limit);
        if (e == SPAMM_ERR_NOMEM) {
            cudaGetLastError();
            return SPAMM_ERR_UNSUPPORTED;  // too large to hold at once: solved one by one
        }
        if (e) return e;
        slot->key = key;
    }
    Batch* b = slot.get();
    cudaStream_t st = static_cast<cudaStream_t>(o.stream);
    BK(cudaEventRecord(b->ev_in, st));
    BK(cudaStreamWaitEvent(b->gst, b->ev_in, 0));
    BK(cudaGraphLaunch(b->exec, b->gst));
    BK(cudaEventRecord(b->ev_out, b->gst));
    BK(cudaStreamWaitEvent(st, b->ev_out, 0));
    return collect(b, o, st, stats, statuses);
}

}  // namespace

// Batched solve of `count` problems in one graph (see the top of this file), in the batch cached for the
// current device.
int batched_solve(int count, const double* const* S, const int* n, const double* tau, int maxit,
                  double* const* Y, double* const* Z, const spamm_opts& o, spamm_stats* stats) {
    if (!engine_covers(o)) return SPAMM_ERR_UNSUPPORTED;
    int dev = 0;
    BK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SPAMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    return solve_in_slot(g_batch[dev], count, S, n, tau, maxit, Y, Z, o, stats, 0);
}

// One solve on the batched engine (the stage schedule), in a batch cached per device apart from the batched
// calls' one, so that the two do not evict each other's graphs.
std::mutex g_stage_mu;
std::unique_ptr<Batch> g_stage_batch[64];
int stage_solve(const double* S, int n, double tau, int maxit, double* Y, double* Z, const spamm_opts& o,
                spamm_stats* stats) {
    if (!engine_covers(o)) return SPAMM_ERR_UNSUPPORTED;
    int dev = 0;
    BK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SPAMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    return solve_in_slot(g_stage_batch[dev], 1, &S, &n, &tau, maxit, &Y, &Z, o, stats, 0);
}

// A batch owned by its caller (one per request-server worker): buffers and graph kept between calls.
struct BatchSlot {
    std::unique_ptr<Batch> b;
};
BatchSlot* batch_slot_create() { return new BatchSlot; }
void batch_slot_destroy(BatchSlot* s) { delete s; }
int batched_solve_slot(BatchSlot* s, int count, const double* const* S, const int* n, const double* tau, int maxit,
                       double* const* Y, double* const* Z, const spamm_opts& o, spamm_stats* stats, size_t limit,
                       int* statuses) {
    return solve_in_slot(s->b, count, S, n, tau, maxit, Y, Z, o, stats, limit, statuses);
}
bool batch_engine_covers(const spamm_opts& o) { return engine_covers(o); }

// Device bytes one matrix adds to a batch (its five tile buffers with trees, slices and maxima, its two task
// lists, its stage-list entries and its share of the tables).
size_t batch_footprint(int n, int nb, int precision, int maxit) {
    const Geometry g = make_geometry(n, nb);
    const size_t mm = (size_t)g.m * g.m;
    size_t b = 5 * (g.elems() + (size_t)g.tree_size) * sizeof(double);
    if (precision == SPAMM_EMU64) b += 5 * (2 * emu_slice_bytes_per_tile() * mm + 2 * (size_t)g.m * g.nb * 8);
    b += 2 * (mm + mm * g.m) * sizeof(int) + ((size_t)g.m + 16 + (size_t)n) * sizeof(double);
    b += 3 * mm * (kTileBuckets + 1) * sizeof(int) + 6 * sizeof(ProdDesc) + 3 * ((mm + 7) / 8) * sizeof(int4);
    b += 4 * sizeof(int) + 4 * sizeof(double) * (size_t)std::max(1, maxit);  // stop flags, t_k and task counts
    return b + 32 * 256;                                                      // alignment of the pieces
}

// Frees the cached batches (no work may be in flight).
void release_batches() {
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        for (auto& b : g_batch) b.reset();
    }
    std::lock_guard<std::mutex> lk(g_stage_mu);
    for (auto& b : g_stage_batch) b.reset();
}

}  // namespace spamm

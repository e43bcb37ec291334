// Internal declarations of libspamm: geometry of the tile grid and quadtree,
// device buffers of one problem, and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "spamm.h"

namespace spamm {

constexpr int kMaxLevels = 24;

// Tile grid of an n x n matrix with nb x nb leaves: m tiles per side, the
// quadtree over it has leaf level L (2^L >= m) and dim[l] existing nodes per
// side at level l.  Level l of a norm tree lives at off[l] of one array; the
// leaf level sits at offset 0, so leaf norms are tree[i*m + j].
struct Geometry {
    int n = 0, nb = 0, m = 0, L = 0;
    int dim[kMaxLevels] = {};
    long off[kMaxLevels] = {};
    long tree_size = 0;
    int coarse = 0;        // level used to pre-filter the cull
    int coarse_shift = 0;  // L - coarse
    size_t tile_elems() const { return (size_t)nb * nb; }
    size_t elems() const { return (size_t)m * m * nb * nb; }
};

Geometry make_geometry(int n, int nb);

// Tile-major FP64 matrix: tile (i,j) is nb*nb row-major doubles at
// t + (i*m + j)*nb*nb.  tree holds the squared Frobenius norms of every
// quadtree node.
// With the tensor-core (SPAMM_EMU64) arithmetic a matrix also carries its
// FP16 digit slices in the operand-A and operand-B layouts and the magnitude
// maxima (IEEE bits) of its rows and columns.
struct TileMat {
    double* t = nullptr;
    double* tree = nullptr;
    uint8_t* sliceA = nullptr;
    uint8_t* sliceB = nullptr;
    unsigned long long* rmax = nullptr;  // [m*nb], followed by
    unsigned long long* cmax = nullptr;  // [m*nb]
    // tensor-core path: the output tiles to slice ([m*m] tile ids, then their count), copied by the
    // leaf-product kernel so that slicing can run beside the next cull; and the event recorded once the
    // slices are written
    int* slice_list = nullptr;
    cudaEvent_t sliced = nullptr;
};

// Geometry passed by value to kernels.
struct TreeDev {
    int m, L, coarse, shift;
    int dim[kMaxLevels];
    long off[kMaxLevels];
};
TreeDev tree_dev(const Geometry& g);

// Leaf-product epilogues: the plain product; X with T = 1.5 I - 0.5 X fused
// (the alpha = 1 map) plus the trace partials; X itself plus the trace
// partials (for a map whose coefficients depend on tr X, applied by k_map
// once the whole product is done).
enum EpiMode { EPI_PLAIN = 0, EPI_NS_X = 1, EPI_X = 2 };

// Counts kernel launches (spamm_kernel_launches); every launcher calls it.
void note_launch(int k = 1);

// Kernels of the product chain (cull -> leaf products -> slicing -> tree) are
// launched as programmatic dependents of the previous kernel in their stream:
// the launch overlaps the tail of the predecessor, and the kernel itself
// waits (grid_dependency_wait, first statement) until the predecessor grid
// has finished and its writes are visible.  Every grid of the chain is
// resident in one wave or waits without holding back its predecessor, whose
// blocks never wait on a dependent.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Device side of the above: wait for the predecessor grid, then let the
// next kernel in the stream start launching.
__device__ __forceinline__ void grid_dependency_wait() {
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Once per device and process: shared-memory limits of the big kernels and
// the SM count (kept out of the launchers so that launches can be captured
// into CUDA graphs).
void init_device_attributes();
int device_sm_count();
void f64_kernel_attributes();
void emu_kernel_attributes();

// ---- kernels_tree.cu -------------------------------------------------------
// c = max_i sum_j |s_ij + mu delta_ij|; mu read from *mu_dev (may be null = 0).
void launch_gershgorin(const double* S, int n, const double* mu_dev, double* rowsum, double* out_c,
                       cudaStream_t st);
// Row-major D = S + (mu_rel * *c0) I.
void launch_shift_copy(const double* S, double* D, int n, double mu_rel, const double* c0, cudaStream_t st);
// Row-major T = A^T (n x n).
void launch_transpose_rm(const double* A, double* T, int n, cudaStream_t st);
// *mu_out = mu_rel * (*c0)
void launch_scale_mu(const double* c0, double mu_rel, double* mu_out, cudaStream_t st);
// Row-major src -> tile-major dst with leaf norms.  When recip_c != null:
// dst = (src + mu delta) * (*recip_c), the scaling by the once-rounded 1/c.  Edge padding is zero.
// f32_norms (scaled 64 x 64 packs): the leaf norms are FP32 sums of squares (f32_of_bits).
void launch_pack(const double* src, int n, const Geometry& g, const double* mu, const double* recip_c,
                 TileMat dst, cudaStream_t st, bool f32_norms = false);
// trace_part[i] = logical trace of diagonal tile (i, i) of a packed matrix.
void launch_trace_parts(const double* X, const Geometry& g, double* trace_part, cudaStream_t st);
// T = h_alpha[eps I + (1 - 2 eps) X] elementwise on tiles (logical identity):
// map SPAMM_MAP_NS (alpha = 1, eps = 0) or SPAMM_MAP_SCALED (alpha, eps from
// t = (n - sum trace_part)/n).  X may be T.t (in place; leafX then T.tree).
// Writes T's leaf norms and, with `maxima`, accumulates T's row/column
// maxima into T.rmax/T.cmax (which must be zero).  Skipped once *done is set.
// f32_norms: T's leaf norms are FP32 sums of squares (f32_of_bits).
void launch_map(const double* X, const double* leafX, TileMat T, const Geometry& g, int map, const double* trace_part,
                bool maxima, const int* done, cudaStream_t st, bool f32_norms = false);
// Plane-diagonal profile of one product's task lists (counts, jlist): adds
// to lens[(*iter * 3 + which) * 3 * bins + q * bins + d] the triples (i,j,k)
// at distance d from plane q (|i-j|, |j-k|, |i-k|; d clamped to bins-1).
// Skipped once *done is set.
void launch_lens(const int* counts, const int* jlist, const Geometry& g, int bins, const int* iter, int which,
                 unsigned long long* lens, const int* done, cudaStream_t st);
// T = A^T on the tile grid (tile (i,j) of T = tile (j,i) of A, transposed) with T's leaf norms; tiles of
// norm 0 are left unwritten.  Skipped once *done is set.
void launch_transpose(const TileMat& A, TileMat T, const Geometry& g, const int* done, cudaStream_t st);
// Z = I_n in tile-major form, with leaf norms.
void launch_identity(const Geometry& g, TileMat Z, cudaStream_t st);
// Work fused into the quadtree pass, all optional.  After the levels:
// *zero_int = 0 (the output-tile counter, ready for the next cull); with
// trace_part set, the iteration's trace error t_k = (n - sum trace_part)/n
// into t_hist[k] with k = *iters, then *iters = k + 1, and the stop:
// *done = 1 (and the graph conditional `cond` cleared, if has_cond) once
// |t_k| <= tol_t > 0 or k + 1 == maxit.
struct TreeExtra {
    int* zero_int = nullptr;  // zero_n ints
    int zero_n = 1;
    const double* trace_part = nullptr;
    int n = 0, maxit = 0;
    double tol_t = 0.0;
    double* t_hist = nullptr;
    int* done = nullptr;
    int* iters = nullptr;
    cudaGraphConditionalHandle cond = 0;
    int has_cond = 0;
};
// Upper quadtree levels from the leaf level (skipped when *done is set).
void launch_tree(const Geometry& g, double* tree, const int* done, cudaStream_t st,
                 const TreeExtra& ex = TreeExtra());
// Task lists of A (x) B: counts[i*m+k], jlist[(i*m+k)*m + ...] ascending j.
// thr = ((tau*tau) * rootA) * rootB.  total (may be null) gets += task count.
// Output tiles with a task (or, with force_diag, on the diagonal) are
// appended to tile_list (*tile_count must be zero on entry, order
// unspecified); for every other output tile leafC[tile] is set to 0: that
// tile is exactly zero and its data are not written (readers check nu == 0).
// zero_u64[0 .. zero_n) is cleared on the way (the output's row/column
// maxima, which the leaf products accumulate with atomics).
// With buckets > 1 the listed tiles are sorted coarsely by cost: a tile with
// cnt tasks goes to bucket tile_bucket(cnt), whose ids sit at
// tile_list[b*m*m ...] with count tile_count[b] (all counts zero on entry).
struct CullOut {
    int* counts;
    int* jlist;
    int* tile_list;
    int* tile_count;
    double* leafC;
    int force_diag;
    unsigned long long* zero_u64 = nullptr;
    long zero_n = 0;
    int buckets = 1;
    const int* iter = nullptr;  // set: the task count goes to total[3 * *iter]
};

// Buckets of listed output tiles by task count, most expensive first: the
// persistent leaf-product kernels draw tiles in this order, so the cheap
// tiles fill the end of a launch (longest-first scheduling).
constexpr int kTileBuckets = 5;
__host__ __device__ inline int tile_bucket(int cnt) {
    return cnt >= 16 ? 0 : cnt >= 8 ? 1 : cnt >= 4 ? 2 : cnt >= 2 ? 3 : 4;
}
#ifdef __CUDACC__
// |v| as FP32 from the IEEE bits b of |v|, its mantissa cut to 23 bits (relative error below 2^-23); 0 for
// zero and for magnitudes outside FP32's normal range.  On the tensor-core path the per-tile sums of
// squares are taken in FP32: they only steer the cull, and a relative error near 1e-6 in a tile norm moves
// a keep decision only for pairs that sit that close to the threshold.  Their squares overflow for
// |v| >= 2^64, far above the magnitudes of the scaled iteration.
__device__ __forceinline__ float f32_of_bits(unsigned long long b) {
    const unsigned hw = (unsigned)(b >> 32);
    const int E = (int)(hw >> 20);
    // the low 9 exponent bits and the leading 23 mantissa bits, the bias moved from 1023 to 127 (mod 2^32)
    const unsigned f = __funnelshift_r((unsigned)b, hw, 29) - (896u << 23);
    return (E > 896 && E < 1151) ? __uint_as_float(f) : 0.f;
}
// Number of listed tiles, and the id of the t-th one (buckets in order).
__device__ __forceinline__ int listed_total(const int* tile_count, int buckets) {
    int n = 0;
    for (int b = 0; b < buckets; ++b) n += tile_count[b];
    return n;
}
__device__ __forceinline__ int listed_tile(const int* tile_list, const int* tile_count, int buckets, int mm, int t) {
    for (int b = 0; b < buckets; ++b) {
        const int c = tile_count[b];
        if (t < c) return tile_list[(size_t)b * mm + t];
        t -= c;
    }
    return -1;
}
#endif
void launch_cull(const Geometry& g, const double* treeA, const double* treeB, double tau, const CullOut& out,
                 unsigned long long* total, double* thr_out, const int* done, cudaStream_t st);
// Tile-major -> row-major with out = in * (*mul) or in / (*div) (one of them
// null or both null).  Tiles whose leaf norm is 0 are written as zeros.
// With `iters` set, the source is src/leaf when *iters - iters_src is even and
// src_alt/leaf_alt when it is odd: the iterates alternate between two buffers,
// and a solve that stopped on the device (|t_k| <= tol_t) ran *iters of the
// iters_src iterations its launch sequence holds.
// dst = src * (*scale) when scale != null, else src.
void launch_unpack(const double* src, const double* leaf, const Geometry& g, double* dst, const double* scale,
                   cudaStream_t st, const double* src_alt = nullptr, const double* leaf_alt = nullptr,
                   const int* iters = nullptr, int iters_src = 0);
// *sqc = sqrt(*c), *rc = 1 / *c, *rsqc = 1 / sqrt(*c), each rounded once.
void launch_scale_consts(const double* c, double* sqc, double* rc, double* rsqc, cudaStream_t st);
// sum over logical entries of (R - I)^2 -> *out (deterministic)
void launch_resid_norm(const double* R, const Geometry& g, double* partial, double* out, cudaStream_t st);

// ---- kernels_f64.cu --------------------------------------------------------
// C_ik = sum_{j in list(i,k)} A_ij B_jk in FP64 (dense = every j), epilogue
// per mode; writes leaf norms of the stored tile into treeC[0..m*m) and, for
// EPI_NS_X, the diagonal-tile trace partials of X.
// Sparse form: one CTA per entry of the compacted output-tile list; tasks
// whose operand tile has leaf norm 0 are skipped (exact zeros).  Dense form
// (dense = 1, tile_list null): every output tile, every j.
void launch_gemm_f64(const Geometry& g, const double* A, const double* B, double* C, const double* leafA,
                     const double* leafB, double* treeC, const int* counts, const int* jlist, const int* tile_list,
                     const int* tile_count, int dense, EpiMode mode, double* trace_part, const int* done,
                     cudaStream_t st, int buckets = 1);

// ---- spamm_api.cu, for the request server --------------------------------
}  // namespace spamm
struct spamm_opts;
struct spamm_stats;
namespace spamm {
size_t plan_footprint(int n, int nb, int precision, bool host_io);
// Address the kernels use for caller matrix p in work on `device` (null: pageable host memory, staged);
// SPAMM_ERR_ARG for device memory of another GPU.
int pointer_view(const void* p, int device, void** view);
int run_sqrt(const double* S, int n, double tau, int maxit, double* Y, double* Z, const spamm_opts& o,
             spamm_stats* stats);
int check_args(int n, double tau, const spamm_opts& o);
spamm_opts resolved(const spamm_opts* o);
void trim_plans(size_t keep_bytes);
const char* last_error_message();
void set_error_message(const char* msg);

// ---- batched products (spamm_batch.cu) -------------------------------------
// One SpAMM product of a batch of independent solves: operands, output, task lists and the state of the
// matrix it belongs to.  A stage of the batched iteration runs the products of one table in a single
// launch of each kernel (cull, leaf products, slicing, quadtree); a work item is one output tile of one
// product, encoded as (product << kItemShift) | tile.
constexpr int kItemShift = 18;  // tiles per product < 2^18 (m <= 512)
constexpr int kMaxStageProducts = 1 << 13;
struct ProdDesc {
    const double* At;
    const double* Atree;
    const uint8_t* AsliceA;
    const unsigned long long* Armax;
    const double* Bt;
    const double* Btree;
    const uint8_t* BsliceB;
    const unsigned long long* Bcmax;
    double* Ct;
    double* Ctree;
    uint8_t* CsliceA;
    uint8_t* CsliceB;
    unsigned long long* Crmax;  // followed by Ccmax (2 m N_b words, cleared by the cull)
    unsigned long long* Ccmax;
    int* counts;                // [m*m] task counts of the output tiles
    int* jlist;                 // [m*m*m] ascending j per output tile
    int* mflags;                // the matrix's [0] stop, [1] iterations run
    double* trace_part;         // the matrix's [m] diagonal-tile trace partials (X product)
    double* t_hist;             // the matrix's [maxit] trace errors
    unsigned long long* task_ctr;  // the matrix's [3 maxit] task counts (y, z, x of each iteration)
    double tau;
    double tol_t;
    int mode;                   // EPI_PLAIN or EPI_NS_X
    int which;                  // 0 y, 1 z, 2 x product (task counter slot; 2 also takes t_k and the stop)
    int n, maxit;
    TreeDev td;
};
#ifdef __CUDACC__
__device__ __forceinline__ int item_prod(int item) { return item >> kItemShift; }
__device__ __forceinline__ int item_tile(int item) { return item & ((1 << kItemShift) - 1); }
#endif

// Leaf products of every product of a stage on the tensor cores (leaf 64): the items listed by the batched
// cull (tile_list / tile_count in kTileBuckets cost classes), drawn most expensive first; slice_items gets
// the drawn items and their count at slice_items[cap] for the slicing pass.  all_done: the batch has
// stopped (every kernel returns at once).
void launch_gemm_emu_batched(const ProdDesc* prods, const int* tile_list, const int* tile_count, int cap,
                             int* slice_items, int* sched, const int* all_done, int* err, cudaStream_t st,
                             unsigned long long* units = nullptr);
// FP64 leaf products of every product of a stage (leaf nb): one CTA per listed item, grid cap.
void launch_gemm_f64_batched(int nb, const ProdDesc* prods, const int* tile_list, const int* tile_count, int cap,
                             const int* all_done, cudaStream_t st);
// Cull of every product of a stage: blocks[b] = (product, first output tile, blocks of the product, index
// of b among them), 8 output tiles per block; tile_list / tile_count (kTileBuckets classes of stride cap,
// counts zero on entry) get the listed items.
void launch_cull_batched(const ProdDesc* prods, const int4* blocks, int nblocks, int* tile_list, int* tile_count,
                         int cap, const int* all_done, cudaStream_t st);
// Quadtree levels of every product output of a stage (one block per product), the stage's class counters
// cleared; with x_stage the per-matrix trace error, iteration count and stop, and the batch's end
// (all_done, and the graph condition when cond is set).  stage_ctr: one int, zero between launches.
void launch_tree_batched(const ProdDesc* prods, int nprod, int* tile_count, int* stage_ctr, int* ndone, int count,
                         int* all_done, const cudaGraphConditionalHandle* cond, bool x_stage, cudaStream_t st);
// The batched solve engine (spamm_batch.cu): SPAMM_ERR_UNSUPPORTED when the per-matrix path must serve
// the call (options it does not cover, pageable host memory, or a batch larger than the free memory).
int batched_solve(int count, const double* const* S, const int* n, const double* tau, int maxit,
                  double* const* Y, double* const* Z, const spamm_opts& o, spamm_stats* stats);
void release_batches();
// One solve on the batched engine (SPAMM_SCHED_STAGES); SPAMM_ERR_UNSUPPORTED when it does not cover the call.
int stage_solve(const double* S, int n, double tau, int maxit, double* Y, double* Z, const spamm_opts& o,
                spamm_stats* stats);
// Caller-owned batches (the request server's workers): the same engine with buffers and graph kept per slot;
// limit caps the slot's device memory (0: 70 % of the free memory).
struct BatchSlot;
BatchSlot* batch_slot_create();
void batch_slot_destroy(BatchSlot* s);
// statuses (may be null): every problem's own status.
int batched_solve_slot(BatchSlot* s, int count, const double* const* S, const int* n, const double* tau, int maxit,
                       double* const* Y, double* const* Z, const spamm_opts& o, spamm_stats* stats, size_t limit,
                       int* statuses);
bool batch_engine_covers(const spamm_opts& o);
size_t batch_footprint(int n, int nb, int precision, int maxit);
// Digit slices of the items a batched leaf-product launch drew (slice_items, count at slice_items[cap]).
void launch_slice_batched(const ProdDesc* prods, const int* slice_items, int cap, const int* all_done,
                          cudaStream_t st);

// ---- kernels_emu.cu (leaf tile 64 only) -----------------------------------
size_t emu_slice_bytes_per_tile();  // bytes of one tile's slices in one operand role
// Row/column magnitude maxima of a packed matrix (arrays must be zeroed first).
void launch_rowcol_max(const double* X, const Geometry& g, unsigned long long* rmax, unsigned long long* cmax,
                       cudaStream_t st);
// FP16 digit slices of both operand roles from FP64 tiles and row/column maxima,
// for the listed tiles (or all tiles when tile_list is null).  With leaf_out
// null, tiles whose leaf[] norm is zero are skipped, and so are those below
// skip_factor * (*skip_root) when skip_root is set (a matrix whose products all
// cull at tau >= tau_min never reads a tile with nu < tau_min^2 * nu_root: see
// the prologue); with leaf_out set, every listed tile is sliced and its squared
// Frobenius norm written to leaf_out.
void launch_slice(const double* X, const double* leaf, double* leaf_out, const unsigned long long* rmax,
                  const unsigned long long* cmax, uint8_t* sA, uint8_t* sB, const Geometry& g, const int* tile_list,
                  const int* tile_count, const int* done, cudaStream_t st, const double* skip_root = nullptr,
                  double skip_factor = 0.0);
// Leaf products on the tensor cores; writes C's FP64 tiles, leaf norms
// (FP32 sums of squares, about 1e-6 relative), row/column maxima
// (pre-zeroed), trace partials for EPI_NS_X, and C.slice_list; *err set on a
// timed-out internal wait.  units (may be null) gets += the (stack, slice)
// units issued: twelve 128 x 64 x 64 FP16 products per task.  stall_polls > 0
// makes every CTA first wait that many polls on a barrier nothing arrives at:
// the expired-wait path (error 5 in *err, no copy or product issued, tensor
// memory freed, no tile handed to the slicing pass).
// sched: two ints, zero before the first launch; the kernel leaves them zero.
// Leaf-product layout of single products: alternating accumulator columns (true) or one fixed block.
// mode -1 = by size, 0 = never, 1 = always.
void set_emu_alternate(int mode);
bool emu_alternate(int m);
void launch_gemm_emu(const Geometry& g, const TileMat& A, const TileMat& B, const TileMat& C, const int* counts,
                     const int* jlist, const int* tile_list, const int* tile_count, EpiMode mode, double* trace_part,
                     int* sched, const int* done, int* err, double tau, cudaStream_t st, int buckets = 1,
                     unsigned long long* units = nullptr, long long stall_polls = 0);

}  // namespace spamm

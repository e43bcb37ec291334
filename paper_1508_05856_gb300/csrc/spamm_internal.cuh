// Internal declarations of libspamm: geometry of the tile grid and quadtree,
// device buffers of one problem, and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

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
// BF16 slices in the operand-A and operand-B layouts and the magnitude
// maxima (IEEE bits) of its rows and columns.
struct TileMat {
    double* t = nullptr;
    double* tree = nullptr;
    uint8_t* sliceA = nullptr;
    uint8_t* sliceB = nullptr;
    unsigned long long* rmax = nullptr;  // [m*nb], followed by
    unsigned long long* cmax = nullptr;  // [m*nb]
};

// Geometry passed by value to kernels.
struct TreeDev {
    int m, L, coarse, shift;
    int dim[kMaxLevels];
    long off[kMaxLevels];
};
TreeDev tree_dev(const Geometry& g);

enum EpiMode { EPI_PLAIN = 0, EPI_NS_X = 1 };

// Counts kernel launches (spamm_kernel_launches); every launcher calls it.
void note_launch(int k = 1);

// ---- kernels_tree.cu -------------------------------------------------------
// c = max_i sum_j |s_ij + mu delta_ij|; mu read from *mu_dev (may be null = 0).
void launch_gershgorin(const double* S, int n, const double* mu_dev, double* rowsum, double* out_c,
                       cudaStream_t st);
// *mu_out = mu_rel * (*c0)
void launch_scale_mu(const double* c0, double mu_rel, double* mu_out, cudaStream_t st);
// Row-major src -> tile-major dst with leaf norms.  When scale_c != null:
// dst = (src + mu delta) / c.  Edge padding is zero.
void launch_pack(const double* src, int n, const Geometry& g, const double* mu, const double* scale_c,
                 TileMat dst, cudaStream_t st);
// T = 1.5 I_n - 0.5 X elementwise on tiles (logical identity), with leaf norms.
void launch_hmap(const double* X, const Geometry& g, TileMat T, cudaStream_t st);
// Z = I_n in tile-major form, with leaf norms.
void launch_identity(const Geometry& g, TileMat Z, cudaStream_t st);
// Upper quadtree levels from the leaf level.
void launch_tree(const Geometry& g, double* tree, const int* done, cudaStream_t st);
// Task lists of A (x) B: counts[i*m+k], jlist[(i*m+k)*m + ...] ascending j.
// thr = ((tau*tau) * rootA) * rootB.  total (may be null) gets += task count.
void launch_cull(const Geometry& g, const double* treeA, const double* treeB, double tau, int* counts,
                 int* jlist, unsigned long long* total, double* thr_out, const int* done, cudaStream_t st);
// Tile-major -> row-major with out = in * (*mul) or in / (*div) (one of them null or both null).
void launch_unpack(const double* src, const Geometry& g, double* dst, const double* mul, const double* div,
                   cudaStream_t st);
// t_k = (n - sum trace_part)/n into hist[k]; done/iters bookkeeping.
void launch_tk(const double* trace_part, const Geometry& g, int k, double tol_t, double* t_hist, int* done,
               int* iters, cudaStream_t st);
// sqrt of device scalar: out = sqrt(*c)
void launch_sqrt_scalar(const double* c, double* out, cudaStream_t st);
// sum over logical entries of (R - I)^2 -> *out (deterministic)
void launch_resid_norm(const double* R, const Geometry& g, double* partial, double* out, cudaStream_t st);

// ---- kernels_f64.cu --------------------------------------------------------
// C_ik = sum_{j in list(i,k)} A_ij B_jk in FP64 (dense = every j), epilogue
// per mode; writes leaf norms of the stored tile into treeC[0..m*m) and, for
// EPI_NS_X, the diagonal-tile trace partials of X.
void launch_gemm_f64(const Geometry& g, const double* A, const double* B, double* C, double* treeC,
                     const int* counts, const int* jlist, int dense, EpiMode mode, double* trace_part,
                     const int* done, cudaStream_t st);

// ---- kernels_emu.cu (leaf tile 64 only) -----------------------------------
size_t emu_slice_bytes_per_tile();  // bytes of one tile's slices in one operand role
// Row/column magnitude maxima of a packed matrix (arrays must be zeroed first).
void launch_rowcol_max(const double* X, const Geometry& g, unsigned long long* rmax, unsigned long long* cmax,
                       cudaStream_t st);
// BF16 slices of both operand roles from FP64 tiles and row/column maxima.
void launch_slice(const double* X, const double* leaf, const unsigned long long* rmax, const unsigned long long* cmax,
                  uint8_t* sA, uint8_t* sB, const Geometry& g, const int* done, cudaStream_t st);
// Leaf products on the tensor cores; writes C's FP64 tiles, leaf norms and
// row/column maxima (pre-zeroed), trace partials for EPI_NS_X; *err set on a
// timed-out internal wait.
void launch_gemm_emu(const Geometry& g, const TileMat& A, const TileMat& B, const TileMat& C, const int* counts,
                     const int* jlist, EpiMode mode, double* trace_part, const int* done, int* err, cudaStream_t st);

}  // namespace spamm

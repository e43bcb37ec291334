// FP64 leaf-tile products of the SpAMM path (Eq. (newspamm): only the
// surviving a^i . b^i leaf products are formed).
//
// One CTA per output tile (i, k) walks the task list of that tile, j
// ascending, and accumulates C_ik = sum_j A_ij B_jk with FP64 fused
// multiply-adds in registers: no atomics, a fixed order, so results are
// deterministic.  Output tiles with an empty list are written as zeros.
// The epilogue stores the tile, its squared Frobenius norm (the quadtree leaf
// of the product, Sec. 1), and for the X product of the Newton-Schulz
// iteration it stores T = h[X] = 1.5 I - 0.5 X instead of X together with the
// diagonal-tile trace partials of X (for t_k, Sec. 4.2).
#include "spamm_internal.cuh"

namespace spamm {

namespace {

constexpr int kThreads = 256;
constexpr int kKC = 32;  // inner-dimension chunk staged in shared memory

template <int NB>
__global__ void __launch_bounds__(kThreads) k_gemm_f64(const double* __restrict__ A, const double* __restrict__ B,
                                                       double* __restrict__ C, const double* __restrict__ leafA,
                                                       const double* __restrict__ leafB, double* __restrict__ leafC,
                                                       const int* __restrict__ counts, const int* __restrict__ jlist,
                                                       const int* __restrict__ tile_list,
                                                       const int* __restrict__ tile_count, int buckets, int m, int n,
                                                       int dense,
                                                       int mode, double* __restrict__ trace_part,
                                                       const int* __restrict__ done) {
    grid_dependency_wait();
    if (done && *done) return;
    if (tile_list && (int)blockIdx.x >= listed_total(tile_count, buckets)) return;
    constexpr int TM = NB / 16;  // each thread owns TM x TM outputs
    constexpr int LDS = NB + 1;  // padded row of the staged chunks
    extern __shared__ double smem[];
    double* As = smem;              // [kKC][LDS]  A chunk, transposed (k-major)
    double* Bs = smem + kKC * LDS;  // [kKC][LDS]  B chunk
    __shared__ double red[8];

    const int tile = tile_list ? listed_tile(tile_list, tile_count, buckets, m * m, (int)blockIdx.x) : (int)blockIdx.x;
    const int i = tile / m, k = tile - (tile / m) * m;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int nt = dense ? m : counts[tile];
    const int* js = jlist + (size_t)tile * m;

    double acc[TM][TM];
#pragma unroll
    for (int p = 0; p < TM; ++p)
#pragma unroll
        for (int q = 0; q < TM; ++q) acc[p][q] = 0.0;

    for (int t = 0; t < nt; ++t) {
        const int j = dense ? t : js[t];
        // an operand tile with zero norm contributes exact zeros (and its data may be stale)
        if (!dense && (leafA[(size_t)i * m + j] == 0.0 || leafB[(size_t)j * m + k] == 0.0)) continue;
        const double* Aij = A + ((size_t)i * m + j) * NB * NB;
        const double* Bjk = B + ((size_t)j * m + k) * NB * NB;
        for (int kc = 0; kc < NB; kc += kKC) {
            for (int idx = threadIdx.x; idx < NB * kKC; idx += kThreads) {
                const int r = idx / kKC, kk = idx - r * kKC;
                As[kk * LDS + r] = Aij[(size_t)r * NB + kc + kk];
            }
            for (int idx = threadIdx.x; idx < kKC * NB; idx += kThreads) {
                const int kk = idx / NB, c = idx - kk * NB;
                Bs[kk * LDS + c] = Bjk[(size_t)(kc + kk) * NB + c];
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kKC; ++kk) {
                double a[TM], b[TM];
#pragma unroll
                for (int p = 0; p < TM; ++p) a[p] = As[kk * LDS + ty + 16 * p];
#pragma unroll
                for (int q = 0; q < TM; ++q) b[q] = Bs[kk * LDS + tx + 16 * q];
#pragma unroll
                for (int p = 0; p < TM; ++p)
#pragma unroll
                    for (int q = 0; q < TM; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
            }
            __syncthreads();
        }
    }

    double* Ct = C + (size_t)tile * NB * NB;
    double nu = 0.0, tr = 0.0;
#pragma unroll
    for (int p = 0; p < TM; ++p)
#pragma unroll
        for (int q = 0; q < TM; ++q) {
            const int r = ty + 16 * p, c = tx + 16 * q;
            const int gi = i * NB + r, gj = k * NB + c;
            double v = acc[p][q];
            if (mode != EPI_PLAIN) {
                const bool diag = (gi == gj) && (gi < n);
                if (diag) tr += v;
                if (mode == EPI_NS_X) v = diag ? 1.5 - 0.5 * v : -0.5 * v;
            }
            Ct[(size_t)r * NB + c] = v;
            nu = fma(v, v, nu);
        }
    // fixed-order block reductions
    for (int o = 16; o > 0; o >>= 1) nu += __shfl_xor_sync(0xffffffffu, nu, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nu;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        leafC[tile] = s;
    }
    if (mode != EPI_PLAIN && i == k) {
        __syncthreads();
        for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += red[w];
            trace_part[i] = s;
        }
    }
}

template <int NB>
void launch_nb(const Geometry& g, const double* A, const double* B, double* C, const double* leafA,
               const double* leafB, double* treeC, const int* counts, const int* jlist, const int* tile_list,
               const int* tile_count, int dense, EpiMode mode, double* trace_part, const int* done, cudaStream_t st,
               int buckets) {
    const size_t smem = 2 * (size_t)kKC * (NB + 1) * sizeof(double);
    launch_dependent(k_gemm_f64<NB>, dim3(g.m * g.m), dim3(kThreads), smem, st, A, B, C, leafA, leafB, treeC, counts,
                     jlist, tile_list, tile_count, buckets, g.m, g.n, dense, (int)mode, trace_part, done);
    note_launch();
}

template <int NB>
void set_attr() {
    const size_t smem = 2 * (size_t)kKC * (NB + 1) * sizeof(double);
    cudaFuncSetAttribute(k_gemm_f64<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

void f64_kernel_attributes() {
    set_attr<32>();
    set_attr<64>();
    set_attr<128>();
}

void launch_gemm_f64(const Geometry& g, const double* A, const double* B, double* C, const double* leafA,
                     const double* leafB, double* treeC, const int* counts, const int* jlist, const int* tile_list,
                     const int* tile_count, int dense, EpiMode mode, double* trace_part, const int* done,
                     cudaStream_t st, int buckets) {
    switch (g.nb) {
        case 32:
            launch_nb<32>(g, A, B, C, leafA, leafB, treeC, counts, jlist, tile_list, tile_count, dense, mode,
                          trace_part, done, st, buckets);
            break;
        case 64:
            launch_nb<64>(g, A, B, C, leafA, leafB, treeC, counts, jlist, tile_list, tile_count, dense, mode,
                          trace_part, done, st, buckets);
            break;
        case 128:
            launch_nb<128>(g, A, B, C, leafA, leafB, treeC, counts, jlist, tile_list, tile_count, dense, mode,
                           trace_part, done, st, buckets);
            break;
        default: break;
    }
}

}  // namespace spamm

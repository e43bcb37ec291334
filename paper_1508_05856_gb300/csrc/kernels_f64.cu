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

// Batched form (kBatched): the listed entries are items (p << kItemShift) | tile of the products prods[p]
// (class stride cap), and every operand, output and size comes from prods[p].
template <int NB, bool kBatched>
__global__ void __launch_bounds__(kThreads) k_gemm_f64(const double* __restrict__ A0, const double* __restrict__ B0,
                                                       double* __restrict__ C0, const double* __restrict__ leafA0,
                                                       const double* __restrict__ leafB0, double* __restrict__ leafC0,
                                                       const int* __restrict__ counts0, const int* __restrict__ jlist0,
                                                       const int* __restrict__ tile_list,
                                                       const int* __restrict__ tile_count, int buckets, int m0, int n0,
                                                       int dense,
                                                       int mode0, double* __restrict__ trace_part0,
                                                       const int* __restrict__ done,
                                                       const ProdDesc* __restrict__ prods, int cap) {
    grid_dependency_wait();
    if (done && *done) return;
    if (tile_list && (int)blockIdx.x >= listed_total(tile_count, buckets)) return;
    const double* A = A0;
    const double* B = B0;
    double* C = C0;
    const double* leafA = leafA0;
    const double* leafB = leafB0;
    double* leafC = leafC0;
    const int* counts = counts0;
    const int* jlist = jlist0;
    int m = m0, n = n0, mode = mode0;
    double* trace_part = trace_part0;
    int tile;
    if constexpr (kBatched) {
        const int item = listed_tile(tile_list, tile_count, buckets, cap, (int)blockIdx.x);
        const ProdDesc& d = prods[item_prod(item)];
        tile = item_tile(item);
        A = d.At;
        B = d.Bt;
        C = d.Ct;
        leafA = d.Atree;
        leafB = d.Btree;
        leafC = d.Ctree;
        counts = d.counts;
        jlist = d.jlist;
        m = d.td.m;
        n = d.n;
        mode = d.mode;
        trace_part = d.trace_part;
    } else {
        tile = tile_list ? listed_tile(tile_list, tile_count, buckets, m * m, (int)blockIdx.x) : (int)blockIdx.x;
    }
    constexpr int TM = NB / 16;  // each thread owns TM x TM outputs
    constexpr int LDS = NB + 1;  // padded row of the staged chunks
    extern __shared__ double smem[];
    double* As = smem;              // [kKC][LDS]  A chunk, transposed (k-major)
    double* Bs = smem + kKC * LDS;  // [kKC][LDS]  B chunk
    __shared__ double red[8];

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
    launch_dependent(k_gemm_f64<NB, false>, dim3(g.m * g.m), dim3(kThreads), smem, st, A, B, C, leafA, leafB, treeC,
                     counts, jlist, tile_list, tile_count, buckets, g.m, g.n, dense, (int)mode, trace_part, done,
                     (const ProdDesc*)nullptr, 0);
    note_launch();
}

template <int NB>
void launch_batched_nb(const ProdDesc* prods, const int* tile_list, const int* tile_count, int cap,
                       const int* all_done, cudaStream_t st) {
    const size_t smem = 2 * (size_t)kKC * (NB + 1) * sizeof(double);
    launch_dependent(k_gemm_f64<NB, true>, dim3(cap), dim3(kThreads), smem, st, (const double*)nullptr,
                     (const double*)nullptr, (double*)nullptr, (const double*)nullptr, (const double*)nullptr,
                     (double*)nullptr, (const int*)nullptr, (const int*)nullptr, tile_list, tile_count,
                     kTileBuckets, 0, 0, 0, 0, (double*)nullptr, all_done, prods, cap);
    note_launch();
}

template <int NB>
void set_attr() {
    const size_t smem = 2 * (size_t)kKC * (NB + 1) * sizeof(double);
    cudaFuncSetAttribute(k_gemm_f64<NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_gemm_f64<NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

void launch_gemm_f64_batched(int nb, const ProdDesc* prods, const int* tile_list, const int* tile_count, int cap,
                             const int* all_done, cudaStream_t st) {
    switch (nb) {
        case 32: launch_batched_nb<32>(prods, tile_list, tile_count, cap, all_done, st); break;
        case 64: launch_batched_nb<64>(prods, tile_list, tile_count, cap, all_done, st); break;
        case 128: launch_batched_nb<128>(prods, tile_list, tile_count, cap, all_done, st); break;
        default: break;
    }
}

}  // namespace spamm

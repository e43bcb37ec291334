// SPAMM_EMU64: FP64-class SpAMM leaf products on the BF16 tensor cores.
//
// Why: the dual-channel iteration (Eq. (cannonical)) does not damp errors
// injected into its products, so a 1e-8 residual needs products accurate to
// about FP64; GB300 has little FP64 throughput but a large BF16 one.  Every
// matrix is therefore held both as FP64 tiles and as six 8-bit "slices":
//
//   x ~ 2^e * sum_{p=0..5} d_p 2^{-8(p+1)},  balanced digits |d_p| <= 128
//                                            (|d_0| <= 256), error <= 2^{-49} 2^e
//
// where 2^e bounds the largest magnitude of x's row (operand A role) or of
// x's column (operand B role) over the whole matrix.  Each digit times its
// power of two is exact in BF16.  A product of slices p and q is a sum over
// 64 terms of integers of magnitude <= 2^16 in units of 2^{-8(p+q+2)}, so the
// FP32 tensor-core accumulator holds these partial sums exactly (below 2^24
// even for the two pairs that share an accumulator group).  Per output
// tile and per task the partial sums are moved from TMEM to registers in five
// groups (top-half diagonals p+q = 0, 1, 2, 3 exactly, and >= 4 rounded to
// 2^{-48}) and added, as integers, into a 64-bit fixed-point accumulator with
// quantum 2^{-48} relative to 2^{e_row + e_col}.  The dropped pairs
// p+q >= 6 and the truncated digits contribute below ~2^{-46} relative to
// the row/column scales: a normwise FP64-class product.
//
// Layout (no swizzle, K-major canonical core matrices of 8 rows x 16 bytes,
// core (row_group, k_group) at ((row_group * 8 + k_group) * 128) bytes):
//   A role: per tile 3 stacks of 128 x 64 bf16; stack s = slices 2s (rows
//           0-63) and 2s+1 (rows 64-127) of the tile, K = tile column.
//   B role: per tile 6 slices of 64 x 64 bf16, stored transposed (row =
//           tile column c = MMA N index, K = tile row).
// One M=128, N=64, K=16 MMA (stack s, slice q) yields slice pairs (2s, q) in
// TMEM lanes 0-63 and (2s+1, q) in lanes 64-127.
#include <cuda_bf16.h>

#include "spamm_internal.cuh"
#include "tc_ptx.cuh"

namespace spamm {
namespace emu {

constexpr int NB = 64;
constexpr int NSLICE = 6;
constexpr uint32_t A_STACK_BYTES = 128 * 64 * 2;
constexpr uint32_t A_TILE_BYTES = 3 * A_STACK_BYTES;
constexpr uint32_t B_SLICE_BYTES = 64 * 64 * 2;
constexpr uint32_t B_TILE_BYTES = NSLICE * B_SLICE_BYTES;
constexpr uint32_t STAGE_BYTES = A_TILE_BYTES + B_TILE_BYTES;
constexpr int NSTAGE = 2;
constexpr uint32_t SMEM_DYN = NSTAGE * STAGE_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 512;
constexpr int kThreads = 192;
constexpr int kMaxTasks = 1024;
constexpr long long kSpin = 1ll << 22;

// exponent e with |x| < 2^e for every x of a row/column whose largest
// magnitude has the IEEE bits `bits` (0 for an all-zero or subnormal row)
__device__ __forceinline__ int expo_of(unsigned long long bits) {
    const int E = (int)((bits >> 52) & 0x7FF);
    return E == 0 ? 0 : E - 1022;
}

// x * 2^-e rounded to a signed fixed-point integer with 48 fractional bits
// (|result| <= 2^48 because |x| < 2^e).
__device__ __forceinline__ long long fixed48(double x, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0 || E == 0x7FF) return 0ll;
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int s = e + 1027 - E;  // >= 5 when |x| < 2^e
    if (s >= 64) return 0ll;
    const long long F = s < 5 ? (long long)(1ull << 48) : (long long)((M + (1ull << (s - 1))) >> s);
    return (b >> 63) ? -F : F;
}

// Balanced signed base-256 digits of F = sum_p d_p 2^{8(5-p)}: |d_p| <= 128
// for p >= 1 and |d_0| <= 256, so every digit times 2^{-8(p+1)} is exact in
// BF16 and the truncation error is symmetric.
__device__ __forceinline__ void balanced_digits(long long F, int (&d)[6]) {
#pragma unroll
    for (int p = 5; p >= 1; --p) {
        const int lo = (int)((F & 0xFF) ^ 0x80) - 0x80;
        d[p] = lo;
        F = (F - lo) >> 8;
    }
    d[0] = (int)F;
}

__device__ __forceinline__ __nv_bfloat16 digit_bf16(int d, int p) {
    const float scale = __int_as_float((127 - 8 * (p + 1)) << 23);  // 2^{-8(p+1)}
    return __float2bfloat16_rn((float)d * scale);
}

// ------------------------------------------------------------------ slicing
// Leaf tiles with nu == 0 are skipped: the leaf-product kernel never reads
// them (their products are exactly zero).
__global__ void __launch_bounds__(256) k_slice(const double* __restrict__ X, const double* __restrict__ leaf,
                                               const unsigned long long* __restrict__ rmax,
                                               const unsigned long long* __restrict__ cmax,
                                               uint8_t* __restrict__ sA, uint8_t* __restrict__ sB, int m,
                                               const int* __restrict__ done) {
    if (done && *done) return;
    const int tile = blockIdx.x;
    if (leaf[tile] == 0.0) return;
    __shared__ double xs[NB][NB + 1];
    __shared__ int eR[NB], eC[NB];
    const int i = tile / m, j = tile - (tile / m) * m;
    const double* x = X + (size_t)tile * NB * NB;
    for (int idx = threadIdx.x; idx < NB * NB; idx += 256) xs[idx >> 6][idx & 63] = x[idx];
    if (threadIdx.x < NB) eR[threadIdx.x] = expo_of(rmax[i * NB + threadIdx.x]);
    else if (threadIdx.x < 2 * NB) eC[threadIdx.x - NB] = expo_of(cmax[j * NB + threadIdx.x - NB]);
    __syncthreads();
    uint8_t* a = sA + (size_t)tile * A_TILE_BYTES;
    uint8_t* b = sB + (size_t)tile * B_TILE_BYTES;
    for (int item = threadIdx.x; item < 2 * 512; item += 256) {
        const bool arole = item < 512;
        const int it = arole ? item : item - 512;
        const int r = it >> 3, g = it & 7;  // A: row r, k-group g; B: column r, k-group g
        int D[8][6];
        for (int q = 0; q < 8; ++q) {
            const double v = arole ? xs[r][8 * g + q] : xs[8 * g + q][r];
            balanced_digits(fixed48(v, arole ? eR[r] : eC[r]), D[q]);
        }
        for (int p = 0; p < NSLICE; ++p) {
            __align__(16) __nv_bfloat16 w[8];
            for (int q = 0; q < 8; ++q) w[q] = digit_bf16(D[q][p], p);
            uint32_t off;
            if (arole) {
                const int row = (p & 1) * 64 + r;
                off = (uint32_t)(p >> 1) * A_STACK_BYTES + (uint32_t)(((row >> 3) * 8 + g) * 128 + (row & 7) * 16);
                *reinterpret_cast<uint4*>(a + off) = *reinterpret_cast<const uint4*>(w);
            } else {
                off = (uint32_t)p * B_SLICE_BYTES + (uint32_t)(((r >> 3) * 8 + g) * 128 + (r & 7) * 16);
                *reinterpret_cast<uint4*>(b + off) = *reinterpret_cast<const uint4*>(w);
            }
        }
    }
}

// Row and column magnitude maxima (as IEEE bits) of a packed FP64 matrix.
__global__ void __launch_bounds__(256) k_rowcol_max(const double* __restrict__ X, int m,
                                                    unsigned long long* __restrict__ rmax,
                                                    unsigned long long* __restrict__ cmax) {
    __shared__ unsigned long long xs[NB][NB + 1];
    const int tile = blockIdx.x;
    const int i = tile / m, j = tile - (tile / m) * m;
    const double* x = X + (size_t)tile * NB * NB;
    for (int idx = threadIdx.x; idx < NB * NB; idx += 256)
        xs[idx >> 6][idx & 63] = (unsigned long long)__double_as_longlong(fabs(x[idx]));
    __syncthreads();
    if (threadIdx.x < NB) {
        unsigned long long mx = 0;
        for (int c = 0; c < NB; ++c) mx = max(mx, xs[threadIdx.x][c]);
        if (mx) atomicMax(rmax + i * NB + threadIdx.x, mx);
    } else if (threadIdx.x < 2 * NB) {
        const int c = threadIdx.x - NB;
        unsigned long long mx = 0;
        for (int r = 0; r < NB; ++r) mx = max(mx, xs[r][c]);
        if (mx) atomicMax(cmax + j * NB + c, mx);
    }
}

// ------------------------------------------------------------------ leaf products
struct EmuArgs {
    const uint8_t* sliceA;              // A-role slices of the left operand
    const uint8_t* sliceB;              // B-role slices of the right operand
    const double* leafA;                // leaf norms (quadtree leaf level)
    const double* leafB;
    const unsigned long long* rmaxA;    // row maxima of the left operand
    const unsigned long long* cmaxB;    // column maxima of the right operand
    double* C;                          // FP64 output tiles
    double* leafC;
    unsigned long long* rmaxC;          // output row / column maxima (pre-zeroed)
    unsigned long long* cmaxC;
    const int* counts;
    const int* jlist;
    double* trace_part;
    const int* done;
    int* err;
    int m, n, mode;
};

__device__ __forceinline__ uint32_t stage_addr(uint32_t base, int s) { return base + (uint32_t)s * STAGE_BYTES; }

__global__ void __launch_bounds__(kThreads, 1) k_gemm_emu(const EmuArgs a) {
    if (a.done && *a.done) return;
    extern __shared__ uint8_t dyn_smem[];
    __shared__ __align__(8) uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accf, bar_acce;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int tasks_sh[kMaxTasks];
    __shared__ int ntask_sh;
    __shared__ int eA_sh[NB], eB_sh[NB];
    __shared__ double red_sh[4];

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = ptx::smem_addr(smem);
    const int m = a.m;
    const int tile = blockIdx.x;
    const int i = tile / m, k = tile - (tile / m) * m;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        const int cnt = a.counts[tile];
        const int* js = a.jlist + (size_t)tile * m;
        int T = 0;
        for (int t = 0; t < cnt; ++t) {
            const int j = js[t];
            if (a.leafA[(size_t)i * m + j] != 0.0 && a.leafB[(size_t)j * m + k] != 0.0) tasks_sh[T++] = j;
        }
        ntask_sh = T;
        for (int s = 0; s < NSTAGE; ++s) {
            ptx::mbar_init(&bar_full[s], 1);
            ptx::mbar_init(&bar_empty[s], 1);
        }
        ptx::mbar_init(&bar_accf, 1);
        ptx::mbar_init(&bar_acce, 4);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < NB) eA_sh[threadIdx.x] = expo_of(a.rmaxA[i * NB + threadIdx.x]);
    else if (threadIdx.x < 2 * NB) eB_sh[threadIdx.x - NB] = expo_of(a.cmaxB[k * NB + threadIdx.x - NB]);
    if (warp == 0) {
        ptx::tmem_alloc(&tmem_base_sh, TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int T = ntask_sh;

    if (warp == 0) {
        // ---------------- producer: bulk copies of the slices of A_ij and B_jk
        if (lane == 0) {
            for (int t = 0; t < T; ++t) {
                const int s = t & 1;
                if (t >= 2 && !ptx::mbar_wait_bounded(&bar_empty[s], ((t >> 1) & 1) ^ 1, kSpin)) {
                    atomicExch(a.err, 1);
                    break;
                }
                const int j = tasks_sh[t];
                uint8_t* dst = smem + (size_t)s * STAGE_BYTES;
                ptx::mbar_arrive_expect_tx(&bar_full[s], STAGE_BYTES);
                ptx::bulk_g2s(dst, a.sliceA + ((size_t)i * m + j) * A_TILE_BYTES, A_TILE_BYTES, &bar_full[s]);
                ptx::bulk_g2s(dst + A_TILE_BYTES, a.sliceB + ((size_t)j * m + k) * B_TILE_BYTES, B_TILE_BYTES,
                              &bar_full[s]);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = ptx::idesc_bf16_f32(128, 64);
            // (stack, slice) pairs in the order of their accumulator group: the
            // group is the diagonal 2*stack + slice of the top half, capped at 4
            const int8_t ps[12] = {0, 0, 0, 1, 0, 1, 0, 0, 1, 1, 2, 2};
            const int8_t qs[12] = {0, 1, 2, 0, 3, 1, 4, 5, 2, 3, 0, 1};
            for (int t = 0; t < T; ++t) {
                const int s = t & 1;
                if (!ptx::mbar_wait_bounded(&bar_full[s], (t >> 1) & 1, kSpin)) {
                    atomicExch(a.err, 2);
                    break;
                }
                // the accumulators are single-buffered: wait until the epilogue read task t-1
                if (t >= 1 && !ptx::mbar_wait_bounded(&bar_acce, (t - 1) & 1, kSpin)) {
                    atomicExch(a.err, 3);
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t sA = stage_addr(sbase, s), sB = sA + A_TILE_BYTES;
                int prev_g = -1;
                for (int u = 0; u < 12; ++u) {
                    const int sg = ps[u], q = qs[u];
                    const int g = min(2 * sg + q, 4);
                    const uint32_t d = tmem + (uint32_t)(g * 64);
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = ptx::smem_desc(sA + sg * A_STACK_BYTES + ks * 256, 128, 1024);
                        const uint64_t bd = ptx::smem_desc(sB + q * B_SLICE_BYTES + ks * 256, 128, 1024);
                        // the first MMA into a group overwrites it, the rest accumulate
                        ptx::mma_bf16(d, ad, bd, idesc, (ks > 0 || g == prev_g) ? 1u : 0u);
                        prev_g = g;
                    }
                }
                ptx::mma_commit(&bar_empty[s]);
                ptx::mma_commit(&bar_accf);
            }
        }
    }

    // ---------------- epilogue warps 2..5: TMEM lanes 32*(warp%4) + lane
    long long acc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = 0;
    const int quarter = warp & 3;
    const int half = quarter >> 1;  // 0: rows 0-63 of the MMA (even slices), 1: rows 64-127 (odd slices)
    if (warp >= 2) {
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        for (int t = 0; t < T; ++t) {
            if (!ptx::mbar_wait_bounded(&bar_accf, t & 1, kSpin)) {
                atomicExch(a.err, 4);
                break;
            }
            ptx::tc_fence_after();
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                // exact integer partial sums of diagonal g + half in units 2^{-8(diag+2)}
                const int diag = g + half;
                const float up = __int_as_float((127 + 8 * (diag + 2)) << 23);
                const int sh = 32 - 8 * diag;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t r[32];
                    ptx::tmem_ld32(lane_base + (uint32_t)(g * 64 + h * 32), r);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const int v = __float2int_rn(__uint_as_float(r[c]) * up);
                        acc[h * 32 + c] += (long long)v << sh;
                    }
                }
            }
            {
                // diagonals >= 4 (top) / >= 5 (bottom): rounded to the 2^{-48} quantum
                const float up48 = __int_as_float((127 + 48) << 23);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t r[32];
                    ptx::tmem_ld32(lane_base + (uint32_t)(4 * 64 + h * 32), r);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int c = 0; c < 32; ++c) acc[h * 32 + c] += (long long)__float2int_rn(__uint_as_float(r[c]) * up48);
                }
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&bar_acce);
        }
        // combine the odd-slice half (rows 64-127) into the even half (rows 0-63)
        long long* comb = reinterpret_cast<long long*>(smem);  // [64][65] int64; stage memory is idle now
        const int row = (quarter & 1) * 32 + lane;
        if (half == 1) {
#pragma unroll
            for (int c = 0; c < NB; ++c) comb[c * 65 + row] = acc[c];
        }
        ptx::named_sync(1, 128);
        double nu = 0.0, tr = 0.0;
        unsigned long long* colbuf = reinterpret_cast<unsigned long long*>(smem + 65 * 64 * 8);  // [64][65]
        if (half == 0) {
            const int gi = i * NB + row;
            const int eAr = eA_sh[row];
            double* out = a.C + (size_t)tile * NB * NB + (size_t)row * NB;
            unsigned long long rmx = 0;
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                const long long tot = acc[c] + comb[c * 65 + row];
                double x = (double)tot;
                if (tot != 0) {
                    long long bits = __double_as_longlong(x);
                    bits += (long long)(eAr + eB_sh[c] - 48) << 52;
                    x = __longlong_as_double(bits);
                }
                const int gj = k * NB + c;
                double v = x;
                if (a.mode == EPI_NS_X) {
                    const bool dg = (gi == gj) && (gi < a.n);
                    if (dg) tr += x;
                    v = dg ? 1.5 - 0.5 * x : -0.5 * x;
                }
                out[c] = v;
                nu = fma(v, v, nu);
                const unsigned long long vb = (unsigned long long)__double_as_longlong(fabs(v));
                rmx = max(rmx, vb);
                colbuf[c * 65 + row] = vb;
            }
            if (rmx) atomicMax(a.rmaxC + gi, rmx);
        }
        ptx::named_sync(1, 128);
        if (half == 0) {
            // column maxima: thread `row` reduces column `row`
            unsigned long long cmx = 0;
            for (int r = 0; r < NB; ++r) cmx = max(cmx, colbuf[row * 65 + r]);
            if (cmx) atomicMax(a.cmaxC + k * NB + row, cmx);
            // fixed-order reductions of nu and the trace over the 64 rows (2 warps)
            for (int o = 16; o > 0; o >>= 1) {
                nu += __shfl_xor_sync(0xffffffffu, nu, o);
                tr += __shfl_xor_sync(0xffffffffu, tr, o);
            }
            if (lane == 0) {
                red_sh[quarter & 1] = nu;
                red_sh[2 + (quarter & 1)] = tr;
            }
        }
        ptx::named_sync(1, 128);
        if (warp >= 2 && half == 0 && (quarter & 1) == 0 && lane == 0) {
            a.leafC[tile] = red_sh[0] + red_sh[1];
            if (a.mode == EPI_NS_X && i == k) a.trace_part[i] = red_sh[2] + red_sh[3];
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) ptx::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace emu

size_t emu_slice_bytes_per_tile() { return emu::A_TILE_BYTES; }

void launch_rowcol_max(const double* X, const Geometry& g, unsigned long long* rmax, unsigned long long* cmax,
                       cudaStream_t st) {
    emu::k_rowcol_max<<<g.m * g.m, 256, 0, st>>>(X, g.m, rmax, cmax);
    note_launch();
}

void launch_slice(const double* X, const double* leaf, const unsigned long long* rmax, const unsigned long long* cmax,
                  uint8_t* sA, uint8_t* sB, const Geometry& g, const int* done, cudaStream_t st) {
    emu::k_slice<<<g.m * g.m, 256, 0, st>>>(X, leaf, rmax, cmax, sA, sB, g.m, done);
    note_launch();
}

void launch_gemm_emu(const Geometry& g, const TileMat& A, const TileMat& B, const TileMat& C, const int* counts,
                     const int* jlist, EpiMode mode, double* trace_part, const int* done, int* err, cudaStream_t st) {
    emu::EmuArgs a;
    a.sliceA = A.sliceA;
    a.sliceB = B.sliceB;
    a.leafA = A.tree;
    a.leafB = B.tree;
    a.rmaxA = A.rmax;
    a.cmaxB = B.cmax;
    a.C = C.t;
    a.leafC = C.tree;
    a.rmaxC = C.rmax;
    a.cmaxC = C.cmax;
    a.counts = counts;
    a.jlist = jlist;
    a.trace_part = trace_part;
    a.done = done;
    a.err = err;
    a.m = g.m;
    a.n = g.n;
    a.mode = (int)mode;
    cudaFuncSetAttribute(emu::k_gemm_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emu::SMEM_DYN);
    emu::k_gemm_emu<<<g.m * g.m, emu::kThreads, emu::SMEM_DYN, st>>>(a);
    note_launch();
}

}  // namespace spamm

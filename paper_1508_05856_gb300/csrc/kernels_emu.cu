// SPAMM_EMU64: FP64-class SpAMM leaf products on the 16-bit tensor cores.
//
// Why: the dual-channel iteration (Eq. (cannonical)) does not damp errors
// injected into its products, so a 1e-8 residual needs products accurate to
// about FP64; GB300 has little FP64 throughput but a large FP16/BF16 one.  Every
// matrix is therefore held both as FP64 tiles and as six 8-bit "slices":
//
//   x ~ 2^e * sum_{p=0..5} d_p 2^{-8(p+1)},  balanced digits |d_p| <= 128,
//                                            error <= 2^{-49} 2^e,
//
// where 2^(e-1) bounds the largest magnitude of x's row (operand A role) or
// of x's column (operand B role) over the whole matrix.  A slice holds the
// digits d_p themselves, integers that FP16 represents exactly; the power of
// two of a slice pair is applied when its partial sums leave TMEM.  A product
// of slices p and q is a sum over 64 terms of integers of magnitude <= 2^14
// (weight 2^{-8(p+q+2)}): at most 2^20 per pair and task, 2^21 for the two
// pairs that share an accumulator group.  The FP32 tensor-core accumulators in TMEM therefore hold the sums
// of up to 7 tasks exactly (7 * 2^21 < 2^24).  Every 7 tasks (and at the end
// of an output tile) the partial sums are moved from TMEM to registers in
// six groups (diagonals p+q <= 3 exactly, the groups of diagonal >= 4 added
// in FP32 and rounded to 2^{-48}) and added, as integers, into a 64-bit
// fixed-point accumulator
// with quantum 2^{-48} relative to 2^{e_row + e_col}.  Dropped pairs
// (p+q >= 6, except the (1,5), (3,3), (5,1) that come with the stacking) and
// the digit truncation leave an error of a few 2^{-48} per product term
// relative to 2^{e_row + e_col}: a normwise FP64-class product.
//
// Method: this is an instance of the Ozaki scheme (Ozaki, Ogita, Oishi and
// Rump, 2012: split each FP64 operand into slices that a low-precision unit
// multiplies exactly, and sum the slice products at higher precision), in the
// integer-slice form that shares one power of two per row of A and per
// column of B (Ootomo, Ozaki and Yokota, 2024).  The digit width, the
// balanced digits, the pair set, the stacking into M = 128 and the flush
// schedule above are this library's own, fitted to FP16 inputs, FP32 TMEM
// accumulators and 64 x 64 leaf tiles; so is the error model.
//
// Layout (no swizzle, K-major canonical core matrices of 8 rows x 16 bytes;
// per K-half of 32, core (row_group, k_group) at ((row_group * 4 + k_group) *
// 128) bytes, so the descriptors use LBO = 128 and SBO = 512):
//   A role: per tile and K-half 3 stacks of 128 x 32 fp16; stack s = slices
//           2s (rows 0-63) and 2s+1 (rows 64-127), K = tile column.
//   B role: per tile and K-half 6 slices of 64 x 32 fp16, stored transposed
//           (row = tile column c = MMA N index, K = tile row).
// The B slices of a K-half are consecutive 64-column blocks of one N-major
// operand, so one M=128, N=64n, K=16 MMA (stack s, slices q0 .. q0+n-1)
// yields the slice pairs (2s, q) in TMEM lanes 0-63 and (2s+1, q) in lanes
// 64-127 for n slices at once.  Accumulator group g = 2s + q (the top-half
// diagonal) sits at TMEM columns 64g .. 64g+63, so the pairs of one stack land
// in consecutive groups and four MMAs per K step cover all twelve pairs:
// stack 0 with slices 0-3 and 4-5, stack 1 with 0-3, stack 2 with 0-1.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

#include "spamm_internal.cuh"
#include "tc_ptx.cuh"

namespace spamm {
namespace emu {

constexpr int NB = 64;
constexpr int NSLICE = 6;
// One task is split into two K-halves of 32.  Per tile and operand role the
// slices are stored as [K-half][stack or slice][core matrices], so a half-task's
// A data and B data are each one contiguous 24 KB block.
constexpr uint32_t A_HALF_STACK = 128 * 32 * 2;          // 128 rows x 32 K
constexpr uint32_t A_HALF_BYTES = 3 * A_HALF_STACK;      // 3 stacks
constexpr uint32_t A_TILE_BYTES = 2 * A_HALF_BYTES;
constexpr uint32_t B_HALF_SLICE = 64 * 32 * 2;           // 64 columns x 32 K
constexpr uint32_t B_HALF_BYTES = NSLICE * B_HALF_SLICE;  // 6 slices
constexpr uint32_t B_TILE_BYTES = 2 * B_HALF_BYTES;
constexpr uint32_t STAGE_BYTES = A_HALF_BYTES + B_HALF_BYTES;
constexpr int NSTAGE = 3;
constexpr uint32_t EPI_BYTES = 2 * 64 * 65 * 8;          // epilogue staging of the two 64-bit halves
constexpr uint32_t SMEM_DYN = NSTAGE * STAGE_BYTES + EPI_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 512;
constexpr int kEpiWarps = 16;                // four per TMEM lane quarter (16 output columns each)
constexpr int kSchedWarp = 2 + kEpiWarps;   // prepares the tiles' task lists and scales
constexpr int kThreads = 32 * (3 + kEpiWarps);
constexpr int NSLOT = 3;                     // tiles in flight: streamed, prepared, being prepared
constexpr int kGroups = 6;                   // accumulator groups (64 TMEM columns each)
constexpr int kChunk = 7;                    // tasks accumulated in TMEM between flushes (exactness bound)
// tasks of one output tile: at most m, and the API limits SPAMM_EMU64 to m <= 512
constexpr int kMaxTasks = 512;

// exponent e with |x| < 2^(e-1) for every x of a row/column whose largest
// magnitude has the IEEE bits `bits` (0 for an all-zero or subnormal row):
// the scaled entries x * 2^-e lie in (-1/2, 1/2), so every balanced digit,
// the leading one included, is at most 128 in magnitude.
__device__ __forceinline__ int expo_of(unsigned long long bits) {
    const int E = (int)((bits >> 52) & 0x7FF);
    return E == 0 ? 0 : E - 1021;
}

// |x| * 2^(48-e) rounded (half up) to an integer, from the IEEE bits of x and
// se = e + 1027: the shift s = se - E is at least 6 for every entry of a row
// (column) whose largest magnitude defines e, so |F| <= 2^47.  Zeros give 0;
// a shift beyond 63 gives 0.
__device__ __forceinline__ unsigned long long fixed48_mag(unsigned long long b, int se) {
    const unsigned hw = (unsigned)(b >> 32);
    const int E = (int)((hw >> 20) & 0x7FFu);
    const unsigned long long M = E ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : 0ull;
    const int s = min(se - E, 63);
    return ((M >> (s - 1)) + 1ull) >> 1;
}

// Balanced signed base-256 digits of F = sum_p d_p 2^{8(5-p)}: |d_p| <= 128
// (d_p in [-128, 127] for p >= 1), so the truncation error is symmetric.  The
// slicing pass takes the digits of |F| (then 0 <= d_0 <= 128) and negates
// them for a negative entry: still |d_p| <= 128.  Adding 0x80 to each of the
// five low bytes of F turns them into plain bytes d_p + 128 (p = 1..5, byte
// 5-p of G); byte 5 of G is d_0 itself.
struct Digits {
    unsigned lo;  // bytes d_5+128, d_4+128, d_3+128, d_2+128
    unsigned hi;  // byte 0: d_1 + 128, byte 1: d_0
};
__device__ __forceinline__ Digits balanced_digits(unsigned long long F) {
    const unsigned long long G = F + 0x8080808080ull;
    return Digits{(unsigned)G, (unsigned)(G >> 32)};
}
// Digit P of two entries (a: low half, b: high half) as a packed FP16 pair,
// exact: the two bytes go into the FP16 magic pattern 1024 + byte (unit 1),
// and one fused multiply-add by (s_a, s_b) = +-1 with addend -1152 s (bias
// 128 removed; -1024 s for the unbiased top digit) yields s * d_P.
// sgn: bit 15 / bit 31 set for a negative entry a / b.
template <int P>
__device__ __forceinline__ uint32_t digit_pair_f16(const Digits& a, const Digits& b, uint32_t sgn) {
    uint32_t t;
    if (P == 0) t = __byte_perm(a.hi, b.hi, 0x0501);
    else if (P == 1) t = __byte_perm(a.hi, b.hi, 0x0400);
    else t = __byte_perm(a.lo, b.lo, (5 - P) | ((9 - P) << 8));
    const uint32_t mag = (t & 0x00FF00FFu) | 0x64006400u;
    const uint32_t sc = 0x3C003C00u ^ sgn;                                  // (s_a, s_b)
    const uint32_t add = (P == 0 ? 0xE400E400u : 0xE480E480u) ^ sgn;       // -1024 s or -1152 s
    const __half2 r = __hfma2(*reinterpret_cast<const __half2*>(&mag), *reinterpret_cast<const __half2*>(&sc),
                              *reinterpret_cast<const __half2*>(&add));
    return *reinterpret_cast<const uint32_t*>(&r);
}

// The 512 items of one operand role of a staged tile, two per thread: item `it` covers row (A role) or
// column (B role) r and k-group g, 8 entries, i.e. 16 bytes of every slice.  8 consecutive items fill one
// 128-byte core matrix, 32 consecutive items 512 contiguous bytes.  The role is a template parameter, so
// the entries are read and moved as bit patterns with no per-entry selects.
template <bool kA>
__device__ __forceinline__ void slice_role(const double (*xs)[NB + 1], const int* e, uint8_t* dst) {
#pragma unroll 1
    for (int it = threadIdx.x; it < 512; it += 256) {
        const int kgi = (it >> 3) & 3, kh = (it >> 5) & 1;
        const int r = (it >> 6) * 8 + (it & 7), g = kh * 4 + kgi;  // A: row r, k-group g; B: column r, k-group g
        // digits of |F| with F = round(|x| 2^(48-e)); the sign goes onto the FP16 digits afterwards
        Digits D[8];
        unsigned neg = 0;
        const int se = e[r] + 1027;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const unsigned long long bq =
                (unsigned long long)__double_as_longlong(kA ? xs[r][8 * g + q] : xs[8 * g + q][r]);
            neg |= (unsigned)(bq >> 63) << q;
            D[q] = balanced_digits(fixed48_mag(bq, se));
        }
        uint8_t* const base = dst + (uint32_t)kh * (kA ? A_HALF_BYTES : B_HALF_BYTES) +
                              (uint32_t)(((r >> 3) * 4 + kgi) * 128 + (r & 7) * 16);
        // FP16 sign bits of element pairs (2h, 2h+1): bit 15 and bit 31 of word h
        const uint32_t m0 = ((neg & 1u) << 15) | ((neg & 2u) << 30);
        const uint32_t m1 = ((neg & 4u) << 13) | ((neg & 8u) << 28);
        const uint32_t m2 = ((neg & 16u) << 11) | ((neg & 32u) << 26);
        const uint32_t m3 = ((neg & 64u) << 9) | ((neg & 128u) << 24);
        // A role: slice p sits in stack p/2, rows 64 (p%2) + r (the odd rows 8 row groups, 4 KB, further on);
        // B role: slice p is the p-th 64-column block
#define SPAMM_STORE_SLICE(P)                                                                                 \
        {                                                                                                    \
            uint4 w;                                                                                         \
            w.x = digit_pair_f16<P>(D[0], D[1], m0);                                                         \
            w.y = digit_pair_f16<P>(D[2], D[3], m1);                                                         \
            w.z = digit_pair_f16<P>(D[4], D[5], m2);                                                         \
            w.w = digit_pair_f16<P>(D[6], D[7], m3);                                                         \
            constexpr uint32_t off = kA ? (uint32_t)(P >> 1) * A_HALF_STACK + (uint32_t)(P & 1) * 4096u       \
                                        : (uint32_t)P * B_HALF_SLICE;                                        \
            *reinterpret_cast<uint4*>(base + off) = w;                                                       \
        }
        SPAMM_STORE_SLICE(0)
        SPAMM_STORE_SLICE(1)
        SPAMM_STORE_SLICE(2)
        SPAMM_STORE_SLICE(3)
        SPAMM_STORE_SLICE(4)
        SPAMM_STORE_SLICE(5)
#undef SPAMM_STORE_SLICE
    }
}

// ------------------------------------------------------------------ slicing
// Grid-stride over the listed tiles (tile_list / tile_count), or over all
// m*m tiles when tile_list is null.  With leaf_out null, leaf tiles with
// nu == 0 are skipped (the leaf-product kernel never reads them: their
// products are exactly zero).  With leaf_out set, the kernel also computes
// each listed tile's squared Frobenius norm nu (FP64 fused multiply-adds, a
// fixed-order reduction) into leaf_out[tile]; unlisted tiles keep the zero
// the cull wrote for them.
// Batched form (kBatched): tile_list holds items (p << kItemShift) | tile of the products prods[p], whose
// outputs are sliced; leaf_out is null.
template <bool kBatched>
__global__ void __launch_bounds__(256, 5) k_slice(const double* __restrict__ X0, const double* __restrict__ leaf0,
                                               double* __restrict__ leaf_out,
                                               const unsigned long long* __restrict__ rmax0,
                                               const unsigned long long* __restrict__ cmax0,
                                               uint8_t* __restrict__ sA0, uint8_t* __restrict__ sB0, int m0,
                                               const int* __restrict__ tile_list, const int* __restrict__ tile_count,
                                               const int* __restrict__ done, const ProdDesc* __restrict__ prods,
                                               const double* __restrict__ skip_root, double skip_factor) {
    grid_dependency_wait();
    if (done && *done) return;
    const double skip_below = skip_root ? skip_factor * *skip_root : 0.0;
    __shared__ double xs[NB][NB + 1];
    __shared__ int eR[NB], eC[NB];
    __shared__ double nu_sh[8];
    const int ntiles = tile_list ? *tile_count : m0 * m0;
    for (int idx = blockIdx.x; idx < ntiles; idx += gridDim.x) {
    const int item = tile_list ? tile_list[idx] : idx;
    int tile = item, m = m0;
    const double* X = X0;
    const double* leaf = leaf0;
    const unsigned long long* rmax = rmax0;
    const unsigned long long* cmax = cmax0;
    uint8_t* sA = sA0;
    uint8_t* sB = sB0;
    if constexpr (kBatched) {
        const ProdDesc& d = prods[item_prod(item)];
        tile = item_tile(item);
        m = d.td.m;
        X = d.Ct;
        leaf = d.Ctree;
        rmax = d.Crmax;
        cmax = d.Ccmax;
        sA = d.CsliceA;
        sB = d.CsliceB;
    }
    if (!leaf_out) {
        const double nu = leaf[tile];
        if (nu == 0.0 || nu < skip_below) continue;
    }
    __syncthreads();
    const int i = tile / m, j = tile - (tile / m) * m;
    const double* x = X + (size_t)tile * NB * NB;
    double nup[2] = {0.0, 0.0};
    // two batches of eight independent loads per thread
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = x[threadIdx.x + 256 * (8 * h + q)];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int idx = threadIdx.x + 256 * (8 * h + q);
            xs[idx >> 6][idx & 63] = v[q];
            if (leaf_out) nup[q & 1] = fma(v[q], v[q], nup[q & 1]);
        }
    }
    if (leaf_out) {
        double nu = nup[0] + nup[1];
        for (int o = 16; o > 0; o >>= 1) nu += __shfl_xor_sync(0xffffffffu, nu, o);
        if ((threadIdx.x & 31) == 0) nu_sh[threadIdx.x >> 5] = nu;
    }
    if (threadIdx.x < NB) eR[threadIdx.x] = expo_of(rmax[i * NB + threadIdx.x]);
    else if (threadIdx.x < 2 * NB) eC[threadIdx.x - NB] = expo_of(cmax[j * NB + threadIdx.x - NB]);
    __syncthreads();
    if (leaf_out && threadIdx.x == 0) {
        // pairwise, fixed order
        const double s01 = nu_sh[0] + nu_sh[1], s23 = nu_sh[2] + nu_sh[3];
        const double s45 = nu_sh[4] + nu_sh[5], s67 = nu_sh[6] + nu_sh[7];
        leaf_out[tile] = (s01 + s23) + (s45 + s67);
    }
    slice_role<true>(xs, eR, sA + (size_t)tile * A_TILE_BYTES);
    slice_role<false>(xs, eC, sB + (size_t)tile * B_TILE_BYTES);
    }
}

// Row and column magnitude maxima of a packed FP64 matrix, kept as the upper 32 bits of the IEEE pattern
// (sign cleared), which carry the exponent exactly: the maxima feed only the slicing exponents.  Warp w
// takes rows 8w .. 8w+7 of a 64 x 64 tile and lane l the columns l and l + 32, sixteen independent loads
// per thread; rows reduce across the warp, columns across the eight warps in shared memory.
__global__ void __launch_bounds__(256) k_rowcol_max(const double* __restrict__ X, int m,
                                                    unsigned long long* __restrict__ rmax,
                                                    unsigned long long* __restrict__ cmax) {
    __shared__ unsigned cm_sh[8][NB];
    const int tile = blockIdx.x;
    const int i = tile / m, j = tile - (tile / m) * m;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long* x = reinterpret_cast<const unsigned long long*>(X + (size_t)tile * NB * NB);
    unsigned long long a[8], b[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        a[q] = x[(8 * w + q) * NB + lane];
        b[q] = x[(8 * w + q) * NB + 32 + lane];
    }
    unsigned ca = 0, cb = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const unsigned ha = (unsigned)(a[q] >> 32) & 0x7FFFFFFFu, hb = (unsigned)(b[q] >> 32) & 0x7FFFFFFFu;
        ca = max(ca, ha);
        cb = max(cb, hb);
        const unsigned rm = __reduce_max_sync(0xffffffffu, max(ha, hb));
        if (lane == 0 && rm) atomicMax(rmax + i * NB + 8 * w + q, (unsigned long long)rm << 32);
    }
    cm_sh[w][lane] = ca;
    cm_sh[w][lane + 32] = cb;
    __syncthreads();
    if (threadIdx.x < NB) {
        unsigned mx = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) mx = max(mx, cm_sh[q][threadIdx.x]);
        if (mx) atomicMax(cmax + j * NB + threadIdx.x, (unsigned long long)mx << 32);
    }
}

// ------------------------------------------------------------------ leaf products
struct EmuArgs {
    const uint8_t* sliceA;              // A-role slices of the left operand
    const uint8_t* sliceB;              // B-role slices of the right operand
    const double* leafA;                // leaf norms (quadtree leaf level)
    const double* leafB;
    const double* rootA;                // quadtree roots: thr = ((tau*tau) * rootA) * rootB as in the cull
    const double* rootB;
    double tau;
    const unsigned long long* rmaxA;    // row maxima of the left operand
    const unsigned long long* cmaxB;    // column maxima of the right operand
    unsigned long long* units;          // (stack, slice) units issued, summed over the launch (may be null)
    double* C;                          // FP64 output tiles
    double* leafC;                      // output leaf norms (squared Frobenius, FP32 sums)
    int* slice_list;                    // copy of the drawn tiles ([m*m] ids, count at [m*m]) for slicing
    unsigned long long* rmaxC;          // output row / column maxima (pre-zeroed)
    unsigned long long* cmaxC;
    const int* counts;
    const int* jlist;
    const int* tile_list;               // compacted output tiles with work, in `buckets` cost classes
    const int* tile_count;              // [buckets]
    int buckets;
    int* sched;                         // [2] tile ticket counter and finished-CTA counter, zero between launches
    double* trace_part;
    const int* done;
    int* err;
    int m, n, mode;
    // batched form: per-item products (items (p << kItemShift) | tile in tile_list, kTileBuckets classes of
    // stride cap); the drawn items go to slice_items (count at slice_items[cap])
    const ProdDesc* prods;
    int* slice_items;
    int cap;
    long long poll_limit;   // polls of every internal wait before it expires
    long long stall_polls;  // > 0: every CTA first waits this long on a barrier nothing arrives at (the
                            // expired-wait path, taken with nothing in flight)
};

// What the producer warp needs of an output tile's product.
struct ProducerView {
    int m;
    const int* counts;
    const int* jlist;
    const uint8_t* sliceA;
    const uint8_t* sliceB;
    const double* leafA;
    const double* leafB;
    const unsigned long long* rmaxA;
    const unsigned long long* cmaxB;
    bool zero_filter;  // thr = 0: listed tasks may have an exactly zero operand, skipped
};
template <bool kBatched>
__device__ __forceinline__ ProducerView producer_view(const EmuArgs& a, int prod) {
    if constexpr (kBatched) {
        const ProdDesc& d = a.prods[prod];
        const double rA = d.Atree[d.td.off[0]], rB = d.Btree[d.td.off[0]];
        return ProducerView{d.td.m, d.counts, d.jlist, d.AsliceA, d.BsliceB, d.Atree, d.Btree, d.Armax, d.Bcmax,
                            !(((d.tau * d.tau) * rA) * rB > 0.0)};
    } else {
        return ProducerView{a.m, a.counts, a.jlist, a.sliceA, a.sliceB, a.leafA, a.leafB, a.rmaxA, a.cmaxB,
                            !(((a.tau * a.tau) * *a.rootA) * *a.rootB > 0.0)};
    }
}
// What the epilogue warps need of an output tile's product.
struct EpiView {
    int m, n, mode;
    double* C;
    double* leafC;
    unsigned long long* rmaxC;
    unsigned long long* cmaxC;
    double* trace_part;
};
template <bool kBatched>
__device__ __forceinline__ EpiView epi_view(const EmuArgs& a, int prod) {
    if constexpr (kBatched) {
        const ProdDesc& d = a.prods[prod];
        return EpiView{d.td.m, d.n, d.mode, d.Ct, d.Ctree, d.Crmax, d.Ccmax, d.trace_part};
    } else {
        return EpiView{a.m, a.n, a.mode, a.C, a.leafC, a.rmaxC, a.cmaxC, a.trace_part};
    }
}

__device__ __forceinline__ uint32_t stage_addr(uint32_t base, int s) { return base + (uint32_t)s * STAGE_BYTES; }

// int64 -> double as integer operations (round to nearest even), times 2^s;
// results below the normal range flush to zero.
__device__ __forceinline__ double fixed_to_double(long long tot, int s) {
    if (tot == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)tot & 0x8000000000000000ull;
    const unsigned long long u = sign ? 0ull - (unsigned long long)tot : (unsigned long long)tot;
    const int lz = __clzll(u);
    const unsigned long long mnorm = u << lz;  // leading one at bit 63
    const unsigned long long keep = mnorm >> 11;  // 53 bits, leading one at bit 52
    const unsigned rem = (unsigned)mnorm & 0x7FFu;
    const unsigned up = (rem + 0x3FFu + ((unsigned)keep & 1u)) >> 11;  // round half to even
    const int ef = 62 - lz + s + 1023;  // the leading one of keep adds the missing 1 to the exponent field
    if (ef < 0) return 0.0;
    // a rounding carry out of the 52 mantissa bits moves into the exponent field
    const unsigned long long bits = ((unsigned long long)ef << 52) + keep + up;
    return __longlong_as_double((long long)(bits | sign));
}

// IEEE bits of |fixed_to_double(tot, s)|, branch-free (0 for tot = 0 and for a flushed result); the
// caller supplies the sign.
__device__ __forceinline__ unsigned long long fixed_mag_bits(long long tot, int s) {
    const unsigned long long u = tot < 0 ? 0ull - (unsigned long long)tot : (unsigned long long)tot;
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const int lz = hw ? __clz(hw) : 32 + __clz(lw);
    const unsigned long long mnorm = u << (lz & 63);
    const unsigned long long keep = mnorm >> 11;
    const unsigned rem = (unsigned)mnorm & 0x7FFu;
    const unsigned up = (rem + 0x3FFu + ((unsigned)keep & 1u)) >> 11;
    const int ef = 62 - lz + s + 1023;
    const unsigned long long bits = ((unsigned long long)(unsigned)ef << 52) + keep + up;
    return (u == 0 || ef < 0) ? 0ull : bits;
}

// Move one chunk's accumulator groups from TMEM into the 64-bit fixed-point
// sums (unit 2^{-48}) of this thread's row (16 of the 64 output columns).
// Group g holds integer sums of digit products of weight 2^{-8(diag+2)},
// diag = g + half (half = 1 for the odd-slice lanes).  Groups of diagonal
// 0..3 are exact integers, shifted left by 32 - 8 diag.  The groups of
// diagonal >= 4 (weight <= one unit) are added in FP32 first and converted
// once: |sum| < 2^25 units, so the FP32 additions and the final rounding cost
// at most 1.5 units per chunk, the size of the quantum itself.
// The loads are double-buffered: load g+1 is in flight while g is converted.
template <int SH>
__device__ __forceinline__ void flush_exact(const uint32_t (&r)[16], int h, long long (&acc)[16]) {
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[h * 16 + c] += (long long)__float2int_rn(__uint_as_float(r[c])) << SH;
}
__device__ __forceinline__ uint32_t col16(uint32_t base, int g, int h) { return base + (uint32_t)(g * 64 + h * 16); }
__device__ __forceinline__ void flush_groups(uint32_t lane_col_base, int half, long long (&acc)[16]) {
    static_assert(kGroups == 6, "flush schedule written for six groups");
    const uint32_t b = lane_col_base;
    uint32_t ra[16], rb[16];
#pragma unroll
    for (int h = 0; h < 1; ++h) {
        ptx::tmem_ld16(col16(b, 0, h), ra);
        ptx::tmem_ld_wait(ra);
        if (half == 0) {
            // diagonals 0, 1, 2, 3 exact; 4 + 5/2^8 rounded
            ptx::tmem_ld16(col16(b, 1, h), rb);
            flush_exact<32>(ra, h, acc);
            ptx::tmem_ld_wait(rb);
            ptx::tmem_ld16(col16(b, 2, h), ra);
            flush_exact<24>(rb, h, acc);
            ptx::tmem_ld_wait(ra);
            ptx::tmem_ld16(col16(b, 3, h), rb);
            flush_exact<16>(ra, h, acc);
            ptx::tmem_ld_wait(rb);
            ptx::tmem_ld16(col16(b, 4, h), ra);
            flush_exact<8>(rb, h, acc);
            ptx::tmem_ld_wait(ra);
            ptx::tmem_ld16(col16(b, 5, h), rb);
            ptx::tmem_ld_wait(rb);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                acc[h * 16 + c] += (long long)__float2int_rn(
                    fmaf(__uint_as_float(rb[c]), 0x1p-8f, __uint_as_float(ra[c])));
        } else {
            // diagonals 1, 2, 3 exact; 4 + 5/2^8 + 6/2^16 rounded
            ptx::tmem_ld16(col16(b, 1, h), rb);
            flush_exact<24>(ra, h, acc);
            ptx::tmem_ld_wait(rb);
            ptx::tmem_ld16(col16(b, 2, h), ra);
            flush_exact<16>(rb, h, acc);
            ptx::tmem_ld_wait(ra);
            ptx::tmem_ld16(col16(b, 3, h), rb);
            flush_exact<8>(ra, h, acc);
            ptx::tmem_ld_wait(rb);
            ptx::tmem_ld16(col16(b, 4, h), ra);
            ptx::tmem_ld_wait(ra);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                rb[c] = __float_as_uint(fmaf(__uint_as_float(ra[c]), 0x1p-8f, __uint_as_float(rb[c])));
            ptx::tmem_ld16(col16(b, 5, h), ra);
            ptx::tmem_ld_wait(ra);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                acc[h * 16 + c] += (long long)__float2int_rn(
                    fmaf(__uint_as_float(ra[c]), 0x1p-16f, __uint_as_float(rb[c])));
        }
    }
}

// The alternating layout (kernel instances with kAlt): the chunks of a tile of more than one chunk sit at
// TMEM columns 0-383 and 128-511 in turn, so the next chunk overwrites only four of this chunk's six
// groups.  The epilogue reads those four first and releases the accumulator (release()), then reads the
// other two while the next chunk's products already run: with many tasks per tile the MMA warp then waits
// for two thirds of a flush instead of all of it.  kNextHigh: this chunk sits at 0-383 and the next at
// 128-511 (groups 2-5 are shared); otherwise this chunk sits at 128-511 and the next at 0-383 (groups 0-3
// are shared).  The integer sums are the same in any order; the groups of diagonal >= 4 are combined in
// FP32 exactly as flush_groups does, so both layouts give the same bits.
// Each load completes before the next is issued: overlapping them as flush_groups does spills registers in
// this instance and was slower.
__device__ __forceinline__ void tmem_ld16_now(uint32_t taddr, uint32_t (&r)[16]) {
    ptx::tmem_ld16(taddr, r);
    ptx::tmem_ld_wait(r);
}
template <bool kNextHigh, typename Release>
__device__ __forceinline__ void flush_groups_split(uint32_t b, int half, long long (&acc)[16], Release release) {
    uint32_t ra[16], rb[16];
    if (kNextHigh) {
        if (half == 0) {
            tmem_ld16_now(col16(b, 2, 0), ra);
            flush_exact<16>(ra, 0, acc);
            tmem_ld16_now(col16(b, 3, 0), ra);
            flush_exact<8>(ra, 0, acc);
            tmem_ld16_now(col16(b, 4, 0), ra);
            tmem_ld16_now(col16(b, 5, 0), rb);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                acc[c] += (long long)__float2int_rn(fmaf(__uint_as_float(rb[c]), 0x1p-8f, __uint_as_float(ra[c])));
            release();
            tmem_ld16_now(col16(b, 0, 0), ra);
            flush_exact<32>(ra, 0, acc);
            tmem_ld16_now(col16(b, 1, 0), ra);
            flush_exact<24>(ra, 0, acc);
        } else {
            tmem_ld16_now(col16(b, 2, 0), ra);
            flush_exact<8>(ra, 0, acc);
            tmem_ld16_now(col16(b, 3, 0), rb);
            tmem_ld16_now(col16(b, 4, 0), ra);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                rb[c] = __float_as_uint(fmaf(__uint_as_float(ra[c]), 0x1p-8f, __uint_as_float(rb[c])));
            tmem_ld16_now(col16(b, 5, 0), ra);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                acc[c] += (long long)__float2int_rn(fmaf(__uint_as_float(ra[c]), 0x1p-16f, __uint_as_float(rb[c])));
            release();
            tmem_ld16_now(col16(b, 0, 0), ra);
            flush_exact<24>(ra, 0, acc);
            tmem_ld16_now(col16(b, 1, 0), ra);
            flush_exact<16>(ra, 0, acc);
        }
    } else {
        if (half == 0) {
            tmem_ld16_now(col16(b, 0, 0), ra);
            flush_exact<32>(ra, 0, acc);
            tmem_ld16_now(col16(b, 1, 0), ra);
            flush_exact<24>(ra, 0, acc);
            tmem_ld16_now(col16(b, 2, 0), ra);
            flush_exact<16>(ra, 0, acc);
            tmem_ld16_now(col16(b, 3, 0), ra);
            flush_exact<8>(ra, 0, acc);
            release();
            tmem_ld16_now(col16(b, 4, 0), ra);
            tmem_ld16_now(col16(b, 5, 0), rb);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                acc[c] += (long long)__float2int_rn(fmaf(__uint_as_float(rb[c]), 0x1p-8f, __uint_as_float(ra[c])));
        } else {
            tmem_ld16_now(col16(b, 0, 0), ra);
            flush_exact<24>(ra, 0, acc);
            tmem_ld16_now(col16(b, 1, 0), ra);
            flush_exact<16>(ra, 0, acc);
            tmem_ld16_now(col16(b, 2, 0), ra);
            flush_exact<8>(ra, 0, acc);
            tmem_ld16_now(col16(b, 3, 0), rb);  // diagonal 4 of the odd rows: kept for the FP32 combination
            release();
            tmem_ld16_now(col16(b, 4, 0), ra);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                rb[c] = __float_as_uint(fmaf(__uint_as_float(ra[c]), 0x1p-8f, __uint_as_float(rb[c])));
            tmem_ld16_now(col16(b, 5, 0), ra);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                acc[c] += (long long)__float2int_rn(fmaf(__uint_as_float(ra[c]), 0x1p-16f, __uint_as_float(rb[c])));
        }
    }
}

// Polls of the waits that drain an aborted CTA's copies and products before it exits.
constexpr long long kDrainPolls = 1ll << 22;

// Bounded wait that also gives up when another role of this CTA aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                              long long limit) {
    for (long long it = 0; it < limit; ++it) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

// Persistent: one CTA per SM takes output tiles from the compacted list with
// an atomic ticket (a CTA that draws cheap tiles draws more of them).  The
// four roles run decoupled through NSLOT tile slots: the scheduler warp draws
// tiles and writes their task lists and scales up to two tiles ahead, so the
// producer warp streams half-tasks from one tile straight into the next while
// the MMA warp multiplies and the epilogue warps finish the tile before; the
// tile id travels in the slot, and mbarriers order the roles.  The last CTA
// to finish resets the ticket counters for the next launch.
template <bool kBatched, bool kAlt>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_emu(const EmuArgs a) {
    grid_dependency_wait();
    if (a.done && *a.done) return;
    extern __shared__ uint8_t dyn_smem[];
    __shared__ __align__(8) uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accf, bar_acce;
    __shared__ __align__(8) uint64_t bar_tready[NSLOT], bar_tfree[NSLOT];
    __shared__ __align__(8) uint64_t bar_stall, bar_drain;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int tasks_sh[NSLOT][kMaxTasks];
    __shared__ int ntask_sh[NSLOT];
    __shared__ int tile_sh[NSLOT];
    __shared__ int prod_sh[NSLOT];
    __shared__ int eA_sh[NSLOT][NB], eB_sh[NSLOT][NB];
    __shared__ const uint8_t* srcA_sh[NSLOT];  // slices of A_i0 and B_0k; strideB_sh: bytes from B_jk to B_j+1,k
    __shared__ const uint8_t* srcB_sh[NSLOT];
    __shared__ size_t strideB_sh[NSLOT];
    __shared__ double tr_sh[kEpiWarps];
    __shared__ float nu_sh[kEpiWarps];
    __shared__ int abort_sh;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = ptx::smem_addr(smem);
    long long* sTop = reinterpret_cast<long long*>(smem + NSTAGE * STAGE_BYTES);  // [64][65]
    long long* sBot = sTop + NB * 65;                                             // [64][65]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // stride of one cost class in the tile list, and where the drawn tiles are copied for the slicing pass
    const int lstride = kBatched ? a.cap : a.m * a.m;
    int* const drawn = kBatched ? a.slice_items : a.slice_list;
    // bucket counts held in registers: a drawn ticket maps to its tile with one load
    int bcount[kTileBuckets];
    int ntiles = 0;
#pragma unroll
    for (int b = 0; b < kTileBuckets; ++b) {
        bcount[b] = b < a.buckets ? a.tile_count[b] : 0;
        ntiles += bcount[b];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) drawn[lstride] = ntiles;
    if ((int)blockIdx.x >= ntiles) return;

    if (warp == 2 && lane == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            ptx::mbar_init(&bar_full[s], 1);
            ptx::mbar_init(&bar_empty[s], 1);
        }
        ptx::mbar_init(&bar_accf, 1);
        ptx::mbar_init(&bar_acce, kEpiWarps);
        ptx::mbar_init(&bar_stall, 1);
        ptx::mbar_init(&bar_drain, 1);
        for (int q = 0; q < NSLOT; ++q) {
            ptx::mbar_init(&bar_tready[q], 1);
            ptx::mbar_init(&bar_tfree[q], kEpiWarps);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        ptx::tmem_alloc(&tmem_base_sh, TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    volatile int* abort_flag = &abort_sh;
    if (a.stall_polls > 0) {
        // nothing arrives at bar_stall: the wait expires, the CTA records the error and every role stops
        // before issuing a copy or a product
        if (threadIdx.x == 0 && !wait_or_abort(&bar_stall, 0u, abort_flag, a.stall_polls)) atomicExch(a.err, 5);
        __syncthreads();
    }

    if (warp == 0) {
        // ---------------- producer: streams the half-tasks of the tiles the scheduler prepared
        long long H = 0;
        if (lane == 0) {
            for (int tau = 0;; ++tau) {
                const int slot = tau % NSLOT;
                if (!wait_or_abort(&bar_tready[slot], (uint32_t)((tau / NSLOT) & 1), abort_flag, a.poll_limit)) {
                    atomicExch(a.err, 1);
                    break;
                }
                if (tile_sh[slot] < 0) break;
                const int T = ntask_sh[slot];
                const uint8_t* const baseA = srcA_sh[slot];
                const uint8_t* const baseB = srcB_sh[slot];
                const size_t strideB = strideB_sh[slot];
                for (int t = 0; t < T; ++t) {
                    const int j = tasks_sh[slot][t];
                    const uint8_t* srcA = baseA + (size_t)j * A_TILE_BYTES;
                    const uint8_t* srcB = baseB + (size_t)j * strideB;
                    for (int h = 0; h < 2; ++h, ++H) {
                        const int s = (int)(H % NSTAGE);
                        if (H >= NSTAGE &&
                            !wait_or_abort(&bar_empty[s], (uint32_t)(((H / NSTAGE) - 1) & 1), abort_flag, a.poll_limit)) {
                            atomicExch(a.err, 1);
                            break;
                        }
                        uint8_t* dst = smem + (size_t)s * STAGE_BYTES;
                        ptx::mbar_arrive_expect_tx(&bar_full[s], STAGE_BYTES);
                        ptx::bulk_g2s(dst, srcA + h * A_HALF_BYTES, A_HALF_BYTES, &bar_full[s]);
                        ptx::bulk_g2s(dst + A_HALF_BYTES, srcB + h * B_HALF_BYTES, B_HALF_BYTES, &bar_full[s]);
                    }
                    if (*abort_flag) break;
                }
                if (*abort_flag) break;
            }
            // an aborted CTA leaves no copy in flight: wait (bounded) for the last copy issued on every stage
            if (*abort_flag)
                for (int s = 0; s < NSTAGE; ++s)
                    if (H > s) {
                        const long long hl = s + ((H - 1 - s) / NSTAGE) * NSTAGE;
                        ptx::mbar_wait_bounded(&bar_full[s], (uint32_t)((hl / NSTAGE) & 1), kDrainPolls);
                    }
        }
        __syncwarp();
    } else if (warp == kSchedWarp) {
        // ---------------- scheduler: draws tiles and writes each one's task list and scales into a slot, up
        // to two tiles ahead of the one being streamed
        for (int tau = 0;; ++tau) {
            const int slot = tau % NSLOT;
            if (tau >= NSLOT) {
                bool ok = true;
                if (lane == 0)
                    ok = wait_or_abort(&bar_tfree[slot], (uint32_t)(((tau / NSLOT) & 1) ^ 1), abort_flag, a.poll_limit);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) atomicExch(a.err, 1);
                    break;
                }
            }
            // a CTA's first ticket is its block index; later ones come from the counter, after the grid's
            int idx = (int)blockIdx.x;
            if (tau > 0) {
                idx = lane == 0 ? (int)gridDim.x + atomicAdd(a.sched, 1) : 0;
                idx = __shfl_sync(0xffffffffu, idx, 0);
            }
            // lane 0 decides for the warp: the abort flag may change between the lanes' reads
            const int stop = __shfl_sync(0xffffffffu, lane == 0 ? (int)(idx >= ntiles || *abort_flag) : 0, 0);
            if (stop) {
                // no more tiles: the other roles see tile -1 in this slot and stop
                if (lane == 0) {
                    tile_sh[slot] = -1;
                    ptx::mbar_arrive(&bar_tready[slot]);
                }
                break;
            }
            // the first tickets take the cheapest tiles, so every CTA's epilogue starts early; the others take
            // the rest most expensive first (tiles cost the epilogue about the same, the products do not)
            const int g0 = min((int)gridDim.x, ntiles);
            int t = idx < g0 ? ntiles - 1 - idx : idx - g0, b = 0;
#pragma unroll
            for (int q = 0; q < kTileBuckets - 1; ++q)
                if (b == q && t >= bcount[q]) {
                    t -= bcount[q];
                    b = q + 1;
                }
            const int item = a.tile_list[(size_t)b * lstride + t];
            const int prod = kBatched ? item_prod(item) : 0;
            const int tile = kBatched ? item_tile(item) : item;
            const ProducerView v = producer_view<kBatched>(a, prod);
            const int m = v.m;
            const int i = tile / m, k = tile - (tile / m) * m;
            const int cnt = v.counts[tile];
            const int* js = v.jlist + (size_t)tile * m;
            const unsigned long long ra0 = v.rmaxA[i * NB + lane], ra1 = v.rmaxA[i * NB + 32 + lane];
            const unsigned long long cb0 = v.cmaxB[k * NB + lane], cb1 = v.cmaxB[k * NB + 32 + lane];
            int T = 0;
            for (int base = 0; base < cnt; base += 32) {
                const int tt = base + lane;
                bool keep = tt < cnt;
                const int j = keep ? js[tt] : 0;
                // with thr > 0 every listed task has two nonzero operand tiles; with thr = 0 the
                // tasks with an exactly zero operand contribute nothing and are skipped
                if (keep && v.zero_filter) keep = v.leafA[(size_t)i * m + j] != 0.0 && v.leafB[(size_t)j * m + k] != 0.0;
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) tasks_sh[slot][T + __popc(bal & ((1u << lane) - 1u))] = j;
                T += __popc(bal);
            }
            eA_sh[slot][lane] = expo_of(ra0);
            eA_sh[slot][lane + 32] = expo_of(ra1);
            eB_sh[slot][lane] = expo_of(cb0);
            eB_sh[slot][lane + 32] = expo_of(cb1);
            if (lane == 0) {
                ntask_sh[slot] = T;
                tile_sh[slot] = tile;
                prod_sh[slot] = prod;
                srcA_sh[slot] = v.sliceA + (size_t)i * m * A_TILE_BYTES;
                srcB_sh[slot] = v.sliceB + (size_t)k * B_TILE_BYTES;
                strideB_sh[slot] = (size_t)m * B_TILE_BYTES;
                drawn[idx] = item;
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&bar_tready[slot]);  // release: the task list and scales are visible
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: tasks accumulate in TMEM in chunks of kChunk
        if (lane == 0) {
            constexpr uint32_t idesc256 = ptx::idesc_f16_f32(128, 256);
            constexpr uint32_t idesc128 = ptx::idesc_f16_f32(128, 128);
            // descriptors of the other stages and K steps differ from stage 0's by a constant in the address
            // field (shared addresses stay below 2^18, so the 14-bit field never carries)
            const uint64_t dA0 = ptx::smem_desc(stage_addr(sbase, 0), 128, 512);
            const uint64_t dB0 = ptx::smem_desc(stage_addr(sbase, 0) + A_HALF_BYTES, 128, 512);
            constexpr uint64_t kDStage = STAGE_BYTES >> 4, kDK = 256 >> 4, kDStack = A_HALF_STACK >> 4;
            constexpr uint64_t kDSl4 = (4 * B_HALF_SLICE) >> 4;
            long long H = 0, C = 0;
            unsigned long long units = 0;
            int tau = 0;
            bool ok = true;
            for (; ok; ++tau) {
                const int slot = tau % NSLOT;
                if (!wait_or_abort(&bar_tready[slot], (uint32_t)((tau / NSLOT) & 1), abort_flag, a.poll_limit)) {
                    atomicExch(a.err, 2);
                    break;
                }
                if (tile_sh[slot] < 0) break;
                const int T = ntask_sh[slot];
                uint32_t acc0 = tmem;  // kAlt: odd chunks of a tile sit 128 columns on
                for (int t = 0; t < T && ok; ++t) {
                    const bool chunk_start = (t % kChunk) == 0;
                    if (kAlt && chunk_start) acc0 = ((t / kChunk) & 1) ? tmem + 128u : tmem;
                    units += 12;  // twelve stacked (stack, slice) products per task
                    for (int h = 0; h < 2; ++h, ++H) {
                        const int s = (int)(H % NSTAGE);
                        if (!wait_or_abort(&bar_full[s], (uint32_t)((H / NSTAGE) & 1), abort_flag, a.poll_limit)) {
                            atomicExch(a.err, 2);
                            ok = false;
                            break;
                        }
                        // a new chunk overwrites the accumulators: the epilogue must have read the previous one
                        if (chunk_start && h == 0 && C > 0 &&
                            !wait_or_abort(&bar_acce, (uint32_t)((C - 1) & 1), abort_flag, a.poll_limit)) {
                            atomicExch(a.err, 3);
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint64_t dA = dA0 + (uint64_t)s * kDStage, dB = dB0 + (uint64_t)s * kDStage;
                        // the chunk's first K step overwrites groups 0-5 (stack 0 covers them all);
                        // stacks 1 and 2 always accumulate onto it
                        const uint32_t fresh = chunk_start && h == 0;
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {
                            const uint32_t acc = fresh && ks == 0 ? 0u : 1u;
                            const uint64_t a = dA + ks * kDK, b = dB + ks * kDK;
                            ptx::mma_f16(acc0, a, b, idesc256, acc);
                            ptx::mma_f16(acc0 + 256u, a, b + kDSl4, idesc128, acc);
                            ptx::mma_f16(acc0 + 128u, a + kDStack, b, idesc256, 1u);
                            ptx::mma_f16(acc0 + 256u, a + 2 * kDStack, b, idesc128, 1u);
                        }
                        ptx::mma_commit(&bar_empty[s]);
                    }
                    if (ok && ((t % kChunk) == kChunk - 1 || t == T - 1)) {
                        ptx::mma_commit(&bar_accf);
                        ++C;
                    }
                }
            }
            // an aborted CTA leaves no product in flight: commit and wait (bounded) for everything issued
            if (*abort_flag && H > 0) {
                ptx::mma_commit(&bar_drain);
                ptx::mbar_wait_bounded(&bar_drain, 0u, kDrainPolls);
            }
            if (a.units && units) atomicAdd(a.units, units);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps 2..17: TMEM lane quarter warp%4 (lanes 32q .. 32q+31),
        // columns 16*cq .. 16*cq+15 with cq = (warp-2)/4
        const int quarter = warp & 3;
        const int half = quarter >> 1;  // 0: MMA rows 0-63 (even slices), 1: rows 64-127 (odd slices)
        const int cq = (warp - 2) >> 2;
        const int row = (quarter & 1) * 32 + lane;
        const uint32_t lane_col_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cq * 16);
        const int et = threadIdx.x - 64;  // 0..511
        const int ew = warp - 2;          // 0..15
        long long C = 0;
        int tau = 0;
        for (;; ++tau) {
            const int slot = tau % NSLOT;
            if (!wait_or_abort(&bar_tready[slot], (uint32_t)((tau / NSLOT) & 1), abort_flag, a.poll_limit)) {
                atomicExch(a.err, 4);
                break;
            }
            const int tile = tile_sh[slot];
            if (tile < 0) break;
            const EpiView ev = epi_view<kBatched>(a, prod_sh[slot]);
            const int m = ev.m;
            const int i = tile / m, k = tile - (tile / m) * m;
            const int T = ntask_sh[slot];
            const int nchunks = (T + kChunk - 1) / kChunk;
            long long acc[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = 0;
            bool ok = true;
            for (int ck = 0; ck < nchunks; ++ck, ++C) {
                if (!wait_or_abort(&bar_accf, (uint32_t)(C & 1), abort_flag, a.poll_limit)) {
                    atomicExch(a.err, 4);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                auto release = [&] {
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&bar_acce);
                };
                // kAlt: chunk ck of the tile sits at columns 128 (ck & 1) onwards; the tile's next chunk (or the
                // next tile's first, at 0) decides which groups it shares with this one
                const int sel = kAlt ? ck & 1 : 0, next_sel = kAlt && ck + 1 < nchunks ? (ck + 1) & 1 : 0;
                if (!kAlt || sel == next_sel) {
                    flush_groups(lane_col_base, half, acc);
                    release();
                } else if (sel == 0) {
                    flush_groups_split<true>(lane_col_base, half, acc, release);
                } else {
                    flush_groups_split<false>(lane_col_base + 128u, half, acc, release);
                }
            }
            if (!ok) break;
            // stage both halves' 64-bit sums, then finish the tile element-parallel:
            // thread et owns column c and every eighth row
            long long* dst = half ? sBot : sTop;
#pragma unroll
            for (int c = 0; c < 16; ++c) dst[(cq * 16 + c) * 65 + row] = acc[c];
            ptx::named_sync(1, 32 * kEpiWarps);
            const int c = et & 63;
            const int r0 = et >> 6;  // 0..7
            const int gj = k * NB + c;
            const int eBc = eB_sh[slot][c];
            const bool nsx = ev.mode == EPI_NS_X;
            const bool with_tr = ev.mode != EPI_PLAIN;
            // T = 1.5 I - 0.5 X: off the diagonal -x/2 is the conversion of -t64 one binade lower; the one
            // thread per column that owns the diagonal entry computes it up front (and its trace share)
            const int rd = (with_tr && i == k && (c & 7) == r0 && gj < ev.n) ? c : -1;
            double xd = 0.0;
            unsigned long long vdb = 0;  // bits of the diagonal entry of x or T
            if (rd >= 0) {
                xd = fixed_to_double(sTop[c * 65 + c] + sBot[c * 65 + c], eA_sh[slot][c] + eBc - 48);
                vdb = (unsigned long long)__double_as_longlong(nsx ? 1.5 - 0.5 * xd : xd);
            }
            const int sc = eBc - 48 - (nsx ? 1 : 0);
            // the sign of x, or of -x/2 for T: the sign bit of the sum, flipped for T
            const unsigned long long flip = nsx ? 0x8000000000000000ull : 0ull;
            unsigned long long* outb = reinterpret_cast<unsigned long long*>(ev.C) + (size_t)tile * NB * NB;
            unsigned cmx = 0;  // upper words of the column's magnitudes
            float nf = 0.f;
            unsigned rowm = 0;  // lane q: upper magnitude bits of row r0 + 8q over this warp's 32 columns
            long long t64[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) t64[u] = sTop[c * 65 + r0 + 8 * u] + sBot[c * 65 + r0 + 8 * u];
            // the entries are moved as IEEE bit patterns only: no FP64 instruction in the loop
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = r0 + 8 * u;
                unsigned long long vb = fixed_mag_bits(t64[u], eA_sh[slot][r] + sc);
                unsigned long long sb = vb | (vb ? ((unsigned long long)t64[u] ^ flip) & 0x8000000000000000ull : 0ull);
                if (r == rd) {
                    sb = vdb;
                    vb = vdb & 0x7FFFFFFFFFFFFFFFull;
                }
                outb[r * NB + c] = sb;  // consecutive lanes: consecutive columns
                const float f = f32_of_bits(vb);
                nf = fmaf(f, f, nf);
                // the maxima only feed the slicing exponents: the upper 32 bits carry the exponent exactly
                const unsigned hw = (unsigned)(vb >> 32);
                cmx = max(cmx, hw);
                const unsigned rm = __reduce_max_sync(0xffffffffu, hw);
                if (lane == u) rowm = rm;
            }
            // X itself (EPI_X) is not sliced: the maxima are those of the map's output, taken by k_map
            if (ev.mode != EPI_X) {
                if (cmx) atomicMax(ev.cmaxC + gj, (unsigned long long)cmx << 32);
                if (lane < 8 && rowm) atomicMax(ev.rmaxC + i * NB + r0 + 8 * lane, (unsigned long long)rowm << 32);
            }
            for (int o = 16; o > 0; o >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, o);
            if (lane == 0) nu_sh[ew] = nf;
            const bool diag_tile = with_tr && i == k;
            if (diag_tile) {
                double tr = rd >= 0 ? xd : 0.0;
                for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
                if (lane == 0) tr_sh[ew] = tr;
            }
            // every epilogue warp is done with the staging buffer (and tr_sh holds the trace partials)
            ptx::named_sync(1, 32 * kEpiWarps);
            if (ew == 0) {
                float t = lane < kEpiWarps ? nu_sh[lane] : 0.f;
                for (int o = kEpiWarps / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (lane == 0) {
                    ev.leafC[tile] = (double)t;
                    if (diag_tile) {
                        double s8 = 0.0;
                        for (int w = 0; w < kEpiWarps; ++w) s8 += tr_sh[w];
                        ev.trace_part[i] = s8;
                    }
                }
            }
            if (lane == 0) ptx::mbar_arrive(&bar_tfree[slot]);
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) ptx::tmem_dealloc(tmem, TMEM_COLS);
    if (threadIdx.x == 0) {
        // every participating CTA has drawn its last ticket: the last one out resets both counters
        __threadfence();
        const int participants = min((int)gridDim.x, ntiles);
        if (atomicAdd(a.sched + 1, 1) == participants - 1) {
            a.sched[0] = 0;
            a.sched[1] = 0;
            // after an expired wait the drawn-tile list is incomplete: the slicing pass gets none
            if (*a.err) drawn[lstride] = 0;
        }
    }
}

}  // namespace emu

size_t emu_slice_bytes_per_tile() { return emu::A_TILE_BYTES; }

void emu_kernel_attributes() {
    cudaFuncSetAttribute(emu::k_gemm_emu<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emu::SMEM_DYN);
    cudaFuncSetAttribute(emu::k_gemm_emu<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emu::SMEM_DYN);
    cudaFuncSetAttribute(emu::k_gemm_emu<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emu::SMEM_DYN);
}

void launch_rowcol_max(const double* X, const Geometry& g, unsigned long long* rmax, unsigned long long* cmax,
                       cudaStream_t st) {
    emu::k_rowcol_max<<<g.m * g.m, 256, 0, st>>>(X, g.m, rmax, cmax);
    note_launch();
}

void launch_slice(const double* X, const double* leaf, double* leaf_out, const unsigned long long* rmax,
                  const unsigned long long* cmax, uint8_t* sA, uint8_t* sB, const Geometry& g, const int* tile_list,
                  const int* tile_count, const int* done, cudaStream_t st, const double* skip_root,
                  double skip_factor) {
    // five blocks (34 KB shared memory, 48 registers) are resident per SM: one wave, so a dependent launched
    // early never holds slots the grid still needs
    const int grid = std::min(device_sm_count() * 5, g.m * g.m);
    launch_dependent(emu::k_slice<false>, dim3(grid), dim3(256), 0, st, X, leaf, leaf_out, rmax, cmax, sA, sB, g.m,
                     tile_list, tile_count, done, (const ProdDesc*)nullptr, skip_root, skip_factor);
    note_launch();
}

void launch_slice_batched(const ProdDesc* prods, const int* slice_items, int cap, const int* all_done,
                          cudaStream_t st) {
    const int grid = std::min(device_sm_count() * 5, cap);
    launch_dependent(emu::k_slice<true>, dim3(grid), dim3(256), 0, st, (const double*)nullptr,
                     (const double*)nullptr, (double*)nullptr, (const unsigned long long*)nullptr,
                     (const unsigned long long*)nullptr, (uint8_t*)nullptr, (uint8_t*)nullptr, 0, slice_items,
                     slice_items + cap, all_done, prods, (const double*)nullptr, 0.0);
    note_launch();
}

// Which leaf-product layout a single product uses: the alternating one from 128 tiles per side (where this
// library's product-heavy cases live: about 22 tasks per tile on the 3D Gaussian, against 3.4 on the KMS
// headline, whose kernel stays the plain one); spamm_test_emu_alternate forces either.
static std::atomic<int> g_emu_alt_mode{-1};
void set_emu_alternate(int mode) { g_emu_alt_mode.store(mode < 0 ? -1 : (mode ? 1 : 0)); }
bool emu_alternate(int m) {
    const int mode = g_emu_alt_mode.load();
    return mode < 0 ? m >= 128 : mode == 1;
}

void launch_gemm_emu(const Geometry& g, const TileMat& A, const TileMat& B, const TileMat& C, const int* counts,
                     const int* jlist, const int* tile_list, const int* tile_count, EpiMode mode, double* trace_part,
                     int* sched, const int* done, int* err, double tau, cudaStream_t st, int buckets,
                     unsigned long long* units, long long stall_polls) {
    emu::EmuArgs a;
    a.sliceA = A.sliceA;
    a.sliceB = B.sliceB;
    a.leafA = A.tree;
    a.leafB = B.tree;
    a.rootA = A.tree + g.off[0];
    a.rootB = B.tree + g.off[0];
    a.tau = tau;
    a.rmaxA = A.rmax;
    a.cmaxB = B.cmax;
    a.units = units;
    a.C = C.t;
    a.leafC = C.tree;
    a.slice_list = C.slice_list;
    a.rmaxC = C.rmax;
    a.cmaxC = C.cmax;
    a.counts = counts;
    a.jlist = jlist;
    a.tile_list = tile_list;
    a.tile_count = tile_count;
    a.buckets = buckets;
    a.sched = sched;
    a.trace_part = trace_part;
    a.done = done;
    a.err = err;
    a.m = g.m;
    a.n = g.n;
    a.mode = (int)mode;
    a.prods = nullptr;
    a.slice_items = nullptr;
    a.cap = 0;
    a.poll_limit = 1ll << 22;
    a.stall_polls = stall_polls;
    const int grid = std::min(device_sm_count(), g.m * g.m);
    if (emu_alternate(g.m))
        launch_dependent(emu::k_gemm_emu<false, true>, dim3(grid), dim3(emu::kThreads), emu::SMEM_DYN, st, a);
    else
        launch_dependent(emu::k_gemm_emu<false, false>, dim3(grid), dim3(emu::kThreads), emu::SMEM_DYN, st, a);
    note_launch();
}

void launch_gemm_emu_batched(const ProdDesc* prods, const int* tile_list, const int* tile_count, int cap,
                             int* slice_items, int* sched, const int* all_done, int* err, cudaStream_t st,
                             unsigned long long* units) {
    emu::EmuArgs a = {};
    a.prods = prods;
    a.slice_items = slice_items;
    a.cap = cap;
    a.tile_list = tile_list;
    a.tile_count = tile_count;
    a.buckets = kTileBuckets;
    a.sched = sched;
    a.done = all_done;
    a.err = err;
    a.units = units;
    a.poll_limit = 1ll << 22;
    a.stall_polls = 0;
    const int grid = std::min(device_sm_count(), cap);
    launch_dependent(emu::k_gemm_emu<true, false>, dim3(grid), dim3(emu::kThreads), emu::SMEM_DYN, st, a);
    note_launch();
}

}  // namespace spamm

// Norm-tree, cull and bookkeeping kernels of the SpAMM path.
//
//  * pack + leaf norms (the quadtree decoration of Sec. 1: every leaf tile
//    carries its squared Frobenius norm, accumulated in FP64),
//  * upper quadtree levels (parent = sum of its existing children),
//  * the two-sided metric query of Eq. (newspamm) as a per-output-tile scan
//    with a coarse-level pre-filter,
//  * Gershgorin scaling (Sec. 3.2), the NS map h[X] = 1.5 I - 0.5 X, the
//    trace error t_k (Sec. 4.2), unpacking and the residual norm.
//
// All reductions run in a fixed order, so every result is deterministic.
#include "spamm_internal.cuh"

namespace spamm {

Geometry make_geometry(int n, int nb) {
    Geometry g;
    g.n = n;
    g.nb = nb;
    g.m = (n + nb - 1) / nb;
    int L = 0;
    while ((1 << L) < g.m) ++L;
    g.L = L;
    long total = 0;
    for (int l = L; l >= 0; --l) {
        int sh = L - l;
        g.dim[l] = (g.m + (1 << sh) - 1) >> sh;
        g.off[l] = total;
        total += (long)g.dim[l] * g.dim[l];
    }
    g.tree_size = total;
    g.coarse = L >= 3 ? L - 3 : 0;
    g.coarse_shift = L - g.coarse;
    return g;
}

TreeDev tree_dev(const Geometry& g) {
    TreeDev t;
    t.m = g.m;
    t.L = g.L;
    t.coarse = g.coarse;
    t.shift = g.coarse_shift;
    for (int l = 0; l < kMaxLevels; ++l) {
        t.dim[l] = g.dim[l];
        t.off[l] = g.off[l];
    }
    return t;
}

// Deterministic block sum for blockDim.x == 256 (8 warps).
__device__ __forceinline__ double block_sum_256(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < 8; ++q) s += red[q];
    return s;  // valid in thread 0
}

// ---------------------------------------------------------------- Gershgorin
// sum_j |r_j + mu delta_{j,row}| for one row, by one warp: four independent partial sums per lane (FP64
// latency is long), partial p adding the entries lane + 32 (4k + p) in increasing k, then (p0 + p1) +
// (p2 + p3).  Sixteen loads are in flight per lane; kShift = false issues no add for the shift.
template <bool kShift>
__device__ __forceinline__ double row_abs_sum(const double* __restrict__ r, int n, int row, int lane, double mu) {
    double p[4] = {0.0, 0.0, 0.0, 0.0};
    int j = lane;
    for (; j + 480 < n; j += 512) {
        double v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = r[j + 32 * u];
        if (kShift) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (j + 32 * u == row) v[u] += mu;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) p[u & 3] += fabs(v[u]);
    }
    for (; j + 96 < n; j += 128) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            v[u] = r[j + 32 * u];
            if (kShift && j + 32 * u == row) v[u] += mu;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] += fabs(v[u]);
    }
    for (; j < n; j += 32) {
        double v = r[j];
        if (kShift && j == row) v += mu;
        p[0] += fabs(v);
    }
    return (p[0] + p[1]) + (p[2] + p[3]);
}

__global__ void k_rowsum(const double* __restrict__ S, int n, const double* __restrict__ mu_dev,
                         double* __restrict__ rowsum) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double* r = S + (size_t)row * n;
    double s = mu_dev ? row_abs_sum<true>(r, n, row, lane, *mu_dev) : row_abs_sum<false>(r, n, row, lane, 0.0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rowsum[row] = s;
}

__global__ void k_max(const double* __restrict__ v, int n, double* __restrict__ out) {
    __shared__ double red[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = fmax(r, red[q]);
        *out = r;
    }
}

void launch_gershgorin(const double* S, int n, const double* mu_dev, double* rowsum, double* out_c,
                       cudaStream_t st) {
    k_rowsum<<<(n + 7) / 8, 256, 0, st>>>(S, n, mu_dev, rowsum);
    note_launch();
    k_max<<<1, 1024, 0, st>>>(rowsum, n, out_c);
    note_launch();
}

__global__ void k_scale_mu(const double* c0, double mu_rel, double* mu_out) { *mu_out = mu_rel * (*c0); }

// Row-major D = S + (mu_rel * *c0) I (the level shift of Sec. 6, relative to a device-side bound c0).
__global__ void __launch_bounds__(256) k_shift_copy(const double* __restrict__ S, double* __restrict__ D, int n,
                                                    double mu_rel, const double* __restrict__ c0) {
    const double mu = mu_rel * *c0;
    const size_t nn = (size_t)n * n;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += (size_t)gridDim.x * blockDim.x) {
        const size_t i = q / n, j = q - i * n;
        D[q] = i == j ? S[q] + mu : S[q];
    }
}

void launch_shift_copy(const double* S, double* D, int n, double mu_rel, const double* c0, cudaStream_t st) {
    const size_t nn = (size_t)n * n;
    const int blocks = (int)std::min<size_t>((nn + 255) / 256, (size_t)device_sm_count() * 8);
    k_shift_copy<<<blocks, 256, 0, st>>>(S, D, n, mu_rel, c0);
    note_launch();
}

// Row-major T = A^T in 32 x 32 blocks through shared memory (coalesced on both sides).
__global__ void __launch_bounds__(256) k_transpose_rm(const double* __restrict__ A, double* __restrict__ T, int n) {
    __shared__ double sm[32][33];
    const int nbk = (n + 31) / 32;
    for (int b = blockIdx.x; b < nbk * nbk; b += gridDim.x) {
        const int r0 = (b / nbk) * 32, c0 = (b - (b / nbk) * nbk) * 32;  // block of A at rows r0, columns c0
        __syncthreads();
        for (int q = threadIdx.x; q < 1024; q += 256) {
            const int r = q >> 5, c = q & 31;
            if (r0 + r < n && c0 + c < n) sm[r][c] = A[(size_t)(r0 + r) * n + c0 + c];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < 1024; q += 256) {
            const int r = q >> 5, c = q & 31;  // T's row c0 + r, column r0 + c
            if (c0 + r < n && r0 + c < n) T[(size_t)(c0 + r) * n + r0 + c] = sm[c][r];
        }
    }
}

void launch_transpose_rm(const double* A, double* T, int n, cudaStream_t st) {
    const int nbk = (n + 31) / 32;
    const int blocks = std::min(nbk * nbk, device_sm_count() * 8);
    k_transpose_rm<<<blocks, 256, 0, st>>>(A, T, n);
    note_launch();
}

void launch_scale_mu(const double* c0, double mu_rel, double* mu_out, cudaStream_t st) {
    k_scale_mu<<<1, 1, 0, st>>>(c0, mu_rel, mu_out);
    note_launch();
}


// The scaling constants of a solve, once: sqrt(c) for Y, and the once-rounded reciprocals 1/c (for S) and
// 1/sqrt(c) (for Z) that the scaling multiplies by.
__global__ void k_scale_consts(const double* c, double* sqc, double* rc, double* rsqc) {
    const double s = sqrt(*c);
    *sqc = s;
    *rc = 1.0 / *c;
    *rsqc = 1.0 / s;
}

void launch_scale_consts(const double* c, double* sqc, double* rc, double* rsqc, cudaStream_t st) {
    k_scale_consts<<<1, 1, 0, st>>>(c, sqc, rc, rsqc);
    note_launch();
}

// ---------------------------------------------------------------- pack + leaf norms
// Entries of a tile handled per thread of a 256-thread block, and how many of them one batch of
// independent loads covers.
template <int NB, int kMaxBatch>
struct TileSplit {
    static constexpr int kPer = NB * NB / 256;
    static constexpr int kBatch = kPer < kMaxBatch ? kPer : kMaxBatch;
};

// One 256-thread block per tile.  Thread t takes the entries t + 256 q (a warp reads 32 consecutive
// entries of one row), sixteen independent loads at a time, then scales, stores and squares them in order.
// kScale: multiply by rc; kShift (diagonal tiles of a scaled pack): add mu on the logical diagonal first.
template <int NB, bool kScale, bool kShift>
__device__ __forceinline__ double pack_tile(const double* __restrict__ src, int n, int i, int j, double mu, double rc,
                                            double* __restrict__ d) {
    using TS = TileSplit<NB, 16>;
    double acc = 0.0;
#pragma unroll 1
    for (int q0 = 0; q0 < TS::kPer; q0 += TS::kBatch) {
        double v[TS::kBatch];
#pragma unroll
        for (int u = 0; u < TS::kBatch; ++u) {
            const int idx = threadIdx.x + 256 * (q0 + u);
            const int gi = i * NB + idx / NB, gj = j * NB + idx % NB;
            v[u] = (gi < n && gj < n) ? src[(size_t)gi * n + gj] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < TS::kBatch; ++u) {
            const int idx = threadIdx.x + 256 * (q0 + u);
            const int gi = i * NB + idx / NB, gj = j * NB + idx % NB;
            double x = v[u];
            if (kScale && gi < n && gj < n) {
                if (kShift && gi == gj) x += mu;
                x = x * rc;
            }
            d[idx] = x;
            acc = fma(x, x, acc);
        }
    }
    return acc;
}

// Four horizontally adjacent 64 x 64 tiles (i, 4 jb .. 4 jb + 3) per 256-thread block: thread t takes column
// t of the band in every row, so a row of the band is read as one 2 KB run (the eight warps side by side)
// and each thread touches a single tile (t / 64); sixteen independent loads at a time.  The leaf norm of a
// tile is the sum over its two warps of the per-thread sums of squares (rows in order), fixed order.
// kF32 (the tensor-core path): the sums of squares in FP32 from the entries' bits, so the FP64 pipe does one
// multiply per entry instead of two operations.  kShift: add mu on the diagonal (a compile-time switch, so
// that without a shift no entry carries a predicated add).
template <bool kScale, bool kF32, bool kShift>
__device__ __forceinline__ void pack_band64(const double* __restrict__ src, int n, int m, int i, int jb, double mu,
                                            double rc, double* __restrict__ dst, double* __restrict__ leaf,
                                            double* red) {
    const int t = threadIdx.x;
    const int j = 4 * jb + (t >> 6);  // this thread's tile column
    const int c = t & 63;
    const int gj = j * 64 + c;
    const bool colok = j < m && gj < n;
    double* d = dst + ((size_t)i * m + j) * 4096;
    double acc = 0.0;
    float accf = 0.f;
#pragma unroll 1
    for (int r0 = 0; r0 < 64; r0 += 16) {
        double v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int gi = i * 64 + r0 + u;
            v[u] = (colok && gi < n) ? src[(size_t)gi * n + gj] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int gi = i * 64 + r0 + u;
            double x = v[u];
            if (kScale && colok && gi < n) {
                if (kShift && gi == gj) x += mu;
                x = x * rc;
            }
            if (j < m) d[(r0 + u) * 64 + c] = x;
            if (kF32) {
                const float f = f32_of_bits((unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull);
                accf = fmaf(f, f, accf);
            } else {
                acc = fma(x, x, acc);
            }
        }
    }
    if (kF32) acc = (double)accf;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) red[t >> 5] = acc;
    __syncthreads();
    if (t < 4 && 4 * jb + t < m) leaf[(size_t)i * m + 4 * jb + t] = red[2 * t] + red[2 * t + 1];
}

__global__ void __launch_bounds__(256) k_pack_band64(const double* __restrict__ src, int n, int m, int bands,
                                                     const double* __restrict__ mu_dev,
                                                     const double* __restrict__ rc_dev, double* __restrict__ dst,
                                                     double* __restrict__ leaf, int f32_norms) {
    __shared__ double red[8];
    const int i = blockIdx.x / bands, jb = blockIdx.x - (blockIdx.x / bands) * bands;
    if (rc_dev) {
        const double rc = *rc_dev;
        if (mu_dev) {
            if (f32_norms) pack_band64<true, true, true>(src, n, m, i, jb, *mu_dev, rc, dst, leaf, red);
            else pack_band64<true, false, true>(src, n, m, i, jb, *mu_dev, rc, dst, leaf, red);
        } else {
            if (f32_norms) pack_band64<true, true, false>(src, n, m, i, jb, 0.0, rc, dst, leaf, red);
            else pack_band64<true, false, false>(src, n, m, i, jb, 0.0, rc, dst, leaf, red);
        }
    } else {
        pack_band64<false, false, false>(src, n, m, i, jb, 0.0, 1.0, dst, leaf, red);
    }
}

template <int NB>
__global__ void __launch_bounds__(256) k_pack(const double* __restrict__ src, int n, int m,
                                              const double* __restrict__ mu_dev, const double* __restrict__ rc_dev,
                                              double* __restrict__ dst, double* __restrict__ leaf) {
    __shared__ double red[8];
    const int tile = blockIdx.x;
    const int i = tile / m, j = tile - (tile / m) * m;
    const double mu = mu_dev ? *mu_dev : 0.0;
    double* d = dst + (size_t)tile * NB * NB;
    double acc;
    if (!rc_dev) acc = pack_tile<NB, false, false>(src, n, i, j, 0.0, 1.0, d);
    else if (i == j) acc = pack_tile<NB, true, true>(src, n, i, j, mu, *rc_dev, d);
    else acc = pack_tile<NB, true, false>(src, n, i, j, 0.0, *rc_dev, d);
    const double s = block_sum_256(acc, red);
    if (threadIdx.x == 0) leaf[tile] = s;
}

void launch_pack(const double* src, int n, const Geometry& g, const double* mu, const double* recip_c,
                 TileMat dst, cudaStream_t st, bool f32_norms) {
    const dim3 grid(g.m * g.m), block(256);
    if (g.nb == 32) {
        k_pack<32><<<grid, block, 0, st>>>(src, n, g.m, mu, recip_c, dst.t, dst.tree);
    } else if (g.nb == 64) {
        const int bands = (g.m + 3) / 4;
        k_pack_band64<<<dim3(g.m * bands), block, 0, st>>>(src, n, g.m, bands, mu, recip_c, dst.t, dst.tree,
                                                           f32_norms ? 1 : 0);
    } else {
        k_pack<128><<<grid, block, 0, st>>>(src, n, g.m, mu, recip_c, dst.t, dst.tree);
    }
    note_launch();
}

// ---------------------------------------------------------------- the NS map
// Sum of the diagonal-tile trace partials, fixed order (lane-strided, then a
// butterfly): the same value in every warp that calls it.  Warp-wide.
__device__ __forceinline__ double trace_sum_warp(const double* __restrict__ trace_part, int m) {
    double tr = 0.0;
    for (int i = (int)(threadIdx.x & 31); i < m; i += 32) tr += trace_part[i];
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    return tr;
}

// trace_part[i] = sum of the logical diagonal of tile (i, i), one warp per tile.
__global__ void __launch_bounds__(32) k_trace_parts(const double* __restrict__ X, int n, int m, int nb,
                                                    double* __restrict__ trace_part) {
    const int i = blockIdx.x;
    const double* x = X + ((size_t)i * m + i) * nb * nb;
    const int cnt = min(nb, n - i * nb);
    double s = 0.0;
    for (int r = threadIdx.x; r < cnt; r += 32) s += x[(size_t)r * nb + r];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) trace_part[i] = s;
}

void launch_trace_parts(const double* X, const Geometry& g, double* trace_part, cudaStream_t st) {
    k_trace_parts<<<g.m, 32, 0, st>>>(X, g.n, g.m, g.nb, trace_part);
    note_launch();
}

// T = h_alpha[U], U = eps I + (1 - 2 eps) X, the NS logistic after the
// stabilising shift-and-scale (Sec. 4.2 "Mapping"), written as T = c0 I + c1 X
// with c0 = (sqrt(alpha)/2)(3 - alpha eps), c1 = -(sqrt(alpha)/2) alpha (1 - 2 eps).
// SPAMM_MAP_SCALED takes alpha and eps from the sigmoidal damping functions of
// t = (n - tr X)/n; SPAMM_MAP_NS is alpha = 1, eps = 0 (c0 = 1.5, c1 = -0.5,
// both exact).  Grid-stride over tiles; a tile whose X is exactly zero (leaf
// norm 0, data unwritten) off the diagonal stays zero.  Writes T's leaf
// norms and, when rmax is set (64 x 64 tiles), T's row/column magnitude maxima.
// -x/2 as the multiply gives it, from the bits where that is exact: for a normal x whose half is normal the
// exponent field drops by one and the sign flips; +-0 flips its sign; anything else (a half below the
// normal range, inf, nan) takes the FP64 multiply, which this part runs at a small fraction of its integer
// rate.
__device__ __forceinline__ double neg_half(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned E = (unsigned)(b >> 52) & 0x7FFu;
    if (E > 1u && E < 0x7FFu) return __longlong_as_double((long long)((b - (1ull << 52)) ^ 0x8000000000000000ull));
    if ((b << 1) == 0ull) return __longlong_as_double((long long)(b ^ 0x8000000000000000ull));
    return -0.5 * x;
}

// The entries of one tile of the map, thread t taking t + 256 q: T = c1 X + c0 I (kHalf: c1 = -1/2, the
// entries off the diagonal from their bits), the thread's sum of squares (FP32 from the bits when f32 is
// set, then widened) and, with rmax, the row maxima by warp reductions and the thread's column maximum.
template <int NB, bool kHalf, bool kDiag>
__device__ __forceinline__ double map_entries(const double* x, double* t, int i, int j, int n, double c0, double c1,
                                              bool f32, unsigned long long* __restrict__ rmax, int lane,
                                              unsigned long long& cmx) {
    using TS = TileSplit<NB, 8>;
    double acc = 0.0;
    float accf = 0.f;
#pragma unroll 1
    for (int q0 = 0; q0 < TS::kPer; q0 += TS::kBatch) {
        // a batch of independent loads first (in place, each thread reads its entries before writing them)
        double xb[TS::kBatch];
#pragma unroll
        for (int u = 0; u < TS::kBatch; ++u) xb[u] = x[threadIdx.x + 256 * (q0 + u)];
#pragma unroll
        for (int u = 0; u < TS::kBatch; ++u) {
            const int idx = threadIdx.x + 256 * (q0 + u);
            const int r = idx / NB, cc = idx % NB;
            const double xv = xb[u];
            double v = kHalf ? neg_half(xv) : c1 * xv;
            if (kDiag) {
                const int gi = i * NB + r, gj = j * NB + cc;
                if (gi == gj && gi < n) v = fma(c1, xv, c0);
            }
            t[idx] = v;
            if (f32) {
                const float f = f32_of_bits((unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull);
                accf = fmaf(f, f, accf);
            } else {
                acc = fma(v, v, acc);
            }
            if (NB == 64 && rmax) {
                // 64-wide tiles: this thread keeps column threadIdx.x & 63, and the row's 64 entries sit in
                // two consecutive warps; the maxima feed only the slicing exponents, so the upper 32 bits
                // (sign cleared) carry what is needed
                const unsigned long long vb = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
                cmx = max(cmx, vb);
                const unsigned rm = __reduce_max_sync(0xffffffffu, (unsigned)(vb >> 32));
                if (lane == 0 && rm) atomicMax(rmax + (size_t)i * NB + r, (unsigned long long)rm << 32);
            }
        }
    }
    return f32 ? (double)accf : acc;
}

template <int NB>
__global__ void __launch_bounds__(256, 4) k_map(const double* X, double* T, const double* leafX, double* leafT,
                                                int n, int m, int map, const double* __restrict__ trace_part,
                                                unsigned long long* __restrict__ rmax,
                                                unsigned long long* __restrict__ cmax, const int* __restrict__ done,
                                                int f32_norms) {
    grid_dependency_wait();
    if (done && *done) return;
    __shared__ double red[8];
    __shared__ double coef[2];
    __shared__ unsigned long long cm_sh[4][64];
    if (threadIdx.x < 32) {
        double alpha = 1.0, eps = 0.0;
        if (map == SPAMM_MAP_SCALED) {
            const double t = ((double)n - trace_sum_warp(trace_part, m)) / (double)n;
            alpha = 1.0 + 1.85 / (1.0 + exp(-50.0 * (t - 0.35)));
            eps = 0.1 / (1.0 + exp(-75.0 * (t - 0.30)));
        }
        if (threadIdx.x == 0) {
            const double hr = 0.5 * sqrt(alpha);
            coef[0] = hr * (3.0 - alpha * eps);
            coef[1] = -(hr * alpha) * (1.0 - 2.0 * eps);
        }
    }
    __syncthreads();
    const double c0 = coef[0], c1 = coef[1];
    // alpha = 1: c1 = -1/2 exactly, so the entries off the diagonal are -x/2 from their bits
    const bool half_neg = map != SPAMM_MAP_SCALED;
    constexpr int ne = NB * NB;
    const int lane = threadIdx.x & 31;
    for (int tile = blockIdx.x; tile < m * m; tile += gridDim.x) {
        const int i = tile / m, j = tile - (tile / m) * m;
        const double* x = X + (size_t)tile * ne;
        double* t = T + (size_t)tile * ne;
        const double nu_x = leafX[tile];
        __syncthreads();  // every thread has read leafX[tile] before thread 0 may overwrite it (in place)
        if (nu_x == 0.0 && i != j) {
            if (T != X)
                for (int idx = threadIdx.x; idx < ne; idx += 256) t[idx] = 0.0;
            if (threadIdx.x == 0) leafT[tile] = 0.0;
            continue;
        }
        double acc = 0.0;
        unsigned long long cmx = 0;
        // every switch of the entry loop is uniform over the tile, so each case is its own loop: no entry of
        // an off-diagonal tile carries a predicated fused multiply-add, and alpha = 1 no multiply
        if (i == j) {
            if (half_neg) acc = map_entries<NB, true, true>(x, t, i, j, n, c0, c1, f32_norms, rmax, lane, cmx);
            else acc = map_entries<NB, false, true>(x, t, i, j, n, c0, c1, f32_norms, rmax, lane, cmx);
        } else {
            if (half_neg) acc = map_entries<NB, true, false>(x, t, i, j, n, c0, c1, f32_norms, rmax, lane, cmx);
            else acc = map_entries<NB, false, false>(x, t, i, j, n, c0, c1, f32_norms, rmax, lane, cmx);
        }
        if (NB == 64 && rmax) {
            cm_sh[threadIdx.x >> 6][threadIdx.x & 63] = cmx;
            __syncthreads();
            if (threadIdx.x < 64) {
                const unsigned long long mx =
                    max(max(cm_sh[0][threadIdx.x], cm_sh[1][threadIdx.x]), max(cm_sh[2][threadIdx.x], cm_sh[3][threadIdx.x]));
                if (mx) atomicMax(cmax + (size_t)j * NB + threadIdx.x, mx);
            }
        }
        const double s = block_sum_256(acc, red);
        if (threadIdx.x == 0) leafT[tile] = s;
    }
}

void launch_map(const double* X, const double* leafX, TileMat T, const Geometry& g, int map, const double* trace_part,
                bool maxima, const int* done, cudaStream_t st, bool f32_norms) {
    // one resident wave (four 256-thread blocks per SM), so a dependent launch never waits on a later wave
    const int grid = std::min(device_sm_count() * 4, g.m * g.m);
    unsigned long long* rmax = maxima ? T.rmax : nullptr;
    unsigned long long* cmax = maxima ? T.cmax : nullptr;
    if (g.nb == 32)
        launch_dependent(k_map<32>, dim3(grid), dim3(256), 0, st, X, T.t, leafX, T.tree, g.n, g.m, map, trace_part,
                         rmax, cmax, done, f32_norms ? 1 : 0);
    else if (g.nb == 64)
        launch_dependent(k_map<64>, dim3(grid), dim3(256), 0, st, X, T.t, leafX, T.tree, g.n, g.m, map, trace_part,
                         rmax, cmax, done, f32_norms ? 1 : 0);
    else
        launch_dependent(k_map<128>, dim3(grid), dim3(256), 0, st, X, T.t, leafX, T.tree, g.n, g.m, map, trace_part,
                         rmax, cmax, done, f32_norms ? 1 : 0);
    note_launch();
}

// Plane-diagonal profile (Sec. 7.2 "lensing") of a product's task lists: a warp per output tile (i, k)
// walks its surviving j; block histograms in shared memory, then one atomic per non-empty bin.  Launched
// in stream order after the cull (not as a programmatic dependent: its grid may take several waves).
__global__ void __launch_bounds__(256) k_lens(const int* __restrict__ counts, const int* __restrict__ jlist, int m,
                                              int bins, const int* __restrict__ iter, int which,
                                              unsigned long long* __restrict__ lens, const int* __restrict__ done) {
    if (done && *done) return;
    extern __shared__ unsigned hist[];  // [3][bins]
    for (int q = threadIdx.x; q < 3 * bins; q += blockDim.x) hist[q] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int wid = blockIdx.x * 8 + (threadIdx.x >> 5); wid < m * m; wid += gridDim.x * 8) {
        const int i = wid / m, k = wid - (wid / m) * m;
        const int cnt = counts[wid];
        const int* js = jlist + (size_t)wid * m;
        for (int t = lane; t < cnt; t += 32) {
            const int j = js[t];
            atomicAdd(&hist[min(abs(i - j), bins - 1)], 1u);
            atomicAdd(&hist[bins + min(abs(j - k), bins - 1)], 1u);
        }
        if (lane == 0 && cnt) atomicAdd(&hist[2 * bins + min(abs(i - k), bins - 1)], (unsigned)cnt);
    }
    __syncthreads();
    unsigned long long* out = lens + ((size_t)*iter * 3 + which) * 3 * bins;
    for (int q = threadIdx.x; q < 3 * bins; q += blockDim.x)
        if (hist[q]) atomicAdd(out + q, (unsigned long long)hist[q]);
}

void launch_lens(const int* counts, const int* jlist, const Geometry& g, int bins, const int* iter, int which,
                 unsigned long long* lens, const int* done, cudaStream_t st) {
    const int blocks = std::min((g.m * g.m + 7) / 8, device_sm_count() * 4);
    k_lens<<<blocks, 256, 3 * (size_t)bins * sizeof(unsigned), st>>>(counts, jlist, g.m, bins, iter, which, lens, done);
    note_launch();
}

// T = A^T on the tile grid: tile (i,j) of T is tile (j,i) of A transposed, moved through shared memory in
// 32 x 32 blocks (coalesced reads along A's rows, writes along T's rows).  T's leaf norms are A's, transposed
// (a tile's Frobenius norm does not depend on the order of its entries).  Tiles of norm 0 are not written:
// every reader goes by the norm.  Grid-stride over output tiles; skipped once *done is set.
__global__ void __launch_bounds__(256) k_transpose(const double* __restrict__ A, const double* __restrict__ leafA,
                                                   double* __restrict__ T, double* __restrict__ leafT, int m, int nb,
                                                   const int* __restrict__ done) {
    grid_dependency_wait();
    if (done && *done) return;
    __shared__ double sm[32][33];
    const size_t ne = (size_t)nb * nb;
    for (int tile = blockIdx.x; tile < m * m; tile += gridDim.x) {
        const int i = tile / m, j = tile - (tile / m) * m;
        const int src = j * m + i;
        const double nu = leafA[src];
        if (threadIdx.x == 0) leafT[tile] = nu;
        if (nu == 0.0) continue;
        const double* a = A + (size_t)src * ne;
        double* t = T + (size_t)tile * ne;
        for (int r0 = 0; r0 < nb; r0 += 32)
            for (int c0 = 0; c0 < nb; c0 += 32) {
                __syncthreads();
                for (int q = threadIdx.x; q < 1024; q += 256) {
                    const int c = q >> 5, r = q & 31;
                    sm[c][r] = a[(size_t)(c0 + c) * nb + r0 + r];  // A's row c0 + c, column r0 + r
                }
                __syncthreads();
                for (int q = threadIdx.x; q < 1024; q += 256) {
                    const int r = q >> 5, c = q & 31;
                    t[(size_t)(r0 + r) * nb + c0 + c] = sm[c][r];  // T's row r0 + r, column c0 + c
                }
            }
    }
}

void launch_transpose(const TileMat& A, TileMat T, const Geometry& g, const int* done, cudaStream_t st) {
    // one resident wave (34 KB of shared memory and 256 threads per block leave room for 4 per SM)
    const int grid = std::min(device_sm_count() * 4, g.m * g.m);
    launch_dependent(k_transpose, dim3(grid), dim3(256), 0, st, (const double*)A.t, (const double*)A.tree, T.t,
                     T.tree, g.m, g.nb, done);
    note_launch();
}

__global__ void __launch_bounds__(256) k_identity(int n, int m, int nb, double* __restrict__ Z,
                                                  double* __restrict__ leaf) {
    const int tile = blockIdx.x;
    const int i = tile / m, j = tile % m;
    const int ne = nb * nb;
    double* z = Z + (size_t)tile * ne;
    for (int idx = threadIdx.x; idx < ne; idx += 256) {
        const int r = idx / nb, cc = idx - r * nb;
        const int gi = i * nb + r, gj = j * nb + cc;
        z[idx] = (gi == gj && gi < n) ? 1.0 : 0.0;
    }
    if (threadIdx.x == 0) {
        int cnt = 0;
        if (i == j) cnt = min(nb, n - i * nb);
        leaf[tile] = (double)cnt;
    }
}

void launch_identity(const Geometry& g, TileMat Z, cudaStream_t st) {
    k_identity<<<g.m * g.m, 256, 0, st>>>(g.n, g.m, g.nb, Z.t, Z.tree);
    note_launch();
}

// ---------------------------------------------------------------- quadtree levels
// Parent = sum of its existing children, summed pairwise (rows first).
__device__ __forceinline__ double child_sum(const double* ch, int dc, int I, int J) {
    const int ci = 2 * I, cj = 2 * J;
    const bool r1 = ci + 1 < dc, c1 = cj + 1 < dc;
    const double s0 = ch[ci * dc + cj] + (c1 ? ch[ci * dc + cj + 1] : 0.0);
    const double s1 = r1 ? ch[(ci + 1) * dc + cj] + (c1 ? ch[(ci + 1) * dc + cj + 1] : 0.0) : 0.0;
    return s0 + s1;
}

// t_k = (n - tr X)/n from the diagonal-tile trace partials (fixed-order warp
// reduction) into t_hist[k], k = *iters the iterations done so far; then the
// count and the stop (tolerance reached, or the last of maxit iterations),
// which also ends a graph's conditional loop.
template <bool kLoop>
__device__ __forceinline__ void trace_error(const double* __restrict__ trace_part, int n, int m, const TreeExtra& ex) {
    const double tr = trace_sum_warp(trace_part, m);
    if (threadIdx.x != 0) return;
    const int k = *ex.iters;
    const double t = ((double)n - tr) / (double)n;
    ex.t_hist[k] = t;
    *ex.iters = k + 1;
    if ((ex.tol_t > 0.0 && fabs(t) <= ex.tol_t) || k + 1 >= ex.maxit) {
        *ex.done = 1;
        if constexpr (kLoop) cudaGraphSetConditional(ex.cond, 0u);
    }
}

// Upper levels of one quadtree from its leaf level, by a block of kThr threads.  Levels whose children
// exceed 64 x 64 go through global memory; from there on the children are held in shared memory (bufA:
// 64 x 64, bufB: 32 x 32; each level is still written out), so the top levels cost shared-memory latency
// instead of global.
template <int kThr>
__device__ __forceinline__ void tree_levels(const TreeDev& td, double* __restrict__ tree, double* bufA,
                                            double* bufB) {
    int l = td.L - 1;
    for (; l >= 0 && td.dim[l + 1] > 64; --l) {
        const int d = td.dim[l], dc = td.dim[l + 1];
        const double* ch = tree + td.off[l + 1];
        double* pa = tree + td.off[l];
        for (int idx = threadIdx.x; idx < d * d; idx += kThr) {
            const int I = idx / d, J = idx - I * d;
            const int ci = 2 * I, cj = 2 * J;
            const bool r1 = ci + 1 < dc, c1 = cj + 1 < dc;
            const double s0 = ch[(size_t)ci * dc + cj] + (c1 ? ch[(size_t)ci * dc + cj + 1] : 0.0);
            const double s1 = r1 ? ch[(size_t)(ci + 1) * dc + cj] + (c1 ? ch[(size_t)(ci + 1) * dc + cj + 1] : 0.0) : 0.0;
            pa[idx] = s0 + s1;
        }
        __syncthreads();
    }
    if (l >= 0) {
        const int dc0 = td.dim[l + 1];
        const double* ch0 = tree + td.off[l + 1];
        // up to 4096 children: independent loads first, then the shared-memory stores
        constexpr int kPer = 4096 / kThr;
        double v[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int idx = threadIdx.x + q * kThr;
            v[q] = idx < dc0 * dc0 ? ch0[idx] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int idx = threadIdx.x + q * kThr;
            if (idx < dc0 * dc0) bufA[idx] = v[q];
        }
        __syncthreads();
        double* cur = bufA;
        double* nxt = bufB;
        for (; l >= 0; --l) {
            const int d = td.dim[l], dc = td.dim[l + 1];
            double* pa = tree + td.off[l];
            for (int idx = threadIdx.x; idx < d * d; idx += kThr) {
                const int I = idx / d, J = idx - I * d;
                const double s = child_sum(cur, dc, I, J);
                nxt[idx] = s;
                pa[idx] = s;
            }
            __syncthreads();
            double* t = cur;
            cur = nxt;
            nxt = t;
        }
    }
}

// The same levels for trees of at most 64 x 64 leaves (L <= 6), by 1024 threads with one block barrier.
// The leaf grid is taken as 64 x 64 with zeros beyond m (adding a zero child is exact), so real level l is
// level l + 6 - L of the padded tree.  Thread t holds the level-5 node whose Morton code is t (even bits:
// column, odd bits: row) and sums its four leaves as child_sum does; the next two levels are groups of 4
// and 16 consecutive lanes, combined with shuffles in child_sum's order (the two top-row children first,
// then the two bottom-row ones, then the two sums).  The 64 level-3 nodes go through shared memory to one
// warp, which finishes levels 2, 1 and 0 the same way.  Every node is written to its level of the tree.
__device__ __forceinline__ int compact_bits(int x) {  // bits 0, 2, 4, 6, 8 of x to bits 0..4
    x &= 0x155;
    x = (x | (x >> 1)) & 0x133;
    x = (x | (x >> 2)) & 0x10F;
    x = (x | (x >> 4)) & 0x01F;
    return x;
}
__device__ __forceinline__ void put_node(const TreeDev& td, double* __restrict__ tree, int vlevel, int I, int J,
                                         double v) {
    const int l = vlevel - (6 - td.L);
    if (l >= 0 && l < td.L && I < td.dim[l] && J < td.dim[l]) tree[td.off[l] + (long)I * td.dim[l] + J] = v;
}
__device__ __forceinline__ void tree_levels_small(const TreeDev& td, double* __restrict__ tree, double* lvl3) {
    const int t = threadIdx.x, lane = t & 31;
    const int J = compact_bits(t), I = compact_bits(t >> 1);  // level-5 node (I, J)
    const int m = td.m;
    const double* leaf = tree + td.off[td.L];
    const int r0 = 2 * I, c0 = 2 * J;
    const double a00 = (r0 < m && c0 < m) ? leaf[r0 * m + c0] : 0.0;
    const double a01 = (r0 < m && c0 + 1 < m) ? leaf[r0 * m + c0 + 1] : 0.0;
    const double a10 = (r0 + 1 < m && c0 < m) ? leaf[(r0 + 1) * m + c0] : 0.0;
    const double a11 = (r0 + 1 < m && c0 + 1 < m) ? leaf[(r0 + 1) * m + c0 + 1] : 0.0;
    double v = (a00 + a01) + (a10 + a11);
    put_node(td, tree, 5, I, J, v);
    // level 4: lanes 4q .. 4q+3 hold (top-left, top-right, bottom-left, bottom-right)
    double h = v + __shfl_xor_sync(0xffffffffu, v, 1);
    v = h + __shfl_xor_sync(0xffffffffu, h, 2);
    if ((t & 3) == 0) put_node(td, tree, 4, I >> 1, J >> 1, v);
    // level 3: the level-4 nodes sit on lanes 16q + 4p
    h = v + __shfl_xor_sync(0xffffffffu, v, 4);
    v = h + __shfl_xor_sync(0xffffffffu, h, 8);
    if ((t & 15) == 0) {
        put_node(td, tree, 3, I >> 2, J >> 2, v);
        lvl3[t >> 4] = v;
    }
    __syncthreads();
    if (t < 32) {
        // level 2: lane q pairs level-3 nodes 2q, 2q+1 (Morton-consecutive), then combines with lane q ^ 1
        h = lvl3[2 * lane] + lvl3[2 * lane + 1];
        v = h + __shfl_xor_sync(0xffffffffu, h, 1);
        const int q2 = lane >> 1;  // Morton code of the level-2 node
        if ((lane & 1) == 0) put_node(td, tree, 2, compact_bits(q2 >> 1), compact_bits(q2), v);
        h = v + __shfl_xor_sync(0xffffffffu, v, 2);
        v = h + __shfl_xor_sync(0xffffffffu, h, 4);
        const int q1 = lane >> 3;
        if ((lane & 7) == 0) put_node(td, tree, 1, q1 >> 1, q1 & 1, v);
        h = v + __shfl_xor_sync(0xffffffffu, v, 8);
        v = h + __shfl_xor_sync(0xffffffffu, h, 16);
        if (lane == 0) put_node(td, tree, 0, 0, 0, v);
    }
    __syncthreads();
}

// kLoop: the instance in a graph's conditional loop body, the only one that calls the device runtime
// (profilers skip kernels that do, so every other launch uses the plain instance).
template <bool kLoop>
__global__ void __launch_bounds__(1024) k_tree(TreeDev td, double* __restrict__ tree, const int* __restrict__ done,
                                               TreeExtra ex) {
    grid_dependency_wait();
    if (done && *done) return;
    __shared__ double bufA[64 * 64];
    __shared__ double bufB[32 * 32];
    if (td.L <= 6) tree_levels_small(td, tree, bufB);
    else tree_levels<1024>(td, tree, bufA, bufB);
    if (ex.zero_int && threadIdx.x < ex.zero_n) ex.zero_int[threadIdx.x] = 0;
    if (ex.trace_part && threadIdx.x < 32)
        trace_error<kLoop>(ex.trace_part, ex.n, td.m, ex);
}

void launch_tree(const Geometry& g, double* tree, const int* done, cudaStream_t st, const TreeExtra& ex) {
    if (ex.has_cond)
        launch_dependent(k_tree<true>, dim3(1), dim3(1024), 0, st, tree_dev(g), tree, done, ex);
    else
        launch_dependent(k_tree<false>, dim3(1), dim3(1024), 0, st, tree_dev(g), tree, done, ex);
    note_launch();
}

// ---------------------------------------------------------------- the cull
// Leaf test of Eq. (newspamm) in squared form: a pair is kept unless fl(nu_a * nu_b) < thr (FP64, strict).
// Most pairs are decided from the binary exponents alone: with nu_a in [2^ea, 2^(ea+1)) and nu_b in
// [2^eb, 2^(eb+1)), the product lies in [2^(ea+eb), 2^(ea+eb+2)); for thr in [2^et, 2^(et+1)) it is culled
// when ea+eb+2 < et and kept when ea+eb >= et+1, and its rounded value falls on the same side (rounding is
// monotone and powers of two are exact).  Only pairs within a factor of about eight of the threshold, and
// zero, subnormal or non-finite operands, take the FP64 multiply: the same decision as the multiply, at a
// fraction of the FP64 work this part's slow FP64 pipe would spend on every candidate.
__device__ __forceinline__ int biased_exponent(double x) {
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFull);
}
__device__ __forceinline__ bool keep_pair(double a, double b, double thr, int et) {
    const int ea = biased_exponent(a), eb = biased_exponent(b);
    if (ea > 0 && ea < 0x7FF && eb > 0 && eb < 0x7FF && et > 0 && et < 0x7FF) {
        const int s = ea + eb - 1023;  // biased exponent of 2^(ea'+eb')
        if (s + 2 < et) return false;
        if (s >= et + 1) return true;
    }
    return !(a * b < thr);
}

// Task list of output tile (i, k) by one warp: lanes test 32 consecutive j at a time and the survivors are
// compacted with a ballot in ascending j.  A chunk of 32 j is skipped when no coarse block J under it passes
// the coarse test (parents hold sums of non-negative children, so a coarse pair below the threshold has no
// surviving leaf pair under it).  The surviving set is exactly the leaf test nuA(i,j) * nuB(j,k) >= thr,
// i.e. the recursion of Eq. (newspamm).  Returns the count (in every lane).
__device__ __forceinline__ int cull_tile(const TreeDev& td, const double* __restrict__ treeA,
                                         const double* __restrict__ treeB, double thr, int i, int k, int lane,
                                         int* __restrict__ out) {
    const int m = td.m;
    const int et = biased_exponent(thr);
    const int dc = td.dim[td.coarse];
    const double* cA = treeA + td.off[td.coarse];
    const double* cB = treeB + td.off[td.coarse];
    const int I = i >> td.shift, K = k >> td.shift;
    int cnt = 0;
    for (int j0 = 0; j0 < m; j0 += 32) {
        const int j = j0 + lane;
        bool coarse = false;
        if (j < m) {
            const int J = j >> td.shift;
            coarse = keep_pair(cA[(size_t)I * dc + J], cB[(size_t)J * dc + K], thr, et);
        }
        if (!__any_sync(0xffffffffu, coarse)) continue;
        const bool keep = coarse && keep_pair(treeA[(size_t)i * m + j], treeB[(size_t)j * m + k], thr, et);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) out[cnt + __popc(bal & ((1u << lane) - 1u))] = j;
        cnt += __popc(bal);
    }
    return cnt;
}

// Up to 64 candidates (m <= 64), the list of cull_tile without its coarse pre-filter: every candidate's two
// leaf norms are loaded at once, before the threshold's roots have arrived, so the test waits for one round
// trip instead of one per chunk and level.  The list is the same: a coarse node is the rounded sum of its
// non-negative children, so it is at least each of them, and the rounded product is monotone; a pair the
// pre-filter would have skipped fails the leaf test too.
struct LeafPre {
    double a0, b0, a1, b1;
};
__device__ __forceinline__ LeafPre cull_preload(const double* __restrict__ treeA, const double* __restrict__ treeB,
                                                int m, int i, int k, int lane) {
    LeafPre p{0.0, 0.0, 0.0, 0.0};
    if (lane < m) {
        p.a0 = treeA[(size_t)i * m + lane];
        p.b0 = treeB[(size_t)lane * m + k];
    }
    if (lane + 32 < m) {
        p.a1 = treeA[(size_t)i * m + lane + 32];
        p.b1 = treeB[(size_t)(lane + 32) * m + k];
    }
    return p;
}
__device__ __forceinline__ int cull_tile_small(const LeafPre& p, double thr, int m, int lane, int* __restrict__ out) {
    const int et = biased_exponent(thr);
    const bool k0 = lane < m && keep_pair(p.a0, p.b0, thr, et);
    const unsigned b0 = __ballot_sync(0xffffffffu, k0);
    if (k0) out[__popc(b0 & ((1u << lane) - 1u))] = lane;
    int cnt = __popc(b0);
    if (m > 32) {
        const bool k1 = lane + 32 < m && keep_pair(p.a1, p.b1, thr, et);
        const unsigned b1 = __ballot_sync(0xffffffffu, k1);
        if (k1) out[cnt + __popc(b1 & ((1u << lane) - 1u))] = lane + 32;
        cnt += __popc(b1);
    }
    return cnt;
}

// One warp per output tile (i, k), the task list by cull_tile.
__global__ void __launch_bounds__(256) k_cull(TreeDev td, const double* __restrict__ treeA,
                                              const double* __restrict__ treeB, double tau, CullOut co,
                                              unsigned long long* __restrict__ total, double* __restrict__ thr_out,
                                              const int* __restrict__ done) {
    grid_dependency_wait();
    if (done && *done) return;
    __shared__ int red[8];
    __shared__ int lst[8];
    __shared__ int bkt[8];
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < co.zero_n; q += (long)gridDim.x * blockDim.x)
        co.zero_u64[q] = 0ull;
    const int m = td.m;
    const int wid = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const bool small = m <= 64;
    const LeafPre pre = small && wid < m * m ? cull_preload(treeA, treeB, m, wid / m, wid % m, lane) : LeafPre{};
    const double thr = ((tau * tau) * treeA[td.off[0]]) * treeB[td.off[0]];
    int cnt = 0;
    bool listed = false;
    if (wid < m * m) {
        const int i = wid / m, k = wid - (wid / m) * m;
        int* const out = co.jlist + (size_t)wid * m;
        cnt = small ? cull_tile_small(pre, thr, m, lane, out) : cull_tile(td, treeA, treeB, thr, i, k, lane, out);
        if (lane == 0) {
            co.counts[wid] = cnt;
            if (co.tile_list) {
                listed = cnt > 0 || (co.force_diag && i == k);
                if (!listed && co.leafC) co.leafC[wid] = 0.0;
            }
        }
    }
    if (co.tile_list) {
        // one atomic per block and bucket appends the block's listed output tiles
        if (lane == 0) {
            lst[threadIdx.x >> 5] = listed ? wid : -1;
            bkt[threadIdx.x >> 5] = co.buckets > 1 ? tile_bucket(cnt) : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int c[kTileBuckets] = {0, 0, 0, 0, 0};
            for (int w = 0; w < 8; ++w)
                if (lst[w] >= 0) ++c[bkt[w]];
            int q[kTileBuckets];
            for (int b = 0; b < kTileBuckets; ++b) q[b] = c[b] ? atomicAdd(co.tile_count + b, c[b]) : 0;
            const size_t mm = (size_t)m * m;
            for (int w = 0; w < 8; ++w)
                if (lst[w] >= 0) co.tile_list[bkt[w] * mm + q[bkt[w]]++] = lst[w];
        }
    }
    if (thr_out && wid == 0 && lane == 0) *thr_out = thr;
    if (total) {
        if (lane == 0) red[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            int sacc = 0;
            for (int w = 0; w < 8; ++w) sacc += red[w];
            if (sacc) atomicAdd(co.iter ? total + 3 * (size_t)*co.iter : total, (unsigned long long)sacc);
        }
    }
}

void launch_cull(const Geometry& g, const double* treeA, const double* treeB, double tau, const CullOut& out,
                 unsigned long long* total, double* thr_out, const int* done, cudaStream_t st) {
    const int warps = g.m * g.m;
    launch_dependent(k_cull, dim3((warps + 7) / 8), dim3(256), 0, st, tree_dev(g), treeA, treeB, tau, out, total,
                     thr_out, done);
    note_launch();
}

// ---------------------------------------------------------------- batched cull and quadtree
// The cull of every product of a stage of a batched solve in one launch.  Block b takes 8 output tiles of
// one product: blocks[b] = (product, first tile, blocks of that product, index of b among them).  Per
// output tile the test is the one of k_cull (the leaf test with the coarse pre-filter, ascending j);
// listed tiles become items (p << kItemShift) | tile in the stage's cost classes (stride cap).  The
// products of a matrix that has stopped are skipped, and the output's row/column maxima are cleared for
// the tensor-core products.
__global__ void __launch_bounds__(256) k_cull_batched(const ProdDesc* __restrict__ prods,
                                                      const int4* __restrict__ blocks, int* __restrict__ tile_list,
                                                      int* __restrict__ tile_count, int cap,
                                                      const int* __restrict__ all_done) {
    grid_dependency_wait();
    if (*all_done) return;
    const int4 bt = blocks[blockIdx.x];
    const ProdDesc& d = prods[bt.x];
    if (d.mflags[0]) return;
    __shared__ int red[8];
    __shared__ int lst[8];
    __shared__ int bkt[8];
    const TreeDev& td = d.td;
    const int m = td.m;
    if (d.Crmax) {
        const long zn = 2L * m * 64;
        for (long q = (long)bt.w * blockDim.x + threadIdx.x; q < zn; q += (long)bt.z * blockDim.x) d.Crmax[q] = 0ull;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wid = bt.y + warp;
    const double* treeA = d.Atree;
    const double* treeB = d.Btree;
    const bool small = m <= 64;
    const LeafPre pre = small && wid < m * m ? cull_preload(treeA, treeB, m, wid / m, wid % m, lane) : LeafPre{};
    const double thr = ((d.tau * d.tau) * treeA[td.off[0]]) * treeB[td.off[0]];
    int cnt = 0;
    bool listed = false;
    if (wid < m * m) {
        const int i = wid / m, k = wid - (wid / m) * m;
        int* const out = d.jlist + (size_t)wid * m;
        cnt = small ? cull_tile_small(pre, thr, m, lane, out) : cull_tile(td, treeA, treeB, thr, i, k, lane, out);
        if (lane == 0) {
            d.counts[wid] = cnt;
            listed = cnt > 0 || (d.mode != EPI_PLAIN && i == k);
            if (!listed) d.Ctree[wid] = 0.0;
        }
    }
    if (lane == 0) {
        lst[warp] = listed ? ((bt.x << kItemShift) | wid) : -1;
        bkt[warp] = tile_bucket(cnt);
        red[warp] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int c[kTileBuckets] = {0, 0, 0, 0, 0};
        int sacc = 0;
        for (int w = 0; w < 8; ++w) {
            if (lst[w] >= 0) ++c[bkt[w]];
            sacc += red[w];
        }
        int q[kTileBuckets];
        for (int b = 0; b < kTileBuckets; ++b) q[b] = c[b] ? atomicAdd(tile_count + b, c[b]) : 0;
        for (int w = 0; w < 8; ++w)
            if (lst[w] >= 0) tile_list[(size_t)bkt[w] * cap + q[bkt[w]]++] = lst[w];
        if (sacc) atomicAdd(d.task_ctr + 3 * (size_t)d.mflags[1] + d.which, (unsigned long long)sacc);
    }
}

void launch_cull_batched(const ProdDesc* prods, const int4* blocks, int nblocks, int* tile_list, int* tile_count,
                         int cap, const int* all_done, cudaStream_t st) {
    launch_dependent(k_cull_batched, dim3(nblocks), dim3(256), 0, st, prods, blocks, tile_list, tile_count, cap,
                     all_done);
    note_launch();
}

// Upper quadtree levels of every product output of a stage, one block per product; the stage's cost-class
// counters are cleared for its next cull.  In the X stage (x_stage) each live matrix also records its
// trace error t_k = (n - tr X)/n, counts the iteration and stops (|t_k| <= tol_t > 0, or maxit steps), as
// k_tree does for one solve; the last block to finish ends the batch once every matrix has stopped (and,
// in a graph's loop body, clears the loop's condition).
template <bool kLoop>
__global__ void __launch_bounds__(1024) k_tree_batched(const ProdDesc* __restrict__ prods, int nprod,
                                                      int* __restrict__ tile_count, int* __restrict__ stage_ctr,
                                                      int* __restrict__ ndone, int count, int* __restrict__ all_done,
                                                      cudaGraphConditionalHandle cond, int x_stage) {
    grid_dependency_wait();
    if (*all_done) return;
    __shared__ double bufA[64 * 64];
    __shared__ double bufB[32 * 32];
    const ProdDesc& d = prods[blockIdx.x];
    const bool live = d.mflags[0] == 0;
    if (live) {
        if (d.td.L <= 6) tree_levels_small(d.td, d.Ctree, bufB);
        else tree_levels<1024>(d.td, d.Ctree, bufA, bufB);
    }
    if (blockIdx.x == 0 && threadIdx.x < kTileBuckets) tile_count[threadIdx.x] = 0;
    if (!x_stage) return;
    if (live && threadIdx.x < 32) {
        const double tr = trace_sum_warp(d.trace_part, d.td.m);
        if (threadIdx.x == 0) {
            const int k = d.mflags[1];
            const double t = ((double)d.n - tr) / (double)d.n;
            d.t_hist[k] = t;
            d.mflags[1] = k + 1;
            if ((d.tol_t > 0.0 && fabs(t) <= d.tol_t) || k + 1 >= d.maxit) {
                d.mflags[0] = 1;
                atomicAdd(ndone, 1);
            }
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(stage_ctr, 1) == nprod - 1) {
            *stage_ctr = 0;
            if (atomicAdd(ndone, 0) >= count) {
                *all_done = 1;
                if constexpr (kLoop) cudaGraphSetConditional(cond, 0u);
            }
        }
    }
}

void launch_tree_batched(const ProdDesc* prods, int nprod, int* tile_count, int* stage_ctr, int* ndone, int count,
                         int* all_done, const cudaGraphConditionalHandle* cond, bool x_stage, cudaStream_t st) {
    if (cond)
        launch_dependent(k_tree_batched<true>, dim3(nprod), dim3(1024), 0, st, prods, nprod, tile_count, stage_ctr,
                         ndone, count, all_done, *cond, x_stage ? 1 : 0);
    else
        launch_dependent(k_tree_batched<false>, dim3(nprod), dim3(1024), 0, st, prods, nprod, tile_count, stage_ctr,
                         ndone, count, all_done, (cudaGraphConditionalHandle)0, x_stage ? 1 : 0);
    note_launch();
}

// ---------------------------------------------------------------- unpack
// One 256-thread block per tile, entries t + 256 q per thread, sixteen independent loads at a time; an
// all-zero tile (leaf norm 0) is written as zeros without reading it.
template <int NB, bool kScale>
__device__ __forceinline__ void unpack_tile(const double* __restrict__ s, bool zero, int n, int i, int j, double f,
                                            double* __restrict__ dst) {
    using TS = TileSplit<NB, 16>;
    if (zero) {
        // an all-zero tile (its scale factor is positive, so +0 either way) costs stores only
        for (int idx = threadIdx.x; idx < NB * NB; idx += 256) {
            const int gi = i * NB + idx / NB, gj = j * NB + idx % NB;
            if (gi < n && gj < n) dst[(size_t)gi * n + gj] = 0.0;
        }
        return;
    }
#pragma unroll 1
    for (int q0 = 0; q0 < TS::kPer; q0 += TS::kBatch) {
        double v[TS::kBatch];
#pragma unroll
        for (int u = 0; u < TS::kBatch; ++u) v[u] = s[threadIdx.x + 256 * (q0 + u)];
#pragma unroll
        for (int u = 0; u < TS::kBatch; ++u) {
            const int idx = threadIdx.x + 256 * (q0 + u);
            const int gi = i * NB + idx / NB, gj = j * NB + idx % NB;
            if (gi < n && gj < n) dst[(size_t)gi * n + gj] = kScale ? v[u] * f : v[u];
        }
    }
}

template <int NB>
__global__ void __launch_bounds__(256) k_unpack(const double* __restrict__ src, const double* __restrict__ leaf,
                                                int n, int m, double* __restrict__ dst,
                                                const double* __restrict__ scale_dev,
                                                const double* __restrict__ src_alt, const double* __restrict__ leaf_alt,
                                                const int* __restrict__ iters, int iters_src) {
    const int tile = blockIdx.x;
    const int i = tile / m, j = tile - (tile / m) * m;
    if (iters && ((*iters - iters_src) & 1)) {
        src = src_alt;
        leaf = leaf_alt;
    }
    const double* s = src + (size_t)tile * NB * NB;
    const bool zero = leaf && leaf[tile] == 0.0;
    if (scale_dev) unpack_tile<NB, true>(s, zero, n, i, j, *scale_dev, dst);
    else unpack_tile<NB, false>(s, zero, n, i, j, 1.0, dst);
}

void launch_unpack(const double* src, const double* leaf, const Geometry& g, double* dst, const double* scale,
                   cudaStream_t st, const double* src_alt, const double* leaf_alt, const int* iters, int iters_src) {
    const dim3 grid(g.m * g.m), block(256);
    if (g.nb == 32)
        k_unpack<32><<<grid, block, 0, st>>>(src, leaf, g.n, g.m, dst, scale, src_alt, leaf_alt, iters, iters_src);
    else if (g.nb == 64)
        k_unpack<64><<<grid, block, 0, st>>>(src, leaf, g.n, g.m, dst, scale, src_alt, leaf_alt, iters, iters_src);
    else
        k_unpack<128><<<grid, block, 0, st>>>(src, leaf, g.n, g.m, dst, scale, src_alt, leaf_alt, iters, iters_src);
    note_launch();
}

// ---------------------------------------------------------------- residual ||R - I||_F
__global__ void __launch_bounds__(256) k_resid_tiles(const double* __restrict__ R, int n, int m, int nb,
                                                     double* __restrict__ partial) {
    __shared__ double red[8];
    const int tile = blockIdx.x;
    const int i = tile / m, j = tile % m;
    const int ne = nb * nb;
    const double* r = R + (size_t)tile * ne;
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < ne; idx += 256) {
        const int rr = idx / nb, cc = idx - rr * nb;
        const int gi = i * nb + rr, gj = j * nb + cc;
        if (gi < n && gj < n) {
            const double d = r[idx] - (gi == gj ? 1.0 : 0.0);
            acc = fma(d, d, acc);
        }
    }
    const double s = block_sum_256(acc, red);
    if (threadIdx.x == 0) partial[tile] = s;
}

__global__ void k_sum_sqrt(const double* __restrict__ partial, int cnt, double* __restrict__ out) {
    double s = 0.0;
    for (int q = 0; q < cnt; ++q) s += partial[q];
    *out = sqrt(s);
}

void launch_resid_norm(const double* R, const Geometry& g, double* partial, double* out, cudaStream_t st) {
    k_resid_tiles<<<g.m * g.m, 256, 0, st>>>(R, g.n, g.m, g.nb, partial);
    note_launch();
    k_sum_sqrt<<<1, 1, 0, st>>>(partial, g.m * g.m, out);
    note_launch();
}

}  // namespace spamm

/*
 * Plain FP64 CPU oracle for the SpAMM product and the dual-channel
 * Newton-Schulz square-root iteration (Challacombe, Haut & Bock,
 * "A N-Body Solver for Square Root Iteration").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only the tests, the package smoke check and the bench's CPU-baseline leg
 * load it.  It shares no code, header or constant with the CUDA library.
 *
 * Everything is written the slow, obvious way:
 *   - matrices are dense, row-major, n x n, double precision;
 *   - the quadtree is built over a grid of m = ceil(n/nb) leaf tiles;
 *     tiles on the ragged edge are zero-padded inside the tile, and quadtree
 *     nodes that cover no tile of the matrix do not exist;
 *   - node norms are squared Frobenius norms ("nu"), a parent being the sum
 *     of its existing children in the order 00, 01, 10, 11 (Sec. 1, the
 *     quadtree and its norm recursion);
 *   - the cull is the recursive two-sided query of Eq. (newspamm) with the
 *     relative criterion ||a^i|| ||b^i|| < tau ||a|| ||b||, evaluated in
 *     squared form nu_a * nu_b < (tau*tau) * nu_A * nu_B, strict "<" culls;
 *   - the 2x2 block product inside the recursion is the ordinary one
 *     (c00 = a00 b00 + a01 b10, c01 = a00 b01 + a01 b11,
 *      c10 = a10 b00 + a11 b10, c11 = a10 b01 + a11 b11);
 *   - leaf products are triple loops, accumulated per output tile with the
 *     surviving j in ascending order and the inner index ascending;
 *   - the square-root iteration is Eq. (cannonical) (or Eq. (single), the
 *     single channel instance), started from
 *     X0 = Y0 = S / c, Z0 = I, where c is the Gershgorin bound of the
 *     largest eigenvalue (Sec. 3.2), with T = h_alpha[U] the NS logistic of
 *     Sec. 4.2 "Mapping" applied to the stabilised U = eps I + (1-2 eps) X:
 *     map 0 is alpha = 1, eps = 0 (T = 1.5 I - 0.5 X); map 1 takes alpha
 *     and eps from the sigmoidal damping functions of the trace error t of
 *     the X being mapped.
 *
 * Parity-pinned by tests/test_oracle_pins.py, every function:
 *   - products and culls: the tau = 0 dense product (bitwise), a worked 4x4,
 *     the tile-level closed form of the lemma, recursive == brute-force cull
 *     sets, the Proposition's bounds, the norm-tree levels;
 *   - the iteration: eigen-decomposition iterates, diagonal S against the
 *     scalar recursion (bitwise), the 2x2 closed form, convergence
 *     identities, the KMS inverse, padding invariance, the order variants;
 *   - the damped map: the sigmoid landmarks, eigen iterates, its fixed point;
 *   - the single channel: a hand-worked 2x2, eigen iterates, diagonal S;
 *   - lensing histograms: a dense closed form, an identity operand, hand
 *     triples;
 *   - the product representation: telescoping at tau = 0, conditioning, the
 *     transpose;
 *   - the Gershgorin bound and the residual: closed forms.
 * No function is left "parity unpinned".
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (see oracle/__init__.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_NOMEM -2
#define OR_ERR_CAP -3

/* ------------------------------------------------------------------------- */
/* quadtree of squared Frobenius norms                                        */
/* ------------------------------------------------------------------------- */

typedef struct {
    int m;          /* leaf tiles per side                                    */
    int L;          /* leaf level: smallest L with 2^L >= m                    */
    int dim[32];    /* existing nodes per side at level l                     */
    long off[32];   /* offset of level l in nu[]                              */
    double* nu;     /* all levels, level l row-major dim[l] x dim[l]          */
} or_tree;

static int ceil_log2(int m) {
    int L = 0;
    while ((1 << L) < m) ++L;
    return L;
}

int or_tiles_per_side(int n, int nb) { return (n + nb - 1) / nb; }
int or_leaf_level(int m) { return ceil_log2(m); }

/* Leaf norm nu_ij = sum of squares of tile (i,j), summed in row-major order
 * inside the tile over the entries that lie in the matrix (Sec. 1). */
void or_leaf_norms(const double* A, int n, int nb, double* nu) {
    int m = or_tiles_per_side(n, nb);
    #pragma omp parallel for schedule(static)
    for (int t = 0; t < m * m; ++t) {
        int i = t / m, j = t % m;
        double acc = 0.0;
        for (int r = i * nb; r < (i + 1) * nb && r < n; ++r)
            for (int c = j * nb; c < (j + 1) * nb && c < n; ++c) {
                double a = A[(long)r * n + c];
                acc += a * a;
            }
        nu[t] = acc;
    }
}

static int tree_build(or_tree* T, const double* leaf, int m) {
    T->m = m;
    T->L = ceil_log2(m);
    long total = 0;
    for (int l = T->L; l >= 0; --l) {
        int shift = T->L - l;
        T->dim[l] = (m + (1 << shift) - 1) >> shift;
        T->off[l] = total;
        total += (long)T->dim[l] * T->dim[l];
    }
    T->nu = (double*)malloc(sizeof(double) * (size_t)total);
    if (!T->nu) return OR_ERR_NOMEM;
    memcpy(T->nu + T->off[T->L], leaf, sizeof(double) * (size_t)m * m);
    for (int l = T->L - 1; l >= 0; --l) {
        int d = T->dim[l], dc = T->dim[l + 1];
        for (int I = 0; I < d; ++I)
            for (int J = 0; J < d; ++J) {
                double s = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        int ci = 2 * I + a, cj = 2 * J + b;
                        if (ci < dc && cj < dc) s += T->nu[T->off[l + 1] + (long)ci * dc + cj];
                    }
                T->nu[T->off[l] + (long)I * d + J] = s;
            }
    }
    return OR_OK;
}

static void tree_free(or_tree* T) { free(T->nu); T->nu = NULL; }

static double tree_at(const or_tree* T, int l, int I, int J) {
    return T->nu[T->off[l] + (long)I * T->dim[l] + J];
}

/* Whole tree, exported for tests: levels from leaf (L) up to root (0).
 * out must hold sum_l dim[l]^2 doubles; level_off/level_dim get L+1 entries. */
int or_norm_tree(const double* A, int n, int nb, double* out, long* level_off, int* level_dim) {
    int m = or_tiles_per_side(n, nb);
    double* leaf = (double*)malloc(sizeof(double) * (size_t)m * m);
    if (!leaf) return OR_ERR_NOMEM;
    or_leaf_norms(A, n, nb, leaf);
    or_tree T;
    int st = tree_build(&T, leaf, m);
    free(leaf);
    if (st) return st;
    long total = 0;
    for (int l = 0; l <= T.L; ++l) total += (long)T.dim[l] * T.dim[l];
    memcpy(out, T.nu, sizeof(double) * (size_t)total);
    for (int l = 0; l <= T.L; ++l) { level_off[l] = T.off[l]; level_dim[l] = T.dim[l]; }
    tree_free(&T);
    return T.L;
}

/* ------------------------------------------------------------------------- */
/* the two-sided metric query, Eq. (newspamm)                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    const or_tree* A;
    const or_tree* B;
    double thr;
    int* out;       /* triples (i, j, k)                                      */
    long cap;
    long count;
} cull_ctx;

/* Node triple at level l: A(I,J) times B(J,K) contributes to C(I,K). */
static void cull_rec(cull_ctx* cx, int l, int I, int J, int K) {
    const or_tree* A = cx->A;
    int d = A->dim[l];
    if (I >= d || J >= d || K >= d) return;            /* node does not exist */
    if (tree_at(cx->A, l, I, J) * tree_at(cx->B, l, J, K) < cx->thr) return;  /* culled */
    if (l == A->L) {                                    /* leaf: a^i . b^i    */
        if (cx->count < cx->cap) {
            cx->out[3 * cx->count + 0] = I;
            cx->out[3 * cx->count + 1] = J;
            cx->out[3 * cx->count + 2] = K;
        }
        cx->count++;
        return;
    }
    /* c_ab = a_a0 b_0b + a_a1 b_1b for the four quadrants (ab = 00, 01, 10, 11) */
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e)
                cull_rec(cx, l + 1, 2 * I + a, 2 * J + e, 2 * K + b);
}

double or_threshold(double tau, double nuA_root, double nuB_root) {
    return ((tau * tau) * nuA_root) * nuB_root;
}

static int cmp_ikj(const void* pa, const void* pb) {
    const int* a = (const int*)pa;
    const int* b = (const int*)pb;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;   /* i */
    if (a[2] != b[2]) return a[2] < b[2] ? -1 : 1;   /* k */
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;   /* j */
    return 0;
}

/* Recursive cull of A x B: writes surviving leaf triples (i,j,k) sorted by
 * (i, k, j) into tasks (3*cap ints) and returns how many survive (may exceed
 * cap, in which case only the first cap found are stored and the list is not
 * sorted; callers size cap = m^3).  thr_out receives the threshold used. */
long or_cull(const double* A, const double* B, int n, int nb, double tau, int* tasks, long cap,
             double* thr_out) {
    int m = or_tiles_per_side(n, nb);
    double* la = (double*)malloc(sizeof(double) * (size_t)m * m);
    double* lb = (double*)malloc(sizeof(double) * (size_t)m * m);
    if (!la || !lb) { free(la); free(lb); return OR_ERR_NOMEM; }
    or_leaf_norms(A, n, nb, la);
    or_leaf_norms(B, n, nb, lb);
    or_tree TA, TB;
    if (tree_build(&TA, la, m) || tree_build(&TB, lb, m)) { free(la); free(lb); return OR_ERR_NOMEM; }
    free(la); free(lb);
    cull_ctx cx;
    cx.A = &TA; cx.B = &TB;
    cx.thr = or_threshold(tau, tree_at(&TA, 0, 0, 0), tree_at(&TB, 0, 0, 0));
    cx.out = tasks; cx.cap = cap; cx.count = 0;
    cull_rec(&cx, 0, 0, 0, 0);
    if (cx.count <= cap) qsort(tasks, (size_t)cx.count, 3 * sizeof(int), cmp_ikj);
    if (thr_out) *thr_out = cx.thr;
    tree_free(&TA); tree_free(&TB);
    return cx.count;
}

/* Brute force over all m^3 leaf triples with the same leaf test, for the
 * recursive == flat check.  Leaf norms and root norms come from the same tree
 * construction as or_cull. */
long or_cull_flat(const double* A, const double* B, int n, int nb, double tau, int* tasks, long cap) {
    int m = or_tiles_per_side(n, nb);
    double* la = (double*)malloc(sizeof(double) * (size_t)m * m);
    double* lb = (double*)malloc(sizeof(double) * (size_t)m * m);
    if (!la || !lb) { free(la); free(lb); return OR_ERR_NOMEM; }
    or_leaf_norms(A, n, nb, la);
    or_leaf_norms(B, n, nb, lb);
    or_tree TA, TB;
    if (tree_build(&TA, la, m) || tree_build(&TB, lb, m)) { free(la); free(lb); return OR_ERR_NOMEM; }
    double thr = or_threshold(tau, tree_at(&TA, 0, 0, 0), tree_at(&TB, 0, 0, 0));
    long cnt = 0;
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k)
            for (int j = 0; j < m; ++j)
                if (!(la[i * m + j] * lb[j * m + k] < thr)) {
                    if (cnt < cap) {
                        tasks[3 * cnt + 0] = i;
                        tasks[3 * cnt + 1] = j;
                        tasks[3 * cnt + 2] = k;
                    }
                    cnt++;
                }
    free(la); free(lb);
    tree_free(&TA); tree_free(&TB);
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* leaf products                                                               */
/* ------------------------------------------------------------------------- */

/* C = sum over the given (i,j,k) triples (sorted by (i,k,j)) of A_ij B_jk.
 * Output tiles with no triple are zero.  Per output element the sum runs over
 * j ascending, then the inner index ascending. */
void or_leaf_products(const double* A, const double* B, double* C, int n, int nb,
                      const int* tasks, long ntasks) {
    int m = or_tiles_per_side(n, nb);
    long* start = (long*)calloc((size_t)m * m + 1, sizeof(long));
    for (long t = 0; t < ntasks; ++t) start[tasks[3 * t] * m + tasks[3 * t + 2] + 1]++;
    for (long q = 0; q < (long)m * m; ++q) start[q + 1] += start[q];
    #pragma omp parallel for schedule(dynamic, 1)
    for (long q = 0; q < (long)m * m; ++q) {
        int i = (int)(q / m), k = (int)(q % m);
        int r0 = i * nb, r1 = (i + 1) * nb < n ? (i + 1) * nb : n;
        int c0 = k * nb, c1 = (k + 1) * nb < n ? (k + 1) * nb : n;
        double* acc = (double*)calloc((size_t)nb * nb, sizeof(double));
        for (long t = start[q]; t < start[q + 1]; ++t) {
            int j = tasks[3 * t + 1];
            int l0 = j * nb, l1 = (j + 1) * nb < n ? (j + 1) * nb : n;
            for (int r = r0; r < r1; ++r)
                for (int l = l0; l < l1; ++l) {
                    double a = A[(long)r * n + l];
                    const double* brow = B + (long)l * n;
                    double* arow = acc + (long)(r - r0) * nb;
                    for (int c = c0; c < c1; ++c) arow[c - c0] += a * brow[c];
                }
        }
        for (int r = r0; r < r1; ++r)
            for (int c = c0; c < c1; ++c) C[(long)r * n + c] = acc[(long)(r - r0) * nb + (c - c0)];
        free(acc);
    }
    free(start);
}

/* C = A (x)_tau B.  tasks may be NULL (the triples are then kept internally).
 * Returns the number of surviving leaf triples, or a negative error. */
long or_spamm(const double* A, const double* B, double* C, int n, int nb, double tau,
              int* tasks, long cap) {
    int m = or_tiles_per_side(n, nb);
    long full = (long)m * m * m;
    int* own = NULL;
    if (!tasks || cap < full) {
        own = (int*)malloc(sizeof(int) * 3 * (size_t)full);
        if (!own) return OR_ERR_NOMEM;
    }
    int* tl = own ? own : tasks;
    long cnt = or_cull(A, B, n, nb, tau, tl, full, NULL);
    if (cnt < 0) { free(own); return cnt; }
    or_leaf_products(A, B, C, n, nb, tl, cnt);
    if (own && tasks) memcpy(tasks, own, sizeof(int) * 3 * (size_t)(cnt < cap ? cnt : cap));
    free(own);
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* dual-channel Newton-Schulz square-root iteration, Eq. (cannonical)         */
/* ------------------------------------------------------------------------- */

/* Gershgorin bound max_i sum_j |s_ij| of S + mu I (Sec. 3.2 rescaling). */
double or_gershgorin(const double* S, int n, double mu) {
    double c = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = 0; j < n; ++j) {
            double v = S[(long)i * n + j];
            if (i == j) v += mu;
            r += fabs(v);
        }
        if (r > c) c = r;
    }
    return c;
}

/*
 * Damping of the NS map, Sec. 4.2 "Mapping": with the relative trace error t
 * of the matrix being mapped, the logistic scale is
 *   alpha(t) = 1 + 1.85 / (1 + exp(-50 (t - 0.35)))
 * and the stabiliser width
 *   eps(t)   = 0.1 / (1 + exp(-75 (t - 0.30))),
 * so that both are switched off (alpha -> 1, eps -> 0) as t -> 0.
 * map 0 is the plain map: alpha = 1, eps = 0 for every t.
 */
void or_map_params(int map, double t, double* alpha, double* eps) {
    if (map == 0) {
        *alpha = 1.0;
        *eps = 0.0;
        return;
    }
    *alpha = 1.0 + 1.85 / (1.0 + exp(-50.0 * (t - 0.35)));
    *eps = 0.1 / (1.0 + exp(-75.0 * (t - 0.30)));
}

/*
 * T = h_alpha[U] = (sqrt(alpha)/2) (3 I - alpha U) with U = eps I + (1 - 2 eps) X,
 * the stabilising shift-and-scale of [0,1] onto [eps, 1-eps] followed by the
 * NS logistic (Sec. 4.2 "Mapping"); alpha and eps from t (or_map_params).
 */
static void or_apply_map(const double* X, double* T, int n, int map, double t) {
    double alpha, eps;
    or_map_params(map, t, &alpha, &eps);
    const double half_root = 0.5 * sqrt(alpha);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double x = X[(long)i * n + j];
            const double u = (i == j) ? eps + (1.0 - 2.0 * eps) * x : (1.0 - 2.0 * eps) * x;
            T[(long)i * n + j] = half_root * ((i == j ? 3.0 : 0.0) - alpha * u);
        }
}

/* t = (n - tr X) / n, the relative trace error (Sec. 4.2). */
static double or_trace_error(const double* X, int n) {
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += X[(long)i * n + i];
    return ((double)n - tr) / (double)n;
}

/*
 * Plane-diagonal profile of a task list (the "lensing" of Sec. 7.2: the
 * culled volume collapsing onto the plane diagonals of the ijk cube).
 * hist[q * bins + d] += number of surviving triples (i, j, k) whose distance
 * d from plane q is that many tiles: q = 0 |i - j| (plane i = j, the left
 * operand's diagonal), q = 1 |j - k| (the right operand's), q = 2 |i - k|
 * (the product's); d >= bins counts in the last bin.
 */
void or_lens_hist(const int* tasks, long cnt, int bins, long* hist) {
    for (long t = 0; t < cnt; ++t) {
        const int i = tasks[3 * t], j = tasks[3 * t + 1], k = tasks[3 * t + 2];
        const int d[3] = {abs(i - j), abs(j - k), abs(i - k)};
        for (int q = 0; q < 3; ++q) hist[q * bins + (d[q] < bins ? d[q] : bins - 1)] += 1;
    }
}

/* T = A^T (n x n). */
static void or_transpose(const double* A, double* T, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) T[(long)j * n + i] = A[(long)i * n + j];
}

/*
 * Y -> S^{1/2}, Z -> S^{-1/2} by the dual channel iteration with
 * T = h_alpha[eps I + (1 - 2 eps) X] (or_apply_map; map 0: T = 1.5 I - 0.5 X):
 *   order 0 (as printed):  Y <- T (x)_{tau_s} Y,  Z <- Z (x)_tau T
 *   order 1 (transposed):  Y <- Y (x)_{tau_s} T,  Z <- T (x)_tau Z
 *   then X <- Y (x)_tau Z (order 0) or X <- Z (x)_tau Y (order 1), and
 *   t_k = (n - tr X) / n (Sec. 4.2).
 * mu_rel > 0 regularises with S + mu I, mu = mu_rel * (Gershgorin bound of S)
 * (Sec. 6).  The map applied to X_k takes alpha and eps from t_k of that same
 * X_k (t_0 from X0 = S / c).
 *
 * channel 1 is the single channel instance, Eq. (single), from X0 = s = S / c
 * and Z0 = I:
 *   Z <- Z (x)_tau T,   W <- s (x)_{tau_s} Z,   X <- Z^T (x)_tau W,
 * i.e. x_k = z_k^T s z_k with the inner product s z_k taken first, at the
 * sensitive threshold tau_s as in the volume plots of the single instance
 * (Sec. 5.3); Y = W (s z -> s^{1/2}).  Only the printed order (order 0) is
 * defined for it.
 *
 * The iteration stops after maxit steps or once |t_k| <= tol_t (tol_t > 0).
 * t_hist (maxit) and task_hist (3*maxit: the y, z, x products of the dual
 * channel; z, s z, x of the single channel) may be NULL.  lens_hist may be
 * NULL or hold maxit * 3 * 3 * lens_bins counts: the plane-diagonal profile
 * (or_lens_hist) of product p of iteration k at ((k * 3 + p) * 3) * lens_bins.
 * Returns the number of iterations run; *scale_c receives c.
 */
int or_ns(const double* S, int n, int nb, double tau, double tau_s, double mu_rel, int maxit,
          int order, double tol_t, int map, int channel, double* Y, double* Z, double* t_hist,
          long* task_hist, long* lens_hist, int lens_bins, double* scale_c) {
    if (n <= 0 || nb <= 0 || maxit < 0 || !(tau >= 0.0) || !(tau_s >= 0.0) || map < 0 || map > 1 ||
        channel < 0 || channel > 1 || (channel == 1 && order != 0) || (lens_hist && lens_bins <= 0))
        return OR_ERR_ARG;
    const int m = or_tiles_per_side(n, nb);
    const long full = (long)m * m * m;
    size_t nn = (size_t)n * n;
    double* X = (double*)malloc(sizeof(double) * nn);
    double* T = (double*)malloc(sizeof(double) * nn);
    double* W = (double*)malloc(sizeof(double) * nn);
    double* s1 = channel == 1 ? (double*)malloc(sizeof(double) * nn) : NULL;
    double* Zt = channel == 1 ? (double*)malloc(sizeof(double) * nn) : NULL;
    int* tl = lens_hist ? (int*)malloc(sizeof(int) * 3 * (size_t)full) : NULL;
    if (!X || !T || !W || (channel == 1 && (!s1 || !Zt)) || (lens_hist && !tl)) {
        free(X); free(T); free(W); free(s1); free(Zt); free(tl);
        return OR_ERR_NOMEM;
    }
    const long cap = tl ? full : 0;
#define OR_LENS(p, cnt) \
    if (tl && (cnt) >= 0) or_lens_hist(tl, (cnt), lens_bins, lens_hist + ((long)k * 3 + (p)) * 3 * lens_bins)

    double mu = 0.0;
    if (mu_rel > 0.0) mu = mu_rel * or_gershgorin(S, n, 0.0);
    double c = or_gershgorin(S, n, mu);
    /* s <- s / c (Sec. 3.2, rescaling into (0, 1]), applied as a product with the once-rounded 1/c */
    const double rc = 1.0 / c;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = S[(long)i * n + j];
            if (i == j) v += mu;
            Y[(long)i * n + j] = v * rc;
            Z[(long)i * n + j] = (i == j) ? 1.0 : 0.0;
        }
    memcpy(X, Y, sizeof(double) * nn);
    if (channel == 1) memcpy(s1, Y, sizeof(double) * nn);
    double t_cur = or_trace_error(X, n);

    int it = 0;
    for (int k = 0; k < maxit; ++k) {
        or_apply_map(X, T, n, map, t_cur);
        long ty, tz, tx;
        if (channel == 1) {
            /* Eq. (single): z_k = z_{k-1} h[x_{k-1}], x_k = z_k^T s z_k */
            tz = or_spamm(Z, T, W, n, nb, tau, tl, cap);
            OR_LENS(0, tz);
            memcpy(Z, W, sizeof(double) * nn);
            ty = or_spamm(s1, Z, Y, n, nb, tau_s, tl, cap);
            OR_LENS(1, ty);
            or_transpose(Z, Zt, n);
            tx = or_spamm(Zt, Y, X, n, nb, tau, tl, cap);
            OR_LENS(2, tx);
            if (ty < 0 || tz < 0 || tx < 0) {
                free(X); free(T); free(W); free(s1); free(Zt); free(tl);
                return OR_ERR_NOMEM;
            }
            const double tk = or_trace_error(X, n);
            t_cur = tk;
            if (t_hist) t_hist[k] = tk;
            if (task_hist) { task_hist[3 * k] = tz; task_hist[3 * k + 1] = ty; task_hist[3 * k + 2] = tx; }
            it = k + 1;
            if (tol_t > 0.0 && fabs(tk) <= tol_t) break;
            continue;
        }
        if (order == 0) {
            ty = or_spamm(T, Y, W, n, nb, tau_s, tl, cap);
            OR_LENS(0, ty);
            memcpy(Y, W, sizeof(double) * nn);
            tz = or_spamm(Z, T, W, n, nb, tau, tl, cap);
            OR_LENS(1, tz);
            memcpy(Z, W, sizeof(double) * nn);
        } else {
            ty = or_spamm(Y, T, W, n, nb, tau_s, tl, cap);
            OR_LENS(0, ty);
            memcpy(Y, W, sizeof(double) * nn);
            tz = or_spamm(T, Z, W, n, nb, tau, tl, cap);
            OR_LENS(1, tz);
            memcpy(Z, W, sizeof(double) * nn);
        }
        /* X = Y Z as printed; the transposed variant needs X = Z Y (the exact
         * transpose of the printed iteration for symmetric iterates).  Pairing
         * Y T / T Z with X = Y Z is unstable near the fixed point. */
        if (order == 0) tx = or_spamm(Y, Z, X, n, nb, tau, tl, cap);
        else tx = or_spamm(Z, Y, X, n, nb, tau, tl, cap);
        OR_LENS(2, tx);
        if (ty < 0 || tz < 0 || tx < 0) {
            free(X); free(T); free(W); free(s1); free(Zt); free(tl);
            return OR_ERR_NOMEM;
        }
        const double tk = or_trace_error(X, n);
        t_cur = tk;
        if (t_hist) t_hist[k] = tk;
        if (task_hist) { task_hist[3 * k] = ty; task_hist[3 * k + 1] = tz; task_hist[3 * k + 2] = tx; }
        it = k + 1;
        if (tol_t > 0.0 && fabs(tk) <= tol_t) break;
    }
    /* single channel with no iteration: Y = s Z0 = s, already in Y */
    /* undo the scaling: Y sqrt(c), Z / sqrt(c), the latter as a product with the once-rounded 1/sqrt(c) */
    const double sc = sqrt(c), rsc = 1.0 / sc;
    for (size_t q = 0; q < nn; ++q) { Y[q] = Y[q] * sc; Z[q] = Z[q] * rsc; }
    if (scale_c) *scale_c = c;
#undef OR_LENS
    free(X); free(T); free(W); free(s1); free(Zt); free(tl);
    return it;
}

/*
 * Product representation of the regularised inverse factor (Sec. 6,
 * Eq. (spammsandwich), with the iterative regularisation of Eq. (product_rep)):
 *   z_0 = (S + mu_0 c0 I)^{-1/2} by or_ns at tau0 (dual channel, map 0,
 *         mu_rel = mu_0; the most-approximate-yet-effective slice),
 *   Z = z_0, and for l = 1 .. levels-1:
 *     R_l = Z^T (x)_{tau1} ((S + mu_l c0 I) (x)_{tau1} Z)   (the residual),
 *     z_l = R_l^{-1/2} by or_ns at tau0 (no shift),
 *     Z  <- Z (x)_{tau1} z_l,
 * so that Z^T (S + mu_{levels-1} c0 I) Z -> I.  c0 is the Gershgorin bound of
 * S (shifts relative to it, like mu_rel).  Each or_ns runs maxit iterations,
 * or fewer with tol_t > 0.  iters (levels) may be NULL.  Returns 0 or an
 * OR_ERR code.
 */
int or_invsqrt_product(const double* S, int n, int nb, int levels, const double* mu, double tau0, double tau1,
                       int maxit, double tol_t, double* Zout, int* iters) {
    if (n <= 0 || nb <= 0 || levels < 1 || maxit < 0 || !(tau0 >= 0.0) || !(tau1 >= 0.0)) return OR_ERR_ARG;
    for (int l = 0; l < levels; ++l)
        if (!(mu[l] >= 0.0)) return OR_ERR_ARG;
    const size_t nn = (size_t)n * n;
    double* Y = (double*)malloc(sizeof(double) * nn);
    double* z = (double*)malloc(sizeof(double) * nn);
    double* Sm = (double*)malloc(sizeof(double) * nn);
    double* W = (double*)malloc(sizeof(double) * nn);
    double* Zt = (double*)malloc(sizeof(double) * nn);
    double* R = (double*)malloc(sizeof(double) * nn);
    int rc = OR_OK;
    if (!Y || !z || !Sm || !W || !Zt || !R) { rc = OR_ERR_NOMEM; goto done; }
    {
        const double c0 = or_gershgorin(S, n, 0.0);
        int it = or_ns(S, n, nb, tau0, 0.01 * tau0, mu[0], maxit, 0, tol_t, 0, 0, Y, Zout, NULL, NULL, NULL, 0,
                       NULL);
        if (it < 0) { rc = it; goto done; }
        if (iters) iters[0] = it;
        for (int l = 1; l < levels; ++l) {
            memcpy(Sm, S, sizeof(double) * nn);
            for (int i = 0; i < n; ++i) Sm[(long)i * n + i] += mu[l] * c0;
            if (or_spamm(Sm, Zout, W, n, nb, tau1, NULL, 0) < 0) { rc = OR_ERR_NOMEM; goto done; }
            or_transpose(Zout, Zt, n);
            if (or_spamm(Zt, W, R, n, nb, tau1, NULL, 0) < 0) { rc = OR_ERR_NOMEM; goto done; }
            it = or_ns(R, n, nb, tau0, 0.01 * tau0, 0.0, maxit, 0, tol_t, 0, 0, Y, z, NULL, NULL, NULL, 0, NULL);
            if (it < 0) { rc = it; goto done; }
            if (iters) iters[l] = it;
            if (or_spamm(Zout, z, W, n, nb, tau1, NULL, 0) < 0) { rc = OR_ERR_NOMEM; goto done; }
            memcpy(Zout, W, sizeof(double) * nn);
        }
    }
done:
    free(Y); free(z); free(Sm); free(W); free(Zt); free(R);
    return rc;
}

/* ||Z S Z - I||_F with plain triple loops (verification of a finished solve). */
double or_residual(const double* S, const double* Z, int n) {
    size_t nn = (size_t)n * n;
    double* W = (double*)calloc(nn, sizeof(double));
    double* R = (double*)calloc(nn, sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < n; ++l) {
            double a = Z[(long)i * n + l];
            for (int j = 0; j < n; ++j) W[(long)i * n + j] += a * S[(long)l * n + j];
        }
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < n; ++l) {
            double a = W[(long)i * n + l];
            for (int j = 0; j < n; ++j) R[(long)i * n + j] += a * Z[(long)l * n + j];
        }
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double d = R[(long)i * n + j] - (i == j ? 1.0 : 0.0);
            s += d * d;
        }
    free(W); free(R);
    return sqrt(s);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

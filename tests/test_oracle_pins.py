"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a hand-worked
example, a closed form, an independent brute force, a theorem's bound or an
eigen-decomposition identity.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _tiles(n, nb):
    return (n + nb - 1) // nb


def _np_leaf_norms_int(A, nb):
    """Tile norms for integer-valued inputs (every sum is exact, so the order does not matter)."""
    n = A.shape[0]
    m = _tiles(n, nb)
    P = np.zeros((m * nb, m * nb))
    P[:n, :n] = A
    return (P.reshape(m, nb, m, nb) ** 2).sum(axis=(1, 3))


def _decaying_int(n, seed, length=4.0, amp=6):
    """Integer matrix with an exponentially decaying envelope: tile norms spread over orders of magnitude,
    and every FP64 sum of products is exact."""
    rng = np.random.default_rng(seed)
    i = np.arange(n)
    env = np.floor(amp * np.exp(-np.abs(i[:, None] - i[None, :]) / length) + 0.5)
    return env * rng.integers(-2, 3, size=(n, n))


# --------------------------------------------------------------------------- hand-worked example


def test_worked_example_4x4():
    g = json.load(open(os.path.join(GOLD, "spamm_worked_4x4.json")))
    A = np.array(g["A"], dtype=np.float64)
    for case in g["cases"]:
        C, cnt = oracle.spamm(A, A, g["nb"], case["tau"])
        np.testing.assert_array_equal(C, np.array(case["C"], dtype=np.float64))
        tasks, _ = oracle.cull(A, A, g["nb"], case["tau"])
        want = sorted((i, j, k) for i, j, k in case["tasks_ikj"])
        assert sorted(map(tuple, tasks.tolist())) == want
        assert cnt == len(want)
        # the list is ordered by output tile (i, k), then j ascending
        assert [tuple(t) for t in tasks.tolist()] == sorted(want, key=lambda t: (t[0], t[2], t[1]))


# --------------------------------------------------------------------------- P1: tau = 0 is the dense product


@pytest.mark.parametrize("n,nb", [(16, 4), (37, 8), (64, 16), (100, 32), (5, 8)])
def test_tau_zero_is_dense_product_bitwise(n, nb):
    A = synth.integer_matrix(n, seed=1)
    B = synth.integer_matrix(n, seed=2)
    C, cnt = oracle.spamm(A, B, nb, 0.0)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(C, exact)
    assert cnt == _tiles(n, nb) ** 3


# --------------------------------------------------------------------------- P2: tile-level closed form of the lemma


@pytest.mark.parametrize("n,nb,tau", [(64, 8, 1e-2), (64, 8, 5e-2), (96, 16, 2e-2), (70, 8, 3e-2), (128, 16, 1e-3)])
def test_tile_closed_form(n, nb, tau):
    """C_ik = sum_j A_ij B_jk [nu_A(i,j) nu_B(j,k) >= tau^2 nu_A nu_B] (the lemma of the Proposition at tile
    granularity; the recursion is equivalent to this flat test because parent norms dominate their children)."""
    A = _decaying_int(n, 3)
    B = _decaying_int(n, 4, length=6.0)
    m = _tiles(n, nb)
    na, nbm = _np_leaf_norms_int(A, nb), _np_leaf_norms_int(B, nb)
    thr = ((tau * tau) * na.sum()) * nbm.sum()
    P = m * nb
    Ap = np.zeros((P, P), dtype=np.int64)
    Bp = np.zeros((P, P), dtype=np.int64)
    Ap[:n, :n] = A
    Bp[:n, :n] = B
    want = np.zeros((P, P), dtype=np.int64)
    kept = 0
    for i in range(m):
        for k in range(m):
            for j in range(m):
                if not (na[i, j] * nbm[j, k] < thr):
                    kept += 1
                    want[i * nb:(i + 1) * nb, k * nb:(k + 1) * nb] += \
                        Ap[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] @ Bp[j * nb:(j + 1) * nb, k * nb:(k + 1) * nb]
    C, cnt = oracle.spamm(A, B, nb, tau)
    assert 0 < cnt < m ** 3, "choose tau so that the cull is not trivial"
    assert cnt == kept
    np.testing.assert_array_equal(C, want[:n, :n].astype(np.float64))


def test_elementwise_lemma_nb1():
    """At N_b = 1 every culled term satisfies |a_il||b_lj| < tau ||a|| ||b|| and every kept one does not."""
    n = 24
    A = _decaying_int(n, 5, length=3.0)
    B = _decaying_int(n, 6, length=3.0)
    tau = 0.02
    C, _ = oracle.spamm(A, B, 1, tau)
    tab2 = (tau * tau) * (A * A).sum() * (B * B).sum()
    keep = (A[:, :, None] ** 2) * (B[None, :, :] ** 2) >= tab2          # [i, l, j]
    want = np.einsum("il,lj,ilj->ij", A, B, keep.astype(np.float64))
    np.testing.assert_array_equal(C, want)


# --------------------------------------------------------------------------- P3: recursion == brute force


@pytest.mark.parametrize("n,nb,tau", [(64, 4, 1e-2), (100, 8, 1e-3), (128, 8, 5e-2), (33, 4, 0.0), (200, 16, 1e-3)])
def test_recursive_cull_equals_flat(n, nb, tau):
    A = synth.decay_matrix(n, seed=7, length=5.0)
    B = synth.decay_matrix(n, seed=8, length=9.0)
    rec, thr = oracle.cull(A, B, nb, tau)
    flat = oracle.cull_flat(A, B, nb, tau)
    np.testing.assert_array_equal(rec, flat)
    # independent numpy brute force with the oracle's own leaf norms and threshold
    la, lb = oracle.leaf_norms(A, nb), oracle.leaf_norms(B, nb)
    keep = ~((la[:, :, None] * lb[None, :, :]) < thr)           # [i, j, k]
    ii, jj, kk = np.nonzero(keep)
    brute = np.stack([ii, jj, kk], 1)
    brute = brute[np.lexsort((brute[:, 1], brute[:, 2], brute[:, 0]))]
    np.testing.assert_array_equal(rec, brute)


def test_norm_tree_levels():
    """Each level is the sum of its existing children; the root is ||A||_F^2; ragged grids have no phantom nodes."""
    n, nb = 77, 8
    A = synth.integer_matrix(n, seed=9)
    levels = oracle.norm_tree(A, nb)
    m = _tiles(n, nb)
    assert levels[-1].shape == (m, m)
    np.testing.assert_array_equal(levels[-1], _np_leaf_norms_int(A, nb))
    assert levels[0].shape == (1, 1) and levels[0][0, 0] == (A * A).sum()
    for l in range(len(levels) - 1):
        child = levels[l + 1]
        d = levels[l].shape[0]
        pad = np.zeros((2 * d, 2 * d))
        pad[:child.shape[0], :child.shape[1]] = child
        np.testing.assert_array_equal(levels[l], pad.reshape(d, 2, d, 2).sum(axis=(1, 3)))


# --------------------------------------------------------------------------- P4: the Proposition's bounds


@pytest.mark.parametrize("tau", [1e-1, 3e-2, 1e-2, 1e-3])
@pytest.mark.parametrize("nb", [1, 4, 16])
def test_proposition_bounds(tau, nb):
    n = 64
    A = synth.decay_matrix(n, seed=11, length=4.0)
    B = synth.decay_matrix(n, seed=12, length=6.0)
    C, _ = oracle.spamm(A, B, nb, tau)
    D = C - A @ B
    tab = tau * np.linalg.norm(A) * np.linalg.norm(B)
    slack = 1e-12 * np.abs(A) .sum() * np.abs(B).sum()     # rounding of the two products
    assert np.abs(D).max() <= n * tab + slack
    assert np.linalg.norm(D) <= n * n * tab + slack
    # sharper: the error is at most the sum over culled tile pairs of ||A_ij|| ||B_jk||
    tasks, _ = oracle.cull(A, B, nb, tau)
    la, lb = oracle.leaf_norms(A, nb), oracle.leaf_norms(B, nb)
    m = la.shape[0]
    kept = np.zeros((m, m, m), dtype=bool)
    kept[tasks[:, 0], tasks[:, 1], tasks[:, 2]] = True
    cullsum = (np.sqrt(la[:, :, None] * lb[None, :, :]) * (~kept)).sum()
    assert np.linalg.norm(D) <= cullsum * (1 + 1e-12) + slack


def test_normwise_tau_bound_is_not_a_theorem():
    """||A(x)B - AB|| <= tau ||A|| ||B|| without the n^2 factor fails on the all-ones matrix (reading of the bound)."""
    n = 16
    A = np.ones((n, n))
    tau = 1.01 / (n * n)        # every leaf |a||b| = 1 < tau * n^2 at N_b = 1
    C, cnt = oracle.spamm(A, A, 1, tau)
    assert cnt == 0 and not C.any()
    err = np.linalg.norm(C - A @ A)
    tab = tau * np.linalg.norm(A) ** 2
    assert err > 10 * tab
    assert err <= n * n * tab


# --------------------------------------------------------------------------- P5: NS iterates in the eigenbasis


def _scalar_ns(lam, iters, order=0):
    y = lam.copy()
    z = np.ones_like(lam)
    x = lam.copy()
    for _ in range(iters):
        t = 1.5 - 0.5 * x
        if order == 0:
            y = t * y
            z = z * t
        else:
            y = y * t
            z = t * z
        x = y * z
    return y, z


@pytest.mark.parametrize("iters", [1, 2, 5, 12])
def test_ns_iterates_match_eigen_recursion(iters):
    n, nb = 40, 8
    S = synth.gaussian_lattice(n, sigma=0.7, seed=0)
    c = np.abs(S).sum(1).max()
    lam, Q = np.linalg.eigh(S / c)
    y, z = _scalar_ns(lam, iters)
    r = oracle.sqrt_invsqrt(S, nb, 0.0, iters)
    Yk = (Q * (y * math.sqrt(c))) @ Q.T
    Zk = (Q * (z / math.sqrt(c))) @ Q.T
    assert r["iters"] == iters
    assert np.linalg.norm(r["Y"] - Yk) <= 1e-12 * np.linalg.norm(Yk)
    assert np.linalg.norm(r["Z"] - Zk) <= 1e-11 * np.linalg.norm(Zk)


@pytest.mark.parametrize("scale", [1.0, 0.95])
def test_ns_diagonal_is_scalar_recursion_bitwise(scale):
    # scale 0.95 makes c = 1.9, where s * RN(1/c) and s / c differ in 10 of the 12 entries
    d = np.array([0.9, 0.05, 0.3, 1.7, 0.011, 0.6, 2.0, 0.25, 0.125, 1.0, 0.75, 0.4]) * scale
    S = np.diag(d)
    c = d.max()
    for order in (0, 1):
        r = oracle.sqrt_invsqrt(S, 4, 0.0, 9, order=order)
        # the scaling is a product with the once-rounded reciprocals 1/c and 1/sqrt(c)
        y, z = _scalar_ns(d * (1.0 / c), 9, order)
        np.testing.assert_array_equal(np.diag(r["Y"]), y * math.sqrt(c))
        np.testing.assert_array_equal(np.diag(r["Z"]), z * (1.0 / math.sqrt(c)))
        assert not (r["Y"] - np.diag(np.diag(r["Y"]))).any()


# --------------------------------------------------------------------------- P6/P7: convergence, KMS


def test_sqrt_2x2_closed_form():
    g = json.load(open(os.path.join(GOLD, "sqrt_2x2.json")))
    S = np.array(g["S"], dtype=np.float64)
    ev = {"sqrt": math.sqrt}
    Yw = np.array([[eval(e, {"__builtins__": {}}, ev) for e in row] for row in g["sqrt_expr"]])
    Zw = np.array([[eval(e, {"__builtins__": {}}, ev) for e in row] for row in g["invsqrt_expr"]])
    r = oracle.sqrt_invsqrt(S, 1, 0.0, 40)
    np.testing.assert_allclose(r["Y"], Yw, rtol=0, atol=4e-16 * 4)
    np.testing.assert_allclose(r["Z"], Zw, rtol=0, atol=4e-16 * 4)


@pytest.mark.parametrize("kind", ["gauss", "kms"])
def test_ns_converges_to_square_roots(kind):
    n, nb = 96, 16
    S = synth.gaussian_lattice(n, 0.6, seed=0) if kind == "gauss" else synth.kms(n, 0.9)
    r = oracle.sqrt_invsqrt(S, nb, 0.0, 30)
    lam, Q = np.linalg.eigh(S)
    Sh = (Q * np.sqrt(lam)) @ Q.T
    Smh = (Q / np.sqrt(lam)) @ Q.T
    Y, Z = r["Y"], r["Z"]
    kappa = lam.max() / lam.min()
    tol = 1e-13 * kappa
    assert np.linalg.norm(Y - Sh) <= tol * np.linalg.norm(Sh)
    assert np.linalg.norm(Z - Smh) <= tol * np.linalg.norm(Smh)
    assert np.linalg.norm(Y @ Z - np.eye(n)) <= tol * math.sqrt(n)
    assert oracle.residual(S, Z) <= tol * math.sqrt(n)
    assert np.linalg.norm(Y @ Y - S) <= tol * np.linalg.norm(S)
    assert abs(r["t_hist"][-1]) <= 1e-14


def test_kms_inverse_closed_form():
    n, rho = 64, 0.9
    S = synth.kms(n, rho)
    Sinv = synth.kms_inverse(n, rho)
    # the closed form itself: S * Sinv = I
    np.testing.assert_allclose(S @ Sinv, np.eye(n), atol=1e-12)
    r = oracle.sqrt_invsqrt(S, 16, 0.0, 30)
    Z = r["Z"]
    assert np.linalg.norm(Z @ Z - Sinv) <= 1e-11 * np.linalg.norm(Sinv)
    # spectrum of KMS lies in [(1-rho)/(1+rho), (1+rho)/(1-rho)]
    lam = np.linalg.eigvalsh(S)
    assert lam.min() >= (1 - rho) / (1 + rho) - 1e-12 and lam.max() <= (1 + rho) / (1 - rho) + 1e-12


# --------------------------------------------------------------------------- P8: padding invariance, order


@pytest.mark.parametrize("tau", [0.0, 1e-3])
def test_zero_padding_invariance(tau):
    n, nb = 50, 16
    A = synth.decay_matrix(n, seed=21)
    B = synth.decay_matrix(n, seed=22)
    C, _ = oracle.spamm(A, B, nb, tau)
    P = 64
    Ap = np.zeros((P, P)); Ap[:n, :n] = A
    Bp = np.zeros((P, P)); Bp[:n, :n] = B
    Cp, _ = oracle.spamm(Ap, Bp, nb, tau)
    np.testing.assert_array_equal(Cp[:n, :n], C)
    assert not Cp[n:, :].any() and not Cp[:, n:].any()


def test_transpose_consistency_integer():
    n, nb, tau = 72, 8, 2e-2
    A = _decaying_int(n, 31)
    B = _decaying_int(n, 32, length=7.0)
    C, c1 = oracle.spamm(A, B, nb, tau)
    Ct, c2 = oracle.spamm(B.T.copy(), A.T.copy(), nb, tau)
    assert c1 == c2
    np.testing.assert_array_equal(C.T, Ct)


def test_order_variants_agree():
    n, nb = 64, 8
    S = synth.gaussian_lattice(n, 0.7, seed=2)
    a = oracle.sqrt_invsqrt(S, nb, 0.0, 25, order=0)
    b = oracle.sqrt_invsqrt(S, nb, 0.0, 25, order=1)
    assert np.linalg.norm(a["Z"] - b["Z"]) <= 1e-12 * np.linalg.norm(a["Z"])


def test_tol_stop_and_regularisation():
    n, nb = 64, 16
    S = synth.kms(n, 0.8)
    r = oracle.sqrt_invsqrt(S, nb, 0.0, 50, tol_t=1e-12)
    assert r["iters"] < 50 and abs(r["t_hist"][-1]) <= 1e-12
    mu_rel = 1e-3
    c0 = oracle.gershgorin(S)
    r2 = oracle.sqrt_invsqrt(S, nb, 0.0, 40, mu_rel=mu_rel)
    Smu = S + mu_rel * c0 * np.eye(n)
    lam, Q = np.linalg.eigh(Smu)
    assert np.linalg.norm(r2["Z"] - (Q / np.sqrt(lam)) @ Q.T) <= 1e-12 * np.linalg.norm(r2["Z"]) * 10
    assert r2["scale_c"] == pytest.approx(c0 + mu_rel * c0, rel=1e-15)


# --------------------------------------------------------------------------- the damped, stabilised NS map (Sec. 4.2)


def test_map_sigmoid_landmarks():
    """alpha(t) and eps(t) against the landmarks of their definitions: the plain map, the asymptotes, the
    midpoints (where the logistic factor is exactly 1/2) and the slopes there (amplitude * rate / 4)."""
    assert oracle.map_params(0.7, oracle.MAP_NS) == (1.0, 0.0)
    a, e = oracle.map_params(0.35)
    assert a == pytest.approx(1.0 + 1.85 / 2, rel=1e-15)
    a, e = oracle.map_params(0.30)
    assert e == pytest.approx(0.1 / 2, rel=1e-15)
    assert oracle.map_params(20.0) == (pytest.approx(2.85, rel=1e-15), pytest.approx(0.1, rel=1e-15))
    a, e = oracle.map_params(-20.0)
    assert a == 1.0 and 0.0 <= e < 1e-300
    h = 1e-6
    da = (oracle.map_params(0.35 + h)[0] - oracle.map_params(0.35 - h)[0]) / (2 * h)
    de = (oracle.map_params(0.30 + h)[1] - oracle.map_params(0.30 - h)[1]) / (2 * h)
    assert da == pytest.approx(1.85 * 50 / 4, rel=1e-7)
    assert de == pytest.approx(0.1 * 75 / 4, rel=1e-7)
    # both damp monotonically towards the plain map as t -> 0
    ts = np.linspace(-0.2, 1.0, 61)
    al = [oracle.map_params(t)[0] for t in ts]
    ep = [oracle.map_params(t)[1] for t in ts]
    assert all(np.diff(al) >= 0) and all(np.diff(ep) >= 0)


def _scalar_scaled_ns(lam, iters, order=0):
    """The scaled, stabilised map acting on the eigenvalues: for symmetric S = Q diag(lam) Q^T every iterate is
    Q f(lam) Q^T, and t = (n - tr X)/n = 1 - mean(x) couples the eigenvalues only through alpha and eps."""
    y = lam.copy()
    z = np.ones_like(lam)
    x = lam.copy()
    for _ in range(iters):
        a, e = oracle.map_params(1.0 - x.mean())
        u = e + (1.0 - 2.0 * e) * x
        t = 0.5 * math.sqrt(a) * (3.0 - a * u)
        y = t * y
        z = z * t
        x = y * z
    return y, z


@pytest.mark.parametrize("iters", [1, 3, 8])
def test_scaled_map_matches_eigen_recursion(iters):
    n, nb = 40, 8
    S = synth.gaussian_lattice(n, sigma=0.9, seed=0)
    c = np.abs(S).sum(1).max()
    lam, Q = np.linalg.eigh(S / c)
    y, z = _scalar_scaled_ns(lam, iters)
    for order in (0, 1):
        r = oracle.sqrt_invsqrt(S, nb, 0.0, iters, order=order, map=oracle.MAP_SCALED)
        Yk = (Q * (y * math.sqrt(c))) @ Q.T
        Zk = (Q * (z / math.sqrt(c))) @ Q.T
        assert np.linalg.norm(r["Y"] - Yk) <= 1e-12 * np.linalg.norm(Yk)
        assert np.linalg.norm(r["Z"] - Zk) <= 1e-11 * np.linalg.norm(Zk)


def test_scaled_map_fixed_point():
    """At convergence h_alpha[u] = 1 with u = eps + (1 - 2 eps) x, i.e. u* = (3 - 2/sqrt(alpha))/alpha and
    x* = (u* - eps)/(1 - 2 eps), with alpha and eps taken at t* = 1 - x* (solved here by fixed-point
    iteration of that scalar equation).  The stabiliser leaves the trace error at t* ~ -eps(0), not 0."""
    xs = 1.0
    for _ in range(60):
        a, e = oracle.map_params(1.0 - xs)
        us = (3.0 - 2.0 / math.sqrt(a)) / a
        xs = (us - e) / (1.0 - 2.0 * e)
    t_star = 1.0 - xs
    assert -1.8e-11 < t_star < -1.6e-11
    S = synth.kms(128, 0.9)
    r = oracle.sqrt_invsqrt(S, 16, 0.0, 40, map=oracle.MAP_SCALED)
    assert abs(r["t_hist"][-1] - t_star) <= 2e-14
    # ZSZ = x* I at the fixed point
    assert oracle.residual(S, r["Z"]) == pytest.approx(abs(t_star) * math.sqrt(128), rel=2e-3)


@pytest.mark.parametrize("kind", ["kms", "gauss"])
def test_scaled_map_accelerates(kind):
    """The scaled map needs fewer iterations than alpha = 1 on ill-conditioned inputs (Sec. 4.2)."""
    S = synth.kms(200, 0.99) if kind == "kms" else synth.gaussian_lattice(125, 0.9, seed=0)

    def iters_to(mp):
        r = oracle.sqrt_invsqrt(S, 16, 0.0, 60, map=mp, tol_t=1e-9)
        assert abs(r["t_hist"][-1]) <= 1e-9
        return r["iters"]

    assert iters_to(oracle.MAP_SCALED) + 3 <= iters_to(oracle.MAP_NS)


# --------------------------------------------------------------------------- the single channel instance, Eq. (single)


def test_single_channel_worked_2x2():
    g = json.load(open(os.path.join(GOLD, "single_channel_2x2.json")))
    S = np.array(g["S"])
    r = oracle.sqrt_invsqrt(S, 1, 0.0, 1, channel=oracle.CHANNEL_SINGLE)
    assert r["scale_c"] == g["scale_c"]
    assert r["t_hist"][0] == g["t1"]
    sc = math.sqrt(g["scale_c"])
    np.testing.assert_array_equal(r["Y"], np.array(g["w1"]) * sc)
    np.testing.assert_array_equal(r["Z"], np.array(g["z1"]) * (1.0 / sc))


def _scalar_single(lam, iters, scaled=False):
    """Eq. (single) on the eigenvalues: z <- z h[x], x = z^2 lam (z^T s z for commuting symmetric factors)."""
    z = np.ones_like(lam)
    x = lam.copy()
    for _ in range(iters):
        a, e = oracle.map_params(1.0 - x.mean(), oracle.MAP_SCALED if scaled else oracle.MAP_NS)
        t = 0.5 * math.sqrt(a) * (3.0 - a * (e + (1.0 - 2.0 * e) * x))
        z = z * t
        x = z * z * lam
    return lam * z, z


@pytest.mark.parametrize("iters,scaled", [(1, False), (4, False), (12, False), (3, True), (9, True)])
def test_single_channel_matches_eigen_recursion(iters, scaled):
    n, nb = 40, 8
    S = synth.gaussian_lattice(n, sigma=0.8, seed=1)
    c = np.abs(S).sum(1).max()
    lam, Q = np.linalg.eigh(S / c)
    y, z = _scalar_single(lam, iters, scaled)
    r = oracle.sqrt_invsqrt(S, nb, 0.0, iters, channel=oracle.CHANNEL_SINGLE,
                            map=oracle.MAP_SCALED if scaled else oracle.MAP_NS)
    Yk = (Q * (y * math.sqrt(c))) @ Q.T
    Zk = (Q * (z / math.sqrt(c))) @ Q.T
    assert np.linalg.norm(r["Y"] - Yk) <= 1e-12 * np.linalg.norm(Yk)
    assert np.linalg.norm(r["Z"] - Zk) <= 1e-11 * np.linalg.norm(Zk)


def test_single_channel_diagonal_is_scalar_recursion_bitwise():
    d = np.array([0.9, 0.05, 0.3, 1.7, 0.011, 0.6, 2.0, 0.25, 0.125, 1.0, 0.75, 0.4])
    c = d.max()
    r = oracle.sqrt_invsqrt(np.diag(d), 4, 0.0, 9, channel=oracle.CHANNEL_SINGLE)
    lam = d * (1.0 / c)
    z = np.ones_like(lam)
    x = lam.copy()
    for _ in range(9):
        z = z * (1.5 - 0.5 * x)
        w = lam * z
        x = z * w
    np.testing.assert_array_equal(np.diag(r["Z"]), z * (1.0 / math.sqrt(c)))
    np.testing.assert_array_equal(np.diag(r["Y"]), w * math.sqrt(c))


@pytest.mark.parametrize("iters", [2, 7, 20])
def test_single_and_dual_channels_agree_at_tau0(iters):
    """In exact arithmetic y_k = s z_k, so x_k = y_k z_k = z_k^T s z_k: both instances give the same iterates."""
    S = synth.kms(96, 0.9)
    a = oracle.sqrt_invsqrt(S, 16, 0.0, iters)
    b = oracle.sqrt_invsqrt(S, 16, 0.0, iters, channel=oracle.CHANNEL_SINGLE)
    assert np.linalg.norm(a["Z"] - b["Z"]) <= 1e-12 * np.linalg.norm(a["Z"])
    assert np.linalg.norm(a["Y"] - b["Y"]) <= 1e-12 * np.linalg.norm(a["Y"])
    np.testing.assert_allclose(a["t_hist"], b["t_hist"], rtol=0, atol=1e-13)


def test_single_channel_rejects_transposed_order():
    with pytest.raises(RuntimeError):
        oracle.sqrt_invsqrt(synth.kms(16, 0.5), 4, 0.0, 2, order=1, channel=oracle.CHANNEL_SINGLE)


def test_single_channel_s_product_threshold_is_tau_s():
    """W = s (x)_{tau_s} z (the single instance's sensitive product): after one step its task count is the
    brute-force count of the leaf test at tau_s, which differs here from the count at tau."""
    n, nb, tau = 96, 8, 2e-3
    S = synth.gaussian_lattice(n, 0.6, seed=5)
    r = oracle.sqrt_invsqrt(S, nb, tau, 1, tau_s=0.01 * tau, channel=oracle.CHANNEL_SINGLE)
    c = r["scale_c"]
    s = S * (1.0 / c)
    z1 = r["Z"] * math.sqrt(c)
    n_tau_s = len(oracle.cull_flat(s, z1, nb, 0.01 * tau))
    n_tau = len(oracle.cull_flat(s, z1, nb, tau))
    assert n_tau_s != n_tau
    assert r["task_hist"][0][1] == n_tau_s


# --------------------------------------------------------------------------- plane-diagonal profile ("lensing", Sec. 7.2)


def test_lens_profile_dense_closed_form():
    """At tau = 0 every (i, j, k) survives: for each plane, distance 0 holds m^2 triples and distance d > 0
    holds m * 2 (m - d); the task counts of every product are m^3."""
    n, nb = 70, 10  # m = 7
    m = 7
    S = synth.kms(n, 0.9)
    r = oracle.sqrt_invsqrt(S, nb, 0.0, 2, lens_bins=m)
    want = np.array([m * m] + [m * 2 * (m - d) for d in range(1, m)])
    for k in range(2):
        for p in range(3):
            assert r["task_hist"][k][p] == m ** 3
            for q in range(3):
                np.testing.assert_array_equal(r["lens_hist"][k, p, q], want)


def test_lens_profile_identity_operand_lies_on_its_plane():
    """With Z0 = I the first z product Z0 (x) T0 has a left operand supported on tile diagonal only, so its
    whole volume lies on the plane i = j; the counts agree with the task count; a narrow last bin collects
    every distance beyond it."""
    n, nb = 96, 8
    S = synth.gaussian_lattice(n, 0.6, seed=3)
    r = oracle.sqrt_invsqrt(S, nb, 1e-6, 3, lens_bins=4)
    h = r["lens_hist"]
    z0 = h[0, 1]
    assert z0[0, 0] == r["task_hist"][0][1] and z0[0, 1:].sum() == 0
    assert (h.sum(axis=3) == r["task_hist"][:, :, None]).all()
    tasks, _ = oracle.cull(S, S, nb, 1e-3)
    full = oracle.lens_hist(tasks, 12)  # m = 12: every distance has its own bin
    narrow = oracle.lens_hist(tasks, 4)
    np.testing.assert_array_equal(narrow[:, :3], full[:, :3])
    np.testing.assert_array_equal(narrow[:, 3], full[:, 3:].sum(axis=1))


def test_lens_profile_hand_triples():
    # (i, j, k) = (0, 1, 3): 1 tile from plane i = j, 2 from j = k, 3 from i = k; (5, 5, 0): 0, 5 -> last bin, 5
    h = oracle.lens_hist(np.array([[0, 1, 3], [5, 5, 0]]), 5)
    want = np.zeros((3, 5), dtype=np.int64)
    want[0, 1] += 1; want[1, 2] += 1; want[2, 3] += 1
    want[0, 0] += 1; want[1, 4] += 1; want[2, 4] += 1
    np.testing.assert_array_equal(h, want)


# --------------------------------------------------------------------------- product representation (Sec. 6)


@pytest.mark.parametrize("mus", [[0.1, 0.0], [0.1, 0.01, 0.001], [0.05, 0.005, 0.0005, 0.0]])
def test_product_representation_telescopes_at_tau0(mus):
    """At tau = 0 every slice is a function of S, so Z = z_0 z_1 ... is (S + mu_last c0 I)^{-1/2} exactly
    (each residual is (S + mu_l c0)(S + mu_{l-1} c0)^{-1} in its eigenbasis)."""
    S = synth.gaussian_lattice(125, 0.9, seed=0)
    lam, Q = np.linalg.eigh(S)
    c0 = oracle.gershgorin(S)
    r = oracle.invsqrt_product(S, 16, mus, 0.0, 0.0, 60)
    Zw = (Q / np.sqrt(lam + mus[-1] * c0)) @ Q.T
    assert np.linalg.norm(r["Z"] - Zw) <= 1e-12 * np.linalg.norm(Zw)
    assert len(r["iters"]) == len(mus)


def test_product_representation_improves_conditioning():
    """Each level improves the effective condition number of Z^T S Z (Sec. 6, iterative regularisation):
    here by about an order per level at tau0 = 1e-3, tau1 = 1e-5, and the residual shrinks."""
    S = synth.gaussian_lattice(125, 0.9, seed=0)
    kap, res = [], []
    for L in (1, 2, 3):
        r = oracle.invsqrt_product(S, 16, [0.1, 0.01, 0.001][:L], 1e-3, 1e-5, 40)
        M = r["Z"].T @ S @ r["Z"]
        ev = np.linalg.eigvalsh(0.5 * (M + M.T))
        kap.append(ev.max() / ev.min())
        res.append(np.linalg.norm(M - np.eye(len(M))))
    assert kap[0] > 5 * kap[1] > 25 * kap[2], kap
    assert res[0] > res[1] > res[2], res


def test_product_representation_residual_uses_the_transpose():
    """The residual is z0^T (S + mu_1 c0 I) z0 as printed (Sec. 6).  On a nonsymmetric S whose slices are not
    symmetric, the result must equal z0 (z0^T S_mu1 z0)^{-1/2} built from scipy's principal square roots
    (the NS map converges to the principal root); without the transpose it differs by ~7e-2."""
    sl = pytest.importorskip("scipy.linalg")
    S = np.array([[2.0, 1.0, 0.0], [0.0, 3.0, 1.0], [0.5, 0.0, 4.0]])
    c0 = oracle.gershgorin(S)
    mus = [0.1, 0.0]
    z0 = np.linalg.inv(sl.sqrtm(S + mus[0] * c0 * np.eye(3))).real
    r1 = z0.T @ (S + mus[1] * c0 * np.eye(3)) @ z0
    want = z0 @ np.linalg.inv(sl.sqrtm(r1)).real
    r = oracle.invsqrt_product(S, 1, mus, 0.0, 0.0, 80)
    np.testing.assert_allclose(r["Z"], want, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------- Gershgorin bound and residual


def test_gershgorin_closed_form():
    """max_i sum_j |s_ij + mu delta_ij| (the rescaling bound of Sec. 3.2): row sums of absolute values with
    the shift on the diagonal.  Here the row sums are 3.5 and 6.5; column sums (a transposed loop) would give
    5.5, signed sums (a dropped |.|) -0.5 in both rows, and an ignored shift 7.0."""
    S = np.array([[1.0, -2.0], [3.0, -4.0]])
    assert oracle.gershgorin(S, 0.5) == 6.5
    assert oracle.gershgorin(S) == 7.0
    assert oracle.gershgorin(S.T, 0.5) == 5.5


def test_residual_closed_forms():
    """||Z S Z - I||_F: zero for an exact inverse square root, sqrt(sum (d_i - 1)^2) for Z = I and diagonal S,
    and (Z S Z)_{01} = z00 s01 z11 for a triangular Z that a transposed product would get wrong."""
    S = np.diag([4.0, 16.0, 0.25])
    assert oracle.residual(S, np.diag([0.5, 0.25, 2.0])) == 0.0
    d = np.array([2.0, 0.5, 3.0])
    assert oracle.residual(np.diag(d), np.eye(3)) == pytest.approx(math.sqrt(((d - 1.0) ** 2).sum()), rel=1e-15)
    Z = np.array([[1.0, 2.0], [0.0, 1.0]])
    S2 = np.array([[1.0, 0.0], [0.0, 1.0]])
    # Z S Z = Z^2 = [[1, 4], [0, 1]]: residual 4 (Z S Z^T would give [[5, 2], [2, 1]], residual sqrt(24))
    assert oracle.residual(S2, Z) == 4.0

"""Plain FP64 CPU oracle for SpAMM and dual-channel Newton-Schulz iteration.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the library never does.  The
arithmetic lives in ``spamm_oracle.c`` (plain loops, no BLAS), compiled with
gcc into ``oracle/_build/liboracle.so``; this module only marshals numpy
arrays.  It shares no code with the CUDA path.

Paper references (Challacombe, Haut & Bock, "A N-Body Solver for Square Root
Iteration"): the quadtree and its Frobenius-norm recursion (Sec. 1), the
stable SpAMM occlusion cull, Eq. (newspamm), the dual-channel square-root
iteration, Eq. (cannonical), the trace error t_k and the damped, stabilised
NS map (Sec. 4.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spamm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over output tiles, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lp = ctypes.POINTER(ctypes.c_long)
            L.or_leaf_norms.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            L.or_leaf_norms.restype = None
            L.or_norm_tree.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, lp, ip]
            L.or_norm_tree.restype = ctypes.c_int
            L.or_threshold.argtypes = [ctypes.c_double] * 3
            L.or_threshold.restype = ctypes.c_double
            L.or_cull.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ip, ctypes.c_long, dp]
            L.or_cull.restype = ctypes.c_long
            L.or_cull_flat.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ip, ctypes.c_long]
            L.or_cull_flat.restype = ctypes.c_long
            L.or_leaf_products.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_long]
            L.or_leaf_products.restype = None
            L.or_spamm.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ip, ctypes.c_long]
            L.or_spamm.restype = ctypes.c_long
            L.or_gershgorin.argtypes = [dp, ctypes.c_int, ctypes.c_double]
            L.or_gershgorin.restype = ctypes.c_double
            L.or_ns.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp, dp, lp,
                                lp, ctypes.c_int, dp]
            L.or_invsqrt_product.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, ip]
            L.or_invsqrt_product.restype = ctypes.c_int
            L.or_lens_hist.argtypes = [ip, ctypes.c_long, ctypes.c_int, lp]
            L.or_lens_hist.restype = None
            L.or_map_params.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
            L.or_map_params.restype = None
            L.or_ns.restype = ctypes.c_int
            L.or_residual.argtypes = [dp, dp, ctypes.c_int]
            L.or_residual.restype = ctypes.c_double
            L.or_num_threads.argtypes = []
            L.or_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _l(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _mat(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square matrix expected")
    return a


def tiles_per_side(n: int, nb: int) -> int:
    return (n + nb - 1) // nb


def num_threads() -> int:
    return lib().or_num_threads()


def leaf_norms(A, nb: int) -> np.ndarray:
    """Squared Frobenius norm of every nb x nb leaf tile (m x m array)."""
    A = _mat(A)
    m = tiles_per_side(A.shape[0], nb)
    out = np.zeros((m, m))
    lib().or_leaf_norms(_d(A), A.shape[0], nb, _d(out))
    return out


def norm_tree(A, nb: int) -> list[np.ndarray]:
    """All quadtree levels of squared norms, index 0 = root ... L = leaves."""
    A = _mat(A)
    n = A.shape[0]
    m = tiles_per_side(n, nb)
    L = max(0, int(np.ceil(np.log2(m)))) if m > 1 else 0
    total = sum(((m + (1 << (L - l)) - 1) >> (L - l)) ** 2 for l in range(L + 1))
    buf = np.zeros(total)
    off = np.zeros(L + 1, dtype=np.int64)
    dim = np.zeros(L + 1, dtype=np.int32)
    got = lib().or_norm_tree(_d(A), n, nb, _d(buf), _l(off), _i(dim))
    assert got == L
    return [buf[off[l]:off[l] + dim[l] * dim[l]].reshape(dim[l], dim[l]).copy() for l in range(L + 1)]


def threshold(tau: float, nuA_root: float, nuB_root: float) -> float:
    return lib().or_threshold(tau, nuA_root, nuB_root)


def cull(A, B, nb: int, tau: float) -> tuple[np.ndarray, float]:
    """Recursive two-sided query: surviving (i, j, k) leaf triples sorted by (i, k, j), and the threshold."""
    A, B = _mat(A), _mat(B)
    m = tiles_per_side(A.shape[0], nb)
    cap = m ** 3
    buf = np.zeros((cap, 3), dtype=np.int32)
    thr = np.zeros(1)
    cnt = lib().or_cull(_d(A), _d(B), A.shape[0], nb, tau, _i(buf), cap, _d(thr))
    if cnt < 0:
        raise MemoryError("oracle cull failed")
    return buf[:cnt].copy(), float(thr[0])


def cull_flat(A, B, nb: int, tau: float) -> np.ndarray:
    """Brute force over all m^3 leaf triples, in (i, k, j) order."""
    A, B = _mat(A), _mat(B)
    m = tiles_per_side(A.shape[0], nb)
    cap = m ** 3
    buf = np.zeros((cap, 3), dtype=np.int32)
    cnt = lib().or_cull_flat(_d(A), _d(B), A.shape[0], nb, tau, _i(buf), cap)
    return buf[:cnt].copy()


def leaf_products(A, B, nb: int, tasks: np.ndarray) -> np.ndarray:
    """Sum of A_ij B_jk over an explicit list of (i, j, k) triples sorted by (i, k, j)."""
    A, B = _mat(A), _mat(B)
    tasks = np.ascontiguousarray(tasks, dtype=np.int32).reshape(-1, 3)
    C = np.zeros_like(A)
    lib().or_leaf_products(_d(A), _d(B), _d(C), A.shape[0], nb, _i(tasks), tasks.shape[0])
    return C


def spamm(A, B, nb: int, tau: float) -> tuple[np.ndarray, int]:
    """C = A (x)_tau B and the number of surviving leaf products."""
    A, B = _mat(A), _mat(B)
    C = np.zeros_like(A)
    cnt = lib().or_spamm(_d(A), _d(B), _d(C), A.shape[0], nb, tau, None, 0)
    if cnt < 0:
        raise MemoryError("oracle spamm failed")
    return C, int(cnt)


def gershgorin(S, mu: float = 0.0) -> float:
    S = _mat(S)
    return lib().or_gershgorin(_d(S), S.shape[0], mu)


MAP_NS = 0      # alpha = 1, eps = 0: T = 1.5 I - 0.5 X
MAP_SCALED = 1  # sigmoidal alpha(t), eps(t) of Sec. 4.2 "Mapping"


def map_params(t: float, map: int = MAP_SCALED) -> tuple[float, float]:
    """(alpha, eps) of the NS map for relative trace error t."""
    a = np.zeros(1)
    e = np.zeros(1)
    lib().or_map_params(int(map), float(t), _d(a), _d(e))
    return float(a[0]), float(e[0])


CHANNEL_DUAL = 0    # Eq. (cannonical)
CHANNEL_SINGLE = 1  # Eq. (single): z <- z h[x], x = z^T s z


def lens_hist(tasks, bins: int) -> np.ndarray:
    """Plane-diagonal profile of a task list: [3, bins] counts of |i-j|, |j-k|, |i-k| (last bin: >= bins-1)."""
    tasks = np.ascontiguousarray(tasks, dtype=np.int32).reshape(-1, 3)
    h = np.zeros((3, bins), dtype=np.int64)
    lib().or_lens_hist(_i(tasks), tasks.shape[0], int(bins), _l(h))
    return h


def sqrt_invsqrt(S, nb: int, tau: float, maxit: int, tau_s: float | None = None, mu_rel: float = 0.0,
                 order: int = 0, tol_t: float = 0.0, map: int = MAP_NS, channel: int = CHANNEL_DUAL,
                 lens_bins: int = 0) -> dict:
    """NS square-root iteration (dual or single channel); returns Y ~ S^{1/2}, Z ~ S^{-1/2} and the
    per-iteration history (with lens_bins > 0 also the plane-diagonal profile of every product,
    [iters, 3 products, 3 planes, lens_bins])."""
    S = _mat(S)
    n = S.shape[0]
    if tau_s is None:
        tau_s = 0.01 * tau
    Y = np.zeros_like(S)
    Z = np.zeros_like(S)
    th = np.zeros(max(maxit, 1))
    kh = np.zeros((max(maxit, 1), 3), dtype=np.int64)
    c = np.zeros(1)
    lh = np.zeros((max(maxit, 1), 3, 3, max(lens_bins, 1)), dtype=np.int64)
    it = lib().or_ns(_d(S), n, nb, tau, tau_s, mu_rel, maxit, order, tol_t, int(map), int(channel), _d(Y), _d(Z),
                     _d(th), _l(kh), _l(lh) if lens_bins > 0 else None, int(lens_bins), _d(c))
    if it < 0:
        raise RuntimeError(f"oracle NS failed ({it})")
    out = {"Y": Y, "Z": Z, "iters": it, "t_hist": th[:it].copy(), "task_hist": kh[:it].copy(),
           "scale_c": float(c[0])}
    if lens_bins > 0:
        out["lens_hist"] = lh[:it].copy()
    return out


def invsqrt_product(S, nb: int, mus, tau0: float, tau1: float, maxit: int, tol_t: float = 0.0) -> dict:
    """Product representation of the regularised inverse factor: slice z_0 = (S + mu_0 c0 I)^{-1/2}, then per
    level the residual Z^T (S + mu_l c0 I) Z, its inverse square root z_l and Z <- Z z_l.  Returns Z (with
    Z^T (S + mu_last c0 I) Z -> I) and the NS iterations of every level."""
    S = _mat(S)
    n = S.shape[0]
    mus = np.ascontiguousarray(mus, dtype=np.float64)
    Z = np.zeros_like(S)
    its = np.zeros(len(mus), dtype=np.int32)
    rc = lib().or_invsqrt_product(_d(S), n, nb, len(mus), _d(mus), tau0, tau1, maxit, tol_t, _d(Z), _i(its))
    if rc != 0:
        raise RuntimeError(f"oracle product representation failed ({rc})")
    return {"Z": Z, "iters": its.copy(), "scale_c0": gershgorin(S)}


def residual(S, Z) -> float:
    """||Z S Z - I||_F by plain triple loops."""
    S, Z = _mat(S), _mat(Z)
    return lib().or_residual(_d(S), _d(Z), S.shape[0])

"""Python binding of libspamm, the GB300 SpAMM / Newton-Schulz library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/spamm.h``.  Matrices may be
numpy arrays (host memory) or torch tensors (host or CUDA); results come back
in the same kind of container as the first matrix argument.

Method: Challacombe, Haut & Bock, "A N-Body Solver for Square Root
Iteration" -- the SpAMM product of Eq. (newspamm) and the dual-channel
Newton-Schulz iteration of Eq. (cannonical).

Loading fails loudly when the CUDA library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build_lib

__all__ = ["FP64", "EMU64", "ORDER_PAPER", "ORDER_TRANSPOSED", "MAP_NS", "MAP_SCALED", "CHANNEL_DUAL",
           "CHANNEL_SINGLE", "SCHED_BRANCHES", "SCHED_STAGES", "SCHED_AUTO", "SpammError", "lib", "build", "multiply", "sqrt_invsqrt", "sqrt_invsqrt_batched",
           "invsqrt_product", "autotune_leaf", "norm_tree", "cull", "release", "version", "HEADER_SYMBOLS", "Server"]

FP64 = 0
EMU64 = 1
ORDER_PAPER = 0
ORDER_TRANSPOSED = 1
MAP_NS = 0       # T = (3I - X)/2 (alpha = 1)
MAP_SCALED = 1   # damped, stabilised h_alpha (Sec. 4.2 "Mapping")
CHANNEL_DUAL = 0    # Eq. (cannonical)
CHANNEL_SINGLE = 1  # Eq. (single): Z <- Z h[X], X = Z^T s Z
SCHED_BRANCHES = 0  # y and z products on two streams, launches per product
SCHED_STAGES = 1    # the batched engine with one problem (the y and z products share launches)
SCHED_AUTO = 2      # timed on the call's own input, cached

STATUS = {0: "SPAMM_OK", -1: "SPAMM_ERR_ARG", -2: "SPAMM_ERR_NOMEM", -3: "SPAMM_ERR_DIVERGED",
          -4: "SPAMM_ERR_NOTCONVERGED", -5: "SPAMM_ERR_TIMEOUT", -6: "SPAMM_ERR_ADMIT", -7: "SPAMM_ERR_CUDA",
          -8: "SPAMM_ERR_UNSUPPORTED", -9: "SPAMM_ERR_NOTFOUND"}

# every extern "C" function declared in include/spamm.h
HEADER_SYMBOLS = ["spamm_opts_init", "spamm_autotune_leaf", "spamm_multiply", "spamm_sqrt_invsqrt",
                  "spamm_invsqrt_product",
                  "spamm_sqrt_invsqrt_batched", "spamm_norm_tree", "spamm_cull", "spamm_last_error", "spamm_strerror",
                  "spamm_release",
                  "spamm_kernel_launches", "spamm_version", "spamm_multiply_noalloc", "spamm_test_expire_next_wait",
                  "spamm_test_emu_alternate",
                  "spamm_server_create",
                  "spamm_server_submit", "spamm_server_poll", "spamm_server_wait", "spamm_server_destroy"]


class SpammError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("precision", ctypes.c_int), ("tau_s", ctypes.c_double),
                ("mu_rel", ctypes.c_double), ("tol_t", ctypes.c_double), ("order", ctypes.c_int),
                ("residual", ctypes.c_int), ("profile", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("map", ctypes.c_int), ("channel", ctypes.c_int), ("schedule", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("t_final", ctypes.c_double), ("resid_F", ctypes.c_double),
                ("scale_c", ctypes.c_double), ("tasks_total", ctypes.c_longlong),
                ("tasks_dense", ctypes.c_longlong), ("flops", ctypes.c_double),
                ("t_hist", ctypes.POINTER(ctypes.c_double)), ("task_hist", ctypes.POINTER(ctypes.c_longlong)),
                ("gemm_ms", ctypes.c_double), ("gemm_launches", ctypes.c_longlong),
                ("lens_hist", ctypes.POINTER(ctypes.c_longlong)), ("lens_bins", ctypes.c_int),
                ("tensor_units", ctypes.c_longlong), ("cull_ms", ctypes.c_double),
                ("cull_launches", ctypes.c_longlong), ("tree_ms", ctypes.c_double),
                ("tree_launches", ctypes.c_longlong), ("slice_ms", ctypes.c_double),
                ("slice_launches", ctypes.c_longlong), ("schedule", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    return _build_lib.build(force=force)


def lib_path() -> str:
    return _build_lib.LIB


def lib(build_if_missing: bool = True):
    """Load libspamm.so (building it with nvcc first when it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build_lib.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"libspamm.so not built at {path}")
            _build_lib.build()
        L = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.spamm_opts_init.argtypes = [ctypes.POINTER(Opts)]
        L.spamm_opts_init.restype = None
        L.spamm_autotune_leaf.argtypes = [vp, ip, ctypes.c_double, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_int)]
        L.spamm_autotune_leaf.restype = ip
        L.spamm_multiply.argtypes = [vp, vp, vp, ip, ctypes.c_double, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]
        L.spamm_invsqrt_product.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                            ctypes.c_double, ip, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Opts)]
        L.spamm_invsqrt_product.restype = ip
        L.spamm_multiply.restype = ip
        L.spamm_sqrt_invsqrt.argtypes = [vp, ip, ctypes.c_double, ip, vp, vp, ctypes.POINTER(Opts),
                                         ctypes.POINTER(Stats)]
        L.spamm_sqrt_invsqrt.restype = ip
        L.spamm_sqrt_invsqrt_batched.argtypes = [ip, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(ctypes.c_double), ip, ctypes.POINTER(vp),
                                                 ctypes.POINTER(vp), ctypes.POINTER(Opts), ctypes.POINTER(Stats)]
        L.spamm_sqrt_invsqrt_batched.restype = ip
        L.spamm_norm_tree.argtypes = [vp, ip, ip, vp, dp, vp]
        L.spamm_norm_tree.restype = ip
        L.spamm_cull.argtypes = [vp, vp, ip, ctypes.c_double, ip, vp, vp, dp, ctypes.POINTER(ctypes.c_longlong), vp]
        L.spamm_cull.restype = ip
        L.spamm_last_error.argtypes = []
        L.spamm_last_error.restype = ctypes.c_char_p
        L.spamm_strerror.argtypes = [ip]
        L.spamm_strerror.restype = ctypes.c_char_p
        L.spamm_release.argtypes = []
        L.spamm_release.restype = ip
        L.spamm_multiply_noalloc.argtypes = [vp, vp, vp, ip, ctypes.c_double, ip, vp]
        L.spamm_multiply_noalloc.restype = ip
        L.spamm_server_create.argtypes = [ctypes.c_size_t, ip, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
        L.spamm_server_create.restype = ip
        L.spamm_server_submit.argtypes = [vp, vp, ip, ctypes.c_double, ip, vp, vp, ctypes.POINTER(ctypes.c_longlong)]
        L.spamm_server_submit.restype = ip
        L.spamm_server_poll.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
        L.spamm_server_poll.restype = ip
        L.spamm_server_wait.argtypes = [vp, ctypes.c_longlong, ctypes.c_double, ctypes.POINTER(Stats),
                                        ctypes.POINTER(ctypes.c_double)]
        L.spamm_server_wait.restype = ip
        L.spamm_server_destroy.argtypes = [vp]
        L.spamm_server_destroy.restype = ip
        L.spamm_test_expire_next_wait.argtypes = [ctypes.c_longlong]
        L.spamm_test_expire_next_wait.restype = ip
        L.spamm_test_emu_alternate.argtypes = [ip]
        L.spamm_test_emu_alternate.restype = ip
        L.spamm_kernel_launches.argtypes = []
        L.spamm_kernel_launches.restype = ctypes.c_longlong
        L.spamm_version.argtypes = []
        L.spamm_version.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(status: int, allow=()) -> int:
    if status != 0 and status not in allow:
        raise SpammError(status, lib().spamm_last_error().decode())
    return status


# ---------------------------------------------------------------------------- marshalling helpers


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _prep(x, n=None):
    """Return (object kept alive, raw pointer, n, is_cuda)."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float64:
            raise TypeError("float64 tensors expected")
        x = x.contiguous()
        if x.dim() != 2 or x.shape[0] != x.shape[1]:
            raise ValueError("square matrix expected")
        return x, x.data_ptr(), x.shape[0], x.is_cuda
    a = np.ascontiguousarray(x, dtype=np.float64)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square matrix expected")
    return a, a.ctypes.data, a.shape[0], False


def _like(ref, n):
    if _is_torch(ref):
        import torch
        return torch.empty((n, n), dtype=torch.float64, device=ref.device)
    return np.empty((n, n), dtype=np.float64)


def _ptr(x) -> int:
    return x.data_ptr() if _is_torch(x) else x.ctypes.data


def _stream_of(ref, stream):
    if stream is not None:
        return int(stream) if not hasattr(stream, "cuda_stream") else int(stream.cuda_stream)
    if _is_torch(ref) and ref.is_cuda:
        import torch
        return int(torch.cuda.current_stream(ref.device).cuda_stream)
    return None


def _opts(leaf=64, precision=FP64, tau_s=None, mu_rel=0.0, tol_t=0.0, order=ORDER_PAPER, residual=False,
          stream=None, profile=False, map=MAP_NS, channel=CHANNEL_DUAL, schedule=SCHED_BRANCHES) -> Opts:
    o = Opts()
    lib().spamm_opts_init(ctypes.byref(o))
    o.leaf = int(leaf)
    o.precision = int(precision)
    o.tau_s = -1.0 if tau_s is None else float(tau_s)
    o.mu_rel = float(mu_rel)
    o.tol_t = float(tol_t)
    o.order = int(order)
    o.residual = 1 if residual else 0
    o.profile = 1 if profile else 0
    o.stream = stream
    o.map = int(map)
    o.channel = int(channel)
    o.schedule = int(schedule)
    return o


def _stats_dict(s: Stats, th=None, kh=None) -> dict:
    d = {"iters": s.iters, "t_final": s.t_final, "resid_F": s.resid_F, "scale_c": s.scale_c,
         "tasks_total": s.tasks_total, "tasks_dense": s.tasks_dense, "flops": s.flops, "gemm_ms": s.gemm_ms,
         "gemm_launches": s.gemm_launches, "tensor_units": s.tensor_units, "cull_ms": s.cull_ms,
         "cull_launches": s.cull_launches, "tree_ms": s.tree_ms, "tree_launches": s.tree_launches,
         "slice_ms": s.slice_ms, "slice_launches": s.slice_launches, "schedule": s.schedule}
    if th is not None:
        d["t_hist"] = th[:s.iters].copy()
    if kh is not None:
        d["task_hist"] = kh[:s.iters].copy()
    return d


# ---------------------------------------------------------------------------- public calls


def multiply(A, B, tau: float, leaf: int = 64, precision: int = FP64, out=None, stream=None, profile=False):
    """C = A (x)_tau B (Eq. (newspamm)); returns (C, stats).  profile: time the leaf-product kernel with CUDA
    events (stats["gemm_ms"])."""
    a, pa, n, _ = _prep(A)
    b, pb, nb_, _ = _prep(B)
    if nb_ != n:
        raise ValueError("A and B differ in size")
    C = out if out is not None else _like(a, n)
    st = Stats()
    o = _opts(leaf=leaf, precision=precision, stream=_stream_of(a, stream), profile=profile)
    _check(lib().spamm_multiply(pa, pb, _ptr(C), n, float(tau), ctypes.byref(o), ctypes.byref(st)))
    return C, _stats_dict(st)


def invsqrt_product(S, mus, tau0: float, tau1: float, maxit: int, leaf: int = 64, precision: int = FP64,
                    tau_s=None, tol_t=0.0, map=None, channel=None, Z=None, stream=None, raise_on=True):
    """Product representation of the regularised inverse factor (Sec. 6, spamm_invsqrt_product): slice
    z_0 = (S + mus[0] c0 I)^{-1/2} at tau0, then per level the residual Z^T (S + mus[l] c0 I) Z at tau1, its
    inverse square root z_l at tau0 and Z <- Z (x)_tau1 z_l.  Returns (Z, {"iters": [...], "status": s}),
    with Z^T (S + mus[-1] c0 I) Z ~ I."""
    s, ps, n, _ = _prep(S)
    Z = Z if Z is not None else _like(s, n)
    mu = (ctypes.c_double * len(mus))(*[float(x) for x in mus])
    its = (ctypes.c_int * len(mus))()
    o = _opts(leaf, precision, tau_s, 0.0, tol_t, ORDER_PAPER, False, _stream_of(s, stream), False,
              MAP_NS if map is None else map, CHANNEL_DUAL if channel is None else channel)
    status = lib().spamm_invsqrt_product(ps, n, len(mus), mu, float(tau0), float(tau1), int(maxit), _ptr(Z), its,
                                         ctypes.byref(o))
    if raise_on:
        _check(status)
    return Z, {"iters": list(its), "status": status}


def autotune_leaf(S, tau: float, precision: int = FP64, stream=None) -> int:
    """Fastest leaf size for problems like S (spamm_autotune_leaf); cached per device, n, arithmetic and
    decade of tau.  Calls given leaf=0 use the same choice."""
    s, ps, n, _ = _prep(S)
    o = _opts(leaf=0, precision=precision, stream=_stream_of(s, stream))
    leaf = ctypes.c_int(0)
    _check(lib().spamm_autotune_leaf(ps, n, float(tau), ctypes.byref(o), ctypes.byref(leaf)))
    return leaf.value


def sqrt_invsqrt(S, tau: float, maxit: int, leaf: int = 64, precision: int = FP64, tau_s=None, mu_rel=0.0,
                 tol_t=0.0, order=ORDER_PAPER, residual=False, Y=None, Z=None, stream=None, raise_on=True,
                 profile=False, map=None, channel=None, lens_bins=0, schedule=SCHED_BRANCHES):
    """Y ~ S^{1/2}, Z ~ S^{-1/2} by dual-channel Newton-Schulz on SpAMM products; returns (Y, Z, stats).
    With lens_bins > 0, stats["lens_hist"] holds the plane-diagonal profile of every product's surviving tile
    triples, [iters, 3 products, 3 planes (|i-j|, |j-k|, |i-k|), lens_bins]."""
    s, ps, n, _ = _prep(S)
    Y = Y if Y is not None else _like(s, n)
    Z = Z if Z is not None else _like(s, n)
    th = np.zeros(max(1, maxit))
    kh = np.zeros((max(1, maxit), 3), dtype=np.int64)
    st = Stats()
    st.t_hist = th.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st.task_hist = kh.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    lh = None
    if lens_bins > 0:
        lh = np.zeros((max(1, maxit), 3, 3, int(lens_bins)), dtype=np.int64)
        st.lens_hist = lh.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
        st.lens_bins = int(lens_bins)
    o = _opts(leaf, precision, tau_s, mu_rel, tol_t, order, residual, _stream_of(s, stream), profile,
              MAP_NS if map is None else map, CHANNEL_DUAL if channel is None else channel, schedule)
    status = lib().spamm_sqrt_invsqrt(ps, n, float(tau), int(maxit), _ptr(Y), _ptr(Z), ctypes.byref(o),
                                      ctypes.byref(st))
    d = _stats_dict(st, th, kh)
    if lh is not None:
        d["lens_hist"] = lh[:st.iters].copy()
    d["status"] = status
    if raise_on:
        _check(status)
    return Y, Z, d


def sqrt_invsqrt_batched(Ss, taus, maxit: int, leaf: int = 64, precision: int = FP64, tau_s=None, mu_rel=0.0,
                         tol_t=0.0, order=ORDER_PAPER, residual=False, stream=None, map=None, channel=None,
                         raise_on=True, Ys=None, Zs=None):
    """Many independent solves in one call; returns (list of Y, list of Z, list of stats).  With raise_on
    False a failed status (the first nonzero one) is returned in every stats dict as "call_status".  Ys, Zs:
    optional output matrices (the library reuses its captured batch while the inputs, outputs and options
    stay the same)."""
    cnt = len(Ss)
    keep = [_prep(S) for S in Ss]
    Ys = list(Ys) if Ys is not None else [_like(k[0], k[2]) for k in keep]
    Zs = list(Zs) if Zs is not None else [_like(k[0], k[2]) for k in keep]
    VP = ctypes.c_void_p * cnt
    sp = VP(*[k[1] for k in keep])
    yp = VP(*[_ptr(y) for y in Ys])
    zp = VP(*[_ptr(z) for z in Zs])
    ns = (ctypes.c_int * cnt)(*[k[2] for k in keep])
    ts = (ctypes.c_double * cnt)(*[float(t) for t in taus])
    stats = (Stats * cnt)()
    o = _opts(leaf, precision, tau_s, mu_rel, tol_t, order, residual, _stream_of(keep[0][0], stream) if cnt else None,
              map=MAP_NS if map is None else map, channel=CHANNEL_DUAL if channel is None else channel)
    status = lib().spamm_sqrt_invsqrt_batched(cnt, sp, ns, ts, int(maxit), yp, zp, ctypes.byref(o), stats)
    if raise_on:
        _check(status)
    out = [_stats_dict(stats[q]) for q in range(cnt)]
    for d in out:
        d["call_status"] = status
    return Ys, Zs, out


def norm_tree(A, leaf: int = 64, stream=None):
    """Leaf squared norms (m x m numpy array) and the root squared norm, computed on the GPU."""
    a, pa, n, _ = _prep(A)
    m = (n + leaf - 1) // leaf
    nu = np.zeros((m, m))
    root = ctypes.c_double(0.0)
    _check(lib().spamm_norm_tree(pa, n, int(leaf), nu.ctypes.data, ctypes.byref(root), _stream_of(a, stream)))
    return nu, root.value


def cull(A, B, tau: float, leaf: int = 64, stream=None):
    """GPU task list: sorted (i, j, k) triples (ordered by i, k, then j), the squared threshold and the count."""
    a, pa, n, _ = _prep(A)
    b, pb, _, _ = _prep(B)
    m = (n + leaf - 1) // leaf
    counts = np.zeros(m * m, dtype=np.int32)
    jl = np.zeros(m * m * m, dtype=np.int32)
    thr = ctypes.c_double(0.0)
    tot = ctypes.c_longlong(0)
    _check(lib().spamm_cull(pa, pb, n, float(tau), int(leaf), counts.ctypes.data, jl.ctypes.data,
                            ctypes.byref(thr), ctypes.byref(tot), _stream_of(a, stream)))
    jl = jl.reshape(m * m, m)
    rows = []
    for q in np.nonzero(counts)[0]:
        i, k = divmod(int(q), m)
        for j in jl[q, :counts[q]]:
            rows.append((i, int(j), k))
    tasks = np.array(rows, dtype=np.int32).reshape(-1, 3)
    return tasks, thr.value, tot.value


class Server:
    """Request loop over sqrt_invsqrt: submit() queues a solve, wait() returns (Y, Z, stats, latency_s).

    Requests are admitted in arrival order when a worker is free and their device footprint fits in the
    memory budget; admitted requests run concurrently on separate CUDA streams."""

    def __init__(self, bytes_budget: int, max_active: int = 4, leaf: int = 64, precision: int = FP64, tau_s=None,
                 mu_rel=0.0, tol_t=0.0, order=ORDER_PAPER, map=None, channel=None):
        self._h = ctypes.c_void_p(0)
        o = _opts(leaf, precision, tau_s, mu_rel, tol_t, order, False, None, map=MAP_NS if map is None else map,
                  channel=CHANNEL_DUAL if channel is None else channel)
        _check(lib().spamm_server_create(int(bytes_budget), int(max_active), ctypes.byref(o), ctypes.byref(self._h)))
        self._keep = {}

    def submit(self, S, tau: float, maxit: int):
        s, ps, n, _ = _prep(S)
        Y, Z = _like(s, n), _like(s, n)
        rid = ctypes.c_longlong(0)
        _check(lib().spamm_server_submit(self._h, ps, n, float(tau), int(maxit), _ptr(Y), _ptr(Z), ctypes.byref(rid)))
        self._keep[rid.value] = (s, Y, Z)
        return rid.value

    def poll(self, rid: int) -> int:
        st = ctypes.c_int(0)
        _check(lib().spamm_server_poll(self._h, int(rid), ctypes.byref(st)))
        return st.value

    def wait(self, rid: int, timeout: float = -1.0, raise_on=True):
        stats = Stats()
        lat = ctypes.c_double(0.0)
        status = lib().spamm_server_wait(self._h, int(rid), float(timeout), ctypes.byref(stats), ctypes.byref(lat))
        if status == -5 and timeout >= 0:
            raise TimeoutError(f"request {rid} still pending")
        s, Y, Z = self._keep.pop(rid, (None, None, None))
        d = _stats_dict(stats)
        d["status"] = status
        if raise_on:
            _check(status)
        return Y, Z, d, lat.value

    def close(self):
        if self._h:
            _check(lib().spamm_server_destroy(self._h))
            self._h = ctypes.c_void_p(0)
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def kernel_launches() -> int:
    """Kernels launched by libspamm since load (all threads)."""
    return int(lib().spamm_kernel_launches())


def release():
    _check(lib().spamm_release())


def version() -> str:
    return lib().spamm_version().decode()

"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no SpAMM or Newton-Schulz arithmetic: it only draws the
workload matrices (and request traces) that both sides receive unchanged.

The paper's own data (TubeGen nanotube overlaps, gromacs water boxes,
bcsstk14; Sec. 4.3) are not available here.  Stand-ins, with the decay and
metric locality the method relies on:

* ``kms(n, rho)``: the Kac-Murdock-Szego matrix S_ij = rho^|i-j|, a quasi-1D
  exponential decay whose inverse is tridiagonal in closed form.
* ``gaussian_lattice(n, sigma, seed)``: S_ij = exp(-|r_i - r_j|^2 / (2 sigma^2))
  for n points on a jittered 3D cubic lattice (spacing 1, jitter U(-0.1, 0.1)),
  i.e. the overlap matrix of normalised s-type Gaussians, a 3D Gramian like the
  water-box overlaps.  Lattice sites are ordered along a 3D Morton
  (Z-order) space-filling curve, the locality-preserving ordering the paper
  uses for its bases (Sec. 1, block-by-magnitude structure).
"""
from __future__ import annotations

import math

import numpy as np


def kms(n: int, rho: float) -> np.ndarray:
    """Kac-Murdock-Szego matrix rho^|i-j| (n x n, float64)."""
    i = np.arange(n)
    return np.power(float(rho), np.abs(i[:, None] - i[None, :]).astype(np.float64))


def kms_inverse(n: int, rho: float) -> np.ndarray:
    """Closed-form tridiagonal inverse of the KMS matrix:
    (1/(1-rho^2)) * tridiag(-rho, [1, 1+rho^2, ..., 1+rho^2, 1], -rho)."""
    r = float(rho)
    T = np.zeros((n, n))
    d = np.full(n, 1.0 + r * r)
    d[0] = d[-1] = 1.0
    if n == 1:
        d[0] = 1.0 - r * r
    T[np.arange(n), np.arange(n)] = d
    T[np.arange(n - 1), np.arange(1, n)] = -r
    T[np.arange(1, n), np.arange(n - 1)] = -r
    return T / (1.0 - r * r)


def _part1by2(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def morton3(ix: np.ndarray, iy: np.ndarray, iz: np.ndarray) -> np.ndarray:
    """3D Morton key with x in the lowest interleaved bit."""
    return _part1by2(ix) | (_part1by2(iy) << np.uint64(1)) | (_part1by2(iz) << np.uint64(2))


def lattice_points(n: int, seed: int = 0, jitter: float = 0.1) -> np.ndarray:
    """First n sites of a ceil(n^(1/3))^3 integer lattice in Morton order, jittered U(-jitter, jitter)."""
    side = 1
    while side ** 3 < n:
        side += 1
    g = np.arange(side)
    ix, iy, iz = np.meshgrid(g, g, g, indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    order = np.argsort(morton3(ix, iy, iz), kind="stable")[:n]
    pts = np.stack([ix[order], iy[order], iz[order]], axis=1).astype(np.float64)
    rng = np.random.default_rng(seed)
    pts += rng.uniform(-jitter, jitter, size=pts.shape)
    return pts


def gaussian_lattice(n: int, sigma: float = 0.6, seed: int = 0, jitter: float = 0.1) -> np.ndarray:
    """3D Gaussian-decay Gramian exp(-|r_i - r_j|^2 / (2 sigma^2)) on jittered Morton-ordered lattice points."""
    r = lattice_points(n, seed, jitter)
    d2 = ((r[:, None, :] - r[None, :, :]) ** 2).sum(-1)
    return np.exp(-d2 / (2.0 * sigma * sigma))


def integer_matrix(n: int, seed: int = 0, lo: int = -2, hi: int = 2) -> np.ndarray:
    """Integer-valued float64 matrix with entries uniform in {lo..hi}: every FP sum of products is exact."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n, n)).astype(np.float64)


def decay_matrix(n: int, seed: int = 0, length: float = 8.0) -> np.ndarray:
    """Random matrix with exponential off-diagonal decay exp(-|i-j|/length) times U(-1,1) entries (non-symmetric)."""
    rng = np.random.default_rng(seed)
    i = np.arange(n)
    env = np.exp(-np.abs(i[:, None] - i[None, :]) / float(length))
    return env * rng.uniform(-1.0, 1.0, size=(n, n))


def round_up(x: int, q: int) -> int:
    return ((int(x) + q - 1) // q) * q


def log_uniform_sizes(count: int, lo: int, hi: int, multiple: int, rng: np.random.Generator) -> np.ndarray:
    """Sizes drawn log-uniform in [lo, hi], rounded to a multiple and clipped into [lo, hi]."""
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    s = np.array([round_up(int(round(math.exp(v))), multiple) for v in u])
    return np.clip(s, lo, hi)


def batch_mix(count: int = 512, lo: int = 128, hi: int = 2048, seed: int = 0) -> list[dict]:
    """Mixed batch of SPD decay matrices: 50% 1D KMS with rho ~ U(0.5, 0.95), 50% 3D Gaussian with
    sigma ~ U(0.6, 0.9); sizes log-uniform in [lo, hi], multiples of 32.  Matrices are built lazily."""
    rng = np.random.default_rng(seed)
    sizes = log_uniform_sizes(count, lo, hi, 32, rng)
    out = []
    for q in range(count):
        if rng.uniform() < 0.5:
            out.append({"kind": "kms", "n": int(sizes[q]), "rho": float(rng.uniform(0.5, 0.95))})
        else:
            out.append({"kind": "gauss", "n": int(sizes[q]), "sigma": float(rng.uniform(0.6, 0.9)),
                        "seed": int(rng.integers(0, 2 ** 31 - 1))})
    return out


def make(spec: dict) -> np.ndarray:
    """Materialise a matrix from a batch_mix / serving_trace spec."""
    if spec["kind"] == "kms":
        return kms(spec["n"], spec["rho"])
    return gaussian_lattice(spec["n"], spec["sigma"], spec.get("seed", 0))


def serving_trace(count: int = 2000, rate: float = 200.0, lo: int = 256, hi: int = 8192, seed: int = 0,
                  taus=(1e-4, 1e-6, 1e-8)) -> list[dict]:
    """Poisson arrivals (seeded exponential gaps) of square-root requests on 3D Gaussian-decay matrices;
    sizes log-uniform in [lo, hi] rounded to 32, tau drawn uniformly from taus."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    sizes = log_uniform_sizes(count, lo, hi, 32, rng)
    out = []
    for q in range(count):
        out.append({"kind": "gauss", "n": int(sizes[q]), "sigma": float(rng.uniform(0.6, 0.9)),
                    "seed": int(rng.integers(0, 2 ** 31 - 1)), "tau": float(taus[int(rng.integers(len(taus)))]),
                    "arrival": float(t[q])})
    return out

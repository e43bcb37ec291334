"""The synthetic inputs match their stated recipes (CPU only).

Both the oracle and the CUDA path receive these matrices unchanged, so a drift in a recipe would change every
parity case and every benchmark workload at once without failing a parity test.
"""
import math

import numpy as np
import pytest

import synth


def test_kms_entries_and_symmetry():
    S = synth.kms(7, 0.9)
    i = np.arange(7)
    assert np.array_equal(S, 0.9 ** np.abs(i[:, None] - i[None, :]))
    assert np.array_equal(S, S.T) and (np.diag(S) == 1.0).all()


def test_morton_key_interleaves_x_lowest():
    key = lambda x, y, z: int(synth.morton3(np.array([x]), np.array([y]), np.array([z]))[0])
    assert [key(1, 0, 0), key(0, 1, 0), key(0, 0, 1), key(1, 1, 1), key(2, 0, 0), key(0, 0, 2)] == [1, 2, 4, 7, 8, 32]
    assert key(3, 5, 6) == 0b110101011  # bits (z y x) per level, lowest level first: 011, 101, 110


@pytest.mark.parametrize("n", [1, 8, 27, 30, 256])
def test_lattice_points_are_the_first_morton_sites_jittered(n):
    side = 1
    while side ** 3 < n:
        side += 1
    p = synth.lattice_points(n, seed=3)
    assert p.shape == (n, 3)
    sites = np.rint(p).astype(np.int64)
    assert np.abs(p - sites).max() <= 0.1
    assert sites.min() >= 0 and sites.max() < side
    keys = synth.morton3(sites[:, 0], sites[:, 1], sites[:, 2])
    # the n smallest keys of the side^3 cube, in increasing order, each site once
    assert (np.diff(keys.astype(np.int64)) > 0).all()
    g = np.arange(side)
    all_keys = np.sort(synth.morton3(*[a.ravel() for a in np.meshgrid(g, g, g, indexing="ij")]))
    assert np.array_equal(keys, all_keys[:n])
    assert np.array_equal(p, synth.lattice_points(n, seed=3))  # seeded
    assert not np.array_equal(p, synth.lattice_points(n, seed=4)) or n == 0


def test_gaussian_lattice_is_the_gaussian_gramian_of_the_points():
    n, sigma = 40, 0.7
    S = synth.gaussian_lattice(n, sigma, seed=2)
    r = synth.lattice_points(n, seed=2)
    i, j = 5, 31
    assert S[i, j] == pytest.approx(math.exp(-((r[i] - r[j]) ** 2).sum() / (2 * sigma * sigma)), rel=1e-15)
    assert np.array_equal(S, S.T) and (np.diag(S) == 1.0).all()
    assert np.linalg.eigvalsh(S).min() > 0.0


def test_batch_mix_recipe():
    specs = synth.batch_mix(512, seed=0)
    assert len(specs) == 512
    sizes = np.array([s["n"] for s in specs])
    assert (sizes % 32 == 0).all() and sizes.min() >= 128 and sizes.max() <= 2048
    kinds = [s["kind"] for s in specs]
    assert 0.4 < kinds.count("kms") / 512 < 0.6
    assert all(0.5 <= s["rho"] <= 0.95 for s in specs if s["kind"] == "kms")
    assert all(0.6 <= s["sigma"] <= 0.9 for s in specs if s["kind"] == "gauss")
    # log-uniform: the median size sits near the geometric mean of the range, not the arithmetic one
    assert abs(math.log(np.median(sizes)) - 0.5 * math.log(128 * 2048)) < 0.25
    assert synth.batch_mix(512, seed=0) == specs


def test_serving_trace_recipe():
    tr = synth.serving_trace(2000, rate=200.0, seed=0)
    arr = np.array([r["arrival"] for r in tr])
    assert (np.diff(arr) > 0).all()
    # Poisson arrivals at 200/s: exponential gaps with mean 5 ms
    assert np.mean(np.diff(arr)) == pytest.approx(1 / 200.0, rel=0.08)
    sizes = np.array([r["n"] for r in tr])
    assert (sizes % 32 == 0).all() and sizes.min() >= 256 and sizes.max() <= 8192
    assert {r["tau"] for r in tr} == {1e-4, 1e-6, 1e-8}
    assert all(r["kind"] == "gauss" for r in tr)

"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

Tolerances (FP64 path):
  * leaf norms: relative 1e-13 (sums of nb^2 squares in a different order,
    with fused multiply-adds: bound nb^2 u, observed ~1e-15);
  * task lists: identical except triples within the band
    |nu_a nu_b / thr - 1| <= 2e-6 (the norms feeding the test differ in the
    last bits because the summation orders differ);
  * one product with identical task lists: |C - C_oracle| <= 4 K u (|A||B|)
    elementwise, K = inner length, u = 2^-53 (same summation order, fused vs
    separate multiply-add);
  * Newton-Schulz: ||Z - Z_oracle||_F / ||Z_oracle||_F <= 1e-10 (and Y alike).
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_1508_05856_gb300")

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else t


def _band_ok(A, B, nb, tau, gpu_tasks, or_tasks, thr):
    la, lb = oracle.leaf_norms(A, nb), oracle.leaf_norms(B, nb)
    g = set(map(tuple, gpu_tasks.tolist()))
    o = set(map(tuple, or_tasks.tolist()))
    diff = g ^ o
    for (i, j, k) in diff:
        r = la[i, j] * lb[j, k] / thr if thr > 0 else math.inf
        assert abs(r - 1.0) <= 2e-6, f"task {(i, j, k)} differs outside the tolerance band (ratio {r})"
    return len(diff)


# ------------------------------------------------------------------------------------------ norm tree


@pytest.mark.parametrize("n,nb", [(256, 32), (200, 64), (1000, 128), (64, 64), (4096, 64)])
def test_norm_tree(n, nb):
    A = synth.decay_matrix(n, seed=n + nb)
    nu, root = sp.norm_tree(dev(A), nb)
    ref = oracle.leaf_norms(A, nb)
    np.testing.assert_allclose(nu, ref, rtol=1e-13, atol=0)
    tree = oracle.norm_tree(A, nb)
    assert root == pytest.approx(tree[0][0, 0], rel=1e-13)


# ------------------------------------------------------------------------------------------ cull


@pytest.mark.parametrize("n,nb,tau", [(256, 32, 1e-3), (500, 32, 1e-4), (1024, 64, 1e-5), (640, 128, 1e-6),
                                      (200, 64, 0.0), (4096, 64, 1e-8)])
def test_cull_lists(n, nb, tau):
    A = synth.decay_matrix(n, seed=1, length=n / 20)
    B = synth.decay_matrix(n, seed=2, length=n / 15)
    gt, thr, tot = sp.cull(dev(A), dev(B), tau, nb)
    ot, othr = oracle.cull(A, B, nb, tau)
    assert thr == pytest.approx(othr, rel=1e-12, abs=0)
    assert tot == gt.shape[0]
    nd = _band_ok(A, B, nb, tau, gt, ot, othr)
    assert nd == 0 or nd < 3
    if nd == 0:
        np.testing.assert_array_equal(gt, ot)       # same canonical (i, k, j) order


# ------------------------------------------------------------------------------------------ products


@pytest.mark.parametrize("n,nb", [(64, 32), (100, 32), (256, 64), (300, 64), (384, 128), (129, 128)])
def test_tau_zero_integer_bitwise(n, nb):
    A = synth.integer_matrix(n, seed=3)
    B = synth.integer_matrix(n, seed=4)
    C, st = sp.multiply(dev(A), dev(B), 0.0, leaf=nb)
    Co, cnt = oracle.spamm(A, B, nb, 0.0)
    np.testing.assert_array_equal(host(C), Co)
    assert st["tasks_total"] == cnt


@pytest.mark.parametrize("n,nb,tau", [(256, 32, 1e-3), (333, 32, 1e-4), (512, 64, 1e-6), (768, 128, 1e-7),
                                      (1000, 64, 0.0)])
def test_multiply_matches_oracle(n, nb, tau):
    A = synth.decay_matrix(n, seed=5, length=n / 16)
    B = synth.decay_matrix(n, seed=6, length=n / 10)
    C, st = sp.multiply(dev(A), dev(B), tau, leaf=nb)
    C = host(C)
    ot, thr = oracle.cull(A, B, nb, tau)
    gt, _, _ = sp.cull(dev(A), dev(B), tau, nb)
    _band_ok(A, B, nb, tau, gt, ot, thr)
    Co = oracle.leaf_products(A, B, nb, gt)           # oracle arithmetic on the GPU's (valid) list
    K = (max(1, int(np.bincount(gt[:, 0] * 10000 + gt[:, 2]).max())) if len(gt) else 1) * nb
    bound = 4 * K * U * (np.abs(A) @ np.abs(B)) + 1e-300
    assert (np.abs(C - Co) <= bound).all()
    assert st["tasks_total"] == len(gt)


def test_host_and_device_pointers_agree():
    n, nb, tau = 300, 32, 1e-5
    A = synth.decay_matrix(n, seed=8)
    B = synth.decay_matrix(n, seed=9)
    Ch, _ = sp.multiply(A, B, tau, leaf=nb)                # numpy in, numpy out (host staging)
    Cd, _ = sp.multiply(dev(A), dev(B), tau, leaf=nb)
    np.testing.assert_array_equal(Ch, host(Cd))


# ------------------------------------------------------------------------------------------ Newton-Schulz


def _ns_compare(S, nb, tau, maxit, **kw):
    Y, Z, st = sp.sqrt_invsqrt(dev(S), tau, maxit, leaf=nb, **kw)
    Y, Z = host(Y), host(Z)
    kw2 = {k: v for k, v in kw.items() if k in ("tau_s", "mu_rel", "order", "tol_t", "map", "channel")}
    ref = oracle.sqrt_invsqrt(S, nb, tau, maxit, **kw2)
    assert st["iters"] == ref["iters"]
    ez = np.linalg.norm(Z - ref["Z"]) / np.linalg.norm(ref["Z"])
    ey = np.linalg.norm(Y - ref["Y"]) / np.linalg.norm(ref["Y"])
    assert ez <= 1e-10, ez
    assert ey <= 1e-10, ey
    assert st["scale_c"] == pytest.approx(ref["scale_c"], rel=1e-14)
    np.testing.assert_allclose(st["t_hist"], ref["t_hist"], rtol=0, atol=1e-12)
    return Y, Z, st, ref


def test_ns_gaussian_256_leaf32():
    """Gaussian decay, 256 jittered lattice points (sigma 0.6, seed 0), N_b 32, tau 1e-6, 30 iterations."""
    S = synth.gaussian_lattice(256, 0.6, seed=0)
    Y, Z, st, ref = _ns_compare(S, 32, 1e-6, 30)
    np.testing.assert_array_equal(st["task_hist"], ref["task_hist"])


@pytest.mark.parametrize("n,nb,tau,order", [(200, 32, 1e-5, 0), (200, 64, 1e-7, 1), (333, 128, 1e-6, 0),
                                            (96, 32, 0.0, 1), (600, 64, 1e-9, 0)])
def test_ns_ragged_and_orders(n, nb, tau, order):
    S = synth.gaussian_lattice(n, 0.7, seed=n)
    _ns_compare(S, nb, tau, 25, order=order)


def test_ns_kms_regularised_and_tol():
    S = synth.kms(320, 0.9)
    _ns_compare(S, 64, 1e-8, 30, mu_rel=1e-3)
    Y, Z, st, ref = _ns_compare(S, 32, 1e-10, 40, tol_t=1e-13)
    assert st["iters"] < 40


def test_ns_diagonal_bitwise():
    d = np.linspace(0.01, 2.0, 150)
    S = np.diag(d)
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 0.0, 12, leaf=32)
    ref = oracle.sqrt_invsqrt(S, 32, 0.0, 12)
    np.testing.assert_array_equal(host(Y), ref["Y"])
    np.testing.assert_array_equal(host(Z), ref["Z"])


def test_residual_matches_oracle():
    S = synth.kms(256, 0.8)
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 1e-9, 25, leaf=32, residual=True)
    r = oracle.residual(S, host(Z))
    assert st["resid_F"] == pytest.approx(r, rel=1e-6, abs=1e-14)


def test_batched_equals_single_bitwise():
    specs = synth.batch_mix(6, lo=128, hi=512, seed=3)
    Ss = [synth.make(s) for s in specs]
    taus = [1e-6] * len(Ss)
    Ys, Zs, sts = sp.sqrt_invsqrt_batched([dev(S) for S in Ss], taus, 20, leaf=32)
    for S, Yb, Zb in zip(Ss, Ys, Zs):
        Y1, Z1, _ = sp.sqrt_invsqrt(dev(S), 1e-6, 20, leaf=32)
        assert torch.equal(Yb, Y1) and torch.equal(Zb, Z1)


def test_divergence_reported():
    """An indefinite S has no real square root: the trace error leaves [0,1) and the call says so."""
    S = synth.kms(128, 0.5)
    S[0, 0] = -3.0
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 0.0, 30, leaf=32, raise_on=False)
    assert st["status"] == -3


@pytest.mark.slow
def test_ns_kms_4096_full_size():
    """KMS rho 0.9, N 4096, N_b 64 (the benchmark workload's geometry) at tau 1e-8: full iteration vs oracle."""
    S = synth.kms(4096, 0.9)
    _ns_compare(S, 64, 1e-8, 30)


def test_ns_kms_4096_benchmark_tau():
    """The benchmark's configuration on the FP64 path (KMS rho 0.9, N 4096, N_b 64, tau 1e-14, 30
    iterations): Y and Z within 1e-10 of the oracle, every per-iteration task count equal."""
    S = synth.kms(4096, 0.9)
    Y, Z, st, ref = _ns_compare(S, 64, 1e-14, 30)
    np.testing.assert_array_equal(st["task_hist"], ref["task_hist"])


def test_residual_at_least_one_is_reported_as_divergence():
    """At tau 1e-4 culling carries Y and Z off the roots while X = YZ still looks converged: the residual
    ||ZSZ - I||_F exceeds 1 and the call reports SPAMM_ERR_DIVERGED (outputs written).  The oracle's solve
    shows the same residual, so this is the method at that threshold, not the GPU."""
    S = synth.kms(1024, 0.9)
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 1e-4, 30, leaf=64, residual=True, raise_on=False)
    ref = oracle.sqrt_invsqrt(S, 64, 1e-4, 30)
    r_or = oracle.residual(S, ref["Z"])
    assert r_or >= 1.0 and abs(ref["t_hist"][-1]) < 1e-12
    assert st["status"] == -3
    assert st["resid_F"] == pytest.approx(r_or, rel=1e-6)
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 1e-12, 30, leaf=64, residual=True, raise_on=False)
    assert st["status"] == 0 and st["resid_F"] < 1.0


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs a second GPU to hold memory the current device cannot reach")
def test_device_memory_of_another_gpu_is_an_argument_error():
    """Only pointer attributes are read: no kernel sees the other GPU's memory."""
    other = torch.zeros((64, 64), dtype=torch.float64, device="cuda:1")
    here = torch.zeros((64, 64), dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(0):
        with pytest.raises(sp.SpammError) as ei:
            sp.multiply(other, here, 0.0, leaf=32, out=here.clone())
        assert ei.value.status == -1
        assert sp.lib().spamm_multiply_noalloc(other.data_ptr(), here.data_ptr(), here.data_ptr(), 64, 0.0, 32,
                                               None) == -1


def test_graph_replay_identical_and_profiled():
    """Repeated fixed-iteration solves replay a captured CUDA graph: identical results, kernel timings recorded,
    and no CUDA error left behind for the caller."""
    S = dev(synth.kms(512, 0.9))
    outs = [sp.sqrt_invsqrt(S, 1e-10, 12, leaf=64, profile=True) for _ in range(3)]
    for Y, Z, st in outs[1:]:
        assert torch.equal(Y, outs[0][0]) and torch.equal(Z, outs[0][1])
        assert st["gemm_ms"] > 0 and st["gemm_launches"] == 36
    torch.zeros(4, device="cuda").add_(1)
    torch.cuda.synchronize()


def test_leaf_autotuner():
    """leaf = 0 resolves to the autotuner's choice on the call's input: one of the supported sizes, cached,
    and the solve is the one that leaf size gives explicitly (bitwise)."""
    S = dev(synth.gaussian_lattice(600, 0.7, seed=11))
    leaf = sp.autotune_leaf(S, 1e-8)
    assert leaf in (32, 64, 128)
    assert sp.autotune_leaf(S, 1e-8) == leaf
    Y0, Z0, _ = sp.sqrt_invsqrt(S, 1e-8, 12, leaf=0)
    Y1, Z1, _ = sp.sqrt_invsqrt(S, 1e-8, 12, leaf=leaf)
    assert torch.equal(Y0, Y1) and torch.equal(Z0, Z1)
    assert sp.autotune_leaf(S, 1e-8, precision=sp.EMU64) == 64


# ------------------------------------------------------------------------------------------ damped, stabilised map


@pytest.mark.parametrize("n,nb,tau,order", [(200, 32, 1e-6, 0), (333, 64, 1e-8, 1), (96, 128, 0.0, 0),
                                            (129, 32, 1e-10, 1)])
def test_ns_scaled_map(n, nb, tau, order):
    """alpha(t), eps(t) of Sec. 4.2 "Mapping" on an ill-conditioned Gaussian decay (sigma 0.9): the map runs
    after the X product (it needs tr X), in place, with T's leaf norms."""
    S = synth.gaussian_lattice(n, 0.9, seed=n)
    Y, Z, st, ref = _ns_compare(S, nb, tau, 20, order=order, map=sp.MAP_SCALED)
    assert st["t_hist"][0] > 0.35          # the first steps run with alpha well above 1


def test_ns_scaled_map_converges_sooner():
    S = synth.kms(300, 0.99)
    # tau 1e-12 keeps the SpAMM error floor of t_k below the tolerance for both maps (17 vs 11 steps)
    _, _, s1, _ = _ns_compare(S, 32, 1e-12, 40, tol_t=1e-9, map=sp.MAP_SCALED)
    _, _, s0, _ = _ns_compare(S, 32, 1e-12, 40, tol_t=1e-9)
    assert s1["iters"] + 3 <= s0["iters"]


def test_ns_plain_map_is_default():
    S = synth.gaussian_lattice(150, 0.7, seed=3)
    a = sp.sqrt_invsqrt(dev(S), 1e-7, 10, leaf=32)
    b = sp.sqrt_invsqrt(dev(S), 1e-7, 10, leaf=32, map=sp.MAP_NS)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_ns_scaled_map_batched_equals_single():
    Ss = [synth.gaussian_lattice(n, 0.9, seed=n) for n in (120, 257)]
    Ys, Zs, _ = sp.sqrt_invsqrt_batched([dev(S) for S in Ss], [1e-8, 1e-8], 15, leaf=32, map=sp.MAP_SCALED)
    for S, Yb, Zb in zip(Ss, Ys, Zs):
        Y1, Z1, _ = sp.sqrt_invsqrt(dev(S), 1e-8, 15, leaf=32, map=sp.MAP_SCALED)
        assert torch.equal(Yb, Y1) and torch.equal(Zb, Z1)


@pytest.mark.parametrize("tol,mp", [(1e-2, 0), (1e-3, 0), (1e-3, 1), (1e-4, 1)])
def test_ns_tolerance_stop_in_graph(tol, mp):
    """A solve that stops on |t_k| <= tol_t runs as one captured graph: the kernels after the stop return on
    the device flag and the unpack takes the buffer of the last executed iteration (odd and even counts)."""
    S = synth.kms(320, 0.9)
    Y, Z, st, ref = _ns_compare(S, 32, 1e-10, 40, tol_t=tol, map=mp)
    assert st["iters"] == ref["iters"] < 40
    assert (st["task_hist"][st["iters"]:] == 0).all() if len(st["task_hist"]) > st["iters"] else True
    # a second call replays the same graph
    Y2, Z2, st2 = sp.sqrt_invsqrt(dev(S), 1e-10, 40, leaf=32, tol_t=tol, map=mp)
    assert st2["iters"] == st["iters"] and np.array_equal(host(Y2), Y) and np.array_equal(host(Z2), Z)


def test_loop_graph_launches_only_the_iterations_run():
    """The iteration is a WHILE conditional node of the solve's graph: a solve stopped by tol_t launches the
    kernels of the iterations it ran (rounded up to the two-iteration body), not those of maxit."""
    S = synth.kms(256, 0.9)
    kw = dict(leaf=32)

    def launches(**extra):
        sp.sqrt_invsqrt(dev(S), 1e-10, 30, **kw, **extra)          # captures the graph
        torch.cuda.synchronize()
        l0 = sp.kernel_launches()
        _, _, st = sp.sqrt_invsqrt(dev(S), 1e-10, 30, **kw, **extra)
        return sp.kernel_launches() - l0, st["iters"]

    fixed, it_fixed = launches()
    stopped, it_stop = launches(tol_t=1e-3)
    assert it_fixed == 30 and it_stop < 12
    per_iter = fixed / 30.0
    assert stopped <= per_iter * (it_stop + 1) + 20, (stopped, fixed, it_stop)


# ------------------------------------------------------------------------------------------ single channel


def test_ns_single_channel_gaussian_256_leaf32():
    """Eq. (single) on the small Gaussian configuration: per-iteration task counts of the z, s z and x
    products equal the oracle's."""
    S = synth.gaussian_lattice(256, 0.6, seed=0)
    Y, Z, st, ref = _ns_compare(S, 32, 1e-6, 30, channel=sp.CHANNEL_SINGLE)
    np.testing.assert_array_equal(st["task_hist"], ref["task_hist"])


@pytest.mark.parametrize("n,nb,tau,mp", [(333, 64, 1e-8, 0), (200, 128, 0.0, 0), (300, 32, 1e-9, 1),
                                         (129, 64, 1e-10, 1)])
def test_ns_single_channel(n, nb, tau, mp):
    S = synth.gaussian_lattice(n, 0.8, seed=n)
    _ns_compare(S, nb, tau, 20, channel=sp.CHANNEL_SINGLE, map=mp)


def test_ns_single_channel_tolerance_stop():
    S = synth.kms(320, 0.9)
    Y, Z, st, ref = _ns_compare(S, 32, 1e-10, 40, tol_t=1e-3, channel=sp.CHANNEL_SINGLE)
    assert st["iters"] == ref["iters"] < 40


def test_ns_single_channel_batched_equals_single():
    Ss = [synth.gaussian_lattice(n, 0.7, seed=n) for n in (96, 200)]
    Ys, Zs, _ = sp.sqrt_invsqrt_batched([dev(S) for S in Ss], [1e-8, 1e-8], 12, leaf=32,
                                        channel=sp.CHANNEL_SINGLE)
    for S, Yb, Zb in zip(Ss, Ys, Zs):
        Y1, Z1, _ = sp.sqrt_invsqrt(dev(S), 1e-8, 12, leaf=32, channel=sp.CHANNEL_SINGLE)
        assert torch.equal(Yb, Y1) and torch.equal(Zb, Z1)


# ------------------------------------------------------------------------------------------ plane-diagonal profile


@pytest.mark.parametrize("channel,tol", [(0, 0.0), (1, 0.0), (0, 1e-3)])
def test_lens_profile_matches_oracle(channel, tol):
    """Per-iteration |i-j|, |j-k|, |i-k| histograms of every product's surviving triples (Sec. 7.2 lensing):
    identical to the oracle's where the task lists are (the Gaussian 256 / N_b 32 case)."""
    S = synth.gaussian_lattice(256, 0.6, seed=0)
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 1e-6, 16, leaf=32, channel=channel, tol_t=tol, lens_bins=5)
    ref = oracle.sqrt_invsqrt(S, 32, 1e-6, 16, channel=channel, tol_t=tol, lens_bins=5)
    assert st["iters"] == ref["iters"]
    np.testing.assert_array_equal(st["task_hist"], ref["task_hist"])
    np.testing.assert_array_equal(st["lens_hist"], ref["lens_hist"])
    # the profile changes the results in no way
    Y0, Z0, _ = sp.sqrt_invsqrt(dev(S), 1e-6, 16, leaf=32, channel=channel, tol_t=tol)
    assert torch.equal(Y, Y0) and torch.equal(Z, Z0)


# ------------------------------------------------------------------------------------------ product representation


def test_product_representation_matches_oracle():
    """Sec. 6 product representation on an ill-conditioned Gaussian decay (sigma 0.9): three slices at
    tau0 = 1e-3 with residual products at tau1 = 1e-5, against the oracle's."""
    S = synth.gaussian_lattice(200, 0.9, seed=7)
    mus = [0.1, 0.01, 0.001]
    Z, info = sp.invsqrt_product(dev(S), mus, 1e-3, 1e-5, 30, leaf=32)
    ref = oracle.invsqrt_product(S, 32, mus, 1e-3, 1e-5, 30)
    assert info["iters"] == list(ref["iters"])
    Z = host(Z)
    assert np.linalg.norm(Z - ref["Z"]) <= 1e-9 * np.linalg.norm(ref["Z"])
    # host pointers give the same factor
    Zh, _ = sp.invsqrt_product(S, mus, 1e-3, 1e-5, 30, leaf=32)
    np.testing.assert_array_equal(Zh, Z)


def test_product_representation_telescopes_at_tau0():
    S = synth.gaussian_lattice(150, 0.9, seed=8)
    lam, Q = np.linalg.eigh(S)
    c0 = np.abs(S).sum(1).max()
    Z, _ = sp.invsqrt_product(dev(S), [0.1, 0.01, 0.0], 0.0, 0.0, 60, leaf=64)
    Zw = (Q / np.sqrt(lam)) @ Q.T
    assert np.linalg.norm(host(Z) - Zw) <= 1e-10 * np.linalg.norm(Zw)
    assert c0 > 0


# ------------------------------------------------------------------------------------------ edge cases of the options


@pytest.mark.parametrize("n", [1, 2, 33])
def test_options_on_tiny_and_ragged_sizes(n):
    """Single channel, damped map and product representation at n = 1, 2 and a ragged 33 (one partial leaf)."""
    S = synth.kms(n, 0.7) if n > 1 else np.array([[2.5]])
    for kw in (dict(channel=sp.CHANNEL_SINGLE), dict(map=sp.MAP_SCALED), dict(channel=sp.CHANNEL_SINGLE,
                                                                             map=sp.MAP_SCALED)):
        _ns_compare(S, 32, 1e-9, 15, **kw)
    Z, info = sp.invsqrt_product(dev(S), [0.1, 0.0], 1e-9, 1e-12, 30, leaf=32)
    ref = oracle.invsqrt_product(S, 32, [0.1, 0.0], 1e-9, 1e-12, 30)
    assert np.linalg.norm(host(Z) - ref["Z"]) <= 1e-10 * np.linalg.norm(ref["Z"])


def test_one_level_product_representation_is_the_regularised_solve():
    S = synth.gaussian_lattice(150, 0.8, seed=11)
    Z1, info = sp.invsqrt_product(dev(S), [0.01], 1e-7, 1e-9, 20, leaf=32)
    _, Z2, st = sp.sqrt_invsqrt(dev(S), 1e-7, 20, leaf=32, mu_rel=0.01)
    assert torch.equal(Z1, Z2) and info["iters"] == [st["iters"]]


def test_lens_single_bin_counts_every_task():
    S = synth.gaussian_lattice(128, 0.6, seed=12)
    _, _, st = sp.sqrt_invsqrt(dev(S), 1e-6, 6, leaf=32, lens_bins=1)
    assert (st["lens_hist"][:, :, :, 0] == st["task_hist"][:, :, None]).all()


@pytest.mark.parametrize("precision", [sp.FP64, sp.EMU64])
def test_profiled_single_product(precision):
    """opts.profile on an uncaptured call (one product): the leaf-product kernel is timed, the result is the
    unprofiled one."""
    A = synth.decay_matrix(512, seed=3, length=20.0)
    C0, _ = sp.multiply(dev(A), dev(A), 1e-10, leaf=64, precision=precision)
    C1, st = sp.multiply(dev(A), dev(A), 1e-10, leaf=64, precision=precision, profile=True)
    assert torch.equal(C0, C1)
    assert st["gemm_ms"] > 0 and st["gemm_launches"] == 1
    if precision == sp.EMU64:
        assert st["tensor_units"] == 12 * st["tasks_total"]


def test_pinned_host_buffers_are_used_in_place():
    """Page-locked host S, Y, Z: the pack and unpack kernels read and write them directly (no staging);
    the result equals the device-pointer solve's bit for bit, and pageable host buffers (staged) agree too."""
    S = synth.gaussian_lattice(300, 0.7, seed=13)
    Sp = torch.from_numpy(S).pin_memory()
    Yp = torch.empty_like(Sp).pin_memory()
    Zp = torch.empty_like(Sp).pin_memory()
    sp.sqrt_invsqrt(Sp, 1e-8, 15, leaf=64, Y=Yp, Z=Zp)
    Yd, Zd, _ = sp.sqrt_invsqrt(dev(S), 1e-8, 15, leaf=64)
    Yh, Zh, _ = sp.sqrt_invsqrt(S, 1e-8, 15, leaf=64)
    assert np.array_equal(Yp.numpy(), host(Yd)) and np.array_equal(Zp.numpy(), host(Zd))
    assert np.array_equal(Yh, host(Yd)) and np.array_equal(Zh, host(Zd))
    for prec in (sp.FP64, sp.EMU64):
        Cp = torch.empty_like(Sp).pin_memory()
        sp.multiply(Sp, Sp, 1e-8, leaf=64, precision=prec, out=Cp)
        Cd, _ = sp.multiply(dev(S), dev(S), 1e-8, leaf=64, precision=prec)
        assert np.array_equal(Cp.numpy(), host(Cd))

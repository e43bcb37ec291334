"""GPU parity of the tensor-core (SPAMM_EMU64) leaf products against the FP64 CPU oracle.

Error model (derived in kernels_emu.cu): each operand entry is held to
2^-49 2^e of its row (A role) or column (B role) scale 2^e <= 4 max|.|;
slice pairs p+q >= 6 are dropped except (1,5), (3,3), (5,1).  Per product
element the error is at most a few K 2^-48 2^(eA_r + eB_c) plus the FP64
rounding of the final value, K = inner length.  The tests use
  |C - C_oracle| <= K 2^-42 rowmax(A)_r colmax(B)_c + 4 K u (|A||B|)_rc
(2^(eA) <= 4 rowmax, 2^(eB) <= 4 colmax).  Integer inputs whose row and column
maxima are powers of two are represented exactly, so tau = 0 products are
then bitwise equal to the exact product.  Newton-Schulz with these products:
||Z - Z_oracle||_F / ||Z_oracle||_F <= 1e-9 (the iteration carries product
errors forward without damping them; a numpy model of this arithmetic gives
about 1e-10 residuals on KMS at N = 512-1024).
"""
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


def _tol(A, B, K):
    ra = np.abs(A).max(axis=1)[:, None]
    cb = np.abs(B).max(axis=0)[None, :]
    return K * 2.0 ** -42 * ra * cb + 4 * K * U * (np.abs(A) @ np.abs(B)) + 1e-300


@pytest.mark.parametrize("n", [64, 128, 200, 512])
def test_emu_integer_tau0_bitwise(n):
    rng = np.random.default_rng(n)
    A = rng.integers(-2, 3, size=(n, n)).astype(np.float64)
    B = rng.integers(-2, 3, size=(n, n)).astype(np.float64)
    A[:, 0] = 2.0          # every row / column maximum is exactly 2
    B[0, :] = -2.0
    C, st = sp.multiply(dev(A), dev(B), 0.0, leaf=64, precision=sp.EMU64)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(C.cpu().numpy(), exact)


@pytest.mark.parametrize("n,tau", [(256, 1e-3), (300, 1e-6), (640, 0.0), (1024, 1e-8)])
def test_emu_multiply_matches_oracle(n, tau):
    A = synth.decay_matrix(n, seed=11, length=n / 10)
    B = synth.decay_matrix(n, seed=12, length=n / 14)
    C, st = sp.multiply(dev(A), dev(B), tau, leaf=64, precision=sp.EMU64)
    C = C.cpu().numpy()
    gt, _, _ = sp.cull(dev(A), dev(B), tau, 64)
    Co = oracle.leaf_products(A, B, 64, gt)
    assert st["tasks_total"] == len(gt)
    m = (n + 63) // 64
    assert (np.abs(C - Co) <= _tol(A, B, m * 64)).all()


def test_emu_multiply_kms_scales():
    """Rows with very different magnitudes (scaled KMS): per-row scales keep small rows accurate."""
    n = 384
    S = synth.kms(n, 0.8)
    d = np.exp(np.linspace(-8, 3, n))
    A = d[:, None] * S
    B = S * d[None, :]
    C, _ = sp.multiply(dev(A), dev(B), 0.0, leaf=64, precision=sp.EMU64)
    Co, _ = oracle.spamm(A, B, 64, 0.0)
    assert (np.abs(C.cpu().numpy() - Co) <= _tol(A, B, n)).all()


def _emu_ns(S, tau, maxit, **kw):
    Y, Z, st = sp.sqrt_invsqrt(dev(S), tau, maxit, leaf=64, precision=sp.EMU64, **kw)
    ref = oracle.sqrt_invsqrt(S, 64, tau, maxit,
                              **{k: v for k, v in kw.items() if k in ("order", "mu_rel", "map", "channel")})
    ez = np.linalg.norm(Z.cpu().numpy() - ref["Z"]) / np.linalg.norm(ref["Z"])
    ey = np.linalg.norm(Y.cpu().numpy() - ref["Y"]) / np.linalg.norm(ref["Y"])
    return ez, ey, st, ref


@pytest.mark.parametrize("kind,n,tau", [("gauss", 256, 1e-6), ("kms", 512, 1e-10), ("gauss", 700, 1e-9)])
def test_emu_ns_matches_oracle(kind, n, tau):
    S = synth.gaussian_lattice(n, 0.6, seed=0) if kind == "gauss" else synth.kms(n, 0.9)
    ez, ey, st, ref = _emu_ns(S, tau, 30)
    assert ez <= 1e-9 and ey <= 1e-9, (ez, ey)


def test_emu_ns_transposed_order():
    S = synth.gaussian_lattice(320, 0.7, seed=4)
    ez, ey, st, ref = _emu_ns(S, 1e-9, 25, order=sp.ORDER_TRANSPOSED)
    assert ez <= 1e-9 and ey <= 1e-9, (ez, ey)


def test_emu_ns_benchmark_configuration():
    """The configuration the benchmark times, against the oracle at full size: KMS rho 0.9, N 4096, N_b 64,
    tau 1e-14, tau_s 1e-16, 30 iterations of the dual channel with tensor-core leaf products.  Y and Z agree
    with the oracle to the tensor-core path's 1e-9 and the residual meets the 1e-8 gate.

    The task lists are not compared triple by triple here.  The tensor-core products are FP64-class
    normwise: an entry carries an absolute error of a few 2^-48 of its row and column scale, whatever its own
    size.  Far from the diagonal, where the FP64 products are many orders below that level, the tensor-core
    products hold rounding noise at that level instead, and at tau_s = 1e-16 the y product's threshold sits
    just below it: those noise tiles pass the cull and add leaf products (measured: 17 % more over the solve,
    up to 3x in single late products), each contributing below tau_s ||T|| ||Y||.  So the test bounds the
    solve's task total to [0.95, 1.25] x the oracle's; the FP64 path's lists are compared exactly
    (test_ns_kms_4096_benchmark_tau)."""
    S = synth.kms(4096, 0.9)
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 1e-14, 30, leaf=64, precision=sp.EMU64, residual=True)
    ref = oracle.sqrt_invsqrt(S, 64, 1e-14, 30)
    ez = np.linalg.norm(Z.cpu().numpy() - ref["Z"]) / np.linalg.norm(ref["Z"])
    ey = np.linalg.norm(Y.cpu().numpy() - ref["Y"]) / np.linalg.norm(ref["Y"])
    kg = np.asarray(st["task_hist"], dtype=np.float64)
    ko = np.asarray(ref["task_hist"], dtype=np.float64)
    print(f"ez {ez:.3e} ey {ey:.3e} resid {st['resid_F']:.3e} tasks gpu {kg.sum():.0f} oracle {ko.sum():.0f} "
          f"max per-product rel diff {np.max(np.abs(kg - ko) / np.maximum(ko, 1)):.3f}")
    assert st["iters"] == ref["iters"] == 30
    assert ez <= 1e-9 and ey <= 1e-9, (ez, ey)
    assert st["resid_F"] <= 1e-8, st["resid_F"]
    np.testing.assert_allclose(st["t_hist"], ref["t_hist"], rtol=0, atol=1e-12)
    assert 0.95 * ko.sum() <= kg.sum() <= 1.25 * ko.sum()


def test_emu_ns_residual_gate():
    S = synth.kms(1024, 0.9)
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 1e-14, 30, leaf=64, precision=sp.EMU64, residual=True)
    assert st["resid_F"] <= 1e-8, st["resid_F"]


def test_emu_batched_equals_single():
    specs = synth.batch_mix(5, lo=128, hi=640, seed=7)
    Ss = [synth.make(s) for s in specs]
    Ys, Zs, _ = sp.sqrt_invsqrt_batched([dev(S) for S in Ss], [1e-8] * len(Ss), 20, leaf=64, precision=sp.EMU64)
    for S, Yb, Zb in zip(Ss, Ys, Zs):
        Y1, Z1, _ = sp.sqrt_invsqrt(dev(S), 1e-8, 20, leaf=64, precision=sp.EMU64)
        assert torch.equal(Yb, Y1) and torch.equal(Zb, Z1)


def test_emu_rejects_other_leaf_sizes():
    S = synth.kms(128, 0.5)
    with pytest.raises(sp.SpammError):
        sp.sqrt_invsqrt(dev(S), 1e-8, 5, leaf=32, precision=sp.EMU64)


def test_emu_output_tile_with_more_than_256_tasks():
    """m = 257 leaf tiles per side: only block row 0 of A and block column 0 of B are nonzero, so output tile
    (0, 0) carries all 257 products (more tasks than one 256-entry list could hold) and every other tile is
    exactly zero."""
    nb, m = 64, 257
    n = nb * m
    rng = np.random.default_rng(257)
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    A[:nb, :] = rng.standard_normal((nb, n))
    B[:, :nb] = rng.standard_normal((n, nb))
    C, st = sp.multiply(dev(A), dev(B), 1e-12, leaf=nb, precision=sp.EMU64)
    assert st["tasks_total"] == m
    C00 = C[:nb, :nb].cpu().numpy()
    rest = C.clone()
    rest[:nb, :nb] = 0
    assert int(torch.count_nonzero(rest)) == 0
    del rest, C
    tasks = np.array([(0, j, 0) for j in range(m)], dtype=np.int32)
    Co = oracle.leaf_products(A, B, nb, tasks)[:nb, :nb]
    As, Bs = A[:nb, :], B[:, :nb]
    assert (np.abs(C00 - Co) <= _tol(As, Bs, n)).all()


@pytest.mark.parametrize("n,tau,order", [(256, 1e-8, 0), (700, 1e-10, 1)])
def test_emu_ns_scaled_map(n, tau, order):
    """Damped, stabilised map on the tensor-core path: X is written plain, the map kernel forms T in place
    with its leaf norms and row/column maxima, then T is sliced."""
    S = synth.gaussian_lattice(n, 0.9, seed=1)
    ez, ey, st, ref = _emu_ns(S, tau, 20, order=order, map=sp.MAP_SCALED)
    assert ez <= 1e-9 and ey <= 1e-9, (ez, ey)
    np.testing.assert_allclose(st["t_hist"], ref["t_hist"], rtol=0, atol=1e-11)


@pytest.mark.parametrize("n,tau,mp", [(256, 1e-9, 0), (700, 1e-12, 0), (320, 1e-10, 1)])
def test_emu_ns_single_channel(n, tau, mp):
    """Eq. (single) on the tensor-core path: Z^T's slices come from the tile transpose with Z's column maxima
    as its row maxima."""
    S = synth.gaussian_lattice(n, 0.7, seed=2)
    ez, ey, st, ref = _emu_ns(S, tau, 20, channel=sp.CHANNEL_SINGLE, map=mp)
    assert ez <= 1e-9 and ey <= 1e-9, (ez, ey)
    np.testing.assert_allclose(st["t_hist"], ref["t_hist"], rtol=0, atol=1e-11)


def test_emu_lens_profile_counts():
    """The plane-diagonal profile on the tensor-core path: every product's histogram sums to its task count,
    and the first z product (Z0 = I on the left) lies on the plane i = j."""
    S = synth.kms(512, 0.9)
    Y, Z, st = sp.sqrt_invsqrt(dev(S), 1e-10, 10, leaf=64, precision=sp.EMU64, lens_bins=8)
    h = st["lens_hist"]
    assert h.shape == (10, 3, 3, 8)
    assert (h.sum(axis=3) == st["task_hist"][:, :, None]).all()
    assert h[0, 1, 0, 0] == st["task_hist"][0][1] and h[0, 1, 0, 1:].sum() == 0


def test_emu_product_representation_matches_oracle():
    S = synth.gaussian_lattice(256, 0.8, seed=9)
    mus = [0.05, 0.0005]
    Z, info = sp.invsqrt_product(dev(S), mus, 1e-8, 1e-10, 25, leaf=64, precision=sp.EMU64)
    ref = oracle.invsqrt_product(S, 64, mus, 1e-8, 1e-10, 25)
    assert info["iters"] == list(ref["iters"])
    Z = Z.cpu().numpy()
    assert np.linalg.norm(Z - ref["Z"]) <= 1e-8 * np.linalg.norm(ref["Z"])


def test_expired_device_wait_returns_timeout_and_the_next_call_succeeds():
    """Every wait inside the tensor-core kernel gives up after a bounded number of polls.  Here one is made to
    expire (a barrier nothing arrives at, before any copy or product is issued): the call reports
    SPAMM_ERR_TIMEOUT instead of hanging, the kernel frees its tensor memory, and the next calls (and other
    work on the device) run normally with the same results as before."""
    A = dev(synth.decay_matrix(448, seed=21, length=40.0))
    B = dev(synth.decay_matrix(448, seed=22, length=30.0))
    C0, _ = sp.multiply(A, B, 1e-9, leaf=64, precision=sp.EMU64)
    assert sp.lib().spamm_test_expire_next_wait(-1) == -1
    assert sp.lib().spamm_test_expire_next_wait(64) == 0
    with pytest.raises(sp.SpammError) as ei:
        sp.multiply(A, B, 1e-9, leaf=64, precision=sp.EMU64)
    assert ei.value.status == -5
    C1, _ = sp.multiply(A, B, 1e-9, leaf=64, precision=sp.EMU64)
    assert torch.equal(C0, C1)
    Y, Z, st = sp.sqrt_invsqrt(dev(synth.kms(256, 0.8)), 1e-10, 12, leaf=64, precision=sp.EMU64)
    assert st["status"] == 0
    x = torch.arange(1, 1025, device="cuda", dtype=torch.float64).sum()
    torch.cuda.synchronize()
    assert float(x) == 1024 * 1025 / 2


@pytest.mark.parametrize("n,length", [(1000, 400.0), (2048, 900.0)])
def test_alternating_accumulator_layout_gives_the_same_bits(n, length):
    """The leaf kernel can place the accumulator chunks of one output tile at alternating tensor-memory
    columns (the next chunk's products overlap the read-out of this one).  Tiles of one, two, three and more
    chunks (7 tasks each) exercise every hand-over between the two positions; products and solves must come
    out bit for bit as with the fixed position."""
    A = dev(synth.decay_matrix(n, seed=31, length=length))
    B = dev(synth.decay_matrix(n, seed=32, length=length))
    S = dev(synth.gaussian_lattice(n, 0.7, seed=3))
    out = {}
    try:
        for mode in (0, 1):
            assert sp.lib().spamm_test_emu_alternate(mode) == 0
            sp.release()
            C, st = sp.multiply(A, B, 1e-10, leaf=64, precision=sp.EMU64)
            Y, Z, s2 = sp.sqrt_invsqrt(S, 1e-10, 8, leaf=64, precision=sp.EMU64, raise_on=False)
            out[mode] = (C, st["tasks_total"], Y, Z, s2["tasks_total"])
    finally:
        sp.lib().spamm_test_emu_alternate(-1)
        sp.release()
    assert sp.lib().spamm_test_emu_alternate(2) == -1
    (C0, t0, Y0, Z0, k0), (C1, t1, Y1, Z1, k1) = out[0], out[1]
    m = (n + 63) // 64
    assert t0 == t1 and t0 > 7 * m * m, (t0, m)   # more than one chunk per tile on average
    assert torch.equal(C0, C1) and torch.equal(Y0, Y1) and torch.equal(Z0, Z1) and k0 == k1

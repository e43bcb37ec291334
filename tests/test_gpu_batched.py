"""The batched solve engine: many independent square-root solves advanced together, one stage of the
dual-channel iteration (Eq. (cannonical)) at a time, each stage one launch of each kernel over every
matrix's products, captured once as a CUDA graph.

Every matrix's result must be the one a single call gives, bit for bit: the same task lists, iterations,
trace errors and outputs, whatever it is batched with.  And the launches per iteration must not grow with
the number of matrices.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_1508_05856_gb300")

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _check_equal_to_single(Ss, taus, maxit, **kw):
    Ys, Zs, sts = sp.sqrt_invsqrt_batched([dev(S) for S in Ss], taus, maxit, raise_on=False, **kw)
    for S, t, Yb, Zb, sb in zip(Ss, taus, Ys, Zs, sts):
        Y1, Z1, s1 = sp.sqrt_invsqrt(dev(S), t, maxit, raise_on=False, **kw)
        assert torch.equal(Yb, Y1) and torch.equal(Zb, Z1)
        assert sb["iters"] == s1["iters"] and sb["tasks_total"] == s1["tasks_total"]
        assert sb["t_final"] == s1["t_final"] and sb["scale_c"] == s1["scale_c"]
    return Ys, Zs, sts


@pytest.mark.parametrize("precision,leaf", [(0, 32), (0, 64), (0, 128), (1, 64)])
def test_batch_of_mixed_sizes_equals_single_calls(precision, leaf):
    """Sizes from one tile (n <= leaf) to many, ragged edges, KMS and Gaussian types."""
    sizes = [40, 64, 97, 200, 333, 512, 700]
    Ss = [synth.kms(n, 0.6 + 0.05 * (q % 6)) if q % 2 else synth.gaussian_lattice(n, 0.7, seed=q)
          for q, n in enumerate(sizes)]
    taus = [1e-6, 1e-8, 1e-7, 1e-9, 1e-6, 1e-10, 1e-8]
    _check_equal_to_single(Ss, taus, 16, leaf=leaf, precision=precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_transposed_order_shift_and_tau_s(precision):
    Ss = [synth.gaussian_lattice(n, 0.8, seed=n) for n in (128, 256, 384)]
    _check_equal_to_single(Ss, [1e-7] * 3, 14, leaf=64, precision=precision, order=sp.ORDER_TRANSPOSED,
                           mu_rel=1e-3, tau_s=3e-9)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_stops_each_matrix_at_its_own_tolerance(precision):
    """With tol_t the matrices stop after different iteration counts (odd and even): each stops where its
    single call stops, the others go on."""
    Ss = [synth.kms(256, 0.5), synth.kms(320, 0.9), synth.gaussian_lattice(448, 0.9, seed=1), synth.kms(128, 0.7)]
    Ys, Zs, sts = _check_equal_to_single(Ss, [1e-10] * 4, 40, leaf=64, precision=precision, tol_t=1e-11)
    iters = [s["iters"] for s in sts]
    assert len(set(iters)) > 1 and max(iters) < 40, iters
    assert len({i % 2 for i in iters}) == 2, iters


def test_batch_matches_oracle():
    Ss = [synth.kms(300, 0.85), synth.gaussian_lattice(260, 0.6, seed=5)]
    Ys, Zs, sts = sp.sqrt_invsqrt_batched([dev(S) for S in Ss], [1e-8, 1e-7], 25, leaf=32)
    for S, t, Y, Z, st in zip(Ss, [1e-8, 1e-7], Ys, Zs, sts):
        ref = oracle.sqrt_invsqrt(S, 32, t, 25)
        assert np.linalg.norm(Z.cpu().numpy() - ref["Z"]) <= 1e-10 * np.linalg.norm(ref["Z"])
        assert np.linalg.norm(Y.cpu().numpy() - ref["Y"]) <= 1e-10 * np.linalg.norm(ref["Y"])
        assert st["iters"] == ref["iters"]


def test_batch_launches_per_iteration_do_not_grow_with_the_count():
    """Launches of a batched call grow with the count only by each matrix's setup and finish passes: the
    extra launches of ten more iterations are the same for 2 and for 6 matrices."""
    def launches(count, maxit):
        Ss = [dev(synth.kms(192 + 32 * q, 0.8)) for q in range(count)]
        sp.sqrt_invsqrt_batched(Ss, [1e-8] * count, maxit, leaf=64, precision=sp.EMU64)   # capture
        torch.cuda.synchronize()
        l0 = sp.kernel_launches()
        sp.sqrt_invsqrt_batched(Ss, [1e-8] * count, maxit, leaf=64, precision=sp.EMU64)
        torch.cuda.synchronize()
        return sp.kernel_launches() - l0

    d2 = launches(2, 20) - launches(2, 10)
    d6 = launches(6, 20) - launches(6, 10)
    assert d2 == d6 and d2 > 0, (d2, d6)
    assert launches(6, 10) - launches(2, 10) == 4 * (launches(3, 10) - launches(2, 10))


def test_batch_repeated_calls_replay_and_stay_identical():
    Ss = [dev(synth.gaussian_lattice(n, 0.75, seed=n)) for n in (192, 256)]
    a = sp.sqrt_invsqrt_batched(Ss, [1e-8, 1e-9], 12, leaf=64, precision=sp.EMU64)
    b = sp.sqrt_invsqrt_batched(Ss, [1e-8, 1e-9], 12, leaf=64, precision=sp.EMU64)
    for x, y in zip(a[0] + a[1], b[0] + b[1]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("precision", [0, 1])
def test_stage_schedule_for_one_solve_equals_the_branch_schedule(precision):
    """SPAMM_SCHED_STAGES runs one solve on the batched engine (the y and z products share each launch):
    the same result bit for bit; options the engine does not cover (the residual) fall back to branches."""
    S = dev(synth.gaussian_lattice(448, 0.75, seed=9))
    Y0, Z0, s0 = sp.sqrt_invsqrt(S, 1e-9, 18, leaf=64, precision=precision)
    Y1, Z1, s1 = sp.sqrt_invsqrt(S, 1e-9, 18, leaf=64, precision=precision, schedule=sp.SCHED_STAGES)
    assert s0["schedule"] == sp.SCHED_BRANCHES and s1["schedule"] == sp.SCHED_STAGES
    assert torch.equal(Y0, Y1) and torch.equal(Z0, Z1)
    assert np.array_equal(s0["task_hist"], s1["task_hist"]) and np.array_equal(s0["t_hist"], s1["t_hist"])
    _, _, s2 = sp.sqrt_invsqrt(S, 1e-9, 18, leaf=64, precision=precision, schedule=sp.SCHED_STAGES, residual=True)
    assert s2["schedule"] == sp.SCHED_BRANCHES and s2["resid_F"] >= 0


def test_schedule_autotuner_picks_a_schedule_and_keeps_it():
    S = dev(synth.kms(1536, 0.9))
    Y0, Z0, s0 = sp.sqrt_invsqrt(S, 1e-10, 14, leaf=64, precision=sp.EMU64)
    Y1, Z1, s1 = sp.sqrt_invsqrt(S, 1e-10, 14, leaf=64, precision=sp.EMU64, schedule=sp.SCHED_AUTO)
    assert s1["schedule"] in (sp.SCHED_BRANCHES, sp.SCHED_STAGES)
    assert torch.equal(Y0, Y1) and torch.equal(Z0, Z1)
    _, _, s2 = sp.sqrt_invsqrt(S, 1e-10, 14, leaf=64, precision=sp.EMU64, schedule=sp.SCHED_AUTO)
    assert s2["schedule"] == s1["schedule"]

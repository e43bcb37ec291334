"""Why the leaf products are FP64-class on every sweep: reduced-precision products early in the dual-channel
iteration leave an error that later sweeps at full precision do not remove.

The model: the dual-channel iteration of Eq. (cannonical) with alpha = 1 (T = (3I - X)/2), S scaled by its
Gershgorin bound, dense products (tau = 0), each product rounded by a stated arithmetic:
  * fp64   -- IEEE double;
  * fp32   -- operands rounded to IEEE single, single-precision sums (numpy float32 matmul);
  * tf32   -- operands rounded to nearest to 10 explicit mantissa bits (the TF32 tensor-core operand
              format), single-precision sums;
  * 3xtf32 -- the split-precision product a_hi b_hi + a_hi b_lo + a_lo b_hi with a = a_hi + a_lo,
              a_hi = tf32(a), a_lo = tf32(a - a_hi), single-precision sums;
  * bf16   -- operands rounded to bfloat16, single-precision sums.
The FP64 model is first pinned to the oracle's solve at tau = 0.  Near the fixed point the iteration's
Frechet derivative is idempotent (Sec. 3.2, Sec. 5.1): an error injected into Y and Z is neither amplified
nor damped, so whatever the early sweeps leave stays in the result.  The tests show it for every schedule a
reduced-precision plan could take: all sweeps reduced, the reduced sweeps followed by 3xTF32 and then FP64
sweeps, and the reduced sweeps followed by FP64 sweeps of the single channel, Eq. (single), whose map is
formed from s directly.  None comes within two orders of the 1e-8 gate on ||Z S Z - I||_F; all-FP64 products
reach 1e-12.
"""
import numpy as np
import pytest

import oracle
import synth

GATE = 1e-8


def _tf32(a):
    """Round float32 values to nearest (ties away from zero) at 10 explicit mantissa bits."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + (1 << 12)) & ~np.uint64((1 << 13) - 1)).astype(np.uint32)
    return b.view(np.float32)


def _bf16(a):
    """Round float32 values to nearest even at 7 explicit mantissa bits."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & ~np.uint64(0xFFFF)).astype(np.uint32)
    return b.view(np.float32)


def p_fp64(A, B):
    return A @ B


def p_fp32(A, B):
    return (A.astype(np.float32) @ B.astype(np.float32)).astype(np.float64)


def p_tf32(A, B):
    return (_tf32(A) @ _tf32(B)).astype(np.float64)


def p_bf16(A, B):
    return (_bf16(A) @ _bf16(B)).astype(np.float64)


def p_3xtf32(A, B):
    a, b = A.astype(np.float32), B.astype(np.float32)
    ah, bh = _tf32(a), _tf32(b)
    al, bl = _tf32(a - ah), _tf32(b - bh)
    return (ah @ bh + (ah @ bl + al @ bh)).astype(np.float64)


def dual_model(S, maxit, schedule, single_tail=0):
    """Dual channel for maxit sweeps with the product of sweep k given by schedule(k), then single_tail
    sweeps of the single channel in FP64 (z <- z h[z^T s z]).  Returns (Y, Z) unscaled."""
    n = S.shape[0]
    c = np.abs(S).sum(axis=1).max()
    s = S * (1.0 / c)
    eye = np.eye(n)
    Y, Z, T = s.copy(), eye.copy(), 1.5 * eye - 0.5 * s
    for k in range(maxit):
        P = schedule(k)
        Y = P(T, Y)
        Z = P(Z, T)
        T = 1.5 * eye - 0.5 * P(Y, Z)
    for _ in range(single_tail):
        Z = Z @ (1.5 * eye - 0.5 * (Z.T @ (s @ Z)))
        Y = s @ Z
    return Y * np.sqrt(c), Z * (1.0 / np.sqrt(c))


def resid(S, Z):
    return float(np.linalg.norm(Z @ S @ Z - np.eye(S.shape[0])))


def test_fp64_model_is_the_oracle_at_tau0():
    """The model with FP64 products follows the oracle's solve at tau = 0 to rounding."""
    S = synth.kms(192, 0.9)
    Y, Z = dual_model(S, 20, lambda k: p_fp64)
    ref = oracle.sqrt_invsqrt(S, 32, 0.0, 20)
    assert np.linalg.norm(Z - ref["Z"]) <= 1e-12 * np.linalg.norm(ref["Z"])
    assert np.linalg.norm(Y - ref["Y"]) <= 1e-12 * np.linalg.norm(ref["Y"])


def test_rounding_models():
    x = np.array([1.0 + 2.0 ** -11, 1.0 + 2.0 ** -10 + 2.0 ** -12, -3.0 - 2.0 ** -9], dtype=np.float32)
    assert list(_tf32(x)) == [1.0 + 2.0 ** -10, 1.0 + 2.0 ** -10, -3.0 - 2.0 ** -9]
    y = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8], dtype=np.float32)
    assert list(_bf16(y)) == [1.0, 1.0 + 2.0 ** -6]


@pytest.fixture(scope="module")
def kms384():
    return synth.kms(384, 0.9)


def test_all_fp64_meets_the_gate(kms384):
    _, Z = dual_model(kms384, 30, lambda k: p_fp64)
    assert resid(kms384, Z) <= 1e-11


@pytest.mark.parametrize("name,prod", [("fp32", p_fp32), ("tf32", p_tf32), ("3xtf32", p_3xtf32),
                                       ("bf16", p_bf16)])
def test_reduced_precision_everywhere_misses_the_gate(kms384, name, prod):
    _, Z = dual_model(kms384, 30, lambda k: prod)
    assert resid(kms384, Z) >= 100 * GATE, name


@pytest.mark.parametrize("name,sched", [
    ("tf32 x22, 3xtf32 x5, fp64 x3", lambda k: p_tf32 if k < 22 else (p_3xtf32 if k < 27 else p_fp64)),
    ("tf32 x20, fp64 x10", lambda k: p_tf32 if k < 20 else p_fp64),
    ("3xtf32 x20, fp64 x10", lambda k: p_3xtf32 if k < 20 else p_fp64),
    ("fp32 x20, fp64 x10", lambda k: p_fp32 if k < 20 else p_fp64),
    ("bf16 x20, fp64 x10", lambda k: p_bf16 if k < 20 else p_fp64),
])
def test_fp64_final_sweeps_do_not_remove_the_early_error(kms384, name, sched):
    _, Z = dual_model(kms384, 30, sched)
    assert resid(kms384, Z) >= 100 * GATE, name


@pytest.mark.parametrize("name,prod,k_low", [("tf32", p_tf32, 10), ("fp32", p_fp32, 10), ("3xtf32", p_3xtf32, 10)])
def test_single_channel_fp64_refinement_does_not_remove_it(kms384, name, prod, k_low):
    """The single channel's map comes from z^T s z, so it corrects the part of the error that z^T s z sees;
    the error the dual sweeps left includes a part z^T s z does not see, and it stays."""
    _, Z = dual_model(kms384, k_low, lambda k: prod, single_tail=5)
    assert resid(kms384, Z) >= 100 * GATE, name

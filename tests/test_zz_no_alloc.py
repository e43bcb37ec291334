"""spamm_multiply_noalloc, the allocation-free SpAMM product, checked against spamm_multiply.

The entry point serves callers that cannot let a library allocate device
memory: for example a service that reserves its whole GPU memory budget at
start-up and forbids allocation afterwards.  It keeps its scratch in one
fixed device array instead of cudaMalloc'd buffers.  These tests call it
through the C ABI on device pointers, several times in a row on one stream
with different inputs and leaf sizes.  Each result must equal
spamm_multiply's bit for bit (the same kernels on the same task lists), and
one is also checked against the CPU oracle within the product tolerance the
other parity tests use (4 K u |A||B| elementwise).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_1508_05856_gb300")

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def _noalloc(A, B, C, tau, leaf, stream):
    return sp.lib().spamm_multiply_noalloc(A.data_ptr(), B.data_ptr(), C.data_ptr(), A.shape[0], float(tau),
                                           int(leaf), stream)


def test_noalloc_two_calls_match_multiply():
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = [(300, 64, 1e-5, 1, 2), (512, 32, 1e-6, 3, 4), (512, 128, 1e-7, 5, 6)]
    mats = []
    for n, leaf, tau, sa, sb in cases:
        A = torch.from_numpy(synth.decay_matrix(n, seed=sa, length=n / 12)).to(dev)
        B = torch.from_numpy(synth.decay_matrix(n, seed=sb, length=n / 9)).to(dev)
        mats.append((A, B, torch.empty_like(A), tau, leaf))
    # the first call on this device looks up the array's address, and CUDA loads the code of each leaf size
    # on its first use: one call per leaf size before the free memory is read
    for A, B, C, tau, leaf in mats:
        assert _noalloc(A, B, C, tau, leaf, stream) == 0, sp.lib().spamm_last_error()
    torch.cuda.synchronize()
    for A, B, C, tau, leaf in mats:
        C.fill_(float("nan"))
    torch.cuda.synchronize()

    free_before = torch.cuda.mem_get_info(dev)[0]
    for A, B, C, tau, leaf in mats:             # calls in a row, ordered on one stream
        st = _noalloc(A, B, C, tau, leaf, stream)
        assert st == 0, sp.lib().spamm_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free_before

    for A, B, C, tau, leaf in mats:
        Cref, _ = sp.multiply(A, B, tau, leaf=leaf)
        assert torch.equal(C, Cref)
    # the first case against the oracle's product at the same tau
    A, B, C, tau, leaf = mats[0]
    An, Bn = A.cpu().numpy(), B.cpu().numpy()
    Co, _ = oracle.spamm(An, Bn, leaf, tau)
    bound = 4 * An.shape[0] * U * (np.abs(An) @ np.abs(Bn)) + 1e-300
    assert (np.abs(C.cpu().numpy() - Co) <= bound).all()


def test_noalloc_rejects_sizes_beyond_its_array_and_host_pointers():
    dev = torch.device("cuda:0")
    n = 513
    A = torch.zeros((n, n), dtype=torch.float64, device=dev)
    assert _noalloc(A, A, A, 0.0, 64, None) == -8
    assert b"512" in sp.lib().spamm_last_error()
    h = torch.zeros((8, 8), dtype=torch.float64)
    assert _noalloc(h, h, h, 0.0, 64, None) == -1

"""The request server: results equal standalone solves (bitwise), admission by device footprint."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_1508_05856_gb300")

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _mix(count, seed):
    tr = synth.serving_trace(count, rate=1e9, lo=128, hi=640, seed=seed, taus=(1e-6, 1e-8, 1e-10))
    return [(synth.make(r), r["tau"]) for r in tr]


@pytest.mark.parametrize("precision", [sp.FP64, sp.EMU64])
def test_server_results_equal_standalone(precision):
    reqs = _mix(8, seed=1)
    with sp.Server(bytes_budget=8 << 30, max_active=4, leaf=64, precision=precision) as srv:
        ids = []
        for q, (S, tau) in enumerate(reqs):
            ids.append(srv.submit(dev(S) if q % 2 == 0 else S, tau, 20))   # device and host requests mixed
        outs = [srv.wait(i) for i in ids]
    for (S, tau), (Y, Z, st, lat) in zip(reqs, outs):
        Y1, Z1, st1 = sp.sqrt_invsqrt(dev(S), tau, 20, leaf=64, precision=precision)
        Yn = Y.cpu().numpy() if hasattr(Y, "cpu") else Y
        Zn = Z.cpu().numpy() if hasattr(Z, "cpu") else Z
        np.testing.assert_array_equal(Yn, Y1.cpu().numpy())
        np.testing.assert_array_equal(Zn, Z1.cpu().numpy())
        assert st["tasks_total"] == st1["tasks_total"] and lat > 0


def test_server_tight_budget_still_completes():
    reqs = _mix(4, seed=2)
    with sp.Server(bytes_budget=24 << 20, max_active=4, leaf=64) as srv:   # about one n=640 request at a time
        ids = [srv.submit(dev(S), tau, 12) for S, tau in reqs]
        outs = [srv.wait(i) for i in ids]
    assert all(o[2]["status"] == 0 for o in outs)


def test_server_rejects_oversize_and_unknown():
    with sp.Server(bytes_budget=64 << 20, max_active=2, leaf=64) as srv:
        S = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
        with pytest.raises(sp.SpammError) as ei:
            srv.submit(S, 1e-8, 5)
        assert ei.value.status == -6
        with pytest.raises(sp.SpammError) as ei:
            srv.poll(12345)
        assert ei.value.status == -9


def test_plan_cache_stays_bounded_over_many_sizes():
    """Plans are cached per size; across many distinct sizes the idle cache is evicted (least recently used
    first) so that it never holds more than a quarter of the device, and the caller's own allocations keep
    succeeding."""
    free0, total = torch.cuda.mem_get_info()
    for k in range(48):
        n = 3008 + 64 * k
        S = torch.eye(n, dtype=torch.float64, device="cuda") * 0.5
        Y, Z, st = sp.sqrt_invsqrt(S, 1e-8, 1, leaf=64, precision=sp.EMU64)
        del S, Y, Z
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        # idle plans <= total/4, plus the plan in use, plus torch's own tensors of this step
        assert free0 - free <= total // 4 + (4 << 30), (k, free0 - free)
    sp.release()


@pytest.mark.parametrize("precision", [sp.FP64, sp.EMU64])
def test_server_groups_queued_requests_into_shared_launches(precision):
    """Device-resident requests queued behind a busy worker are solved as one batch: every stage of their
    iterations is one launch over all of them (far fewer launches than one solve per request), and each
    result is still bitwise the standalone one."""
    reqs = _mix(12, seed=5)
    mats = [dev(S) for S, _ in reqs]
    alone = [sp.sqrt_invsqrt(S, tau, 16, leaf=64, precision=precision) for S, (_, tau) in zip(mats, reqs)]
    torch.cuda.synchronize()
    l0 = sp.kernel_launches()
    for S, (_, tau) in zip(mats, reqs):
        sp.sqrt_invsqrt(S, tau, 16, leaf=64, precision=precision)
    torch.cuda.synchronize()
    l_alone = sp.kernel_launches() - l0
    with sp.Server(bytes_budget=16 << 30, max_active=1, leaf=64, precision=precision) as srv:
        l0 = sp.kernel_launches()
        ids = [srv.submit(S, tau, 16) for S, (_, tau) in zip(mats, reqs)]
        outs = [srv.wait(i) for i in ids]
        l_served = sp.kernel_launches() - l0
    for (Y1, Z1, st1), (Y, Z, st, lat) in zip(alone, outs):
        assert torch.equal(Y, Y1) and torch.equal(Z, Z1)
        assert st["status"] == 0 and st["iters"] == st1["iters"] and st["tasks_total"] == st1["tasks_total"]
    assert l_served < 0.6 * l_alone, (l_served, l_alone)

"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every symbol include/spamm.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

import paper_1508_05856_gb300 as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    txt = open(os.path.join(ROOT, "include", "spamm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(spamm_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_loads():
    path = sp.build()
    assert os.path.exists(path)
    L = sp.lib()
    assert sp.version().startswith("spamm-gb300")


def test_every_header_symbol_is_exported():
    syms = _header_symbols()
    assert syms, "no declarations parsed"
    assert sorted(sp.HEADER_SYMBOLS) == syms
    raw = ctypes.CDLL(sp.lib_path())
    for s in syms:
        assert hasattr(raw, s), s


def test_strerror_and_defaults():
    L = sp.lib()
    assert L.spamm_strerror(0) == b"SPAMM_OK"
    assert L.spamm_strerror(-3) == b"SPAMM_ERR_DIVERGED"
    o = sp.Opts()
    L.spamm_opts_init(ctypes.byref(o))
    assert o.leaf == 64 and o.precision == sp.FP64 and o.tau_s < 0 and o.order == sp.ORDER_PAPER
    assert o.map == sp.MAP_NS and o.channel == sp.CHANNEL_DUAL and o.schedule == sp.SCHED_BRANCHES


@pytest.mark.parametrize("n,tau,leaf", [(0, 1e-6, 64), (-5, 1e-6, 64), (64, -1.0, 64), (64, float("nan"), 64),
                                        (64, 1e-6, 48), (64, float("inf"), 64)])
def test_bad_arguments_rejected_without_device(n, tau, leaf):
    L = sp.lib()
    o = sp.Opts()
    L.spamm_opts_init(ctypes.byref(o))
    o.leaf = leaf
    buf = (ctypes.c_double * 16)()
    st = L.spamm_multiply(buf, buf, buf, n, tau, ctypes.byref(o), None)
    assert st == -1
    assert L.spamm_last_error()
    st = L.spamm_sqrt_invsqrt(buf, n, tau, 5, buf, buf, ctypes.byref(o), None)
    assert st == -1


def test_bad_option_fields_rejected():
    L = sp.lib()
    o = sp.Opts()
    L.spamm_opts_init(ctypes.byref(o))
    o.order = 7
    buf = (ctypes.c_double * 16)()
    assert L.spamm_sqrt_invsqrt(buf, 4, 0.0, 5, buf, buf, ctypes.byref(o), None) == -1
    L.spamm_opts_init(ctypes.byref(o))
    o.map = 2
    assert L.spamm_sqrt_invsqrt(buf, 4, 0.0, 5, buf, buf, ctypes.byref(o), None) == -1
    assert b"map" in L.spamm_last_error()
    L.spamm_opts_init(ctypes.byref(o))
    o.channel = 3
    assert L.spamm_sqrt_invsqrt(buf, 4, 0.0, 5, buf, buf, ctypes.byref(o), None) == -1
    L.spamm_opts_init(ctypes.byref(o))
    o.channel = sp.CHANNEL_SINGLE
    o.order = sp.ORDER_TRANSPOSED
    assert L.spamm_sqrt_invsqrt(buf, 4, 0.0, 5, buf, buf, ctypes.byref(o), None) == -1
    assert b"single channel" in L.spamm_last_error()
    L.spamm_opts_init(ctypes.byref(o))
    o.schedule = 3
    assert L.spamm_sqrt_invsqrt(buf, 4, 0.0, 5, buf, buf, ctypes.byref(o), None) == -1
    assert b"schedule" in L.spamm_last_error()
    L.spamm_opts_init(ctypes.byref(o))
    o.mu_rel = -1.0
    assert L.spamm_sqrt_invsqrt(buf, 4, 0.0, 5, buf, buf, ctypes.byref(o), None) == -1
    L.spamm_opts_init(ctypes.byref(o))
    assert L.spamm_sqrt_invsqrt(None, 4, 0.0, 5, buf, buf, ctypes.byref(o), None) == -1
    assert L.spamm_sqrt_invsqrt_batched(-1, None, None, None, 5, None, None, None, None) == -1
    assert L.spamm_sqrt_invsqrt_batched(0, None, None, None, 5, None, None, None, None) == 0


def test_server_create_rejects_bad_budget_without_device():
    L = sp.lib()
    h = ctypes.c_void_p(0)
    assert L.spamm_server_create(0, 2, None, ctypes.byref(h)) == -1
    assert L.spamm_server_create(1 << 20, 0, None, ctypes.byref(h)) == -1
    assert L.spamm_server_destroy(None) == -1


def test_autotune_rejects_bad_arguments_without_device():
    L = sp.lib()
    buf = (ctypes.c_double * 16)()
    leaf = ctypes.c_int(-1)
    assert L.spamm_autotune_leaf(buf, 0, 1e-6, None, ctypes.byref(leaf)) == -1
    assert L.spamm_autotune_leaf(buf, 4, -1.0, None, ctypes.byref(leaf)) == -1
    assert L.spamm_autotune_leaf(None, 4, 1e-6, None, ctypes.byref(leaf)) == -1
    assert L.spamm_autotune_leaf(buf, 4, 1e-6, None, None) == -1
    assert leaf.value == -1


def test_product_representation_rejects_bad_arguments_without_device():
    L = sp.lib()
    o = sp.Opts()
    L.spamm_opts_init(ctypes.byref(o))
    buf = (ctypes.c_double * 16)()
    mu = (ctypes.c_double * 2)(0.1, 0.01)
    its = (ctypes.c_int * 2)()
    assert L.spamm_invsqrt_product(buf, 4, 0, mu, 1e-3, 1e-5, 10, buf, its, ctypes.byref(o)) == -1
    assert L.spamm_invsqrt_product(buf, 4, 2, mu, 1e-3, -1.0, 10, buf, its, ctypes.byref(o)) == -1
    bad = (ctypes.c_double * 2)(0.1, float("nan"))
    assert L.spamm_invsqrt_product(buf, 4, 2, bad, 1e-3, 1e-5, 10, buf, its, ctypes.byref(o)) == -1
    assert L.spamm_invsqrt_product(None, 4, 2, mu, 1e-3, 1e-5, 10, buf, its, ctypes.byref(o)) == -1


def test_test_hooks_reject_bad_arguments_without_device():
    """The two check hooks validate their argument on the host; a valid call only records the request."""
    L = sp.lib()
    assert L.spamm_test_expire_next_wait(-1) == -1
    assert L.spamm_test_expire_next_wait(0) == 0
    for bad in (-2, 2, 7):
        assert L.spamm_test_emu_alternate(bad) == -1
        assert "mode" in sp.lib().spamm_last_error().decode()
    for ok in (1, 0, -1):   # -1 last: the library's own choice again
        assert L.spamm_test_emu_alternate(ok) == 0

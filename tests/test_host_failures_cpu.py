"""Failure paths of the C ABI that need no GPU: a simulated out-of-memory.

kubo_debug_fail_allocations(n) makes the library's next n device allocations fail the way a
full device does.  The workspace allocation is the first device work of kubo_ahc after the
host-side validation, so on a machine without a GPU the call still reaches it and must
return KUBO_ERR_OOM -- without dereferencing the (dummy) device pointers -- and the pending
count must be consumed, so the next call's allocation is attempted for real.
"""
import ctypes

import numpy as np
import pytest

import tbgen

OOM = 5


@pytest.fixture(scope="module")
def L():
    from paper_2309_06675_gb300 import _build
    _build.build()
    import paper_2309_06675_gb300 as kubo
    return kubo, kubo.lib()


def _call_ahc(kubo, L, m, prec=0):
    o = kubo.Options()
    L.kubo_options_init(ctypes.byref(o))
    o.precision = prec
    R = np.ascontiguousarray(m.R, dtype=np.int32)
    km = np.array([3, 2, 2], dtype=np.int32)
    dummy = ctypes.c_void_p(256)   # never dereferenced: the call fails before any launch
    return L.kubo_ahc(dummy, R.ctypes.data_as(ctypes.c_void_p), m.W, m.N_R,
                      km.ctypes.data_as(ctypes.c_void_p), dummy, 1, 1e-3, dummy, ctypes.byref(o))


@pytest.mark.parametrize("prec", [0, 1, 4])
def test_simulated_allocation_failure_returns_oom(L, prec):
    kubo, lib = L
    m = tbgen.random_tb(4, 1, 1.0, 0)
    kubo.debug_fail_allocations(1)
    assert _call_ahc(kubo, lib, m, prec) == OOM
    kubo.debug_fail_allocations(0)


def test_pending_failures_are_consumed_one_per_allocation(L):
    kubo, lib = L
    m = tbgen.random_tb(4, 1, 1.0, 0)
    kubo.debug_fail_allocations(2)
    assert _call_ahc(kubo, lib, m) == OOM
    assert _call_ahc(kubo, lib, m) == OOM
    # the count is spent: the third call attempts the real allocation (which, without a GPU,
    # fails for another reason or, with one, proceeds) -- either way not via the hook
    kubo.debug_fail_allocations(0)


def test_invalid_options_are_rejected_before_allocation(L):
    kubo, lib = L
    m = tbgen.random_tb(4, 1, 1.0, 0)
    o = kubo.Options()
    lib.kubo_options_init(ctypes.byref(o))
    o.ql_max_sweeps = -1
    R = np.ascontiguousarray(m.R, dtype=np.int32)
    km = np.array([3, 2, 2], dtype=np.int32)
    dummy = ctypes.c_void_p(256)
    kubo.debug_fail_allocations(1)
    code = lib.kubo_ahc(dummy, R.ctypes.data_as(ctypes.c_void_p), m.W, m.N_R,
                        km.ctypes.data_as(ctypes.c_void_p), dummy, 1, 1e-3, dummy, ctypes.byref(o))
    assert code == 1   # KUBO_ERR_INVALID_ARG: validation comes first, the hook stays pending
    assert _call_ahc(kubo, lib, m) == OOM
    kubo.debug_fail_allocations(0)

"""The no-allocation selector replay (ampcg_selector_trace_noalloc).

It exists for callers that must not call cudaMalloc -- for example code that
runs while a caching allocator has reserved the device's free memory, or a
latency-critical loop that cannot afford cudaMalloc's implicit device
synchronisation -- and keeps its device scratch in a static array compiled
into the library.  Its output must equal the allocating entry point's
(ampcg_selector_trace) on the same input; the outputs are integer precision
codes, so equality is exact.  Two calls in a row check that the shared static
array carries no state from one call into the next.  This file is collected
last so that a run stopping at the first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_04155_b300")


def _call(fn_name, delta, nb, tol, policy):
    lib = P.load_library()
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    out = np.full(delta.size, 0xEE, dtype=np.uint8)
    pol = policy.to_c()
    st = getattr(lib, fn_name)(C.byref(pol), delta.ctypes.data_as(C.POINTER(C.c_double)),
                               delta.size - 1, nb, tol, out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return st, out


def _sequences():
    rng = np.random.default_rng(21)
    geo = 5.0 * 0.9 ** np.arange(600)
    osc = np.abs(3.0 * 0.97 ** np.arange(900) * (1.0 + 0.9 * np.sin(0.5 * np.arange(900))))
    noisy = np.exp(np.cumsum(rng.normal(-0.04, 0.25, 2000)))
    return [geo, osc, noisy]


@pytest.mark.parametrize("policy", [
    P.Policy(u0=P.FP64, criterion=P.CRIT_WINDOW),
    P.Policy(u0=P.FP16, criterion=P.CRIT_LINEAR),
    P.Policy(u0=P.FP32, criterion=P.CRIT_WINDOW, latch=0),
    P.Policy(criterion=P.CRIT_FIXED, fixed_uz=P.FP16, fixed_ur=P.FP32),
])
def test_noalloc_matches_allocating_entry_point_twice(policy):
    nb, tol = 3.0, 1e-9
    for delta in _sequences():
        st_ref, ref = _call("ampcg_selector_trace", delta, nb, tol, policy)
        assert st_ref == P.OK
        # two calls in a row, with a different (longer, then shorter) call in between
        st1, got1 = _call("ampcg_selector_trace_noalloc", delta, nb, tol, policy)
        _call("ampcg_selector_trace_noalloc", np.concatenate([delta, delta[::-1]]), nb * 2, tol, policy)
        st2, got2 = _call("ampcg_selector_trace_noalloc", delta, nb, tol, policy)
        assert st1 == P.OK and st2 == P.OK
        assert np.array_equal(got1, ref)
        assert np.array_equal(got2, ref)


def test_noalloc_python_wrapper_and_limit():
    delta = 2.0 * 0.95 ** np.arange(65536)      # m + 1 = 65536: the largest accepted
    pol = P.Policy()
    assert np.array_equal(P.selector_trace_noalloc(delta, 1.0, 1e-10, pol),
                          P.selector_trace(delta, 1.0, 1e-10, pol))
    too_long = np.ones(65537)
    st, _ = _call("ampcg_selector_trace_noalloc", too_long, 1.0, 1e-10, pol)
    assert st == P.ERR_INVALID_ARG
    assert "65536" in P.load_library().ampcg_last_error().decode()

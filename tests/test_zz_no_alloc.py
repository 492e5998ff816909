"""The no-allocation gradient-moment entry point.

sim_gradient_moments_noalloc exists for callers that cannot allocate device
memory themselves or through the library -- for example code whose GPU memory
is owned by another allocator or held to a fixed budget, or loops that must not
risk the synchronisation an allocation can bring.  It keeps its scratch in a
fixed array inside the library instead.  These tests call it through the C ABI
and check that two calls in a row give what the regular entry point gives, and
that requests larger than its fixed scratch are refused.  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1502_02908_gb300 import binding as B
from paper_1502_02908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12          # the tolerance the GPU parity tests use for floating point


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()


def _noalloc(s, days):
    d = np.ascontiguousarray(days, np.int32)
    out = np.zeros((d.size, B.N_MOMENTS), np.float64)
    per = np.zeros((s.R, 8), np.float64)
    st = s.L.sim_gradient_moments_noalloc(s.h, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), d.size,
                                          per.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    return st, out, per


def test_noalloc_matches_regular_entry_point_on_two_calls():
    w = W.sise_plain(N=150, T=40, n_events=1500, R=96)
    s = B.Sim.from_workload(w, score_reverse=True)
    s.run(w.T)
    s.score_backward()
    days = np.array([9, 19, 39])
    ref_out, ref_per = s.gradient_moments(days)
    import torch
    free = []
    for _ in range(2):
        st, out, per = _noalloc(s, days)
        free.append(torch.cuda.mem_get_info()[0])
        assert st == B.SIM_OK, s.L.sim_last_error(s.h)
        np.testing.assert_allclose(out, ref_out, rtol=RTOL, atol=0)
        np.testing.assert_allclose(per, ref_per, rtol=RTOL, atol=0)
    # the first call on a device may place the library's array in device memory
    # (lazy module loading); a later call takes no device memory at all
    assert free[1] == free[0]
    # a different request reuses the same scratch
    st, out, _ = _noalloc(s, days[:1])
    assert st == B.SIM_OK
    np.testing.assert_allclose(out, ref_out[:1], rtol=RTOL, atol=0)
    s.close()


def test_noalloc_refuses_requests_beyond_its_scratch():
    w = W.tiny_node(model=W.SISE, herd=4, infected=1, R=8193, T=2,
                    params=dict(upsilon=0.1, gamma=0.1, alpha=0.1, beta=0.1, epsilon=0.0))
    s = B.Sim.from_workload(w, score=True)
    st, _, _ = _noalloc(s, [0])
    assert st == B.SIM_E_INVALID_ARG
    assert b"8192" in s.L.sim_last_error(s.h)
    s.close()
    w = W.tiny_node(model=W.SISE, herd=4, infected=1, R=2, T=600,
                    params=dict(upsilon=0.1, gamma=0.1, alpha=0.1, beta=0.1, epsilon=0.0))
    s = B.Sim.from_workload(w, score=True)
    st, _, _ = _noalloc(s, np.arange(513))
    assert st == B.SIM_E_INVALID_ARG
    assert b"512" in s.L.sim_last_error(s.h)
    s.close()


def test_noalloc_returns_a_latched_device_error_as_the_regular_entry_point():
    # under the ERROR policy a run whose events ask for absent animals latches
    # SIM_E_UNDERFLOW; both entry points report it (and clear it) the same way
    w = W.sise3_national(N=3000, T=12, n_events=20_000, e1_source="powerlaw")
    days = np.array([5, 11])
    status = []
    for regular in (True, False):
        s = B.Sim.from_workload(w, underflow_error=True, score=True)
        s.run(w.T)
        if regular:
            with pytest.raises(B.SimError) as ei:
                s.gradient_moments(days)
            status.append(ei.value.status)
            ref_out, _ = s.gradient_moments(days)         # the error was cleared
        else:
            status.append(_noalloc(s, days)[0])
            st, out, _ = _noalloc(s, days)
            assert st == B.SIM_OK
            np.testing.assert_allclose(out, ref_out, rtol=RTOL, atol=0)
        s.close()
    assert status == [B.SIM_E_UNDERFLOW, B.SIM_E_UNDERFLOW]

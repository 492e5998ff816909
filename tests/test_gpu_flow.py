"""The dataflow day loop (SIM_LAUNCH_FLOW): one persistent launch over a call's
days with per-herd readiness instead of per-day barriers.  Its results equal the
per-day kernels and the oracle bit for bit (counts, phi, daily statistics,
counters) on every stochastic-step path, with several replicates, across split
calls, on components too large for a lane's staging slots, under the ERROR
policy and with the pre-event phi; and a wait that runs out returns
SIM_E_TIMEOUT with the device usable."""
import numpy as np
import pytest

import oracle
from paper_1502_02908_gb300 import binding as B
from paper_1502_02908_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()


def _run(w, launch, splits=None, warp=-1, group=-1, **kw):
    s = B.Sim.from_workload(w, **kw)
    s.set_group_threshold(group)
    s.tune(warp)
    s.set_launch(launch)
    status = None
    for nd in (splits or [w.T]):
        s.run(nd)
    try:
        s.sync()
    except B.SimError as e:
        status = e.status
    c, p, day = s.state()
    pi, pn, ctr = s.stats()
    s.close()
    return c, p, day, pi, pn, ctr, status


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("warp,group", [(400, 100), (1 << 30, 200), (1 << 30, 1 << 30)])
def test_flow_national_shape_equals_per_day_kernels(warp, group):
    w = W.sise3_national(N=4000, T=60, n_events=150_000)
    _same(_run(w, "flow", warp=warp, group=group), _run(w, "stream", warp=warp, group=group))


def test_flow_equals_oracle_with_replicates_and_split_calls():
    w = W.sise3_batched(R=3, T=50, base=W.sise3_national(N=2000, T=50, n_events=60_000))
    ref = oracle.run(w)
    c, p, day, pi, pn, ctr, st = _run(w, "flow", splits=[1, 17, 32], warp=300, group=100)
    assert st is None and day == w.T
    assert np.array_equal(c, ref.counts) and np.array_equal(p, ref.phi)
    assert np.array_equal(pi[:, :w.T], ref.prev_i) and np.array_equal(pn[:, :w.T], ref.prev_n)
    assert np.array_equal(ctr, ref.counters)


def test_flow_sise_plain_and_pre_event_phi():
    w = W.sise_plain(N=1500, T=80, n_events=8000)
    _same(_run(w, "flow"), _run(w, "stream"))
    ref = oracle.run(w, phi_pre_event=True)
    c, p, *_ = _run(w, "flow", phi_pre_event=True)
    assert np.array_equal(c, ref.counts) and np.array_equal(p, ref.phi)


@pytest.mark.parametrize("underflow_error", [False, True])
def test_flow_large_components_clamps_and_error_policy(underflow_error):
    # "powerlaw" puts ~8 % of the events on one small herd: day components larger
    # than a lane's staging slots, many clamped (or, under ERROR, skipped) events
    w = W.sise3_national(N=3000, T=40, n_events=60_000, e1_source="powerlaw")
    ref = oracle.run(w, underflow_error=underflow_error)
    c, p, day, pi, pn, ctr, st = _run(w, "flow", underflow_error=underflow_error)
    assert st == (B.SIM_E_UNDERFLOW if underflow_error else None)
    assert np.array_equal(c, ref.counts) and np.array_equal(p, ref.phi)
    assert np.array_equal(ctr, ref.counters)


def test_flow_without_events_and_one_node():
    w = W.sise3_national(N=500, T=20, n_events=0)
    _same(_run(w, "flow"), _run(w, "stream"))
    t = W.tiny_node(model=W.SISE, herd=40, infected=3, T=15,
                    params=dict(upsilon=0.05, gamma=0.1, alpha=1.0, beta=0.1, epsilon=1e-3))
    _same(_run(t, "flow"), _run(t, "stream"))


def test_flow_wait_runs_out_and_reports_timeout():
    import ctypes
    w = W.sise3_national(N=800, T=10, n_events=8000)
    s = B.Sim.from_workload(w)
    s.set_launch("flow")
    s.run(2)
    st = s.L.sim_debug_flow_stall(s.h, 3, ctypes.c_int64(20000))
    assert st == B.SIM_E_TIMEOUT
    # the device stays usable: reset and run the whole horizon
    s.reset()
    s.run(w.T)
    c, p, _ = s.state()
    s.close()
    ref = oracle.run(w)
    assert np.array_equal(c, ref.counts) and np.array_equal(p, ref.phi)

"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same
seeded inputs.  Counts, statistics and counters must be bit-identical; phi must
agree to 1e-12 relative (the kernels follow the oracle's IEEE operation order, so
it is expected to be identical too); per-node score terms to 1e-12 relative."""
import numpy as np
import pytest

import oracle
from paper_1502_02908_gb300 import binding as B
from paper_1502_02908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PHI_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()


def _assert_phi(got, ref):
    np.testing.assert_allclose(got, ref, rtol=PHI_RTOL, atol=0)


def _run_gpu(w, ndays=None, event_variant=None, **kw):
    s = B.Sim.from_workload(w, event_variant=event_variant, **kw)
    s.run(w.T if ndays is None else ndays)
    counts, phi, day = s.state()
    pi, pn, ctr = s.stats()
    sc = s.score() if kw.get("score") else None
    s.close()
    return counts, phi, pi, pn, ctr, sc


def _compare(w, ndays=None, replicates=None, global_events=False, **kw):
    nd = w.T if ndays is None else ndays
    counts, phi, pi, pn, ctr, sc = _run_gpu(w, ndays=nd, global_events=global_events, **kw)
    reps = list(range(w.R)) if replicates is None else replicates
    ref = oracle.run(w, ndays=nd, replicates=reps, **kw)
    assert np.array_equal(counts[reps], ref.counts)
    _assert_phi(phi[reps], ref.phi)
    assert np.array_equal(pi[reps][:, :nd], ref.prev_i)
    assert np.array_equal(pn[reps][:, :nd], ref.prev_n)
    assert np.array_equal(ctr[reps], ref.counters)
    if kw.get("score"):
        np.testing.assert_allclose(sc[reps], ref.score, rtol=PHI_RTOL, atol=1e-300)
    return ref


def test_neglog_kernel_bitexact():
    import torch
    rng = np.random.default_rng(11)
    js = rng.integers(0, 1 << 52, size=1 << 20, dtype=np.uint64)
    js[:6] = [0, 1, (1 << 52) - 1, (1 << 51), (1 << 51) - 1, 12345]
    jd = torch.from_numpy(js.view(np.int64)).cuda()
    out = torch.empty(js.size, dtype=torch.float64, device="cuda")
    B.debug_neglog(jd.data_ptr(), out.data_ptr(), js.size)
    got = out.cpu().numpy()
    L = oracle.lib()
    ref = np.array([L.orc_neglog(int(j)) for j in js[:20000]])
    assert np.array_equal(got[:20000], ref)
    # the rest against the float64 library log within the oracle's bound
    u = (2 * js.astype(np.float64) + 1) / 2.0 ** 53
    assert np.all(np.abs(got - (-np.log(u))) <= np.spacing(got) + 2.0 ** -55 + 4e-16 * np.abs(got))


def test_sise_plain_full_horizon_bitexact():
    _compare(W.sise_plain())


def test_sise_plain_phi_pre_event_bitexact():
    _compare(W.sise_plain(T=120), phi_pre_event=True)


def test_sise3_national_bitexact_120_days():
    w = W.sise3_national()
    w.T = 120
    _compare(w)


@pytest.mark.slow
def test_sise3_national_full_horizon_bitexact():
    _compare(W.sise3_national())


def test_replicates_with_own_parameters_bitexact():
    base = W.sise3_national(N=3000, T=60, n_events=150_000)
    w = W.sise3_batched(R=6, T=60, base=base)
    _compare(w)


def test_resume_equals_uninterrupted():
    w = W.sise_plain()
    full = B.Sim.from_workload(w)
    full.run(w.T)
    c_full, p_full, _ = full.state()
    a = B.Sim.from_workload(w)
    a.run(100)
    c, p, day = a.state()
    assert day == 100
    b = B.Sim.from_workload(w)
    b.set_state(c, p, day)
    b.run(w.T - 100)
    c2, p2, day2 = b.state()
    assert day2 == w.T
    assert np.array_equal(c2, c_full) and np.array_equal(p2, p_full)
    # and splitting one handle's run into several calls changes nothing
    a.run(50); a.run(w.T - 150)
    c3, p3, _ = a.state()
    assert np.array_equal(c3, c_full) and np.array_equal(p3, p_full)
    for s in (full, a, b):
        s.close()


def test_score_terms_match_oracle():
    w = W.sise_plain(N=300, T=60, n_events=3000, R=3)
    w.params.upsilon[:, 0] = [0.02, 0.03, 0.04]
    _compare(w, score=True)


def test_score_terms_sise3_match_oracle():
    base = W.sise3_national(N=500, T=40, n_events=20_000)
    _compare(base, score=True)


def test_underflow_error_policy_latches_and_skips():
    w = W.sise_plain(N=50, T=30, n_events=3000)
    ref = oracle.run(w, underflow_error=True)
    assert ref.counters[0, 3] > 0
    s = B.Sim.from_workload(w, underflow_error=True)
    s.run(w.T)
    with pytest.raises(B.SimError) as ei:
        s.sync()
    assert ei.value.status == B.SIM_E_UNDERFLOW
    counts, phi, _ = s.state()                      # latch was cleared by sync
    assert np.array_equal(counts, ref.counts)
    _, _, ctr = s.stats()
    assert np.array_equal(ctr, ref.counters)
    s.close()


def test_edge_cases_single_node_no_events_zero_days():
    w = W.tiny_node(model=W.SISE, herd=40, infected=3, T=20,
                    params=dict(upsilon=0.05, gamma=0.1, alpha=1.0, beta=0.1, epsilon=1e-3))
    _compare(w)
    s = B.Sim.from_workload(w)
    s.run(0)
    c, p, day = s.state()
    assert day == 0 and np.array_equal(c[0], w.u0)
    with pytest.raises(B.SimError) as ei:
        s.run(w.T + 1)
    assert ei.value.status == B.SIM_E_INVALID_ARG
    s.close()


def test_empty_herds_and_zero_rates():
    u0 = np.array([[0, 5, 0], [0, 0, 4]], np.int32)       # empty node, all-S node, all-I node
    w = W.tiny_node(model=W.SISE, herd=1, infected=0, copies=3, T=10,
                    params=dict(upsilon=0.2, gamma=0.3, alpha=0.5, beta=0.2, epsilon=0.0))
    w.u0 = u0
    _compare(w)


def test_global_event_variant_bitexact():
    w = W.sise3_national()
    w.T = 60
    _compare(w, global_events=True)


def test_day_too_large_for_shared_memory_falls_back():
    # 30,000 events on three days: ~10,000 per day needs more than 220 KB staged
    w = W.sise_plain(N=2000, T=3, n_events=30_000)
    _compare(w)


def test_integer_pipe_division_matches_hardware_divide():
    import torch
    g = torch.Generator(device="cpu").manual_seed(3)
    n = 1 << 22
    ex = torch.randint(1023 - 60, 1023 + 60, (n,), generator=g, dtype=torch.int64)
    ey = torch.randint(1023 - 60, 1023 + 60, (n,), generator=g, dtype=torch.int64)
    mx = torch.randint(0, 1 << 52, (n,), generator=g, dtype=torch.int64)
    my = torch.randint(0, 1 << 52, (n,), generator=g, dtype=torch.int64)
    my[::5] &= 0xF
    x = ((ex << 52) | mx).view(torch.float64).cuda()
    y = ((ey << 52) | my).view(torch.float64).cuda()
    out = torch.empty_like(x); ref = torch.empty_like(x)
    B.debug_div(x.data_ptr(), y.data_ptr(), out.data_ptr(), ref.data_ptr(), n, device=True)
    assert torch.equal(out.view(torch.int64), ref.view(torch.int64))
    assert torch.equal(out.view(torch.int64), (x / y).view(torch.int64))


@pytest.mark.parametrize("threshold", [0, 60])
def test_warp_per_node_path_bitexact_sise3(threshold):
    w = W.sise3_national(N=4000, T=90, n_events=80_000)
    s = B.Sim.from_workload(w)
    nwarp = s.tune(threshold)
    expect = 4000 if threshold == 0 else int((w.u0.sum(0) >= threshold).sum())
    assert nwarp == expect
    s.run(w.T)
    counts, phi, _ = s.state()
    pi, pn, ctr = s.stats()
    s.close()
    ref = oracle.run(w)
    assert np.array_equal(counts, ref.counts)
    _assert_phi(phi, ref.phi)
    assert np.array_equal(ctr, ref.counters) and np.array_equal(pi, ref.prev_i)


def test_warp_per_node_path_bitexact_sise_many_transitions():
    # prevalence near 1: ~19 transitions per node-day, long warp chains
    w = W.sise_plain(N=600, T=200, n_events=12_000)
    s = B.Sim.from_workload(w)
    assert s.tune(0) == 600
    s.run(w.T)
    counts, phi, _ = s.state()
    _, _, ctr = s.stats()
    s.close()
    ref = oracle.run(w)
    assert np.array_equal(counts, ref.counts)
    _assert_phi(phi, ref.phi)
    assert np.array_equal(ctr, ref.counters)


def test_reverse_score_sweep_matches_oracle_tangents():
    w = W.sise_plain(N=300, T=60, n_events=3000, R=3)
    s = B.Sim.from_workload(w, score_reverse=True)
    s.run(w.T)
    s.score_backward()
    sc = s.score()
    s.close()
    ref = oracle.run(w, score=True)
    # upsilon / gamma terms: same operation order, identical
    np.testing.assert_allclose(sc[:, :6], ref.score[:, :6], rtol=PHI_RTOL, atol=1e-300)
    # beta / alpha: reverse sweep vs forward tangents, a different summation order
    for k in (6, 7):
        scale = np.abs(ref.score[:, k]).max()
        assert np.max(np.abs(sc[:, k] - ref.score[:, k])) <= 1e-9 * scale


@pytest.mark.parametrize("variant,e1_source", [(0, "herd"), (2, "herd"), (0, "powerlaw"), (2, "powerlaw")])
def test_event_kernel_variants_bitexact(variant, e1_source):
    # 0: owner-computes kernel (default), 2: level-scheduled kernels; "powerlaw"
    # puts ~8% of all events on one small herd (a long chain every day)
    w = W.sise3_national(e1_source=e1_source)
    w.T = 90
    counts, phi, pi, pn, ctr, _ = _run_gpu(w, event_variant=variant)
    ref = oracle.run(w)
    assert np.array_equal(counts, ref.counts) and np.array_equal(ctr, ref.counters)
    _assert_phi(phi, ref.phi)


@pytest.mark.parametrize("launch", ["stream", "graph"])
def test_programmatic_overlap_on_and_off_bitexact(launch):
    # the day's kernels launched with programmatic dependent launch (default) or
    # in plain stream order give the oracle's result either way
    w = W.sise3_national(N=5000, T=60, n_events=60_000)
    ref = oracle.run(w)
    for on in (True, False):
        s = B.Sim.from_workload(w)
        s.set_overlap(on)
        s.set_launch(launch)
        s.run(w.T)
        counts, phi, _ = s.state()
        pi, pn, ctr = s.stats()
        s.close()
        assert np.array_equal(counts, ref.counts)
        _assert_phi(phi, ref.phi)
        assert np.array_equal(ctr, ref.counters) and np.array_equal(pi, ref.prev_i)


@pytest.mark.parametrize("launch,split", [("stream", False), ("graph", False), ("graph", True)])
def test_tracing_times_every_launch_and_keeps_results(launch, split):
    # sim_profile: one timed pair per kernel launch (graph mode: event-record
    # nodes inside a one-shot graph); traced runs give the untraced result
    w = W.sise3_national(N=3000, T=20, n_events=20_000)
    ref = oracle.run(w)
    s = B.Sim.from_workload(w)
    s.set_launch(launch)
    s.set_split(split)
    s.profile(True)
    s.run(w.T)
    prof = s.profile_read()
    s.profile(False)
    counts, _, _ = s.state()
    s.close()
    assert np.array_equal(counts, ref.counts)
    ms, n = prof["ssa"]
    # one launch per day, plus the touched herds' launch of each day after a day
    # with events (split day step)
    ev_days = set(np.asarray(w.events.day).tolist()) & set(range(w.T))
    assert n == w.T + (len([d for d in range(1, w.T) if d - 1 in ev_days]) if split else 0) and ms > 0
    ems, en = prof["events"]
    assert en == len(set(np.asarray(w.events.day).tolist()) & set(range(w.T))) and ems > 0
    assert prof["finalize"][1] == 1


@pytest.mark.parametrize("launch,threshold,R", [("stream", 400, 1), ("graph", 400, 1), ("graph", 0, 2),
                                                 ("graph", 1 << 30, 1)])
def test_split_day_step_bitexact(launch, threshold, R):
    # the next day's untouched herds on a second stream alongside the event step,
    # the touched ones after it, or one launch per day: the oracle's result both ways
    w = W.sise3_national(N=5000, T=45, n_events=60_000, R=R)
    ref = oracle.run(w)
    for split in (True, False):
        s = B.Sim.from_workload(w)
        s.tune(threshold)
        s.set_split(split)
        s.set_launch(launch)
        s.run(20)
        s.run(w.T - 20)                              # a second call starts with a full launch
        counts, phi, _ = s.state()
        pi, pn, ctr = s.stats()
        s.close()
        assert np.array_equal(counts, ref.counts)
        _assert_phi(phi, ref.phi)
        assert np.array_equal(ctr, ref.counters) and np.array_equal(pi, ref.prev_i) and np.array_equal(pn, ref.prev_n)


@pytest.mark.parametrize("underflow_error", [False, True])
def test_event_step_bitexact_with_clamps_and_error_policy(underflow_error):
    # "powerlaw" puts ~8 % of the events on one small herd: a long daily chain in
    # one component, many of its events clamped or, under the ERROR policy, skipped
    w = W.sise3_national(N=3000, T=40, n_events=60_000, e1_source="powerlaw")
    ref = oracle.run(w, underflow_error=underflow_error)
    assert ref.counters[0, 2 + int(underflow_error)] > 0
    s = B.Sim.from_workload(w, underflow_error=underflow_error)
    s.run(w.T)
    if underflow_error:
        with pytest.raises(B.SimError) as ei:
            s.sync()
        assert ei.value.status == B.SIM_E_UNDERFLOW
    counts, phi, _ = s.state()
    _, _, ctr = s.stats()
    s.close()
    assert np.array_equal(counts, ref.counts)
    _assert_phi(phi, ref.phi)
    assert np.array_equal(ctr, ref.counters)


@pytest.mark.parametrize("warp,group", [(400, 1 << 30), (1 << 30, 100), (1 << 30, 1 << 30)])
def test_synthetic_benchmark_bitexact(warp, group):
    # Sec. 4.2 benchmark shape (about S + I transitions per node-day), small
    w = W.synthetic_sis(N=64, T=12, S0=300, I0=300, rho=0.5, k=8)
    ref = oracle.run(w)
    s = B.Sim.from_workload(w)
    s.set_group_threshold(group)
    s.tune(warp)
    s.run(w.T)
    counts, phi, _ = s.state()
    pi, pn, ctr = s.stats()
    s.close()
    assert np.array_equal(counts, ref.counts)
    assert np.all(phi == 1.0)
    assert np.array_equal(ctr, ref.counters) and np.array_equal(pi, ref.prev_i)
    assert ctr[0, 0] > 64 * 12 * 500                  # SSA-dense


def test_state_in_caller_tensors_bitexact():
    # sim_create_on: the live counts and phi are the caller's tensors, updated in place;
    # they outlive the handle
    import torch
    w = W.sise3_national(N=2000, T=30, n_events=20_000, R=2)
    counts_t = torch.empty((w.R, w.nc, w.N), dtype=torch.int32, device="cuda")
    phi_t = torch.empty((w.R, w.N), dtype=torch.float64, device="cuda")
    s = B.Sim.from_workload(w, state=(counts_t, phi_t))
    s.run(w.T)
    s.sync()
    counts, phi, _ = s.state()
    s.close()
    torch.cuda.synchronize()
    ref = oracle.run(w)
    assert np.array_equal(counts_t.cpu().numpy(), ref.counts) and np.array_equal(counts, ref.counts)
    np.testing.assert_allclose(phi_t.cpu().numpy(), ref.phi, rtol=1e-12, atol=0)
    counts_t += 1                                   # still the caller's memory after sim_destroy
    assert int(counts_t.sum().item()) == int(ref.counts.sum()) + counts_t.numel()


def test_state_in_caller_tensors_rejects_host_memory():
    import torch
    w = W.sise_plain(N=64, T=5, n_events=0)
    with pytest.raises((B.SimError, ValueError)):
        B.Sim.from_workload(w, state=(torch.empty((1, 2, 64), dtype=torch.int32),
                                      torch.empty((1, 64), dtype=torch.float64)))

"""GPU: the general compartment model through the C ABI (gen_*) against the
general-model oracle, bit for bit on counts, continuous variables and counters:
the SIR example (frequency-dependent and mass-action), an SEIRS model with two
continuous variables under the three update sources, an Erlang-staged model with
11 transitions (the wide kernel), SISe3 in the general form on a national-shaped
network, the ERROR policy, CUDA-graph launches, split runs and state round
trips, one node, no events, no transitions."""
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


def _run(w, launch="stream", splits=None, warp=-1, group=-1, margin=16):
    s = B.GenSim.from_workload(w)
    s.set_launch(launch)
    s.set_warp_threshold(warp)
    s.set_group_threshold(group)
    s.set_clock_margin(margin)
    for nd in (splits or [w.T]):
        s.run(nd)
    counts, y, day = s.state()
    ctr = s.counters()
    s.close()
    assert day == sum(splits or [w.T])
    return counts, y, ctr


def _same(w, got, ref=None):
    ref = oracle.run_general(w) if ref is None else ref
    counts, y, ctr = got
    assert np.array_equal(counts, ref.counts)
    assert np.array_equal(y, ref.y)
    assert np.array_equal(ctr, ref.counters)
    return ref


@pytest.mark.parametrize("freq", [True, False])
def test_sir_bitexact(freq):
    w = W.sir_general(N=2000 + 37, T=60, n_events=12_000, R=2, freq=freq, beta=0.4 if freq else 0.004)
    w.rates[1] *= np.array([1.2, 0.9])
    ref = _same(w, _run(w))
    assert ref.counters[:, 0].min() > 10_000 and ref.counters[:, 2].sum() > 0


@pytest.mark.parametrize("source", [W.Y_POST_EVENT, W.Y_PRE_EVENT, W.Y_MIDPOINT])
def test_seirs_two_variables_bitexact(source):
    w = W.seirs_env(N=3000 + 5, T=60, n_events=30_000, R=2, y_source=source)
    ref = _same(w, _run(w))
    assert ref.counters[:, 0].min() > 100_000


# warp per node for every node (0), for none (2^30), for the largest (default)
@pytest.mark.parametrize("warp", [0, 1 << 30, -1, 100])
def test_warp_method_bitexact(warp):
    w = W.seirs_env(N=2000 + 11, T=40, n_events=20_000, R=2, y_source=W.Y_MIDPOINT)
    _same(w, _run(w, warp=warp))


# four nodes per warp (8-lane segments) for every node (group 0), for the middle
# tier, and mixed with a warp tier; the tail warp holds fewer than four nodes
@pytest.mark.parametrize("warp,group", [(1 << 30, 0), (1 << 30, 60), (300, 80), (-1, -1)])
def test_group_method_bitexact(warp, group):
    w = W.seirs_env(N=2000 + 7, T=40, n_events=20_000, R=2, y_source=W.Y_MIDPOINT)
    _same(w, _run(w, warp=warp, group=group))


@pytest.mark.parametrize("freq", [True, False])
def test_group_method_sir_runs_out_of_transitions(freq):
    w = W.sir_general(N=900 + 2, T=40, n_events=3000, R=1, freq=freq, beta=0.6 if freq else 0.01)
    _same(w, _run(w, warp=1 << 30, group=0))


@pytest.mark.parametrize("warp,group", [(0, 0), (1 << 30, 0), (-1, -1)])
def test_erlang_eleven_transitions_bitexact(warp, group):
    w = W.erlang_sis(N=1500 + 3, T=40, n_events=8000, R=2)
    w.rates[1] *= 1.5
    ref = _same(w, _run(w, warp=warp, group=group))
    assert ref.counters[:, 0].min() > 1_000_000


@pytest.mark.parametrize("freq,warp", [(True, 0), (False, 0), (True, 60)])
def test_sir_warp_bitexact(freq, warp):
    # SIR nodes run out of transitions (a0 = 0) inside a round
    w = W.sir_general(N=900, T=40, n_events=3000, R=1, freq=freq, beta=0.6 if freq else 0.01)
    _same(w, _run(w, warp=warp))


@pytest.mark.parametrize("warp", [-1, 0])
def test_sise3_general_national_shape_bitexact(warp):
    w = W.as_general(W.sise3_national(N=3000, T=60, n_events=40_000, R=2))
    w.rates[1] *= 1.4
    ref = _same(w, _run(w, warp=warp))
    assert ref.counters[:, 1].min() > 1000


def test_sise_general_matches_the_sise_kernels():
    # SISe in the general form is the same model as the SISe path
    w = W.sise_plain(N=1200, T=50, n_events=9000)
    s = B.Sim.from_workload(w)
    s.run(w.T)
    counts, phi, _ = s.state()
    _, _, ctr = s.stats()
    s.close()
    g_counts, g_y, g_ctr = _run(W.as_general(w))
    assert np.array_equal(counts, g_counts) and np.array_equal(phi, g_y[:, 0, :])
    assert np.array_equal(ctr, g_ctr)


def test_many_components_share_warps_bitexact():
    # about 20,000 components a day: past 8,192 warps the event step puts several
    # components on the lanes of one warp (each still alone on its nodes)
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    w = W.sir_general(N=40_000, T=4, n_events=160_000, R=1)
    ev = w.events
    for d in range(w.T):
        m = ev.day == d
        tr = m & (ev.kind == W.EXTERNAL)
        touched = np.unique(np.concatenate([ev.node[m], ev.dest[tr]]))
        _, label = connected_components(coo_matrix((np.ones(tr.sum()), (ev.node[tr], ev.dest[tr])), shape=(w.N, w.N)),
                                        directed=False)
        assert len(np.unique(label[touched])) > 2 * 8192
    ref = _same(w, _run(w))
    assert ref.counters[0, 1] == len(ev)


def test_graph_launch_and_split_runs_bitexact():
    w = W.seirs_env(N=1000, T=40, n_events=8000, R=1, y_source=W.Y_MIDPOINT)
    ref = oracle.run_general(w)
    _same(w, _run(w, launch="graph"), ref)
    _same(w, _run(w, splits=[7, 1, 20, 12]), ref)
    _same(w, _run(w, launch="graph", splits=[13, 27], warp=0), ref)


def test_set_state_round_trip_continues_bitexact():
    w = W.sir_general(N=700, T=30, n_events=3000, R=1)
    ref = oracle.run_general(w)
    s = B.GenSim.from_workload(w)
    s.run(12)
    c12, y12, _ = s.state()
    s.run(18)
    s.set_state(c12, y12, 12)
    s.run(18)
    counts, y, day = s.state()
    s.close()
    assert day == 30 and np.array_equal(counts, ref.counts)


def test_error_policy_latches_underflow():
    w = W.sir_general(N=300, T=20, n_events=4000, R=1)
    w.events.count[:] = w.events.count * 40
    w.underflow_error = True
    ref = oracle.run_general(w)
    assert ref.counters[0, 3] > 0
    s = B.GenSim.from_workload(w)
    s.run(w.T)
    with pytest.raises(B.SimError) as e:
        s.state()
    assert e.value.status == B.SIM_E_UNDERFLOW
    counts, y, _ = s.state()                       # latched once, then cleared
    assert np.array_equal(counts, ref.counts)
    assert np.array_equal(s.counters(), ref.counters)
    s.close()


def test_one_node_no_events_no_transitions():
    w = W.seirs_env(N=1, T=25, n_events=0, R=3)
    _same(w, _run(w))
    m = W.general_model(("A", "B"), [], variables=[(("A",), ("A", "B"))], selects=[("A",)])
    g = W.GeneralWorkload("static", m, 50, 10, 1, np.full((2, 50), 3, np.int32), np.zeros((1, 50)),
                          np.zeros((1, 0)), W._var_params(1, 1, (0.5,), (0.1,), (0.0,)), W.GeneralEvents.empty(), 3)
    _same(g, _run(g))


def test_replicate_base_shifts_streams():
    w = W.sir_general(N=400, T=20, n_events=2000, R=3)
    ref = oracle.run_general(w)
    s = B.GenSim(w.model, w.u0, w.y0, w.rates[1:], w.var_params[1:], w.T, seed=w.seed, replicate_base=1)
    s.load_events(w.events)
    s.run(w.T)
    counts, _, _ = s.state()
    s.close()
    assert np.array_equal(counts, ref.counts[1:])


def test_rejects_bad_events():
    w = W.sir_general(N=50, T=5, n_events=100)
    s = B.GenSim.from_workload(w, events=False)
    bad = w.events.take(np.arange(len(w.events)))
    bad.kind[0] = W.INTERNAL
    bad.select[0] = 0                   # mask {S, I, R} with offset +2: S -> R lands in the mask
    bad.shift[0] = 0
    with pytest.raises(B.SimError):
        s.load_events(bad)
    bad = w.events.take(np.arange(len(w.events)))
    bad.day[3] = -1
    with pytest.raises(B.SimError):
        s.load_events(bad)
    s.close()


def test_events_past_the_horizon_are_never_reached():
    w = W.seirs_env(N=800, T=40, n_events=6000, R=1)
    ref = oracle.run_general(w, ndays=25)
    s = B.GenSim.from_workload(w, max_days=25)     # days 25..39 stay unreached
    s.run(25)
    counts, y, _ = s.state()
    s.close()
    assert np.array_equal(counts, ref.counts) and np.array_equal(y, ref.y)


@pytest.mark.parametrize("warp,group", [(0, 0), (1 << 30, 0), (1 << 30, 1 << 30)])
def test_largest_model_bitexact(warp, group):
    # 16 compartments and 32 transitions (the limits): a ring C_i -> C_(i+1) at
    # k C_i and C_i -> C_(i+2) at k' C_i C_(i+1) / N, four continuous variables;
    # the stochastic step then needs more than 48 KB of shared memory per block
    comps = tuple(f"C{i}" for i in range(16))
    tr = []
    for i in range(16):
        tr.append(dict(change={comps[i]: -1, comps[(i + 1) % 16]: 1}, a=comps[i], cont=i % 4))
    for i in range(16):
        tr.append(dict(change={comps[i]: -1, comps[(i + 2) % 16]: 1}, a=comps[i], b=comps[(i + 1) % 16], pop=comps))
    variables = [((comps[q],), comps) for q in range(3)] + [((comps[3], comps[4]), ())]
    m = W.general_model(comps, tr, variables=variables, selects=[comps, comps[:4]], shifts=[{c: 4 for c in comps[:4]}],
                        y_source=W.Y_MIDPOINT)
    assert m.nc == 16 and m.nt == 32
    N, T, R = 700, 12, 2
    rng = np.random.default_rng(8)
    u0 = rng.integers(0, 40, size=(16, N)).astype(np.int32)
    y0 = rng.uniform(0.5, 1.5, size=(4, N))
    rates = rng.uniform(0.01, 0.2, size=(R, 32))
    vp = W._var_params(R, 4, (1.0, 0.5, 0.2, 0.01), (0.1, 0.2, 0.3, 0.05), (1e-3, 0.0, 0.0, 1e-4))
    ev = W._general_events(rng, N, T, 3000, [(0.3, W.EXIT, [0, 1], [-1]), (0.2, W.ENTER, [1], [-1, 0]),
                                             (0.2, W.INTERNAL, [1], [0]), (0.3, W.EXTERNAL, [0, 1], [-1, 0])])
    w = W.GeneralWorkload("ring16", m, N, T, R, u0, y0, rates, vp, ev, 21)
    ref = _same(w, _run(w, warp=warp, group=group))
    assert ref.counters[:, 0].min() > 10_000


def _exact_component_days(counts, N, R, seed=5):
    """A SIR workload whose day d holds exactly counts[d] transfer-graph components:
    each component is one event on a node of its own (exit of any animal, entry of
    susceptibles or vaccination), or a transfer a -> b followed by an exit at b."""
    w = W.sir_general(N=N, T=len(counts), n_events=0, R=R)
    rng = np.random.default_rng(seed)
    cols = [[] for _ in range(7)]
    for d, c in enumerate(counts):
        nodes = rng.permutation(N)[:2 * c]
        for i in range(c):
            a, b = int(nodes[2 * i]), int(nodes[2 * i + 1])
            n = int(rng.integers(1, 6))
            kind = int(rng.integers(0, 4))
            if kind == 3:
                rows = [(W.EXTERNAL, a, b, n, 0, -1), (W.EXIT, b, -1, n, 0, -1)]
            else:
                rows = [((W.EXIT, W.ENTER, W.INTERNAL)[kind], a, -1, n, (0, 1, 1)[kind], (-1, -1, 0)[kind])]
            for kd, nd, ds, ct, sel, sh in rows:
                for col, v in zip(cols, (d, kd, nd, ds, ct, sel, sh)):
                    col.append(v)
    w.events = W.GeneralEvents(*(np.asarray(c, np.int32) for c in cols))
    return w


@pytest.mark.parametrize("counts", [(8193, 8250, 8300, 8192, 8191), (1, 17, 31, 32, 33, 95)])
def test_component_counts_at_the_warp_deal_edges_bitexact(counts):
    # just above 8,192 components (the lane-major deal puts a second component on a
    # warp's lanes), counts that are not multiples of 32, and fewer than one warp's
    # worth; two replicates, so the event grid's second dimension varies
    w = _exact_component_days(counts, N=20_000, R=2)
    ref = _same(w, _run(w))
    assert ref.counters[:, 1].sum() == 2 * len(w.events)
    _same(w, _run(w, launch="graph"), ref)


@pytest.mark.parametrize("margin", [16, 12, 6, 1, 0])
def test_binary32_clock_bitexact_at_every_margin(margin):
    # the one-per-thread nodes' binary32 clock and selections against the general
    # oracle: from the tightest safe margin (2^-16) to none (0: exact only); SEIRS
    # with two continuous variables and frequency-dependent rates, one per thread
    w = W.seirs_env(N=1200, T=40, n_events=10_000, R=2)
    ref = oracle.run_general(w)
    _same(w, _run(w, warp=1 << 30, group=1 << 30, margin=margin), ref)


@pytest.mark.parametrize("freq", [True, False])
def test_binary32_clock_sir_and_erlang(freq):
    w = W.sir_general(N=1500, T=50, n_events=6000, R=2, freq=freq)
    _same(w, _run(w, warp=1 << 30, group=1 << 30))
    e = W.erlang_sis(N=900, T=30, n_events=4000, R=2)
    _same(e, _run(e, warp=1 << 30, group=1 << 30))


def test_binary32_clock_falls_back_outside_its_bounds():
    # a rate constant beyond 2^30 and a node of more than 2^21 animals take the
    # exact method; the results stay the specification's
    w = W.sir_general(N=300, T=12, n_events=1200, R=2, freq=True, beta=0.4, gamma=0.1)
    w.rates = w.rates.copy()
    w.rates[1, 1] = 3.0e9                            # replicate 1: recovery constant above 2^30
    w.u0 = w.u0.copy()
    w.u0[0, 7] = 3_000_000                           # node 7: above 2^21 animals
    _same(w, _run(w, warp=1 << 30, group=1 << 30))


def test_binary32_clock_national_sise3_general_bitexact():
    w = W.as_general(W.sise3_national(N=6000, T=60, n_events=180_000))
    ref = oracle.run_general(w)
    _same(w, _run(w, launch="graph", warp=600, group=300), ref)
    _same(w, _run(w, launch="graph", warp=1 << 30, group=1 << 30, margin=3), ref)


@pytest.mark.parametrize("margin", [16, 6, 1])
@pytest.mark.parametrize("tier", ["warp", "group"])
def test_binary32_segment_methods_bitexact_at_margins(margin, tier):
    # the warp (32-lane) and group (8-lane) methods' binary32 choices and Q62
    # clock scan against the general oracle, every node on the one tier; smaller
    # margins hand more node-days back to the binary64 segment method
    w = W.seirs_env(N=600, T=30, n_events=5000, R=2)
    ref = oracle.run_general(w)
    kw = dict(warp=0) if tier == "warp" else dict(warp=1 << 30, group=0)
    _same(w, _run(w, margin=margin, **kw), ref)


@pytest.mark.parametrize("tier", ["warp", "group"])
def test_binary32_segment_methods_fall_back_outside_bounds(tier):
    # a rate constant beyond 2^30 (replicate 1) and a node of more than 2^21
    # animals: those segments run the binary64 method while the others of their
    # warp keep the binary32 one
    w = W.sir_general(N=300, T=12, n_events=1200, R=2, freq=True, beta=0.4, gamma=0.1)
    w.rates = w.rates.copy()
    w.rates[1, 1] = 3.0e9
    w.u0 = w.u0.copy()
    w.u0[0, 7] = 3_000_000
    kw = dict(warp=0) if tier == "warp" else dict(warp=1 << 30, group=0)
    _same(w, _run(w, **kw))

"""The node-sharded single replicate on the GPU: several ranks' handles in one
process on one device, exchanging the day's touched herds through the C ABI
(sim_pack_touched / sim_unpack_touched) between the two halves of each day.  The
ranks' own nodes joined together equal a single handle's run and the oracle bit
for bit; statistics add up over the ranks."""
import numpy as np
import pytest

import oracle
from paper_1502_02908_gb300 import binding as B
from paper_1502_02908_gb300 import sharded
from paper_1502_02908_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()


def _single(w):
    s = B.Sim.from_workload(w)
    s.run(w.T)
    c, p, _ = s.state()
    pi, pn, ctr = s.stats()
    s.close()
    return c, p, pi, pn, ctr


def _sharded(w, world, warp=-1, group=-1):
    engines = [sharded.EngineShard(w, k, world) for k in range(world)]
    for e in engines:
        e.sim.set_group_threshold(group)
        e.sim.tune(warp)
    sharded.run_in_process(engines, w.T)
    parts = [e.own_state() for e in engines]
    stats = [e.sim.stats() for e in engines]
    for e in engines:
        e.close()
    counts, phi = sharded.merge_own(parts, engines[0].bounds, w.R, w.nc, w.N)
    pi = sum(s[0] for s in stats)
    pn = sum(s[1] for s in stats)
    trans = sum(s[2][:, 0] for s in stats)
    return counts, phi, pi, pn, trans, stats[0][2]


@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_national_shape_equals_single_handle_and_oracle(world):
    w = W.sise3_national(N=4000, T=40, n_events=120_000)
    c, p, pi, pn, ctr = _single(w)
    sc, sp, spi, spn, strans, sctr0 = _sharded(w, world)
    assert np.array_equal(sc, c) and np.array_equal(sp, p)
    assert np.array_equal(spi, pi) and np.array_equal(spn, pn)
    assert np.array_equal(strans, ctr[:, 0]) and np.array_equal(sctr0[:, 1:], ctr[:, 1:])
    if world == 2:
        ref = oracle.run(w)
        assert np.array_equal(sc, ref.counts) and np.array_equal(sp, ref.phi)


def test_sharded_warp_and_group_paths_and_more_ranks_than_some_days_touch():
    # warp- and group-path herds on every rank; seven ranks on a small network
    w = W.sise3_national(N=900, T=30, n_events=20_000)
    c, p, pi, pn, ctr = _single(w)
    sc, sp, spi, spn, strans, _ = _sharded(w, 7, warp=400, group=100)
    assert np.array_equal(sc, c) and np.array_equal(sp, p) and np.array_equal(spi, pi)


def test_sharded_with_empty_ranges_and_replicates():
    # more ranks than nodes (some ranges empty), two replicates, SISe
    w = W.sise_plain(N=5, T=20, n_events=300, R=2)
    c, p, pi, pn, ctr = _single(w)
    sc, sp, spi, spn, strans, _ = _sharded(w, 8)
    assert np.array_equal(sc, c) and np.array_equal(sp, p) and np.array_equal(spi, pi)


def test_day_halves_without_exchange_equal_whole_days_and_guard_the_state():
    w = W.sise_plain(N=400, T=25, n_events=4000)
    c, p, *_ = _single(w)
    s = B.Sim.from_workload(w)
    for d in range(w.T):
        s.run_day_stochastic()
        if d == 3:
            with pytest.raises(B.SimError) as ei:
                s.state()
            assert ei.value.status == B.SIM_E_STATE
            with pytest.raises(B.SimError):
                s.run(1)
        s.run_day_events()
    gc, gp, day = s.state()
    s.close()
    assert day == w.T and np.array_equal(gc, c) and np.array_equal(gp, p)


def test_touched_nodes_are_those_the_days_events_name():
    w = W.sise3_national(N=700, T=10, n_events=5000)
    s = B.Sim.from_workload(w)
    for d in range(w.T):
        m = w.events.day == d
        want = np.unique(np.concatenate([w.events.node[m], w.events.dest[m & (w.events.kind == W.EXTERNAL)]]))
        got = s.touched_nodes(d)
        assert s.touched_count(d) == got.size and np.array_equal(np.sort(got), want)
    assert s.touched_count(-1) == -1 and s.touched_count(w.T) == -1
    s.close()

"""GPU: the speculative binary32 clock of the stochastic step.  Every node-day
first runs with a binary32 clock accumulated in Q62 fixed point and decides
stop/continue only outside a margin around the day's end; inside it, the
node-day reruns with the specification's binary64 arithmetic.  Whatever the
margin (including margins so wide that most node-days rerun, and 0 = always
exact), results must equal the oracle's bit for bit, on both the per-thread and
the warp-per-node method."""
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


def test_neglog_f32_within_relative_bound():
    # the clock's error analysis assumes |E~ - E| <= 16 * 2^-24 * E
    import torch
    rng = np.random.default_rng(21)
    js = rng.integers(0, 1 << 52, size=1 << 20, dtype=np.uint64)
    # edges: smallest and largest u, both sides of u = 1/2, u near 1 (E tiny)
    edge = [0, 1, 2, (1 << 51) - 2, (1 << 51) - 1, 1 << 51, (1 << 51) + 1, (1 << 52) - 1, (1 << 52) - 2,
            (1 << 52) - 1000, (1 << 52) - (1 << 30)]
    js[:len(edge)] = edge
    # long runs of ones/zeros in the bits below the 24 kept ones; both sides of
    # the 1/sqrt2 split of the two formulas
    js[len(edge):len(edge) + 52] = [((1 << 52) - 1) >> s for s in range(52)]
    split = 3184525836262886
    js[100:4100] = np.arange(split - 2000, split + 2000, dtype=np.uint64)
    jd = torch.from_numpy(js.view(np.int64)).cuda()
    out = torch.empty(js.size, dtype=torch.float32, device="cuda")
    B.debug_neglog_f32(jd.data_ptr(), out.data_ptr(), js.size)
    got = out.cpu().numpy().astype(np.float64)
    L = oracle.lib()
    ref = np.array([L.orc_neglog(int(j)) for j in js[:100_000]])
    assert np.all(np.abs(got[:100_000] - ref) <= 2.0 ** -20 * ref)
    u = (2 * js.astype(np.float64) + 1) / 2.0 ** 53      # exact
    e64 = np.where(u < 0.5, -np.log(u), -np.log1p(-((2.0 ** 53 - 2 * js.astype(np.float64) - 1) / 2.0 ** 53)))
    assert np.all(np.abs(got - e64) <= 2.0 ** -20 * e64)


_REF = {}


def _oracle(key, w):
    if key not in _REF:
        _REF[key] = oracle.run(w)
    return _REF[key]


@pytest.mark.parametrize("threshold", [0, 1 << 30])     # every node one per warp / one per thread
@pytest.mark.parametrize("k", [17, 6, 1, 0])
def test_clock_margin_bitexact_sise3(threshold, k):
    w = W.sise3_national(N=3000, T=60, n_events=40_000)
    s = B.Sim.from_workload(w)
    s.tune(threshold)
    s.set_clock_margin(k)
    s.run(w.T)
    counts, phi, _ = s.state()
    pi, pn, ctr = s.stats()
    s.close()
    ref = _oracle("sise3", w)
    assert np.array_equal(counts, ref.counts)
    np.testing.assert_allclose(phi, ref.phi, rtol=1e-12, atol=0)
    assert np.array_equal(ctr, ref.counters) and np.array_equal(pi, ref.prev_i) and np.array_equal(pn, ref.prev_n)


@pytest.mark.parametrize("threshold", [0, 1 << 30])
@pytest.mark.parametrize("k", [17, 1])
def test_clock_margin_bitexact_sise_many_transitions(threshold, k):
    # prevalence near 1: ~19 transitions per node-day, so many decisions fall
    # inside a wide margin
    w = W.sise_plain(N=600, T=120, n_events=8_000)
    s = B.Sim.from_workload(w)
    s.tune(threshold)
    s.set_clock_margin(k)
    s.run(w.T)
    counts, phi, _ = s.state()
    _, _, ctr = s.stats()
    s.close()
    ref = _oracle("sise", w)
    assert np.array_equal(counts, ref.counts)
    np.testing.assert_allclose(phi, ref.phi, rtol=1e-12, atol=0)
    assert np.array_equal(ctr, ref.counters)


def test_clock_margin_rejects_unsafe_values():
    w = W.sise_plain(N=50, T=5, n_events=0)
    s = B.Sim.from_workload(w)
    for bad in (-1, 18, 40):
        with pytest.raises(B.SimError):
            s.set_clock_margin(bad)
    s.close()


@pytest.mark.parametrize("warp,group", [(1 << 30, 0), (400, 50), (1 << 30, 150)])
@pytest.mark.parametrize("k", [17, 1])
def test_group_path_bitexact_sise3(warp, group, k):
    # herds below the warp threshold and at or above the group threshold run four
    # to a warp, eight lanes each; group 0: every node in a group
    w = W.sise3_national(N=3000, T=60, n_events=40_000)
    s = B.Sim.from_workload(w)
    s.set_group_threshold(group)
    s.tune(warp)
    s.set_clock_margin(k)
    s.run(w.T)
    counts, phi, _ = s.state()
    pi, pn, ctr = s.stats()
    s.close()
    ref = _oracle("sise3", w)
    assert np.array_equal(counts, ref.counts)
    np.testing.assert_allclose(phi, ref.phi, rtol=1e-12, atol=0)
    assert np.array_equal(ctr, ref.counters) and np.array_equal(pi, ref.prev_i) and np.array_equal(pn, ref.prev_n)


@pytest.mark.parametrize("k", [17, 1])
def test_group_path_bitexact_sise_many_transitions(k):
    w = W.sise_plain(N=600, T=120, n_events=8_000)
    s = B.Sim.from_workload(w)
    s.set_group_threshold(0)
    s.tune(1 << 30)
    s.set_clock_margin(k)
    s.run(w.T)
    counts, phi, _ = s.state()
    _, _, ctr = s.stats()
    s.close()
    ref = _oracle("sise", w)
    assert np.array_equal(counts, ref.counts)
    np.testing.assert_allclose(phi, ref.phi, rtol=1e-12, atol=0)
    assert np.array_equal(ctr, ref.counters)

"""The persistent work-stealing batch kernel: results identical to running each
simulation alone (and to the oracle), score mode inside a batch, and the failure
path of its bounded dependency waits."""
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


def _state(s):
    c, p, d = s.state()
    pi, pn, ctr = s.stats()
    return c, p, d, pi, pn, ctr


def test_uneven_batch_equals_individual_runs_and_oracle():
    ws = W.uneven_batch(n_inst=12, N_lo=50, N_hi=3000, T_lo=20, T_hi=120, seed=7)
    ws[0].R = 3
    ws[0].params = W.Params.broadcast(3, ws[0].params.upsilon[0, :1], ws[0].params.gamma[0, :1],
                                      ws[0].params.alpha[0], ws[0].params.beta[0, 0], 1e-6)
    batch = [B.Sim.from_workload(w) for w in ws]
    batch[1].tune(0)                               # one instance on the warp-per-node path
    B.run_batch(batch)
    for w, s in zip(ws, batch):
        alone = B.Sim.from_workload(w)
        alone.run(w.T)
        a, b = _state(s), _state(alone)
        assert b[2] == w.T and a[2] == w.T
        for x, y in zip(a, b):
            assert np.array_equal(np.asarray(x), np.asarray(y)), w.name
        alone.close()
    for i in (0, 1, 5):
        ref = oracle.run(ws[i])
        c, p, _, pi, pn, ctr = _state(batch[i])
        assert np.array_equal(c, ref.counts) and np.array_equal(ctr, ref.counters)
        np.testing.assert_allclose(p, ref.phi, rtol=1e-12, atol=0)
    for s in batch:
        s.close()


def test_batch_partial_horizons_and_resume():
    ws = W.uneven_batch(n_inst=4, N_lo=100, N_hi=800, T_lo=30, T_hi=60, seed=9)
    sims = [B.Sim.from_workload(w) for w in ws]
    B.run_batch(sims, until=[10, 0, 17, 5])
    B.run_batch(sims)                              # the rest of every horizon
    for w, s in zip(ws, sims):
        ref = oracle.run(w)
        c, p, d = s.state()
        assert d == w.T and np.array_equal(c, ref.counts)
        s.close()


def test_batch_with_score_mode_matches_plain_run():
    w = W.sise_plain(N=300, T=40, n_events=3000, R=4)
    a = B.Sim.from_workload(w, score=True)
    b = B.Sim.from_workload(w, score=True)
    B.run_batch([a])
    b.run(w.T)
    assert np.array_equal(a.score(), b.score())
    assert np.array_equal(a.state()[0], b.state()[0])
    a.close(); b.close()


def test_batch_wait_runs_out_and_reports_timeout():
    w = W.sise_plain(N=200, T=20, n_events=1000)
    s = B.Sim.from_workload(w)
    s.run(1)
    st = s.L.sim_debug_batch_stall(s.h, 5, 20_000)
    assert st == B.SIM_E_TIMEOUT
    # the context is still usable: a fresh run matches the oracle
    t = B.Sim.from_workload(w)
    t.run(w.T)
    assert np.array_equal(t.state()[0], oracle.run(w).counts)
    s.close(); t.close()


def test_graph_and_persistent_launch_modes_match_stream_launches():
    w = W.sise3_national(N=3000, T=40, n_events=60_000)
    out = {}
    for mode in ("stream", "graph", "persistent"):
        s = B.Sim.from_workload(w)
        s.set_launch(mode)
        s.run(15); s.run(25)                       # two calls: two graphs / two batch launches
        out[mode] = _state(s)
        s.reset()                                  # replaying a cached graph after a reset
        s.run(15); s.run(25)
        again = _state(s)
        for x, y in zip(out[mode], again):
            assert np.array_equal(np.asarray(x), np.asarray(y))
        s.close()
    for mode in ("graph", "persistent"):
        for x, y in zip(out[mode], out["stream"]):
            assert np.array_equal(np.asarray(x), np.asarray(y)), mode


def test_autotuner_keeps_results_and_picks_a_setting():
    from paper_1502_02908_gb300 import autotune
    w = W.sise3_national(N=2000, T=30, n_events=40_000)
    best, table = autotune.autotune(w, days=20, thresholds=(1 << 30, 200), repeats=1, groups=(1 << 30, 100))
    assert len(table) == 12 and best["launch"] in autotune.LAUNCH_MODES
    assert best["group_threshold"] in (1 << 30, 100)


def test_batch_and_graph_on_caller_tensors():
    # handles whose state lives in caller tensors (sim_create_on): the persistent
    # batch kernel and the CUDA-graph day loop update the tensors in place
    import torch
    ws = W.uneven_batch(n_inst=5, N_lo=100, N_hi=2000, T_lo=20, T_hi=70, seed=11)
    tensors = [(torch.zeros((w.R, w.nc, w.N), dtype=torch.int32, device="cuda"),
                torch.zeros((w.R, w.N), dtype=torch.float64, device="cuda")) for w in ws]
    sims = [B.Sim.from_workload(w, state=t) for w, t in zip(ws, tensors)]
    B.run_batch(sims[:3])
    for s, w in zip(sims[3:], ws[3:]):
        s.set_launch("graph")
        s.run(w.T // 2)
        s.run(w.T - w.T // 2)
    for s in sims:
        s.sync()
    torch.cuda.synchronize()
    for w, (ct, pt), s in zip(ws, tensors, sims):
        ref = oracle.run(w)
        assert np.array_equal(ct.cpu().numpy(), ref.counts), w.name
        np.testing.assert_allclose(pt.cpu().numpy(), ref.phi, rtol=1e-12, atol=0)
        s.close()


@pytest.mark.parametrize("shape", B.BATCH_SHAPES)
def test_batch_shapes_agree_and_match_oracle(shape):
    # 12,000 events a day on 3,000 herds: the staged event step of a day needs
    # more shared memory than one of two (or four) blocks an SM may take, so those
    # shapes run such days through the global-memory variant
    big = W.sise3_national(N=3000, T=16, n_events=192_000)
    ws = [big] + W.uneven_batch(n_inst=5, N_lo=50, N_hi=2000, T_lo=10, T_hi=40, seed=13)
    try:
        B.batch_shape(*shape)
        sims = [B.Sim.from_workload(w) for w in ws]
        B.run_batch(sims)
    finally:
        B.batch_shape(*B.BATCH_SHAPES[0])
    for w, s in zip(ws, sims):
        ref = oracle.run(w)
        c, p, d, pi, pn, ctr = _state(s)
        assert d == w.T and np.array_equal(c, ref.counts), (shape, w.name)
        assert np.array_equal(ctr, ref.counters), (shape, w.name)
        np.testing.assert_allclose(p, ref.phi, rtol=1e-12, atol=0)
        s.close()


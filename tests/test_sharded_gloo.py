"""The node-sharded single replicate on several ranks (gloo, CPU): each rank runs
the day loop and exchange of ``sharded.run_days`` with the CPU oracle standing in
for its GPU engine (stochastic step and phi update of its own nodes, the whole
event list on every rank), and the ranks' own nodes joined together equal one
oracle run of the whole network bit for bit."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1502_02908_gb300 import sharded
from paper_1502_02908_gb300 import workloads as W


class OracleShard:
    """One rank of the sharded day loop, computed by the oracle's day steps."""

    def __init__(self, w, rank, world):
        self.w, self.rank = w, rank
        self.bounds = sharded.node_bounds(w.N, world)
        self.lo, self.hi = int(self.bounds[rank]), int(self.bounds[rank + 1])
        self.counts = np.ascontiguousarray(w.u0, np.int32).copy()
        self.phi = np.ascontiguousarray(w.phi0, np.float64).copy()
        self.day = 0
        self.transitions = 0
        self.order = np.argsort(w.events.day, kind="stable")          # day-stable positions
        self.first = np.searchsorted(w.events.day[self.order], np.arange(w.T + 1))

    def _today(self):
        s0, s1 = self.first[self.day], self.first[self.day + 1]
        return np.arange(s0, s1), self.w.events.select(self.order[s0:s1])

    def _touched(self):
        _, ev = self._today()
        return np.unique(np.concatenate([ev.node, ev.dest[ev.kind == W.EXTERNAL]]))

    def stochastic(self):
        self.transitions += oracle.ssa_nodes(self.w, self.counts, self.phi, self.day, self.lo, self.hi)

    def touched_count(self):
        return int(self._touched().size)

    def pack(self, n):
        return np.ascontiguousarray(self.counts[:, self._touched()]).ravel()

    def unpack(self, gathered):
        t = self._touched()
        g = np.asarray(gathered).reshape(len(self.bounds) - 1, self.w.nc, t.size)
        owner = np.searchsorted(self.bounds, t, side="right") - 1
        self.counts[:, t] = g[owner, :, np.arange(t.size)].T

    def events(self):
        pos, ev = self._today()
        oracle.apply_events(self.w, self.counts, pos, ev)
        oracle.phi_nodes(self.w, self.counts, self.phi, self.day, self.lo, self.hi)
        self.day += 1


def _workloads():
    return [W.sise3_national(N=500, T=25, n_events=8000), W.sise_plain(N=300, T=30, n_events=3000)]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = []
    for w in _workloads():
        e = OracleShard(w, rank, world)
        sharded.run_days(e, w.T, sharded.allgather_exchange())
        res.append((e.counts[:, e.lo:e.hi].tolist(), e.phi[e.lo:e.hi].tolist(), int(e.transitions)))
    out[rank] = res
    dist.destroy_process_group()


def _check(w, parts, bounds):
    ref = oracle.run(w)
    counts, phi = sharded.merge_own([(np.array(c)[None], np.array(p)[None]) for c, p, _ in parts], bounds,
                                    1, w.nc, w.N)
    assert np.array_equal(counts[0], ref.counts[0])
    assert np.array_equal(phi[0], ref.phi[0])
    assert sum(t for _, _, t in parts) == ref.counters[0, 0]


def test_two_gloo_ranks_equal_one_oracle_run():
    world = 2
    port = 29600 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(k, world, port, out)) for k in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = [out[k] for k in range(world)]
    for i, w in enumerate(_workloads()):
        _check(w, [res[k][i] for k in range(world)], sharded.node_bounds(w.N, world))


@pytest.mark.parametrize("world", [1, 3, 5])
def test_ranks_in_one_process_equal_one_oracle_run(world):
    # the same exchange joined in one process, including more ranks than a
    # day's touched herds would need and uneven node ranges
    w = W.sise3_national(N=203, T=12, n_events=3000)
    engines = [OracleShard(w, k, world) for k in range(world)]
    sharded.run_in_process(engines, w.T)
    parts = [(e.counts[:, e.lo:e.hi], e.phi[e.lo:e.hi], e.transitions) for e in engines]
    _check(w, parts, engines[0].bounds)


def test_node_bounds_cover_the_nodes():
    for N, world in ((10, 3), (7, 8), (37_000, 4)):
        b = sharded.node_bounds(N, world)
        assert b[0] == 0 and b[-1] == N and np.all(np.diff(b) >= 0) and b.size == world + 1

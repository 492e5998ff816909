"""Node-sharded single replicate over several GPUs (one process per GPU).

The paper splits the nodes of one trajectory over workers and exchanges the
events that cross their boundaries once per day (Sec. 3.4, Alg. 2), and names
larger machines as the way forward (Sec. 5).  Here each rank owns a contiguous
node range and holds the whole state.  A day is:

1. the stochastic step of the rank's own nodes (Eq. (numstep3));
2. the exchange: every rank packs the post-stochastic-step counts of the herds
   the day's events touch, the packs are gathered in rank order, and every rank
   takes each touched herd's counts from its owner's pack;
3. the whole day's event list on every rank (Eq. (numstep4)); the event step is
   bound by its longest dependency chain, not by its size, so running it on every
   rank costs no more than running a share of it;
4. the phi update and statistics of the own nodes (Eq. (numstep5)).

The random numbers are keyed by node, day and event position, so each rank's own
nodes end every day exactly as in a single-GPU run.  The day loop is written
against a small engine interface (stochastic / touched_count / pack / unpack /
events) so that the exchange logic is the same for the GPU engine and for the
CPU oracle standing in for it in multi-process tests.
"""
from __future__ import annotations

import numpy as np

from . import binding as B
from . import replicas
from . import workloads as W


def node_bounds(N: int, world: int) -> np.ndarray:
    """[world + 1] boundaries of the ranks' contiguous node ranges."""
    return np.array([replicas.shard(N, world, k)[0] for k in range(world)] + [N], np.int32)


class EngineShard:
    """One rank's part on the GPU: a handle over the whole state whose stochastic
    step, phi update and statistics cover nodes [lo, hi) (sim_shard)."""

    def __init__(self, w: W.Workload, rank: int, world: int, **sim_kw):
        import torch
        self.w, self.rank, self.world = w, rank, world
        self.bounds = node_bounds(w.N, world)
        self.lo, self.hi = int(self.bounds[rank]), int(self.bounds[rank + 1])
        self.sim = B.Sim(w.model, w.u0, w.phi0, w.params, w.T, seed=w.seed, **sim_kw)
        if len(w.events):
            self.sim.load_events(w.events)
        self.sim.shard(self.lo, self.hi)
        self.day = 0
        self.planes = w.R * w.nc
        self._torch = torch

    def stochastic(self):
        self.sim.run_day_stochastic()

    def touched_count(self):
        return self.sim.touched_count(self.day)

    def pack(self, n):
        buf = self._torch.empty(self.planes * n, dtype=self._torch.int32, device="cuda")
        self.sim.pack_touched(buf.data_ptr())
        return buf

    def unpack(self, gathered):
        self.sim.unpack_touched(gathered.data_ptr(), self.bounds)

    def events(self):
        self.sim.run_day_events()
        self.day += 1

    def own_state(self):
        """(counts [R][Nc][hi-lo], phi [R][hi-lo]) of the own nodes, host arrays."""
        c, p, _ = self.sim.state()
        return c[:, :, self.lo:self.hi], p[:, self.lo:self.hi]

    def close(self):
        self.sim.close()


def run_days(engine, days: int, exchange):
    """Runs `days` days of one rank; exchange(pack) returns the ranks' packs
    gathered back to back in rank order."""
    for _ in range(days):
        engine.stochastic()
        n = engine.touched_count()
        if n > 0:
            engine.unpack(exchange(engine.pack(n)))
        engine.events()


def allgather_exchange(group=None):
    """exchange() over torch.distributed: an all-gather of the packs in rank order
    (NCCL on device buffers; gloo through host copies)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    nccl = dist.get_backend(group) == "nccl"

    def exchange(buf):
        if nccl:
            out = torch.empty(world * buf.numel(), dtype=buf.dtype, device=buf.device)
            dist.all_gather_into_tensor(out, buf, group=group)
            return out
        host = torch.as_tensor(buf).cpu() if not isinstance(buf, np.ndarray) else torch.from_numpy(buf)
        parts = [torch.empty_like(host) for _ in range(world)]
        dist.all_gather(parts, host, group=group)
        out = torch.cat(parts)
        return out if isinstance(buf, np.ndarray) else out.to(buf.device)

    return exchange


def run_in_process(engines, days: int):
    """Every rank's engine in one process (one device): the same day, the packs
    joined in rank order on the host side of the call.  Used to check the sharded
    path on a single GPU; no kernel of one engine waits for another's."""
    for _ in range(days):
        for e in engines:
            e.stochastic()
        n = engines[0].touched_count()
        if n > 0:
            packs = [e.pack(n) for e in engines]
            if isinstance(packs[0], np.ndarray):
                gathered = np.concatenate(packs)
            else:
                import torch
                gathered = torch.cat(packs)
            for e in engines:
                e.unpack(gathered)
        for e in engines:
            e.events()


def merge_own(parts, bounds, R, nc, N):
    """Joins the ranks' own-node states [(counts, phi), ...] into whole arrays."""
    counts = np.zeros((R, nc, N), np.int32)
    phi = np.zeros((R, N), np.float64)
    for k, (c, p) in enumerate(parts):
        counts[:, :, bounds[k]:bounds[k + 1]] = c
        phi[:, bounds[k]:bounds[k + 1]] = p
    return counts, phi

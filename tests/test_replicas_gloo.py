"""Replicas on several ranks (world size 2, gloo, CPU): sharding of replicate
ranges and the rank-ordered reduction of gradient-moment sums give exactly the
single-process result.  Each rank evaluates its replicates with the CPU oracle,
which stands in for the per-GPU engine here (the host logic is what is tested)."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1502_02908_gb300 import replicas
from paper_1502_02908_gb300 import workloads as W


def _moments(w, r0, r1):
    """Per-replicate final prevalence and score sums -> the 42 moment sums, in
    replicate order (same definition as the library's moment kernel)."""
    import oracle
    res = oracle.run(w, replicates=range(r0, r1), score=True)
    m = np.zeros(42)
    for i in range(r1 - r0):
        f = res.prev_i[i, -1] / res.prev_n[i, -1]
        s = res.score[i].sum(axis=1)
        m[0] += f; m[1] += f * f
        for k in range(8):
            m[2 + 4 * k] += s[k]; m[3 + 4 * k] += s[k] ** 2
            m[4 + 4 * k] += f * s[k]; m[5 + 4 * k] += (f * s[k]) ** 2
            m[34 + k] += f * s[k] ** 2
    return m


def _workload():
    return W.sise_plain(N=40, T=15, n_events=200, R=6)


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _workload()
    r0, r1 = replicas.shard(w.R, world, rank)
    m = replicas.allreduce_moments(_moments(w, r0, r1))
    out[rank] = m.tolist()
    dist.destroy_process_group()


def test_shards_cover_replicates_exactly():
    for R in (1, 5, 6, 4096):
        for world in (1, 2, 3, 8):
            spans = [replicas.shard(R, world, k) for k in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == R
            assert all(spans[k][1] == spans[k + 1][0] for k in range(world - 1))


def test_two_gloo_ranks_match_single_process():
    world = 2
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(k, world, port, out)) for k in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        ms = [np.array(out[k]) for k in range(world)]
    w = _workload()
    parts = [_moments(w, *replicas.shard(w.R, world, k)) for k in range(world)]
    single = replicas.combine(parts)
    for m in ms:
        assert np.array_equal(m, single)
    # and the sum equals the unsharded sum up to the order of additions
    np.testing.assert_allclose(single, _moments(w, 0, w.R), rtol=1e-12)

"""Runs one workload for a number of days with one kernel launch per step and
day, for kernel captures (e.g. ``ncu -k regex:k_node_day_dealt -s D -c 1``
captures day D's stochastic step).

    python -m paper_1502_02908_gb300.profile_case national --days 301
    python -m paper_1502_02908_gb300.profile_case batched --days 201
    python -m paper_1502_02908_gb300.profile_case national --days 60 --launch flow
    python -m paper_1502_02908_gb300.profile_case batched --days 30 --launch persistent
    python -m paper_1502_02908_gb300.profile_case uneven --instances 64

Cases: ``national`` (SISe3, 37,000 herds, 3M events; warp path from 800
animals, group path from 200, the bench's tuned shape), ``batched`` (the national
network with 256 replicates, every herd on the per-thread path), ``general``
(SISe3 written in the general model), ``uneven`` (the first `--instances` of the
512-instance uneven batch, whole horizons, in one persistent launch).  Launches go
to the stream one by one (no CUDA graph), so each kernel launch is capturable;
with ``--launch flow`` the days run as one dataflow launch, with ``--launch
persistent`` as one persistent batch launch (block shape ``--shape``).
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["national", "batched", "general", "uneven"])
    ap.add_argument("--days", type=int, default=301)
    ap.add_argument("--launch", choices=["stream", "flow", "persistent"], default="stream",
                    help="stream: one launch per kernel and day; flow: one dataflow launch for all days; "
                         "persistent: one persistent batch launch")
    ap.add_argument("--shape", default="256x2", help="persistent batch block shape, threads x blocks an SM")
    ap.add_argument("--instances", type=int, default=64, help="uneven: how many of the 512 instances")
    args = ap.parse_args(argv)
    import torch
    from . import binding as B
    from . import workloads as W
    from .build import build
    build()
    B.batch_shape(*(int(x) for x in args.shape.split("x")))
    if args.case == "uneven":
        ws = W.uneven_batch()[:args.instances]
        sims = [B.Sim.from_workload(w) for w in ws]
        B.run_batch(sims)
        torch.cuda.synchronize()
        for s in sims:
            s.close()
        print(f"uneven: {len(ws)} instances, {sum(w.N * w.T for w in ws)} node-days done")
        return 0
    if args.case == "general":
        w = W.as_general(W.sise3_national())
        w.T = min(args.days, w.T)
        s = B.GenSim.from_workload(w)
        s.set_warp_threshold(600)
        s.set_group_threshold(300)
    else:
        w = W.sise3_national() if args.case == "national" else W.sise3_batched(R=256, T=365)
        w.T = min(args.days, w.T)
        s = B.Sim.from_workload(w)
        if args.case == "national":
            s.set_group_threshold(200)
            s.tune(800)
        else:
            s.set_group_threshold(1 << 30)
            s.tune(1 << 30)
    s.set_launch(args.launch if args.case != "general" else "stream")
    s.run(w.T)
    torch.cuda.synchronize()
    s.close()
    print(f"{args.case}: {w.T} days done")
    return 0


if __name__ == "__main__":
    sys.exit(main())

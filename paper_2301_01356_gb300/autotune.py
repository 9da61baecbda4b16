"""Autotuner: the best configuration per graph-size bucket (and per benchmark graph).

For every size bucket of a sample batch, each candidate configuration (ruler
stride of the list ranking; First-CC variant: plain hooking, local-first in
shared memory, or sampled; Last-CC sampling) is timed with CUDA events on the
bucket's batched solve (mean of a few runs), the three fastest are timed again
over many more runs (a sampled variant can be slow now and then, and a short
mean can miss it), and the fastest of those is written to ``tuning.json`` beside
this module, which ``batch.BatchRunner`` and ``bench.py`` read.

    python -m paper_2301_01356_gb300.autotune [--graphs 512] [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import batch as B
from . import fbcc, graphgen as gg

CANDIDATES = [dict(ruler_stride=s, cc_local=l, cc_sample=c, lcc_sample=q)
              for s in (8, 16, 32) for (l, c) in ((0, 0), (8192, 0), (16384, 0), (0, 2)) for q in (0, 2)]


def _time(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    # the mean, not the median: a configuration that is slow now and then (a
    # sampled skip that misses) must pay for it
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def _finalists(times: dict, k: int = 3) -> list:
    return sorted(times, key=times.get)[:k]


def tune_batch(batch, reps: int = 8, candidates=CANDIDATES, buckets=B.BUCKETS, final_reps: int = 30) -> list:
    out = []
    sizes = batch.sizes()
    for lo, hi in buckets:
        idx = np.nonzero((sizes >= lo) & (sizes < hi))[0]
        if idx.size == 0:
            continue
        runner = B.BatchRunner(batch.subset(idx), buckets=((lo, hi),), tuning={})

        def configure(cfg):
            for b in runner.buckets:      # every chunk of the bucket
                fbcc.fbcc_workspace_configure(b.ws, **cfg)
        times = {}
        for cfg in candidates:
            configure(cfg)
            times[json.dumps(cfg, sort_keys=True)] = _time(runner.run, reps)
        final = {}
        for key in _finalists(times):   # the closest few again, long enough to see rare slow runs
            configure(json.loads(key))
            final[key] = _time(runner.run, final_reps)
        best = min(final, key=final.get)
        times.update(final)
        out.append({"lo": lo, "hi": hi, "graphs": int(idx.size), "config": json.loads(best), "ms": times[best],
                    "candidates_ms": times})
        runner.close()
    return out


def tune_graph(g, off64: bool, reps: int = 8, candidates=CANDIDATES, final_reps: int = 30) -> dict:
    import torch
    off = torch.from_numpy(g.offsets.astype(np.int64 if off64 else np.int32)).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    s = fbcc.Solver(g.n, g.nnz)
    times = {}
    for cfg in candidates:
        s.configure(**cfg)
        times[json.dumps(cfg, sort_keys=True)] = _time(lambda: s.enqueue(off, adj), reps)
    final = {}
    for key in _finalists(times):
        s.configure(**json.loads(key))
        final[key] = _time(lambda: s.enqueue(off, adj), final_reps)
    s.close()
    best = min(final, key=final.get)
    times.update(final)
    return {"config": json.loads(best), "ms": times[best], "candidates_ms": times}


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--graphs", type=int, default=512, help="graphs in the sample batch (config-4 recipe)")
    ap.add_argument("--out", default=B.TUNING_PATH)
    ap.add_argument("--reps", type=int, default=8)
    args = ap.parse_args(argv)
    t0 = time.time()
    sample = gg.batch(args.graphs, 44, 1000, 1000000)
    table = {"device": torch.cuda.get_device_name(0), "sample": f"{args.graphs} graphs, config-4 recipe, seed 44",
             "buckets": tune_batch(sample, args.reps)}
    table["graphs"] = {
        "grid4096": tune_graph(gg.workload_grid_4096(), False, args.reps),
        "uniform64k": tune_graph(gg.workload_uniform_64k(), False, args.reps),
        "rmat24": tune_graph(gg.workload_rmat_24(), True, args.reps),
    }
    table["seconds"] = round(time.time() - t0, 1)
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps({k: (v if k != "buckets" else [{kk: b[kk] for kk in ("lo", "hi", "config", "ms")} for b in v])
                      for k, v in table.items() if k != "graphs"}))
    print(json.dumps({k: {"config": v["config"], "ms": v["ms"]} for k, v in table["graphs"].items()}))


if __name__ == "__main__":
    main()

"""Autotuner for the launch shape of the FCFS kernels; its choices go into plans.

Knobs are tuned by timing real calls with CUDA events, each candidate run
through a Plan (fcfs_plan_* of the C ABI), so no process-wide hook changes:

* single clip: the form of the contraction (over the corners, split-FP16 over
  y, pruned FFT along y), and for the contraction over the corners its vertex
  splits (split-K) and tile shape (CTA pairs or one-CTA tiles);
* batch: chunks per (clip, tile, split) unit, tile shape, grouping by y.

The winning knobs are cached in a JSON file keyed by GPU name, T, K, precision,
the power-of-two bucket of the corner count and the clip count, so a workload
is tuned once per machine; tune_* return a Plan carrying them.  The cache lives
at $FCFS_AUTOTUNE_CACHE, else ~/.cache/fcfs_gb300/autotune.json.
"""
import json
import math
import os
import statistics

import torch

from . import fcfs

SPLIT_CANDIDATES = (0, 2, 4, 8, 12, 19, 38, 76, 152)
UNIT_CANDIDATES = (8, 16, 32, 64, 128)   # longer FP32 accumulation runs lose accuracy


def cache_path():
    return os.environ.get("FCFS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fcfs_gb300", "autotune.json"))


def _load():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(db):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(db, fh, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _key(kind, T, K, prec, V, n=1):
    gpu = torch.cuda.get_device_name()
    vb = int(math.log2(max(1, V)))
    return "plan|%s|%s|T%d|K%d|%s|V2^%d|n%d" % (kind, gpu, T, K, prec, vb, n)


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def _forward_candidates(prec, K):
    """Knob sets tried for one clip: each form with the library's own split
    count, then the contraction over the corners with other split counts and,
    for split FP16, one-CTA tiles."""
    cands = [{"form": 0}, {"form": 2}]
    if prec == "split_f16" and 2 * K >= 256:
        cands.insert(1, {"form": 1})
        cands.append({"form": 0, "pair": 0})
    cands += [{"form": 0, "splits": sp} for sp in SPLIT_CANDIDATES if sp]
    return cands


def _best(kind, key, cands, make, run, reps, force):
    db = _load()
    if key in db and not force:
        return make(db[key]["knobs"])
    best, results = None, {}
    for kn in cands:
        try:
            plan = make(kn)
            ms = _time(run(plan), reps)
        except fcfs.FCFSError:
            continue   # a knob set the sizes do not allow
        results[json.dumps(kn, sort_keys=True)] = ms
        if best is None or ms < best[0]:
            best = (ms, kn)
    db[key] = {"knobs": best[1], "ms": best[0], "tried": results}
    _store(db)
    return make(best[1])


def tune_forward(x, y, s, T, K, prec="split_f16", reps=5, force=False):
    """A forward Plan with the fastest knobs for one clip (measured; cached)."""
    V = x.numel()
    W = 2 * K + 1
    out = torch.empty((W, W), dtype=torch.complex64, device=x.device)
    area = torch.empty(1, dtype=torch.int64, device=x.device)
    nchunks = (V + 63) // 64
    cands = [c for c in _forward_candidates(prec, K) if c.get("splits", 0) <= nchunks]

    def make(kn):
        return fcfs.Plan("forward", V, T, K, prec, **kn)

    def run(plan):
        ws = fcfs.alloc_workspace(plan.workspace_size(), x.device)
        return lambda: plan.forward(x, y, s, out=out, area_out=area, workspace=ws)

    return _best("forward", _key("forward", T, K, prec, V), cands, make, run, reps, force)


def tune_batch(x, y, s, offsets, T, K, prec="split_f16", reps=3, force=False):
    """A batch Plan with the fastest knobs (chunks per unit, tile shape, grouping
    by y) for these clips (measured; cached)."""
    n = offsets.numel() - 1
    V = x.numel()
    W = 2 * K + 1
    out = torch.empty((n, W, W), dtype=torch.complex64, device=x.device)
    area = torch.empty(n, dtype=torch.int64, device=x.device)
    cands = [{"form": 0, "unit_chunks": uc} for uc in UNIT_CANDIDATES]
    if prec == "split_f16" and 2 * K >= 256:
        cands += [{"form": 0, "unit_chunks": uc, "pair": 0} for uc in UNIT_CANDIDATES]
        cands.append({"form": 1})

    def make(kn):
        return fcfs.Plan("batch", V, T, K, prec, n_clips=n, **kn)

    def run(plan):
        ws = fcfs.alloc_workspace(plan.workspace_size(), x.device)
        return lambda: plan.batch(x, y, s, offsets, out=out, area_out=area, workspace=ws)

    return _best("batch", _key("batch", T, K, prec, V, n), cands, make, run, reps, force)

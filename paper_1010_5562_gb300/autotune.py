"""Autotuner for the launch shape of the FCFS kernels.

Two knobs are tuned by timing real calls with CUDA events:

* single clip: the number of vertex splits of the contraction (split-K), which
  trades parallelism against the size of the partial sums;
* batch: the number of pipeline chunks per (clip, tile, split) unit, which
  trades load balance against the number of partial tiles.

Results are cached in a JSON file keyed by GPU name, T, K, precision and the
power-of-two bucket of the corner count, so a workload is tuned once per
machine.  The cache lives at $FCFS_AUTOTUNE_CACHE, else
~/.cache/fcfs_gb300/autotune.json.
"""
import json
import math
import os
import statistics

import torch

from . import fcfs

SPLIT_CANDIDATES = (0, 1, 2, 4, 8, 12, 16, 19, 24, 32, 38, 48, 64, 76, 96, 152)
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
    return "%s|%s|T%d|K%d|%s|V2^%d|n%d" % (kind, gpu, T, K, prec, vb, n)


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


def tune_forward(x, y, s, T, K, prec="split_f16", reps=5, force=False):
    """Best split count for one clip (0 = the library's own choice); cached."""
    db = _load()
    key = _key("forward", T, K, prec, x.numel())
    if key in db and not force:
        return db[key]["splits"]
    W = 2 * K + 1
    out = torch.empty((W, W), dtype=torch.complex64, device=x.device)
    area = torch.empty(1, dtype=torch.int64, device=x.device)
    best = (float("inf"), 0)
    results = {}
    nchunks = (x.numel() + 63) // 64
    for sp in SPLIT_CANDIDATES:
        if sp > nchunks:
            continue
        fcfs.set_splits(sp)
        try:
            ws = torch.empty(fcfs.workspace_size(x.numel(), T, K, prec), dtype=torch.uint8, device=x.device)
            ms = _time(lambda: fcfs.forward(x, y, s, T, K, prec=prec, out=out, area_out=area, workspace=ws), reps)
        finally:
            fcfs.set_splits(0)
        results[str(sp)] = ms
        best = min(best, (ms, sp))
    db[key] = {"splits": best[1], "ms": best[0], "tried": results}
    _store(db)
    return best[1]


def tune_batch(x, y, s, offsets, T, K, prec="split_f16", reps=3, force=False):
    """Best chunks per unit for a batch (0 = default); cached."""
    n = offsets.numel() - 1
    db = _load()
    key = _key("batch", T, K, prec, x.numel(), n)
    if key in db and not force:
        return db[key]["unit_chunks"]
    W = 2 * K + 1
    out = torch.empty((n, W, W), dtype=torch.complex64, device=x.device)
    area = torch.empty(n, dtype=torch.int64, device=x.device)
    lib = fcfs._lib.load()
    best = (float("inf"), 0)
    results = {}
    for uc in UNIT_CANDIDATES:
        fcfs.set_batch_unit_chunks(uc)
        try:
            need = lib.fcfs_batch_workspace_size(x.numel(), n, T, K, fcfs.PREC[prec])
            ws = torch.empty(need, dtype=torch.uint8, device=x.device)
            ms = _time(lambda: fcfs.batch(x, y, s, offsets, T, K, prec=prec, out=out, area_out=area,
                                          workspace=ws), reps)
        finally:
            fcfs.set_batch_unit_chunks(0)
        results[str(uc)] = ms
        best = min(best, (ms, uc))
    db[key] = {"unit_chunks": best[1], "ms": best[0], "tried": results}
    _store(db)
    return best[1]

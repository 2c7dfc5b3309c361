#!/usr/bin/env python3
"""Throughput of the FCFS block transform on GB300, one JSON line on stdout.

Step: one forward block F(k,l), |k|,|l| <= 256, of the synthetic Manhattan clip
T=4096 with 2000 polygons (~12.6k signed corners), through the C ABI on the
split-FP16 tensor-core path: tables, exact area and axis lines, tcgen05
contraction, compensated split-K reduction and epilogue (five kernels).
Metric: vertex-coefficient terms per second, V * (2K+1)^2 per step.

Default run: N=1, warm-up 50, 5000 timed steps.  The clip's inputs are far
smaller than L2, so L2 is flushed (a 256 MiB write) before every timed step,
outside the timed events.  Under torchrun each rank runs its own replica of the
clip on its own GPU (no collective; weak scaling); rank 0 prints the line.

--impl reference times the FP64 oracle instead (the plain CPU implementation
of the definition, on the host cores), on row samples of the same block.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vertex·coefficient terms/s (fwd, adjoint) vs plain FP32 GPU at stated rel error"
UNIT = "terms/s"
WORKLOAD = ("clip T=4096, 2000 rectilinear polygons (rect/L/T/U/plus/stair, sides 20-89), "
            "V=12576 signed corners, K=256 (513x513 complex64 block), forward")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "gemm_tc_T4096_K256.md")
FALLBACK_BF16_TFLOPS = 1900.0
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint, batch, large-clip and cosine-series measurements")
    ap.add_argument("--no-pair", action="store_true",
                    help="--only: one-CTA tiles instead of CTA pairs (profiling)")
    ap.add_argument("--no-fuse", action="store_true",
                    help="--only: separate axis and reduce kernels (profiling)")
    ap.add_argument("--prec", choices=["split_f16", "fp32"], default="split_f16",
                    help="--only adjoint / adjoint_large / cosine / cosine_large: contraction precision")
    ap.add_argument("--only", choices=["step", "large", "batch", "adjoint", "adjoint_large", "cosine",
                                       "cosine_large", "haar", "haar_large"], default=None,
                    help="run one workload warmup + steps times and print its mean time "
                         "(for profiler command lines; not the benchmark line)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def host_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"),
                default=0)
        if n:
            return int(n)
    except Exception:
        pass
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def workload():
    from synth import config_clip
    clip, K = config_clip(2)
    return clip, K


def terms(clip, K):
    return clip.V * (2 * K + 1) ** 2


# ---------------------------------------------------------------------------
# the oracle as CPU baseline (the only place bench.py runs oracle/)
# ---------------------------------------------------------------------------
def oracle_rows(clip, K, rows, start):
    """F(k, l) for `rows` consecutive k (cycling over [-K, K]) and every l."""
    import numpy as np
    import oracle
    f = np.arange(-K, K + 1)
    ks = f[(start + np.arange(rows)) % f.shape[0]]
    return oracle.block_entries(clip.x, clip.y, clip.s, clip.T, ks, f)


def cpu_baseline(clip, K, seconds):
    """Full oracle blocks, repeated for about `seconds` of CPU time."""
    import oracle
    t0 = time.perf_counter()
    runs = 0
    F = None
    while True:
        F = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
        runs += 1
        el = time.perf_counter() - t0
        if runs >= 2 and el >= seconds:
            break
    value = terms(clip, K) * runs / el
    info = {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": "%d full 513x513 blocks of the T=4096 clip in %.1f s (FP64 numpy, BLAS matmul)"
                      % (runs, el)}
    return info, F, oracle.area_exact(clip.x, clip.y, clip.s, clip.T)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    clip, K = workload()
    W = 2 * K + 1
    t0 = time.perf_counter()
    oracle_rows(clip, K, 8, 0)
    per_row = (time.perf_counter() - t0) / 8
    budget = 90.0
    rows = int(max(1, min(W, budget / max(1, args.steps + args.warmup) / per_row)))
    for i in range(args.warmup):
        oracle_rows(clip, K, rows, i * rows)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle_rows(clip, K, rows, (args.warmup + i) * rows)
    el = time.perf_counter() - t0
    n_terms = clip.V * rows * W * args.steps
    value = n_terms / el
    cores = host_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_rows_per_step": rows,
                                        "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d block rows x 513 columns per step (FP64 numpy)" % rows},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
            if self.idx is not None:
                cmd += ["-i", str(self.idx)]
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [c.strip() for c in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_index_for_smi(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local < len(ids):
            return ids[local]
    return local


# ---------------------------------------------------------------------------
# our path
# ---------------------------------------------------------------------------
def measured_peak():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return FALLBACK_BF16_TFLOPS, "fallback"


KERNEL_SOURCES = ("fcfs_tc.cu", "fcfs_epilogue.cuh", "fcfs_common.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1010_5562_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch():
    """DRAM bytes per launch of the contraction kernel from the committed ncu
    summary, if it was taken on the current kernel source (the kernel file and
    the two device headers it includes)."""
    try:
        h = kernel_source_hash()
        txt = open(TRAFFIC_FILE).read()
        got = {}
        for line in txt.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                v = v.strip().split()
                if v:
                    got[k.strip().strip("-* `")] = v[0].strip("`")
        if got.get("source_sha256_16") == h:
            return float(got["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def whole_job_rate(local_ms, units_per_step, steps, world, device="cpu"):
    """Throughput of `world` replicas that each process `units_per_step` units
    in each of `steps` steps: the slowest rank bounds the job, so the time is
    the maximum over ranks (one all-reduce when world > 1) and the rate is
    world * units_per_step * steps / that time.  Returns (rate per second, ms)."""
    t = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * units_per_step * steps / (t * 1e-3), t


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs

    clip, K = workload()
    T, V = clip.T, clip.V
    W = 2 * K + 1
    n_terms = terms(clip, K)
    x = torch.from_numpy(clip.x).to(dev)
    y = torch.from_numpy(clip.y).to(dev)
    s = torch.from_numpy(clip.s).to(dev)
    F = torch.empty((W, W), dtype=torch.complex64, device=dev)
    area = torch.empty((1,), dtype=torch.int64, device=dev)
    ws = torch.empty(fcfs.workspace_size(V, T, K, "split_f16"), dtype=torch.uint8, device=dev)
    F32 = torch.empty_like(F)
    ws32 = torch.empty(fcfs.workspace_size(V, T, K, "fp32"), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(prec="split_f16"):
        if prec == "split_f16":
            fcfs.forward(x, y, s, T, K, prec=prec, out=F, area_out=area, workspace=ws, stream=stream)
        else:
            fcfs.forward(x, y, s, T, K, prec=prec, out=F32, area_out=area, workspace=ws32, stream=stream)

    def timed(n, fn):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for a, b in evs:
            flush.fill_(1)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(b) for a, b in evs]

    for _ in range(max(3, args.warmup)):
        flush.fill_(1)
        step()
    step("fp32")
    torch.cuda.synchronize(dev)

    # ---- main timed region ----
    # The timed steps can take only milliseconds, less than the sampling period
    # of nvidia-smi, so the same step also runs (untimed) for a few sampling
    # periods before and after them: the clock samples are taken under that load.
    def keep_busy(seconds):
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            for _ in range(20):
                flush.fill_(1)
                step()
            torch.cuda.synchronize(dev)

    sampler = ClockSampler(gpu_index_for_smi(local)) if rank == 0 else None
    if sampler:
        sampler.start()
        keep_busy(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    l0 = fcfs.launch_count()
    ms = timed(args.steps, step)
    launches = fcfs.launch_count() - l0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        keep_busy(0.3)
    clocks = sampler.stop() if sampler else None
    if clocks is not None:
        clocks["window"] = "nvidia-smi every 100 ms, the step running 0.3 s before and after the timed steps"
    value, total_ms = whole_job_rate(sum(ms), n_terms, args.steps, world, dev)

    # ---- per-kernel roofline of the contraction (events around the kernel) ----
    reps = min(args.steps, 500)
    fcfs.profile_enable(True)
    stage = []
    for _ in range(reps):
        flush.fill_(1)
        step()
        stage.append(fcfs.profile_read())
    fcfs.profile_enable(False)
    gemm_ms = statistics.mean(r[2] for r in stage)
    stage_ms = [statistics.mean(r[i] for r in stage) for i in range(4)]
    alg_flops = 2.0 * V * (2 * K) ** 2          # one real MAC per off-axis term
    issued_flops = 3.0 * alg_flops               # hi*hi + hi*lo + lo*hi
    peak_tf, peak_kind = measured_peak()
    achieved = alg_flops / (gemm_ms * 1e-3) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf, "traffic": traffic_per_launch(),
                "kernel": ("gemm_tc_kernel<256,3,full,pair> (tcgen05 cta_group::2 split-FP16 contraction on "
                           "CTA pairs; fused split-K sum, axis DFT and output behind a grid barrier)"),
                "kernel_ms": gemm_ms, "peak_source": "%s bf16 dense burst (fp16 same rate)" % peak_kind,
                "issued_tflops": issued_flops / (gemm_ms * 1e-3) / 1e12,
                "issued_frac": issued_flops / (gemm_ms * 1e-3) / 1e12 / peak_tf,
                # the axis lines and the split-K sum run inside the contraction kernel
                "stage_ms": {"prep": stage_ms[0], "contraction_with_fused_tail": stage_ms[2]}}

    # ---- plain FP32 path on the same clip ----
    ms32 = timed(min(args.steps, 1000), lambda: step("fp32"))
    value32 = world * n_terms / (statistics.mean(ms32) * 1e-3)

    # ---- end to end: pinned host inputs in, block out ----
    # x, y and s travel in one pinned staging buffer (16-byte aligned views on
    # both sides), F and the area come back as one block: one copy each way
    a16 = lambda n: (n + 15) // 16 * 16
    ox, oy, osg = 0, a16(4 * V), 2 * a16(4 * V)
    nin = osg + a16(V)
    hin = torch.zeros(nin, dtype=torch.uint8).pin_memory()
    hin[ox:ox + 4 * V].copy_(torch.from_numpy(clip.x).view(torch.uint8))
    hin[oy:oy + 4 * V].copy_(torch.from_numpy(clip.y).view(torch.uint8))
    hin[osg:osg + V].copy_(torch.from_numpy(clip.s).view(torch.uint8))
    din = torch.empty(nin, dtype=torch.uint8, device=dev)
    ex, ey = din[ox:ox + 4 * V].view(torch.int32), din[oy:oy + 4 * V].view(torch.int32)
    es = din[osg:osg + V].view(torch.int8)
    nout = W * W * 8 + 8
    dout = torch.empty(nout, dtype=torch.uint8, device=dev)
    eF = dout[:W * W * 8].view(torch.complex64).view(W, W)
    ea = dout[W * W * 8:].view(torch.int64)
    hout = torch.empty(nout, dtype=torch.uint8).pin_memory()

    def e2e_step():
        din.copy_(hin, non_blocking=True)
        fcfs.forward(ex, ey, es, T, K, prec="split_f16", out=eF, area_out=ea, workspace=ws, stream=stream)
        hout.copy_(dout, non_blocking=True)

    for _ in range(5):
        e2e_step()
    mse = timed(min(args.steps, 1000), e2e_step)
    torch.cuda.synchronize(dev)
    e2e_ok = bool(torch.equal(hout[:W * W * 8].view(torch.complex64).view(W, W), F.cpu()))

    # Pipelined: steps alternate between two streams, so one step's copies run on
    # the copy engines while another step computes.  Eight buffer sets (inputs,
    # block, workspace) rotate; together they exceed L2 (129 MB), so a set comes
    # back cold, and set i is reused on the same stream 8 steps later (no race).
    n_sets = 8
    sets = []
    for _ in range(n_sets):
        d_in = torch.empty(nin, dtype=torch.uint8, device=dev)
        d_out = torch.empty(nout, dtype=torch.uint8, device=dev)
        sets.append(dict(din=d_in, dout=d_out, ws=torch.empty_like(ws),
                         hout=torch.empty(nout, dtype=torch.uint8).pin_memory(),
                         x=d_in[ox:ox + 4 * V].view(torch.int32), y=d_in[oy:oy + 4 * V].view(torch.int32),
                         s=d_in[osg:osg + V].view(torch.int8),
                         F=d_out[:W * W * 8].view(torch.complex64).view(W, W), a=d_out[W * W * 8:].view(torch.int64)))
    set_bytes = nin + nout + ws.numel()
    lanes = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]

    def e2e_pipelined(n):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for ln in lanes:
            ln.wait_stream(stream)
        for i in range(n):
            ln, b = lanes[i % 2], sets[i % n_sets]
            with torch.cuda.stream(ln):
                b["din"].copy_(hin, non_blocking=True)
                fcfs.forward(b["x"], b["y"], b["s"], T, K, prec="split_f16", out=b["F"], area_out=b["a"],
                             workspace=b["ws"], stream=ln)
                b["hout"].copy_(b["dout"], non_blocking=True)
        for ln in lanes:
            stream.wait_stream(ln)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        return t0.elapsed_time(t1) / n

    e2e_pipelined(2 * n_sets)
    ms_pipe = e2e_pipelined(min(args.steps, 1000))
    pipe_ok = all(bool(torch.equal(b["hout"][:W * W * 8].view(torch.complex64).view(W, W), F.cpu())) for b in sets)
    e2e = {"value": world * n_terms / (ms_pipe * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": int(nin), "d2h_bytes_per_step": int(nout),
           "copies": ("every step: one H2D of x, y, s from pinned host memory and one D2H of F and the area; "
                      "steps alternate between two streams so copies overlap another step's compute; "
                      "%d buffer sets in rotation (%.0f MB, more than L2)" % (n_sets, n_sets * set_bytes / 1e6)),
           "ms_per_step": ms_pipe, "matches_device_step": bool(e2e_ok and pipe_ok),
           "serial": {"value": world * n_terms / (statistics.mean(mse) * 1e-3), "ms_per_step": statistics.mean(mse),
                      "note": "one stream, events around each step, L2 flushed between steps"}}

    extras = {} if (world > 1 or args.no_extras) else run_extras(fcfs, dev, flush, stream, args)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic (seeded Manhattan clip; stands in for the paper's proprietary 22 nm layout)",
        "config": {"workload": WORKLOAD, "precision": "split_f16 (hi+lo FP16 operands, FP32 accumulate, "
                   "TwoSum-compensated split-K sum)", "T": T, "K": K, "V": V,
                   "l2": "flushed before every timed step (256 MiB write, outside the events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "plain_fp32": {"value": value32, "unit": UNIT, "ms_per_step": statistics.mean(ms32)},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    for k in ("adjoint", "batch", "large", "cosine", "haar", "crossover"):
        if k in extras:
            line[k] = extras[k]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import numpy as np
        cb, Fo, A = cpu_baseline(clip, K, args.cpu_seconds)
        line["cpu_baseline"] = cb
        step()
        step("fp32")
        torch.cuda.synchronize(dev)
        errs = {}
        for name, t in (("split_f16", F), ("fp32", F32)):
            Fg = t.cpu().numpy().astype(np.complex128)
            errs[name] = float(np.max(np.abs(Fg - Fo)) / A)
        line["accuracy"] = {"max_abs_err_over_area": errs, "area_exact": int(area.item()) == A,
                            "reference": "FP64 oracle (direct signed-quadrant vertex sum)"}
        if extras:
            extras_accuracy(line, extras)
    if rank == 0:
        print(json.dumps(strip_private(line)), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def strip_private(obj):
    """Drop the bookkeeping entries (keys starting with '_') that the accuracy
    pass consumes, e.g. when it is skipped."""
    if isinstance(obj, dict):
        return {k: strip_private(v) for k, v in obj.items() if not str(k).startswith("_")}
    return obj


# ---------------------------------------------------------------------------
# the other workloads: adjoint, batch, large clip (reported beside the step)
# ---------------------------------------------------------------------------
def _timed_ms(torch, fn, n, flush, stream):
    fn()
    torch.cuda.synchronize()
    out = []
    for _ in range(n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        a.record(stream)
        fn()
        b.record(stream)
        out.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in out)


def run_extras(fcfs, dev, flush, stream, args):
    import numpy as np
    import torch
    from synth import config_clip, config4_target, batch_clips, concat_clips
    from paper_1010_5562_gb300 import autotune
    out = {}

    # adjoint: workload 4, pupil loss, FP32
    clip, K = config_clip(4)
    tgt, _ = config4_target(clip)
    T, W = clip.T, 2 * K + 1
    x, y, s = (torch.from_numpy(a).to(dev) for a in (clip.x, clip.y, clip.s))
    F, _ = fcfs.forward(x, y, s, T, K, prec="fp32")
    Ft, _ = fcfs.forward(*(torch.from_numpy(a).to(dev) for a in (tgt.x, tgt.y, tgt.s)), T, K, prec="fp32")
    f = torch.arange(-K, K + 1, device=dev)
    mask = ((f[:, None] ** 2 + f[None, :] ** 2) <= K * K)
    G = (2.0 * (F - Ft) * mask).contiguous()
    gx = torch.empty(clip.V, dtype=torch.float32, device=dev)
    gy = torch.empty_like(gx)
    wsa = torch.empty(fcfs._lib.load().fcfs_adjoint_workspace_size(clip.V, T, K, 0), dtype=torch.uint8, device=dev)
    ms = _timed_ms(torch, lambda: fcfs.adjoint(x, y, s, T, K, G, gx=gx, gy=gy, workspace=wsa, stream=stream),
                   20, flush, stream)
    gx16 = torch.empty_like(gx)
    gy16 = torch.empty_like(gx)
    wsa16 = torch.empty(fcfs._lib.load().fcfs_adjoint_workspace_size(clip.V, T, K, 1), dtype=torch.uint8,
                        device=dev)
    ms16 = _timed_ms(torch, lambda: fcfs.adjoint(x, y, s, T, K, G, prec="split_f16", gx=gx16, gy=gy16,
                                                 workspace=wsa16, stream=stream), 20, flush, stream)
    out["adjoint"] = {"workload": "clip T=2048, 5000 polygons, V=%d, K=128, pupil-disc loss vs edges "
                                  "jittered +-2; corner derivatives" % clip.V,
                      "value": clip.V * W * W / (ms16 * 1e-3), "unit": UNIT, "ms": ms16,
                      "precision": "split_f16 (tcgen05 contraction)",
                      "fp32": {"value": clip.V * W * W / (ms * 1e-3), "ms": ms},
                      "_check": (clip, tgt, K, G.cpu().numpy(), gx.cpu().numpy(), gy.cpu().numpy(),
                                 gx16.cpu().numpy(), gy16.cpu().numpy())}

    # batch: workload 3, one launch replayed from a CUDA graph vs one call per clip
    clips, K = batch_clips()
    T, W = clips[0].T, 2 * K + 1
    bx, by, bs, boff = (torch.from_numpy(a).to(dev) for a in concat_clips(clips))
    n = len(clips)
    terms_b = float(sum(c.V for c in clips)) * W * W
    uc = autotune.tune_batch(bx, by, bs, boff, T, K, prec="split_f16")
    fcfs.set_batch_unit_chunks(uc)
    Fb = torch.empty((n, W, W), dtype=torch.complex64, device=dev)
    Ab = torch.empty(n, dtype=torch.int64, device=dev)
    wsb = torch.empty(fcfs._lib.load().fcfs_batch_workspace_size(bx.numel(), n, T, K, 1), dtype=torch.uint8,
                      device=dev)
    cap = torch.cuda.Stream(dev)   # graphs are captured on a side stream
    with torch.cuda.stream(cap):
        fcfs.batch(bx, by, bs, boff, T, K, out=Fb, area_out=Ab, workspace=wsb, stream=cap)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        fcfs.batch(bx, by, bs, boff, T, K, out=Fb, area_out=Ab, workspace=wsb, stream=cap)
    ms_b = _timed_ms(torch, g.replay, 5, flush, stream)
    fcfs.set_batch_unit_chunks(0)
    per = [tuple(torch.from_numpy(a).to(dev) for a in (c.x, c.y, c.s)) for c in clips]
    wsc = torch.empty(max(fcfs.workspace_size(c.V, T, K) for c in clips), dtype=torch.uint8, device=dev)
    Fc = torch.empty((W, W), dtype=torch.complex64, device=dev)
    Ac = torch.empty(1, dtype=torch.int64, device=dev)

    def per_clip():
        for (cx, cy, cs) in per:
            fcfs.forward(cx, cy, cs, T, K, out=Fc, area_out=Ac, workspace=wsc, stream=stream)

    ms_c = _timed_ms(torch, per_clip, 3, flush, stream)
    out["batch"] = {"workload": "512 clips, T=2048, V_c log-uniform 1e3..1e5 (sum %d), K=128, split_f16"
                                % bx.numel(),
                    "value": terms_b / (ms_b * 1e-3), "unit": UNIT, "ms": ms_b,
                    "per_clip_calls_value": terms_b / (ms_c * 1e-3), "per_clip_calls_ms": ms_c,
                    "unit_chunks": uc, "launch": "one fcfs_batch call replayed from a CUDA graph",
                    "_check": (clips, K, Fb, Ab)}

    # large clip: workload 5, both precisions
    clip5, K5 = config_clip(5)
    W5 = 2 * K5 + 1
    x5, y5, s5 = (torch.from_numpy(a).to(dev) for a in (clip5.x, clip5.y, clip5.s))
    big = {}
    for prec in ("split_f16", "fp32"):
        F5 = torch.empty((W5, W5), dtype=torch.complex64, device=dev)
        A5 = torch.empty(1, dtype=torch.int64, device=dev)
        ws5 = torch.empty(fcfs.workspace_size(clip5.V, clip5.T, K5, prec), dtype=torch.uint8, device=dev)
        ms5 = _timed_ms(torch, lambda: fcfs.forward(x5, y5, s5, clip5.T, K5, prec=prec, out=F5, area_out=A5,
                                                    workspace=ws5, stream=stream), 3, flush, stream)
        big[prec] = {"value": clip5.V * W5 * W5 / (ms5 * 1e-3), "ms": ms5, "_F": F5, "_A": A5}
    big["split_f16"]["contraction"] = "corners grouped by y: T+1 contraction columns instead of V corners"
    # the direct contraction over the V corners on the same clip, for comparison
    fcfs.set_hybrid(0)
    try:
        F5d = torch.empty((W5, W5), dtype=torch.complex64, device=dev)
        A5d = torch.empty(1, dtype=torch.int64, device=dev)
        ws5d = torch.empty(fcfs.workspace_size(clip5.V, clip5.T, K5, "split_f16"), dtype=torch.uint8, device=dev)
        ms5d = _timed_ms(torch, lambda: fcfs.forward(x5, y5, s5, clip5.T, K5, prec="split_f16", out=F5d,
                                                     area_out=A5d, workspace=ws5d, stream=stream), 3, flush, stream)
    finally:
        fcfs.set_hybrid(1)
    big["split_f16_direct"] = {"value": clip5.V * W5 * W5 / (ms5d * 1e-3), "ms": ms5d,
                               "contraction": "over the V corners (CTA pairs)"}
    # adjoint of the large clip (FP32), seeded random cotangent over the full block
    rng = np.random.default_rng(5)
    G5 = torch.from_numpy((rng.standard_normal((W5, W5)) + 1j * rng.standard_normal((W5, W5)))
                          .astype(np.complex64)).to(dev)
    gx5 = torch.empty(clip5.V, dtype=torch.float32, device=dev)
    gy5 = torch.empty_like(gx5)
    wsa5 = torch.empty(fcfs._lib.load().fcfs_adjoint_workspace_size(clip5.V, clip5.T, K5, 0), dtype=torch.uint8,
                       device=dev)
    ms_a5 = _timed_ms(torch, lambda: fcfs.adjoint(x5, y5, s5, clip5.T, K5, G5, gx=gx5, gy=gy5, workspace=wsa5,
                                                  stream=stream), 2, flush, stream)
    big["adjoint_fp32"] = {"value": clip5.V * W5 * W5 / (ms_a5 * 1e-3), "ms": ms_a5,
                           "cotangent": "seeded standard complex normal over the block",
                           "_G": G5, "_g": (gx5, gy5)}
    gx5h = torch.empty_like(gx5)
    gy5h = torch.empty_like(gx5)
    wsa5h = torch.empty(fcfs._lib.load().fcfs_adjoint_workspace_size(clip5.V, clip5.T, K5, 1), dtype=torch.uint8,
                        device=dev)
    ms_a5h = _timed_ms(torch, lambda: fcfs.adjoint(x5, y5, s5, clip5.T, K5, G5, prec="split_f16", gx=gx5h, gy=gy5h,
                                                   workspace=wsa5h, stream=stream), 3, flush, stream)
    big["adjoint_split_f16"] = {"value": clip5.V * W5 * W5 / (ms_a5h * 1e-3), "ms": ms_a5h,
                                "cotangent": "as adjoint_fp32", "_g": (gx5h, gy5h)}
    out["cosine"] = cosine_extras(fcfs, dev, flush, stream)
    out["haar"] = haar_extras(fcfs, dev, flush, stream)
    out["crossover"] = crossover_extras(fcfs, dev, flush, stream)
    out["large"] = {"workload": "clip T=65536, 150000 polygons, V=%d, K=1024 (2049x2049)" % clip5.V,
                    "unit": UNIT, "split_f16": big["split_f16"], "split_f16_direct": big["split_f16_direct"],
                    "fp32": big["fp32"],
                    "adjoint_split_f16": big["adjoint_split_f16"], "adjoint_fp32": big["adjoint_fp32"],
                    "_check": (clip5, K5)}
    return out


def cosine_large_clip():
    """~0.95M corners at T = 32768 (the largest period of the cosine series),
    the corner density of the T = 65536 workload."""
    from synth import make_clip
    return make_clip(32768, 150000, 1006, smin=20, smax=80, wmin=4, margin=1), 1024


def cosine_extras(fcfs, dev, flush, stream):
    """Continuous cosine series C(k, l), 0 <= k, l <= K: the bench clip
    (T = 4096, K = 256) and a large clip (T = 32768, ~0.95M corners, K = 1024),
    both precisions.  Terms: V (K + 1)^2 vertex-coefficient pairs per call."""
    import torch
    from synth import config_clip
    res = {"unit": UNIT}
    for key, (clip, K) in (("clip_T4096_K256", config_clip(2)), ("clip_T32768_K1024", cosine_large_clip())):
        x, y, s = (torch.from_numpy(a).to(dev) for a in (clip.x, clip.y, clip.s))
        d = {"V": clip.V, "T": clip.T, "K": K}
        for prec in ("split_f16", "fp32"):
            C = torch.empty((K + 1, K + 1), dtype=torch.float32, device=dev)
            A = torch.empty(1, dtype=torch.int64, device=dev)
            ws = torch.empty(fcfs.cosine_workspace_size(clip.V, clip.T, K, prec), dtype=torch.uint8, device=dev)
            n = 20 if K <= 256 else 3
            ms = _timed_ms(torch, lambda: fcfs.cosine(x, y, s, clip.T, K, prec=prec, out=C, area_out=A,
                                                      workspace=ws, stream=stream), n, flush, stream)
            e = {"value": clip.V * (K + 1) ** 2 / (ms * 1e-3), "ms": ms, "_C": C, "_A": A}
            if prec == "split_f16":   # 3 split products of a K x K x V contraction, whole call
                e["issued_tflops_whole_call"] = 3 * 2.0 * clip.V * K * K / (ms * 1e-3) / 1e12
            d[prec] = e
        d["_clip"] = clip
        res[key] = d
    return res


CROSSOVER_CLIPS = (
    # (T, polygons, seed, sides min/max, min sub-width, K)
    (4096, 500, 1101, 20, 200, 4, 256),
    (4096, 2000, 1102, 20, 200, 4, 256),
    (4096, 8000, 1103, 4, 40, 1, 256),
    (4096, 32000, 1104, 4, 18, 1, 256),
    (65536, 20000, 1105, 20, 300, 4, 1024),
    (65536, 150000, 1106, 20, 200, 4, 1024),
)


def crossover_extras(fcfs, dev, flush, stream):
    """Split-FP16 forward with the contraction over the V corners (direct) and
    over the T + 1 values of y after grouping the corners by y (the pruned
    sparse-image DFT of the off-axis block), across corner densities V / (T + 1).
    "auto" is the library's automatic choice for the sizes (a cost estimate of both)."""
    import torch
    from synth import make_clip
    rows = []
    for (T, n, seed, smin, smax, wmin, K) in CROSSOVER_CLIPS:
        clip = make_clip(T, n, seed, smin=smin, smax=smax, wmin=wmin)
        x, y, s = (torch.from_numpy(a).to(dev) for a in (clip.x, clip.y, clip.s))
        W = 2 * K + 1
        F = torch.empty((W, W), dtype=torch.complex64, device=dev)
        A = torch.empty(1, dtype=torch.int64, device=dev)
        r = {"T": T, "K": K, "V": clip.V, "V_per_y": round(clip.V / (T + 1), 2)}
        for mode, key in ((0, "direct_ms"), (2, "grouped_ms")):
            fcfs.set_hybrid(mode)
            try:
                ws = torch.empty(fcfs.workspace_size(clip.V, T, K, "split_f16"), dtype=torch.uint8, device=dev)
                r[key] = _timed_ms(torch, lambda: fcfs.forward(x, y, s, T, K, out=F, area_out=A, workspace=ws,
                                                               stream=stream), 10 if T <= 4096 else 3, flush, stream)
            finally:
                fcfs.set_hybrid(1)
        r["auto"] = "grouped" if fcfs.forward_grouped(clip.V, T, K) == 1 else "direct"
        r["faster"] = "grouped" if r["grouped_ms"] < r["direct_ms"] else "direct"
        rows.append(r)
    return {"unit": "ms per forward call (split FP16)", "rows": rows}


def measured_hbm():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def haar_extras(fcfs, dev, flush, stream):
    """Continuous Haar transform (all 4^J coefficients up to level J): the bench
    clip at full depth (T = 4096, J = 12) and the T = 65536 clip at J = 14.
    HBM roofline of the whole call: algorithmic bytes = the corners read once
    (9 B each) plus the FP64 coefficients written once (8 B each); the pipeline
    moves more per cell: 3 passes over the level-J grid of 4 B per cell (int32
    grid, cells up to 1024 wide) or 8 B (the row build's write, the column sums'
    read, the strip kernel's read), plus the 8 B coefficient per cell."""
    import torch
    from synth import config_clip
    peak, src = measured_hbm()
    res = {"unit": "coefficients/s", "hbm_peak_gbs": peak, "peak_source": src}
    for key, ci, J in (("clip_T4096_J12", 2, 12), ("clip_T65536_J14", 5, 14)):
        clip, _ = config_clip(ci)
        x, y, s = (torch.from_numpy(a).to(dev) for a in (clip.x, clip.y, clip.s))
        G = 1 << J
        W = torch.empty((G, G), dtype=torch.float64, device=dev)
        ws = torch.empty(fcfs.haar_workspace_size(clip.V, clip.T, J), dtype=torch.uint8, device=dev)
        ms = _timed_ms(torch, lambda: fcfs.haar(x, y, s, clip.T, J, out=W, workspace=ws, stream=stream),
                       10 if J <= 12 else 3, flush, stream)
        alg = 9.0 * clip.V + 8.0 * G * G
        elem = 4.0 if (clip.T >> J) <= 1024 else 8.0
        moved = (3.0 * elem + 8.0) * G * G + 9.0 * clip.V
        d = {"V": clip.V, "T": clip.T, "J": J, "value": G * G / (ms * 1e-3), "ms": ms,
             "algorithmic_bytes": alg, "achieved_gbs": alg / (ms * 1e-3) / 1e9,
             "frac_of_hbm_peak": alg / (ms * 1e-3) / 1e9 / peak,
             "moved_bytes_est": moved, "moved_gbs_est": moved / (ms * 1e-3) / 1e9}
        if J == 12:
            d["_check"] = (clip, W)
        res[key] = d
    return res


def extras_accuracy(line, extras):
    """Errors of the extra workloads against the oracle (CPU leg); strips the
    bookkeeping fields from the reported objects."""
    import numpy as np
    import oracle
    if "adjoint" in extras:
        clip, tgt, K, G, gx, gy, gx16, gy16 = extras["adjoint"].pop("_check")
        rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, clip.T, K, G.astype(np.complex128))

        def rel(a, b_, c, d):
            return max(float(np.max(np.abs(a - c)) / np.max(np.abs(c))), float(np.max(np.abs(b_ - d)) / np.max(np.abs(d))))
        line["adjoint"]["max_rel_err"] = rel(gx16, gy16, rx, ry)
        line["adjoint"]["fp32"]["max_rel_err"] = rel(gx, gy, rx, ry)
    if "batch" in extras:
        clips, K, Fb, Ab = extras["batch"].pop("_check")
        Fb = Fb.cpu().numpy()
        Ab = Ab.cpu().numpy()
        order = np.argsort([c.V for c in clips])
        worst = 0.0
        for c in order[[0, 255, 511]]:
            A = oracle.area_exact(clips[c].x, clips[c].y, clips[c].s, clips[c].T)
            Fo = oracle.block(clips[c].x, clips[c].y, clips[c].s, clips[c].T, K)
            worst = max(worst, float(np.max(np.abs(Fb[c] - Fo)) / A))
        line["batch"]["max_abs_err_over_area_sampled"] = worst
        line["batch"]["areas_exact"] = bool(all(int(Ab[c]) == oracle.area_exact(cl.x, cl.y, cl.s, cl.T)
                                                for c, cl in enumerate(clips)))
    if "cosine" in extras:
        for key, d in line["cosine"].items():
            if not isinstance(d, dict):
                continue
            clip, K = d.pop("_clip"), d["K"]
            Aexact = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
            if K <= 256:
                pick = np.arange(K + 1)
                sampled = False
            else:
                pick = np.unique(np.concatenate([[0, 1, 2, K - 1, K], np.random.default_rng(6).integers(0, K + 1, 20)]))
                sampled = True
            Co = oracle.cosine_entries(clip.x, clip.y, clip.s, clip.T, pick, pick)
            for prec in ("split_f16", "fp32"):
                e = d[prec]
                C = e.pop("_C").cpu().numpy().astype(np.float64)[np.ix_(pick, pick)]
                e["max_abs_err_over_area" + ("_sampled" if sampled else "")] = float(np.max(np.abs(C - Co)) / Aexact)
                e["area_exact"] = int(e.pop("_A").item()) == Aexact
    if "haar" in extras:
        import time as _t
        from oracle import haar as _haar
        d = line["haar"]["clip_T4096_J12"]
        clip, W = d.pop("_check")
        # the oracle (per-polygon pruned recursion) on the first 200 polygons;
        # its cost is linear in the polygons, so the full clip takes about 10x
        n_s = 200
        sub = clip.poly_offsets[:n_s + 1]
        t0 = _t.perf_counter()
        _haar.pcht(clip.x[:sub[-1]], clip.y[:sub[-1]], sub, clip.T, 12)
        dt = _t.perf_counter() - t0
        d["cpu_oracle"] = {"kind": "oracle", "cores": 1, "sample": "first %d of %d polygons, J = 12" % (n_s, clip.n_polys),
                           "value": (1 << 24) / (dt * clip.n_polys / n_s), "unit": "coefficients/s",
                           "seconds_sample": dt}
        Wg = W.cpu().numpy()
        A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
        d["parseval_rel_err"] = abs(float(np.sum(Wg * Wg)) - A) / A
        d["scaling_coefficient_exact"] = bool(Wg[0, 0] == A / clip.T)
    if "large" in extras:
        clip5, K5 = extras["large"].pop("_check")
        A = oracle.area_exact(clip5.x, clip5.y, clip5.s, clip5.T)
        pick = np.unique(np.array([0, 1, -1, 2, -2, 7, -13, 100, -333, 512, K5, -K5, K5 - 1]))
        Fo = oracle.block_entries(clip5.x, clip5.y, clip5.s, clip5.T, pick, pick)
        for prec in ("split_f16", "fp32"):
            d = line["large"][prec]
            F5 = d.pop("_F").cpu().numpy()[np.ix_(pick + K5, pick + K5)]
            d["max_abs_err_over_area_sampled"] = float(np.max(np.abs(F5 - Fo)) / A)
            d["area_exact"] = int(d.pop("_A").item()) == A
        d = line["large"]["adjoint_fp32"]
        G5 = d.pop("_G").cpu().numpy().astype(np.complex128)
        idx = np.sort(np.random.default_rng(55).choice(clip5.V, 32, replace=False))
        rx, ry = oracle.vertex_gradient(clip5.x[idx], clip5.y[idx], clip5.s[idx], clip5.T, K5, G5)
        for key in ("adjoint_fp32", "adjoint_split_f16"):
            d = line["large"][key]
            gx5, gy5 = (t.cpu().numpy().astype(np.float64) for t in d.pop("_g"))
            d["max_rel_err_sampled"] = max(float(np.max(np.abs(gx5[idx] - rx)) / np.max(np.abs(rx))),
                                           float(np.max(np.abs(gy5[idx] - ry)) / np.max(np.abs(ry))))


def run_only(args):
    """One workload, warmup + steps calls, for profiler command lines."""
    import torch
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    from synth import config_clip, config4_target, batch_clips, concat_clips
    dev = torch.device("cuda", 0)
    if args.no_pair:
        fcfs.set_pair(0)
    if args.no_fuse:
        fcfs.set_fuse(0)
    if args.only in ("haar", "haar_large"):
        clip, _ = config_clip(2 if args.only == "haar" else 5)
        x, y, s = (torch.from_numpy(a).to(dev) for a in (clip.x, clip.y, clip.s))
        J = 12 if args.only == "haar" else 14
        fn = lambda: fcfs.haar(x, y, s, clip.T, J)
    elif args.only in ("cosine", "cosine_large"):
        clip, K = config_clip(2) if args.only == "cosine" else cosine_large_clip()
        x, y, s = (torch.from_numpy(a).to(dev) for a in (clip.x, clip.y, clip.s))
        fn = lambda: fcfs.cosine(x, y, s, clip.T, K, prec=args.prec)
    elif args.only in ("step", "large", "adjoint", "adjoint_large"):
        clip, K = config_clip({"step": 2, "large": 5, "adjoint": 4, "adjoint_large": 5}[args.only])
        x, y, s = (torch.from_numpy(a).to(dev) for a in (clip.x, clip.y, clip.s))
        if args.only.startswith("adjoint"):
            gen = torch.Generator(device="cpu").manual_seed(7)
            G = torch.randn((2 * K + 1, 2 * K + 1), dtype=torch.complex64, generator=gen).to(dev)
            fn = lambda: fcfs.adjoint(x, y, s, clip.T, K, G, prec=args.prec)
        else:
            fn = lambda: fcfs.forward(x, y, s, clip.T, K, prec="split_f16")
    else:
        clips, K = batch_clips()
        x, y, s, off = (torch.from_numpy(a).to(dev) for a in concat_clips(clips))
        fn = lambda: fcfs.batch(x, y, s, off, clips[0].T, K, prec="split_f16")
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fn()
    torch.cuda.synchronize()
    print(json.dumps({"only": args.only, "steps": args.steps,
                      "ms_per_call": 1e3 * (time.perf_counter() - t0) / max(1, args.steps)}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

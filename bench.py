#!/usr/bin/env python3
"""Throughput of the FCFS block transform on GB300, one JSON line on stdout.

Step: one forward block F(k,l), |k|,|l| <= 256, of the synthetic Manhattan clip
T=4096 with 2000 polygons (~12.6k signed corners), through the C ABI on the
split-FP16 tensor-core path: tables, exact area and axis lines, tcgen05
contraction, FP64 split-K reduction and epilogue (four kernels).
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
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


def traffic_per_launch():
    """DRAM bytes per launch of the contraction kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        src = open(os.path.join(ROOT, "paper_1010_5562_gb300", "csrc", "fcfs_tc.cu"), "rb").read()
        h = hashlib.sha256(src).hexdigest()[:16]
        txt = open(TRAFFIC_FILE).read()
        got = {}
        for line in txt.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                got[k.strip().strip("-* `")] = v.strip().strip("`")
        if got.get("source_sha256_16") == h:
            return float(got["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


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
    sampler = ClockSampler(gpu_index_for_smi(local)) if rank == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    l0 = fcfs.launch_count()
    ms = timed(args.steps, step)
    launches = fcfs.launch_count() - l0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop() if sampler else None
    total_ms = sum(ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * n_terms * args.steps / (total_ms * 1e-3)

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
                "kernel": "gemm_tc_kernel<256,2,full> (tcgen05 split-FP16 contraction)",
                "kernel_ms": gemm_ms, "peak_source": "%s bf16 dense burst (fp16 same rate)" % peak_kind,
                "issued_tflops": issued_flops / (gemm_ms * 1e-3) / 1e12,
                "issued_frac": issued_flops / (gemm_ms * 1e-3) / 1e12 / peak_tf,
                "stage_ms": {"prep": stage_ms[0], "axis": stage_ms[1], "contraction": stage_ms[2],
                             "reduce": stage_ms[3]}}

    # ---- plain FP32 path on the same clip ----
    ms32 = timed(min(args.steps, 1000), lambda: step("fp32"))
    value32 = world * n_terms / (statistics.mean(ms32) * 1e-3)

    # ---- end to end: pinned host inputs in, block out ----
    hx = torch.from_numpy(clip.x).pin_memory()
    hy = torch.from_numpy(clip.y).pin_memory()
    hs = torch.from_numpy(clip.s).pin_memory()
    hF = torch.empty((W, W), dtype=torch.complex64).pin_memory()
    ha = torch.empty((1,), dtype=torch.int64).pin_memory()

    def e2e_step():
        x.copy_(hx, non_blocking=True)
        y.copy_(hy, non_blocking=True)
        s.copy_(hs, non_blocking=True)
        step()
        hF.copy_(F, non_blocking=True)
        ha.copy_(area, non_blocking=True)

    for _ in range(5):
        e2e_step()
    mse = timed(min(args.steps, 1000), e2e_step)
    e2e = {"value": world * n_terms / (statistics.mean(mse) * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": int(V * (4 + 4 + 1)), "d2h_bytes_per_step": int(W * W * 8 + 8)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic (seeded Manhattan clip; stands in for the paper's proprietary 22 nm layout)",
        "config": {"workload": WORKLOAD, "precision": "split_f16 (hi+lo FP16 operands, FP32 accumulate, "
                   "FP64 split-K sum)", "T": T, "K": K, "V": V,
                   "l2": "flushed before every timed step (256 MiB write, outside the events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "plain_fp32": {"value": value32, "unit": UNIT, "ms_per_step": statistics.mean(ms32)},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
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
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

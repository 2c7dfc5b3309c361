#!/usr/bin/env python3
"""Throughput of the FCFS block transform on GB300, one JSON line on stdout.

Step: one forward block F(k,l), |k|,|l| <= 1024, of the synthetic Manhattan
clip T=65536 with 150000 polygons (945450 signed corners), and one adjoint of
that block (the derivative of every corner for a seeded complex cotangent over
the whole block), through the C ABI on the split-FP16 precision class (the
library picks its fastest form per call: the forward groups the corners by y
and takes a pruned FFT along y, the adjoint groups them by y and by x for its
tensor-core contraction).  Metric: vertex-coefficient terms per second,
2 V (2K+1)^2 per step (the adjoint counts the forward's terms).

Default run: N=1, warm-up 5, 20 timed steps; the workspaces (over 1 GB)
exceed L2 and L2 is also flushed (a 256 MiB write) before every timed step,
outside the timed events.  Under torchrun each rank runs its own replica of
the clip on its own GPU (no collective; weak scaling); rank 0 prints the line.

--impl reference times the FP64 oracle instead (the plain CPU implementation
of the definition, on the host cores), on a bounded sample of the same step.
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
WORKLOAD = ("clip T=65536, 150000 rectilinear polygons (rect/L/T/U/plus/stair, sides 20-166), V=945450 signed "
            "corners, K=1024 (2049x2049 complex64 block); step = forward block + adjoint (corner derivatives "
            "for a seeded complex cotangent over the block)")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "gemm_tc_T4096_K256.md")
FALLBACK_BF16_TFLOPS = 1900.0
FALLBACK_HBM_GBS = 6800.0
SMS, FP32_LANES = 152, 128   # GB300: SMs, FP32 lanes per SM (the FP32 FMA peak)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (adjoint, batch, T=4096 clip, forms, cosine, Haar, crossover)")
    ap.add_argument("--no-pair", action="store_true",
                    help="--only: one-CTA tiles instead of CTA pairs (profiling)")
    ap.add_argument("--no-fuse", action="store_true",
                    help="--only: separate axis and reduce kernels (profiling)")
    ap.add_argument("--prec", choices=["split_f16", "fp32"], default="split_f16",
                    help="--only adjoint / adjoint_large / cosine / cosine_large: contraction precision")
    ap.add_argument("--only", choices=["step", "clip4096", "large", "batch", "adjoint", "adjoint_large", "cosine",
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
    return config_clip(5)


def cotangent(K):
    """The seeded cotangent of the step's adjoint: standard complex normal over the block."""
    import numpy as np
    W = 2 * K + 1
    rng = np.random.default_rng(5)
    return (rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))).astype(np.complex64)


def terms(clip, K):
    """Terms of one step: the forward's V (2K+1)^2 and the adjoint's as many."""
    return 2 * clip.V * (2 * K + 1) ** 2


# ---------------------------------------------------------------------------
# the oracle as CPU baseline (the only place bench.py runs oracle/)
# ---------------------------------------------------------------------------
SAMPLE_N = 24   # frequencies per axis of one oracle sample's sub-block of F


def sample_corners(clip, K):
    """Corners of one sample's adjoint half: as many terms as its forward half."""
    return max(1, int(round(SAMPLE_N * SAMPLE_N * clip.V / (2 * K + 1) ** 2)))


def oracle_sample(clip, K, G, i):
    """The i-th bounded sample of the step on the oracle: a SAMPLE_N x SAMPLE_N
    sub-block of F (seeded rows and columns; the first sample holds 0, +-1 and
    +-K on both axes) and the derivatives of sample_corners() seeded corners for
    the full cotangent (both halves have SAMPLE_N^2 V terms).
    Returns (rows, cols, F sub-block, corner indices, gx, gy, terms)."""
    import numpy as np
    import oracle
    W = 2 * K + 1
    rng = np.random.default_rng(100 + i)
    f = np.arange(-K, K + 1)
    if i == 0:
        fixed = np.array([0, 1, -1, K, -K])
        rest = rng.choice(np.setdiff1d(f, fixed), 2 * (SAMPLE_N - fixed.size), replace=False)
        rows = np.sort(np.concatenate([fixed, rest[:SAMPLE_N - fixed.size]]))
        cols = np.sort(np.concatenate([fixed, rest[SAMPLE_N - fixed.size:]]))
    else:
        rows = np.sort(rng.choice(f, SAMPLE_N, replace=False))
        cols = np.sort(rng.choice(f, SAMPLE_N, replace=False))
    nc = sample_corners(clip, K)
    idx = np.sort(rng.choice(clip.V, nc, replace=False))
    Fr = oracle.block_entries(clip.x, clip.y, clip.s, clip.T, rows, cols)
    gx, gy = oracle.vertex_gradient(clip.x[idx], clip.y[idx], clip.s[idx], clip.T, K, G.astype(np.complex128))
    return rows, cols, Fr, idx, gx, gy, SAMPLE_N * SAMPLE_N * clip.V + nc * W * W


def cpu_baseline(clip, K, G, seconds):
    """Oracle samples of the step, repeated for about `seconds` of CPU time."""
    t0 = time.perf_counter()
    n_terms = 0
    samples = []
    while True:
        r = oracle_sample(clip, K, G, len(samples))
        samples.append(r)
        n_terms += r[6]
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    info = {"value": n_terms / el, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": ("%d samples in %.1f s, each a %dx%d sub-block of the 2049x2049 forward block and the "
                       "derivatives of %d corners (adjoint, full cotangent) of the T=65536 clip (FP64 numpy, "
                       "BLAS matmul)" % (len(samples), el, SAMPLE_N, SAMPLE_N, len(samples[0][3])))}
    return info, samples


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    clip, K = workload()
    G = cotangent(K)
    for i in range(args.warmup):
        oracle_sample(clip, K, G, i)
    t0 = time.perf_counter()
    n_terms = 0
    for i in range(args.steps):
        n_terms += oracle_sample(clip, K, G, args.warmup + i)[6]
    el = time.perf_counter() - t0
    value = n_terms / el
    cores = host_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (host)",
                                        "sample_per_step": "a %dx%d sub-block of F + the adjoint of %d corners"
                                                           % (SAMPLE_N, SAMPLE_N, sample_corners(clip, K))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step: a %dx%d sub-block of F and the derivatives of %d corners (FP64 numpy)"
                                   % (SAMPLE_N, SAMPLE_N, sample_corners(clip, K))},
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


# committed ncu summaries that carry per-launch DRAM traffic: stage -> (file,
# kernel line tag, the sources the kernel is built from)
STAGE_TRAFFIC = {
    "h_poly": ("step_T65536_K1024.md", "hyb_h_kernel<1>", ("fcfs_hybrid.cu", "fcfs_fft.cuh", "fcfs_common.cuh")),
    "fft_y": ("step_T65536_K1024.md", "fft_y_fused_kernel", ("fcfs_fft.cu", "fcfs_fft.cuh", "fcfs_common.cuh")),
    "adj_fft": ("step_T65536_K1024.md", "adj_fft_kernel<11>", ("fcfs_adjoint_fft.cu", "fcfs_fft.cuh", "fcfs_common.cuh")),
    "adj_dot": ("step_T65536_K1024.md", "adj_dot_kernel", ("fcfs_adjoint_fft.cu", "fcfs_fft.cuh", "fcfs_common.cuh")),
}


def stage_traffic(stage):
    """DRAM bytes per launch of a stage's kernel from its committed ncu summary,
    if the summary was taken on the kernel's current sources, else None."""
    import re
    if stage not in STAGE_TRAFFIC:
        return None
    fname, tag, srcs = STAGE_TRAFFIC[stage]
    try:
        h = hashlib.sha256()
        for name in srcs:
            with open(os.path.join(ROOT, "paper_1010_5562_gb300", "csrc", name), "rb") as fh:
                h.update(fh.read())
        for line in open(os.path.join(ROOT, "profiles", fname)):
            if line.startswith("- " + tag + ":"):
                sh = re.search(r"source_sha256_16: `([0-9a-f]+)`", line)
                by = re.search(r"dram_bytes_per_launch: `([0-9]+)`", line)
                if sh and by and sh.group(1) == h.hexdigest()[:16]:
                    return float(by.group(1))
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


def peaks():
    """(bf16 dense TFLOP/s burst, HBM GB/s, SM max MHz, source) from MEASURED_PEAKS.json."""
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return FALLBACK_BF16_TFLOPS, FALLBACK_HBM_GBS, 2070.0, "fallback"


ADJOINT_FORMS = {0: "per_corner", 1: "grouped_tc", 2: "grouped_fft"}
FORM_TEXT = {
    "forward": {"direct": "contraction over the corners (tcgen05, split FP16)",
                "grouped_tc": "corners grouped by y, FP32 pair sums, split-FP16 tcgen05 contraction over y",
                "grouped_fft": "corners grouped by y, FP32 pair sums and pruned FFT along y (FP32 arithmetic)"},
    "adjoint": {"per_corner": "split-FP16 tcgen05 contraction per corner",
                "grouped_tc": "split-FP16 tcgen05 contraction grouped by y and by x",
                "grouped_fft": "corners grouped by y and by x, one input-pruned FFT along the grouped coordinate "
                               "per frequency and one dot per corner (FP32 arithmetic)"},
}


def stage_work(name, clip, K):
    """Roofline of one library stage on the step's clip: (bound, algorithmic work
    per launch, unit of the rate, what the work counts), or None for stages
    that are latency-bound glue (prep, grouping, outputs)."""
    V, T, M2 = float(clip.V), float(clip.T), 2.0 * K
    if name in ("h_poly", "h_rows"):
        return ("alu", 8.0 * V * K, "TFLOP/s",
                "8 FP32 flops per corner-frequency term (form s e^{j 2 pi k x / T} from table values, add it)")
    if name == "fft_y":
        return ("hbm", K * T * 8.0 + 2.0 * K * (2 * K) * 8.0, "GB/s",
                "conj(H) read once (K T complex64) + rows k and -k of the block written once")
    if name == "gemm_y":
        return ("tensor", 2.0 * (T + 1) * M2 * M2, "TFLOP/s", "2 (T+1) (2K)^2: one real MAC per y-frequency term")
    if name in ("gemm_tc", "gemm_tc_fused"):
        return ("tensor", 2.0 * V * M2 * M2, "TFLOP/s", "2 V (2K)^2: one real MAC per corner-coefficient term")
    if name == "adj_tc_grouped":
        return ("tensor", 4.0 * (T + 1) * M2 * M2, "TFLOP/s",
                "2 matrices (gx, gy) x 2 (T+1) (2K)^2: one real MAC per b-value-coefficient term")
    if name == "adj_tc":
        return ("tensor", 4.0 * V * M2 * M2, "TFLOP/s", "2 matrices x 2 V (2K)^2")
    if name == "adj_fft":
        return ("hbm", 2.0 * T * (K + 1) * 8.0 + 2.0 * (2 * K + 1) ** 2 * 8.0, "GB/s",
                "V_k(b) of both matrices written once (2 T (K+1) complex64) + the cotangent read once per matrix")
    if name == "adj_dot":
        return ("alu", 10.0 * 2.0 * V * (K + 1), "TFLOP/s",
                "10 FP32 flops per corner-frequency term, 2 V (K+1) terms (E_k(a) by one complex rotation, "
                "Re(E_k V_k) accumulated)")
    if name == "axis_lines":
        return ("alu", 4.0 * K * (T + 1), "Tops/s", "4 K (T+1) exact integer MACs (the two axis lines)")
    return None


def roofline_of(stages, clip, K):
    """The dominant stage of the step (largest mean time) against its roofline."""
    bf16, hbm, mhz, src = peaks()
    fp32 = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
    ranked = sorted(stages.items(), key=lambda kv: -kv[1])
    name, ms = ranked[0]
    w = stage_work(name, clip, K)
    out = {"kernel": name, "kernel_ms": ms,
           "stage_ms": {k: round(v, 4) for k, v in ranked}}
    if w is None:
        out.update({"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None})
        return out
    bound, work, unit, what = w
    if bound == "tensor":
        peak, psrc = bf16, "%s bf16 dense burst (fp16 same rate)" % src
        achieved = work / (ms * 1e-3) / 1e12
        out["issued_tflops"] = 3.0 * achieved     # hi*hi + hi*lo + lo*hi
        out["issued_frac"] = 3.0 * achieved / peak
    elif bound == "hbm":
        peak, psrc = hbm, "%s STREAM-style copy" % src
        achieved = work / (ms * 1e-3) / 1e9
    else:
        peak = fp32
        psrc = "derived: %d SMs x %d FP32 lanes x 2 flops x %.0f MHz (%s SM max clock)" % (SMS, FP32_LANES, mhz, src)
        achieved = work / (ms * 1e-3) / 1e12
    out.update({"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": stage_traffic(name), "work": what, "peak_source": psrc})
    return out


def run_ours(args):
    import numpy as np
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
    lib = fcfs._lib.load()

    clip, K = workload()
    T, V = clip.T, clip.V
    W = 2 * K + 1
    n_terms = terms(clip, K)
    Gh = cotangent(K)
    x = torch.from_numpy(clip.x).to(dev)
    y = torch.from_numpy(clip.y).to(dev)
    s = torch.from_numpy(clip.s).to(dev)
    G = torch.from_numpy(Gh).to(dev)
    F = torch.empty((W, W), dtype=torch.complex64, device=dev)
    area = torch.empty((1,), dtype=torch.int64, device=dev)
    gx = torch.empty(V, dtype=torch.float32, device=dev)
    gy = torch.empty_like(gx)
    ws = torch.empty(fcfs.workspace_size(V, T, K, "split_f16"), dtype=torch.uint8, device=dev)
    wsa = torch.empty(lib.fcfs_adjoint_workspace_size(V, T, K, 1), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        fcfs.forward(x, y, s, T, K, prec="split_f16", out=F, area_out=area, workspace=ws, stream=stream)
        fcfs.adjoint(x, y, s, T, K, G, prec="split_f16", gx=gx, gy=gy, workspace=wsa, stream=stream)

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
    torch.cuda.synchronize(dev)

    # ---- main timed region ----
    # The clock samples are taken while the same step keeps the GPU busy for a
    # few sampling periods before and after the timed steps.
    def keep_busy(seconds):
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            for _ in range(4):
                flush.fill_(1)
                step()
            torch.cuda.synchronize(dev)

    sampler = ClockSampler(gpu_index_for_smi(local)) if rank == 0 else None
    if sampler:
        sampler.start()
        keep_busy(0.4)
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
        keep_busy(0.4)
    clocks = sampler.stop() if sampler else None
    if clocks is not None:
        clocks["window"] = "nvidia-smi every 100 ms, the step running 0.4 s before and after the timed steps"
    value, total_ms = whole_job_rate(sum(ms), n_terms, args.steps, world, dev)

    # ---- per-stage times (events around each library stage, separate pass) ----
    reps = 3
    acc = {}
    fwd_ms = adj_ms = 0.0
    fcfs.set_overlap(False)   # each stage alone on the call's stream
    for _ in range(reps):
        flush.fill_(1)
        fcfs.kernel_timing_enable(True)
        step()
        for name, t in fcfs.kernel_timing():
            acc[name] = acc.get(name, 0.0) + t / reps
            if name.startswith("adj_"):
                adj_ms += t / reps
            else:
                fwd_ms += t / reps
    fcfs.kernel_timing_enable(False)
    fcfs.set_overlap(True)
    roofline = roofline_of(acc, clip, K)
    forms = {0: "direct", 1: "grouped_tc", 2: "grouped_fft"}
    parts = {"forward": {"form": forms.get(fcfs.forward_grouped(V, T, K), "?"), "stages_ms": round(fwd_ms, 4),
                         "value": V * W * W / (fwd_ms * 1e-3)},
             "adjoint": {"form": ADJOINT_FORMS.get(fcfs.adjoint_grouped(V, T, K), "?"),
                         "stages_ms": round(adj_ms, 4), "value": V * W * W / (adj_ms * 1e-3)}}

    # ---- plain FP32 on the same clip (forward and adjoint) ----
    F32 = torch.empty_like(F)
    gx32 = torch.empty_like(gx)
    gy32 = torch.empty_like(gx)
    ws32 = torch.empty(fcfs.workspace_size(V, T, K, "fp32"), dtype=torch.uint8, device=dev)
    wsa32 = torch.empty(lib.fcfs_adjoint_workspace_size(V, T, K, 0), dtype=torch.uint8, device=dev)

    def step32():
        fcfs.forward(x, y, s, T, K, prec="fp32", out=F32, area_out=area, workspace=ws32, stream=stream)
        fcfs.adjoint(x, y, s, T, K, G, prec="fp32", gx=gx32, gy=gy32, workspace=wsa32, stream=stream)

    step32()
    ms32 = timed(2, step32)
    value32 = world * n_terms / (statistics.mean(ms32) * 1e-3)

    # ---- end to end: pinned host inputs in, block and derivatives out ----
    # x, y, s and the cotangent travel in one pinned staging buffer (16-byte
    # aligned views on both sides); F, the area and the derivatives come back as
    # one block: one copy each way per step.
    a16 = lambda n: (n + 15) // 16 * 16
    ox, oy, osg = 0, a16(4 * V), 2 * a16(4 * V)
    og = osg + a16(V)
    nin = og + W * W * 8
    hin = torch.zeros(nin, dtype=torch.uint8).pin_memory()
    hin[ox:ox + 4 * V].copy_(torch.from_numpy(clip.x).view(torch.uint8))
    hin[oy:oy + 4 * V].copy_(torch.from_numpy(clip.y).view(torch.uint8))
    hin[osg:osg + V].copy_(torch.from_numpy(clip.s).view(torch.uint8))
    hin[og:].copy_(torch.from_numpy(Gh).view(torch.uint8).reshape(-1))
    of, oa, ogx = 0, W * W * 8, W * W * 8 + 16
    ogy = ogx + a16(4 * V)
    nout = ogy + a16(4 * V)
    Fref, gxref, gyref = F.cpu(), gx.cpu(), gy.cpu()

    def make_set():
        d_in = torch.empty(nin, dtype=torch.uint8, device=dev)
        d_out = torch.empty(nout, dtype=torch.uint8, device=dev)
        return dict(din=d_in, dout=d_out, ws=torch.empty_like(ws), wsa=torch.empty_like(wsa),
                    hout=torch.empty(nout, dtype=torch.uint8).pin_memory(),
                    x=d_in[ox:ox + 4 * V].view(torch.int32), y=d_in[oy:oy + 4 * V].view(torch.int32),
                    s=d_in[osg:osg + V].view(torch.int8), G=d_in[og:].view(torch.complex64).view(W, W),
                    F=d_out[of:of + W * W * 8].view(torch.complex64).view(W, W),
                    a=d_out[oa:oa + 8].view(torch.int64), gx=d_out[ogx:ogx + 4 * V].view(torch.float32),
                    gy=d_out[ogy:ogy + 4 * V].view(torch.float32))

    def run_set(b, st):
        b["din"].copy_(hin, non_blocking=True)
        fcfs.forward(b["x"], b["y"], b["s"], T, K, prec="split_f16", out=b["F"], area_out=b["a"],
                     workspace=b["ws"], stream=st)
        fcfs.adjoint(b["x"], b["y"], b["s"], T, K, b["G"], prec="split_f16", gx=b["gx"], gy=b["gy"],
                     workspace=b["wsa"], stream=st)
        b["hout"].copy_(b["dout"], non_blocking=True)

    def same(b):
        h = b["hout"]
        return (torch.equal(h[of:of + W * W * 8].view(torch.complex64).view(W, W), Fref)
                and torch.equal(h[ogx:ogx + 4 * V].view(torch.float32), gxref)
                and torch.equal(h[ogy:ogy + 4 * V].view(torch.float32), gyref))

    one = make_set()
    for _ in range(2):
        run_set(one, stream)
    mse = timed(min(args.steps, 10), lambda: run_set(one, stream))
    torch.cuda.synchronize(dev)
    e2e_ok = bool(same(one))
    # Pipelined: steps alternate between two streams, so one step's copies run on
    # the copy engines while the other computes; sets are reused on the same
    # stream only (no race), and together they exceed L2.
    n_sets = 2
    sets = [one, make_set()]
    lanes = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]

    def e2e_pipelined(n):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for ln in lanes:
            ln.wait_stream(stream)
        for i in range(n):
            ln, b = lanes[i % 2], sets[i % n_sets]
            with torch.cuda.stream(ln):
                run_set(b, ln)
        for ln in lanes:
            stream.wait_stream(ln)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        return t0.elapsed_time(t1) / n

    e2e_pipelined(4)
    ms_pipe = e2e_pipelined(max(4, min(args.steps, 20)))
    pipe_ok = all(same(b) for b in sets)
    set_bytes = nin + nout + ws.numel() + wsa.numel()
    e2e = {"value": world * n_terms / (ms_pipe * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": int(nin), "d2h_bytes_per_step": int(nout),
           "copies": ("every step: one H2D of x, y, s and the cotangent from pinned host memory and one D2H "
                      "of F, the area and both derivatives; steps alternate between two streams so copies "
                      "overlap the other step's compute; %d buffer sets (%.0f MB each)"
                      % (n_sets, set_bytes / 1e6)),
           "ms_per_step": ms_pipe, "matches_device_step": bool(e2e_ok and pipe_ok),
           "serial": {"value": world * n_terms / (statistics.mean(mse) * 1e-3), "ms_per_step": statistics.mean(mse),
                      "note": "one stream, events around each step, L2 flushed between steps"}}
    del sets, one

    extras = {} if (world > 1 or args.no_extras) else run_extras(fcfs, dev, flush, stream, args)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Manhattan clip; stands in for the paper's proprietary 22 nm layout)",
        "config": {"workload": WORKLOAD,
                   "precision": ("split_f16 class (max|dF|/area <= 1e-5): the library's fastest form per call; "
                                 "forward: %s; adjoint: %s" % (FORM_TEXT["forward"].get(parts["forward"]["form"], "?"),
                                                              FORM_TEXT["adjoint"].get(parts["adjoint"]["form"], "?"))),
                   "T": T, "K": K, "V": V,
                   "l2": "workspaces exceed L2, and L2 is flushed before every timed step (256 MiB write, "
                         "outside the events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "parts": parts,
        "plain_fp32": {"value": value32, "unit": UNIT, "ms_per_step": statistics.mean(ms32),
                       "forward_form": forms.get(fcfs.forward_grouped(V, T, K, prec="fp32"), "?"),
                       "adjoint_form": ADJOINT_FORMS.get(fcfs.adjoint_grouped(V, T, K, prec="fp32"), "?")},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    for k in ("adjoint", "batch", "clip_T4096", "large", "cosine", "haar", "crossover"):
        if k in extras:
            line[k] = extras[k]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, samples = cpu_baseline(clip, K, Gh, args.cpu_seconds)
        line["cpu_baseline"] = cb
        import oracle
        A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
        Fg, F32g = F.cpu().numpy().astype(np.complex128), F32.cpu().numpy().astype(np.complex128)
        gxs, gys = gx.cpu().numpy().astype(np.float64), gy.cpu().numpy().astype(np.float64)
        gx3, gy3 = gx32.cpu().numpy().astype(np.float64), gy32.cpu().numpy().astype(np.float64)
        err_f = err_f32 = err_g = err_g32 = 0.0
        for rows, cols, Fr, idx, ox_, oy_, _ in samples:
            sub = np.ix_(rows + K, cols + K)
            err_f = max(err_f, float(np.max(np.abs(Fg[sub] - Fr)) / A))
            err_f32 = max(err_f32, float(np.max(np.abs(F32g[sub] - Fr)) / A))
            sc = max(float(np.max(np.abs(ox_))), float(np.max(np.abs(oy_))))
            err_g = max(err_g, float(max(np.max(np.abs(gxs[idx] - ox_)), np.max(np.abs(gys[idx] - oy_)))) / sc)
            err_g32 = max(err_g32, float(max(np.max(np.abs(gx3[idx] - ox_)), np.max(np.abs(gy3[idx] - oy_)))) / sc)
        line["accuracy"] = {
            "forward_max_abs_err_over_area_sampled": err_f, "fp32_forward_max_abs_err_over_area_sampled": err_f32,
            "adjoint_max_rel_err_sampled": err_g, "fp32_adjoint_max_rel_err_sampled": err_g32,
            "area_exact": int(area.item()) == A,
            "sample": "the oracle samples of cpu_baseline: sub-blocks of F and the derivatives of their corners",
            "reference": "FP64 oracle (direct signed-quadrant vertex sum and its derivative)"}
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
                      "precision": "split_f16 class (%s)" % ADJOINT_FORMS.get(fcfs.adjoint_grouped(clip.V, T, K), "?"),
                      "fp32": {"value": clip.V * W * W / (ms * 1e-3), "ms": ms},
                      "_check": (clip, tgt, K, G.cpu().numpy(), gx.cpu().numpy(), gy.cpu().numpy(),
                                 gx16.cpu().numpy(), gy16.cpu().numpy())}

    # batch: workload 3, one launch replayed from a CUDA graph vs one call per clip
    clips, K = batch_clips()
    T, W = clips[0].T, 2 * K + 1
    bx, by, bs, boff = (torch.from_numpy(a).to(dev) for a in concat_clips(clips))
    n = len(clips)
    terms_b = float(sum(c.V for c in clips)) * W * W
    plan = autotune.tune_batch(bx, by, bs, boff, T, K, prec="split_f16")
    Fb = torch.empty((n, W, W), dtype=torch.complex64, device=dev)
    Ab = torch.empty(n, dtype=torch.int64, device=dev)
    wsb = torch.empty(plan.workspace_size(), dtype=torch.uint8, device=dev)
    cap = torch.cuda.Stream(dev)   # graphs are captured on a side stream
    with torch.cuda.stream(cap):
        plan.batch(bx, by, bs, boff, out=Fb, area_out=Ab, workspace=wsb, stream=cap)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        plan.batch(bx, by, bs, boff, out=Fb, area_out=Ab, workspace=wsb, stream=cap)
    ms_b = _timed_ms(torch, g.replay, 5, flush, stream)
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
                    "plan": plan.knobs(), "launch": "one fcfs_plan_batch call replayed from a CUDA graph",
                    "_check": (clips, K, Fb, Ab)}

    # large clip (the step's clip): every forward form, forced
    clip5, K5 = config_clip(5)
    W5 = 2 * K5 + 1
    x5, y5, s5 = (torch.from_numpy(a).to(dev) for a in (clip5.x, clip5.y, clip5.s))
    forms = {}
    for mode, key, prec in ((0, "direct_tc", "split_f16"), (2, "grouped_tc", "split_f16"),
                            (3, "grouped_fft", "split_f16")):
        fcfs.set_hybrid(mode)
        try:
            F5 = torch.empty((W5, W5), dtype=torch.complex64, device=dev)
            A5 = torch.empty(1, dtype=torch.int64, device=dev)
            ws5 = torch.empty(fcfs.workspace_size(clip5.V, clip5.T, K5, prec), dtype=torch.uint8, device=dev)
            fn = lambda: fcfs.forward(x5, y5, s5, clip5.T, K5, prec=prec, out=F5, area_out=A5, workspace=ws5,
                                      stream=stream)
            ms5 = _timed_ms(torch, fn, 3, flush, stream)
            flush.fill_(1)
            fcfs.set_overlap(False)   # each stage alone on the call's stream
            fcfs.kernel_timing_enable(True)
            fn()
            kt = fcfs.kernel_timing()
            fcfs.kernel_timing_enable(False)
            fcfs.set_overlap(True)
        finally:
            fcfs.set_hybrid(1)
        forms[key] = {"ms": ms5, "value": clip5.V * W5 * W5 / (ms5 * 1e-3),
                      "stages_ms": {n: round(t, 4) for n, t in kt}, "_F": F5, "_A": A5}
    # the same clip's adjoint (the step's cotangent), every form forced
    G5 = torch.from_numpy(cotangent(K5)).to(dev)
    aforms = {}
    for mode, key in ((0, "per_corner_tc"), (2, "grouped_tc"), (3, "grouped_fft")):
        fcfs.set_hybrid(mode)
        try:
            g5x = torch.empty(clip5.V, dtype=torch.float32, device=dev)
            g5y = torch.empty_like(g5x)
            wsa5 = torch.empty(fcfs._lib.load().fcfs_adjoint_workspace_size(clip5.V, clip5.T, K5, 1),
                               dtype=torch.uint8, device=dev)
            fn = lambda: fcfs.adjoint(x5, y5, s5, clip5.T, K5, G5, prec="split_f16", gx=g5x, gy=g5y, workspace=wsa5,
                                      stream=stream)
            ms5 = _timed_ms(torch, fn, 3, flush, stream)
            flush.fill_(1)
            fcfs.set_overlap(False)   # each stage alone on the call's stream
            fcfs.kernel_timing_enable(True)
            fn()
            kt = fcfs.kernel_timing()
            fcfs.kernel_timing_enable(False)
            fcfs.set_overlap(True)
            del wsa5
        finally:
            fcfs.set_hybrid(1)
        aforms[key] = {"ms": ms5, "value": clip5.V * W5 * W5 / (ms5 * 1e-3),
                       "stages_ms": {n: round(t, 4) for n, t in kt}, "_g": (g5x, g5y)}
    out["large"] = {"workload": "clip T=65536, 150000 polygons, V=%d, K=1024 (2049x2049), forward and adjoint "
                                "forms forced one by one (split-FP16 class)" % clip5.V, "unit": UNIT,
                    "auto": {0: "direct_tc", 1: "grouped_tc", 2: "grouped_fft"}[fcfs.forward_grouped(clip5.V, clip5.T, K5)],
                    "forms": forms,
                    "adjoint_auto": ADJOINT_FORMS.get(fcfs.adjoint_grouped(clip5.V, clip5.T, K5), "?"),
                    "adjoint_forms": aforms, "_check": (clip5, K5)}

    # the T = 4096 clip: one forward block (the contraction over its corners)
    clip2, K2 = config_clip(2)
    W2 = 2 * K2 + 1
    x2, y2, s2 = (torch.from_numpy(a).to(dev) for a in (clip2.x, clip2.y, clip2.s))
    F2 = torch.empty((W2, W2), dtype=torch.complex64, device=dev)
    A2 = torch.empty(1, dtype=torch.int64, device=dev)
    d2 = {"workload": "clip T=4096, 2000 polygons, V=%d, K=256 (513x513), forward" % clip2.V, "unit": UNIT}
    for prec in ("split_f16", "fp32"):
        ws2 = torch.empty(fcfs.workspace_size(clip2.V, clip2.T, K2, prec), dtype=torch.uint8, device=dev)
        fn = lambda: fcfs.forward(x2, y2, s2, clip2.T, K2, prec=prec, out=F2, area_out=A2, workspace=ws2,
                                  stream=stream)
        ms2 = _timed_ms(torch, fn, 200, flush, stream)
        st = {}
        for _ in range(20):
            flush.fill_(1)
            fcfs.set_overlap(False)   # each stage alone on the call's stream
            fcfs.kernel_timing_enable(True)
            fn()
            for n, t in fcfs.kernel_timing():
                st[n] = st.get(n, 0.0) + t / 20
        fcfs.kernel_timing_enable(False)
        fcfs.set_overlap(True)
        e = {"ms": ms2, "value": clip2.V * W2 * W2 / (ms2 * 1e-3),
             "form": {0: "direct", 1: "grouped_tc", 2: "grouped_fft"}[fcfs.forward_grouped(clip2.V, clip2.T, K2, prec=prec)],
             "_F": F2.cpu()}
        if prec == "split_f16":
            rf = roofline_of(st, clip2, K2)
            rf["traffic"] = traffic_per_launch()
            e["roofline"] = rf
        else:
            e["stages_ms"] = {n: round(t, 4) for n, t in st.items()}
        d2[prec] = e
    d2["_check"] = clip2, K2
    out["clip_T4096"] = d2
    out["cosine"] = cosine_extras(fcfs, dev, flush, stream)
    out["haar"] = haar_extras(fcfs, dev, flush, stream)
    out["crossover"] = crossover_extras(fcfs, dev, flush, stream)
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
    """Forward with the contraction over the V corners (direct), with the corners
    grouped by y and the split-FP16 contraction over the T + 1 values of y
    (grouped_tc), and with the pruned FFT along y (grouped_fft), across corner
    densities V / (T + 1).  "auto" is the library's automatic choice for the
    sizes (cost estimates of all three)."""
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
        for mode, key in ((0, "direct_ms"), (2, "grouped_tc_ms"), (3, "grouped_fft_ms")):
            fcfs.set_hybrid(mode)
            try:
                ws = torch.empty(fcfs.workspace_size(clip.V, T, K, "split_f16"), dtype=torch.uint8, device=dev)
                r[key] = _timed_ms(torch, lambda: fcfs.forward(x, y, s, T, K, out=F, area_out=A, workspace=ws,
                                                               stream=stream), 10 if T <= 4096 else 3, flush, stream)
            finally:
                fcfs.set_hybrid(1)
        r["auto"] = {0: "direct", 1: "grouped_tc", 2: "grouped_fft"}[fcfs.forward_grouped(clip.V, T, K)]
        r["fastest"] = min(("direct", "grouped_tc", "grouped_fft"), key=lambda f: r[f + "_ms"])
        rows.append(r)
    return {"unit": "ms per forward call (split-FP16 class)", "rows": rows}


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
    (9 B each) plus the FP64 coefficients written once (8 B each).  What the
    pipeline moves: on grids of >= 256 cells a side (the banded kernels, 32-bit
    cells) the coefficients, the band sums (4 B per 32 cells, written, read
    twice by the band scan, written again, read by the bands: 0.5 B per cell)
    and the corners twice (band sums, bands); on smaller grids 3 passes over the
    level-J grid of 4 B (or 8 B) per cell plus the coefficients."""
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
        if G >= 256 and elem == 4.0:
            moved = 8.5 * G * G + 18.0 * clip.V
        else:
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
        for key, d in line["large"]["forms"].items():
            F5 = d.pop("_F").cpu().numpy()[np.ix_(pick + K5, pick + K5)]
            d["max_abs_err_over_area_sampled"] = float(np.max(np.abs(F5 - Fo)) / A)
            d["area_exact"] = int(d.pop("_A").item()) == A
        # adjoint forms: 64 sampled corners against the oracle's derivatives
        rng = np.random.default_rng(64)
        idx = np.sort(rng.choice(clip5.V, 64, replace=False))
        Gq = cotangent(K5).astype(np.complex128)
        rx, ry = oracle.vertex_gradient(clip5.x[idx], clip5.y[idx], clip5.s[idx], clip5.T, K5, Gq)
        sc = max(float(np.max(np.abs(rx))), float(np.max(np.abs(ry))))
        for key, d in line["large"]["adjoint_forms"].items():
            g5x, g5y = (t.cpu().numpy().astype(np.float64)[idx] for t in d.pop("_g"))
            d["max_rel_err_sampled"] = max(float(np.max(np.abs(g5x - rx))), float(np.max(np.abs(g5y - ry)))) / sc
    if "clip_T4096" in extras:
        clip2, K2 = extras["clip_T4096"].pop("_check")
        A = oracle.area_exact(clip2.x, clip2.y, clip2.s, clip2.T)
        Fo = oracle.block(clip2.x, clip2.y, clip2.s, clip2.T, K2)
        for prec in ("split_f16", "fp32"):
            d = line["clip_T4096"][prec]
            d["max_abs_err_over_area"] = float(np.max(np.abs(d.pop("_F").numpy().astype(np.complex128) - Fo)) / A)


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
    elif args.only == "step":   # the benchmark step: forward and adjoint of the large clip
        clip, K = workload()
        x, y, s = (torch.from_numpy(a).to(dev) for a in (clip.x, clip.y, clip.s))
        G = torch.from_numpy(cotangent(K)).to(dev)

        def fn():
            fcfs.forward(x, y, s, clip.T, K, prec="split_f16")
            fcfs.adjoint(x, y, s, clip.T, K, G, prec="split_f16")
    elif args.only in ("clip4096", "large", "adjoint", "adjoint_large"):
        clip, K = config_clip({"clip4096": 2, "large": 5, "adjoint": 4, "adjoint_large": 5}[args.only])
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

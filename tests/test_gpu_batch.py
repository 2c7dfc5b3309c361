"""Batch of clips on the GPU against the FP64 oracle, clip by clip.

Same error measure and bounds as the single-clip forward (max |dF| / area per
clip: 1e-6 plain FP32, 1e-5 split FP16; exact areas).
"""
import numpy as np
import pytest
import torch

import oracle
from synth import make_clip, concat_clips, batch_clips, clip_from_rings, rect_ring

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-6, "split_f16": 1e-5}
PRECS = ["fp32", "split_f16"]


@pytest.fixture(scope="module")
def fc():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import fcfs
    assert torch.cuda.is_available()
    fcfs.set_batch_unit_chunks(0)
    return fcfs


def run_batch(fc, clips, K, prec):
    x, y, s, off = concat_clips(clips)
    d = [torch.from_numpy(a).cuda() for a in (x, y, s, off)]
    F, area = fc.batch(d[0], d[1], d[2], d[3], clips[0].T, K, prec=prec)
    torch.cuda.synchronize()
    return F.cpu().numpy().astype(np.complex128), area.cpu().numpy()


_ORACLE_CACHE = {}


def _oracle_block(clip, K):
    key = (clip.T, K, clip.V, clip.x.tobytes(), clip.y.tobytes(), clip.s.tobytes())
    if key not in _ORACLE_CACHE:   # both precisions compare with the same block
        _ORACLE_CACHE[key] = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    return _ORACLE_CACHE[key]


def check_clip(F, area, clip, K, prec):
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert int(area) == A
    Fo = _oracle_block(clip, K)
    err = np.max(np.abs(F - Fo)) / max(A, 1)
    assert err <= TOL[prec], err


def small_batch():
    empty = clip_from_rings(512, [rect_ring(1, 1, 2, 2)])
    empty.x, empty.y, empty.s = empty.x[:0], empty.y[:0], empty.s[:0]
    return [make_clip(512, n, 800 + n, smin=6, smax=40) for n in (3, 40, 1, 90, 17)] + \
           [empty, make_clip(512, 60, 999, smin=6, smax=40)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("chunks", [0, 1, 3])
def test_small_batch_against_oracle(fc, prec, chunks):
    clips = small_batch()
    fc.set_batch_unit_chunks(chunks)
    try:
        F, area = run_batch(fc, clips, 40, prec)
    finally:
        fc.set_batch_unit_chunks(0)
    for c, clip in enumerate(clips):
        if clip.V == 0:
            assert area[c] == 0 and not np.any(F[c])
        else:
            check_clip(F[c], area[c], clip, 40, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_matches_single_clip_calls(fc, prec):
    clips = small_batch()[:5]
    F, _ = run_batch(fc, clips, 40, prec)
    for c, clip in enumerate(clips):
        x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
        Fs, _ = fc.forward(x, y, s, clip.T, 40, prec=prec)
        A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
        assert np.max(np.abs(F[c] - Fs.cpu().numpy())) / A <= 2 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_config3_full_batch(fc, prec):
    """512 clips, T=2048, V_c log-uniform in [1e3, 1e5], K=128; 64 clips spread
    evenly over the range of V (the smallest and largest included) are checked
    against the oracle element by element, every area exactly."""
    clips, K = batch_clips()
    F, area = run_batch(fc, clips, K, prec)
    for c, clip in enumerate(clips):
        assert int(area[c]) == oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    order = np.argsort([cl.V for cl in clips])
    for c in order[np.unique(np.linspace(0, len(clips) - 1, 64).round().astype(int))]:
        check_clip(F[c], area[c], clips[c], K, prec)


def test_batch_in_cuda_graph(fc):
    clips = small_batch()
    x, y, s, off = (torch.from_numpy(a).cuda() for a in concat_clips(clips))
    K, T = 40, clips[0].T
    W = 2 * K + 1
    F = torch.empty((len(clips), W, W), dtype=torch.complex64, device="cuda")
    area = torch.empty((len(clips),), dtype=torch.int64, device="cuda")
    ws = torch.empty(fc._lib.load().fcfs_batch_workspace_size(x.numel(), len(clips), T, K, 1),
                     dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        fc.batch(x, y, s, off, T, K, out=F, area_out=area, workspace=ws, stream=st)   # warm-up
    torch.cuda.synchronize()
    ref = F.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        fc.batch(x, y, s, off, T, K, out=F, area_out=area, workspace=ws, stream=st)
    F.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(F, ref)


def test_autotune_plans(fc, tmp_path, monkeypatch):
    """The autotuner times knob sets through plans and returns a plan carrying
    the winner (served from its cache the second time); the tuned plan's
    blocks match the automatic call's, and no process-wide hook was changed."""
    from paper_1010_5562_gb300 import autotune
    monkeypatch.setenv("FCFS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    clips = small_batch()[:4]
    T, K = clips[0].T, 40
    x, y, s, off = (torch.from_numpy(a).cuda() for a in concat_clips(clips))
    plan = autotune.tune_batch(x, y, s, off, T, K, reps=1)
    assert plan.get("unit_chunks") in autotune.UNIT_CANDIDATES or plan.get("form") == 1
    assert (tmp_path / "tune.json").exists()
    again = autotune.tune_batch(x, y, s, off, T, K)
    assert again.knobs() == plan.knobs()
    Fp, ap = plan.batch(x, y, s, off)
    Fa, aa = fc.batch(x, y, s, off, T, K)
    assert torch.equal(ap, aa)
    A = [oracle.area_exact(c.x, c.y, c.s, c.T) for c in clips]
    for c in range(len(clips)):
        assert float(torch.max(torch.abs(Fp[c] - Fa[c]))) / max(A[c], 1) <= 2 * TOL["split_f16"]
    v0 = clips[0].V
    fplan = autotune.tune_forward(x[:v0], y[:v0], s[:v0], T, K, reps=1)
    F1, a1 = fplan.forward(x[:v0], y[:v0], s[:v0])
    F0, a0 = fc.forward(x[:v0], y[:v0], s[:v0], T, K)
    assert int(a1) == int(a0) == A[0]
    assert float(torch.max(torch.abs(F1 - F0))) / A[0] <= 2 * TOL["split_f16"]
    lib = fc._lib.load()
    assert lib.fcfs_forward_grouped(12576, 4096, 256, 1) == 0   # the hooks still automatic


@pytest.mark.parametrize("form", [0, 1, 2])
def test_forward_plans_match_oracle(fc, form):
    """Each forward form through a plan, against the oracle; the plan reports
    the form it runs and leaves the process-wide hook alone."""
    clip = make_clip(1024, 200, 31, smin=6, smax=60)
    K = 160
    plan = fc.Plan("forward", clip.V, clip.T, K, "split_f16", form=form, splits=3 if form == 0 else 0)
    assert plan.get("form") == form
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    F, a = plan.forward(x, y, s)
    torch.cuda.synchronize()
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    assert int(a) == A
    Fo = oracle.block(clip.x, clip.y, clip.s, clip.T, K)
    assert np.max(np.abs(F.cpu().numpy() - Fo)) / A <= TOL["split_f16"]
    assert fc.forward_grouped(clip.V, clip.T, K) == fc._lib.load().fcfs_forward_grouped(clip.V, clip.T, K, 1)


def test_adjoint_plan_matches_call(fc):
    clip = make_clip(1024, 100, 32, smin=6, smax=60)
    K = 130
    rng = np.random.default_rng(9)
    W = 2 * K + 1
    G = torch.from_numpy((rng.standard_normal((W, W)) + 1j * rng.standard_normal((W, W))).astype(np.complex64)).cuda()
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    for form in (0, 1, 2):
        plan = fc.Plan("adjoint", clip.V, clip.T, K, "split_f16", form=form)
        assert plan.get("form") == form
        gx, gy = plan.adjoint(x, y, s, G)
        rx, ry = oracle.vertex_gradient(clip.x, clip.y, clip.s, clip.T, K, G.cpu().numpy().astype(np.complex128))
        gx, gy = gx.cpu().numpy(), gy.cpu().numpy()
        err = max(np.max(np.abs(gx - rx)) / np.max(np.abs(rx)), np.max(np.abs(gy - ry)) / np.max(np.abs(ry)))
        assert err <= 1e-5, (form, err)


def run_batch_mode(fc, clips, K, mode):
    fc.set_hybrid(mode)   # the batch sizes its workspace inside the call
    try:
        return run_batch(fc, clips, K, "split_f16")
    finally:
        fc.set_hybrid(1)


@pytest.mark.parametrize("K", [128, 129, 200])
def test_grouped_batch_against_oracle(fc, K):
    """Each clip's corners grouped by y and contracted over its T + 1 values of y
    (one launch per stage for the whole batch), forced on the small batch: an
    empty clip, a one-polygon clip, ragged 2K."""
    clips = small_batch()
    F, area = run_batch_mode(fc, clips, K, 2)
    for c, clip in enumerate(clips):
        if clip.V == 0:
            assert area[c] == 0 and not np.any(F[c])
        else:
            check_clip(F[c], area[c], clip, K, "split_f16")


def test_grouped_batch_matches_direct(fc):
    """24 clips of workload 3 (T=2048, K=128): grouped and direct (unit-list)
    batches agree to FP32 rounding; repeated grouped calls are bit-identical."""
    clips, K = batch_clips(n_clips=24)
    Fg, ag = run_batch_mode(fc, clips, K, 2)
    Fg2, _ = run_batch_mode(fc, clips, K, 2)
    Fd, ad = run_batch_mode(fc, clips, K, 0)
    assert np.array_equal(Fg, Fg2)
    assert np.array_equal(ag, ad)
    for c, clip in enumerate(clips):
        A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
        assert np.max(np.abs(Fg[c] - Fd[c])) / A <= 2e-6


def test_grouped_batch_in_cuda_graph(fc):
    clips = small_batch()
    x, y, s, off = (torch.from_numpy(a).cuda() for a in concat_clips(clips))
    K, T = 128, clips[0].T
    W = 2 * K + 1
    F = torch.empty((len(clips), W, W), dtype=torch.complex64, device="cuda")
    area = torch.empty((len(clips),), dtype=torch.int64, device="cuda")
    fc.set_hybrid(2)
    try:
        ws = torch.empty(fc._lib.load().fcfs_batch_workspace_size(x.numel(), len(clips), T, K, 1),
                         dtype=torch.uint8, device="cuda")
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            fc.batch(x, y, s, off, T, K, out=F, area_out=area, workspace=ws, stream=st)   # warm-up
        torch.cuda.synchronize()
        ref = F.clone()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            fc.batch(x, y, s, off, T, K, out=F, area_out=area, workspace=ws, stream=st)
        F.zero_()
        g.replay()
        torch.cuda.synchronize()
    finally:
        fc.set_hybrid(1)
    assert torch.equal(F, ref)

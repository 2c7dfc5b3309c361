"""Torch-facing binding of the FCFS library.

Every function marshals device tensors into the C ABI of include/fcfs.h; the
arithmetic runs in the library's CUDA kernels.  PyTorch provides the device
memory (outputs and workspaces) and the current stream.
"""
import torch

from . import _lib
from ._lib import FCFSError, PREC, FLAG_VALIDATE

__all__ = ["forward", "adjoint", "edge_chain", "batch", "cosine", "haar", "workspace_size",
           "cosine_workspace_size", "haar_workspace_size", "forward_grouped", "adjoint_grouped",
           "get_status", "launch_count", "Plan", "FCFSError"]


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check_vertices(x, y, s):
    for name, t, dt in (("x", x, torch.int32), ("y", y, torch.int32), ("s", s, torch.int8)):
        if not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.dtype != dt:
            raise ValueError("%s must be %s" % (name, dt))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if not (x.shape == y.shape == s.shape) or x.dim() != 1:
        raise ValueError("x, y, s must be 1-D of equal length")


def _prec(prec):
    return PREC[prec] if isinstance(prec, str) else int(prec)


def workspace_size(V, T, K, prec="split_f16"):
    return int(_lib.load().fcfs_workspace_size(int(V), int(T), int(K), _prec(prec)))


def alloc_workspace(nbytes, device):
    # torch allocations are 512-byte aligned; the library asks for 256
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def forward(x, y, s, T, K, prec="split_f16", validate=False, out=None, area_out=None, workspace=None,
            stream=None):
    """F(k, l), |k|,|l| <= K, of one clip: complex64 (2K+1, 2K+1) and the int64 area."""
    _check_vertices(x, y, s)
    lib = _lib.load()
    dev = x.device
    W = 2 * int(K) + 1
    if out is None:
        out = torch.empty((W, W), dtype=torch.complex64, device=dev)
    if area_out is None:
        area_out = torch.empty((1,), dtype=torch.int64, device=dev)
    if workspace is None:   # (a given workspace is checked by the library)
        workspace = alloc_workspace(workspace_size(x.numel(), T, K, prec), dev)
    code = lib.fcfs_forward(_ptr(x), _ptr(y), _ptr(s), x.numel(), int(T), int(K), _prec(prec),
                            FLAG_VALIDATE if validate else 0, _ptr(out), _ptr(area_out),
                            _ptr(workspace), workspace.numel(), _stream(stream))
    _lib.check("fcfs_forward", code)
    return out, area_out


def adjoint(x, y, s, T, K, dF, prec="fp32", gx=None, gy=None, workspace=None, stream=None):
    """Corner derivatives (gx, gy) of a real loss with cotangent dF (complex64 block)."""
    _check_vertices(x, y, s)
    if dF.dtype != torch.complex64 or not dF.is_contiguous() or dF.shape != (2 * K + 1, 2 * K + 1):
        raise ValueError("dF must be a contiguous complex64 (2K+1, 2K+1) tensor")
    lib = _lib.load()
    dev = x.device
    V = x.numel()
    gx = torch.empty(V, dtype=torch.float32, device=dev) if gx is None else gx
    gy = torch.empty(V, dtype=torch.float32, device=dev) if gy is None else gy
    need = int(lib.fcfs_adjoint_workspace_size(V, int(T), int(K), _prec(prec)))
    if workspace is None:
        workspace = alloc_workspace(need, dev)
    code = lib.fcfs_adjoint(_ptr(x), _ptr(y), _ptr(s), V, int(T), int(K), _prec(prec), _ptr(dF),
                            _ptr(gx), _ptr(gy), _ptr(workspace), workspace.numel(), _stream(stream))
    _lib.check("fcfs_adjoint", code)
    return gx, gy


def edge_chain(gx, gy, ev0, ev1, eaxis, out=None, stream=None):
    """Per-edge derivative: a vertical edge moves both corners in x, a horizontal one in y."""
    lib = _lib.load()
    E = ev0.numel()
    out = torch.empty(E, dtype=torch.float32, device=gx.device) if out is None else out
    code = lib.fcfs_edge_chain(_ptr(gx), _ptr(gy), _ptr(ev0), _ptr(ev1), _ptr(eaxis), E, _ptr(out),
                               _stream(stream))
    _lib.check("fcfs_edge_chain", code)
    return out


def batch(x, y, s, offsets, T, K, prec="split_f16", validate=False, out=None, area_out=None,
          workspace=None, stream=None):
    """Blocks of n clips (offsets: int64 CUDA tensor [n+1]): (n, 2K+1, 2K+1) and (n,)."""
    _check_vertices(x, y, s)
    lib = _lib.load()
    dev = x.device
    n = offsets.numel() - 1
    W = 2 * int(K) + 1
    out = torch.empty((n, W, W), dtype=torch.complex64, device=dev) if out is None else out
    area_out = torch.empty((n,), dtype=torch.int64, device=dev) if area_out is None else area_out
    need = int(lib.fcfs_batch_workspace_size(x.numel(), n, int(T), int(K), _prec(prec)))
    if workspace is None:
        workspace = alloc_workspace(need, dev)
    code = lib.fcfs_batch(_ptr(x), _ptr(y), _ptr(s), _ptr(offsets), n, x.numel(), int(T), int(K),
                          _prec(prec), FLAG_VALIDATE if validate else 0, _ptr(out), _ptr(area_out),
                          _ptr(workspace), workspace.numel(), _stream(stream))
    _lib.check("fcfs_batch", code)
    return out, area_out


PLAN_KINDS = {"forward": 0, "batch": 1, "adjoint": 2}
KNOBS = {"form": 0, "splits": 1, "pair": 2, "unit_chunks": 3}


class Plan:
    """A workload's sizes and launch-shape choices (fcfs_plan_* of the C ABI).

    Knobs: form (forward: 0 over the corners, 1 split-FP16 contraction over y,
    2 pruned FFT along y; adjoint: 0 per corner, 1 grouped split-FP16
    contraction, 2 grouped pruned FFT; batch: 0 direct, 1 grouped), splits, pair,
    unit_chunks; -1 or 0 leaves a knob to the library.  get() returns the value
    a call will use.  The plan is released when the object is."""

    def __init__(self, kind, V, T, K, prec="split_f16", n_clips=1, **knobs):
        import ctypes as C
        lib = _lib.load()
        h = C.c_void_p()
        code = lib.fcfs_plan_create(C.byref(h), PLAN_KINDS[kind], int(V), int(n_clips), int(T), int(K),
                                    _prec(prec))
        _lib.check("fcfs_plan_create", code)
        self._h, self.kind, self.V, self.T, self.K, self.prec, self.n_clips = h, kind, int(V), int(T), int(K), prec, int(n_clips)
        for k, v in knobs.items():
            self.set(k, v)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.load().fcfs_plan_destroy(h)
            self._h = None

    def set(self, knob, value):
        _lib.check("fcfs_plan_set", _lib.load().fcfs_plan_set(self._h, KNOBS[knob], int(value)))
        return self

    def get(self, knob):
        return int(_lib.load().fcfs_plan_get(self._h, KNOBS[knob]))

    def knobs(self):
        return {k: self.get(k) for k in KNOBS}

    def workspace_size(self):
        return int(_lib.load().fcfs_plan_workspace_size(self._h))

    def forward(self, x, y, s, out=None, area_out=None, workspace=None, stream=None):
        _check_vertices(x, y, s)
        dev = x.device
        W = 2 * self.K + 1
        out = torch.empty((W, W), dtype=torch.complex64, device=dev) if out is None else out
        area_out = torch.empty((1,), dtype=torch.int64, device=dev) if area_out is None else area_out
        workspace = alloc_workspace(self.workspace_size(), dev) if workspace is None else workspace
        code = _lib.load().fcfs_plan_forward(self._h, _ptr(x), _ptr(y), _ptr(s), x.numel(), 0, _ptr(out),
                                             _ptr(area_out), _ptr(workspace), workspace.numel(), _stream(stream))
        _lib.check("fcfs_plan_forward", code)
        return out, area_out

    def batch(self, x, y, s, offsets, out=None, area_out=None, workspace=None, stream=None):
        _check_vertices(x, y, s)
        dev = x.device
        n = offsets.numel() - 1
        W = 2 * self.K + 1
        out = torch.empty((n, W, W), dtype=torch.complex64, device=dev) if out is None else out
        area_out = torch.empty((n,), dtype=torch.int64, device=dev) if area_out is None else area_out
        workspace = alloc_workspace(self.workspace_size(), dev) if workspace is None else workspace
        code = _lib.load().fcfs_plan_batch(self._h, _ptr(x), _ptr(y), _ptr(s), _ptr(offsets), x.numel(),
                                           _ptr(out), _ptr(area_out), _ptr(workspace), workspace.numel(),
                                           _stream(stream))
        _lib.check("fcfs_plan_batch", code)
        return out, area_out

    def adjoint(self, x, y, s, dF, gx=None, gy=None, workspace=None, stream=None):
        _check_vertices(x, y, s)
        dev = x.device
        V = x.numel()
        gx = torch.empty(V, dtype=torch.float32, device=dev) if gx is None else gx
        gy = torch.empty(V, dtype=torch.float32, device=dev) if gy is None else gy
        workspace = alloc_workspace(self.workspace_size(), dev) if workspace is None else workspace
        code = _lib.load().fcfs_plan_adjoint(self._h, _ptr(x), _ptr(y), _ptr(s), V, _ptr(dF), _ptr(gx), _ptr(gy),
                                             _ptr(workspace), workspace.numel(), _stream(stream))
        _lib.check("fcfs_plan_adjoint", code)
        return gx, gy


def cosine_workspace_size(V, T, K, prec="split_f16"):
    return int(_lib.load().fcfs_cosine_workspace_size(int(V), int(T), int(K), _prec(prec)))


def cosine(x, y, s, T, K, prec="split_f16", out=None, area_out=None, workspace=None, stream=None):
    """Continuous cosine series C(k, l), 0 <= k, l <= K, of one clip: float32
    (K+1, K+1) and the int64 area."""
    _check_vertices(x, y, s)
    lib = _lib.load()
    dev = x.device
    n1 = int(K) + 1
    if out is None:
        out = torch.empty((n1, n1), dtype=torch.float32, device=dev)
    if area_out is None:
        area_out = torch.empty((1,), dtype=torch.int64, device=dev)
    if workspace is None:
        workspace = alloc_workspace(cosine_workspace_size(x.numel(), T, K, prec), dev)
    code = lib.fcfs_cosine(_ptr(x), _ptr(y), _ptr(s), x.numel(), int(T), int(K), _prec(prec), 0,
                           _ptr(out), _ptr(area_out), _ptr(workspace), workspace.numel(), _stream(stream))
    _lib.check("fcfs_cosine", code)
    return out, area_out


def haar_workspace_size(V, T, J):
    return int(_lib.load().fcfs_haar_workspace_size(int(V), int(T), int(J)))


def haar(x, y, s, T, J, out=None, workspace=None, stream=None):
    """Continuous Haar coefficients of one clip up to level J: float64 (2^J, 2^J)
    in the square layout of include/fcfs.h (W[0, 0] = area / T)."""
    _check_vertices(x, y, s)
    lib = _lib.load()
    dev = x.device
    G = 1 << int(J)
    if out is None:
        out = torch.empty((G, G), dtype=torch.float64, device=dev)
    if workspace is None:
        workspace = alloc_workspace(haar_workspace_size(x.numel(), T, J), dev)
    code = lib.fcfs_haar(_ptr(x), _ptr(y), _ptr(s), x.numel(), int(T), int(J), 0, _ptr(out),
                         _ptr(workspace), workspace.numel(), _stream(stream))
    _lib.check("fcfs_haar", code)
    return out


def forward_grouped(V, T, K, prec="split_f16"):
    """Which form forward() takes for these sizes: 0 the contraction over the
    corners, 1 corners grouped by y with the split-FP16 contraction over y, 2
    corners grouped by y with the pruned FFT along y (FP32); -1 if the sizes are
    unsupported."""
    return int(_lib.load().fcfs_forward_grouped(int(V), int(T), int(K), _prec(prec)))


def adjoint_grouped(V, T, K, prec="split_f16"):
    """Which form adjoint() takes for these sizes: 0 per corner, 1 corners
    grouped by the contracted coordinate with the split-FP16 contraction over
    its values, 2 grouped with one pruned FFT along it per frequency and a dot
    per corner (FP32); -1 if the sizes or the precision are unsupported."""
    return int(_lib.load().fcfs_adjoint_grouped(int(V), int(T), int(K), _prec(prec)))


def get_status(workspace, stream=None):
    """Synchronise and return the device status name of the last call on ``workspace``."""
    code = _lib.load().fcfs_get_status(_ptr(workspace), _stream(stream))
    return _lib.STATUS.get(code, str(code))


def launch_count():
    return int(_lib.load().fcfs_launch_count())


def set_splits(n):
    """Force the number of vertex splits (0: automatic); a test hook."""
    _lib.load().fcfs_debug_set_splits(int(n))


def set_fuse(on):
    """1 (default): the split-FP16 forward sums its splits and takes the axis DFT
    inside the contraction kernel when its CTAs fit at once; 0: separate kernels."""
    _lib.load().fcfs_debug_set_fuse(1 if on else 0)


def set_pair(on):
    """1 (default): single clips with 2K >= 256 run on CTA pairs (2-SM MMA);
    0: one-CTA tiles.  Allocate workspaces after changing it."""
    _lib.load().fcfs_debug_set_pair(1 if on else 0)


def set_barrier_extra(n):
    """Failure-detection test hook: fused calls wait for n CTAs that do not exist
    (bounded), ending with FCFS_ETIMEOUT; 0 restores normal calls."""
    _lib.load().fcfs_debug_set_barrier_extra(int(n))


def set_hybrid(mode):
    """Form of single-clip forward and adjoint calls: 0 direct / per corner, 1
    automatic (cost estimates; see forward_grouped and adjoint_grouped), 2 the
    grouped split-FP16 contraction whenever eligible, 3 the grouped pruned FFT
    whenever eligible."""
    _lib.load().fcfs_debug_set_hybrid(int(mode))


def set_overlap(on):
    """Run the stages of a call that do not depend on its main sequence on a
    second stream (True, the default) or every stage in order on the call's
    stream (False: what per-stage timing needs)."""
    _lib.load().fcfs_debug_set_overlap(1 if on else 0)


def set_batch_unit_chunks(n):
    """Vertex-split granularity of batch(): n pipeline chunks per unit (0: default)."""
    _lib.load().fcfs_set_batch_unit_chunks(int(n))


def profile_enable(on=True):
    """Bracket every stage of later calls with CUDA events (see profile_read)."""
    _lib.load().fcfs_profile_enable(1 if on else 0)


def profile_read():
    """Durations in ms of the last call's stages: prep, axis, contraction, reduce."""
    import ctypes as C
    buf = (C.c_float * 4)()
    n = _lib.load().fcfs_profile_read(buf, 4)
    return [float(buf[i]) for i in range(n)]


def kernel_timing_enable(on=True):
    """Start (clearing earlier records) or stop recording stage times of later calls."""
    _lib.load().fcfs_kernel_timing_enable(1 if on else 0)


def kernel_timing():
    """[(stage name, ms)] of the calls made since kernel_timing_enable(True)."""
    lib = _lib.load()
    n = lib.fcfs_kernel_timing_count()
    return [(lib.fcfs_kernel_timing_name(i).decode(), float(lib.fcfs_kernel_timing_ms(i))) for i in range(n)]


def vertices_from_edges(pos, ev0, ev1, eaxis, V):
    """Integer corner coordinates from edge positions: a vertical edge (axis 0)
    gives the x of both its corners, a horizontal edge (axis 1) their y."""
    p = torch.round(pos).to(torch.int32)
    vert = eaxis == 0
    x = torch.empty(V, dtype=torch.int32, device=pos.device)
    y = torch.empty(V, dtype=torch.int32, device=pos.device)
    for ends in (ev0, ev1):
        x[ends[vert].long()] = p[vert]
        y[ends[~vert].long()] = p[~vert]
    return x, y


class BlockFunction(torch.autograd.Function):
    """F(k,l) of a clip as a differentiable function of its edge positions.

    forward(pos, ev0, ev1, eaxis, s, T, K, prec) -> complex64 (2K+1, 2K+1).
    `pos` holds lattice-valued edge positions (float); the block is evaluated at
    those integer positions and the gradient is the exact derivative of the
    continuous transform with respect to each edge position (both corners of an
    edge move together), computed by the adjoint kernels and edge chaining.
    """

    @staticmethod
    def forward(ctx, pos, ev0, ev1, eaxis, s, T, K, prec="fp32"):
        x, y = vertices_from_edges(pos, ev0, ev1, eaxis, s.numel())
        F, _ = forward(x, y, s, T, K, prec=prec)
        ctx.save_for_backward(x, y, s, ev0, ev1, eaxis)
        ctx.T, ctx.K, ctx.prec = int(T), int(K), prec
        return F

    @staticmethod
    def backward(ctx, gF):
        x, y, s, ev0, ev1, eaxis = ctx.saved_tensors
        gx, gy = adjoint(x, y, s, ctx.T, ctx.K, gF.contiguous(), prec=ctx.prec)
        gE = edge_chain(gx, gy, ev0, ev1, eaxis)
        return gE, None, None, None, None, None, None, None


def block(pos, ev0, ev1, eaxis, s, T, K, prec="fp32"):
    """Differentiable block of a clip from its edge positions (see BlockFunction)."""
    return BlockFunction.apply(pos, ev0, ev1, eaxis, s, T, K, prec)

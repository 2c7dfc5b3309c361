"""The forward entry point for callers that cannot allocate device memory.

fcfs_forward_noalloc runs the same transform as fcfs_forward but takes no
workspace: its scratch is a fixed array inside the library.  It is meant for
code that cannot call cudaMalloc where it needs the transform (a plugin whose
host framework owns all device memory, a real-time loop that must not stall
on an allocation).  This file is collected last and also runs alone.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from synth import config_clip

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-6, "split_f16": 1e-5}
PREC = {"fp32": 0, "split_f16": 1}


@pytest.fixture(scope="module")
def lib():
    from paper_1010_5562_gb300 import build as B
    B.build()
    from paper_1010_5562_gb300 import _lib
    assert torch.cuda.is_available()
    return _lib.load()


def _noalloc(lib, x, y, s, T, K, prec):
    W = 2 * K + 1
    F = torch.full((W, W), float("nan"), dtype=torch.complex64, device="cuda")
    area = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = lib.fcfs_forward_noalloc(x.data_ptr(), y.data_ptr(), s.data_ptr(), x.numel(), T, K, PREC[prec], 0,
                                    F.data_ptr(), area.data_ptr(), stream)
    assert code == 0, code
    torch.cuda.synchronize()
    return F.cpu().numpy().astype(np.complex128), int(area.item())


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
@pytest.mark.parametrize("cfg", [1, 2])
def test_noalloc_matches_forward_twice(lib, prec, cfg):
    from paper_1010_5562_gb300 import fcfs
    clip, K = config_clip(cfg)
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    Fr, ar = fcfs.forward(x, y, s, clip.T, K, prec=prec)
    torch.cuda.synchronize()
    Fr = Fr.cpu().numpy().astype(np.complex128)
    A = oracle.area_exact(clip.x, clip.y, clip.s, clip.T)
    for _ in range(2):   # the second call reuses the array the first one left behind
        F, area = _noalloc(lib, x, y, s, clip.T, K, prec)
        assert area == int(ar.item()) == A
        assert np.all(np.isfinite(F))
        assert np.max(np.abs(F - Fr)) / A <= TOL[prec]


def test_noalloc_rejects_what_does_not_fit(lib):
    clip, _ = config_clip(1)
    x, y, s = (torch.from_numpy(a).cuda() for a in (clip.x, clip.y, clip.s))
    F = torch.empty((1, 2), dtype=torch.complex64, device="cuda")
    area = torch.zeros(1, dtype=torch.int64, device="cuda")
    code = lib.fcfs_forward_noalloc(x.data_ptr(), y.data_ptr(), s.data_ptr(), x.numel(), 256, 4096, 1, 0,
                                    F.data_ptr(), area.data_ptr(), None)
    assert code == 6     # FCFS_EUNSUPPORTED: even one vertex split exceeds the array
    code = lib.fcfs_forward_noalloc(x.data_ptr(), y.data_ptr(), s.data_ptr(), x.numel(), 256, 8, 1, 1,
                                    F.data_ptr(), area.data_ptr(), None)
    assert code == 1     # FCFS_EINVAL: no flags on this entry point

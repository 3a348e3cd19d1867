"""The allocation-free feasibility check (pecc_check_feasible_noalloc).

Callers that cannot allocate device memory (code running under CUDA graph capture, plug-ins
whose host owns the device memory, real-time loops) check one instance with scratch held in a
fixed device array.  Its answers must equal those of the context-based check, call after call,
although every call reuses the same scratch.  This file sorts last so that a run stopping at
the first failure has run every other test first.
"""
import numpy as np
import pytest

from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu


def _layout(n, u, seed, scale):
    R = synth.radius(n, u)
    xy = synth.random_layout(n, R, seed, spread=1.0) * 0.7 * scale
    return xy, R


@pytest.mark.gpu
def test_noalloc_matches_context_check_twice():
    torch, pecc = need_gpu()
    cases = [_layout(3000, 0.8, 1, 1.0), _layout(777, 0.5, 2, 0.6), _layout(4096, 0.84, 3, 1.0)]
    for xy, R in cases:  # consecutive calls share the scratch array
        t = torch.from_numpy(xy).cuda()
        f1, m1 = pecc.check_feasible_noalloc(t, R, 2.5, 1e-9)
        with pecc.Context(np.array([xy.shape[0]], dtype=np.int32), precision=pecc.FP64) as c:
            c.set_radius(np.array([R]))
            c.set_positions(t)
            f2, m2 = c.check_feasible(1e-9)
        torch.cuda.synchronize()
        assert m1.item() == m2.item()
        assert f1.item() == f2.item()
    # a feasible packing (hexagon of 7 circles in R = 3) after the larger calls
    xy = np.vstack([[0, 0], 2 * np.stack([np.cos(np.arange(6) * np.pi / 3), np.sin(np.arange(6) * np.pi / 3)], 1)])
    f, m = pecc.check_feasible_noalloc(torch.from_numpy(xy).cuda(), 3.0)
    assert f.item() == 1 and m.item() <= 1e-15


@pytest.mark.gpu
def test_noalloc_rejects_oversize():
    torch, pecc = need_gpu()
    xy = torch.zeros((pecc.NOALLOC_MAX_N + 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(pecc.PeccError, match="PECC_ERR_ARG"):
        pecc.check_feasible_noalloc(xy, 100.0)

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
def test_noalloc_over_dense_layouts_match_context_and_oracle(orc):
    """Layouts far denser than any packing, on both sides of the list capacity 2 (16 n + 64) the
    two checks share: 4096 circles with about 19 neighbors each (77576 entries, under 131200:
    finite) and 1000 circles with about 53 each (52938 entries, over 32128: NaN, not checkable).
    The allocation-free check equals the context check, NaN included, and a finite result equals
    the oracle's brute-force depth; two calls in a row give the same answer."""
    torch, pecc = need_gpu()
    for n, half, finite in [(4096, 32.0, True), (1000, 9.0, False)]:
        xy = synth.random_layout(n, half, seed=9)
        R = 40.0
        t = torch.from_numpy(xy).cuda()
        f1, m1 = pecc.check_feasible_noalloc(t, R, 2.5, 1e-9)
        f1b, m1b = pecc.check_feasible_noalloc(t, R, 2.5, 1e-9)
        with pecc.Context(np.array([n], dtype=np.int32), precision=pecc.FP64) as c:
            c.set_radius(np.array([R]))
            c.set_positions(t)
            f2, m2 = c.check_feasible(1e-9)
        torch.cuda.synchronize()
        a, b, a2 = m1.item(), m2.item(), m1b.item()
        assert np.isnan(a) == np.isnan(b) == np.isnan(a2) == (not finite)
        assert f1.item() == f2.item() == f1b.item() == 0
        if finite:
            assert a == b == a2 == orc.max_overlap(xy, R)[0]


@pytest.mark.gpu
def test_noalloc_equals_oracle_on_descended_layouts(orc):
    """Feasible and nearly feasible layouts the descent itself produced: the allocation-free check
    returns the oracle's brute-force depth bit for bit, instance after instance."""
    torch, pecc = need_gpu()
    n = np.array([300, 420, 1000], dtype=np.int32)
    R = np.array([synth.radius(int(v), 0.8) for v in n])
    with pecc.Context(n, precision=pecc.FP32_POLISH64) as c:
        c.set_radius(R)
        c.init_random(5)
        c.descend()
        xy = c.get_positions()
    off = np.concatenate([[0], np.cumsum(n)])
    for q in range(len(n)):
        part = xy[off[q]:off[q + 1]].contiguous()
        f, m = pecc.check_feasible_noalloc(part, float(R[q]), 2.5, 1e-9)
        ref = orc.max_overlap(part.cpu().numpy(), float(R[q]))[0]
        assert m.item() == ref and f.item() == (ref <= 1e-9)


@pytest.mark.gpu
def test_noalloc_rejects_oversize():
    torch, pecc = need_gpu()
    xy = torch.zeros((pecc.NOALLOC_MAX_N + 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(pecc.PeccError, match="PECC_ERR_ARG"):
        pecc.check_feasible_noalloc(xy, 100.0)

"""The framework of Sec. 5.1 on the GPU (pecc_frame_run), marked gpu.

- At the exact radii of 2, 3 and 7 circles the record is that radius within 1e-9, as in the
  oracle.
- On dense instances the record never grows, ends feasible, and improves on the first
  adjustment for some instances.
- A context with other instances is refused.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, split

pytestmark = pytest.mark.gpu

R3 = 1.0 + 2.0 / np.sqrt(3.0)


def test_framework_keeps_the_exact_radii(orc):
    torch, pecc = need_gpu()
    n = np.array([2, 3, 7, 7], dtype=np.int32)
    Rb = np.array([2.0, R3, 3.0, 3.0])
    with pecc.Sed(n, precision=0, s_iter=5) as s, pecc.Context(n, precision=0) as adj:
        Rbest, xbest, trace = pecc.frame_run(s, adj, Rb, seed=5, outer=2, sed_iters=5)
        torch.cuda.synchronize()
        Rbest, xbest, trace = Rbest.cpu().numpy(), xbest.cpu().numpy(), trace.cpu().numpy()
    np.testing.assert_allclose(Rbest, Rb, rtol=0, atol=1e-9)
    assert np.all(np.diff(trace, axis=0) <= 0.0)
    for q, part in enumerate(split(xbest, n)):
        assert orc.max_overlap(part, Rbest[q])[0] <= 1e-9
        x, R, tr = orc.frame(int(n[q]), float(Rb[q]), 5, inst=q, outer=2, s_iter=5)
        assert abs(R - Rbest[q]) <= 1e-9


@pytest.mark.parametrize("prec", [0, 2])
def test_framework_on_dense_instances(orc, prec):
    torch, pecc = need_gpu()
    num = 8
    n = np.full(num, 40, dtype=np.int32)
    Rb = np.full(num, np.sqrt(40 / 0.78))
    with pecc.Sed(n, precision=prec, s_iter=3, max_iter=300) as s, \
            pecc.Context(n, precision=prec, max_iter=300) as adj:
        Rbest, xbest, trace = pecc.frame_run(s, adj, Rb, seed=2, outer=3, sed_iters=3)
        torch.cuda.synchronize()
        Rbest, xbest, trace = Rbest.cpu().numpy(), xbest.cpu().numpy(), trace.cpu().numpy()
    assert np.all(np.diff(trace, axis=0) <= 0.0)
    np.testing.assert_array_equal(Rbest, trace[-1])
    assert np.sum(trace[-1] < trace[0]) >= 1
    for q, part in enumerate(split(xbest, n)):
        assert orc.max_overlap(part, Rbest[q])[0] <= 1e-9, q


def test_framework_refuses_other_instances():
    torch, pecc = need_gpu()
    with pecc.Sed(np.array([10, 12], dtype=np.int32), precision=0) as s, \
            pecc.Context(np.array([10, 13], dtype=np.int32), precision=0) as adj:
        with pytest.raises(pecc.PeccError):
            pecc.frame_run(s, adj, np.array([3.0, 3.5]), seed=1)

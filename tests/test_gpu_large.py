"""Whole-GPU descent of large instances (n >= 16384 circles): parity with the FP64 oracle
(marked gpu).  The same Algorithm GBO (Sec. 4.1) with ANM (Sec. 4.3) as the per-block path,
with grid-wide partition, neighbor build and reductions."""
import numpy as np
import pytest

from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu, split

pytestmark = pytest.mark.gpu


def _ctx(pecc, n, R, **kw):
    c = pecc.Context(n, **kw)
    c.set_radius(R)
    return c


@pytest.mark.parametrize("k,sweeps", [(1, 1), (5, 1), (5, 3)])
def test_grid_descent_short_runs_fp64(orc, k, sweeps):
    """A few sweeps of the whole-GPU FP64 descent take the oracle's steps (positions to 1e-9 R)."""
    torch, pecc = need_gpu()
    n = np.array([20000], dtype=np.int32)
    R = np.array([synth.radius(20000, 0.82)])
    with _ctx(pecc, n, R, precision=0, k_batches=k, max_iter=sweeps) as c:
        c.init_random(5)
        x0 = c.get_positions().cpu().numpy()
        iters, status = c.descend()
        x1 = c.get_positions().cpu().numpy()
        E = c.get_energy().cpu().numpy()
    r = orc.gbo(x0, float(R[0]), k=k, max_iter=sweeps)
    assert int(iters.cpu()[0]) == r.iters
    np.testing.assert_allclose(x1, r.x, rtol=0, atol=1e-9 * float(R[0]))
    assert E[0] == pytest.approx(r.E, rel=1e-9)


def test_grid_descent_fp32_polish_feasible(orc):
    """The whole-GPU FP32 + FP64 polish descent of a 20000-circle instance at u = 0.78 reaches a
    feasible packing; the reported max overlap equals the oracle's brute force on the result."""
    torch, pecc = need_gpu()
    n = np.array([20000], dtype=np.int32)
    R = np.array([synth.radius(20000, 0.78)])
    with _ctx(pecc, n, R, precision=2) as c:
        c.init_random(9)
        iters, status = c.descend()
        feas, mo = c.check_feasible()
        xy = c.get_positions().cpu().numpy()
    ref = orc.max_overlap(xy, float(R[0]))[0]
    assert float(mo.cpu()[0]) == ref
    assert int(status.cpu()[0]) in (0, 1, 2, 3)
    assert int(feas.cpu()[0]) == 1, (int(status.cpu()[0]), ref)


def test_mixed_small_and_large_instances(orc):
    """One context holding block-sized and whole-GPU instances runs both paths."""
    torch, pecc = need_gpu()
    n = np.array([300, 17000, 64], dtype=np.int32)
    R = np.array([synth.radius(int(v), 0.78) for v in n])
    with _ctx(pecc, n, R, precision=2) as c:
        c.init_random(3)
        iters, status = c.descend()
        feas, mo = c.check_feasible()
        xy = c.get_positions().cpu().numpy()
    for q, x in enumerate(split(xy, n)):
        assert float(mo.cpu()[q]) == orc.max_overlap(x, float(R[q]))[0]
    assert int(iters.cpu()[1]) > 0
    assert feas.cpu().numpy().sum() >= 2


def test_grid_barrier_wait_is_bounded(orc):
    """The grid barrier of the whole-GPU descent never waits past its limit: at a barrier that
    nothing releases, every block's wait ends by itself (%globaltimer), the error flag is seen,
    and the device stays usable for the next descent."""
    torch, pecc = need_gpu()
    failed, waited = pecc.selftest_grid_barrier(50_000_000)
    assert failed == 1
    assert 50_000_000 <= waited < 2_000_000_000
    n = np.array([300], dtype=np.int32)
    R = np.array([synth.radius(300, 0.8)])
    with _ctx(pecc, n, R, precision=0, max_iter=2) as c:
        c.init_random(5)
        iters, status = c.descend()
        assert int(iters.cpu()[0]) == 2 and int(status.cpu()[0]) == 3

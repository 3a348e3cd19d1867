"""GBO with the explicit per-batch inverse Hessian (Sec. 4.1, Eq. 10, Eq. 11) on the GPU against the
oracle's dense mode, through the C ABI (marked gpu).

- Short binary64 runs: the GPU (warp-per-row products in a fixed order, FMA) and the oracle
  (sequential sums, correctly rounded) take the same steps up to rounding.  Positions agree to
  1e-9 R, energies to 1e-9 relative, and sweep counts exactly.
- Zero energy, up to rounding, at the exact radius of 7 circles.
- Argument checks.
"""
import numpy as np
import pytest

from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu, split

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,sweeps,part", [(1, 1, 0), (1, 3, 0), (3, 2, 0), (5, 3, 0), (4, 2, 3), (3, 2, 2)])
def test_short_dense_runs_match_the_oracle(orc, k, sweeps, part):
    torch, pecc = need_gpu()
    n = np.array([300, 257, 640, 41], dtype=np.int32)
    R = np.array([synth.radius(int(v), 0.8) for v in n])
    with pecc.Context(n, precision=0, qn_dense=1, k_batches=k, max_iter=sweeps, partition=part,
                      partition_seed=99) as c:
        c.set_radius(R)
        c.init_random(51)
        x0 = c.get_positions().cpu().numpy()
        iters, status = c.descend()
        x1 = c.get_positions().cpu().numpy()
        E = c.get_energy().cpu().numpy()
        iters = iters.cpu().numpy()
        ms = c.phase_times()
    assert ms[0] > 0.0
    for q, (a, b) in enumerate(zip(split(x0, n), split(x1, n))):
        r = orc.gbo(a, float(R[q]), k=k, max_iter=sweeps, dense=1, partition=part, part_seed=99, part_inst=q)
        assert iters[q] == r.iters, q
        np.testing.assert_allclose(b, r.x, rtol=0, atol=1e-9 * float(R[q]))
        assert E[q] == pytest.approx(r.E, rel=1e-9)


def test_dense_descent_differs_from_limited_memory():
    """The explicit H and the m = 10 secant pairs agree on the first sweep of one batch (both
    start from a gradient step) and part ways after it."""
    torch, pecc = need_gpu()
    n = np.array([200], dtype=np.int32)
    R = np.array([synth.radius(200, 0.8)])
    out = {}
    for dense in (0, 1):
        with pecc.Context(n, precision=0, qn_dense=dense, k_batches=1, max_iter=6) as c:
            c.set_radius(R)
            c.init_random(3)
            c.descend()
            out[dense] = c.get_positions().cpu().numpy()
    assert not np.allclose(out[0], out[1], rtol=0, atol=1e-12)


def test_exact_radius_of_seven_reaches_zero_energy(orc):
    torch, pecc = need_gpu()
    num = 12
    n = np.full(num, 7, dtype=np.int32)
    R = np.full(num, 3.0)
    with pecc.Context(n, precision=0, qn_dense=1, k_batches=1, e_tol=1e-28) as c:
        c.set_radius(R)
        c.init_random(8)
        c.descend()
        E = c.get_energy().cpu().numpy()
        xy = c.get_positions().cpu().numpy()
    feasible = [orc.max_overlap(p, 3.0)[0] <= 1e-9 for p in split(xy, n)]
    assert np.min(E) <= 1e-24
    assert np.sum(feasible) >= num // 2


def test_dense_arguments():
    torch, pecc = need_gpu()
    with pytest.raises(pecc.PeccError):
        pecc.Context(np.array([10], dtype=np.int32), precision=2, qn_dense=1)
    with pytest.raises(pecc.PeccError):
        pecc.Context(np.array([10], dtype=np.int32), precision=0, qn_dense=2)
    with pecc.Context(np.array([16384], dtype=np.int32), precision=0, qn_dense=1) as c:
        c.set_radius(np.array([synth.radius(16384, 0.8)]))
        c.init_random(1)
        with pytest.raises(pecc.PeccError):
            c.descend()

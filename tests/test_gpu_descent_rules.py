"""GPU parity of the descent's bookkeeping and of its binary32 path, through the C ABI (marked gpu).

- Algorithm ANM (Sec. 4.3): the GPU decides "Gamma' != Gamma" with a digest of the pair set, the
  oracle by comparing CSR arrays; the counts of builds, of builds that changed Gamma and of
  line-search trials must be equal after short binary64 runs, and the deferral must double on a
  layout whose lists no longer change.
- Eq. 9's line search (Armijo with c1 and halving) and the stationary stop of Algorithm GBO: the
  hand-computed cases of the oracle's pins run on the GPU too.
- Two-level lists: lists filtered from an outer list keep every count of the oracle, and an outer
  list that overflows its capacity falls back to cell-grid builds.
- The binary32 descent: the neighbor lists it builds itself (binary32 grid, binary32 predicate,
  16-bit indices in partition order) equal the oracle's brute force on the coordinates of that
  build, and a few binary32 sweeps follow the oracle's binary64 sweeps from the same binary32
  coordinates within a bound derived below.
"""
import math

import numpy as np
import pytest

from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu, split

pytestmark = pytest.mark.gpu


def _radii(n, u):
    return np.array([synth.radius(max(int(v), 1), u) for v in n])


def _run(pecc, torch, n, R, x0=None, seed=None, **cfg):
    with pecc.Context(n, **cfg) as c:
        c.set_radius(R)
        if x0 is not None:
            c.set_positions(torch.from_numpy(np.ascontiguousarray(x0)))
        else:
            c.init_random(seed)
        xin = c.get_positions().cpu().numpy()
        iters, status = c.descend()
        b, ch, tr = [t.cpu().numpy() for t in c.get_counters()]
        return dict(x0=xin, x=c.get_positions().cpu().numpy(), iters=iters.cpu().numpy(),
                    status=status.cpu().numpy(), E=c.get_energy().cpu().numpy(), builds=b, changes=ch, trials=tr)


# ------------------------------------------------------------------ ANM and trial counters
@pytest.mark.parametrize("k,m,step_max,sweeps", [(1, 10, 0.1, 4), (3, 10, 0.1, 3), (2, 5, 0.3, 6), (5, 10, 0.1, 2)])
def test_anm_and_trial_counters_match_oracle(orc, k, m, step_max, sweeps):
    """Short binary64 runs from random layouts: the lists change after most sweeps (len stays 1)
    and the Verlet rule forces builds at step cap 0.3; builds, changes and trials equal the
    oracle's counts, and the positions agree to 1e-9 R as in the other short-run tests."""
    torch, pecc = need_gpu()
    n = np.array([300, 257, 640, 1000], dtype=np.int32)
    R = _radii(n, 0.82)
    out = _run(pecc, torch, n, R, seed=91, precision=0, k_batches=k, lbfgs_m=m, step_max=step_max,
               max_iter=sweeps)
    for q, (a, b) in enumerate(zip(split(out["x0"], n), split(out["x"], n))):
        r = orc.gbo(a, float(R[q]), k=k, m=m, step_max=step_max, max_iter=sweeps)
        assert out["iters"][q] == r.iters, q
        assert (out["builds"][q], out["changes"][q], out["trials"][q]) == (r.builds, r.changes, r.trials), q
        np.testing.assert_allclose(b, r.x, rtol=0, atol=1e-9 * float(R[q]))


@pytest.mark.parametrize("outer", [0.0, 2.0 ** -9, 0.5, 1.5])
def test_two_level_lists_keep_the_counts(orc, outer):
    """The lists of Sec. 4.3 filtered from an outer list (cutoff l_cut + list_outer) are the sets a
    cell-grid build gives: builds, changes and trials equal the oracle's for an outer reach that is
    rebuilt at almost every list build (2^-9), the default (0.5), and one whose list can outgrow its
    shared-memory share (1.5, about 12 entries per circle), and positions agree to 1e-9 R."""
    torch, pecc = need_gpu()
    n = np.array([300, 257, 640, 1000], dtype=np.int32)
    R = _radii(n, 0.82)
    out = _run(pecc, torch, n, R, seed=93, precision=0, k_batches=2, lbfgs_m=5, step_max=0.3, max_iter=8,
               list_outer=outer)
    for q, (a, b) in enumerate(zip(split(out["x0"], n), split(out["x"], n))):
        r = orc.gbo(a, float(R[q]), k=2, m=5, step_max=0.3, max_iter=8)
        assert out["iters"][q] == r.iters, q
        assert (out["builds"][q], out["changes"][q], out["trials"][q]) == (r.builds, r.changes, r.trials), q
        np.testing.assert_allclose(b, r.x, rtol=0, atol=1e-9 * float(R[q]))


def test_two_level_lists_fall_back_when_the_outer_list_overflows():
    """With room for 6 entries per circle the lists (about 5 per circle at density 0.82) fit but an
    outer list of cutoff 3 (about 7) does not: the descent falls back to cell-grid builds from the
    start, bit for bit the run with list_outer = 0; with the default room the two-level run orders
    its rows differently, so its coordinates differ in the last bits (the fallback is what makes
    the first pair equal)."""
    torch, pecc = need_gpu()
    n = np.array([1000, 640], dtype=np.int32)
    R = _radii(n, 0.82)
    kw = dict(seed=95, precision=0, k_batches=2, lbfgs_m=5, step_max=0.3, max_iter=6)
    a = _run(pecc, torch, n, R, list_outer=0.5, nbr_capacity=6.0, **kw)
    b = _run(pecc, torch, n, R, list_outer=0.0, nbr_capacity=6.0, **kw)
    assert np.all(a["status"] == 3) and np.all(b["status"] == 3)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["builds"], b["builds"])
    c = _run(pecc, torch, n, R, list_outer=0.5, **kw)
    d = _run(pecc, torch, n, R, list_outer=0.0, **kw)
    assert np.array_equal(c["builds"], d["builds"]) and np.array_equal(c["changes"], d["changes"])
    assert not np.array_equal(c["x"], d["x"])
    np.testing.assert_allclose(c["x"], d["x"], rtol=0, atol=1e-9 * float(R.max()))


def test_anm_deferral_doubles_on_stable_layout_gpu(orc):
    """A slightly compressed hexagonal patch relaxes by tiny moves while Gamma never changes: the
    GPU's ANM builds after sweeps 1, 3, 7, 15, 31 (cnt reaching len = 1, 2, 4, 8, 16) besides the
    initial build, with no change of Gamma, exactly as the oracle; an uncompressed patch stalls
    after one sweep and one ANM build."""
    torch, pecc = need_gpu()
    xy = synth.hex_patch(4, 1.999)
    n = np.array([xy.shape[0]], dtype=np.int32)
    out = _run(pecc, torch, n, np.array([1e3]), x0=xy, precision=0, max_iter=31, e_tol=-1.0, gsum_tol=-1.0)
    r = orc.gbo(out["x0"], 1e3, max_iter=31, e_tol=-1.0, gsum_tol=-1.0)
    assert r.iters == out["iters"][0] and r.disp_builds == 0 and r.changes == 0
    assert out["builds"][0] == r.builds == 1 + sum(1 for t in (1, 3, 7, 15, 31) if t <= r.iters)
    assert out["changes"][0] == 0
    xy = synth.hex_patch(4, 2.2)
    out = _run(pecc, torch, n, np.array([100.0]), x0=xy, precision=0, max_iter=40, e_tol=-1.0, gsum_tol=-1.0)
    assert out["status"][0] == 2 and out["builds"][0] == 2 and out["changes"][0] == 0 and out["iters"][0] == 1


def test_anm_off_builds_only_by_the_verlet_rule(orc):
    """With ANM off only the Verlet rule rebuilds: the counts equal the oracle's with anm = 0."""
    torch, pecc = need_gpu()
    n = np.array([300, 640], dtype=np.int32)
    R = _radii(n, 0.82)
    out = _run(pecc, torch, n, R, seed=5, precision=0, k_batches=2, lbfgs_m=5, step_max=0.3, max_iter=8, anm=0)
    for q, a in enumerate(split(out["x0"], n)):
        r = orc.gbo(a, float(R[q]), k=2, m=5, step_max=0.3, max_iter=8, anm=0)
        assert (out["builds"][q], out["changes"][q], out["trials"][q]) == (r.builds, r.changes, r.trials), q
        assert r.builds == 1 + r.disp_builds


# ------------------------------------------------------------------ Armijo and the stationary stop
ARMIJO_KW = dict(k_batches=2, lbfgs_m=5, step_max=2.0, l_cut=6.0, rebuild_disp=2.0, max_iter=1)
ARMIJO_ORC = dict(k=2, m=5, step_max=2.0, l_cut=6.0, rebuild_disp=2.0, max_iter=1)


def _armijo_case(eps):
    w = 0.5 * math.sqrt(1.0 - eps)
    return np.array([[1.0, 0.0], [-0.5, 0.0]]), np.array([3.0 - w])


@pytest.mark.parametrize("eps,c1,trials,xm", [(3.9e-4, 1e-4, 2, 1.5), (4.1e-4, 1e-4, 1, 2.0), (3.9e-4, 0.0, 1, 2.0),
                                              (3.9e-4, 1e-5, 1, 2.0)])
def test_armijo_acceptance_by_hand_gpu(orc, eps, c1, trials, xm):
    """The two-circle layout of the oracle's Armijo pin (M at (1, 0) in batch 0, F at (-1/2, 0),
    first trial alpha = 1, wall depth sqrt(1 - eps) / 2 there): alpha = 1 is accepted exactly when
    eps / 4 >= c1.  The GPU takes the hand-computed number of trials to the hand-computed
    position, as the oracle does."""
    torch, pecc = need_gpu()
    xy, R = _armijo_case(eps)
    out = _run(pecc, torch, np.array([2], dtype=np.int32), R, x0=xy, precision=0, c1=c1, **ARMIJO_KW)
    assert out["trials"][0] == trials
    assert out["x"][0].tolist() == [xm, 0.0] and out["x"][1].tolist() == [-0.5, 0.0]
    r = orc.gbo(xy, float(R[0]), c1=c1, **ARMIJO_ORC)
    assert r.trials == trials
    np.testing.assert_array_equal(out["x"], r.x)


def test_armijo_threshold_gpu(orc):
    """The same layout over a range of eps and c1 (a larger c1 rejects more trials): the GPU's
    trial counts and positions equal the oracle's on both sides of every threshold."""
    torch, pecc = need_gpu()
    seen = set()
    for eps in (1e-4, 3.9e-4, 4.1e-4, 1e-3, 0.2, 0.9):
        xy, R = _armijo_case(eps)
        for c1 in (1e-4, 0.0, 0.05, 0.3):
            out = _run(pecc, torch, np.array([2], dtype=np.int32), R, x0=xy, precision=0, c1=c1, **ARMIJO_KW)
            r = orc.gbo(xy, float(R[0]), c1=c1, **ARMIJO_ORC)
            assert out["trials"][0] == r.trials, (eps, c1)
            np.testing.assert_array_equal(out["x"], r.x)
            seen.add(r.trials)
    assert len(seen) >= 2


def test_stationary_stop_gpu(orc):
    """Two circles 6 sqrt(2) h away (in gradient norm) from their symmetric stationary point in a
    container of radius 2 - delta: the GPU stops after sweep 1 with status stationary when
    gsum_tol = 1e-9 >= 8.49e-10, runs on with 8e-10, and at h = 0 (a gradient of rounding size)
    stops as stationary with the library's 1e-12, as the oracle; with the rule off it does not
    report stationary."""
    torch, pecc = need_gpu()
    delta = 3e-3
    t = 1.0 - delta / 3.0
    n = np.array([2], dtype=np.int32)
    R = np.array([2.0 - delta])
    for h, tol in [(1e-10, 1e-9), (0.0, 1e-12)]:
        xy = np.array([[t + h, 0.0], [-(t + h), 0.0]])
        out = _run(pecc, torch, n, R, x0=xy, precision=0, max_iter=5, gsum_tol=tol)
        r = orc.gbo(xy, float(R[0]), max_iter=5, gsum_tol=tol)
        assert r.status == "stationary" and r.iters == 1
        assert (out["status"][0], out["iters"][0]) == (1, 1)
        assert out["E"][0] == pytest.approx(4.0 * delta ** 2 / 3.0, rel=1e-9)
    xy = np.array([[t + 1e-10, 0.0], [-(t + 1e-10), 0.0]])
    out = _run(pecc, torch, n, R, x0=xy, precision=0, max_iter=5, gsum_tol=8e-10)
    assert out["iters"][0] >= 2
    xy = np.array([[t, 0.0], [-t, 0.0]])
    out = _run(pecc, torch, n, R, x0=xy, precision=0, max_iter=5, gsum_tol=-1.0)
    assert out["status"][0] != 1


# ------------------------------------------------------------------ the binary32 descent
def _rows(cnt, col, lo, hi):
    return [np.sort(col[i, :cnt[i]]) for i in range(lo, hi)]


@pytest.mark.parametrize("cfg", [dict(max_iter=1), dict(max_iter=3, k_batches=2, lbfgs_m=5, step_max=0.3),
                                 dict(max_iter=60, k_batches=2, lbfgs_m=5, step_max=0.3),
                                 dict(max_iter=60, k_batches=2, lbfgs_m=5, step_max=0.3, list_outer=0.0),
                                 dict(max_iter=20, k_batches=2, lbfgs_m=5, step_max=0.3, list_outer=2.0 ** -9),
                                 dict(max_iter=20, k_batches=2, lbfgs_m=5, step_max=0.3, list_outer=1.5)])
def test_fp32_descent_lists_bit_exact(orc, cfg):
    """The lists the binary32 descent builds for itself (cell grid of side l_cut (1 + 2^-10) in
    binary32, the predicate s = dx dx + dy dy < l_cut^2 in binary32 without FMA, 16-bit indices in
    partition order) equal, row by row, the oracle's brute force with the binary32 predicate on the
    coordinates of that build.  Some circles start outside the container (clamped cell keys) and
    some coincide; after 60 sweeps ANM has deferred builds on stable instances."""
    torch, pecc = need_gpu()
    n = np.array([1000, 300, 57, 2, 640, 1], dtype=np.int32)
    R = _radii(n, 0.83)
    rng = np.random.default_rng(17)
    with pecc.Context(n, precision=1, **cfg) as c:
        c.set_radius(R)
        c.init_random(29)
        x0 = c.get_positions().cpu().numpy()
        x0[:40] *= 1.08  # outside the container
        x0[300:305] = x0[305]  # coincident centres
        x0 += rng.normal(scale=1e-3, size=x0.shape)
        c.set_positions(torch.from_numpy(x0))
        cnt, col, xb = c.set_list_dump(64)
        c.descend()
        cnt, col, xb = cnt.cpu().numpy(), col.cpu().numpy(), xb.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(n)])
    assert np.all(cnt >= 0)
    for q in range(len(n)):
        a, b = off[q], off[q + 1]
        x = xb[a:b]
        assert np.array_equal(x.astype(np.float32).astype(np.float64), x)  # binary32 values
        rref, cref = orc.neighbors_brute(x, 2.5, prec32=True)
        got = _rows(cnt, col, a, b)
        for i in range(b - a):
            assert np.array_equal(got[i], cref[rref[i]:rref[i + 1]]), (q, i)


def _fp32_bound(R, k, sweeps, step_max):
    """Position bound of a binary32 run against the binary64 oracle from the same coordinates.  Per
    batch step the binary32 step differs from the binary64 one by alpha |delta d| <= step_max 1e-5
    (the direction inherits the gradient's 1e-5 relative error, and alpha max|d| <= step_max) plus
    the rounding of the new coordinate, ulp32(R) / 2, and of alpha itself.  An earlier difference
    e enters the next gradients through the pair forces' Lipschitz constant (2 per overlapping
    pair, at most 6 pairs and the wall: L = 14), moved by at most alpha max|d| <= step_max per
    unit of gradient, so it grows by at most 1 + 14 step_max per step.  Over k sweeps x steps:"""
    u = float(np.spacing(np.float32(R)))
    steps = k * sweeps
    per = step_max * 1e-5 + u
    return steps * per * (1.0 + 14.0 * step_max) ** steps


@pytest.mark.parametrize("k,sweeps,step_max", [(1, 1, 0.1), (2, 1, 0.1), (2, 2, 0.1), (1, 3, 0.1), (2, 2, 0.3)])
def test_fp32_short_runs_follow_the_oracle(orc, k, sweeps, step_max):
    """A few sweeps of the binary32 descent (binary32 coordinates, pair terms, gradients,
    quasi-Newton vectors and energy sums) against the oracle's binary64 descent from the same
    binary32 coordinates, with the binary32 list predicate on both sides: the same iteration and
    trial counts, positions within the bound of _fp32_bound, and the energy of the GPU's final
    layout equal to its reported binary32 energy to 1e-5 relative plus the binary32 depth floor."""
    torch, pecc = need_gpu()
    n = np.array([300, 257, 640, 1000], dtype=np.int32)
    R = _radii(n, 0.82)
    out = _run(pecc, torch, n, R, seed=61, precision=1, k_batches=k, lbfgs_m=5, step_max=step_max,
               max_iter=sweeps, stall_window=0)
    worst = 0.0
    for q, (a, b) in enumerate(zip(split(out["x0"], n), split(out["x"], n))):
        r = orc.gbo(a, float(R[q]), k=k, m=5, step_max=step_max, max_iter=sweeps, prec32_pred=1)
        assert out["iters"][q] == r.iters and out["trials"][q] == r.trials, q
        err = np.max(np.abs(b - r.x))
        bound = _fp32_bound(float(R[q]), k, sweeps, step_max)
        worst = max(worst, err / bound)
        assert err <= bound, (q, err, bound)
        e_ref = orc.energy_allpairs(b, float(R[q]))
        sum_d = 2 * math.sqrt(max(e_ref, 0.0)) * math.sqrt(3 * n[q])
        u2 = float(np.spacing(np.float32(2.0)))
        assert abs(out["E"][q] - e_ref) <= 1e-5 * e_ref + 4 * u2 * sum_d, q
    print(f"worst position error / bound: {worst:.3g}")

"""GPU parity against the FP64 oracle, through the C ABI (marked gpu).

Bit-exact: random init (Philox, correctly rounded FP64), cell keys and stable order, neighbor
lists (Sec. 4.3 predicate in the coordinates' precision, no FMA), feasibility depths (Eq. 1,
Eq. 2 with correctly rounded operations).  Within tolerance: energy and gradient (Eq. 5 and its
gradient) in FP64 (1e-12 relative), FP32 and the mixed polish arithmetic (bounds derived in
the test docstrings), and short descents (Algorithm GBO) in FP64.
"""
import math

import numpy as np
import pytest

from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu, ragged_sizes, split

pytestmark = pytest.mark.gpu


def _ctx(pecc, n, R, **kw):
    c = pecc.Context(n, **kw)
    c.set_radius(R)
    return c


def _radii(n, u=0.83):
    return np.array([synth.radius(max(int(v), 1), u) for v in n])


# ------------------------------------------------------------------ init / cells / lists
@pytest.mark.parametrize("prec", [0, 1])
def test_init_bit_exact(orc, prec):
    torch, pecc = need_gpu()
    n = ragged_sizes()
    R = _radii(n)
    with _ctx(pecc, n, R, precision=prec) as c:
        c.init_random(12345)
        xy = c.get_positions().cpu().numpy()
    for q, part in enumerate(split(xy, n)):
        ref = orc.init_positions(int(n[q]), float(R[q]), 12345, inst=q)
        if prec == 1:
            ref = ref.astype(np.float32).astype(np.float64)
        assert np.array_equal(part, ref), q


def test_init_square_mode_bit_exact(orc):
    torch, pecc = need_gpu()
    n = np.array([100, 37], dtype=np.int32)
    R = _radii(n)
    with _ctx(pecc, n, R, precision=0, init_mode=1) as c:
        c.init_random(99)
        xy = c.get_positions().cpu().numpy()
    for q, part in enumerate(split(xy, n)):
        assert np.array_equal(part, orc.init_positions(int(n[q]), float(R[q]), 99, inst=q, mode=1))


@pytest.mark.parametrize("prec", [0, 1])
def test_cells_and_neighbors_bit_exact(orc, prec):
    torch, pecc = need_gpu()
    n = ragged_sizes()
    R = _radii(n, 0.85)
    rng = np.random.default_rng(3)
    with _ctx(pecc, n, R, precision=prec) as c:
        c.init_random(7)
        xy = c.get_positions().cpu().numpy()
        # perturb so that some circles leave the container and some coincide
        xy = xy + rng.normal(scale=0.3, size=xy.shape)
        xy[5] = xy[4]
        c.set_positions(torch.from_numpy(xy))
        xy = c.get_positions().cpu().numpy()
        c.rebuild_neighbors(force=True)
        key, order = [t.cpu().numpy() for t in c.export_cells()]
        rp, col = [t.cpu().numpy() for t in c.export_neighbors()]
    off = np.concatenate([[0], np.cumsum(n)])
    for q in range(len(n)):
        a, b = off[q], off[q + 1]
        x = xy[a:b]
        kref = orc.cell_keys(x, float(R[q]), 2.5)
        assert np.array_equal(key[a:b].astype(np.uint32), kref), q
        assert np.array_equal(order[a:b], np.argsort(kref, kind="stable")), q
        rref, cref = orc.neighbors_brute(x, 2.5, prec32=(prec == 1))
        rows = rp[a:b + 1] - rp[a]
        assert np.array_equal(rows, rref), q
        assert np.array_equal(col[rp[a]:rp[b]] - a, cref), q


# ------------------------------------------------------------------ energy and gradient
def _oracle_eg(orc, xy, n, R):
    Es, gs = [], []
    for q, x in enumerate(split(xy, n)):
        rp, col = orc.neighbors_brute(x, 2.5)
        E, g, _ = orc.energy_grad_csr(x, float(R[q]), rp, col)
        assert E == pytest.approx(orc.energy_allpairs(x, float(R[q])), rel=1e-12, abs=1e-300)
        Es.append(E)
        gs.append(g)
    return np.array(Es), np.concatenate(gs) if gs else np.zeros((0, 2))


def _contrib_scale(orc, xy, n, R):
    """Per circle, the sum of the norms of the terms its gradient adds up (2 d_ij per pair,
    2 d_i0 for the wall): the scale a normwise rounding bound on a sum refers to."""
    out = []
    for q, x in enumerate(split(xy, n)):
        s = np.zeros(len(x))
        if len(x):
            rp, col = orc.neighbors_brute(x, 2.5)
            for i in range(len(x)):
                js = col[rp[i]:rp[i + 1]]
                l = np.hypot(*(x[i] - x[js]).T) if len(js) else np.zeros(0)
                s[i] = np.sum(2 * np.maximum(0.0, 2 - l)) + 2 * max(0.0, np.hypot(*x[i]) + 1 - float(R[q]))
        out.append(s)
    return np.concatenate(out) if out else np.zeros(0)


def _layout(c, torch, seed, scale=1.0):
    c.init_random(seed)
    xy = c.get_positions().cpu().numpy() * scale
    c.set_positions(torch.from_numpy(xy))
    return c.get_positions().cpu().numpy()


def test_energy_grad_fp64(orc):
    torch, pecc = need_gpu()
    n = ragged_sizes()
    R = _radii(n, 0.83)
    with _ctx(pecc, n, R, precision=0) as c:
        xy = _layout(c, torch, 11, 1.03)
        c.rebuild_neighbors()
        E, g = [t.cpu().numpy() for t in c.energy_grad()]
    Er, gr = _oracle_eg(orc, xy, n, R)
    np.testing.assert_allclose(E, Er, rtol=1e-12, atol=1e-300)
    gn = np.linalg.norm(gr, axis=1)
    assert np.all(np.linalg.norm(g - gr, axis=1) <= 1e-12 * np.maximum(gn, 1e-300) + 1e-13)


def test_energy_grad_staged_and_per_circle_paths(orc):
    """Instances up to PECC_ENERGY_STAGE_BYTES of coordinates take the block kernel (coordinates
    staged in shared memory), larger ones the per-circle kernel and its reduction; one call with
    both kinds (7000 circles is past the FP64 limit of 6144) matches the oracle on every instance."""
    torch, pecc = need_gpu()
    n = np.array([7000, 300, 0, 50, 6144], dtype=np.int32)
    R = _radii(n, 0.83)
    with _ctx(pecc, n, R, precision=0) as c:
        xy = _layout(c, torch, 12, 1.03)
        c.rebuild_neighbors()
        E, g = [t.cpu().numpy() for t in c.energy_grad()]
    Er, gr = _oracle_eg(orc, xy, n, R)
    np.testing.assert_allclose(E, Er, rtol=1e-12, atol=1e-300)
    gn = np.linalg.norm(gr, axis=1)
    assert np.all(np.linalg.norm(g - gr, axis=1) <= 1e-12 * np.maximum(gn, 1e-300) + 1e-13)


def test_energy_grad_over_dense_instance(orc):
    """An over-dense instance (about 19 neighbors per circle, rows far longer than at the
    method's densities) beside ordinary and empty ones: every instance matches the oracle."""
    torch, pecc = need_gpu()
    n = np.array([300, 200, 0, 37], dtype=np.int32)
    R = np.array([math.sqrt(300 / 2.5), synth.radius(200, 0.83), 5.0, synth.radius(37, 0.83)])
    with _ctx(pecc, n, R, precision=0, nbr_capacity=40.0) as c:
        xy = _layout(c, torch, 21)
        c.rebuild_neighbors(force=True)
        rp, col = [t.cpu().numpy() for t in c.export_neighbors()]
        E, g = [t.cpu().numpy() for t in c.energy_grad()]
    assert rp[300] - rp[0] > 12 * 300  # long rows
    Er, gr = _oracle_eg(orc, xy, n, R)
    np.testing.assert_allclose(E, Er, rtol=1e-12, atol=1e-300)
    gn = np.linalg.norm(gr, axis=1)
    assert np.all(np.linalg.norm(g - gr, axis=1) <= 1e-12 * np.maximum(gn, 1e-300) + 1e-13)


def test_energy_grad_after_list_overflow_is_nan(orc):
    """Every circle of the first instance at one point: its list needs n - 1 entries per circle,
    over a capacity of 2 + 64 / n.  Its energy and gradient come back NaN (nothing past the
    capacity is read); the other instance, sparse enough for its capacity, is unaffected."""
    torch, pecc = need_gpu()
    n = np.array([64, 10], dtype=np.int32)
    R = np.array([20.0, 20.0])
    with _ctx(pecc, n, R, precision=0, nbr_capacity=2.0) as c:
        c.init_random(5)
        xy = c.get_positions().cpu().numpy()
        xy[:64] = 0.0
        c.set_positions(torch.from_numpy(xy))
        c.rebuild_neighbors(force=True)
        E, g = [t.cpu().numpy() for t in c.energy_grad()]
    assert np.isnan(E[0]) and np.all(np.isnan(g[:64]))
    Er, gr = _oracle_eg(orc, xy[64:], n[1:], R[1:])
    assert E[1] == pytest.approx(Er[0], rel=1e-12)
    assert np.all(np.isfinite(g[64:]))


def test_energy_grad_fp32(orc):
    """FP32: d = 2 - l carries an absolute error of about ulp(2) = 2.4e-7 per pair (and the
    wall depth about ulp(R)), so E is compared to 1e-5 relative plus 4 ulp32(2) * sum 2 d, and
    each circle's gradient to 1e-5 times the sum of its terms' norms plus 8 ulp32(R) times a
    neighbor count of 8."""
    torch, pecc = need_gpu()
    n = ragged_sizes()
    R = _radii(n, 0.83)
    with _ctx(pecc, n, R, precision=1) as c:
        xy = _layout(c, torch, 13, 1.03)
        c.rebuild_neighbors()
        E, g = [t.cpu().numpy().astype(np.float64) for t in c.energy_grad()]
    Er, gr = _oracle_eg(orc, xy, n, R)
    u2 = np.spacing(np.float32(2.0)).astype(np.float64)
    for q, (x, Rq) in enumerate(zip(split(xy, n), R)):
        if n[q] == 0:
            assert E[q] == 0.0
            continue
        sum_d = 2 * math.sqrt(max(Er[q], 0.0)) * math.sqrt(3 * n[q]) + 1e-30
        assert abs(E[q] - Er[q]) <= 1e-5 * Er[q] + 4 * u2 * sum_d + 1e-30, q
    uR = np.spacing(np.float32(R.max())).astype(np.float64)
    err = np.linalg.norm(g - gr, axis=1)
    assert np.all(err <= 1e-5 * _contrib_scale(orc, xy, n, R) + 8 * 8 * uR), err.max()


def test_energy_grad_mixed_polish_arithmetic(orc):
    """The polish arithmetic computes 4 - l^2 and |c|^2 - (R-1)^2 in FP64 and the depths from
    them in FP32: every depth and unit vector carries a relative error <= 4 ulp32 = 4.8e-7,
    so E is within 1e-6 relative and each gradient within 1e-6 times the sum of its terms'
    norms (the gradient itself can cancel to much less)."""
    torch, pecc = need_gpu()
    n = ragged_sizes()
    R = _radii(n, 0.83)
    with _ctx(pecc, n, R, precision=2) as c:
        xy = _layout(c, torch, 17, 1.02)
        c.rebuild_neighbors(eval=2)
        E, g = [t.cpu().numpy().astype(np.float64) for t in c.energy_grad(eval=2)]
    Er, gr = _oracle_eg(orc, xy, n, R)
    np.testing.assert_allclose(E, Er, rtol=1e-6, atol=1e-300)
    err = np.linalg.norm(g - gr, axis=1)
    assert np.all(err <= 1e-6 * _contrib_scale(orc, xy, n, R) + 1e-12)


def _mixed_bounds(e_ref, n, R):
    """Bounds of the polish arithmetic against the oracle at the same binary64 coordinates.  Each
    depth carries 3e-7 relative from its binary32 part, and an absolute delta from binary64
    rounding that neither side can avoid: the squared distance (rounded once with FMA on the GPU,
    twice in the oracle: ulp64(4)) and the oracle's wall depth (|c| + 1) - R (two roundings of
    size ulp64(R + 1)); delta = 4 ulp64(max(4, R + 1)).  With at most 4 n terms, sum d <=
    sqrt(4 n E) (Cauchy-Schwarz), so |dE| <= 1e-6 E + 2 delta sqrt(4 n E) + 4 n delta^2; each
    circle's gradient (at most 7 terms of 2 d) gains at most 16 delta."""
    delta = 4 * float(np.spacing(max(4.0, R + 1.0)))
    e_bound = 1e-6 * e_ref + 2 * delta * math.sqrt(4 * n * e_ref) + 4 * n * delta ** 2
    return e_bound, 16 * delta


def test_energy_near_contact_mixed_vs_fp64(orc):
    """Near contact the mixed arithmetic keeps relative accuracy: 4 - l^2 (and |c|^2 - (R-1)^2) are
    formed in binary64, where they cancel exactly (Sterbenz), and only the depths derived from them
    are binary32, each within about 5 ulp32 = 3e-7 relative (one rounding of 4 - s, the reciprocal
    square root, l, 2 + l and the division).  A squared depth then carries 6e-7, so E is within
    1e-6 relative of the oracle's and each circle's gradient within 1e-6 times the sum of its
    terms' norms; the same coordinates in a binary64 context give 1e-12.
    Two layouts: (1) a square lattice of 8 x 8 circles at spacing 2 - 2^-20, whose coordinates are
    binary32 values (so an FP32_POLISH64 context keeps them), E = 2 k (k - 1) 2^-40 by hand; (2) the
    binary64 layouts the polish itself reached, with contact depths down to 1e-10 and below."""
    torch, pecc = need_gpu()
    k, s_ = 8, 2.0 - 2.0 ** -20
    g1, g2 = np.meshgrid(np.arange(k), np.arange(k), indexing="ij")
    lat = np.stack([g1.ravel() * s_, g2.ravel() * s_], axis=1) - (k - 1) * s_ / 2
    assert np.array_equal(lat.astype(np.float32).astype(np.float64), lat)
    n = np.array([k * k], dtype=np.int32)
    R = np.array([100.0])
    with _ctx(pecc, n, R, precision=2) as c:
        c.set_positions(torch.from_numpy(lat))
        c.rebuild_neighbors(eval=2)
        E, g = [t.cpu().numpy().astype(np.float64) for t in c.energy_grad(eval=2)]
    assert E[0] == pytest.approx(2 * k * (k - 1) * 2.0 ** -40, rel=1e-6)
    Er, gr = _oracle_eg(orc, lat, n, R)
    err = np.linalg.norm(g - gr, axis=1)
    assert np.all(err <= 1e-6 * _contrib_scale(orc, lat, n, R) + _mixed_bounds(Er[0], int(n[0]), 100.0)[1])
    # the polish's own binary64 layouts: converged (u = 0.80) and jammed (u = 0.87) instances
    n = np.array([300, 300, 300, 300, 420, 420], dtype=np.int32)
    R = np.concatenate([_radii(n[:4], 0.80), _radii(n[4:], 0.87)])
    with _ctx(pecc, n, R, precision=2, polish_gate=1.0) as c:
        c.init_random(57)
        c.descend()
        pol = c.get_stats().cpu().numpy()[:, 7]
        xy = c.get_positions().cpu().numpy()
        c.rebuild_neighbors(eval=2)
        E, g = [t.cpu().numpy().astype(np.float64) for t in c.energy_grad(eval=2)]
    assert pol.sum() >= 4
    Er, gr = _oracle_eg(orc, xy, n, R)
    assert np.any(Er < 1e-18) and np.any(Er > 1e-10)
    floors = []
    for q in range(len(n)):
        eb, gf = _mixed_bounds(Er[q], int(n[q]), float(R[q]))
        assert abs(E[q] - Er[q]) <= eb, (q, E[q], Er[q])
        floors.append(np.full(n[q], gf))
    err = np.linalg.norm(g - gr, axis=1)
    assert np.all(err <= 1e-6 * _contrib_scale(orc, xy, n, R) + np.concatenate(floors))
    with _ctx(pecc, n, R, precision=0) as c64:
        c64.set_positions(torch.from_numpy(xy))
        c64.rebuild_neighbors()
        E64, g64 = [t.cpu().numpy() for t in c64.energy_grad()]
    # binary64 throughout: 1e-12 relative, down to the same binary64 rounding floor
    for q in range(len(n)):
        eb = _mixed_bounds(Er[q], int(n[q]), float(R[q]))[0] - 1e-6 * Er[q]
        assert abs(E64[q] - Er[q]) <= 1e-12 * Er[q] + eb, (q, E64[q], Er[q])
    assert np.all(np.linalg.norm(g64 - gr, axis=1) <= 1e-12 * _contrib_scale(orc, xy, n, R) + np.concatenate(floors))


# ------------------------------------------------------------------ feasibility
def test_check_feasible_bit_exact(orc):
    torch, pecc = need_gpu()
    n = ragged_sizes()
    R = _radii(n, 0.6)
    with _ctx(pecc, n, R, precision=0) as c:
        xy = _layout(c, torch, 5, 0.9)
        feas, mo = [t.cpu().numpy() for t in c.check_feasible(1e-9)]
    for q, x in enumerate(split(xy, n)):
        ref = orc.max_overlap(x, float(R[q]))[0]
        assert mo[q] == ref, (q, mo[q], ref)
        assert feas[q] == (ref <= 1e-9)


def test_check_feasible_exact_packings(orc):
    torch, pecc = need_gpu()
    pts = [np.array([[-1.0, 0.0], [1.0, 0.0]]),
           np.vstack([[0, 0], 2 * np.stack([np.cos(np.arange(6) * np.pi / 3), np.sin(np.arange(6) * np.pi / 3)], 1)])]
    n = np.array([2, 7], dtype=np.int32)
    R = np.array([2.0, 3.0])
    with _ctx(pecc, n, R, precision=0) as c:
        c.set_positions(torch.from_numpy(np.concatenate(pts)))
        feas, mo = [t.cpu().numpy() for t in c.check_feasible(1e-9)]
    assert feas.tolist() == [1, 1]
    assert mo[0] == 0.0 and mo[1] <= 1e-15


# ------------------------------------------------------------------ descent
@pytest.mark.parametrize("k,sweeps", [(1, 1), (1, 4), (3, 1), (3, 3), (5, 2)])
def test_descend_short_runs_fp64(orc, k, sweeps):
    """A few GBO sweeps in FP64 from the same layout: the GPU (vector-free two-loop, FMA pair
    arithmetic) and the oracle (explicit two-loop, correctly rounded) take the same steps up to
    rounding: positions agree to 1e-9 and energies to 1e-9 relative."""
    torch, pecc = need_gpu()
    n = np.array([300, 257, 1000], dtype=np.int32)
    R = _radii(n, 0.8)
    with _ctx(pecc, n, R, precision=0, k_batches=k, max_iter=sweeps) as c:
        c.init_random(21)
        x0 = c.get_positions().cpu().numpy()
        iters, status = c.descend()
        x1 = c.get_positions().cpu().numpy()
        E = c.get_energy().cpu().numpy()
        iters = iters.cpu().numpy()
    for q, (a, b) in enumerate(zip(split(x0, n), split(x1, n))):
        r = orc.gbo(a, float(R[q]), k=k, max_iter=sweeps)
        assert iters[q] == r.iters
        np.testing.assert_allclose(b, r.x, rtol=0, atol=1e-9 * float(R[q]))
        assert E[q] == pytest.approx(r.E, rel=1e-9)


@pytest.mark.parametrize("sweeps", [1, 3, 6])
def test_descend_short_runs_at_the_batch_settings_fp64(orc, sweeps):
    """The batch workload's settings (k = 2, m = 5 secant pairs, step cap 0.3, so that the Verlet
    rule rebuilds once the largest displacement passes 0.1): a few binary64 sweeps follow the
    oracle's at the same settings to 1e-9."""
    torch, pecc = need_gpu()
    n = np.array([300, 257, 640, 1000], dtype=np.int32)
    R = _radii(n, 0.82)
    with _ctx(pecc, n, R, precision=0, k_batches=2, lbfgs_m=5, step_max=0.3, max_iter=sweeps) as c:
        c.init_random(71)
        x0 = c.get_positions().cpu().numpy()
        iters, status = c.descend()
        x1 = c.get_positions().cpu().numpy()
        E = c.get_energy().cpu().numpy()
        iters = iters.cpu().numpy()
    for q, (a, b) in enumerate(zip(split(x0, n), split(x1, n))):
        r = orc.gbo(a, float(R[q]), k=2, m=5, step_max=0.3, max_iter=sweeps)
        assert iters[q] == r.iters
        np.testing.assert_allclose(b, r.x, rtol=0, atol=1e-9 * float(R[q]))
        assert E[q] == pytest.approx(r.E, rel=1e-9)


@pytest.mark.parametrize("part,k,sweeps", [(3, 3, 2), (3, 5, 3), (1, 3, 2), (2, 4, 2)])
def test_descend_short_runs_other_partitions_fp64(orc, part, k, sweeps):
    """The annulus, fence and random partitions of Sec. 4.1 (random: Philox-keyed order under
    partition_seed, instance word q): a few binary64 sweeps follow the oracle's to 1e-9."""
    torch, pecc = need_gpu()
    n = np.array([300, 257, 640], dtype=np.int32)
    R = _radii(n, 0.8)
    with _ctx(pecc, n, R, precision=0, k_batches=k, max_iter=sweeps, partition=part, partition_seed=4242) as c:
        c.init_random(33)
        x0 = c.get_positions().cpu().numpy()
        iters, status = c.descend()
        x1 = c.get_positions().cpu().numpy()
        E = c.get_energy().cpu().numpy()
        iters = iters.cpu().numpy()
    for q, (a, b) in enumerate(zip(split(x0, n), split(x1, n))):
        r = orc.gbo(a, float(R[q]), k=k, max_iter=sweeps, partition=part, part_seed=4242, part_inst=q)
        assert iters[q] == r.iters
        np.testing.assert_allclose(b, r.x, rtol=0, atol=1e-9 * float(R[q]))
        assert E[q] == pytest.approx(r.E, rel=1e-9)


def _solve(pecc, torch, n, R, seed, **kw):
    with _ctx(pecc, n, R, **kw) as c:
        c.init_random(seed)
        iters, status = c.descend()
        feas, mo = c.check_feasible()
        xy = c.get_positions().cpu().numpy()
        E = c.get_energy().cpu().numpy()
        return dict(iters=iters.cpu().numpy(), status=status.cpu().numpy(), feasible=feas.cpu().numpy(),
                    max_overlap=mo.cpu().numpy(), xy=xy, E=E, polished=c.get_stats().cpu().numpy()[:, 7],
                    precision=c.precision)


@pytest.mark.parametrize("prec", [0, 2])
def test_descend_statistics_vs_oracle(orc, prec):
    """Whole descents diverge from the oracle's after many nonconvex steps (rounding order), so
    they are compared as outcomes: at u = 0.80, n = 300 both reach E <= 1e-20 on most seeds,
    every instance the GPU calls converged is feasible by the oracle's own brute-force check,
    and the GPU's max overlap equals the oracle's on the GPU's final layout."""
    torch, pecc = need_gpu()
    num = 16
    n = np.full(num, 300, dtype=np.int32)
    R = _radii(n, 0.80)
    out = _solve(pecc, torch, n, R, 31, precision=prec)
    _, ref = orc.solve_batch(n, R, 31, nthreads=8)
    for q, x in enumerate(split(out["xy"], n)):
        mo = orc.max_overlap(x, float(R[q]))[0]
        assert out["max_overlap"][q] == mo
        if out["status"][q] == 0:
            assert out["E"][q] <= 1e-20 and mo <= 1e-9
    assert out["feasible"].sum() >= num - 4
    assert abs(int(out["feasible"].sum()) - int(ref["feasible"].sum())) <= 5


def _check_outcomes(orc, out, n, R):
    """Per instance: the max overlap equals the oracle's on the GPU's own final layout, the energy
    the GPU reports is the oracle's energy of that layout, and converged means feasible.  The
    energy bound follows the arithmetic that produced it:
    - binary64 (plain FP64 context): 1e-12 relative plus the binary64 rounding floor of
      _mixed_bounds (at converged layouts, E ~ 1e-21, the floor is the larger term);
    - a polished instance reports its energy in the polish arithmetic (binary64 4 - l^2, binary32
      depths within 3e-7 relative, squared and summed in binary64): 1e-6 relative plus the binary64
      rounding floor of _mixed_bounds;
    - an instance left unpolished reports its binary32 energy: each depth 2 - l carries up to
      4 ulp32(2) absolute, so 1e-5 relative plus 4 ulp32(2) times the sum of 2 d over the pairs,
      which Cauchy-Schwarz bounds by 2 sqrt(3 n E)."""
    u2 = float(np.spacing(np.float32(2.0)))
    for q, x in enumerate(split(out["xy"], n)):
        mo = orc.max_overlap(x, float(R[q]))[0]
        assert out["max_overlap"][q] == mo, q
        e_ref = orc.energy_allpairs(x, float(R[q]))
        if out.get("precision", 2) == 0:
            bound = 1e-12 * e_ref + _mixed_bounds(e_ref, int(n[q]), float(R[q]))[0] - 1e-6 * e_ref
        elif out["polished"][q]:
            bound = _mixed_bounds(e_ref, int(n[q]), float(R[q]))[0]
        else:
            bound = 1e-5 * e_ref + 4 * u2 * 2 * math.sqrt(3 * n[q] * e_ref) + 1e-30
        assert abs(out["E"][q] - e_ref) <= bound, (q, out["E"][q], e_ref, out["polished"][q])
        if out["status"][q] == 0:
            assert out["E"][q] <= 1e-20 and mo <= 1e-9, q


def test_descend_outcomes_at_the_batch_settings(orc):
    """The batch workload's settings on the FP32 + polish path (k = 2, m = 5, step cap 0.3, polish
    gate 1e-5, stagnation checks every 5 / 50 sweeps): the same per-instance checks as at the
    library's settings, and a feasible count within 5 of the oracle's at the same k, m and cap."""
    torch, pecc = need_gpu()
    n = np.array([300, 420, 640, 900, 1000, 512] * 4, dtype=np.int32)
    R = _radii(n, 0.80)
    cfg = dict(k_batches=2, lbfgs_m=5, step_max=0.3, polish_gate=1e-5, stall_window=5, polish_stall_window=50)
    out = _solve(pecc, torch, n, R, 43, precision=2, **cfg)
    _check_outcomes(orc, out, n, R)
    _, ref = orc.solve_batch(n, R, 43, nthreads=8, k=2, m=5, step_max=0.3)
    assert out["feasible"].sum() >= len(n) - 8
    assert abs(int(out["feasible"].sum()) - int(ref["feasible"].sum())) <= 5


@pytest.mark.parametrize("block", [128, 512])
def test_descend_launch_shapes(orc, block):
    """FP32 descent and FP64 polish at 128 and 512 threads per block (the polish at min(block,
    256)), over instances of one batch (n < 300, and every polish) and of several: the same
    outcomes as the oracle's (22 of these 24 reach zero energy in the oracle)."""
    torch, pecc = need_gpu()
    n = np.array([120, 200, 299, 300, 420, 640] * 4, dtype=np.int32)
    R = _radii(n, 0.80)
    out = _solve(pecc, torch, n, R, 41, precision=2, block_threads=block)
    _check_outcomes(orc, out, n, R)
    _, ref = orc.solve_batch(n, R, 41, nthreads=8)
    assert out["feasible"].sum() >= len(n) - 6
    assert abs(int(out["feasible"].sum()) - int(ref["feasible"].sum())) <= 5


@pytest.mark.parametrize("num,bps,smem", [(21, 0, 0), (600, 1, 8192)])
def test_fused_phases_equal_two_kernels(orc, num, bps, smem):
    """The fused kernel (each instance's FP32 descent and polish back to back in one block) runs
    the same arithmetic in the same order as the two-kernel path: with the same threads per block
    the final coordinates, statuses and sweep counts are identical bit for bit.  The second case
    puts about four instances on each block and caps shared memory at 8 KB, so the working sets
    live in global memory while FP32 phases and polishes of different instances run at once."""
    torch, pecc = need_gpu()
    if num == 21:
        n = np.array([120, 200, 299, 300, 420, 640, 1000] * 3, dtype=np.int32)
        R = _radii(n, 0.80)
    else:
        n, R = synth.batch_manifest(num, seed=44)
    outs = []
    for fuse in (1, 0):
        with _ctx(pecc, n, R, precision=2, block_threads=128, blocks_per_sm=bps, smem_per_block=smem,
                  fuse_phases=fuse) as c:
            c.init_random(17)
            iters, status = c.descend()
            outs.append((c.get_positions().cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy(),
                         c.get_stats().cpu().numpy(), c.get_energy().cpu().numpy()))
            ms = c.phase_times()
            assert (ms[1] < 0.05) == bool(fuse)  # fused: the polish event follows the kernel at once
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)


def test_autotune_restores_coordinates_and_descends(orc):
    """pecc_autotune times short descents at every launch shape, then hands the caller back its
    coordinates bit for bit; the descent that follows runs at the chosen shape with the same
    outcomes as the oracle's."""
    torch, pecc = need_gpu()
    n = np.array([120, 200, 299, 300, 420, 640] * 4, dtype=np.int32)
    R = _radii(n, 0.80)
    with _ctx(pecc, n, R, precision=2) as c:
        c.init_random(41)
        x0 = c.get_positions().cpu().numpy()
        b, t = c.autotune(sweeps=5, seed=9)
        assert b in (128, 256, 512) and t in (1, 2, 4)
        assert np.array_equal(c.get_positions().cpu().numpy(), x0)
        iters, status = c.descend()
        assert c.launch_shape()[0] == b
        feas, mo = c.check_feasible()
        out = dict(status=status.cpu().numpy(), feasible=feas.cpu().numpy(), max_overlap=mo.cpu().numpy(),
                   xy=c.get_positions().cpu().numpy(), E=c.get_energy().cpu().numpy(),
                   polished=c.get_stats().cpu().numpy()[:, 7], precision=c.precision)
    _check_outcomes(orc, out, n, R)
    assert out["feasible"].sum() >= len(n) - 6


def test_descend_infeasible_density_small(orc):
    """n = 50 at u = 0.80 is denser than any packing of 50 circles: no descent reaches zero
    energy, on the GPU or in the oracle, and every run ends by stalling or at max_iter."""
    torch, pecc = need_gpu()
    n = np.full(8, 50, dtype=np.int32)
    R = _radii(n, 0.80)
    out = _solve(pecc, torch, n, R, 1, precision=0)
    assert out["feasible"].sum() == 0
    assert set(out["status"].tolist()) <= {1, 2, 3}
    assert np.all(out["E"] > 1e-6)


def test_descend_ragged_and_degenerate(orc):
    torch, pecc = need_gpu()
    n = ragged_sizes()
    R = _radii(n, 0.7)
    out = _solve(pecc, torch, n, R, 3, precision=2)
    assert out["status"][0] == 0 and out["feasible"][0] == 1   # n = 0
    assert out["status"][1] == 0 and out["feasible"][1] == 1   # n = 1
    for q, x in enumerate(split(out["xy"], n)):
        assert out["max_overlap"][q] == orc.max_overlap(x, float(R[q]))[0]
    assert out["feasible"][2:].sum() >= 6


def test_descend_nonfinite_input_flagged(orc):
    torch, pecc = need_gpu()
    n = np.array([20, 20], dtype=np.int32)
    R = _radii(n, 0.5)
    with _ctx(pecc, n, R, precision=1) as c:
        c.init_random(1)
        xy = c.get_positions().cpu().numpy()
        xy[3, 0] = np.nan
        c.set_positions(torch.from_numpy(xy))
        iters, status = c.descend()
        assert status.cpu().numpy().tolist()[0] == 5
        assert status.cpu().numpy().tolist()[1] in (0, 1, 2)


def test_descend_capacity_overflow_flagged(orc):
    """Every circle at one point: each list holds n - 1 entries, over a capacity of 1 per circle."""
    torch, pecc = need_gpu()
    n = np.array([200], dtype=np.int32)
    with _ctx(pecc, n, np.array([20.0]), precision=1, nbr_capacity=1.0) as c:
        c.set_positions(torch.zeros((200, 2), dtype=torch.float64))
        iters, status = c.descend()
        assert int(status.cpu()[0]) == 4


def test_descend_time_budget(orc):
    torch, pecc = need_gpu()
    n = np.full(4, 1000, dtype=np.int32)
    with _ctx(pecc, n, _radii(n, 0.84), precision=1, time_budget_ns=1) as c:
        c.init_random(2)
        iters, status = c.descend()
        assert set(status.cpu().numpy().tolist()) == {6}
        assert np.all(iters.cpu().numpy() == 1)


def test_solve_host_matches_device_path(orc):
    torch, pecc = need_gpu()
    n = np.array([300, 420, 64], dtype=np.int32)
    R = _radii(n, 0.8)
    with _ctx(pecc, n, R, precision=2) as c:
        h = c.solve_host(R, 77)
    d = _solve(pecc, torch, n, R, 77, precision=2)
    np.testing.assert_array_equal(h["xy"], d["xy"])
    np.testing.assert_array_equal(h["feasible"], d["feasible"])
    np.testing.assert_array_equal(h["iters"], d["iters"])

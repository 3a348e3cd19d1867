"""Pins of the oracle's SED heuristic (Sec. 5.2, Algorithm SED, the select operator of Eq. 18).

- J(E) = ceil(-log10 E) is checked against exact rational arithmetic:
  10^-J <= E < 10^(1-J).
- The perturbation is checked against the uniform law U(-0.8, 0.8) by moments, a KS test and
  independence of x and y, and against the printed form (one r for both coordinates) when shared.
- select is checked against its two branches: the argmin, and the softmax law over J by a
  chi-square test.
- The search is checked against invariants of Algorithm SED: E(x*) never rises,
  m = max(1, J(E(x))), and the descent count is 1 + the sum of m.
- Its purpose is checked too: it reaches zero energy at the exact radius of 7 circles, and it
  lowers the energy of dense jammed layouts.
- The framework of Sec. 5.1 keeps the exact radii of 2, 3 and 7 circles, its record never
  grows, and on a dense instance it ends below R_b with a feasible layout.
"""
from fractions import Fraction

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")


def _near_power_of_ten(E):
    k = np.round(np.log10(E))
    return abs(E / 10.0 ** k - 1.0) < 1e-12


def test_J_is_the_ceiling_of_minus_log10(orc):
    rng = np.random.default_rng(3)
    Es = 10.0 ** rng.uniform(-32, 4, size=3000)
    for E in Es:
        if _near_power_of_ten(E):
            continue
        J = orc.sed_J(E)
        f = Fraction(float(E))
        assert Fraction(10) ** (-J) <= f < Fraction(10) ** (1 - J), (E, J)
    assert [orc.sed_J(v) for v in (0.5, 2.0, 50.0, 0.05, 3e-7, 1.0)] == [1, 0, -1, 2, 7, 0]
    assert orc.sed_J(0.0) == 1 << 30


def test_perturbation_is_uniform_and_independent(orc):
    n = 200_000
    x0 = np.zeros((n, 2))
    p = orc.sed_perturb(x0, seed=7, inst=3, it=5, j=2)
    r = p.ravel()
    assert r.min() >= -0.8 and r.max() < 0.8
    assert abs(r.mean()) < 5 * 0.8 / np.sqrt(3 * r.size)
    assert r.var() == pytest.approx(0.64 / 3.0, rel=0.01)
    assert scipy_stats.kstest((r + 0.8) / 1.6, "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(p[:, 0], p[:, 1])[0, 1]) < 5 / np.sqrt(n)
    # the printed form: one r shared by both coordinates of a circle
    ps = orc.sed_perturb(x0[:1000], seed=7, inst=3, it=5, j=2, shared=1)
    assert np.array_equal(ps[:, 0], ps[:, 1])
    assert np.array_equal(ps[:, 0], p[:1000, 0])


def test_perturbation_adds_to_the_layout_and_streams_are_distinct(orc):
    rng = np.random.default_rng(1)
    x = rng.uniform(-5, 5, size=(300, 2))
    a = orc.sed_perturb(x, 11, 0, 0, 0)
    assert np.array_equal(a, orc.sed_perturb(x, 11, 0, 0, 0))  # counter-based: reproducible
    d = a - x
    assert np.all(np.abs(d) <= 0.8)
    others = [orc.sed_perturb(x, 11, 0, 0, 1), orc.sed_perturb(x, 11, 0, 1, 0), orc.sed_perturb(x, 11, 1, 0, 0),
              orc.sed_perturb(x, 12, 0, 0, 0)]
    for o in others:
        assert not np.any(o == a)
    # the initial layouts use the counters with c3 = 0: none of the perturbation's draws repeat them
    init = orc.init_positions(300, 7.0, 11, inst=0, mode=1)
    assert not np.any(np.isclose((d / 0.8), init / 7.0, rtol=0, atol=1e-15))


def test_select_takes_the_least_energy_when_it_improves(orc):
    assert orc.sed_select([3.0, 1.0, 2.0], 5.0, 1, 0, 0) == 1
    assert orc.sed_select([1.0, 1.0, 3.0], 5.0, 1, 0, 0) == 0  # the first of equal energies
    assert orc.sed_select([10.0], 1.0, 1, 0, 0) == 0  # one candidate: always taken
    assert orc.sed_select([2e-3, 5e-4, 1e-3], 1e-3, 1, 0, 0) == 1


def test_select_draws_by_softmax_of_J_otherwise(orc):
    E = [1e-3 * 1.7, 1e-5 * 2.3, 0.5]  # J = 3, 5, 1
    J = np.array([orc.sed_J(v) for v in E])
    assert J.tolist() == [3, 5, 1]
    draws = 30000
    counts = np.zeros(3)
    for it in range(draws):
        counts[orc.sed_select(E, 1e-9, 5, 2, it)] += 1
    p = np.exp(J - J.max())
    p /= p.sum()
    chi2 = scipy_stats.chisquare(counts, p * draws)
    assert chi2.pvalue > 1e-4, (counts, p * draws)
    # equal J: uniform
    counts = np.zeros(4)
    for it in range(8000):
        counts[orc.sed_select([0.5, 0.3, 0.2, 0.6], 0.01, 9, 0, it)] += 1
    assert scipy_stats.chisquare(counts).pvalue > 1e-4


def test_reaches_zero_energy_at_the_exact_radius_of_seven(orc):
    """R = 3 packs 7 circles exactly (hexagonal).  The search ends with E(x*) <= 1e-25."""
    for seed in range(1, 6):
        r = orc.sed(7, 3.0, seed, s_iter=20)
        assert r.status == "converged" and r.E <= 1e-25, (seed, r.E, r.iters)
        assert orc.max_overlap(r.x, 3.0)[0] <= 1e-9


@pytest.mark.parametrize("n,R", [(1, 1.0), (2, 2.0), (3, 1.0 + 2.0 / np.sqrt(3.0))])
def test_reaches_zero_energy_at_the_smallest_exact_radii(orc, n, R):
    """One circle at R = 1, two at R = 2 and three at R = 1 + 2/sqrt(3) pack exactly: the search
    ends converged (E(x*) <= e_feas = 1e-25) with a feasible layout."""
    for seed in range(1, 4):
        r = orc.sed(n, R, seed, s_iter=20)
        assert r.status == "converged" and r.E <= 1e-25, (seed, r.E)
        assert orc.max_overlap(r.x, R)[0] <= 1e-9


def test_trace_invariants_on_a_dense_instance(orc):
    n, R = 30, np.sqrt(30 / 0.80)
    r = orc.sed(n, R, 2, s_iter=10)
    assert r.iters == 10 and r.status == "max_iter"
    Eprev = r.E0
    for t in range(r.iters):
        assert r.m[t] == min(25, max(1, orc.sed_J(Eprev)))
        assert 0 <= r.sel[t] < r.m[t]
        Eprev = r.Ex[t]
    assert np.all(np.diff(np.concatenate([[r.E0], r.Eb])) <= 0.0)  # E(x*) never rises
    assert r.E == r.Eb[-1] == min(r.E0, r.Ex.min())
    assert r.descents == 1 + int(r.m.sum())
    assert orc.energy_allpairs(r.x, R) == pytest.approx(r.E, rel=1e-9)


def test_lowers_the_energy_of_jammed_layouts(orc):
    """Dense layouts (u = 0.80 at n = 30): the first descent jams above zero energy; exploring
    finds lower minima in some runs and never a higher one."""
    n, R = 30, np.sqrt(30 / 0.80)
    lowered = 0
    for seed in (2, 4):
        r = orc.sed(n, R, seed, s_iter=12)
        assert r.E <= r.E0
        lowered += r.E < 0.5 * r.E0
    assert lowered >= 1


def test_easy_instance_needs_no_exploring(orc):
    r = orc.sed(19, np.sqrt(19 / 0.80), 3, s_iter=10)
    assert r.iters == 0 and r.status == "converged" and r.descents == 1


# ---------------------------------------------------------------- the framework (Sec. 5.1)
R3 = 1.0 + 2.0 / np.sqrt(3.0)


@pytest.mark.parametrize("n,Rb", [(2, 2.0), (3, R3), (7, 3.0)])
def test_framework_keeps_the_exact_radius(orc, n, Rb):
    """At the exact radius of 2, 3 and 7 circles the framework's record is that radius (to
    rounding) with a feasible layout, and the record never grows."""
    x, R, tr = orc.frame(n, Rb, 5, outer=2, s_iter=5)
    assert abs(R - Rb) <= 1e-9
    assert orc.max_overlap(x, R)[0] <= 1e-9
    assert np.all(np.diff(tr) <= 0.0)


def test_framework_improves_a_dense_instance(orc):
    """n = 40 at R_b = sqrt(40 / 0.78): the first adjustment enlarges the container; searching at
    min(R_b, R*) then finds a feasible layout below R_b.  The record only shrinks."""
    n, Rb = 40, np.sqrt(40 / 0.78)
    x, R, tr = orc.frame(n, Rb, 2, outer=3, s_iter=3, max_iter=300)
    assert np.all(np.diff(tr) <= 0.0)
    assert tr[0] > Rb and R < Rb
    assert R == tr[-1]
    assert orc.max_overlap(x, R)[0] <= 1e-9


@pytest.mark.parametrize("Rb", [1.0, 1.5, 3.0])
def test_framework_one_circle_reaches_the_unit_radius(orc, Rb):
    """One circle packs exactly into R = 1 (its centre at the origin). From any R_b >= 1 the
    adjustments take the record there, within the schedule's last lambda, feasibly."""
    x, R, tr = orc.frame(1, Rb, 3, outer=2, s_iter=3)
    assert abs(R - 1.0) <= 1e-9
    assert orc.max_overlap(x, R)[0] <= 1e-9
    assert np.all(np.diff(tr) <= 0.0)


def test_framework_empty_instance_keeps_its_radius(orc):
    x, R, tr = orc.frame(0, 2.0, 3, outer=1, s_iter=2)
    assert x.shape == (0, 2) and R == 2.0 and np.all(tr == 2.0)

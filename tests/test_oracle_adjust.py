"""Pins of the oracle's container adjustment (Sec. 4.2, Algorithm adjust_container, Eq. 12).

U(z, lambda) = E(x, R) + lambda R^2 over z = (x, R).  The gradient is checked against finite
differences; the minimiser over R is checked against closed forms.  Just below the exact radius
of n = 2, 3 and 7 circles, the symmetric stationary energies are 4 d^2/3, 9 d^2/4 and 4 d^2
(d = R_exact - R, the same closed forms that pin E).  So the radius minimising E + lambda R^2
is R_exact / (1 + c lambda) with c = 3/4, 4/9 and 1/4: setting dU/dR = -2 a (R_exact - R)
+ 2 lambda R to zero (a = 4/3, 9/4, 4) gives R = R_exact / (1 + lambda / a).
"""
import numpy as np
import pytest

from paper_2303_02650_gb300 import synth

R3 = 1.0 + 2.0 / np.sqrt(3.0)


def _sym(n, R):
    """The symmetric stationary layout of n = 2, 3 or 7 circles in a container of radius R (below
    the exact radius): the ring radius a that minimises E for that R."""
    if n == 2:
        a = (1.0 + R) / 3.0
        return np.array([[a, 0.0], [-a, 0.0]])
    if n == 3:
        # E = 3 (2 - a sqrt3)^2 + 3 (a + 1 - R)^2, stationary at a = (2 sqrt3 + R - 1) / 4
        a = (2.0 * np.sqrt(3.0) + R - 1.0) / 4.0
        ang = np.pi / 2 + np.arange(3) * 2 * np.pi / 3
        return np.c_[a * np.cos(ang), a * np.sin(ang)]
    if n == 7:
        s = 1.0 + R / 3.0
        ang = np.arange(6) * np.pi / 3
        return np.vstack([[0.0, 0.0], np.c_[s * np.cos(ang), s * np.sin(ang)]])
    raise ValueError(n)


EXACT = {2: (2.0, 4.0 / 3.0), 3: (R3, 9.0 / 4.0), 7: (3.0, 4.0)}


def test_u_gradient_finite_differences(orc):
    rng = np.random.default_rng(5)
    n = 30
    R = synth.radius(n, 0.9)
    x = rng.uniform(-R, R, size=(n, 2)) * 0.9
    lam = 0.37
    U, g = orc.u_energy_grad(x, R, lam)
    assert U == pytest.approx(orc.energy_allpairs(x, R) + lam * R * R, rel=1e-13)
    h = 1e-6
    fd = np.zeros(2 * n + 1)
    for i in range(2 * n):
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[i] += h
        xm[i] -= h
        fd[i] = (orc.u_energy_grad(xp.reshape(n, 2), R, lam)[0] - orc.u_energy_grad(xm.reshape(n, 2), R, lam)[0]) / (2 * h)
    fd[2 * n] = (orc.u_energy_grad(x, R + h, lam)[0] - orc.u_energy_grad(x, R - h, lam)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6)
    assert g[2 * n] < 0 or lam * R > 0  # the wall pushes R outwards, the penalty inwards


@pytest.mark.parametrize("n", [2, 3, 7])
@pytest.mark.parametrize("lam", [0.1, 0.01])
def test_adjust_single_round_closed_forms(orc, n, lam):
    Rx, a = EXACT[n]
    R0 = Rx - 0.1
    xs, Rs, res = orc.adjust_container(_sym(n, R0), R0, lambda0=lam, rounds=1)
    assert Rs == pytest.approx(Rx / (1.0 + lam / a), rel=1e-9)


@pytest.mark.parametrize("n", [2, 3, 7])
def test_adjust_full_schedule_reaches_the_exact_radius(orc, n):
    """35 rounds from lambda = 1e-4: the last lambda is 1e-4 / 2^34, so the radius ends within
    about 1e-14 of the exact one, and the layout is feasible."""
    Rx, _ = EXACT[n]
    R0 = Rx - 0.1
    xs, Rs, res = orc.adjust_container(_sym(n, R0), R0)
    assert abs(Rs - Rx) <= 1e-9
    assert orc.max_overlap(xs, Rs)[0] <= 1e-9


def test_adjust_random_infeasible_layout_becomes_feasible(orc):
    """A GBO local minimum above zero energy (n = 40 at u = 0.86, denser than the best known
    packings) is made feasible by enlarging the container, and the radius grows only a little."""
    n = 40
    R0 = synth.radius(n, 0.86)
    x0 = orc.init_positions(n, R0, 3)
    r = orc.gbo(x0, R0)
    assert orc.max_overlap(r.x, R0)[0] > 1e-6
    xs, Rs, res = orc.adjust_container(r.x, R0)
    assert orc.max_overlap(xs, Rs)[0] <= 1e-9
    assert R0 < Rs < 1.1 * R0


@pytest.mark.parametrize("lam", [0.3, 0.05])
def test_one_circle_closed_form(orc, lam):
    """One circle: U = (|c| + 1 - R)^2 + lambda R^2 is least at c = 0 with R = 1 / (1 + lambda)
    (dU/dR = -2 (1 - R) + 2 lambda R = 0); the full schedule ends at R = 1 (the circle itself).
    |c| is a cone at the centre, so the wall's force keeps its size 2 (1 - R) as c -> 0 and the
    search stalls once c oscillates about 0: one round settles R to about 1e-8 (measured
    1.2e-8), the schedule (1 - R -> 0) to 1e-9."""
    x0 = np.array([[0.3, -0.2]])
    xs, Rs, res = orc.adjust_container(x0, 0.9, lambda0=lam, rounds=1)
    assert Rs == pytest.approx(1.0 / (1.0 + lam), rel=1e-7)
    assert np.abs(xs).max() <= 1e-6
    xs, Rs, res = orc.adjust_container(x0, 0.9)
    assert abs(Rs - 1.0) <= 1e-9

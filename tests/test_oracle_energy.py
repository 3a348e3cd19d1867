"""Pins for the oracle's energy (Eq. 3, Eq. 5, Eq. 7) and gradient (CPU only)."""
import math

import numpy as np
import pytest

from paper_2303_02650_gb300 import synth


def _hexagon7(R_in=2.0, rot=0.0):
    ang = rot + np.arange(6) * math.pi / 3
    return np.vstack([[0.0, 0.0], np.stack([R_in * np.cos(ang), R_in * np.sin(ang)], 1)])


def _triangle(rho, rot=0.3):
    ang = rot + np.arange(3) * 2 * math.pi / 3
    return np.stack([rho * np.cos(ang), rho * np.sin(ang)], 1)


def test_closed_form_zero_energy(orc):
    """Eq. 5 vanishes on the optimal packings n = 2 (R = 2), 3 (R = 1 + 2/sqrt 3), 7 (R = 3)."""
    assert orc.energy_allpairs(np.array([[-1.0, 0.0], [1.0, 0.0]]), 2.0) == 0.0
    E3 = orc.energy_allpairs(_triangle(2 / math.sqrt(3)), 1 + 2 / math.sqrt(3))
    E7 = orc.energy_allpairs(_hexagon7(), 3.0)
    assert E3 <= 1e-28 and E7 <= 1e-28


@pytest.mark.parametrize("delta", [1e-3, 0.05])
def test_closed_form_compressed(orc, delta):
    """Symmetric stationary energies just below the optimal radii (derived from Eq. 5):
    n=2: 4 d^2/3 at a = 1 - d/3; n=3: 9 d^2/4 at rho = 2/sqrt3 - d/4; n=7: 4 d^2 at rho = 2 - d/3."""
    a = 1 - delta / 3
    E2 = orc.energy_allpairs(np.array([[-a, 0.0], [a, 0.0]]), 2.0 - delta)
    assert E2 == pytest.approx(4 * delta ** 2 / 3, rel=1e-12)
    E3 = orc.energy_allpairs(_triangle(2 / math.sqrt(3) - delta / 4), 1 + 2 / math.sqrt(3) - delta)
    assert E3 == pytest.approx(9 * delta ** 2 / 4, rel=1e-10)
    E7 = orc.energy_allpairs(_hexagon7(2 - delta / 3, 0.1), 3.0 - delta)
    assert E7 == pytest.approx(4 * delta ** 2, rel=1e-10)
    # and the gradient vanishes there (a stationary point)
    for xy, R in [(np.array([[-a, 0.0], [a, 0.0]]), 2 - delta),
                  (_hexagon7(2 - delta / 3, 0.1), 3 - delta)]:
        g = orc.grad_allpairs(xy, R)
        assert np.abs(g).max() < 1e-12


def test_hex_patch_energy(orc):
    """Hex patch with k rings, spacing s in [1.45, 2), far from the wall: E = (9k^2 + 3k)(2 - s)^2,
    interior gradient zero."""
    for k, s in [(4, 1.5), (12, 1.9)]:
        xy = synth.hex_patch(k, s)
        R = 1e3
        rp, col = orc.neighbors_cells(xy, R, 2.5)
        E, g, _ = orc.energy_grad_csr(xy, R, rp, col)
        assert E == pytest.approx((9 * k * k + 3 * k) * (2 - s) ** 2, rel=1e-12)
        r = np.hypot(xy[:, 0], xy[:, 1])
        interior = r < s * (k - 1) * 0.8
        assert np.abs(g[interior]).max() < 1e-11


def test_two_circles_gradient_analytic(orc):
    """n = 2 on the x axis: dE/dx_1 = -2 (2 - l) + 2 (x_1 + 1 - R) for x_1 = -x_2 = a."""
    a, R = 0.7, 1.5
    xy = np.array([[a, 0.0], [-a, 0.0]])
    g = orc.grad_allpairs(xy, R)
    want = -2 * (2 - 2 * a) + 2 * (a + 1 - R)
    assert g[0, 0] == pytest.approx(want, rel=1e-14)
    assert g[1, 0] == pytest.approx(-want, rel=1e-14)
    assert g[0, 1] == 0.0


def _away_from_kinks(xy, R, tol=1e-3):
    d = np.sqrt(((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(d, 10.0)
    r = np.hypot(xy[:, 0], xy[:, 1])
    return np.all(np.abs(d - 2.0) > tol) and np.all(np.abs(r - (R - 1.0)) > tol)


def test_gradient_finite_differences(orc):
    rng = np.random.default_rng(0)
    n, R = 40, synth.radius(40, 0.9)
    for trial in range(20):
        xy = orc.init_positions(n, R, seed=100 + trial)
        xy *= 1.05  # some boundary overlaps too
        if not _away_from_kinks(xy, R):
            continue
        g = orc.grad_allpairs(xy, R)
        h = 1e-6
        for _ in range(10):
            i, c = rng.integers(n), rng.integers(2)
            xp, xm = xy.copy(), xy.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd = (orc.energy_allpairs(xp, R) - orc.energy_allpairs(xm, R)) / (2 * h)
            assert abs(fd - g[i, c]) <= 1e-6 * max(1.0, abs(g[i, c]))


def test_pair_forces_sum_to_zero(orc):
    """Pair terms act equal and opposite (Newton's third law): with R large, sum_i g_i = 0."""
    n = 300
    xy = synth.random_layout(n, 12.0, seed=9)
    g = orc.grad_allpairs(xy, 1e6)
    assert np.abs(g.sum(0)).max() <= 1e-12 * np.abs(g).sum()


def test_csr_equals_allpairs(orc):
    for n, u in [(10, 0.7), (600, 0.84), (1500, 0.9)]:
        R = synth.radius(n, u)
        xy = orc.init_positions(n, R, seed=n)
        rp, col = orc.neighbors_cells(xy, R, 2.5)
        E, g, _ = orc.energy_grad_csr(xy, R, rp, col)
        assert E == pytest.approx(orc.energy_allpairs(xy, R), rel=1e-13)
        np.testing.assert_allclose(g, orc.grad_allpairs(xy, R), rtol=1e-12, atol=1e-12)


def test_rotation_and_permutation_invariance(orc):
    n, R = 500, synth.radius(500, 0.85)
    xy = orc.init_positions(n, R, seed=4)
    E = orc.energy_allpairs(xy, R)
    rot = np.stack([-xy[:, 1], xy[:, 0]], 1)  # exact 90 degree rotation
    assert orc.energy_allpairs(rot, R) == pytest.approx(E, rel=1e-15)
    p = np.random.default_rng(1).permutation(n)
    assert orc.energy_allpairs(xy[p], R) == pytest.approx(E, rel=1e-13)
    np.testing.assert_allclose(orc.grad_allpairs(xy[p], R), orc.grad_allpairs(xy, R)[p], rtol=1e-13,
                               atol=1e-13)


def test_batch_energy_identity(orc):
    """Eq. 7: E(x_p) = E(x) minus every term with no endpoint in B_p, and a move of x_p changes
    E(x_p) and E(x) by the same amount."""
    n, R, k = 700, synth.radius(700, 0.83), 5
    xy = orc.init_positions(n, R, seed=21)
    perm, bounds = orc.partition(xy, k)
    batch_of = np.zeros(n, dtype=np.int32)
    for p in range(k):
        batch_of[perm[bounds[p]:bounds[p + 1]]] = p
    rp, col = orc.neighbors_cells(xy, R, 2.5)
    E = orc.energy_allpairs(xy, R)
    for p in range(k):
        mb = perm[bounds[p]:bounds[p + 1]]
        Ep = orc.batch_energy(xy, R, rp, col, mb, batch_of, p)
        rest = np.setdiff1d(np.arange(n), mb)
        Erest = orc.energy_allpairs(xy[rest], R)  # pairs and walls with no endpoint in B_p
        assert Ep == pytest.approx(E - Erest, rel=1e-12, abs=1e-12)
        moved = xy.copy()
        moved[mb] += 0.01 * np.random.default_rng(p).standard_normal((len(mb), 2))
        dEp = orc.batch_energy(moved, R, rp, col, mb, batch_of, p) - Ep
        dE = orc.energy_allpairs(moved, R) - E
        assert dEp == pytest.approx(dE, rel=1e-9, abs=1e-12)


def test_degenerate_coincident_centres(orc):
    """Coincident centres: d = 2, the pair adds 4 to E and nothing to the gradient."""
    xy = np.array([[0.5, 0.5], [0.5, 0.5], [5.0, 0.0]])
    R = 100.0
    rp, col = orc.neighbors_brute(xy, 2.5)
    E, g, deg = orc.energy_grad_csr(xy, R, rp, col)
    assert E == 4.0 and deg == 2 and np.all(g == 0.0)


def test_max_overlap_matches_definition(orc):
    xy = np.array([[0.0, 0.0], [1.5, 0.0], [0.0, 3.0]])
    m, mp, mb = orc.max_overlap(xy, 3.5)
    assert mp == pytest.approx(0.5) and mb == pytest.approx(0.5) and m == pytest.approx(0.5)
    m, mp, mb = orc.max_overlap(np.array([[-1.0, 0.0], [1.0, 0.0]]), 2.0)
    assert m == 0.0

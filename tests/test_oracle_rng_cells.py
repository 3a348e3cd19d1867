"""Pins for the oracle's random init, cell binning and neighbor sets (CPU only).

Init: Sec. 5.1 (read as uniform in the disk of radius R-1).  Neighbor set:
Sec. 4.3, Gamma(i) = {j != i : l_ij < l_cut}.
"""
import math
import os

import numpy as np
import pytest

from paper_2303_02650_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    for ctr, key, out in _kat():
        assert list(orc.philox4x32_10(ctr, key)) == out


def test_init_in_disk_and_deterministic(orc):
    n, R = 5000, synth.radius(5000, 0.83)
    a = orc.init_positions(n, R, seed=7, inst=3)
    b = orc.init_positions(n, R, seed=7, inst=3)
    c = orc.init_positions(n, R, seed=7, inst=4)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    r = np.hypot(a[:, 0], a[:, 1])
    assert r.max() <= R - 1.0 + 1e-12


def test_init_uniform_in_disk_chi2(orc):
    """Uniform in a disk: r^2/(R-1)^2 ~ U(0,1) and the polar angle ~ U(0, 2 pi)."""
    from scipy import stats

    n, R = 400000, 40.0
    a = orc.init_positions(n, R, seed=11, inst=0)
    u = (a[:, 0] ** 2 + a[:, 1] ** 2) / (R - 1.0) ** 2
    th = np.arctan2(a[:, 1], a[:, 0])
    h1, _ = np.histogram(u, bins=40, range=(0.0, 1.0))
    h2, _ = np.histogram(th, bins=40, range=(-math.pi, math.pi))
    assert stats.chisquare(h1).pvalue > 1e-4
    assert stats.chisquare(h2).pvalue > 1e-4


def test_init_square_mode(orc):
    n, R = 20000, 30.0
    a = orc.init_positions(n, R, seed=3, inst=0, mode=1)
    assert np.abs(a).max() <= R
    assert np.abs(a).max() > R - 0.05  # fills the square, not the disk


@pytest.mark.parametrize("n,u,l_cut,prec32", [(2, 0.5, 2.5, False), (57, 0.8, 2.5, False),
                                              (800, 0.83, 2.5, False), (800, 0.83, 2.5, True),
                                              (500, 0.85, 4.0, False), (300, 0.3, 2.5, True)])
def test_cells_equal_brute_force(orc, n, u, l_cut, prec32):
    R = synth.radius(n, u)
    xy = orc.init_positions(n, R, seed=n, inst=1)
    if prec32:
        xy = xy.astype(np.float32).astype(np.float64)
    rb, cb = orc.neighbors_brute(xy, l_cut, prec32)
    rc, cc = orc.neighbors_cells(xy, R, l_cut, prec32)
    assert np.array_equal(rb, rc) and np.array_equal(cb, cc)
    # symmetric, no self loops, rows ascending
    pairs = {(i, int(j)) for i in range(n) for j in cc[rc[i]:rc[i + 1]]}
    assert all((j, i) in pairs for (i, j) in pairs)
    assert all(i != j for (i, j) in pairs)
    for i in range(n):
        row = cc[rc[i]:rc[i + 1]]
        assert np.all(np.diff(row) > 0)


def test_cells_points_outside_container(orc):
    """Clamped cells keep every neighbor pair (points far outside the container)."""
    n, R = 400, 10.0
    xy = synth.random_layout(n, R, seed=5, spread=2.5)
    xy[:50] *= 3.0
    rb, cb = orc.neighbors_brute(xy, 2.5)
    rc, cc = orc.neighbors_cells(xy, R, 2.5)
    assert np.array_equal(rb, rc) and np.array_equal(cb, cc)


def test_neighbors_hex_patch_bonds(orc):
    """A hexagonal patch with spacing s in [1.45, 2): Gamma holds exactly the lattice bonds
    (second neighbours are s sqrt(3) >= 2.51 > 2.5 apart)."""
    for rings, s in [(3, 1.45), (5, 1.7), (8, 1.99)]:
        xy = synth.hex_patch(rings, s)
        rp, col = orc.neighbors_brute(xy, 2.5)
        n = xy.shape[0]
        assert n == 3 * rings * (rings + 1) + 1
        assert len(col) // 2 == 9 * rings * rings + 3 * rings


def test_cell_keys_and_stable_sort(orc):
    n, R, l_cut = 3000, synth.radius(3000, 0.8), 2.5
    xy = orc.init_positions(n, R, seed=1)
    key = orc.cell_keys(xy, R, l_cut)
    inv, nc = orc.cell_grid(R, l_cut, n)
    assert nc == math.ceil(2 * R / (l_cut * (1 + 2 ** -20)))
    # a sparse instance: at most max(16, ceil(2 sqrt n)) cells per side, side >= l_cut
    inv2, nc2 = orc.cell_grid(1000.0, l_cut, 10)
    assert nc2 == 16 and 1.0 / inv2 >= l_cut
    # independent restatement of the cell index with numpy floor
    cx = np.clip(np.floor((xy[:, 0] + R) * inv), 0, nc - 1).astype(np.int64)
    cy = np.clip(np.floor((xy[:, 1] + R) * inv), 0, nc - 1).astype(np.int64)
    assert np.array_equal(key, (cy * nc + cx).astype(np.uint32))
    order, start = orc.cell_sort(key, nc * nc)
    assert np.array_equal(order, np.argsort(key, kind="stable"))
    assert start[-1] == n and np.array_equal(np.diff(start), np.bincount(key, minlength=nc * nc))

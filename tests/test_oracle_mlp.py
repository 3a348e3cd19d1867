"""Pins of the learned warm start's oracle (not in the paper; CPU only)."""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_2303_02650_gb300 import synth


def test_bf16_rounding_known_values():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1; 1 + 3*2^-8 -> 1 + 2^-6
    v = mlp.bf16(np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 3.0e38, 0.0]))
    assert v.tolist()[:4] == [1.0, 1.0, 1 + 2 ** -6, -2.5]
    assert v[5] == 0.0 and math.isfinite(v[4])


def test_gradient_finite_differences_unrounded():
    rng = np.random.default_rng(0)
    p = rng.normal(size=mlp.NPAR) * 0.1
    X = rng.normal(size=(40, 25)).astype(np.float32)
    T = rng.normal(size=(40, 2))
    L, g = mlp.loss_grad(p, X, T, round_bf16=False)
    h = 1e-6
    for i in rng.choice(mlp.NPAR, 30, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_grad(pp, X, T, False)[0] - mlp.loss_grad(pm, X, T, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_rounded_gradient_close_to_exact():
    rng = np.random.default_rng(1)
    p = rng.normal(size=mlp.NPAR) * 0.1
    X = rng.normal(size=(200, 25)).astype(np.float32)
    T = rng.normal(size=(200, 2))
    _, g0 = mlp.loss_grad(p, X, T, False)
    _, g1 = mlp.loss_grad(p, X, T, True)
    assert np.linalg.norm(g1 - g0) <= 0.05 * np.linalg.norm(g0)


def test_features_rotation_invariant_exactly():
    """A 90 degree rotation (x, y) -> (-y, x) is exact in binary32 and leaves every feature
    bit-identical (the frame turns with the circle)."""
    n, R = 300, synth.radius(300, 0.8)
    xy = (synth.random_layout(n, R - 1, seed=3) * 0.7).astype(np.float32)
    rot = np.stack([-xy[:, 1], xy[:, 0]], 1)
    assert np.array_equal(mlp.features(xy, R), mlp.features(rot, R))


def test_features_against_brute_force_distances():
    n, R = 200, synth.radius(200, 0.8)
    xy = (synth.random_layout(n, R - 1, seed=4) * 0.7).astype(np.float32)
    f = mlp.features(xy, R)
    for i in range(0, n, 17):
        d = np.hypot(*(xy.astype(np.float64) - xy[i]).T)
        d[i] = np.inf
        near = np.sort(d[d < 4.5])[:12]
        got = np.hypot(f[i, 0:24:2], f[i, 1:24:2])[: len(near)]
        np.testing.assert_allclose(got, near, rtol=1e-5, atol=1e-5)
        assert np.all(f[i, 2 * len(near):24] == 0)
        assert f[i, 24] == pytest.approx(min(R - np.hypot(*xy[i].astype(np.float64)) - 1, 4.5), abs=1e-4)

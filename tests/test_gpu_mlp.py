"""The learned warm start on the GPU against its oracle (marked gpu): features bit-exact, forward
and gradient of the tensor-core network within BF16-derived tolerances, training lowers the loss,
the warm start never raises an instance's energy, and the gain of a briefly trained network over
the plain descent is measured on fresh instances."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu, split

pytestmark = pytest.mark.gpu


def _ctx(pecc, n, R, **kw):
    c = pecc.Context(n, **kw)
    c.set_radius(R)
    return c


def test_features_bit_exact():
    torch, pecc = need_gpu()
    n = np.array([300, 57, 1000, 1], dtype=np.int32)
    R = np.array([synth.radius(int(v), 0.8) for v in n])
    with _ctx(pecc, n, R, precision=pecc.FP32) as c:
        c.init_random(4)
        f = c.features().cpu().numpy()
        xy = c.get_positions().cpu().numpy().astype(np.float32)
    for q, (fq, xq) in enumerate(zip(split(f, n), split(xy, n))):
        assert np.array_equal(fq, omlp.features(xq, float(R[q]))), q


def _data(seed, rows=3000):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(rows, 25)).astype(np.float32)
    T = rng.normal(size=(rows, 2)).astype(np.float32) * 0.1
    return X, T


def test_forward_matches_oracle():
    """Both sides round the same inputs to BF16; they differ by binary32 vs binary64 accumulation,
    which can flip a BF16 rounding of an activation (a 2^-8 relative step): outputs agree to
    2 % of their scale."""
    torch, pecc = need_gpu()
    m = pecc.MLP(seed=3)
    p = m.get_params().cpu().numpy()
    X, _ = _data(0)
    out = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = omlp.forward(p, X, True)
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= 0.02 * scale


def test_gradient_matches_oracle():
    torch, pecc = need_gpu()
    m = pecc.MLP(seed=5)
    p = m.get_params().cpu().numpy()
    X, T = _data(1, 5000)
    g, loss = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    L, gref = omlp.loss_grad(p, X, T, True)
    assert float(loss.item()) == pytest.approx(L, rel=2e-2)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - gref) <= 0.05 * np.linalg.norm(gref)
    for blk in [(omlp.OW1, omlp.OB1), (omlp.OW2, omlp.OB2), (omlp.OW3, omlp.OB3), (omlp.OW4, omlp.OB4)]:
        a, b = blk
        assert np.linalg.norm(g[a:b] - gref[a:b]) <= 0.08 * np.linalg.norm(gref[a:b]) + 1e-12


def test_training_lowers_loss():
    torch, pecc = need_gpu()
    m = pecc.MLP(seed=7)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(4096, 25)).astype(np.float32)
    T = np.stack([0.3 * X[:, 0] - 0.2 * X[:, 24], 0.1 * X[:, 1]], 1).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    l0 = float(m.train_step(Xd, Td, 1e-3).item())
    for _ in range(200):
        l = m.train_step(Xd, Td, 1e-3)
    assert float(l.item()) < 0.2 * l0


def test_warm_start_never_raises_energy():
    torch, pecc = need_gpu()
    n = np.array([400, 650, 300], dtype=np.int32)
    R = np.array([synth.radius(int(v), 0.8) for v in n])
    m = pecc.MLP(seed=11)
    with _ctx(pecc, n, R, precision=pecc.FP32_POLISH64) as c:
        c.init_random(8)
        c.rebuild_neighbors(eval=pecc.FP32)
        E0, _ = c.energy_grad(eval=pecc.FP32)
        acc = c.warm_start(m, 3).cpu().numpy()
        c.rebuild_neighbors(eval=pecc.FP32)
        E1, _ = c.energy_grad(eval=pecc.FP32)
    E0, E1 = E0.cpu().numpy(), E1.cpu().numpy()
    assert np.all(E1 <= E0 * (1 + 1e-6))
    assert np.all((acc >= 0) & (acc <= 3))


def test_learned_warm_start_gain():
    """Train briefly on descent samples, then compare with the plain descent on fresh instances
    (same seeds): the warm start keeps the success rate and reports the change in sweeps."""
    torch, pecc = need_gpu()
    from paper_2303_02650_gb300 import learned

    m = pecc.MLP(seed=1)
    train_set = synth.batch_manifest(96, seed=41)
    losses, rows = learned.train(m, train_set, rounds=4, T=50, steps=15, lr=2e-3)
    assert losses[-1] <= losses[0]
    test_set = synth.batch_manifest(128, seed=4242)
    res = learned.gain(m, test_set, seed=10**6 + 1, warm_rounds=2, precision=pecc.FP32_POLISH64)
    print("learned gain:", res)
    assert res["warm_feasible"] >= res["plain_feasible"] - 6

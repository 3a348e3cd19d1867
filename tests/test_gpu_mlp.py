"""The learned warm start on the GPU against its oracle (marked gpu).

Features are bit-exact.  The network runs on the fifth-generation tensor cores (tcgen05.mma, bf16
operands, binary32 accumulators in TMEM); its forward and backward passes are checked element by
element, one layer at a time: the oracle recomputes each layer in binary64 from the device's own
bf16 inputs of that layer (the traces of pecc_mlp_forward_trace / pecc_mlp_grad_trace), so that a
device element can differ from the oracle's only through the binary32 accumulation of that layer.
For a sum of K terms that accumulation is within K u |terms| (u = 2^-24, any order of additions).
A value that is then rounded to bf16 must lie between the bf16 roundings of (reference - bound)
and (reference + bound): rounding is monotone, so this admits exactly the neighbouring bf16 value
when the reference lies within the bound of a rounding boundary, and nothing else.  Adam is
compared with a binary32 restatement of its update.  Training lowers the loss, the warm start never
raises an instance's energy, and the gain of a trained network over the plain descent is measured.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu, split

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


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


def _data(seed, rows):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(rows, 25)).astype(np.float32)
    T = (rng.normal(size=(rows, 2)) * 0.1).astype(np.float32)
    return X, T


def _between(got, ref, bound, relu=True):
    """got (bf16 values) within the bf16 roundings of ref -/+ bound (after the ReLU when relu);
    returns the fraction of elements equal to the rounding of ref itself."""
    f = (lambda a: np.maximum(a, 0.0)) if relu else (lambda a: a)
    lo, hi, mid = omlp.bf16(f(ref - bound)), omlp.bf16(f(ref + bound)), omlp.bf16(f(ref))
    ok = (got >= lo) & (got <= hi)
    assert ok.all(), (np.argwhere(~ok)[:5], got[~ok][:5], ref[~ok][:5], bound[~ok][:5])
    return float(np.mean(got == mid))


def _check_forward(p, X, tr, out):
    """Every hidden layer from the previous layer's device activations, and the output layer."""
    h = omlp.bf16(X)
    for layer in range(3):
        z, mag = omlp.pre_activation(p, layer, h)
        K = 32 if layer == 0 else 128  # the tensor cores' K (the padded input width for layer 1)
        got = tr[:, layer, :].astype(np.float64)
        exact = _between(got, z, (K + 1) * U32 * mag)
        assert exact > 0.99, (layer, exact)
        h = got
    z, mag = omlp.pre_activation(p, 3, h)
    err = np.abs(out.astype(np.float64) - z)
    assert np.all(err <= 129 * U32 * mag), err.max()


def test_forward_matches_oracle_per_element():
    """1000 rows (seven tiles of 128 and a ragged tail): each layer within the binary32 accumulation
    bound of the oracle's binary64 layer, and the network's outputs against the full oracle forward
    (its own bf16 activations) within 2^-8 of each layer's scale, the size of one bf16 step."""
    torch, pecc = need_gpu()
    m = pecc.MLP(seed=3)
    p = m.get_params().cpu().numpy()
    X, _ = _data(0, 1000)
    out, tr = [t.cpu().numpy() for t in m.forward_trace(torch.from_numpy(X).cuda())]
    _check_forward(p, X, tr, out)
    plain = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.array_equal(plain, out)  # the traced and the plain forward are the same computation
    ref = omlp.forward(p, X, True)
    assert np.abs(out - ref).max() <= 2.0 ** -8 * np.abs(ref).max()


@pytest.mark.parametrize("rows", [100, 40000])
def test_gradient_matches_oracle_per_element(rows):
    """One tile (100 rows) and 40000 rows (more tiles than blocks, so every block accumulates its
    weight gradients in TMEM over two or more tiles): forward layers as above; dO as the device forms
    it; dZ3 = (dO W4) o [H3 > 0], dZ2, dZ1 each within the accumulation bound of the oracle's
    binary64 product of the device's dZ of the layer above; every weight and bias gradient, summed
    over the rows in binary32 (per block, then over blocks), within rows u |terms| of the binary64
    sum of the device's traced factors; the loss likewise."""
    torch, pecc = need_gpu()
    m = pecc.MLP(seed=5)
    p = m.get_params().cpu().numpy()
    X, T = _data(1, rows)
    g, loss, ft, bt = m.grad_trace(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    g, loss, ft, bt = g.cpu().numpy().astype(np.float64), float(loss.item()), ft.cpu().numpy(), bt.cpu().numpy()
    out = bt[:, 3, 2:4]
    _check_forward(p, X, ft, out)
    dO = bt[:, 3, 0:2].astype(np.float64)
    assert np.array_equal(dO, omlp.output_gradient(out, T, rows))
    H = [omlp.bf16(X)] + [ft[:, l, :].astype(np.float64) for l in range(3)]
    dZ = [None, bt[:, 2, :].astype(np.float64), bt[:, 1, :].astype(np.float64), bt[:, 0, :].astype(np.float64)]
    up = dO  # the gradient flowing into layer 3's output
    for layer in (3, 2, 1):  # dZ of hidden layer `layer` (1-based) from the layer above
        z, mag = omlp.back_pre(p, layer, up)
        K = 2 if layer == 3 else 128
        masked_ref = np.where(H[layer] > 0, z, 0.0)
        exact = _between(dZ[layer], masked_ref, np.where(H[layer] > 0, (K + 1) * U32 * mag, 0.0), relu=False)
        assert exact > 0.99, (layer, exact)
        up = dZ[layer]
    # weight and bias gradients from the device's factors
    grads = [(omlp.OW4, omlp.OB4, dO, H[3]), (omlp.OW3, omlp.OB3, dZ[3], H[2]), (omlp.OW2, omlp.OB2, dZ[2], H[1]),
             (omlp.OW1, omlp.OB1, dZ[1], H[0])]
    for ow, ob, d, h in grads:
        ref = d.T @ h
        bound = rows * U32 * (np.abs(d).T @ np.abs(h)) + 1e-30
        got = g[ow:ob].reshape(ref.shape)
        assert np.all(np.abs(got - ref) <= bound), (ow, np.abs(got - ref).max(), bound.max())
        bref, bb = d.sum(0), rows * U32 * np.abs(d).sum(0) + 1e-30
        gb = g[ob:ob + ref.shape[0]]
        assert np.all(np.abs(gb - bref) <= bb), (ob, np.abs(gb - bref).max())
    diff = out.astype(np.float64) - T
    L = np.sum(diff * diff) / rows
    assert abs(loss - L) <= 4 * rows * U32 * L + 1e-30


def test_adam_matches_binary32_restatement():
    """Two Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) against the update restated in binary32
    from the device's own gradients: every parameter within 4 ulp32 of the larger of the parameter
    and its update (the device may fuse the moment updates into FMAs, the restatement rounds each
    operation: about one ulp in each moment, and the ulps of the division, the square root and the
    final subtraction)."""
    torch, pecc = need_gpu()
    m = pecc.MLP(seed=9)
    X, T = _data(2, 3000)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    p = m.get_params().cpu().numpy().astype(np.float32)
    mm = np.zeros_like(p)
    vv = np.zeros_like(p)
    lr = np.float32(1e-3)
    for step in (1, 2):
        g = m.grad(Xd, Td)[0].cpu().numpy().astype(np.float32)
        m.train_step(Xd, Td, float(lr))
        b1c = np.float32(1.0) - np.float32(0.9) ** np.float32(step)
        b2c = np.float32(1.0) - np.float32(0.999) ** np.float32(step)
        mm = (np.float32(0.9) * mm + np.float32(0.1) * g).astype(np.float32)
        vv = (np.float32(0.999) * vv + np.float32(0.001) * g * g).astype(np.float32)
        upd = lr * (mm / b1c) / (np.sqrt(vv / b2c) + np.float32(1e-8))
        ref = (p - upd).astype(np.float32)
        got = m.get_params().cpu().numpy()
        tol = 4 * np.spacing(np.maximum(np.abs(ref), np.abs(upd))).astype(np.float64)
        assert np.all(np.abs(got.astype(np.float64) - ref) <= tol), np.abs(got - ref).max()
        p = got


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
    (same seeds).  The measured gain is reported; the warm start must not cost more than a few
    feasible results (its moves are checked, and the plain descent follows)."""
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

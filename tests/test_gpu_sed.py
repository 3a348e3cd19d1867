"""SED on the GPU (Sec. 5.2, Algorithm SED, Eq. 18) against the oracle, through the C ABI (marked
gpu).

Checked bit for bit:
- the perturbed candidates (Philox counters and correctly rounded binary64 on both sides);
- the candidate counts m = max(1, J(E(x)));
- the select decisions on given candidate energies, with the state they leave (x, x*, E).
Checked within tolerance:
- the start and one full iteration in binary64, with a few descent sweeps: the candidates'
  descents follow the oracle's GBO to 1e-9;
- on the exact radius of 7 circles, every instance reaches zero energy, as in the oracle.
"""
import numpy as np
import pytest

from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu, split

pytestmark = pytest.mark.gpu


def _layouts(orc, n, R, seed):
    return [orc.init_positions(int(v), float(r), seed, inst=q) for q, (v, r) in enumerate(zip(n, R))]


def test_prepare_draws_the_oracles_candidates(orc):
    torch, pecc = need_gpu()
    n = np.array([37, 300, 0, 129, 8], dtype=np.int32)
    R = np.array([synth.radius(max(int(v), 1), 0.8) for v in n])
    # energies chosen to give m = 1 (E > 0.1), 4, 9, 25 (J = 28 capped; e_feas 1e-30) and 1 (E > 1)
    Ex = np.array([0.5, 3e-4, 2e-9, 1e-28, 7.0])
    M = 25
    xs = _layouts(orc, n, R, 5)
    x = np.concatenate(xs)
    seed, it = 1234, 17
    with pecc.Sed(n, max_candidates=M, e_feas=1e-30, precision=0) as s:
        s.set_radius(R)
        s.set_state(torch.from_numpy(x), torch.from_numpy(Ex), seed, it)
        s.prepare()
        out = s.get(candidates=True)
        torch.cuda.synchronize()
        m = out["m"].cpu().numpy()
        cand = out["cand"].cpu().numpy()
    assert m.tolist() == [1, 4, 9, 25, 1]
    # an instance whose E(x*) is at or below e_feas takes no candidates
    with pecc.Sed(n[:1], max_candidates=M, precision=0) as s:
        s.set_radius(R[:1])
        s.set_state(torch.from_numpy(xs[0]), torch.tensor([1e-26]), seed, it)
        s.prepare()
        assert s.get()["m"].cpu().numpy().tolist() == [0]
    off = np.concatenate([[0], np.cumsum(n)])
    for q in range(n.size):
        for j in range(m[q]):
            lo = M * off[q] + j * n[q]
            ref = orc.sed_perturb(xs[q], seed, q, it, j)
            assert np.array_equal(cand[lo:lo + n[q]], ref), (q, j)


def test_prepare_shared_r_form(orc):
    torch, pecc = need_gpu()
    n = np.array([50], dtype=np.int32)
    R = np.array([synth.radius(50, 0.8)])
    x = _layouts(orc, n, R, 2)[0]
    with pecc.Sed(n, max_candidates=3, shared_r=1, precision=0) as s:
        s.set_radius(R)
        s.set_state(torch.from_numpy(x), torch.tensor([2e-3]), 9, 0)
        s.prepare()
        cand = s.get(candidates=True)["cand"].cpu().numpy()
    for j in range(3):
        assert np.array_equal(cand[j * 50:(j + 1) * 50], orc.sed_perturb(x, 9, 0, 0, j, shared=1))


def test_select_matches_the_oracle_on_given_energies(orc):
    """Both branches of Eq. 18 on random candidate energies: argmin when it improves on E(x),
    otherwise the softmax draw; x becomes the chosen candidate and x* follows only when E(x*)
    drops."""
    torch, pecc = need_gpu()
    rng = np.random.default_rng(8)
    num, M = 64, 6
    n = rng.integers(3, 40, size=num).astype(np.int32)
    R = np.array([synth.radius(int(v), 0.8) for v in n])
    x = np.concatenate(_layouts(orc, n, R, 3))
    Ex = 10.0 ** rng.uniform(-12, 0, size=num)
    seed, it = 77, 3
    with pecc.Sed(n, max_candidates=M, precision=0) as s:
        s.set_radius(R)
        s.set_state(torch.from_numpy(x), torch.from_numpy(Ex), seed, it)
        s.prepare()
        st = s.get(candidates=True)
        m = st["m"].cpu().numpy()
        cand = st["cand"].cpu().numpy()
        Ec = np.full(num * M, np.nan)
        for q in range(num):
            # half the instances see an improving candidate, half only worse ones
            scale = 0.5 if q % 2 == 0 else 2.0
            lo, hi = (0.0, 3.0) if q % 2 else (-3.0, 0.0)
            Ec[q * M:q * M + m[q]] = Ex[q] * scale * 10.0 ** rng.uniform(lo, hi, size=m[q])
        s.select(torch.from_numpy(Ec))
        out = s.get()
        torch.cuda.synchronize()
        sel = out["sel"].cpu().numpy()
        x1, xb1 = out["x"].cpu().numpy(), out["xbest"].cpu().numpy()
        Ex1, Eb1 = out["Ex"].cpu().numpy(), out["Eb"].cpu().numpy()
        iters = out["iters"].cpu().numpy()
    off = np.concatenate([[0], np.cumsum(n)])
    softmax = 0
    for q in range(num):
        e = Ec[q * M:q * M + m[q]]
        ref = orc.sed_select(e, Ex[q], seed, q, it)
        assert sel[q] == ref, q
        softmax += e.min() >= Ex[q] and m[q] > 1
        lo = M * off[q] + ref * n[q]
        assert np.array_equal(x1[off[q]:off[q + 1]], cand[lo:lo + n[q]])
        assert Ex1[q] == e[ref]
        if e[ref] < Ex[q]:
            assert Eb1[q] == e[ref] and np.array_equal(xb1[off[q]:off[q + 1]], x1[off[q]:off[q + 1]])
        else:
            assert Eb1[q] == Ex[q] and np.array_equal(xb1[off[q]:off[q + 1]], x[off[q]:off[q + 1]])
        assert iters[q] == 1
    assert softmax >= 10  # the softmax branch was exercised


def test_start_and_one_iteration_follow_the_oracle_fp64(orc):
    """Binary64, three descent sweeps: the start descends the oracle's random layout, and one
    iteration descends the oracle's candidates; positions to 1e-9 R and energies to 1e-9."""
    torch, pecc = need_gpu()
    n = np.array([60, 300, 140], dtype=np.int32)
    R = np.array([synth.radius(int(v), 0.82) for v in n])
    sweeps, seed, M = 3, 21, 4
    with pecc.Sed(n, max_candidates=M, precision=0, max_iter=sweeps) as s:
        s.set_radius(R)
        s.start(seed)
        st0 = s.get()
        x0 = st0["x"].cpu().numpy()
        E0 = st0["Ex"].cpu().numpy()
        s.prepare()
        s.descend()
        s.select()
        st1 = s.get()
        m = st1["m"].cpu().numpy()
        sel = st1["sel"].cpu().numpy()
        x1 = st1["x"].cpu().numpy()
        E1 = st1["Ex"].cpu().numpy()
    k = lambda v: 1 if v < 300 else (3 if v < 500 else 5)  # noqa: E731
    for q, (a, b) in enumerate(zip(split(x0, n), split(x1, n))):
        r = orc.gbo(orc.init_positions(int(n[q]), float(R[q]), seed, inst=q), float(R[q]), k=k(n[q]),
                    max_iter=sweeps, e_tol=1e-25)
        np.testing.assert_allclose(a, r.x, rtol=0, atol=1e-9 * R[q])
        assert E0[q] == pytest.approx(r.E, rel=1e-9)
        mq = min(M, max(1, orc.sed_J(E0[q])))
        assert m[q] == mq
        Ec, xc = [], []
        for j in range(mq):
            c = orc.gbo(orc.sed_perturb(a, seed, q, 0, j), float(R[q]), k=k(n[q]), max_iter=sweeps, e_tol=1e-25)
            Ec.append(c.E)
            xc.append(c.x)
        ref = orc.sed_select(np.array(Ec), E0[q], seed, q, 0)
        assert sel[q] == ref
        np.testing.assert_allclose(b, xc[ref], rtol=0, atol=1e-9 * R[q])
        assert E1[q] == pytest.approx(Ec[ref], rel=1e-9)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_reaches_zero_energy_at_the_exact_radius_of_seven(orc, prec):
    """R = 3 packs 7 circles exactly; every instance of the batch ends with E(x*) <= 1e-25 and a
    feasible layout, as the oracle's searches do."""
    torch, pecc = need_gpu()
    num = 16
    n = np.full(num, 7, dtype=np.int32)
    R = np.full(num, 3.0)
    # a binary32 context cannot resolve 1e-25: its search stops at its own energy floor
    e_feas = 1e-25 if prec != 1 else 1e-12
    with pecc.Sed(n, precision=prec, s_iter=30, e_feas=e_feas) as s:
        s.set_radius(R)
        s.start(5)
        ran, left = s.iterate(30)
        st = s.get()
        Eb = st["Eb"].cpu().numpy()
        status = st["status"].cpu().numpy()
        xb = st["xbest"].cpu().numpy()
    assert left == 0
    assert np.all(status == 0) and np.all(Eb <= e_feas)
    for q, part in enumerate(split(xb, n)):
        assert orc.max_overlap(part, 3.0)[0] <= (1e-9 if prec != 1 else 1e-5)
    r = orc.sed(7, 3.0, 5, inst=0, s_iter=30)
    assert r.status == "converged"


def test_search_lowers_jammed_energies_and_keeps_the_record():
    """Dense instances (u = 0.80, n = 30): E(x*) never rises, the record x* has energy E(x*),
    and exploring lowers it on some instances."""
    torch, pecc = need_gpu()
    num = 32
    n = np.full(num, 30, dtype=np.int32)
    R = np.full(num, np.sqrt(30 / 0.80))
    with pecc.Sed(n, precision=0, s_iter=12, max_candidates=8) as s:
        s.set_radius(R)
        s.start(2)
        E0 = s.get()["Eb"].cpu().numpy()
        ran, left = s.iterate(12)
        st = s.get()
        Eb = st["Eb"].cpu().numpy()
        iters = st["iters"].cpu().numpy()
        xb = st["xbest"]
    assert ran == 12
    assert np.all(Eb <= E0)
    assert np.sum(Eb < 0.5 * E0) >= 1
    assert np.all((iters == 12) | (Eb <= 1e-25))
    # the record's energy is its layout's (binary64 energy of the context's lists)
    with pecc.Context(n, precision=0) as c:
        c.set_radius(R)
        c.set_positions(xb)
        c.rebuild_neighbors(force=True, eval=0)
        E, _ = c.energy_grad(eval=0)
        E = E.cpu().numpy()
    np.testing.assert_allclose(E, Eb, rtol=1e-9, atol=1e-30)


def test_done_instances_are_skipped_and_arguments_checked():
    torch, pecc = need_gpu()
    n = np.array([7, 7], dtype=np.int32)
    R = np.array([3.0, 3.0])
    x = torch.zeros((14, 2), dtype=torch.float64)
    with pecc.Sed(n, precision=0, max_candidates=2) as s:
        s.set_radius(R)
        s.set_state(x, torch.tensor([0.0, 0.3]), 1, 0)  # instance 0 is done: E(x*) = 0
        ran, left = s.iterate(1)
        st = s.get()
        assert st["m"].cpu().numpy().tolist() == [0, 1]
        assert st["iters"].cpu().numpy().tolist() == [0, 1]
        assert st["status"].cpu().numpy()[0] == 0
    with pytest.raises(pecc.PeccError):
        pecc.Sed(np.array([16384], dtype=np.int32))
    with pytest.raises(pecc.PeccError):
        pecc.Sed(np.array([10], dtype=np.int32), max_candidates=0)

"""Stream semantics of the C ABI (marked gpu): which calls return while the context's stream is
still busy (stream-ordered, asynchronous) and which synchronise it, as include/pecc.h lists them
(pecc_phase_times waits for its own last event only, so it is not in either list).

A descent of 2048 instances keeps the stream busy for tens of milliseconds; each asynchronous
call must return before that work ends (the stream still reports pending work), each
synchronising call only after it (the stream reports idle the moment the call returns)."""
import numpy as np
import pytest

from paper_2303_02650_gb300 import synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _busy(c, s):
    c.init_random(3)
    c.descend()
    assert not s.query(), "the descent ended before the call under test: the check is void"


def test_asynchronous_and_synchronising_calls():
    torch, pecc = need_gpu()
    n, R = synth.batch_manifest(2048, seed=2303)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with pecc.Context(n, stream=s, precision=pecc.FP32_POLISH64) as c:
            c.set_radius(R)
            c.init_random(1)
            c.descend()  # first use: graph capture
            s.synchronize()
            xy = c.get_positions()
            R_dev = torch.as_tensor(R, dtype=torch.float64, device="cuda")
            asynchronous = {
                "pecc_init_random": lambda: c.init_random(5),
                "pecc_set_positions": lambda: c.set_positions(xy),
                "pecc_get_positions": c.get_positions,
                "pecc_descend": c.descend,
                "pecc_get_energy": c.get_energy,
                "pecc_get_counters": c.get_counters,
                "pecc_get_stats": c.get_stats,
                "pecc_rebuild_neighbors": lambda: c.rebuild_neighbors(force=True),
                "pecc_check_feasible": c.check_feasible,
                "pecc_set_radius": lambda: c.set_radius(R_dev),
            }
            for call in asynchronous.values():  # first use of every output size in the allocator's cache
                call()
            s.synchronize()
            for name, call in asynchronous.items():
                _busy(c, s)
                call()
                assert not s.query(), f"{name} waited for the stream"
            s.synchronize()
            c.rebuild_neighbors(force=True)
            c.energy_grad()  # the standalone lists are current: energy + gradient is asynchronous too
            synchronising = {
                "pecc_neighbor_count": c.neighbor_count,
                "pecc_solve_host": lambda: c.solve_host(R, 9, want_xy=False),
            }
            for name, call in synchronising.items():
                _busy(c, s)
                if name == "pecc_neighbor_count":
                    c.rebuild_neighbors(force=True)
                call()
                assert s.query(), f"{name} returned with work pending"
        s.synchronize()


def test_bad_radius_marks_its_instance(orc):
    """A radius that is not finite and > 0 is not read on the host: its instance's descent ends
    with status 5 (non-finite) and its feasibility check gives NaN, the other instances are
    unaffected and match the oracle's check."""
    torch, pecc = need_gpu()
    n = np.array([300, 200, 120], dtype=np.int32)
    R = np.array([synth.radius(300, 0.8), float("nan"), synth.radius(120, 0.8)])
    with pecc.Context(n, precision=pecc.FP32_POLISH64) as c:
        c.set_radius(np.where(np.isnan(R), -1.0, R))
        c.set_radius(R)
        c.init_random(3)
        iters, status = c.descend()
        feas, mo = c.check_feasible()
        xy = c.get_positions().cpu().numpy()
    status, feas, mo = status.cpu().numpy(), feas.cpu().numpy(), mo.cpu().numpy()
    assert status[1] == 5 and np.isnan(mo[1]) and feas[1] == 0
    off = np.concatenate([[0], np.cumsum(n)])
    for q in (0, 2):
        assert status[q] in (0, 1, 2, 3)
        assert mo[q] == orc.max_overlap(xy[off[q]:off[q + 1]], float(R[q]))[0]

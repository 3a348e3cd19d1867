"""The bench's per-workload defaults (CPU): the batch workloads run at k = 2 with their tuned
settings, a --cfg field replaces the default of that field only, and every default names a
pecc_config field with a value of the field's type."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

pecc = pytest.importorskip("paper_2303_02650_gb300.pecc")


def _args(workload, k=-1, cfg=()):
    return bench.apply_workload_defaults(argparse.Namespace(workload=workload, k=k, cfg=list(cfg)))


def test_batch_workload_defaults():
    a = _args("c3")
    assert a.k == 2
    f = bench.cfg_fields(a.cfg)
    assert f == {"step_max": 0.3, "polish_gate": 1e-5, "stall_window": 5, "polish_stall_window": 50, "lbfgs_m": 5}
    assert _args("c3", k=0).k == 0  # the paper's k by n on request
    assert _args("c5").k == 0 and _args("c5").cfg == []


def test_cfg_overrides_only_its_field():
    f = bench.cfg_fields(_args("c3", cfg=["lbfgs_m=10"]).cfg)
    assert f["lbfgs_m"] == 10 and f["step_max"] == 0.3


def test_defaults_name_config_fields():
    names = {n for n, _ in pecc.Config._fields_}
    for wl, cfg in bench.CFG_DEFAULT.items():
        for key, val in bench.cfg_fields(cfg).items():
            assert key in names, (wl, key)
            ctype = dict(pecc.Config._fields_)[key]
            assert isinstance(val, float) == (ctype.__name__ == "c_double"), (wl, key)


def _reference_line(*extra):
    import json
    import subprocess

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", *extra], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("extra", [(), ("--workload", "ksweep")])
def test_reference_arm_line(extra):
    """The reference arm (the FP64 oracle on the host cores) prints one JSON line with the bench's
    keys: its own cpu_baseline and an e2e with no host-device copies, both carrying the line's value."""
    r = _reference_line(*extra)
    assert r["impl"] == "reference" and r["value"] > 0 and r["steps"] == 1 and r["warmup"] == 3
    for key in ("metric", "unit", "n_gpus", "ms_per_step", "higher_is_better", "scaling", "dtype", "config"):
        assert key in r, key
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == r["value"]
    assert cb["unit"] == r["unit"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_byte_model_charges_the_configured_memory():
    """The roofline's byte model charges the two-loop recursion 4 m vectors per circle and sweep with
    the m the context runs with: 220 B per circle-sweep in FP32 at the batch workloads' m = 5 (380 B
    at the library's m = 10), and no call of the model passes a fixed m."""
    import re

    assert bench.per_sweep_bytes(5, 8, 8) == 44 + 4 * 5 * 8 + 16 == 220
    assert bench.per_sweep_bytes(10, 8, 8) == 380
    for wl, cfg in bench.CFG_DEFAULT.items():
        m = bench.cfg_fields(cfg).get("lbfgs_m", 10)
        assert bench.per_sweep_bytes(m, 8, 8) == 44 + 32 * m + 16, wl
    src = open(os.path.join(ROOT, "bench.py")).read()
    calls = re.findall(r"algorithmic_bytes_descent\(([^()]*(?:\([^()]*\)[^()]*)*)\)", src)
    assert len(calls) >= 6
    for c in calls:
        args = [a.strip() for a in c.split(",")]
        if args[0].startswith("n, k, iters"):  # the definition
            continue
        assert not re.fullmatch(r"\d+", args[4]), c  # m is the context's, never a literal


def test_oracle_runs_the_workload_settings():
    """The CPU baseline and the reference arm run the oracle with the GPU arm's k, m and step cap."""
    assert bench.oracle_settings(_args("c3")) == {"k": 2, "m": 5, "step_max": 0.3}
    assert bench.oracle_settings(_args("c3", cfg=["lbfgs_m=10"])) == {"k": 2, "m": 10, "step_max": 0.3}
    assert bench.oracle_settings(_args("c1")) == {"k": 0}


def test_paper_runtimes_match_the_golden_table():
    """The paper's per-descent times quoted beside the bench line are the printed table's values."""
    path = os.path.join(ROOT, "tests", "golden", "gbo_batch_numbers.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    table = {int(r[0]): (float(r[1]), int(r[2]), float(r[3])) for r in rows}
    assert bench.PAPER_DESCENT_S == table

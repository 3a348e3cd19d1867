"""The C-ABI library builds for sm_103a, loads without a GPU and exports every call that
include/pecc.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pecc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pecc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2303_02650_gb300 import build

    return build.build()


def test_header_declares_boundary_calls():
    names = _declared()
    for want in ["pecc_create", "pecc_set_radius", "pecc_descend", "pecc_energy_grad", "pecc_rebuild_neighbors",
                 "pecc_check_feasible"]:
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2303_02650_gb300 import pecc

    assert set(_declared()) <= set(pecc._EXPORTS)


def test_config_defaults_without_gpu(libpath):
    from paper_2303_02650_gb300 import pecc

    c = pecc.default_config()
    assert c.l_cut == 2.5 and c.rebuild_disp == 0.25 and c.lbfgs_m == 10 and c.max_iter == 2000
    assert c.e_tol == 1e-20 and c.feas_tol == 1e-9 and c.precision == pecc.FP32_POLISH64


def test_create_rejects_bad_arguments_without_gpu(libpath):
    """Argument checks happen before any device call."""
    from paper_2303_02650_gb300 import pecc

    L = pecc.load()
    n = (ctypes.c_int32 * 1)(10)
    for field, bad in [("l_cut", 2.0), ("lbfgs_m", 11), ("k_batches", 65), ("partition", 4), ("step_max", 0.6)]:
        c = pecc.default_config(**{field: bad})
        c.num_instances = 1
        c.n = ctypes.cast(n, ctypes.POINTER(ctypes.c_int32))
        h = ctypes.c_void_p()
        assert L.pecc_create(ctypes.byref(c), None, ctypes.byref(h)) == 1, field
        assert not h.value


def test_barrier_selftest_rejects_bad_arguments_without_gpu(libpath):
    from paper_2303_02650_gb300 import pecc

    L = pecc.load()
    f, w = ctypes.c_int32(), ctypes.c_int64()
    for t in (0, -5, 20_000_000_000):
        assert L.pecc_selftest_grid_barrier(t, ctypes.byref(f), ctypes.byref(w)) == 1

"""Thin ctypes binding of the C ABI in include/pecc.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libpecc.so``; PyTorch only
provides device memory and the stream.  Importing this module loads the
library and raises if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

FP64, FP32, FP32_POLISH64 = 0, 1, 2
PART_SECTOR, PART_ANNULUS, PART_FENCE, PART_RANDOM = 0, 1, 2, 3
INIT_DISK, INIT_SQUARE = 0, 1
STATUS = {0: "converged", 1: "stationary", 2: "stalled", 3: "max_iter", 4: "nbr_overflow", 5: "nonfinite",
          6: "timeout"}
ERRORS = {1: "PECC_ERR_ARG", 2: "PECC_ERR_CUDA", 3: "PECC_ERR_OOM", 4: "PECC_ERR_NBR_OVERFLOW",
          5: "PECC_ERR_NONFINITE", 6: "PECC_ERR_TIMEOUT"}


class PeccError(RuntimeError):
    pass


class Config(C.Structure):
    _fields_ = [("num_instances", C.c_int32), ("n", C.POINTER(C.c_int32)), ("precision", C.c_int32),
                ("l_cut", C.c_double), ("rebuild_disp", C.c_double), ("step_max", C.c_double),
                ("lbfgs_m", C.c_int32), ("max_iter", C.c_int32), ("polish_max_iter", C.c_int32),
                ("k_batches", C.c_int32), ("partition", C.c_int32), ("max_trials", C.c_int32),
                ("anm", C.c_int32), ("init_mode", C.c_int32), ("e_tol", C.c_double), ("gsum_tol", C.c_double),
                ("c1", C.c_double), ("curv_eps", C.c_double), ("polish_gate", C.c_double),
                ("feas_tol", C.c_double), ("nbr_capacity", C.c_double), ("time_budget_ns", C.c_int64),
                ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32), ("stall_rel", C.c_double),
                ("stall_window", C.c_int32), ("polish_k", C.c_int32),
                ("smem_per_block", C.c_int32), ("polish_stall_rel", C.c_double),
                ("polish_stall_window", C.c_int32), ("fuse_phases", C.c_int32), ("partition_seed", C.c_uint64),
                ("qn_dense", C.c_int32), ("list_outer", C.c_double)]


class SedConfig(C.Structure):
    _fields_ = [("max_candidates", C.c_int32), ("s_iter", C.c_int32), ("e_feas", C.c_double), ("amp", C.c_double),
                ("shared_r", C.c_int32), ("check_every", C.c_int32)]


_lib = None
_EXPORTS = ["pecc_config_default", "pecc_create", "pecc_destroy", "pecc_set_radius", "pecc_set_positions",
            "pecc_init_random", "pecc_get_positions", "pecc_rebuild_neighbors", "pecc_rebuild_neighbors_ex",
            "pecc_neighbor_count", "pecc_export_neighbors", "pecc_export_cells", "pecc_energy_grad",
            "pecc_energy_grad_ex", "pecc_descend", "pecc_get_energy", "pecc_check_feasible", "pecc_solve_host",
            "pecc_get_counters", "pecc_get_launch", "pecc_last_error", "pecc_get_stats", "pecc_phase_times",
            "pecc_check_feasible_noalloc", "pecc_mlp_num_params", "pecc_mlp_create", "pecc_mlp_destroy",
            "pecc_mlp_get_params", "pecc_mlp_set_params", "pecc_mlp_forward", "pecc_mlp_grad", "pecc_mlp_train_step",
            "pecc_features", "pecc_targets", "pecc_warm_start", "pecc_autotune", "pecc_selftest_grid_barrier",
            "pecc_adjust_container", "pecc_sed_config_default", "pecc_sed_create", "pecc_sed_destroy",
            "pecc_sed_last_error", "pecc_sed_set_radius", "pecc_sed_start", "pecc_sed_set_state", "pecc_sed_iterate",
            "pecc_sed_prepare", "pecc_sed_descend", "pecc_sed_select", "pecc_sed_get", "pecc_sed_context",
            "pecc_frame_run", "pecc_set_list_dump", "pecc_warm_start_ex", "pecc_mlp_forward_trace",
            "pecc_mlp_grad_trace"]
NOALLOC_MAX_N = 4096
ENERGY_STAGE_BYTES = 96 * 1024  # PECC_ENERGY_STAGE_BYTES


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpecc.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise PeccError(f"CUDA library not built: {path}")
        _build.build()
    L = C.CDLL(path)
    vp, i32p, i64p, dp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double)
    st = C.c_int
    sig = {
        "pecc_config_default": (None, [C.POINTER(Config)]),
        "pecc_create": (st, [C.POINTER(Config), vp, C.POINTER(vp)]),
        "pecc_destroy": (st, [vp]),
        "pecc_set_radius": (st, [vp, vp]),
        "pecc_set_positions": (st, [vp, vp]),
        "pecc_init_random": (st, [vp, C.c_uint64]),
        "pecc_get_positions": (st, [vp, vp]),
        "pecc_rebuild_neighbors": (st, [vp, C.c_int32, vp]),
        "pecc_rebuild_neighbors_ex": (st, [vp, C.c_int32, C.c_int32, vp]),
        "pecc_neighbor_count": (st, [vp, i64p]),
        "pecc_export_neighbors": (st, [vp, vp, vp, C.c_int64]),
        "pecc_export_cells": (st, [vp, vp, vp]),
        "pecc_energy_grad": (st, [vp, vp, vp]),
        "pecc_energy_grad_ex": (st, [vp, C.c_int32, vp, vp]),
        "pecc_descend": (st, [vp, vp, vp]),
        "pecc_get_energy": (st, [vp, vp]),
        "pecc_check_feasible": (st, [vp, C.c_double, vp, vp]),
        "pecc_solve_host": (st, [vp, vp, C.c_uint64, vp, vp, vp, vp, vp]),
        "pecc_get_counters": (st, [vp, vp, vp, vp]),
        "pecc_get_launch": (st, [vp, i32p, i32p, i32p]),
        "pecc_last_error": (C.c_char_p, [vp]),
        "pecc_get_stats": (st, [vp, vp]),
        "pecc_phase_times": (st, [vp, C.POINTER(C.c_float)]),
        "pecc_check_feasible_noalloc": (st, [vp, C.c_int32, C.c_double, C.c_double, C.c_double, vp, vp, vp]),
        "pecc_selftest_grid_barrier": (st, [C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
        "pecc_adjust_container": (st, [vp, vp, C.c_double, C.c_int32, vp, vp, vp]),
        "pecc_mlp_num_params": (C.c_int32, []),
        "pecc_mlp_create": (st, [C.c_uint64, vp, C.POINTER(vp)]),
        "pecc_mlp_destroy": (st, [vp]),
        "pecc_mlp_get_params": (st, [vp, vp]),
        "pecc_mlp_set_params": (st, [vp, vp]),
        "pecc_mlp_forward": (st, [vp, vp, C.c_int64, vp]),
        "pecc_mlp_grad": (st, [vp, vp, vp, C.c_int64, vp, vp]),
        "pecc_mlp_train_step": (st, [vp, vp, vp, C.c_int64, C.c_float, vp]),
        "pecc_features": (st, [vp, vp, vp]),
        "pecc_targets": (st, [vp, vp, vp]),
        "pecc_warm_start": (st, [vp, vp, C.c_int32, vp]),
        "pecc_autotune": (st, [vp, C.c_int32, C.c_uint64, i32p, i32p]),
        "pecc_sed_config_default": (None, [C.POINTER(SedConfig)]),
        "pecc_sed_create": (st, [C.POINTER(Config), C.POINTER(SedConfig), vp, C.POINTER(vp)]),
        "pecc_sed_destroy": (st, [vp]),
        "pecc_sed_last_error": (C.c_char_p, [vp]),
        "pecc_sed_set_radius": (st, [vp, vp]),
        "pecc_sed_start": (st, [vp, C.c_uint64]),
        "pecc_sed_set_state": (st, [vp, vp, vp, C.c_uint64, C.c_int32]),
        "pecc_sed_iterate": (st, [vp, C.c_int32, i32p, i32p]),
        "pecc_sed_prepare": (st, [vp]),
        "pecc_sed_descend": (st, [vp]),
        "pecc_sed_select": (st, [vp, vp]),
        "pecc_sed_get": (st, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "pecc_sed_context": (vp, [vp]),
        "pecc_frame_run": (st, [vp, vp, vp, C.c_uint64, C.c_int32, C.c_int32, C.c_double, C.c_int32, vp, vp, vp,
                                vp]),
        "pecc_set_list_dump": (st, [vp, C.c_int32, vp, vp, vp]),
        "pecc_warm_start_ex": (st, [vp, vp, C.c_int32, C.c_double, vp]),
        "pecc_mlp_forward_trace": (st, [vp, vp, C.c_int64, vp, vp]),
        "pecc_mlp_grad_trace": (st, [vp, vp, vp, C.c_int64, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def default_config(**kw) -> Config:
    c = Config()
    load().pecc_config_default(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k) or k in ("n", "num_instances"):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def selftest_grid_barrier(timeout_ns=50_000_000):
    """pecc_selftest_grid_barrier: (failed, waited_ns) of a grid barrier that nothing releases."""
    L = load()
    f, w = C.c_int32(), C.c_int64()
    rc = L.pecc_selftest_grid_barrier(int(timeout_ns), C.byref(f), C.byref(w))
    if rc != 0:
        raise PeccError(f"pecc_selftest_grid_barrier: {ERRORS.get(rc, rc)}: {L.pecc_last_error(None).decode()}")
    return f.value, w.value


def check_feasible_noalloc(xy, R, l_cut=2.5, tol=1e-9, stream=None):
    """pecc_check_feasible_noalloc on one instance (device tensor xy [n, 2] float64): returns
    (feasible uint8[1], max_overlap float64[1]) device tensors; allocates no device scratch."""
    L = load()
    n = int(xy.shape[0]) if xy is not None else 0
    dev = xy.device if xy is not None else torch.device("cuda")
    feas = torch.empty(1, dtype=torch.uint8, device=dev)
    mo = torch.empty(1, dtype=torch.float64, device=dev)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    rc = L.pecc_check_feasible_noalloc(_ptr(xy) if n else None, n, float(R), float(l_cut), float(tol), _ptr(feas),
                                       _ptr(mo), C.c_void_p(s))
    if rc != 0:
        raise PeccError(f"pecc_check_feasible_noalloc: {ERRORS.get(rc, rc)}: {L.pecc_last_error(None).decode()}")
    return feas, mo


class MLP:
    """The learned warm start's network (pecc_mlp_*): FP32 master parameters, BF16 tensor-core copies."""

    def __init__(self, seed=0, stream=None):
        self._L = load()
        stream = stream or torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        rc = self._L.pecc_mlp_create(C.c_uint64(seed), C.c_void_p(stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise PeccError(f"pecc_mlp_create: {ERRORS.get(rc, rc)}: {self._L.pecc_last_error(None).decode()}")
        self.h = h
        self.num_params = int(self._L.pecc_mlp_num_params())

    def _check(self, rc, what):
        if rc != 0:
            raise PeccError(f"{what}: {ERRORS.get(rc, rc)}: {self._L.pecc_last_error(None).decode()}")

    def close(self):
        if getattr(self, "h", None):
            self._L.pecc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        self._check(self._L.pecc_mlp_get_params(self.h, _ptr(p)), "pecc_mlp_get_params")
        return p

    def set_params(self, p):
        p = torch.as_tensor(p, dtype=torch.float32, device="cuda").contiguous()
        self._check(self._L.pecc_mlp_set_params(self.h, _ptr(p)), "pecc_mlp_set_params")

    def forward(self, feat):
        feat = feat.contiguous()
        out = torch.empty((feat.shape[0], 2), dtype=torch.float32, device=feat.device)
        self._check(self._L.pecc_mlp_forward(self.h, _ptr(feat), feat.shape[0], _ptr(out)), "pecc_mlp_forward")
        return out

    def grad(self, feat, target):
        g = torch.empty(self.num_params, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        self._check(self._L.pecc_mlp_grad(self.h, _ptr(feat.contiguous()), _ptr(target.contiguous()), feat.shape[0],
                                          _ptr(g), _ptr(loss)), "pecc_mlp_grad")
        return g, loss

    def forward_trace(self, feat):
        """pecc_mlp_forward_trace: (out [rows, 2], trace [rows, 3, 128] of the bf16 hidden activations)."""
        feat = feat.contiguous()
        out = torch.empty((feat.shape[0], 2), dtype=torch.float32, device=feat.device)
        tr = torch.empty((feat.shape[0], 3, 128), dtype=torch.float32, device=feat.device)
        self._check(self._L.pecc_mlp_forward_trace(self.h, _ptr(feat), feat.shape[0], _ptr(out), _ptr(tr)),
                    "pecc_mlp_forward_trace")
        return out, tr

    def grad_trace(self, feat, target):
        """pecc_mlp_grad_trace: (grad, loss, forward trace [rows, 3, 128], backward trace [rows, 4, 128]:
        dZ3, dZ2, dZ1, then dO (2) and the outputs (2))."""
        g = torch.empty(self.num_params, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        ft = torch.empty((feat.shape[0], 3, 128), dtype=torch.float32, device=feat.device)
        bt = torch.empty((feat.shape[0], 4, 128), dtype=torch.float32, device=feat.device)
        self._check(self._L.pecc_mlp_grad_trace(self.h, _ptr(feat.contiguous()), _ptr(target.contiguous()),
                                                feat.shape[0], _ptr(g), _ptr(loss), _ptr(ft), _ptr(bt)),
                    "pecc_mlp_grad_trace")
        return g, loss, ft, bt

    def train_step(self, feat, target, lr):
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        self._check(self._L.pecc_mlp_train_step(self.h, _ptr(feat), _ptr(target), feat.shape[0], C.c_float(lr),
                                                _ptr(loss)), "pecc_mlp_train_step")
        return loss


class Context:
    """One pecc_ctx: independent instances of sizes n[], container radii, positions.

    Device arguments are torch CUDA tensors; host arguments of solve_host are numpy arrays.
    The calls are enqueued on the context's stream, while the tensors the methods allocate (their
    outputs, and device copies of host inputs) come from torch's caching allocator on the stream
    current at the call.  With the default (the current stream at creation) the two are the same
    and memory reuse is stream-ordered.  A caller that passes another stream makes its calls under
    `torch.cuda.stream(ctx.stream)`, or keeps those tensors alive until that stream has run.
    """

    def __init__(self, n, stream=None, **cfg):
        import numpy as np

        self._L = load()
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        self.num = int(self.n.shape[0])
        self.total = int(self.n.sum())
        self.cfg = default_config(**cfg)
        self.cfg.num_instances = self.num
        self.cfg.n = self.n.ctypes.data_as(C.POINTER(C.c_int32))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        rc = self._L.pecc_create(C.byref(self.cfg), C.c_void_p(stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise PeccError(f"pecc_create: {ERRORS.get(rc, rc)}: {self._L.pecc_last_error(None).decode()}")
        self.h = h
        self.precision = int(self.cfg.precision)
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def _check(self, rc, what):
        if rc != 0:
            raise PeccError(f"{what}: {ERRORS.get(rc, rc)}: {self._L.pecc_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            self._L.pecc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --------------------------------------------------------------- calls
    def set_radius(self, R):
        R = torch.as_tensor(R, dtype=torch.float64, device=self.dev).contiguous()
        self._check(self._L.pecc_set_radius(self.h, _ptr(R)), "pecc_set_radius")

    def set_positions(self, xy):
        xy = torch.as_tensor(xy, dtype=torch.float64, device=self.dev).contiguous()
        assert xy.numel() == 2 * self.total
        self._check(self._L.pecc_set_positions(self.h, _ptr(xy)), "pecc_set_positions")

    def init_random(self, seed: int):
        self._check(self._L.pecc_init_random(self.h, C.c_uint64(seed)), "pecc_init_random")

    def get_positions(self):
        out = torch.empty((self.total, 2), dtype=torch.float64, device=self.dev)
        self._check(self._L.pecc_get_positions(self.h, _ptr(out)), "pecc_get_positions")
        return out

    def rebuild_neighbors(self, force=True, eval=None):
        rebuilt = torch.zeros(self.num, dtype=torch.int32, device=self.dev)
        if eval is None:
            rc = self._L.pecc_rebuild_neighbors(self.h, int(force), _ptr(rebuilt))
        else:
            rc = self._L.pecc_rebuild_neighbors_ex(self.h, int(eval), int(force), _ptr(rebuilt))
        self._check(rc, "pecc_rebuild_neighbors")
        return rebuilt

    def neighbor_count(self) -> int:
        v = C.c_int64()
        self._check(self._L.pecc_neighbor_count(self.h, C.byref(v)), "pecc_neighbor_count")
        return v.value

    def export_neighbors(self):
        nnz = self.neighbor_count()
        rp = torch.empty(self.total + 1, dtype=torch.int32, device=self.dev)
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device=self.dev)
        self._check(self._L.pecc_export_neighbors(self.h, _ptr(rp), _ptr(col), C.c_int64(col.numel())),
                    "pecc_export_neighbors")
        return rp, col[:nnz]

    def export_cells(self):
        key = torch.empty(self.total, dtype=torch.int32, device=self.dev)
        order = torch.empty(self.total, dtype=torch.int32, device=self.dev)
        self._check(self._L.pecc_export_cells(self.h, _ptr(key), _ptr(order)), "pecc_export_cells")
        return key, order

    def energy_grad(self, eval=None, out=None):
        """(E, g); out = (E, g) preallocated with the right dtypes reuses those tensors."""
        ev = (FP64 if self.precision == FP64 else FP32) if eval is None else eval
        if out is None:
            E = torch.empty(self.num, dtype=torch.float64, device=self.dev)
            gdt = torch.float64 if ev == FP64 else torch.float32
            g = torch.empty((self.total, 2), dtype=gdt, device=self.dev)
        else:
            E, g = out
        rc = self._L.pecc_energy_grad(self.h, _ptr(E), _ptr(g)) if eval is None else \
            self._L.pecc_energy_grad_ex(self.h, int(eval), _ptr(E), _ptr(g))
        self._check(rc, "pecc_energy_grad")
        return E, g

    def descend(self):
        iters = torch.empty(self.num, dtype=torch.int32, device=self.dev)
        status = torch.empty(self.num, dtype=torch.int32, device=self.dev)
        self._check(self._L.pecc_descend(self.h, _ptr(iters), _ptr(status)), "pecc_descend")
        return iters, status

    def get_energy(self):
        E = torch.empty(self.num, dtype=torch.float64, device=self.dev)
        self._check(self._L.pecc_get_energy(self.h, _ptr(E)), "pecc_get_energy")
        return E

    def set_list_dump(self, stride=32):
        """pecc_set_list_dump: the following descents write the lists in force at the end of their
        first phase; returns the device tensors (cnt int32[total], col int32[total, stride], xb
        float64[total, 2]) they write.  stride=None turns the hook off."""
        if stride is None:
            self._check(self._L.pecc_set_list_dump(self.h, 0, None, None, None), "pecc_set_list_dump")
            self._dump = None
            return None
        cnt = torch.full((self.total,), -2, dtype=torch.int32, device=self.dev)
        col = torch.zeros((self.total, int(stride)), dtype=torch.int32, device=self.dev)
        xb = torch.zeros((self.total, 2), dtype=torch.float64, device=self.dev)
        self._check(self._L.pecc_set_list_dump(self.h, int(stride), _ptr(cnt), _ptr(col), _ptr(xb)),
                    "pecc_set_list_dump")
        self._dump = (cnt, col, xb)  # kept alive while the hook is set
        return self._dump

    def get_counters(self):
        b = torch.empty(self.num, dtype=torch.int32, device=self.dev)
        c = torch.empty_like(b)
        t = torch.empty_like(b)
        self._check(self._L.pecc_get_counters(self.h, _ptr(b), _ptr(c), _ptr(t)), "pecc_get_counters")
        return b, c, t

    def get_stats(self):
        """int32 [num, 10]: iters, status, builds, changes, trials, resets, stalls, polished,
        first-phase sweeps, first-phase trials."""
        st = torch.empty((self.num, 10), dtype=torch.int32, device=self.dev)
        self._check(self._L.pecc_get_stats(self.h, _ptr(st)), "pecc_get_stats")
        return st

    def phase_times(self):
        """Device ms of the last descent: (first phase kernel, polish kernel, whole descent)."""
        ms = (C.c_float * 3)()
        self._check(self._L.pecc_phase_times(self.h, ms), "pecc_phase_times")
        return float(ms[0]), float(ms[1]), float(ms[2])

    def check_feasible(self, tol=None):
        tol = float(self.cfg.feas_tol if tol is None else tol)
        feas = torch.empty(self.num, dtype=torch.uint8, device=self.dev)
        mo = torch.empty(self.num, dtype=torch.float64, device=self.dev)
        self._check(self._L.pecc_check_feasible(self.h, C.c_double(tol), _ptr(feas), _ptr(mo)),
                    "pecc_check_feasible")
        return feas, mo

    def features(self):
        f = torch.empty((self.total, 25), dtype=torch.float32, device=self.dev)
        self._check(self._L.pecc_features(self.h, None, _ptr(f)), "pecc_features")
        return f

    def targets(self, xbefore):
        t = torch.empty((self.total, 2), dtype=torch.float32, device=self.dev)
        self._check(self._L.pecc_targets(self.h, _ptr(xbefore.contiguous()), _ptr(t)), "pecc_targets")
        return t

    def warm_start(self, mlp, rounds=1, max_move=0.25):
        acc = torch.zeros(self.num, dtype=torch.int32, device=self.dev)
        self._check(self._L.pecc_warm_start_ex(self.h, mlp.h, int(rounds), float(max_move), _ptr(acc)),
                    "pecc_warm_start_ex")
        return acc

    def adjust_container(self, R, lambda0=1e-4, rounds=35, out=None, stats=None):
        """pecc_adjust_container: R (float64[num], device or host) -> (R*, iters, status) device
        tensors; the context's coordinates become the adjusted layout.  out: optional (R, iters,
        status) device tensors to reuse (R is then adjusted in place); stats: optional device
        int32[num, 2] receiving {line-search trials, two-loop pair visits}."""
        if out is None:
            Rt = torch.as_tensor(R, dtype=torch.float64).to(self.dev).clone().contiguous()
            iters = torch.empty(self.num, dtype=torch.int32, device=self.dev)
            status = torch.empty(self.num, dtype=torch.int32, device=self.dev)
        else:
            Rt, iters, status = out
        self._check(self._L.pecc_adjust_container(self.h, _ptr(Rt), float(lambda0), int(rounds), _ptr(iters),
                                                  _ptr(status), _ptr(stats) if stats is not None else None),
                    "pecc_adjust_container")
        return Rt, iters, status

    def autotune(self, sweeps=40, seed=99):
        """pecc_autotune: pick threads per block and blocks per SM by timing short descents."""
        b, s = C.c_int32(), C.c_int32()
        self._check(self._L.pecc_autotune(self.h, int(sweeps), C.c_uint64(seed), C.byref(b), C.byref(s)),
                    "pecc_autotune")
        return b.value, s.value

    def launch_shape(self):
        b, s, g = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self._L.pecc_get_launch(self.h, C.byref(b), C.byref(s), C.byref(g)), "pecc_get_launch")
        return b.value, s.value, g.value

    def solve_host(self, R, seed, want_xy=True):
        """Whole path from host memory (pecc_solve_host); R: numpy float64[num]."""
        import numpy as np

        R = np.ascontiguousarray(R, dtype=np.float64)
        xy = np.empty((self.total, 2)) if want_xy else None
        iters = np.empty(self.num, dtype=np.int32)
        status = np.empty(self.num, dtype=np.int32)
        feas = np.empty(self.num, dtype=np.uint8)
        mo = np.empty(self.num, dtype=np.float64)
        a = lambda x: None if x is None else x.ctypes.data_as(C.c_void_p)
        self._check(self._L.pecc_solve_host(self.h, a(R), C.c_uint64(seed), a(xy), a(iters), a(status), a(feas),
                                            a(mo)), "pecc_solve_host")
        return dict(xy=xy, iters=iters, status=status, feasible=feas, max_overlap=mo)


class Sed:
    """One pecc_sed: Algorithm SED (Sec. 5.2) over a batch of instances; every candidate of every
    instance descends in one batched descent.  cfg: the descent's settings (pecc_config fields;
    e_tol defaults to e_feas); sed: pecc_sed_config fields."""

    def __init__(self, n, stream=None, max_candidates=25, s_iter=500, e_feas=1e-25, amp=0.8, shared_r=0,
                 check_every=8, **cfg):
        import numpy as np

        self._L = load()
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        self.num = int(self.n.shape[0])
        self.total = int(self.n.sum())
        cfg.setdefault("e_tol", e_feas)
        self.cfg = default_config(**cfg)
        self.cfg.num_instances = self.num
        self.cfg.n = self.n.ctypes.data_as(C.POINTER(C.c_int32))
        self.sc = SedConfig()
        self._L.pecc_sed_config_default(C.byref(self.sc))
        self.sc.max_candidates, self.sc.s_iter, self.sc.e_feas = int(max_candidates), int(s_iter), float(e_feas)
        self.sc.amp, self.sc.shared_r, self.sc.check_every = float(amp), int(shared_r), int(check_every)
        self.M = int(max_candidates)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        rc = self._L.pecc_sed_create(C.byref(self.cfg), C.byref(self.sc), C.c_void_p(stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise PeccError(f"pecc_sed_create: {ERRORS.get(rc, rc)}: {self._L.pecc_sed_last_error(None).decode()}")
        self.h = h
        self.ctx_h = C.c_void_p(self._L.pecc_sed_context(h))
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def _check(self, rc, what):
        if rc != 0:
            raise PeccError(f"{what}: {ERRORS.get(rc, rc)}: {self._L.pecc_sed_last_error(self.h).decode()}")

    def _check_ctx(self, rc, what):
        if rc != 0:
            raise PeccError(f"{what}: {ERRORS.get(rc, rc)}: {self._L.pecc_last_error(self.ctx_h).decode()}")

    def stats(self, out=None):
        """pecc_get_stats of the candidate context's last descent: int32 [num * M, 10] by slot."""
        st = torch.empty((self.num * self.M, 10), dtype=torch.int32, device=self.dev) if out is None else out
        self._check_ctx(self._L.pecc_get_stats(self.ctx_h, _ptr(st)), "pecc_get_stats")
        return st

    def launch_shape(self):
        b, t, g = C.c_int32(), C.c_int32(), C.c_int32()
        self._check_ctx(self._L.pecc_get_launch(self.ctx_h, C.byref(b), C.byref(t), C.byref(g)), "pecc_get_launch")
        return b.value, t.value, g.value

    def m_counts(self, out=None):
        """The last prepared candidate counts (device int32[num]), without a synchronisation."""
        m = torch.empty(self.num, dtype=torch.int32, device=self.dev) if out is None else out
        self._check(self._L.pecc_sed_get(self.h, None, None, None, None, None, None, _ptr(m), None, None),
                    "pecc_sed_get")
        return m

    def close(self):
        if getattr(self, "h", None):
            self._L.pecc_sed_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_radius(self, R):
        R = torch.as_tensor(R, dtype=torch.float64, device=self.dev).contiguous()
        self._check(self._L.pecc_sed_set_radius(self.h, _ptr(R)), "pecc_sed_set_radius")

    def start(self, seed: int):
        self._check(self._L.pecc_sed_start(self.h, C.c_uint64(seed)), "pecc_sed_start")

    def set_state(self, x, Ex, seed: int, it: int = 0):
        x = torch.as_tensor(x, dtype=torch.float64, device=self.dev).contiguous()
        Ex = torch.as_tensor(Ex, dtype=torch.float64, device=self.dev).contiguous()
        assert x.numel() == 2 * self.total and Ex.numel() == self.num
        self._check(self._L.pecc_sed_set_state(self.h, _ptr(x), _ptr(Ex), C.c_uint64(seed), int(it)),
                    "pecc_sed_set_state")

    def iterate(self, max_iterations):
        ran, left = C.c_int32(), C.c_int32()
        self._check(self._L.pecc_sed_iterate(self.h, int(max_iterations), C.byref(ran), C.byref(left)),
                    "pecc_sed_iterate")
        return ran.value, left.value

    def prepare(self):
        self._check(self._L.pecc_sed_prepare(self.h), "pecc_sed_prepare")

    def descend(self):
        self._check(self._L.pecc_sed_descend(self.h), "pecc_sed_descend")

    def select(self, E_cand=None):
        E = None if E_cand is None else torch.as_tensor(E_cand, dtype=torch.float64, device=self.dev).contiguous()
        if E is not None:
            assert E.numel() == self.num * self.M
        self._check(self._L.pecc_sed_select(self.h, _ptr(E)), "pecc_sed_select")

    def get(self, candidates=False):
        """The state as a dict of device tensors: x, xbest, Ex, Eb, iters, status, m, sel (and
        cand, the candidate slots, when asked)."""
        f64 = dict(dtype=torch.float64, device=self.dev)
        i32 = dict(dtype=torch.int32, device=self.dev)
        out = {"x": torch.empty((self.total, 2), **f64), "xbest": torch.empty((self.total, 2), **f64),
               "Ex": torch.empty(self.num, **f64), "Eb": torch.empty(self.num, **f64),
               "iters": torch.empty(self.num, **i32), "status": torch.empty(self.num, **i32),
               "m": torch.empty(self.num, **i32), "sel": torch.empty(self.num, **i32)}
        cand = torch.empty((self.M * self.total, 2), **f64) if candidates else None
        self._check(self._L.pecc_sed_get(self.h, _ptr(out["x"]), _ptr(out["xbest"]), _ptr(out["Ex"]), _ptr(out["Eb"]),
                                         _ptr(out["iters"]), _ptr(out["status"]), _ptr(out["m"]), _ptr(out["sel"]),
                                         _ptr(cand)), "pecc_sed_get")
        if candidates:
            out["cand"] = cand
        return out


def frame_run(sed, adj, Rb, seed, outer=2, sed_iters=10, lambda0=1e-4, rounds=35, stats=None):
    """pecc_frame_run: the framework of Sec. 5.1 over the instances of `sed` (a Sed), adjusting
    in `adj` (a Context with the same instances).  Returns (R*, x*, R_trace) device tensors;
    stats: optional device int32[3 * num] receiving the adjustments' summed statistics."""
    dev = sed.dev
    Rb = torch.as_tensor(Rb, dtype=torch.float64, device=dev).contiguous()
    Rbest = torch.empty(sed.num, dtype=torch.float64, device=dev)
    xbest = torch.empty((sed.total, 2), dtype=torch.float64, device=dev)
    trace = torch.empty((outer + 1, sed.num), dtype=torch.float64, device=dev)
    sed._check(sed._L.pecc_frame_run(sed.h, adj.h, _ptr(Rb), C.c_uint64(seed), int(outer), int(sed_iters),
                                     float(lambda0), int(rounds), _ptr(Rbest), _ptr(xbest), _ptr(trace), _ptr(stats)),
               "pecc_frame_run")
    return Rbest, xbest, trace

"""Plain FP64 CPU oracle for the elastic-model descent (arXiv 2303.02650).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the CUDA library never does,
and the two share no code.  The arithmetic lives in ``pecc_oracle.c`` (compiled
with ``-O2 -ffp-contract=off``); this module only marshals numpy arrays.

Every function names the passage of the paper it follows:
  * init_positions      Sec. 5.1 random solution (disk of radius R-1, or the square)
  * cell_keys / cell_sort / neighbors_*   Sec. 4.3 neighbor set Gamma(i)
  * energy_* / grad_*   Eq. 3, Eq. 5 (gradient derived from them), Eq. 7
  * partition           Sec. 4.1 sector / annulus / fence partitions
  * lbfgs_direction / dense_bfgs_direction   Eq. 8, Eq. 10, Eq. 11
  * gbo                 Algorithm GBO with ANM (Sec. 4.1, Sec. 4.3)
  * max_overlap         Eq. 1, Eq. 2
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pecc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libpecc_oracle.so")
_lib = None

STATUS = {0: "converged", 1: "stationary", 2: "stalled", 3: "max_iter", 4: "error"}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libpecc_oracle.so (gcc, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-D_POSIX_C_SOURCE=200809L", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Opts(C.Structure):
    _fields_ = [("l_cut", C.c_double), ("rebuild_disp", C.c_double), ("step_max", C.c_double),
                ("e_tol", C.c_double), ("gsum_tol", C.c_double), ("c1", C.c_double),
                ("curv_eps", C.c_double), ("m", C.c_int), ("max_iter", C.c_int), ("k", C.c_int),
                ("partition", C.c_int), ("max_trials", C.c_int), ("anm", C.c_int),
                ("prec32_pred", C.c_int), ("part_seed", C.c_uint64), ("part_inst", C.c_int), ("dense", C.c_int)]


class Result(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("builds", C.c_int), ("changes", C.c_int),
                ("disp_builds", C.c_int), ("trials", C.c_int), ("resets", C.c_int),
                ("stalls", C.c_int), ("E", C.c_double), ("gsum", C.c_double)]


class SedResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("descents", C.c_int), ("E0", C.c_double),
                ("E", C.c_double)]


def _P(t):
    return C.POINTER(t)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i32, u32, i64 = _P(C.c_double), _P(C.c_int32), _P(C.c_uint32), _P(C.c_int64)
        sig = {
            "orc_philox4x32_10": (None, [u32, u32, u32]),
            "orc_init_positions": (None, [C.c_int, C.c_double, C.c_uint64, C.c_int, C.c_int, d]),
            "orc_cell_grid": (None, [C.c_double, C.c_double, C.c_int, d, _P(C.c_int)]),
            "orc_cell_keys": (None, [C.c_int, d, C.c_double, C.c_double, u32]),
            "orc_cell_sort": (None, [C.c_int, u32, C.c_int, i32, i32]),
            "orc_neighbors_brute": (C.c_int64, [C.c_int, d, C.c_double, C.c_int, i32, i32, C.c_int64]),
            "orc_neighbors_cells": (C.c_int64, [C.c_int, d, C.c_double, C.c_double, C.c_int, i32, i32,
                                                C.c_int64]),
            "orc_energy_allpairs": (C.c_double, [C.c_int, d, C.c_double]),
            "orc_energy_csr": (C.c_double, [C.c_int, d, C.c_double, i32, i32]),
            "orc_energy_grad_csr": (C.c_double, [C.c_int, d, C.c_double, i32, i32, d, _P(C.c_int)]),
            "orc_grad_allpairs": (None, [C.c_int, d, C.c_double, d]),
            "orc_batch_energy": (C.c_double, [d, C.c_double, i32, i32, i32, C.c_int, i32, C.c_int]),
            "orc_pseudo_angle": (C.c_double, [C.c_double, C.c_double]),
            "orc_default_k": (C.c_int, [C.c_int]),
            "orc_partition": (None, [C.c_int, d, C.c_int, C.c_int, i32, i32]),
            "orc_partition_seeded": (None, [C.c_int, d, C.c_int, C.c_int, C.c_uint64, C.c_int, i32, i32]),
            "orc_lbfgs_direction": (None, [C.c_int, C.c_int, d, d, d, d]),
            "orc_dense_bfgs_direction": (None, [C.c_int, C.c_int, d, d, d, d]),
            "orc_default_opts": (None, [_P(Opts)]),
            "orc_gbo": (C.c_int, [C.c_int, d, C.c_double, _P(Opts), _P(Result), d]),
            "orc_max_overlap": (C.c_double, [C.c_int, d, C.c_double, d, d]),
            "orc_u_energy_grad": (C.c_double, [C.c_int, d, C.c_double, C.c_double, d]),
            "orc_adjust_container": (C.c_int, [C.c_int, d, d, _P(Opts), C.c_double, C.c_int, _P(Result)]),
            "orc_bfgs_update": (None, [C.c_int, d, d, d]),
            "orc_sed_J": (C.c_int, [C.c_double]),
            "orc_sed_perturb": (None, [C.c_int, d, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, d]),
            "orc_sed_select": (C.c_int, [C.c_int, d, C.c_double, C.c_uint64, C.c_int, C.c_int]),
            "orc_sed": (C.c_int, [C.c_int, C.c_double, C.c_uint64, C.c_int, C.c_int, _P(Opts), C.c_int, C.c_int,
                                  C.c_double, C.c_int, C.c_double, d, _P(SedResult), i32, i32, d, d]),
            "orc_frame": (C.c_int, [C.c_int, C.c_double, C.c_uint64, C.c_int, C.c_int, _P(Opts), C.c_int, C.c_int,
                                    C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, d, d, d]),
            "orc_solve_batch": (C.c_double, [C.c_int, i32, d, C.c_uint64, C.c_int, C.c_int, _P(Opts),
                                             C.c_double, C.c_int, d, i32, i32, d, d, _P(C.c_uint8)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(_P(t))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------- RNG / init
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11) of one 4-word counter under a 2-word key."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def init_positions(n: int, R: float, seed: int, inst: int = 0, mode: int = 0) -> np.ndarray:
    """Random layout of Sec. 5.1: mode 0 uniform in the disk of radius R-1, mode 1 square U(-R,R)^2."""
    xy = np.zeros((n, 2), dtype=np.float64)
    lib().orc_init_positions(n, R, seed, inst, mode, _ptr(xy, C.c_double))
    return xy


# --------------------------------------------------------------------------- cells / neighbors
def cell_grid(R: float, l_cut: float, n: int):
    """Cell grid of an instance: (1 / cell side, cells per side)."""
    inv = C.c_double()
    nc = C.c_int()
    lib().orc_cell_grid(R, l_cut, n, C.byref(inv), C.byref(nc))
    return inv.value, nc.value


def cell_keys(xy, R, l_cut):
    xy = _f64(xy)
    n = xy.shape[0]
    key = np.zeros(n, dtype=np.uint32)
    lib().orc_cell_keys(n, _ptr(xy, C.c_double), R, l_cut, _ptr(key, C.c_uint32))
    return key


def cell_sort(key, ncell):
    key = np.ascontiguousarray(key, dtype=np.uint32)
    n = key.shape[0]
    order = np.zeros(n, dtype=np.int32)
    start = np.zeros(ncell + 1, dtype=np.int32)
    lib().orc_cell_sort(n, _ptr(key, C.c_uint32), ncell, _ptr(order, C.c_int32), _ptr(start, C.c_int32))
    return order, start


def _nbr(fn, n, args, cap):
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    while True:
        col = np.zeros(max(cap, 1), dtype=np.int32)
        r = fn(*args, _ptr(row_ptr, C.c_int32), _ptr(col, C.c_int32), cap)
        if r >= 0:
            return row_ptr, col[:r].copy()
        cap = -r


def neighbors_brute(xy, l_cut=2.5, prec32=False):
    """Gamma(i) of Sec. 4.3 by testing all pairs; rows ascending."""
    xy = _f64(xy)
    n = xy.shape[0]
    return _nbr(lib().orc_neighbors_brute, n, (n, _ptr(xy, C.c_double), l_cut, int(prec32)), 8 * n + 16)


def neighbors_cells(xy, R, l_cut=2.5, prec32=False):
    """Gamma(i) of Sec. 4.3 through cell binning; rows ascending."""
    xy = _f64(xy)
    n = xy.shape[0]
    return _nbr(lib().orc_neighbors_cells, n, (n, _ptr(xy, C.c_double), R, l_cut, int(prec32)), 8 * n + 16)


# --------------------------------------------------------------------------- energy
def energy_allpairs(xy, R):
    """Eq. 5 summed over all pairs i < j and all boundary terms."""
    xy = _f64(xy)
    return lib().orc_energy_allpairs(xy.shape[0], _ptr(xy, C.c_double), R)


def energy_grad_csr(xy, R, row_ptr, col):
    """Eq. 5 in neighbor-list form and its gradient; returns (E, g[n,2], degenerate_pairs)."""
    xy = _f64(xy)
    n = xy.shape[0]
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    if cl.size == 0:
        cl = np.zeros(1, dtype=np.int32)
    g = np.zeros((n, 2), dtype=np.float64)
    deg = C.c_int(0)
    E = lib().orc_energy_grad_csr(n, _ptr(xy, C.c_double), R, _ptr(rp, C.c_int32), _ptr(cl, C.c_int32),
                                  _ptr(g, C.c_double), C.byref(deg))
    return E, g, deg.value


def grad_allpairs(xy, R):
    xy = _f64(xy)
    n = xy.shape[0]
    g = np.zeros((n, 2), dtype=np.float64)
    lib().orc_grad_allpairs(n, _ptr(xy, C.c_double), R, _ptr(g, C.c_double))
    return g


def batch_energy(xy, R, row_ptr, col, members, batch_of, p):
    """Batch energy of Eq. 7 (neighbor-list form)."""
    xy = _f64(xy)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col if len(col) else np.zeros(1), dtype=np.int32)
    mb = np.ascontiguousarray(members, dtype=np.int32)
    bo = np.ascontiguousarray(batch_of, dtype=np.int32)
    return lib().orc_batch_energy(_ptr(xy, C.c_double), R, _ptr(rp, C.c_int32), _ptr(cl, C.c_int32),
                                  _ptr(mb, C.c_int32), mb.shape[0], _ptr(bo, C.c_int32), p)


# --------------------------------------------------------------------------- partition
def pseudo_angle(x, y):
    return lib().orc_pseudo_angle(float(x), float(y))


def default_k(n):
    return lib().orc_default_k(n)


def partition(xy, k, mode=0, seed=0, inst=0):
    """Sec. 4.1 partitions (0 sector, 1 annulus, 2 fence, 3 random with Philox key seed and
    instance word inst): (perm[n], bounds[k+1])."""
    xy = _f64(xy)
    n = xy.shape[0]
    perm = np.zeros(n, dtype=np.int32)
    bounds = np.zeros(k + 1, dtype=np.int32)
    lib().orc_partition_seeded(n, _ptr(xy, C.c_double), k, mode, int(seed), int(inst), _ptr(perm, C.c_int32),
                               _ptr(bounds, C.c_int32))
    return perm, bounds


# --------------------------------------------------------------------------- quasi-Newton
def lbfgs_direction(S, Y, g):
    """-H g for the pairs (S, Y) (oldest first) by the two-loop recursion."""
    S, Y, g = _f64(S), _f64(Y), _f64(g)
    cnt, dim = (S.shape[0], S.shape[1]) if S.ndim == 2 else (0, g.shape[0])
    d = np.zeros(dim)
    lib().orc_lbfgs_direction(dim, cnt, _ptr(S, C.c_double), _ptr(Y, C.c_double), _ptr(g, C.c_double),
                              _ptr(d, C.c_double))
    return d


def dense_bfgs_direction(S, Y, g):
    """-H g with H built by Eq. 11 pair by pair from gamma I (Eq. 10 for beta)."""
    S, Y, g = _f64(S), _f64(Y), _f64(g)
    cnt, dim = (S.shape[0], S.shape[1]) if S.ndim == 2 else (0, g.shape[0])
    d = np.zeros(dim)
    lib().orc_dense_bfgs_direction(dim, cnt, _ptr(S, C.c_double), _ptr(Y, C.c_double), _ptr(g, C.c_double),
                                   _ptr(d, C.c_double))
    return d


# --------------------------------------------------------------------------- descent
@dataclass
class GboResult:
    x: np.ndarray
    iters: int
    status: str
    builds: int
    changes: int
    disp_builds: int
    trials: int
    resets: int
    stalls: int
    E: float
    gsum: float
    trace: np.ndarray


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().orc_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def gbo(xy, R, **kw) -> GboResult:
    """Algorithm GBO (Sec. 4.1) with ANM (Sec. 4.3) on one instance; does not modify xy."""
    o = default_opts(**kw)
    x = _f64(xy).copy()
    n = x.shape[0]
    trace = np.full(o.max_iter + 1, np.nan)
    r = Result()
    lib().orc_gbo(n, _ptr(x, C.c_double), R, C.byref(o), C.byref(r), _ptr(trace, C.c_double))
    return GboResult(x, r.iters, STATUS[r.status], r.builds, r.changes, r.disp_builds, r.trials, r.resets,
                     r.stalls, r.E, r.gsum, trace[: r.iters + 1])


def u_energy_grad(xy, R, lam):
    """Eq. 12: U = E + lam R^2 and its gradient over z = (x, R) (brute-force lists): (U, g[2n + 1])."""
    x = _f64(xy)
    n = x.shape[0]
    g = np.zeros(2 * n + 1)
    U = lib().orc_u_energy_grad(n, _ptr(x, C.c_double), R, lam, _ptr(g, C.c_double))
    return U, g


def adjust_container(xy, R, lambda0=1e-4, rounds=35, **kw):
    """Algorithm adjust_container (Sec. 4.2): returns (x*, R*, result); does not modify xy."""
    o = default_opts(**kw)
    x = _f64(xy).copy()
    n = x.shape[0]
    Rv = np.array([float(R)])
    r = Result()
    lib().orc_adjust_container(n, _ptr(x, C.c_double), _ptr(Rv, C.c_double), C.byref(o), float(lambda0), int(rounds),
                               C.byref(r))
    return x, float(Rv[0]), GboResult(x, r.iters, STATUS[r.status], r.builds, r.changes, r.disp_builds, r.trials,
                                      r.resets, r.stalls, r.E, r.gsum, None)


def bfgs_update(H, s, y):
    """Eq. 11 applied once to H (returns the updated copy), as the dense descent applies it."""
    Hc = _f64(H).copy()
    lib().orc_bfgs_update(Hc.shape[0], _ptr(Hc, C.c_double), _ptr(_f64(s), C.c_double), _ptr(_f64(y), C.c_double))
    return Hc


def sed_J(E):
    """J(E) = ceil(-log10 E) of Sec. 5.2 (2^30 for E <= 0)."""
    return int(lib().orc_sed_J(float(E)))


def sed_perturb(xy, seed, inst, it, j, shared=0, amp=0.8):
    """The perturbation of Sec. 5.2 of layout xy: candidate j of SED iteration it."""
    x = _f64(xy)
    out = np.empty_like(x)
    lib().orc_sed_perturb(x.shape[0], _ptr(x, C.c_double), int(seed), int(inst), int(it), int(j), int(shared),
                          float(amp), _ptr(out, C.c_double))
    return out


def sed_select(E, Ex, seed, inst, it):
    """The select operator of Eq. 18 over candidate energies E, operated solution energy Ex."""
    e = _f64(E)
    return int(lib().orc_sed_select(e.size, _ptr(e, C.c_double), float(Ex), int(seed), int(inst), int(it)))


@dataclass
class SedOut:
    x: np.ndarray
    E: float
    E0: float
    iters: int
    status: str
    descents: int
    m: np.ndarray
    sel: np.ndarray
    Ex: np.ndarray
    Eb: np.ndarray


def sed(n, R, seed, inst=0, s_iter=500, max_cand=25, e_feas=1e-25, shared=0, amp=0.8, init_mode=0, **kw):
    """Algorithm SED (Sec. 5.2) on one instance.  The GBO inside stops at e_tol = e_feas unless
    e_tol is given."""
    kw.setdefault("e_tol", e_feas)
    o = default_opts(**kw)
    x = np.zeros((int(n), 2))
    r = SedResult()
    mt = np.zeros(max(s_iter, 1), dtype=np.int32)
    st = np.zeros(max(s_iter, 1), dtype=np.int32)
    ex = np.zeros(max(s_iter, 1))
    eb = np.zeros(max(s_iter, 1))
    lib().orc_sed(int(n), float(R), int(seed), int(inst), int(init_mode), C.byref(o), int(s_iter), int(max_cand),
                  float(e_feas), int(shared), float(amp), _ptr(x, C.c_double), C.byref(r), _ptr(mt, C.c_int32),
                  _ptr(st, C.c_int32), _ptr(ex, C.c_double), _ptr(eb, C.c_double))
    k = r.iters
    return SedOut(x, r.E, r.E0, k, STATUS[r.status], r.descents, mt[:k], st[:k], ex[:k], eb[:k])


def frame(n, Rb, seed, inst=0, outer=2, s_iter=10, max_cand=25, e_feas=1e-25, amp=0.8, lambda0=1e-4, rounds=35,
          init_mode=0, **kw):
    """The framework of Sec. 5.1 with `outer` iterations in place of the cut-off time:
    (x*, R*, R_trace)."""
    o = default_opts(**kw)
    x = np.zeros((int(n), 2))
    Rb_out = np.zeros(1)
    tr = np.zeros(outer + 1)
    lib().orc_frame(int(n), float(Rb), int(seed), int(inst), int(init_mode), C.byref(o), int(outer), int(s_iter),
                    int(max_cand), float(e_feas), float(amp), float(lambda0), int(rounds), _ptr(x, C.c_double),
                    _ptr(Rb_out, C.c_double), _ptr(tr, C.c_double))
    return x, float(Rb_out[0]), tr


def max_overlap(xy, R):
    """Eq. 1 / Eq. 2 check: (max overall, max pair depth, max boundary depth), brute force."""
    xy = _f64(xy)
    mp, mb = C.c_double(), C.c_double()
    m = lib().orc_max_overlap(xy.shape[0], _ptr(xy, C.c_double), R, C.byref(mp), C.byref(mb))
    return m, mp.value, mb.value


def solve_batch(n, R, seed, inst_base=0, init_mode=0, feas_tol=1e-9, nthreads=1, **kw):
    """Init + GBO + feasibility for many instances on nthreads host threads.

    Returns (wall_seconds, dict of per-instance arrays)."""
    o = default_opts(**kw)
    n = np.ascontiguousarray(n, dtype=np.int32)
    R = _f64(R)
    num = n.shape[0]
    xy = np.zeros((int(n.sum()), 2))
    iters = np.zeros(num, dtype=np.int32)
    status = np.zeros(num, dtype=np.int32)
    E = np.zeros(num)
    mo = np.zeros(num)
    feas = np.zeros(num, dtype=np.uint8)
    t = lib().orc_solve_batch(num, _ptr(n, C.c_int32), _ptr(R, C.c_double), seed, inst_base, init_mode,
                              C.byref(o), feas_tol, nthreads, _ptr(xy, C.c_double), _ptr(iters, C.c_int32),
                              _ptr(status, C.c_int32), _ptr(E, C.c_double), _ptr(mo, C.c_double),
                              _ptr(feas, C.c_uint8))
    return t, dict(xy=xy, iters=iters, status=status, E=E, max_overlap=mo, feasible=feas)

"""Python access to the FP64 CPU oracle (oracle/sph_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` use it; the product package never
imports it. It is built with plain gcc (``build()``), independent of the CUDA
library, and takes problem descriptions from the ``workloads`` input module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsph_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP). Returns the .so path."""
    src = os.path.join(_HERE, "sph_oracle.c")
    hdr = os.path.join(_HERE, "sph_oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wno-unused-function",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Shape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("keep_inside", C.c_int32),
                ("center", C.c_double * 3), ("size", C.c_double * 3)]


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_shapes", C.c_int32),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("shapes", Shape * 4),
                ("field_kind", C.c_int32), ("dist_shape", C.c_int32),
                ("s0", C.c_double), ("a", C.c_double), ("b", C.c_double),
                ("n_poly", C.c_int32), ("eos_general", C.c_int32), ("poly", C.c_double * 8),
                ("rho_scale", C.c_double),
                ("P0", C.c_double), ("gamma", C.c_double), ("sigma0", C.c_double),
                ("tau", C.c_double), ("kappa", C.c_double),
                ("t0", C.c_double), ("t1", C.c_double),
                ("bg_dims", C.c_int32 * 3), ("bg_pad", C.c_int32), ("bg_lo", C.c_double * 3),
                ("bg_hi", C.c_double * 3), ("bg_phi", C.c_void_p), ("bg_s", C.c_void_p),
                ("surface", C.c_void_p)]


class Grid(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("dim", C.c_int32), ("lo", C.c_double * 3), ("h0", C.c_double),
                ("cell", C.c_double * 8), ("dims", (C.c_int32 * 3) * 8), ("base", C.c_uint32 * 9)]


class StepInfo(C.Structure):
    _fields_ = [("sigma", C.c_double), ("dt1", C.c_double), ("dt2", C.c_double),
                ("min_rc_over_a", C.c_double), ("max_a", C.c_double),
                ("sum_rho", C.c_double), ("err_l2", C.c_double), ("err_max", C.c_double),
                ("interface_pairs", C.c_int64), ("force_pairs", C.c_int64),
                ("wall_moved", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def bind(path):
    """Load an oracle library from `path` and declare its function types
    (lib() binds the one build() makes)."""
    L = C.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def _declare(L):
    L.orc_W.restype = C.c_double
    L.orc_W.argtypes = [C.c_double, C.c_double, C.c_int]
    L.orc_dW.restype = C.c_double
    L.orc_dW.argtypes = [C.c_double, C.c_double, C.c_int]
    L.orc_dW_over_r.restype = C.c_double
    L.orc_dW_over_r.argtypes = [C.c_double, C.c_double, C.c_int]
    L.orc_phi.restype = C.c_double
    L.orc_phi.argtypes = [C.POINTER(Problem), _dp]
    L.orc_project.restype = C.c_int
    L.orc_project.argtypes = [C.POINTER(Problem), _dp]
    L.orc_rho_t.restype = C.c_double
    L.orc_rho_t.argtypes = [C.POINTER(Problem), _dp]
    L.orc_h.restype = C.c_double
    L.orc_h.argtypes = [C.POINTER(Problem), _dp]
    L.orc_sigma.restype = C.c_double
    L.orc_sigma.argtypes = [C.POINTER(Problem), C.c_double]
    L.orc_total_mass.restype = C.c_double
    L.orc_total_mass.argtypes = [C.POINTER(Problem), C.c_int]
    L.orc_neighbor_sets.restype = C.c_int
    L.orc_neighbor_sets.argtypes = [C.POINTER(Problem), C.c_int64, _dp, C.c_int,
                                    _i32p, _i32p, _i64p, _i64p, _i64p, _i64p]
    L.orc_step.restype = C.c_int
    L.orc_step.argtypes = [C.POINTER(Problem), C.c_int64, _dp, _u8p, C.c_int64, C.c_int,
                           C.POINTER(StepInfo), C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p]
    L.orc_step_fixed_dt.restype = C.c_int
    L.orc_step_fixed_dt.argtypes = [C.POINTER(Problem), C.c_int64, _dp, _u8p, C.c_int64, C.c_int,
                                    _dp, C.POINTER(StepInfo)]
    L.orc_objective.restype = C.c_int
    L.orc_objective.argtypes = [C.POINTER(Problem), C.c_int64, _dp, _u8p, C.c_double,
                                C.POINTER(C.c_double)]
    L.orc_backward.restype = C.c_int
    L.orc_backward.argtypes = [C.POINTER(Problem), C.c_int64, _dp, _u8p, C.c_int64, C.c_int32,
                               C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                               C.POINTER(C.c_double), _dp, _dp]
    L.orc_num_threads.restype = C.c_int
    L.orc_num_threads.argtypes = []
    L.orc_cell_keys.restype = C.c_int
    L.orc_cell_keys.argtypes = [C.POINTER(Problem), C.c_int64, _dp, C.POINTER(Grid),
                                np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS"), _dp]


def to_c(p) -> Problem:
    """Marshal a workloads.Problem into the oracle's struct."""
    c = Problem()
    c.dim = p.dim
    c.n_shapes = len(p.shapes)
    for k in range(3):
        c.lo[k] = float(p.lo[k]) if k < len(p.lo) else 0.0
        c.hi[k] = float(p.hi[k]) if k < len(p.hi) else 0.0
    for s_i, s in enumerate(p.shapes):
        c.shapes[s_i].kind = s.kind
        c.shapes[s_i].keep_inside = 1 if s.keep_inside else 0
        for k in range(3):
            c.shapes[s_i].center[k] = float(s.center[k]) if k < len(s.center) else 0.0
            c.shapes[s_i].size[k] = float(s.size[k]) if k < len(s.size) else 0.0
    c.field_kind = p.field_kind
    c.dist_shape = p.dist_shape
    c.s0, c.a, c.b = p.s0, p.a, p.b
    c.n_poly = len(p.poly)
    c.eos_general = 1 if getattr(p, 'eos_general', False) else 0
    for k, v in enumerate(p.poly[:8]):
        c.poly[k] = float(v)
    c.rho_scale = p.rho_scale
    c.P0, c.gamma, c.sigma0, c.tau, c.kappa = p.P0, p.gamma, p.sigma0, p.tau, p.kappa
    c.t0, c.t1 = p.t0, p.t1
    keep = []
    surf = getattr(p, "surface", None)
    if surf is not None:
        a = np.ascontiguousarray(np.asarray(surf, dtype=bool).astype(np.uint8))
        keep.append(a)
        c.surface = a.ctypes.data
    bg = getattr(p, "bg", None)
    if bg is not None:
        for k in range(3):
            c.bg_dims[k] = int(bg.dims[k])
            c.bg_lo[k] = float(bg.lo[k])
            c.bg_hi[k] = float(bg.hi[k])
        for name in ("phi", "spacing"):
            v = getattr(bg, name)
            if v is not None:
                a = np.ascontiguousarray(v, dtype=np.float64).ravel(order="F")
                keep.append(a)
                setattr(c, "bg_phi" if name == "phi" else "bg_s", a.ctypes.data)
    c._keep = keep  # the arrays live as long as the struct
    return c


def W(r, H, dim):
    return lib().orc_W(float(r), float(H), int(dim))


def dW(r, H, dim):
    return lib().orc_dW(float(r), float(H), int(dim))


def dW_over_r(r, H, dim):
    return lib().orc_dW_over_r(float(r), float(H), int(dim))


def _pt(p, x):
    v = np.zeros(3)
    v[: p.dim] = np.asarray(x, dtype=np.float64)[: p.dim]
    return v


def phi(p, x):
    return lib().orc_phi(C.byref(to_c(p)), _pt(p, x))


def project(p, x):
    v = _pt(p, x)
    lib().orc_project(C.byref(to_c(p)), v)
    return v[: p.dim]


def rho_t(p, x):
    return lib().orc_rho_t(C.byref(to_c(p)), _pt(p, x))


def h_of(p, x):
    return lib().orc_h(C.byref(to_c(p)), _pt(p, x))


def sigma(p, t):
    return lib().orc_sigma(C.byref(to_c(p)), float(t))


def total_mass(p, res):
    return lib().orc_total_mass(C.byref(to_c(p)), int(res))


def neighbor_sets(p, pos, mode=1):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    dc = np.zeros(n, np.int32); fc = np.zeros(n, np.int32)
    ds = np.zeros(n, np.int64); fs = np.zeros(n, np.int64)
    dx = np.zeros(n, np.int64); fx = np.zeros(n, np.int64)
    rc = lib().orc_neighbor_sets(C.byref(to_c(p)), n, pos, int(mode), dc, fc, ds, fs, dx, fx)
    if rc != 0:
        raise RuntimeError("oracle neighbour search failed")
    return dict(dens_count=dc, force_count=fc, dens_idsum=ds, force_idsum=fs,
                dens_idxor=dx, force_idxor=fx)


def cell_keys(p, pos, grid):
    """Cell key of every particle in the multi-resolution grid `grid` (a dict
    with n_levels, lo, h0, cell[l], dims[l], base[l]: the cell structure's
    configuration) and the smoothing lengths h_i. See orc_cell_keys."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    g = Grid()
    g.n_levels = int(grid["n_levels"])
    g.dim = p.dim
    for k in range(3):
        g.lo[k] = float(grid["lo"][k])
    g.h0 = float(grid["h0"])
    for l in range(g.n_levels):
        g.cell[l] = float(grid["cell"][l])
        for k in range(3):
            g.dims[l][k] = int(grid["dims"][l][k])
    for l in range(g.n_levels + 1):
        g.base[l] = int(grid["base"][l])
    keys = np.zeros(pos.shape[0], np.uint32)
    h = np.zeros(pos.shape[0])
    lib().orc_cell_keys(C.byref(to_c(p)), pos.shape[0], pos, C.byref(g), keys, h)
    return keys, h


def color_volumes(rho, col, n_colors):
    """Per colour c: V_c = sum over its particles of m_i/rho_i (unit mass,
    Eq. mass_SPH_particle; rho from Eq. density_sum) and the particle count,
    the size and mass of each sub-domain of the partition (Sec. 2.1, 2.3).
    FP64 sums in particle order."""
    col = np.asarray(col)
    v = np.zeros(n_colors)
    k = np.zeros(n_colors, np.int64)
    for c in range(n_colors):
        m = col == c
        v[c] = float(np.sum(1.0 / np.asarray(rho, dtype=np.float64)[m]))
        k[c] = int(m.sum())
    return v, k


def cell_order(keys):
    """Particle ids ordered by (cell key, particle id): a stable sort of the
    keys, which leaves equal keys in ascending id order."""
    return np.argsort(np.asarray(keys, dtype=np.int64), kind="stable").astype(np.uint32)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def step(p, pos, col, step_index=0, mode=1, want=True):
    """One relaxation step on a copy of pos. Returns (new_pos, info dict, fields)
    where fields holds rho, acc (a_n), visc (a~), pair_abs_a, pair_abs_b."""
    pos = np.array(pos, dtype=np.float64, order="C", copy=True)
    col = np.ascontiguousarray(col, dtype=np.uint8)
    n, d = pos.shape
    info = StepInfo()
    f = {}
    if want:
        f = dict(rho=np.zeros(n), acc=np.zeros((n, d)), visc=np.zeros((n, d)),
                 pair_abs_a=np.zeros(n), pair_abs_b=np.zeros(n))
    rc = lib().orc_step(C.byref(to_c(p)), n, pos, col, int(step_index), int(mode), C.byref(info),
                        _ptr(f.get("rho")), _ptr(f.get("acc")), _ptr(f.get("visc")),
                        _ptr(f.get("pair_abs_a")), _ptr(f.get("pair_abs_b")))
    if rc != 0:
        raise RuntimeError("oracle step failed")
    return pos, info.as_dict(), f


def run(p, pos, col, n_steps, start_step=0, mode=1):
    """n_steps steps; returns (pos, list of info dicts)."""
    infos = []
    for s in range(n_steps):
        pos, info, _ = step(p, pos, col, start_step + s, mode, want=False)
        infos.append(info)
    return pos, infos


def num_threads():
    return lib().orc_num_threads()


def run_fixed_dt(p, pos, col, dts, start_step=0, mode=1):
    """len(dts) steps with prescribed (dt1, dt2) per step; returns the end state."""
    pos = np.array(pos, dtype=np.float64, order="C", copy=True)
    col = np.ascontiguousarray(col, dtype=np.uint8)
    pc = to_c(p)
    info = StepInfo()
    for s, dt in enumerate(np.asarray(dts, dtype=np.float64).reshape(-1, 2)):
        rc = lib().orc_step_fixed_dt(C.byref(pc), pos.shape[0], pos, col, int(start_step + s), int(mode),
                                     np.ascontiguousarray(dt), C.byref(info))
        if rc != 0:
            raise RuntimeError("oracle step failed")
    return pos


def objective(p, pos, col, lam):
    """L = sum_i (rho_i/rho_t,i - 1)^2 + lam * sum_{i<j, C_i != C_j} W(r_ij, kappa h_ij)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    col = np.ascontiguousarray(col, dtype=np.uint8)
    out = C.c_double()
    if lib().orc_objective(C.byref(to_c(p)), pos.shape[0], pos, col, float(lam), C.byref(out)) != 0:
        raise RuntimeError("oracle objective failed")
    return out.value


GRAD_NAMES = ("sigma0", "gamma", "P0") + tuple(f"poly{m}" for m in range(8))


def backward(p, pos0, col, n_steps, lam, dt=None, seed=None, start_step=0):
    """Sensitivities of L after n_steps steps from pos0 (see orc_backward).
    dt: None (step sizes recomputed and differentiated) or (n_steps, 2) prescribed.
    Returns dict(L, dpos0, grads {name: value}, dt (n_steps, 2))."""
    pos0 = np.ascontiguousarray(pos0, dtype=np.float64)
    col = np.ascontiguousarray(col, dtype=np.uint8)
    n, d = pos0.shape
    dt_in = None if dt is None else np.ascontiguousarray(np.asarray(dt, dtype=np.float64).reshape(-1))
    dt_out = np.zeros(2 * n_steps)
    sd = None if seed is None else np.ascontiguousarray(seed, dtype=np.float64).reshape(-1)
    L = C.c_double()
    dpos = np.zeros((n, d))
    g = np.zeros(11)
    rc = lib().orc_backward(C.byref(to_c(p)), n, pos0, col, int(start_step), int(n_steps), _ptr(dt_in),
                            _ptr(dt_out), float(lam), _ptr(sd), C.byref(L), dpos, g)
    if rc != 0:
        raise RuntimeError("oracle backward failed")
    return dict(L=L.value, dpos0=dpos, grads=dict(zip(GRAD_NAMES, g)), dt=dt_out.reshape(-1, 2))


def convergence_step(counts, window, tol):
    """Index of the step at which the partition is taken as converged (Sec. 3.3:
    the interface topology stays static for a number of iterations, e.g. 50),
    read as: the interface-pair count of every step stays within tol (relative)
    of the count that opened the current run for `window` further steps.
    counts[s] is step s's count; returns the first s that closes such a run,
    or None."""
    ref, stable = None, 0
    for s, c in enumerate(counts):
        if ref is not None and abs(c - ref) <= tol * ref:
            stable += 1
        else:
            ref, stable = c, 0
        if stable >= window:
            return s
    return None


def run_auto_ramp(p, pos, col, n_steps, window, tol, theta, start_step=0, mode=1):
    """n_steps steps with the surface-tension ramp started automatically: once
    convergence_step fires at step s, t0 = s and t1 = (1 + theta) t0 (the ramp
    of Eq. sph_st_sigma over the fraction theta of the steps taken, Sec. 3.3).
    Returns (pos, infos, t0)."""
    import copy
    q = copy.deepcopy(p)
    q.t0, q.t1 = -1.0, -1.0
    infos, counts, t0 = [], [], None
    for s in range(n_steps):
        step_index = start_step + s
        pos, info, _ = step(q, pos, col, step_index, mode, want=False)
        infos.append(info)
        if t0 is None:
            counts.append(info["interface_pairs"])
            if convergence_step(counts, window, tol) == len(counts) - 1:
                t0 = step_index
                q.t0, q.t1 = float(t0), (1.0 + theta) * t0
    return pos, infos, t0

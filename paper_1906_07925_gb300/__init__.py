"""GB300-native multi-phase SPH particle relaxation (arXiv 1906.07925).

Python face of libsphmesh (include/sphmesh.h). Every step of the relaxation
runs in the library's CUDA kernels; this module only marshals arguments and
lends PyTorch's caching allocator and a CUDA stream to the library.

    from paper_1906_07925_gb300 import Relaxation
    r = Relaxation(problem, n_particles=1 << 20, precision="fp32")
    r.step(500); r.ramp_surface_tension(500, 700); r.step(200)
    x, c = r.positions(), r.colors()
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _binding as B

__all__ = ["Batch", "Relaxation", "SphError", "build", "load_library", "problem_structs", "relax_fn"]


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{B.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def build(force=False):
    from .build import build as _b
    return _b(force=force)


def load_library():
    return B.load()


def problem_structs(p, precision="fp32", seed=0, cell_factor=0.0, use_graph=True, record_fields=False, skin=0.0,
                    list_capacity=0):
    """Marshal a problem description (attributes: dim, lo, hi, shapes, field_kind,
    s0, a, b, dist_shape, poly, rho_scale, P0, gamma, sigma0, tau, kappa) into
    the C structs."""
    d = B.sph_domain()
    d.dim = p.dim
    d.n_shapes = len(p.shapes)
    for k in range(3):
        d.lo[k] = float(p.lo[k]) if k < len(p.lo) else 0.0
        d.hi[k] = float(p.hi[k]) if k < len(p.hi) else 0.0
    for i, s in enumerate(p.shapes):
        d.shapes[i].kind = int(s.kind)
        d.shapes[i].keep_inside = 1 if s.keep_inside else 0
        for k in range(3):
            d.shapes[i].center[k] = float(s.center[k]) if k < len(s.center) else 0.0
            d.shapes[i].size[k] = float(s.size[k]) if k < len(s.size) else 0.0
    f = B.sph_field()
    f.kind = int(p.field_kind)
    f.dist_shape = int(p.dist_shape)
    f.s0, f.a, f.b = float(p.s0), float(p.a), float(p.b)
    f.n_poly = len(p.poly)
    for k, v in enumerate(list(p.poly)[:8]):
        f.poly[k] = float(v)
    f.rho_scale = float(p.rho_scale or 0.0)
    q = B.sph_params()
    q.P0, q.gamma, q.sigma0, q.tau, q.kappa = float(p.P0), float(p.gamma), float(p.sigma0), float(p.tau), float(p.kappa)
    q.precision = B.SPH_PREC_FP64 if precision in ("fp64", "f64", "double") else B.SPH_PREC_FP32_SPLIT
    q.kernel_id = 0
    q.seed = int(seed)
    q.cell_factor = float(cell_factor)
    q.use_graph = 1 if use_graph else 0
    q.record_fields = 1 if record_fields else 0
    q.skin = float(skin)
    q.list_capacity = int(list_capacity)
    return d, f, q


def background_struct(bg):
    """Marshal a background mesh (attributes dims, lo, hi, phi, spacing; the
    arrays shaped dims and indexed [i, j, k]) into sph_background. Returns
    (struct, arrays kept alive for the call) or None."""
    if bg is None:
        return None
    import numpy as np
    s = B.sph_background()
    keep = []
    for k in range(3):
        s.dims[k] = int(bg.dims[k])
        s.lo[k] = float(bg.lo[k])
        s.hi[k] = float(bg.hi[k])
    for name in ("phi", "spacing"):
        v = getattr(bg, name, None)
        if v is not None:
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).ravel(order="F"))
            keep.append(a)
            setattr(s, name, a.ctypes.data)
    return s, keep


class Relaxation:
    """One relaxation instance on the current CUDA device.

    problem: geometry/field/parameters (see problem_structs); n_particles and
    n_colors size the initial state drawn by the library (density-proportional
    sampling, nearest-generator colours); set_state() replaces it.
    """

    def __init__(self, problem, n_particles, n_colors=None, precision="fp32", seed=0, cell_factor=0.0,
                 use_graph=True, record_fields=False, device=None, skin=0.0, list_capacity=0):
        import torch
        self._torch = torch
        self.lib = B.load()
        if not torch.cuda.is_available():
            raise SphError(3, "no CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = torch.cuda.Stream(device=self.device)
        self.dim = int(problem.dim)
        self.n = int(n_particles)
        ncol = int(n_colors if n_colors is not None else getattr(problem, "n_colors", 1))
        self.n_colors = ncol
        dom, fld, par = problem_structs(problem, precision, seed, cell_factor, use_graph, record_fields, skin,
                                        list_capacity)
        dev, stream = self.device, self.stream

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            except Exception:  # out of memory -> NULL -> SPH_ERR_OOM
                return None

        def _free(ptr, nbytes, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._cb = (B.ALLOC_FN(_alloc), B.FREE_FN(_free))
        al = B.sph_alloc(self._cb[0], self._cb[1], None)
        h = B.H()
        bg = background_struct(getattr(problem, "bg", None))
        with torch.cuda.device(self.device):
            if bg is None:
                st = self.lib.sph_create(C.byref(dom), C.byref(fld), self.n, ncol, C.byref(par), C.byref(al),
                                         C.c_void_p(stream.cuda_stream), C.byref(h))
            else:
                st = self.lib.sph_create_background(C.byref(dom), C.byref(fld), C.byref(bg[0]), self.n, ncol,
                                                    C.byref(par), C.byref(al), C.c_void_p(stream.cuda_stream),
                                                    C.byref(h))
        if st != B.SPH_OK:
            raise SphError(st, "sph_create failed (details on stderr)")
        self.h = h
        t0 = getattr(problem, "t0", -1.0)
        if t0 is not None and t0 >= 0:
            self.ramp_surface_tension(int(t0), int(problem.t1))

    # ------------------------------------------------------------------ util
    def _check(self, st):
        if st != B.SPH_OK:
            raise SphError(st, self.lib.sph_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.sph_destroy(self.h)
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

    # ------------------------------------------------------------------- API
    def set_state(self, pos, col):
        torch = self._torch
        if isinstance(pos, torch.Tensor) and pos.is_cuda:
            pos = pos.to(torch.float64).contiguous()
            col = col.to(torch.uint8).contiguous()
            self._check(self.lib.sph_set_state(self.h, pos.data_ptr(), col.data_ptr(), 1))
            return
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        col = np.ascontiguousarray(col, dtype=np.uint8)
        assert pos.shape == (self.n, self.dim) and col.shape == (self.n,)
        self._check(self.lib.sph_set_state(self.h, pos.ctypes.data, col.ctypes.data, 0))

    def step(self, n=1):
        self._check(self.lib.sph_step(self.h, int(n)))

    def step_profiled(self, n=1):
        """n steps with per-phase CUDA-event timing: (cells_ms, pass_a_ms, pass_b_ms) summed."""
        ms = (C.c_float * 3)()
        self._check(self.lib.sph_step_profiled(self.h, int(n), ms))
        return tuple(float(v) for v in ms)

    def set_surface(self, flags):
        """Mark feature-surface particles (bool per particle id; None clears)."""
        import numpy as np
        if flags is None:
            self._check(self.lib.sph_set_surface(self.h, None))
            return
        f = np.ascontiguousarray(np.asarray(flags, dtype=bool).astype(np.uint8))
        assert f.shape == (self.n,)
        self._check(self.lib.sph_set_surface(self.h, f.ctypes.data))

    def ramp_surface_tension(self, t0, t1):
        self._check(self.lib.sph_ramp_surface_tension(self.h, int(t0), int(t1)))

    def auto_ramp(self, window=50, tol=1e-3, theta=0.15):
        """Start the ramp when the partition has converged (sph_auto_ramp)."""
        self._check(self.lib.sph_auto_ramp(self.h, int(window), float(tol), float(theta)))

    def positions(self, out=None):
        """(n, dim) float64 in particle-id order: numpy, or into a CUDA tensor `out`."""
        if out is not None:
            self._check(self.lib.sph_get_positions(self.h, out.data_ptr(), 1))
            return out
        x = np.empty((self.n, self.dim), np.float64)
        self._check(self.lib.sph_get_positions(self.h, x.ctypes.data, 0))
        return x

    GRAD_NAMES = ("sigma0", "gamma", "P0") + tuple(f"poly{m}" for m in range(8))

    def backward(self, n_steps, lam=1.0, frozen_dt=False, ckpt_every=5, seed=None, dt=None, density_weight=1.0,
                 out=None):
        """Sensitivities of L (density_weight * density error + lam * interface
        energy) after n_steps steps from the current state; the handle ends at
        the final state.
        seed: optional (n, dim) dL/dx_K of an outer loss; dt: optional (n_steps, 2)
        prescribed step sizes (implies frozen_dt). out: optional CUDA float64
        (n, dim) tensor that receives dpos0 on the device (then seed and dt
        must be CUDA tensors too, or None). Returns dict(L, dpos0 (n, dim),
        grads {name: value}, dt (n_steps, 2))."""
        obj = B.sph_objective(float(density_weight), float(lam), 1 if (frozen_dt or dt is not None) else 0,
                              int(ckpt_every))
        g = B.sph_grad()
        if out is not None:
            torch = self._torch
            dt_dev = getattr(self, "_dt_dev", None)
            if dt_dev is None or dt_dev.shape[0] != max(int(n_steps), 0) or dt_dev.device != out.device:
                dt_dev = torch.zeros((max(int(n_steps), 0), 2), dtype=torch.float64, device=out.device)
                self._dt_dev = dt_dev
            self._check(self.lib.sph_backward(self.h, int(n_steps), C.byref(obj),
                                              None if seed is None else seed.data_ptr(),
                                              None if dt is None else dt.data_ptr(),
                                              dt_dev.data_ptr(), out.data_ptr(), 1, C.byref(g)))
            grads = dict(zip(self.GRAD_NAMES, [g.d_sigma0, g.d_gamma, g.d_P0] + list(g.d_poly)))
            return dict(L=g.L, dpos0=out, grads=grads, dt=dt_dev)
        dpos = np.zeros((self.n, self.dim), np.float64)
        dt_out = np.zeros((max(int(n_steps), 0), 2), np.float64)
        sd = None if seed is None else np.ascontiguousarray(seed, dtype=np.float64)
        di = None if dt is None else np.ascontiguousarray(dt, dtype=np.float64)
        self._check(self.lib.sph_backward(self.h, int(n_steps), C.byref(obj),
                                          None if sd is None else sd.ctypes.data,
                                          None if di is None else di.ctypes.data,
                                          dt_out.ctypes.data, dpos.ctypes.data, 0, C.byref(g)))
        grads = dict(zip(self.GRAD_NAMES, [g.d_sigma0, g.d_gamma, g.d_P0] + list(g.d_poly)))
        return dict(L=g.L, dpos0=dpos, grads=grads, dt=dt_out)

    def colors(self):
        c = np.empty(self.n, np.uint8)
        self._check(self.lib.sph_get_colors(self.h, c.ctypes.data, 0))
        return c

    def stats(self):
        s = B.sph_stats()
        self._check(self.lib.sph_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    def field(self, which):
        k = {"rho": B.SPH_OUT_RHO, "acc": B.SPH_OUT_ACC, "visc": B.SPH_OUT_VISC}[which]
        out = np.empty(self.n if k == B.SPH_OUT_RHO else (self.n, self.dim), np.float64)
        self._check(self.lib.sph_get_field(self.h, k, out.ctypes.data, 0))
        return out

    def neighbor_sets(self):
        n = self.n
        dc = np.zeros(n, np.int32); fc = np.zeros(n, np.int32)
        ds = np.zeros(n, np.int64); fs = np.zeros(n, np.int64)
        self._check(self.lib.sph_neighbor_sets(self.h, dc.ctypes.data, fc.ctypes.data, ds.ctypes.data,
                                               fs.ctypes.data))
        return dict(dens_count=dc, force_count=fc, dens_idsum=ds, force_idsum=fs)

    def set_tuning(self, pass_threads=0, cell_factor=0.0, stage_views=-1):
        """Launch configuration (sph_set_tuning); 0 (stage_views: -1) keeps a value."""
        self._check(self.lib.sph_set_tuning(self.h, int(pass_threads), float(cell_factor), int(stage_views)))

    def tuning(self):
        t, c, s = C.c_int32(), C.c_double(), C.c_int32()
        self._check(self.lib.sph_get_tuning(self.h, C.byref(t), C.byref(c), C.byref(s)))
        return dict(pass_threads=t.value, cell_factor=c.value, stage_views=s.value)

    def stage_info(self):
        """Blocks of 256 particles, how many the last list rebuild staged, and
        the neighbour views they stage (sph_get_stage_info)."""
        b, sb, sv = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.sph_get_stage_info(self.h, C.byref(b), C.byref(sb), C.byref(sv)))
        return dict(blocks=b.value, staged_blocks=sb.value, staged_views=sv.value)

    def color_volumes(self):
        """Per colour: sum of m/rho over its particles (the sub-domain's
        volume, FP64 on the device) and its particle count, from the last step."""
        v = np.zeros(self.n_colors, np.float64)
        k = np.zeros(self.n_colors, np.int64)
        self._check(self.lib.sph_get_color_volumes(self.h, v.ctypes.data, k.ctypes.data))
        return v, k

    def cell_list(self):
        k = np.zeros(self.n, np.uint32); s = np.zeros(self.n, np.uint32)
        self._check(self.lib.sph_get_cell_list(self.h, k.ctypes.data, s.ctypes.data))
        return k, s

    def grid(self):
        g = B.sph_grid_info()
        self._check(self.lib.sph_get_grid(self.h, C.byref(g)))
        L = g.n_levels
        return dict(n_levels=L, dim=g.dim, lo=list(g.lo), h0=g.h0, lip_h=g.lip_h,
                    cell=[g.cell[l] for l in range(L)], dims=[list(g.dims[l]) for l in range(L)],
                    base=[g.base[l] for l in range(L + 1)])

    def sync(self):
        self._check(self.lib.sph_sync(self.h))

    def save(self) -> bytes:
        n = C.c_size_t(0)
        self._check(self.lib.sph_save(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.sph_save(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self.lib.sph_load(self.h, buf, len(blob)))

    def info(self):
        n = C.c_int64(); d = C.c_int32(); rs = C.c_double()
        self._check(self.lib.sph_get_info(self.h, C.byref(n), C.byref(d), C.byref(rs)))
        return dict(n=n.value, dim=d.value, rho_scale=rs.value)


def relax_fn(problem, colors, n_steps, precision="fp32", lam=1.0, density_weight=1.0, frozen_dt=False,
             ckpt_every=5, **handle_kw):
    """K relaxation steps and the objective as a differentiable function:

        f(x0, sigma0, gamma, P0, poly) -> (x_K, L)

    x0: CUDA float64 (n, dim) initial positions (colours `colors` fixed);
    sigma0, gamma, P0: scalar tensors (Eqs. sph_st_sigma, EOS_current); poly:
    (8,) tensor, the coefficients of the target density's polynomial factor
    (Eq. rho_target_function; rho_scale is held at problem.rho_scale, which
    must be > 0). x_K: the positions after n_steps steps; L = density_weight
    * sum_i (rho_i/rho_t,i - 1)^2 + lam * sum_{i<j, C_i != C_j} W(r_ij,
    kappa h_ij) at x_K. Backward is one sph_backward call: the incoming dL/dx_K
    is its seed (kept on the device), the incoming dL/dL scales the objective
    weights, and it returns the gradients of all five inputs. A library handle
    is created for each distinct parameter value and reused while the values
    stay the same."""
    import torch

    col = torch.as_tensor(np.ascontiguousarray(colors, dtype=np.uint8))
    state = {"key": None, "r": None}
    if not (problem.rho_scale > 0):
        raise ValueError("relax_fn needs problem.rho_scale > 0 (held fixed)")

    def handle(values):
        key = tuple(float(v) for v in values)
        if state["key"] != key:
            if state["r"] is not None:
                state["r"].close()
            q = problem.copy(sigma0=key[0], gamma=key[1], P0=key[2], poly=list(key[3:]))
            state["r"] = Relaxation(q, len(col), int(col.max()) + 1, precision=precision, **handle_kw)
            state["key"] = key
        return state["r"]

    def values(sigma0, gamma, P0, poly):
        return [float(sigma0), float(gamma), float(P0)] + [float(v) for v in poly.detach().reshape(-1).tolist()]

    class _Relax(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x0, sigma0, gamma, P0, poly):
            r = handle(values(sigma0, gamma, P0, poly))
            c = col.to(x0.device)
            xs = x0.detach().to(torch.float64).contiguous()
            ctx.save_for_backward(xs, c, sigma0, gamma, P0, poly)
            r.set_state(xs, c)
            r.step(n_steps)
            out = torch.empty_like(xs)
            r.positions(out=out)
            torch.cuda.current_stream().wait_stream(r.stream)
            # L at x_K: a zero-step reverse pass evaluates the objective
            g = r.backward(0, lam=lam, density_weight=density_weight, ckpt_every=1,
                           out=torch.empty_like(xs))
            L = torch.tensor(g["L"], dtype=torch.float64, device=x0.device)
            return out, L

        @staticmethod
        def backward(ctx, g_x, g_L):
            xs, c, sigma0, gamma, P0, poly = ctx.saved_tensors
            r = handle(values(sigma0, gamma, P0, poly))
            r.set_state(xs, c)
            seed = None if g_x is None else g_x.detach().to(torch.float64).contiguous()
            wL = 0.0 if g_L is None else float(g_L)
            dpos = torch.empty_like(xs)
            res = r.backward(n_steps, lam=lam * wL, density_weight=density_weight * wL, frozen_dt=frozen_dt,
                             ckpt_every=ckpt_every, seed=seed, out=dpos)
            torch.cuda.current_stream().wait_stream(r.stream)
            gr = res["grads"]

            def like(t, v):
                return torch.as_tensor(v, dtype=t.dtype, device=t.device).reshape(t.shape)

            dpoly = like(poly, [gr[f"poly{m}"] for m in range(8)][:poly.numel()])
            return dpos, like(sigma0, gr["sigma0"]), like(gamma, gr["gamma"]), like(P0, gr["P0"]), dpoly

    def f(x0, sigma0, gamma, P0, poly):
        return _Relax.apply(x0, sigma0, gamma, P0, poly)

    return f


class Batch:
    """Independent instances stepped together by one CUDA graph per step
    (include/sphmesh.h, sph_batch_*). problems: list of problem descriptions
    (as for Relaxation), each with n_particles / n_colors attributes or given
    in the parallel lists. n_branches = 0: tune with tune() (or 16 by default)."""

    def __init__(self, problems, n_particles, n_colors, precision="fp32", seeds=None, n_branches=0, device=None):
        import torch
        self._torch = torch
        self.lib = B.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = torch.cuda.Stream(device=self.device)
        k = len(problems)
        descs = (B.sph_instance_desc * k)()
        self.dims, self.ns = [], []
        for i, p in enumerate(problems):
            d, f, q = problem_structs(p, precision, 0 if seeds is None else int(seeds[i]), use_graph=False)
            descs[i].dom, descs[i].field, descs[i].params = d, f, q
            descs[i].n_particles = int(n_particles[i])
            descs[i].n_colors = int(n_colors[i])
            self.dims.append(int(p.dim))
            self.ns.append(int(n_particles[i]))
        dev, stream = self.device, self.stream

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            except Exception:
                return None

        def _free(ptr, nbytes, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._cb = (B.ALLOC_FN(_alloc), B.FREE_FN(_free))
        al = B.sph_alloc(self._cb[0], self._cb[1], None)
        h = B.H()
        with torch.cuda.device(self.device):
            st = self.lib.sph_batch_create(descs, k, C.byref(al), C.c_void_p(stream.cuda_stream), int(n_branches),
                                           C.byref(h))
        if st != B.SPH_OK:
            raise SphError(st, "sph_batch_create failed (details on stderr)")
        self.b = h
        self.n_inst = k

    def _check(self, st):
        if st != B.SPH_OK:
            raise SphError(st, self.lib.sph_batch_last_error(self.b).decode())

    def tune(self, candidates=(1, 4, 8, 16, 32, 64, 128), steps_each=2):
        """Autotune the branch count, then the launch configuration (threads
        per block of the pair passes, cell factor); returns dict(chosen,
        trials, n_inst, n_branches)."""
        arr = (C.c_int32 * len(candidates))(*candidates)
        self._check(self.lib.sph_batch_tune(self.b, arr, len(candidates), int(steps_each)))
        return self.info()

    def info(self):
        ni, nb, nt = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self.lib.sph_batch_info(self.b, C.byref(ni), C.byref(nb), C.byref(nt), None, None))
        chosen = B.sph_batch_trial()
        cap = max(nt.value, 1)
        trials = (B.sph_batch_trial * cap)()
        n = C.c_int32()
        self._check(self.lib.sph_batch_tuning(self.b, C.byref(chosen), trials, cap, C.byref(n)))
        return dict(n_inst=ni.value, n_branches=nb.value, chosen=chosen.as_dict(),
                    trials=[trials[i].as_dict() for i in range(min(n.value, cap))])

    def step(self, n=1):
        self._check(self.lib.sph_batch_step(self.b, int(n)))

    def step_each(self, n=1):
        self._check(self.lib.sph_batch_step_each(self.b, int(n)))

    def sync(self):
        self._check(self.lib.sph_batch_sync(self.b))

    def _h(self, k):
        h = B.H()
        self._check(self.lib.sph_batch_get(self.b, int(k), C.byref(h)))
        return h

    def positions(self, k):
        x = np.empty((self.ns[k], self.dims[k]), np.float64)
        h = self._h(k)
        st = self.lib.sph_get_positions(h, x.ctypes.data, 0)
        if st != B.SPH_OK:
            raise SphError(st, self.lib.sph_last_error(h).decode())
        return x

    def colors(self, k):
        c = np.empty(self.ns[k], np.uint8)
        h = self._h(k)
        st = self.lib.sph_get_colors(h, c.ctypes.data, 0)
        if st != B.SPH_OK:
            raise SphError(st, self.lib.sph_last_error(h).decode())
        return c

    def set_state(self, k, pos, col):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        col = np.ascontiguousarray(col, dtype=np.uint8)
        h = self._h(k)
        st = self.lib.sph_set_state(h, pos.ctypes.data, col.ctypes.data, 0)
        if st != B.SPH_OK:
            raise SphError(st, self.lib.sph_last_error(h).decode())

    def stats(self, k):
        s = B.sph_stats()
        h = self._h(k)
        st = self.lib.sph_get_stats(h, C.byref(s))
        if st != B.SPH_OK:
            raise SphError(st, self.lib.sph_last_error(h).decode())
        return s.as_dict()

    def close(self):
        if getattr(self, "b", None):
            self.lib.sph_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Seeded synthetic inputs for the multi-phase SPH relaxation (arXiv 1906.07925).

This module is shared by the oracle's tests and by the GPU path's tests and bench.
It describes geometry (a level set built from a box and spheres, Sec. 3.1), the
user-given target spacing shape s(x) that the target density is built from
(Sec. 2.3, Eq. rho_target_function), and draws particle states:

* a jittered lattice coloured by the nearest of a few seeds;
* density-proportional rejection sampling (particles ~ s(x)^-d inside the
  positive phase), coloured by the nearest Voronoi generator (the
  initialisation of the square case, Sec. 4.2).

It holds none of the relaxation arithmetic (kernel, EOS, forces, time step,
projection). Both sides receive the same numbers from here and do their own
computation. All randomness is numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SPHERE = 0
BOX = 1
GRID = 2  # the level set sampled on the problem's background mesh (Problem.bg.phi)

FIELD_UNIFORM = 0
FIELD_LINEAR_DISTANCE = 1
FIELD_TANH_DISTANCE = 2  # s = a + b tanh(s0 |dist|), s0 a reciprocal length
FIELD_BACKGROUND = 3  # s sampled on the problem's background mesh (Problem.bg.spacing)


@dataclasses.dataclass
class Background:
    """Cartesian background mesh: node (i, j, k) at lo + (i, j, k) (hi - lo) /
    (dims - 1); phi (level set, positive in the region) and spacing are arrays
    of shape dims indexed [i, j, k] (dims[2] = 1 in 2D), either may be None."""

    dims: Sequence[int]
    lo: Sequence[float]
    hi: Sequence[float]
    phi: Optional[np.ndarray] = None
    spacing: Optional[np.ndarray] = None


def bg_interp(bg: Background, v: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Multilinear interpolation of node values v at points x (n, d), x clamped
    into the mesh box (input shaping only: the sampler's density envelope)."""
    n, d = x.shape
    vv = np.asarray(v, dtype=np.float64).reshape(tuple(bg.dims[:d]) if d == 3 else (bg.dims[0], bg.dims[1]))
    i0 = np.zeros((n, d), dtype=np.int64)
    f = np.zeros((n, d))
    for k in range(d):
        m = int(bg.dims[k])
        h = (bg.hi[k] - bg.lo[k]) / (m - 1)
        t = np.clip((x[:, k] - bg.lo[k]) / h, 0.0, m - 1)
        i = np.minimum(np.floor(t).astype(np.int64), m - 2)
        i0[:, k] = i
        f[:, k] = t - i
    out = np.zeros(n)
    for c in range(1 << d):
        w = np.ones(n)
        idx = []
        for k in range(d):
            b = (c >> k) & 1
            idx.append(i0[:, k] + b)
            w *= f[:, k] if b else 1.0 - f[:, k]
        out += w * vv[tuple(idx)]
    return out


@dataclasses.dataclass
class Shape:
    """One level-set constraint: a sphere (size[0] = radius) or an axis box
    (size = half extents). keep_inside=True keeps the region inside it."""

    kind: int
    keep_inside: bool
    center: Sequence[float]
    size: Sequence[float]


@dataclasses.dataclass
class Problem:
    """Geometry, target field and parameters of one relaxation instance.

    Field: rho_t(x) = rho_scale * s(x)^-d * (1 + sum_k poly[k] * b_k(x~)),
    with s = s0 (uniform) or s = a + b * dist(x, shapes[dist_shape]).
    h = tau * rho_t^(-1/d) (unit mass, Eq. scale_SPH_particle); support = kappa*h.
    """

    dim: int
    lo: Sequence[float]
    hi: Sequence[float]
    shapes: List[Shape] = dataclasses.field(default_factory=list)
    field_kind: int = FIELD_UNIFORM
    s0: float = 1.0
    a: float = 0.0
    b: float = 0.0
    dist_shape: int = 0
    poly: List[float] = dataclasses.field(default_factory=list)
    rho_scale: float = 1.0
    P0: float = 1.0
    gamma: float = 2.0
    sigma0: float = 3.0
    tau: float = 2.0
    kappa: float = 1.0
    n_colors: int = 1
    t0: float = -1.0  # surface-tension ramp start (steps); < 0: no ramp
    t1: float = -1.0
    eos_general: bool = False  # use p/rho^2 even at gamma = 2 (identity checks)
    bg: Optional[Background] = None  # background mesh for GRID shapes / FIELD_BACKGROUND
    surface: Optional[np.ndarray] = None  # per particle: feature-surface particle (Sec. 3.5)

    def copy(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------
# geometry helpers used only to shape the inputs
# ----------------------------------------------------------------------------

def _shape_signed(shape: Shape, x: np.ndarray, bg: Optional[Background] = None) -> np.ndarray:
    """Signed distance, positive inside the shape (x: (n, d))."""
    d = x.shape[1]
    if shape.kind == GRID:
        return bg_interp(bg, bg.phi, x)
    c = np.asarray(shape.center[:d], dtype=np.float64)
    if shape.kind == SPHERE:
        return shape.size[0] - np.linalg.norm(x - c, axis=1)
    half = np.asarray(shape.size[:d], dtype=np.float64)
    q = np.abs(x - c) - half
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=1)
    inside = np.minimum(np.max(q, axis=1), 0.0)
    return -(outside + inside)


def inside_mask(p: Problem, x: np.ndarray) -> np.ndarray:
    """True where x lies in the positive phase (inside the box, and inside /
    outside each shape as requested)."""
    d = p.dim
    lo = np.asarray(p.lo[:d]); hi = np.asarray(p.hi[:d])
    m = np.all((x >= lo) & (x <= hi), axis=1)
    for s in p.shapes:
        v = _shape_signed(s, x, p.bg)
        m &= (v > 0) if s.keep_inside else (v < 0)
    return m


def spacing_shape(p: Problem, x: np.ndarray) -> np.ndarray:
    """The user-given spacing shape s(x) times the polynomial modulation
    factor, returned as the un-normalised density weight s^-d (1 + P)."""
    d = p.dim
    if p.field_kind == FIELD_UNIFORM:
        s = np.full(x.shape[0], p.s0)
    elif p.field_kind == FIELD_BACKGROUND:
        s = bg_interp(p.bg, p.bg.spacing, x)
    else:
        dist = np.abs(_shape_signed(p.shapes[p.dist_shape], x, p.bg))
        s = p.a + p.b * (np.tanh(p.s0 * dist) if p.field_kind == FIELD_TANH_DISTANCE else dist)
    w = s ** (-d)
    if p.poly:
        w = w * (1.0 + poly_value(p, x))
    return w


def poly_basis(p: Problem, x: np.ndarray) -> np.ndarray:
    """The 8 monomials of the target-density modulation on x~ = 2(x-lo)/(hi-lo)-1.
    2D: x, y, x^2, xy, y^2, x^3, x^2 y, x y^2.  3D: x, y, z, x^2, y^2, z^2, xy, yz."""
    d = p.dim
    lo = np.asarray(p.lo[:d]); hi = np.asarray(p.hi[:d])
    t = 2.0 * (x - lo) / (hi - lo) - 1.0
    if d == 2:
        X, Y = t[:, 0], t[:, 1]
        return np.stack([X, Y, X * X, X * Y, Y * Y, X ** 3, X * X * Y, X * Y * Y], axis=1)
    X, Y, Z = t[:, 0], t[:, 1], t[:, 2]
    return np.stack([X, Y, Z, X * X, Y * Y, Z * Z, X * Y, Y * Z], axis=1)


def poly_value(p: Problem, x: np.ndarray) -> np.ndarray:
    c = np.zeros(8)
    c[: len(p.poly)] = p.poly
    return poly_basis(p, x) @ c


def rho_scale_for(p: Problem, n: int, res: int = 0) -> float:
    """A value of rho_scale that makes the expected particle count about n
    (midpoint rule of s^-d (1+P) over the positive phase). Any positive value
    is a valid input; this one only keeps the inputs shaped like the paper's
    unit-mass bookkeeping (Sec. 3.2: N = total mass)."""
    d = p.dim
    if res <= 0:
        res = 2048 if d == 2 else 160
    lo = np.asarray(p.lo[:d], dtype=np.float64); hi = np.asarray(p.hi[:d], dtype=np.float64)
    step = (hi - lo) / res
    axes = [lo[k] + (np.arange(res) + 0.5) * step[k] for k in range(d)]
    total = 0.0
    # slab by slab along the last axis to bound memory
    for z in axes[-1]:
        grids = np.meshgrid(*axes[:-1], indexing="ij")
        pts = np.stack([g.ravel() for g in grids] + [np.full(grids[0].size, z)], axis=1)
        m = inside_mask(p, pts)
        total += float(np.sum(spacing_shape(p, pts[m])))
    total *= float(np.prod(step))
    return n / total


# ----------------------------------------------------------------------------
# particle states
# ----------------------------------------------------------------------------

def nearest_color(x: np.ndarray, gens: np.ndarray) -> np.ndarray:
    """Index of the nearest generator, as uint8."""
    if x.shape[0] > 200000:
        from scipy.spatial import cKDTree
        return cKDTree(gens).query(x)[1].astype(np.uint8)
    best = np.full(x.shape[0], np.inf)
    col = np.zeros(x.shape[0], dtype=np.int64)
    for k in range(gens.shape[0]):
        d2 = np.sum((x - gens[k]) ** 2, axis=1)
        better = d2 < best
        best[better] = d2[better]
        col[better] = k
    return col.astype(np.uint8)


def uniform_in_domain(p: Problem, n: int, rng: np.random.Generator) -> np.ndarray:
    d = p.dim
    lo = np.asarray(p.lo[:d]); hi = np.asarray(p.hi[:d])
    out = np.empty((0, d))
    while out.shape[0] < n:
        c = lo + (hi - lo) * rng.random((max(2 * n, 64), d))
        out = np.concatenate([out, c[inside_mask(p, c)]], axis=0)
    return out[:n]


def sample_density(p: Problem, n: int, seed: int, gens: Optional[np.ndarray] = None):
    """n particles drawn with probability ~ s(x)^-d (1+P) in the positive
    phase; coloured by the nearest of p.n_colors generators that are drawn
    uniformly in the positive phase (Voronoi initialisation, Sec. 4.2).
    Returns (pos (n,d) float64, colors (n,) uint8, generators)."""
    rng = np.random.default_rng(seed)
    d = p.dim
    lo = np.asarray(p.lo[:d]); hi = np.asarray(p.hi[:d])
    if gens is None:
        gens = uniform_in_domain(p, p.n_colors, rng)
    # envelope: max weight from a dense probe, padded
    probe = uniform_in_domain(p, 20000, rng)
    wmax = float(np.max(spacing_shape(p, probe))) * 1.5
    for s in p.shapes:  # the densest region may be a thin shell at a shape surface
        if p.field_kind in (FIELD_LINEAR_DISTANCE, FIELD_TANH_DISTANCE):
            wmax = max(wmax, (p.a ** (-d)) * (1.0 + sum(abs(c) for c in p.poly)) * 1.01)
    if p.field_kind == FIELD_BACKGROUND:  # multilinear interpolation stays within the node values
        wmax = max(wmax, float(np.min(p.bg.spacing)) ** (-d) * (1.0 + sum(abs(c) for c in p.poly)) * 1.01)
    chunks = []
    have = 0
    while have < n:
        m = max(4 * (n - have), 4096)
        c = lo + (hi - lo) * rng.random((m, d))
        u = rng.random(m)
        ok = inside_mask(p, c)
        c = c[ok]; u = u[ok]
        w = spacing_shape(p, c)
        acc = u * wmax < w
        c = c[acc]
        chunks.append(c)
        have += c.shape[0]
    pos = np.concatenate(chunks, axis=0)[:n]
    return pos, nearest_color(pos, gens), gens


def lattice_jitter_2d(p: Problem, nx: int, jitter: float, seed: int):
    """nx*nx lattice of the box at spacing (hi-lo)/nx, cell-centred, plus
    uniform jitter in [-jitter*s, jitter*s] per axis; coloured by the nearest of
    one uniform seed per quadrant. Returns (pos, colors, seeds)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(p.lo[:2]); hi = np.asarray(p.hi[:2])
    s = (hi - lo) / nx
    ii, jj = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
    pos = lo + (np.stack([ii.ravel(), jj.ravel()], axis=1) + 0.5) * s
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) * s
    mid = 0.5 * (lo + hi)
    seeds = []
    for qx in range(2):
        for qy in range(2):
            a = np.array([lo[0] if qx == 0 else mid[0], lo[1] if qy == 0 else mid[1]])
            b = np.array([mid[0] if qx == 0 else hi[0], mid[1] if qy == 0 else hi[1]])
            seeds.append(a + (b - a) * rng.random(2))
    seeds = np.array(seeds)
    return pos, nearest_color(pos, seeds), seeds


def lattice(p: Problem, nper: int, margin_cells: int = 0):
    """Perfect cell-centred lattice of nper points per axis over the box."""
    d = p.dim
    lo = np.asarray(p.lo[:d]); hi = np.asarray(p.hi[:d])
    s = (hi - lo) / nper
    idx = np.stack(np.meshgrid(*[np.arange(nper)] * d, indexing="ij"), axis=-1).reshape(-1, d)
    return lo + (idx + 0.5) * s


# ----------------------------------------------------------------------------
# the workloads (shapes and sizes of the paper's benchmark cases)
# ----------------------------------------------------------------------------

def uniform_square_2d(n_side: int = 64, n_colors: int = 4) -> Problem:
    """[0,1]^2, uniform spacing 1/n_side, smoothing length 2 x spacing."""
    s = 1.0 / n_side
    return Problem(dim=2, lo=[0, 0, 0], hi=[1, 1, 0], field_kind=FIELD_UNIFORM, s0=s,
                   rho_scale=1.0, n_colors=n_colors)


def graded_hole_2d(n: int = 1 << 20, n_colors: int = 64, rho_scale: Optional[float] = None) -> Problem:
    """[0,1]^2 minus a disk r=0.2 at the centre; spacing shape
    s = 0.002 + 0.02 dist(x, circle), normalised to about n particles."""
    p = Problem(dim=2, lo=[0, 0, 0], hi=[1, 1, 0],
                shapes=[Shape(SPHERE, False, [0.5, 0.5, 0.0], [0.2, 0, 0])],
                field_kind=FIELD_LINEAR_DISTANCE, a=0.002, b=0.02, dist_shape=0,
                n_colors=n_colors)
    p.rho_scale = rho_scale if rho_scale is not None else rho_scale_for(p, n)
    return p


def graded_inclusion_3d(n: int = 1 << 23, n_colors: int = 256, rho_scale: Optional[float] = None) -> Problem:
    """[0,1]^3 minus a ball r=0.25 at the centre; s = 0.004 + 0.03 dist(x, sphere),
    normalised to about n particles."""
    p = Problem(dim=3, lo=[0, 0, 0], hi=[1, 1, 1],
                shapes=[Shape(SPHERE, False, [0.5, 0.5, 0.5], [0.25, 0, 0])],
                field_kind=FIELD_LINEAR_DISTANCE, a=0.004, b=0.03, dist_shape=0,
                n_colors=n_colors)
    p.rho_scale = rho_scale if rho_scale is not None else rho_scale_for(p, n)
    return p


def circle_2d(n: int = 4289, n_colors: int = 6, h_min: float = 0.391, h_max: float = 3.125,
              rho_scale: Optional[float] = None) -> Problem:
    """The circle of Sec. 4.1: the disk of radius 43 at (50, 50) in
    [0, 100]^2, target size h_min + tanh(2.5 phi / 43) / tanh(2.5) (h_max - h_min)
    with phi the distance to the circle (defaults: the circle_6mpi case, 4,289
    particles, one colour per MPI task of the paper's run)."""
    p = Problem(dim=2, lo=[0, 0, 0], hi=[100, 100, 0],
                shapes=[Shape(SPHERE, True, [50.0, 50.0, 0.0], [43.0, 0, 0])],
                field_kind=FIELD_TANH_DISTANCE, a=h_min, b=(h_max - h_min) / math.tanh(2.5), s0=2.5 / 43.0,
                dist_shape=0, n_colors=n_colors)
    p.rho_scale = rho_scale if rho_scale is not None else rho_scale_for(p, n)
    return p


def circle_with_surface(n_volume: int = 4289, n_colors: int = 6, seed: int = 1, h_min: float = 0.391,
                        h_max: float = 3.125, surface_spacing: float = 1.0):
    """The circle case with feature-surface particles (Sec. 3.5): n_surface
    particles evenly spaced (with a small jitter) on the circle at the target
    spacing there, then n_volume density-proportional particles inside.
    Returns (problem with .surface set, positions, colours); surface particles
    come first and take the colour of the nearest volume generator."""
    p = circle_2d(n_volume, n_colors, h_min=h_min, h_max=h_max)
    vol, col, gens = sample_density(p, n_volume, seed)
    # target spacing on the circle (s = h_min there), times surface_spacing
    spacing = surface_spacing * h_min * p.rho_scale ** -0.5
    n_surface = int(round(2 * math.pi * 43.0 / spacing))
    rng = np.random.default_rng(seed + 7)
    ang = (np.arange(n_surface) + rng.uniform(-0.2, 0.2, n_surface)) * (2 * math.pi / n_surface)
    ring = np.stack([50.0 + 43.0 * np.cos(ang), 50.0 + 43.0 * np.sin(ang)], axis=1)
    pos = np.concatenate([ring, vol])
    colors = np.concatenate([nearest_color(ring, gens), col]).astype(np.uint8)
    surface = np.zeros(len(pos), dtype=bool)
    surface[:n_surface] = True
    return p.copy(surface=surface), pos, colors


def circle_2d_background(n: int = 4289, n_colors: int = 6, h_min: float = 0.391, h_max: float = 3.125,
                         nodes: int = 101, rho_scale: Optional[float] = None) -> Problem:
    """The circle case of Sec. 4.1 given as the paper's method takes geometry in
    (Sec. 3.1, 3.2): the level set 43 - |x - (50, 50)| and the target size
    sampled on a Cartesian background mesh of nodes x nodes points over
    [0, 100]^2, interpolated at the particle positions."""
    t = np.linspace(0.0, 100.0, nodes)
    X, Y = np.meshgrid(t, t, indexing="ij")
    phi = 43.0 - np.hypot(X - 50.0, Y - 50.0)
    size = h_min + np.tanh(2.5 * np.abs(phi) / 43.0) / math.tanh(2.5) * (h_max - h_min)
    bg = Background(dims=[nodes, nodes, 1], lo=[0.0, 0.0, 0.0], hi=[100.0, 100.0, 0.0],
                    phi=phi[:, :, None], spacing=size[:, :, None])
    p = Problem(dim=2, lo=[0, 0, 0], hi=[100, 100, 0], shapes=[Shape(GRID, True, [0.0, 0.0, 0.0], [1.0, 0, 0])],
                field_kind=FIELD_BACKGROUND, n_colors=n_colors, bg=bg)
    p.rho_scale = rho_scale if rho_scale is not None else rho_scale_for(p, n)
    return p


def adjoint_poly_2d(n: int = 1 << 18, n_colors: int = 32, seed: int = 3) -> Problem:
    """The graded-hole field with an 8-coefficient polynomial modulation of the
    target density, coefficients U(-0.05, 0.05) from `seed`."""
    rng = np.random.default_rng(seed)
    p = graded_hole_2d(n, n_colors, rho_scale=1.0)
    p.poly = list(rng.uniform(-0.05, 0.05, size=8))
    p.rho_scale = rho_scale_for(p, n)
    return p


def batch_instances(n_inst: int = 512, seed: int = 4, n_lo: int = 2000, n_hi: int = 200000):
    """Independent instances: half 2D, half 3D; particle counts log-uniform in
    [n_lo, n_hi]; 2..64 colours; a random sphere or box domain inside the unit
    box and a linear spacing grading from a random point's sphere."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_inst):
        dim = 2 if k < n_inst // 2 else 3
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        ncol = int(rng.integers(2, 65))
        lo = [0.0, 0.0, 0.0]
        hi = [1.0, 1.0, 1.0 if dim == 3 else 0.0]
        c = list(rng.uniform(0.4, 0.6, size=3))
        if dim == 2:
            c[2] = 0.0
        if rng.random() < 0.5:
            dom = Shape(SPHERE, True, c, [float(rng.uniform(0.3, 0.4)), 0, 0])
        else:
            dom = Shape(BOX, True, c, list(rng.uniform(0.25, 0.35, size=3)))
        b = float(rng.uniform(0.005, 0.03))
        p = Problem(dim=dim, lo=lo, hi=hi, shapes=[dom], field_kind=FIELD_LINEAR_DISTANCE,
                    a=0.01, b=b, dist_shape=0, n_colors=ncol)
        out.append((p, n))
    return out

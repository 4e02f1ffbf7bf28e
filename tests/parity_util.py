"""Helpers shared by the GPU parity tests: run one step on both sides from the
same seeded input and compare with tolerances stated here.

Tolerances (per-step, identical input state): density relative `tol`; the
force a_i within `tol` of S_i = sum_j |pair term| (the sums cancel, so a
relative bound on a_i itself is meaningless); a~ and the displacement are
downstream of a, so their bound carries the relative error of a,
eps_i = tol * S_i / |a_i|, maximised over the neighbourhood.
tol = 1e-5 for the FP32 split-precision path, 1e-12 for FP64.

One FP32 widening (check_force): a pair near the support edge carries its
kernel factor (1 - q)^3 with a relative error of about 3 q / (1 - q) times the
rounding of q (of r and of the FP32 h, which enter 1 - q unreduced), so a
particle whose force sum such a pair dominates is held to
tol S + 8 ulp S max_j 3 q_j / (1 - q_j); such particles must be rare.
"""
import numpy as np
from scipy.spatial import cKDTree

import oracle

TOL = {"fp32": 1e-5, "fp64": 1e-12}


def oracle_rho_scale(p, n, res=None):
    """rho_scale that makes the problem's field integrate to n particles (Eq.
    total_mass_2 with unit mass), by the oracle's quadrature: the value both
    sides are given when the GPU would otherwise choose it itself."""
    res = res or (2048 if p.dim == 2 else 192)
    return n / oracle.total_mass(p.copy(rho_scale=1.0), res)


def make_gpu(p, pos, col, precision, **kw):
    from paper_1906_07925_gb300 import Relaxation
    r = Relaxation(p, n_particles=len(pos), n_colors=int(col.max()) + 1, precision=precision,
                   record_fields=True, use_graph=kw.pop("use_graph", False), **kw)
    r.set_state(pos, col)
    return r


def h_all(p, pos):
    return np.array([oracle.h_of(p, x) for x in pos])


def local_max(p, pos, h, v):
    """max of v over each particle's neighbourhood (r < kappa max h)."""
    tree = cKDTree(pos)
    R = p.kappa * h.max() * 1.01
    out = np.empty_like(v)
    for i, nb in enumerate(tree.query_ball_point(pos, R)):
        out[i] = v[nb].max()
    return out


def edge_amplification(p, x, idx, tree=None):
    """max over the force pairs of each particle in idx of 3 q / (1 - q),
    q = r / (kappa (h_i + h_j) / 2), from the oracle's h."""
    tree = tree or cKDTree(x)
    out = np.zeros(len(idx))
    for t, i in enumerate(idx):
        hi = oracle.h_of(p, x[i])
        nb = np.array([j for j in tree.query_ball_point(x[i], 2.0 * p.kappa * hi) if j != i], dtype=np.int64)
        if len(nb) == 0:
            continue
        hj = np.array([oracle.h_of(p, x[j]) for j in nb])
        q = np.linalg.norm(x[nb] - x[i], axis=1) / (0.5 * p.kappa * (hi + hj))
        q = q[q < 1.0]
        if len(q):
            out[t] = (3 * q / (1 - q)).max()
    return out


def check_force(p, x, acc, f, precision, tree=None):
    """Force of every particle against the oracle's; returns the relative
    error bound of each a_i (tol, or the widened FP32 bound) for the checks
    downstream of a."""
    tol = TOL[precision]
    n = len(x)
    Sa = f["pair_abs_a"]
    ea = np.abs(acc - f["acc"]).max(axis=1)
    over = np.nonzero(ea > tol * Sa + 1e-300)[0]
    rel_a = np.full(n, tol)
    if precision == "fp64" or len(over) == 0:
        assert len(over) == 0, ("acc", (ea[over] / Sa[over]).max(), int(over[0]))
        return rel_a
    assert len(over) <= max(3, 1e-4 * n), ("acc: too many particles over tol", len(over))
    amp = edge_amplification(p, x, over, tree)
    extra = 8 * 2.0 ** -23 * amp
    bound = (tol + extra) * Sa[over]
    assert (ea[over] <= bound).all(), ("acc", (ea[over] / bound).max())
    rel_a[over] += extra
    return rel_a


def compare_step(p, pos, col, precision, step_index=0, gpu=None):
    """One step on both sides; assert parity; return (gpu, oracle outputs)."""
    tol = TOL[precision]
    r = gpu or make_gpu(p, pos, col, precision)
    r.step(1)
    st = r.stats()
    g = dict(rho=r.field("rho"), acc=r.field("acc"), visc=r.field("visc"), x=r.positions())
    xo, info, f = oracle.step(p, pos, col, step_index)
    n = len(pos)
    # density
    rel = np.abs(g["rho"] - f["rho"]) / f["rho"]
    assert rel.max() <= tol, ("rho", rel.max(), int(rel.argmax()))
    # force a_n, normalised by the sum of pair magnitudes
    Sa = f["pair_abs_a"]
    rel_a = check_force(p, pos, g["acc"], f, precision)
    # time steps: relative error of a at the argmin particle
    an = np.linalg.norm(f["acc"], axis=1)
    cond = np.where(an > 0, Sa / np.maximum(an, 1e-300), 1.0)
    h = h_all(p, pos)
    rc = p.kappa * h
    m = np.where(an > 0, rc / np.maximum(an, 1e-300), np.inf)
    k = int(np.argmin(m))
    dt_tol = 2 * rel_a[k] * (1 + cond[k])
    assert abs(st["dt1"] - info["dt1"]) <= dt_tol * info["dt1"], ("dt1", st["dt1"], info["dt1"])
    assert abs(st["dt2"] - info["dt2"]) <= dt_tol * info["dt2"], ("dt2", st["dt2"], info["dt2"])
    # a~: error carried from a (eps over the neighbourhood), factor 4 for the
    # harmonic-mean coefficient's own dependence on |a|
    eps = local_max(p, pos, h, rel_a * (1 + cond))
    ev = np.abs(g["visc"] - f["visc"]).max(axis=1)
    bound_v = 4 * (eps + dt_tol) * f["pair_abs_b"] + 1e-300
    assert (ev <= bound_v).all(), ("visc", (ev / bound_v).max())
    # displacement
    dg = g["x"] - pos
    do = xo - pos
    dn = np.linalg.norm(do, axis=1)
    ed = np.abs(dg - do).max(axis=1)
    scale = np.abs(pos).max() + 1.0
    rep = (6e-8 if precision == "fp32" else 1e-15) * (scale if precision == "fp32" else scale)
    # representation: FP32 offsets are relative to cells (the rounding of the
    # input positions and of projected points is at most a few ulp of x)
    bound_d = 4 * (eps + 2 * dt_tol) * (dn + 0.5 * info["dt1"] * info["dt2"] * Sa) + 4 * rep
    assert (ed <= bound_d).all(), ("disp", (ed / bound_d).max(), int(np.argmax(ed / bound_d)))
    # integer statistics
    assert st["force_pairs"] == info["force_pairs"] or precision == "fp32"
    return r, dict(info=info, f=f, x=xo, gpu=g, stats=st)


def near_edge_particles(p, pos, rel=1e-5):
    """Particles with any pair within `rel` of a support edge (density or force
    criterion): their FP32 neighbour sets may legitimately differ."""
    h = h_all(p, pos)
    tree = cKDTree(pos)
    R = p.kappa * h.max() * 1.01
    bad = np.zeros(len(pos), bool)
    for i, nb in enumerate(tree.query_ball_point(pos, R)):
        nb = np.asarray(nb)
        r = np.linalg.norm(pos[nb] - pos[i], axis=1)
        Hd = p.kappa * h[i]
        Hf = p.kappa * 0.5 * (h[i] + h[nb])
        if np.any(np.abs(r - Hd) <= rel * Hd) or np.any(np.abs(r - Hf) <= rel * Hf):
            bad[i] = True
    # a particle next to an ambiguous pair sees it too
    return bad

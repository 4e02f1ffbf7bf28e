"""Pins of the oracle's hand-written reverse pass (orc_backward).

The reverse pass is checked against central finite differences of the
oracle's own forward run (which the other pins tie to the paper), for every
parameter and for sampled initial coordinates, in both step-size modes:
prescribed ("frozen") step sizes, and step sizes recomputed from the state.
A second pin is exact: under recomputed step sizes the trajectory does not
depend on P0 at all (a ~ P0, dt1 ~ P0^-1/2, dt2 = 0.8 dt1, so every
displacement term is P0-free), so dL/dP0 must vanish, while under frozen step
sizes it must not.
"""
import copy

import numpy as np
import pytest

import workloads as W

FD_REL = 1e-4  # central differences with step 1e-4 (parameters) / 1e-7 (coordinates)


def _poly_2d(n=260, seed=5):
    """The adjoint workload's field at small n; the coefficients are scaled up
    (x4) so that the polynomial's spatial gradient weighs in the checks."""
    p = W.adjoint_poly_2d(n=n, n_colors=5, seed=3)
    p.poly = [4.0 * c for c in p.poly]
    p.rho_scale = W.rho_scale_for(p, n)
    pos, col, _ = W.sample_density(p, n, seed=seed)
    return p, pos, col


def _general_3d(n=300, seed=7):
    """3D, general EOS (gamma = 1.7), an active surface-tension ramp, a
    polynomial factor, and a box hole on top of the ball hole; six particles
    start inside the box hole, so the first step projects them out through its
    faces (all three projection kinds are in play)."""
    p = W.graded_inclusion_3d(n=n, n_colors=4)
    p.gamma = 1.7
    p.eos_general = True
    p.t0, p.t1 = 0, 4
    p.poly = [0.03, -0.02, 0.01, 0.02, -0.01, 0.015, -0.02, 0.01]
    p.shapes.append(W.Shape(W.BOX, False, [0.2, 0.2, 0.2], [0.08, 0.08, 0.08]))
    p.rho_scale = W.rho_scale_for(p, n)
    pos, col, _ = W.sample_density(p, n, seed=seed)
    inner = 0.2 + np.random.default_rng(seed).uniform(-0.06, 0.06, size=(6, 3))
    pos[:6] = inner
    return p, pos, col


def _tanh_2d(n=260, seed=5):
    """The circle case's tanh-graded field (Sec. 4.1) on the unit square (the
    circle of radius 0.43 at the centre), with a polynomial factor: the field's
    spatial gradient, largest at the circle, enters the reverse pass."""
    p = W.Problem(dim=2, lo=[0, 0, 0], hi=[1, 1, 0], shapes=[W.Shape(W.SPHERE, True, [0.5, 0.5, 0.0], [0.43, 0, 0])],
                  field_kind=W.FIELD_TANH_DISTANCE, a=0.0391, b=(0.3125 - 0.0391) / np.tanh(2.5), s0=2.5 / 0.43,
                  dist_shape=0, n_colors=5)
    p.poly = [0.05, -0.04, 0.03, 0.02, -0.03, 0.01, 0.02, -0.01]
    p.rho_scale = W.rho_scale_for(p, n)
    pos, col, _ = W.sample_density(p, n, seed=seed)
    return p, pos, col


def _loss(orc, p, x, col, K, lam, dt, seed):
    xe = orc.run(p, x, col, K)[0] if dt is None else orc.run_fixed_dt(p, x, col, dt)
    L = orc.objective(p, xe, col, lam)
    if seed is not None:
        L += float((seed * xe).sum())
    return L


def _perturbed(p, name, eps):
    q = copy.deepcopy(p)
    if name.startswith("poly"):
        q.poly = list(p.poly)
        q.poly[int(name[4:])] += eps
    else:
        setattr(q, name, getattr(p, name) + eps)
    return q


def _check(orc, p, pos, col, K, lam, frozen, seed=None, n_coords=10):
    dt = orc.backward(p, pos, col, K, lam)["dt"] if frozen else None
    r = orc.backward(p, pos, col, K, lam, dt=dt, seed=seed)
    # L reports the objective alone (the seed only enters the gradient)
    xe = orc.run(p, pos, col, K)[0] if dt is None else orc.run_fixed_dt(p, pos, col, dt)
    assert np.isclose(r["L"], orc.objective(p, xe, col, lam), rtol=1e-12)
    gvals = np.array([r["grads"][k] for k in orc.GRAD_NAMES])
    scale = np.abs(gvals).max()
    for name in orc.GRAD_NAMES:
        if name == "P0" and not frozen:
            continue  # exactly zero; pinned separately
        if name.startswith("poly") and int(name[4:]) >= len(p.poly):
            assert r["grads"][name] == 0.0
            continue
        eps = 1e-4 * max(abs(getattr(p, name)), 1.0) if not name.startswith("poly") else 1e-4
        fd = (_loss(orc, _perturbed(p, name, eps), pos, col, K, lam, dt, seed)
              - _loss(orc, _perturbed(p, name, -eps), pos, col, K, lam, dt, seed)) / (2 * eps)
        assert abs(r["grads"][name] - fd) <= FD_REL * max(abs(fd), 1e-3 * scale), (name, r["grads"][name], fd)
    rng = np.random.default_rng(11)
    gscale = np.abs(r["dpos0"]).max()
    for t in range(n_coords):
        i, k = (t, t % pos.shape[1]) if t < 3 else (int(rng.integers(pos.shape[0])), int(rng.integers(pos.shape[1])))
        h = 1e-7
        x1, x2 = pos.copy(), pos.copy()
        x1[i, k] += h
        x2[i, k] -= h
        fd = (_loss(orc, p, x1, col, K, lam, dt, seed) - _loss(orc, p, x2, col, K, lam, dt, seed)) / (2 * h)
        assert abs(r["dpos0"][i, k] - fd) <= FD_REL * max(abs(fd), 1e-3 * gscale), (i, k, r["dpos0"][i, k], fd)
    return r


@pytest.mark.parametrize("frozen", [True, False])
def test_adjoint_matches_fd_2d(orc, frozen):
    p, pos, col = _poly_2d()
    _check(orc, p, pos, col, K=3, lam=1.0, frozen=frozen)


@pytest.mark.parametrize("frozen", [True, False])
def test_adjoint_matches_fd_3d_general_eos_seeded(orc, frozen):
    p, pos, col = _general_3d()
    seed = np.random.default_rng(2).normal(size=pos.shape)
    _check(orc, p, pos, col, K=2, lam=0.5, frozen=frozen, seed=seed)


def test_adjoint_P0_invariance(orc):
    """Recomputed step sizes make the trajectory P0-free (bit-identical under
    P0 -> 4 P0, where every scale factor is a power of two), so dL/dP0 = 0;
    with frozen step sizes P0 scales the displacements and dL/dP0 != 0."""
    p, pos, col = _poly_2d()
    K, lam = 3, 1.0
    x1 = orc.run(p, pos, col, K)[0]
    q = copy.deepcopy(p)
    q.P0 = 4.0 * p.P0
    x4 = orc.run(q, pos, col, K)[0]
    assert np.array_equal(x1, x4)
    ra = orc.backward(p, pos, col, K, lam)
    scale = max(abs(v) for v in ra["grads"].values())
    assert abs(ra["grads"]["P0"]) <= 1e-12 * scale
    rf = orc.backward(p, pos, col, K, lam, dt=ra["dt"])
    assert abs(rf["grads"]["P0"]) > 1e-3 * scale
    # the frozen run with the recorded sizes is the same trajectory
    assert np.allclose(orc.run_fixed_dt(p, pos, col, ra["dt"]), x1, rtol=0, atol=1e-15)


def test_adjoint_zero_steps_is_objective_gradient(orc):
    """K = 0: dpos0 is dL/dx of the objective alone (checked by differences)."""
    p, pos, col = _poly_2d(n=200)
    r = orc.backward(p, pos, col, 0, 1.0)
    assert r["dt"].shape == (0, 2)
    rng = np.random.default_rng(3)
    for _ in range(6):
        i, k = int(rng.integers(pos.shape[0])), int(rng.integers(2))
        h = 1e-7
        x1, x2 = pos.copy(), pos.copy()
        x1[i, k] += h
        x2[i, k] -= h
        fd = (orc.objective(p, x1, col, 1.0) - orc.objective(p, x2, col, 1.0)) / (2 * h)
        assert abs(r["dpos0"][i, k] - fd) <= FD_REL * max(abs(fd), 1e-3 * np.abs(r["dpos0"]).max())


@pytest.mark.parametrize("frozen", [True, False])
def test_adjoint_matches_fd_tanh_field(orc, frozen):
    p, pos, col = _tanh_2d()
    _check(orc, p, pos, col, K=3, lam=1.0, frozen=frozen)

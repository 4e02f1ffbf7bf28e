"""GPU reverse pass (sph_backward) vs the oracle's hand-written one.

Both sides start from the same seeded state. With frozen step sizes the GPU
is given the oracle's recorded sizes, so both differentiate the same map;
with recomputed sizes each side chooses its own (equal up to rounding).

Tolerances (relative to the largest component of the compared gradient):
FP64 1e-9 (the two sides differ only in summation order and the integer
state's rounding, amplified over a few steps); FP32 1e-4, the bound the
reverse pass is specified to (measured on GB300: at most 6e-7 for the
parameters and 5e-7 for the positions, here and on the 262,144-particle,
20-step workload).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import make_gpu

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-4}


def poly2d(n=3000, seed=5):
    p = W.adjoint_poly_2d(n=n, n_colors=8, seed=3)
    pos, col, _ = W.sample_density(p, n, seed=seed)
    return p, pos, col


def general3d(n=3000, seed=7):
    p = W.graded_inclusion_3d(n=n, n_colors=6)
    p.gamma = 1.7
    p.eos_general = True
    p.t0, p.t1 = 0, 4
    p.poly = [0.03, -0.02, 0.01, 0.02, -0.01, 0.015, -0.02, 0.01]
    p.shapes.append(W.Shape(W.BOX, False, [0.2, 0.2, 0.2], [0.08, 0.08, 0.08]))
    p.rho_scale = W.rho_scale_for(p, n)
    pos, col, _ = W.sample_density(p, n, seed=seed)
    pos[:6] = 0.2 + np.random.default_rng(seed).uniform(-0.06, 0.06, size=(6, 3))
    return p, pos, col


def _compare(g, o, tol):
    gd, od = g["dpos0"], o["dpos0"]
    scale = np.abs(od).max()
    err = np.abs(gd - od).max()
    assert err <= tol * scale, f"dpos0: max err {err:.3e} vs scale {scale:.3e}"
    pv = np.array([o["grads"][k] for k in oracle.GRAD_NAMES])
    ps = np.abs(pv).max()
    for k in oracle.GRAD_NAMES:
        assert abs(g["grads"][k] - o["grads"][k]) <= tol * ps, (k, g["grads"][k], o["grads"][k], ps)
    assert abs(g["L"] - o["L"]) <= tol * abs(o["L"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("frozen", [True, False])
def test_backward_matches_oracle_2d(precision, frozen):
    p, pos, col = poly2d()
    K, lam = 3, 1.0
    o = oracle.backward(p, pos, col, K, lam)
    dt = o["dt"] if frozen else None
    if frozen:
        o = oracle.backward(p, pos, col, K, lam, dt=dt)
    r = make_gpu(p, pos, col, precision)
    g = r.backward(K, lam=lam, frozen_dt=frozen, ckpt_every=2, dt=dt)
    _compare(g, o, TOL[precision])
    if not frozen:
        # both sides chose (nearly) the same step sizes
        assert np.allclose(g["dt"], o["dt"], rtol=1e-5 if precision == "fp32" else 1e-11)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("frozen", [True, False])
def test_backward_matches_oracle_3d_general_eos(precision, frozen):
    p, pos, col = general3d()
    K, lam = 2, 0.5
    seed = np.random.default_rng(2).normal(size=pos.shape)
    o = oracle.backward(p, pos, col, K, lam)
    dt = o["dt"] if frozen else None
    o = oracle.backward(p, pos, col, K, lam, dt=dt, seed=seed)
    r = make_gpu(p, pos, col, precision)
    g = r.backward(K, lam=lam, frozen_dt=frozen, ckpt_every=1, dt=dt, seed=seed)
    _compare(g, o, TOL[precision])


def test_backward_checkpoint_interval_and_end_state():
    """Every checkpoint interval gives the same gradient (the recomputed steps
    repeat the forward run exactly), and the handle ends at x_K."""
    p, pos, col = poly2d(n=2000)
    K = 5
    res = []
    for c in (1, 2, 5, 7):
        r = make_gpu(p, pos, col, "fp64")
        res.append(r.backward(K, lam=1.0, frozen_dt=False, ckpt_every=c))
        xk = r.positions()
        r2 = make_gpu(p, pos, col, "fp64")
        r2.step(K)
        # x_K comes back through FP64 positions (a round trip of the integer state)
        assert np.abs(xk - r2.positions()).max() <= 1e-14
        assert r.stats()["step"] == K
    for q in res[1:]:
        assert np.allclose(q["dpos0"], res[0]["dpos0"], rtol=0, atol=1e-12 * np.abs(res[0]["dpos0"]).max())
        for k in oracle.GRAD_NAMES:
            assert abs(q["grads"][k] - res[0]["grads"][k]) <= 1e-12 * max(abs(v) for v in res[0]["grads"].values())


def test_backward_seed_alone_is_linear():
    """With both objective weights 0 the reverse pass propagates the seed
    alone: equal to the oracle's gradient with the seed minus without it."""
    p, pos, col = poly2d(n=2000)
    K = 3
    seed = np.random.default_rng(4).normal(size=pos.shape)
    o1 = oracle.backward(p, pos, col, K, 1.0, seed=seed)
    o0 = oracle.backward(p, pos, col, K, 1.0)
    r = make_gpu(p, pos, col, "fp64")
    g = r.backward(K, lam=0.0, density_weight=0.0, seed=seed, ckpt_every=3)
    ref = o1["dpos0"] - o0["dpos0"]
    assert g["L"] == 0.0
    assert np.abs(g["dpos0"] - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_backward_P0_free_with_recomputed_steps(precision):
    """Recomputed step sizes make the run independent of P0: dL/dP0 vanishes
    (to rounding) while the other components do not."""
    p, pos, col = poly2d(n=4000)
    r = make_gpu(p, pos, col, precision)
    g = r.backward(4, lam=1.0, frozen_dt=False, ckpt_every=2)
    scale = max(abs(v) for v in g["grads"].values())
    assert abs(g["grads"]["P0"]) <= (1e-10 if precision == "fp64" else 1e-3) * scale
    gf = make_gpu(p, pos, col, precision).backward(4, lam=1.0, frozen_dt=True, ckpt_every=2)
    assert abs(gf["grads"]["P0"]) > 1e-2 * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_backward_full_size_adjoint_workload(precision):
    """The polynomial-field workload at its full size (262,144 particles, 32
    colours, 20 steps, checkpoint every 5, recomputed step sizes) against the
    oracle's reverse pass from the same seeded state: every position and
    parameter component, and the step sizes; the handle ends at the state 20
    plain steps reach."""
    n = 1 << 18
    p = W.adjoint_poly_2d(n=n, n_colors=32, seed=3)
    pos, col, _ = W.sample_density(p, n, seed=3)
    o = oracle.backward(p, pos, col, 20, 1.0)
    r = make_gpu(p, pos, col, precision, use_graph=True)
    g = r.backward(20, lam=1.0, frozen_dt=False, ckpt_every=5)
    _compare(g, o, TOL[precision])
    assert np.allclose(g["dt"], o["dt"], rtol=1e-5 if precision == "fp32" else 1e-11)
    xk = r.positions()
    r.close()
    r2 = make_gpu(p, pos, col, precision, use_graph=True)
    r2.step(20)
    assert np.abs(xk - r2.positions()).max() <= (1e-6 if precision == "fp32" else 1e-14)
    r2.close()


def test_autograd_function_gradients_match_differences():
    """relax_fn as a torch.autograd.Function of (x0, sigma0, gamma, P0, poly):
    the gradient of w . x_K + 0.5 L against central differences of the same
    GPU forward run (FP64, recomputed step sizes), for every parameter and
    sampled coordinates; and the position gradient of w . x_K alone equals the
    oracle's seeded reverse pass."""
    import torch
    from paper_1906_07925_gb300 import relax_fn
    p, pos, col = poly2d(n=1500)
    K = 3
    f = relax_fn(p, col, K, precision="fp64", lam=0.7, density_weight=1.0, frozen_dt=False, ckpt_every=2,
                 use_graph=False)
    rng = np.random.default_rng(9)
    w = torch.tensor(rng.normal(size=pos.shape), dtype=torch.float64, device="cuda")
    base = dict(sigma0=p.sigma0, gamma=p.gamma, P0=p.P0, poly=list(p.poly))

    def args(v, grad=False):
        x0 = torch.tensor(v["x0"], dtype=torch.float64, device="cuda", requires_grad=grad)
        sc = [torch.tensor(v[k], dtype=torch.float64, requires_grad=grad) for k in ("sigma0", "gamma", "P0")]
        poly = torch.tensor(v["poly"], dtype=torch.float64, requires_grad=grad)
        return [x0] + sc + [poly]

    def loss(v, grad=False):
        a = args(v, grad)
        xk, L = f(*a)
        return (w * xk).sum() + 0.5 * L, a

    v0 = dict(base, x0=pos)
    l0, a = loss(v0, grad=True)
    l0.backward()
    g = {"sigma0": float(a[1].grad), "gamma": float(a[2].grad), "P0": float(a[3].grad)}
    for m in range(8):
        g[f"poly{m}"] = float(a[4].grad[m])
    scale = max(abs(x) for x in g.values())
    for name in g:
        eps = 1e-4
        vp, vm = dict(v0), dict(v0)
        if name.startswith("poly"):
            m = int(name[4:])
            vp["poly"] = list(v0["poly"]); vp["poly"][m] += eps
            vm["poly"] = list(v0["poly"]); vm["poly"][m] -= eps
        else:
            vp[name] = v0[name] + eps
            vm[name] = v0[name] - eps
        fd = (float(loss(vp)[0]) - float(loss(vm)[0])) / (2 * eps)
        assert abs(g[name] - fd) <= 1e-4 * max(abs(fd), 1e-3 * scale), (name, g[name], fd)
    gx = a[0].grad.cpu().numpy()
    gs = np.abs(gx).max()
    for t in range(6):
        i, k = int(rng.integers(len(pos))), int(rng.integers(2))
        h = 1e-7
        xp, xm = pos.copy(), pos.copy()
        xp[i, k] += h
        xm[i, k] -= h
        fd = (float(loss(dict(v0, x0=xp))[0]) - float(loss(dict(v0, x0=xm))[0])) / (2 * h)
        assert abs(gx[i, k] - fd) <= 1e-4 * max(abs(fd), 1e-3 * gs), (i, k, gx[i, k], fd)
    # the seed alone (w . x_K) against the oracle's reverse pass
    a = args(v0, grad=True)
    xk, _ = f(*a)
    (w * xk).sum().backward()
    wn = w.cpu().numpy()
    ref = oracle.backward(p, pos, col, K, 1.0, seed=wn)["dpos0"] - oracle.backward(p, pos, col, K, 1.0)["dpos0"]
    assert np.abs(a[0].grad.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()

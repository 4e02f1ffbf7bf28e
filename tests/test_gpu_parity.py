"""GPU path vs the FP64 oracle, element by element, on seeded inputs.

Sizes span several thread blocks and cell rows with ragged tails; the graded
cases exercise several grid levels. Tolerances are stated in parity_util.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import TOL, compare_step, h_all, make_gpu, near_edge_particles, oracle_rho_scale

pytestmark = pytest.mark.gpu


def c1_state():
    p = W.uniform_square_2d(64, 4)
    pos, col, _ = W.lattice_jitter_2d(p, 64, 0.3, 0)
    return p, pos, col


def circle_state(n=4289, seed=1, ncol=6):
    """The circle_6mpi case of Sec. 4.1 (tanh-graded target size)."""
    p = W.circle_2d(n, ncol)
    pos, col, _ = W.sample_density(p, n, seed)
    return p, pos, col


def circle_bg_state(n=4289, seed=1, ncol=6):
    """The circle case given on a 101 x 101 background mesh (Sec. 3.1, 3.2)."""
    p = W.circle_2d_background(n, ncol)
    pos, col, _ = W.sample_density(p, n, seed)
    return p, pos, col


def graded2d_state(n=20000, seed=1, ncol=16):
    p = W.graded_hole_2d(n, ncol)
    pos, col, _ = W.sample_density(p, n, seed)
    return p, pos, col


def graded3d_state(n=30000, seed=2, ncol=32):
    p = W.graded_inclusion_3d(n, ncol)
    pos, col, _ = W.sample_density(p, n, seed)
    return p, pos, col


# ------------------------------------------------------------ neighbours ----

@pytest.mark.parametrize("case", ["c1", "g2", "g3", "circle", "circle_bg"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_neighbor_sets_match_oracle(case, precision):
    p, pos, col = {"c1": c1_state, "g2": graded2d_state, "g3": graded3d_state, "circle": circle_state,
                   "circle_bg": circle_bg_state}[case]()
    r = make_gpu(p, pos, col, precision)
    got = r.neighbor_sets()
    want = oracle.neighbor_sets(p, pos, 1)
    keep = np.ones(len(pos), bool)
    if precision == "fp32":
        keep = ~near_edge_particles(p, pos)
    assert keep.mean() > 0.9
    for k in ("dens_count", "force_count", "dens_idsum", "force_idsum"):
        assert np.array_equal(got[k][keep], want[k][keep]), k
    if precision == "fp64":
        assert all(np.array_equal(got[k], want[k]) for k in got)
    r.close()


def test_grid_has_several_levels_on_graded_fields():
    p, pos, col = graded3d_state(8000)
    r = make_gpu(p, pos, col, "fp32")
    assert r.grid()["n_levels"] >= 3
    r.close()


# ---------------------------------------------------------------- one step ----

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_parity_uniform_square(precision):
    p, pos, col = c1_state()
    r, out = compare_step(p, pos, col, precision)
    assert out["stats"]["interface_pairs"] == out["info"]["interface_pairs"] or precision == "fp32"
    r.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_parity_graded_2d(precision):
    p, pos, col = graded2d_state()
    r, out = compare_step(p, pos, col, precision)
    assert out["info"]["wall_moved"] > 0  # the hole and the box walls were exercised
    r.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_parity_graded_3d(precision):
    p, pos, col = graded3d_state()
    r, _ = compare_step(p, pos, col, precision)
    r.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_parity_general_gamma_and_poly_field(precision):
    p = W.adjoint_poly_2d(12000, 8)
    p.gamma = 1.4
    pos, col, _ = W.sample_density(p, 12000, 3)
    r, _ = compare_step(p, pos, col, precision)
    r.close()


def test_step_parity_box_and_sphere_domains():
    for k, (p, n) in enumerate(W.batch_instances(6, seed=4, n_lo=3000, n_hi=9000)):
        p.rho_scale = W.rho_scale_for(p, n, res=512 if p.dim == 2 else 96)
        pos, col, _ = W.sample_density(p, n, 10 + k)
        r, _ = compare_step(p, pos, col, "fp64")
        r.close()


def test_ramp_schedule():
    """Steps 0..6 with a ramp over (2, 5]: the sigma each step used matches
    Eq. sph_st_sigma as the oracle evaluates it."""
    p, pos, col = c1_state()
    p = p.copy(t0=2, t1=5)
    r = make_gpu(p, pos, col, "fp64")
    r.ramp_surface_tension(2, 5)
    for s in range(7):
        r.step(1)
        assert r.stats()["sigma"] == pytest.approx(oracle.sigma(p, s), abs=1e-15)
    r.close()


def test_ramped_step_parity():
    """A step taken inside the ramp (sigma = 2) agrees with the oracle."""
    p, pos, col = graded2d_state(8000)
    q = p.copy(t0=0, t1=3)  # step 1 of this schedule uses sigma = 3 (1 - 1/3) = 2
    r = make_gpu(q, pos, col, "fp32")
    # the checkpoint's documented header: 8 int64 then the ramp window
    hdr_t = np.dtype([("magic", "<i8"), ("version", "<i8"), ("n", "<i8"), ("dim", "<i8"), ("step", "<i8"),
                      ("zero", "<i8", 3), ("t0", "<f8"), ("t1", "<f8")])
    blob = bytearray(r.save())
    hdr = np.frombuffer(bytes(blob[:hdr_t.itemsize]), dtype=hdr_t).copy()
    assert hdr["n"][0] == len(pos) and hdr["dim"][0] == 2 and hdr["step"][0] == 0
    hdr["step"] = 1
    blob[:hdr_t.itemsize] = hdr.tobytes()
    r.load(bytes(blob))
    assert r.stats()["step"] == 1
    assert oracle.sigma(q, 1) == pytest.approx(2.0)
    r2, out = compare_step(q, pos, col, "fp32", step_index=1, gpu=r)
    assert out["stats"]["sigma"] == pytest.approx(2.0)
    r.close()


# --------------------------------------------------------- many steps ----

def test_relaxation_trajectory_fp64_stays_close():
    """FP64 path over 20 steps of the 4,096-particle square: trajectories of two
    correct implementations separate only through rounding, so positions agree
    to a small fraction of the spacing."""
    p, pos, col = c1_state()
    r = make_gpu(p, pos, col, "fp64")
    r.step(20)
    xg = r.positions()
    xo, infos = oracle.run(p, pos, col, 20)
    assert np.abs(xg - xo).max() < 1e-6 * (1 / 64)
    assert r.stats()["err_l2"] == pytest.approx(infos[-1]["err_l2"], rel=1e-6)
    r.close()


def test_relaxation_end_state_statistics_fp32():
    """100 steps of the square case: FP32 split vs the FP64 oracle end states
    compared statistically (density error, interface pairs)."""
    p, pos, col = c1_state()
    r = make_gpu(p, pos, col, "fp32", use_graph=True)
    r.step(100)
    st = r.stats()
    xo, infos = oracle.run(p, pos, col, 100)
    io = infos[-1]
    assert st["err_l2"] == pytest.approx(io["err_l2"], rel=0.05)
    assert abs(st["interface_pairs"] - io["interface_pairs"]) <= 0.05 * io["interface_pairs"] + 5
    assert st["err_l2"] < 0.5 * oracle.step(p, pos, col, 0)[1]["err_l2"]  # it relaxed
    r.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_end_state_triangle_quality_matches_oracle(precision):
    """A random start in the square (4,096 particles) relaxed for 100 steps on
    the GPU and in the oracle: the Delaunay triangulations of the two end
    states have the same quality (Sec. 4's G and angle measures). The
    trajectories separate through rounding, so the measures are compared as
    statistics of the point sets, not triangle by triangle."""
    import mesh_quality as MQ
    p = W.uniform_square_2d(64, 4)
    pos, col, _ = W.sample_density(p, 4096, 1)
    r = make_gpu(p, pos, col, precision, use_graph=True)
    r.step(100)
    qg = MQ.quality(r.positions(), r.colors())
    xo, _ = oracle.run(p, pos, col, 100)
    qo = MQ.quality(xo, col)
    r.close()
    assert qg["G_avg"] == pytest.approx(qo["G_avg"], abs=0.01)
    assert qg["theta_min_mean"] == pytest.approx(qo["theta_min_mean"], abs=0.75)
    assert qg["share_55_65"] == pytest.approx(qo["share_55_65"], abs=0.02)
    assert qg["theta_min"] > 15.0 and qg["theta_max"] < 140.0
    assert abs(qg["n_lt30"] - qo["n_lt30"]) <= 0.5 * qo["n_lt30"] + 10
    assert abs(qg["n_tri"] - qo["n_tri"]) <= 0.01 * qo["n_tri"]
    # communication volume of the colour partition, N_eg / N_et
    assert qg["n_eg"] / qg["n_et"] == pytest.approx(qo["n_eg"] / qo["n_et"], rel=0.05)


# ------------------------------------------------------ circle case (Sec. 4.1) ----

@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_step_parity_circle(precision):
    p, pos, col = circle_state()
    compare_step(p, pos, col, precision)


def test_circle_relaxed_quality_matches_oracle():
    """circle_6mpi relaxed for 2,000 steps with the surface tension ramped down
    over steps 1,000-1,200, on the GPU (FP32) and in the oracle: the Delaunay
    meshes of the two end states have the same quality and communication
    volume (Sec. 4 measures), compared as statistics of the point sets."""
    import mesh_quality as MQ
    p, pos, col = circle_state()
    p.t0, p.t1 = 1000, 1200
    r = make_gpu(p, pos, col, "fp32", use_graph=True)
    r.ramp_surface_tension(1000, 1200)
    r.step(2000)
    qg = MQ.quality(r.positions(), r.colors(), max_edge_factor=None, drop_hull=False)
    r.close()
    xo, _ = oracle.run(p, pos, col, 2000)
    qo = MQ.quality(xo, col, max_edge_factor=None, drop_hull=False)
    assert qg["G_avg"] == pytest.approx(qo["G_avg"], abs=0.01)
    assert qg["theta_min_mean"] == pytest.approx(qo["theta_min_mean"], abs=1.0)
    assert abs(qg["n_tri"] - qo["n_tri"]) <= 0.01 * qo["n_tri"]
    assert qg["n_eg"] / qg["n_et"] == pytest.approx(qo["n_eg"] / qo["n_et"], rel=0.25)
    assert abs(qg["n_lt30"] - qo["n_lt30"]) <= 0.5 * qo["n_lt30"] + 10


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_step_parity_background_mesh(precision):
    """Level set and target spacing interpolated from a background mesh, a
    few particles projected back onto the interpolated level set."""
    p, pos, col = circle_bg_state()
    pos = pos.copy()
    pos[:5] = [[50.0, 93.4], [93.5, 50.0], [50.0, 6.8], [19.4, 19.4], [80.6, 80.6]]  # just outside the circle
    compare_step(p, pos, col, precision)


def test_background_mesh_relaxed_quality_matches_oracle():
    """The background-mesh circle relaxed for 1,500 steps (ramp over steps
    800-1,000) on the GPU and in the oracle: the same mesh statistics, and
    every particle inside the interpolated level set."""
    import mesh_quality as MQ
    p, pos, col = circle_bg_state()
    p.t0, p.t1 = 800, 1000
    r = make_gpu(p, pos, col, "fp32", use_graph=True)
    r.ramp_surface_tension(800, 1000)
    r.step(1500)
    xg = r.positions()
    qg = MQ.quality(xg, r.colors(), max_edge_factor=None, drop_hull=False)
    r.close()
    xo, _ = oracle.run(p, pos, col, 1500)
    qo = MQ.quality(xo, col, max_edge_factor=None, drop_hull=False)
    assert qg["G_avg"] == pytest.approx(qo["G_avg"], abs=0.01)
    assert qg["theta_min_mean"] == pytest.approx(qo["theta_min_mean"], abs=1.0)
    assert abs(qg["n_tri"] - qo["n_tri"]) <= 0.01 * qo["n_tri"]
    assert qg["n_eg"] / qg["n_et"] == pytest.approx(qo["n_eg"] / qo["n_et"], rel=0.25)
    assert min(oracle.phi(p, x) for x in xg) > -1e-4


def test_backward_refuses_background_level_set():
    from paper_1906_07925_gb300 import SphError
    p, pos, col = circle_bg_state()
    r = make_gpu(p, pos, col, "fp32")
    with pytest.raises(SphError):
        r.backward(2, lam=1.0)
    r.close()


# ---------------------------------------- feature-surface particles (Sec. 3.5) ----

@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_step_parity_surface_particles(precision):
    """The circle with feature-surface particles on its boundary: one step on
    both sides (surface particles see surface particles only, lose the normal
    force component and are projected back onto the circle)."""
    p, pos, col = W.circle_with_surface(1500, 4)
    r = make_gpu(p, pos, col, precision)
    r.set_surface(p.surface)
    compare_step(p, pos, col, precision, gpu=r)
    x = r.positions()
    s = p.surface
    assert np.abs(np.linalg.norm(x[s] - 50.0, axis=1) - 43.0).max() < (1e-5 if precision == "fp32" else 1e-12)
    r.close()


def test_surface_particles_relaxation_matches_oracle():
    """600 steps with surface particles (ramp over 300-400) on the GPU and in
    the oracle: surface particles stay on the circle and the meshes have the
    same statistics; the backward pass refuses the flagged handle."""
    import mesh_quality as MQ
    from paper_1906_07925_gb300 import SphError
    p, pos, col = W.circle_with_surface(1500, 4)
    p.t0, p.t1 = 300, 400
    r = make_gpu(p, pos, col, "fp32", use_graph=True)
    r.set_surface(p.surface)
    r.ramp_surface_tension(300, 400)
    r.step(600)
    xg = r.positions()
    with pytest.raises(SphError):
        r.backward(1, lam=1.0)
    r.close()
    xo, _ = oracle.run(p, pos, col, 600)
    s = p.surface
    for x in (xg, xo):
        assert np.abs(np.linalg.norm(x[s] - 50.0, axis=1) - 43.0).max() < 1e-5
        assert np.linalg.norm(x[~s] - 50.0, axis=1).max() <= 43.0 + 1e-5
    qg = MQ.quality(xg, col, max_edge_factor=None, drop_hull=False)
    qo = MQ.quality(xo, col, max_edge_factor=None, drop_hull=False)
    assert qg["G_avg"] == pytest.approx(qo["G_avg"], abs=0.015)
    assert qg["theta_min_mean"] == pytest.approx(qo["theta_min_mean"], abs=1.5)
    assert abs(qg["n_tri"] - qo["n_tri"]) <= 0.01 * qo["n_tri"]


def test_circle_paper_schedule():
    """circle_6mpi run as the paper runs it (Sec. 4.1): 20,000 iterations, the
    surface tension ramped down once the partition has converged (automatic
    start, Sec. 3.3). The ramp starts, and the final mesh is of high quality
    with a small communication volume. (The paper's printed measures for this
    case, with its own kernel, are G_avg 0.91, theta_min 28.2 deg, 11 angles
    below 30 deg, for context; the kernel here differs.)"""
    import mesh_quality as MQ
    p, _, _ = circle_state()
    from paper_1906_07925_gb300 import Relaxation
    r = Relaxation(p.copy(rho_scale=0.0), 4289, 6, precision="fp32", seed=1, use_graph=True)
    r.auto_ramp(window=50, tol=1e-3, theta=0.2)
    r.step(20000)
    st = r.stats()
    q = MQ.quality(r.positions(), r.colors(), max_edge_factor=None, drop_hull=False)
    r.close()
    assert 0 < st["ramp_t0"] < st["ramp_t1"] < 20000
    assert q["G_avg"] > 0.78 and q["G_min"] > 0.3
    assert q["theta_min"] > 20.0 and q["theta_max"] < 130.0
    assert q["n_lt30"] <= 0.005 * q["n_tri"]
    assert q["n_eg"] / q["n_et"] < 0.1


# ------------------------------------------------------------- edge cases ----

def test_empty_and_single_particle():
    from paper_1906_07925_gb300 import Relaxation
    p = W.uniform_square_2d(16)
    r0 = Relaxation(p, 0, 1, precision="fp32")
    r0.step(3)
    assert r0.positions().shape == (0, 2)
    r0.close()
    r1 = Relaxation(p, 1, 1, precision="fp64", record_fields=True)
    r1.set_state(np.array([[0.3, 0.4]]), np.array([0], np.uint8))
    r1.step(2)
    # positions are integers of a unit 2^-40 of the finest cell: exact to ~1e-15
    assert np.allclose(r1.positions(), [[0.3, 0.4]], rtol=0, atol=1e-13)
    st = r1.stats()
    assert st["dt1"] == 0.0 and st["force_pairs"] == 0
    r1.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_coincident_particles(precision):
    """Two particles at the same point: the pair's pressure term is 0 and its
    viscous term takes the limit of dW/(r dr), on both sides."""
    p, pos, col = c1_state()
    pos = pos.copy()
    pos[1] = pos[0]
    r, _ = compare_step(p, pos, col, precision)
    assert np.isfinite(r.positions()).all()
    r.close()


def test_ragged_sizes_and_graph_matches_direct():
    for n in (257, 1000, 4097):
        p = W.graded_hole_2d(n, 3)
        pos, col, _ = W.sample_density(p, n, 5)
        a = make_gpu(p, pos, col, "fp32", use_graph=True)
        b = make_gpu(p, pos, col, "fp32", use_graph=False)
        a.step(3); b.step(3)
        assert np.array_equal(a.positions(), b.positions())  # deterministic, same kernels
        a.close(); b.close()


def test_nonfinite_input_is_reported():
    from paper_1906_07925_gb300 import SphError
    p, pos, col = c1_state()
    pos = pos.copy(); pos[5, 0] = np.nan
    with pytest.raises(SphError) as e:
        make_gpu(p, pos, col, "fp32")
    assert e.value.status == 4


def test_save_load_roundtrip():
    p, pos, col = graded2d_state(5000)
    p = p.copy(t0=3, t1=9)
    a = make_gpu(p, pos, col, "fp32")
    a.ramp_surface_tension(3, 9)
    a.step(4)
    blob = a.save()
    b = make_gpu(p, pos, col, "fp32")
    b.load(blob)
    assert np.array_equal(a.positions(), b.positions())
    assert np.array_equal(a.colors(), b.colors())
    a.step(3); b.step(3)
    # same physical state; the restored handle sums in particle-id order, so the
    # trajectories agree to rounding, not bit for bit
    assert np.abs(a.positions() - b.positions()).max() < 1e-7
    assert a.stats()["sigma"] == b.stats()["sigma"]
    assert a.stats()["step"] == b.stats()["step"] == 7
    a.close(); b.close()


def check_cell_list(p, r, precision):
    """Cell keys and sorted order of the handle's current state against the
    oracle's definition of the multi-resolution key (oracle.cell_keys) on the
    handle's grid, and its order (by key, then particle id). Bit-exact, except
    where floating point decides the integer: a smoothing length within
    rounding of a level boundary 2^l h0 (the GPU computes h in its working
    precision) or a position within rounding of a cell face (positions cross
    the boundary as doubles). There the GPU key must be the valid alternative,
    and the order is then compared with the GPU's choice. Returns the number
    of such particles."""
    g = r.grid()
    key, order = r.cell_list()
    x = r.positions()
    want, h = oracle.cell_keys(p, x, g)
    L, d = g["n_levels"], p.dim
    band = 1e-5 if precision == "fp32" else 1e-12
    t = np.log2(h / g["h0"])
    near_level = np.abs(t - np.round(t)) < band
    base = np.array(g["base"], dtype=np.int64)
    lev_w = np.searchsorted(base[1:], want, side="right")
    lev_g = np.searchsorted(base[1:], key, side="right")
    near_face = np.zeros(len(x), bool)
    for l in set(lev_w.tolist()) | set(lev_g.tolist()):
        u = (x - np.array(g["lo"][:d])) / g["cell"][l]
        near_face |= np.any(np.abs(u - np.round(u)) < 1e-9, axis=1)
    bad = key != want
    assert not np.any(bad & ~(near_level | near_face)), np.nonzero(bad & ~(near_level | near_face))[0][:5]
    for i in np.nonzero(bad)[0]:
        lg = int(lev_g[i])
        assert abs(lg - int(lev_w[i])) <= 1
        rel = int(key[i]) - int(base[lg])
        dims = g["dims"][lg]
        c = np.array([rel % dims[0], (rel // dims[0]) % dims[1], rel // (dims[0] * dims[1])])[:d]
        u = (x[i] - np.array(g["lo"][:d])) / g["cell"][lg]
        assert np.all((u >= c - 1e-9) & (u < c + 1 + 1e-9)), i
    expect = want.copy()
    expect[bad] = key[bad]
    assert np.array_equal(order, oracle.cell_order(expect))
    return int(bad.sum())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_cell_keys_and_order_match_oracle(precision):
    """20,000 particles of the graded hole (several levels), after three steps
    (so the order before the sort is a previous cell order, not the id order)."""
    p, pos, col = graded2d_state(20000)
    r = make_gpu(p, pos, col, precision)
    assert r.grid()["n_levels"] >= 2
    check_cell_list(p, r, precision)  # from the id order set by set_state
    r.step(3)
    assert r.stats()["list_rebuilds"] >= 1
    assert check_cell_list(p, r, precision) <= (3 if precision == "fp32" else 0)
    r.close()


def test_cell_keys_and_order_match_oracle_1m():
    """The 1,048,576-particle 2D graded hole as the benchmark creates it (drawn
    on the device), after five graph-replayed steps."""
    from paper_1906_07925_gb300 import Relaxation
    n = 1 << 20
    p = W.graded_hole_2d(n, 64, rho_scale=0.0)
    p = p.copy(rho_scale=oracle_rho_scale(p, n))
    r = Relaxation(p, n, 64, precision="fp32", seed=1, use_graph=True)
    assert r.info()["rho_scale"] == p.rho_scale
    r.step(5)
    assert check_cell_list(p, r, "fp32") <= 1e-4 * n
    r.close()


def test_create_samples_inside_region_with_target_density():
    from paper_1906_07925_gb300 import Relaxation
    p = W.graded_hole_2d(200000, 16, rho_scale=0.0)
    r = Relaxation(p, 200000, 16, precision="fp32", seed=7)
    x = r.positions(); c = r.colors()
    assert np.all(W.inside_mask(p, x))
    assert len(np.unique(c)) == 16
    rs = r.info()["rho_scale"]
    assert rs == pytest.approx(oracle.total_mass(p.copy(rho_scale=1.0), 2048) ** -1 * 200000, rel=2e-3)
    # counts in distance shells follow the target density
    d = np.abs(np.linalg.norm(x - 0.5, axis=1) - 0.2)
    near = np.mean(d < 0.05)
    q = W.sample_density(p.copy(rho_scale=1.0), 100000, 3)[0]
    want = np.mean(np.abs(np.linalg.norm(q - 0.5, axis=1) - 0.2) < 0.05)
    assert near == pytest.approx(want, rel=0.03)
    r.close()


def test_auto_ramp_fires_at_the_oracles_step():
    """Automatic start of the ramp (the convergence test of Sec. 3.3, read as
    in oracle.convergence_step): on the 4,096-particle square in FP64 the GPU
    fires at the same step as the oracle, takes the same ramp window, and the
    trajectories through the ramp stay as close as plain FP64 ones."""
    p, pos, col = c1_state()
    window, tol, theta, n = 10, 0.02, 0.15, 45
    xo, infos, t0 = oracle.run_auto_ramp(p, pos, col, n, window, tol, theta)
    assert t0 is not None and t0 < n - 5
    r = make_gpu(p, pos, col, "fp64")
    r.auto_ramp(window, tol, theta)
    r.step(n)
    st = r.stats()
    assert st["ramp_t0"] == t0
    assert st["ramp_t1"] == pytest.approx((1 + theta) * t0, rel=1e-15)
    assert st["sigma"] == pytest.approx(infos[-1]["sigma"], abs=1e-12)
    assert np.abs(r.positions() - xo).max() < 1e-6 * (1 / 64)
    # an explicit schedule turns the automatic one off
    r.ramp_surface_tension(100, 120)
    r.step(1)
    assert r.stats()["ramp_t0"] == 100
    r.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_color_volumes_match_oracle(precision):
    """Per-colour volume sum m/rho and count (the sizes of the partition's
    sub-domains) after one step from a seeded state, against the oracle's sums
    over its own densities of the same step: FP64 to 1e-12, FP32 to the
    density tolerance. Two calls give identical bits; before any step the call
    is refused."""
    from paper_1906_07925_gb300 import SphError
    p, pos, col = graded2d_state(20000, ncol=16)
    r = make_gpu(p, pos, col, precision)
    with pytest.raises(SphError):
        r.color_volumes()
    r.step(1)
    v, k = r.color_volumes()
    v2, k2 = r.color_volumes()
    assert np.array_equal(v, v2) and np.array_equal(k, k2)
    _, _, f = oracle.step(p, pos, col, 0)
    vo, ko = oracle.color_volumes(f["rho"], col, 16)
    assert np.array_equal(k, ko)
    tol = 1e-12 if precision == "fp64" else 2e-5
    assert np.all(np.abs(v - vo) <= tol * vo), np.abs(v / vo - 1).max()
    r.close()


def test_color_volumes_at_benchmark_size():
    """The 8,388,608-particle 3D workload's 256 colours (FP32): the device
    reduction against the same sums taken on the host from the densities the
    step recorded (FP64 sums), and the counts against the colours."""
    from paper_1906_07925_gb300 import Relaxation
    n = 1 << 23
    p = W.graded_inclusion_3d(n, 256, rho_scale=0.0)
    p = p.copy(rho_scale=oracle_rho_scale(p, n))
    r = Relaxation(p, n, 256, precision="fp32", seed=2, use_graph=True, record_fields=True)
    r.step(2)
    v, k = r.color_volumes()
    rho, col = r.field("rho"), r.colors()
    vo, ko = oracle.color_volumes(rho, col, 256)
    assert np.array_equal(k, ko) and k.sum() == n
    assert np.all(np.abs(v - vo) <= 1e-12 * vo)
    r.close()

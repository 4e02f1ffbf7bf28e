"""Planted mistakes in the oracle, each caught by a pin.

Every case copies oracle/sph_oracle.c, plants one plausible mistake (a changed
printed constant, a dropped factor, a swapped index or sign) in the forward
step or in the hand-written reverse pass, compiles the copy with gcc and runs
the pins named with it against the copy: at least one must fail. This shows
that the pins in test_oracle_pins.py and test_oracle_adjoint.py constrain each
part of the oracle's arithmetic, not only its overall behaviour. The original
oracle passes the same pins (they are the regular CPU tests).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle_adjoint as A
import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "sph_oracle.c")
HDR = os.path.join(os.path.dirname(oracle.__file__), "sph_oracle.h")

# (name, text in sph_oracle.c, replacement of its first occurrence, pins)
FORWARD = [
    ("viscosity nu = 0.2 r_c |v~| (Eq. viscosity_coefficient)",
     "double nu = 0.1 * rc * vn;", "double nu = 0.2 * rc * vn;",
     [(P.test_viscous_force_by_hand, (2, 40))]),
    ("harmonic mean of eta without its factor 2 (Eq. sph_viscous_force)",
     "double hm = es > 0.0 ? 2.0 * eta[i] * eta[j] / es : 0.0;",
     "double hm = es > 0.0 ? eta[i] * eta[j] / es : 0.0;",
     [(P.test_viscous_force_by_hand, (2, 40))]),
    ("viscous pair factor (dW/dr)/r with H^-3",
     "return wendland_alpha(H, dim) / (H * H) * (-20.0 * u * u * u);",
     "return wendland_alpha(H, dim) / (H * H * H) * (-20.0 * u * u * u);",
     [(P.test_viscous_pair_factor_is_kernel_slope_over_distance, (2,))]),
    ("viscous 1/rho_t^2 of i twice (Eq. sph_viscous_force_2)",
     "hm * (1.0 / (rt[i] * rt[i]) + 1.0 / (rt[j] * rt[j])) * orc_dW_over_r",
     "hm * (1.0 / (rt[i] * rt[i]) + 1.0 / (rt[i] * rt[i])) * orc_dW_over_r",
     [(P.test_momentum_conserved, (2, 2.0)), (P.test_viscous_force_by_hand, (2, 40))]),
    ("2D kernel constant 7/(2 pi H^2)",
     "return dim == 2 ? 7.0 / (PI * H * H)", "return dim == 2 ? 7.0 / (2.0 * PI * H * H)",
     [(P.test_kernel_normalised, (2,))]),
    ("kernel slope -10 q (1-q)^3",
     "return wendland_alpha(H, dim) / H * (-20.0 * q * u * u * u);",
     "return wendland_alpha(H, dim) / H * (-10.0 * q * u * u * u);",
     [(P.test_kernel_derivative_and_support, (2,))]),
    ("surface tension with one density term (Eq. sph_st_force)",
     "+ beta * (P0 / (rt[i] * rt[i]) + P0 / (rt[j] * rt[j]));", "+ beta * (P0 / (rt[i] * rt[i]));",
     [(P.test_surface_tension_repels_distinct_colours, ())]),
    ("pressure coefficient P_i + P_i (Eq. sph_pressure_force_2)",
     "double coef = (Pc[i] + Pc[j])", "double coef = (Pc[i] + Pc[i])",
     [(P.test_momentum_conserved, (2, 2.0))]),
    ("body-force time step 0.3 sqrt(r_c/|a|) (Eq. time_step_size)",
     "double t = 0.25 * sqrt(rc / an);", "double t = 0.3 * sqrt(rc / an);",
     [(P.test_time_step_rule_constants, ())]),
    ("CFL divisor 20 (Eq. time_step_size)",
     "double t1 = rc / (40.0 * vn);", "double t1 = rc / (20.0 * vn);",
     [(P.test_time_step_rule_constants, ())]),
    ("e_ij pointing from j to i",
     "ai[k] -= coef * dw * (pos[i * d + k] - pos[j * d + k]) / r;",
     "ai[k] += coef * dw * (pos[i * d + k] - pos[j * d + k]) / r;",
     [(P.test_surface_tension_repels_distinct_colours, ())]),
    ("density summed with the neighbour's smoothing length (Eq. density_sum)",
     "s += orc_W(sqrt(dist2(pos + i * d, pos + j * d, d)), kappa * h[i], d);",
     "s += orc_W(sqrt(dist2(pos + i * d, pos + j * d, d)), kappa * h[j], d);",
     [(P.test_density_gathers_with_own_smoothing_length, ())]),
    ("first kick without 1/2 (Eq. time_int_01)",
     "for (size_t q = 0; q < nd; ++q) vt[q] = 0.5 * a[q] * dt1;",
     "for (size_t q = 0; q < nd; ++q) vt[q] = a[q] * dt1;",
     [(P.test_viscous_force_by_hand, (2, 40))]),
    ("second kick without 1/2 (Eq. time_int_02)",
     "double v = vt[i * d + k] + 0.5 * at[i * d + k] * dt2;", "double v = vt[i * d + k] + at[i * d + k] * dt2;",
     [(P.test_viscous_force_by_hand, (2, 40))]),
    ("pair smoothing length h_i instead of (h_i + h_j)/2",
     "double hij = 0.5 * (h[i] + h[j]);\n      double dw", "double hij = h[i];\n      double dw",
     [(P.test_momentum_conserved, (2, 2.0))]),
    ("smoothing length tau^2 (m/rho_t)^(1/d) (Eq. scale_SPH_particle)",
     "h[i] = p->tau * pow(1.0 / rt[i], 1.0 / d);", "h[i] = p->tau * p->tau * pow(1.0 / rt[i], 1.0 / d);",
     [(P.test_viscous_force_by_hand, (2, 40))]),
    ("ramp measured from t1 (Eq. sph_st_sigma)",
     "return p->sigma0 * (1.0 - (p->t0 - t) / (p->t0 - p->t1));",
     "return p->sigma0 * (1.0 - (p->t1 - t) / (p->t0 - p->t1));",
     [(P.test_sigma_ramp_matches_paper, ())]),
    ("sphere projection to the diameter (Eq. displacement_surface)",
     "x[k] = s->center[k] + s->size[0] * d[k] / r;", "x[k] = s->center[k] + 2.0 * s->size[0] * d[k] / r;",
     [(P.test_projection_and_wall, ())]),
    ("cell level one band too low (multi-resolution cell key)",
     "h >= ldexp(g->h0, l + 1)) ++l;", "h >= ldexp(g->h0, l + 2)) ++l;",
     [(P.test_cell_key_files_each_particle_at_its_level_and_cell, (2,))]),
]

REVERSE = [
    ("reverse: eta = rho_t 0.2 r_c |v~|",
     "rtb[i] += etab[i] * 0.1 * kappa * h[i] * vn;", "rtb[i] += etab[i] * 0.2 * kappa * h[i] * vn;",
     [(A.test_adjoint_matches_fd_2d, (True,))]),
    ("reverse: drift derivative in dt2 with a halved viscous kick",
     "dt2b += gi[k] * (vt[q] + dt2 * at[q]);", "dt2b += gi[k] * (vt[q] + 0.5 * dt2 * at[q]);",
     [(A.test_adjoint_matches_fd_2d, (False,))]),
    ("reverse: pressure pair term with the wrong sign",
     "xb[i * d + k] += Sij * dab;", "xb[i * d + k] -= Sij * dab;",
     [(A.test_adjoint_matches_fd_2d, (True,))]),
    ("reverse: dL/dgamma without the logarithm",
     "pb->gamma += Qb[i] * Q[i] * lr;", "pb->gamma += Qb[i] * Q[i];",
     [(A.test_adjoint_matches_fd_3d_general_eos_seeded, (True,))]),
    ("reverse: density derivative in h halved",
     "hb[i] += rhob[i] * dW_dH(r, H, d) * p->kappa;", "hb[i] += rhob[i] * dW_dH(r, H, d) * 0.5 * p->kappa;",
     [(A.test_adjoint_matches_fd_3d_general_eos_seeded, (True,))]),
    ("reverse: second step size of the argmin with 0.125",
     "dt2b * 0.1 / sqrt(mmin);", "dt2b * 0.125 / sqrt(mmin);",
     [(A.test_adjoint_matches_fd_2d, (False,))]),
    ("reverse: interface term of the objective halved",
     "double c = lambda * orc_dW(r, H, d) / r;", "double c = 0.5 * lambda * orc_dW(r, H, d) / r;",
     [(A.test_adjoint_zero_steps_is_objective_gradient, ())]),
    ("reverse: d(x^2 y)/dx of the polynomial basis as x y",
     "double dX[8] = {1, 0, 2 * X, Y, 0, 3 * X * X, 2 * X * Y, Y * Y};",
     "double dX[8] = {1, 0, 2 * X, Y, 0, 3 * X * X, X * Y, Y * Y};",
     [(A.test_adjoint_matches_fd_2d, (True,))]),
]

CASES = FORWARD + REVERSE


@pytest.fixture(scope="module")
def mutants(tmp_path_factory):
    """Compile every mutated copy once (in parallel); returns name -> .so path."""
    src = open(SRC).read()
    root = tmp_path_factory.mktemp("mutants")
    gcc = shutil.which("gcc") or "gcc"

    def one(k):
        name, old, new, _ = CASES[k]
        assert old in src, name
        d = root / f"m{k}"
        d.mkdir()
        (d / "sph_oracle.c").write_text(src.replace(old, new, 1))
        shutil.copy(HDR, d / "sph_oracle.h")
        so = d / "libmut.so"
        subprocess.run([gcc, "-O1", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-w", "-o", str(so),
                        str(d / "sph_oracle.c"), "-lm"], check=True)
        return name, str(so)

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(ex.map(one, range(len(CASES))))


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(mutants, case):
    name, _, _, pins = CASES[case]
    oracle.lib()  # the real library, restored below
    saved = oracle._lib
    oracle._lib = oracle.bind(mutants[name])
    failed = []
    try:
        for fn, args in pins:
            try:
                fn(oracle, *args)
            except AssertionError:
                failed.append(fn.__name__)
    finally:
        oracle._lib = saved
    assert failed, f"no pin caught: {name}"

"""The C-ABI library builds, loads and exports every declared entry point; the
ctypes mirror of each struct has the C layout; argument validation answers
without touching a GPU."""
import ctypes as C
import os
import subprocess

import pytest

import workloads as W
from paper_1906_07925_gb300 import _binding as B
from paper_1906_07925_gb300 import build as build_lib
from paper_1906_07925_gb300 import problem_structs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib()
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    names = B.declared_symbols()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sphmesh.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(sph_shape),sizeof(sph_domain),sizeof(sph_field),sizeof(sph_params),"
        "sizeof(sph_alloc),sizeof(sph_stats),sizeof(sph_grid_info),"
        "offsetof(sph_params,seed),offsetof(sph_stats,rho_scale),"
        "sizeof(sph_background),offsetof(sph_background,spacing),"
        "sizeof(sph_batch_trial),offsetof(sph_batch_trial,stage_views));return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    want = [C.sizeof(B.sph_shape), C.sizeof(B.sph_domain), C.sizeof(B.sph_field), C.sizeof(B.sph_params),
            C.sizeof(B.sph_alloc), C.sizeof(B.sph_stats), C.sizeof(B.sph_grid_info),
            B.sph_params.seed.offset, B.sph_stats.rho_scale.offset,
            C.sizeof(B.sph_background), B.sph_background.spacing.offset,
            C.sizeof(B.sph_batch_trial), B.sph_batch_trial.stage_views.offset]
    assert got == want


def _create(lib, p, n=100, ncol=4, **kw):
    d, f, q = problem_structs(p, **kw)
    h = B.H()
    st = lib.sph_create(C.byref(d), C.byref(f), n, ncol, C.byref(q), None, None, C.byref(h))
    return st, h


@pytest.mark.parametrize("mutate", [
    lambda p: setattr(p, "dim", 4),
    lambda p: setattr(p, "s0", -1.0),
    lambda p: setattr(p, "tau", 0.0),
    lambda p: setattr(p, "poly", [0.6, 0.6]),
    lambda p: setattr(p, "gamma", -2.0),
])
def test_invalid_arguments_rejected_before_any_device_work(lib, mutate):
    p = W.uniform_square_2d(16)
    mutate(p)
    st, h = _create(lib, p)
    assert st == 1 and not h.value


def test_bad_colour_count_and_particle_count(lib):
    p = W.uniform_square_2d(16)
    assert _create(lib, p, ncol=0)[0] == 1
    assert _create(lib, p, ncol=300)[0] == 1
    assert _create(lib, p, n=-5)[0] == 1


def test_null_handle_calls(lib):
    assert lib.sph_step(None, 1) == 1
    assert lib.sph_sync(None) == 1
    assert lib.sph_last_error(None) == b"null handle"
    assert lib.sph_set_surface(None, None) == 1
    assert lib.sph_set_tuning(None, 256, 1.0, 1) == 1
    assert lib.sph_get_tuning(None, None, None, None) == 1
    assert lib.sph_get_stage_info(None, None, None, None) == 1
    d, f, q = problem_structs(W.uniform_square_2d(16))
    h = B.H()
    assert lib.sph_create_background(C.byref(d), C.byref(f), None, 10, 1, C.byref(q), None, None, C.byref(h)) == 1
    assert not h.value
    lib.sph_destroy(None)


def _create_bg(lib, p, n=100, ncol=4):
    from paper_1906_07925_gb300 import background_struct
    d, f, q = problem_structs(p)
    bg = background_struct(p.bg)
    h = B.H()
    st = lib.sph_create_background(C.byref(d), C.byref(f), C.byref(bg[0]), n, ncol, C.byref(q), None, None,
                                   C.byref(h))
    return st, h


@pytest.mark.parametrize("mutate", [
    lambda p: setattr(p.bg, "dims", [1, 101, 1]),                 # an axis with one node
    lambda p: setattr(p.bg, "dims", [101, 101, 2]),               # 2D mesh with a z extent
    lambda p: setattr(p.bg, "hi", [90.0, 100.0, 0.0]),            # mesh does not cover the box
    lambda p: p.bg.spacing.__setitem__((3, 4, 0), 0.0),            # spacing must be > 0
    lambda p: p.bg.phi.__setitem__((3, 4, 0), float("nan")),       # level set must be finite
    lambda p: setattr(p.bg, "spacing", None),                     # background field without spacing
    lambda p: setattr(p.bg, "phi", None),                         # grid shape without level set
])
def test_invalid_background_rejected_before_any_device_work(lib, mutate):
    p = W.circle_2d_background(100, 4)
    p.bg.phi = p.bg.phi.copy()
    p.bg.spacing = p.bg.spacing.copy()
    mutate(p)
    if p.bg.phi is not None and p.bg.spacing is not None and p.bg.dims[0] == 1:
        p.bg.phi = p.bg.phi[:1]
        p.bg.spacing = p.bg.spacing[:1]
    st, h = _create_bg(lib, p)
    assert st == 1 and not h.value


def test_grid_shape_needs_a_background_mesh(lib):
    p = W.circle_2d_background(100, 4)
    p.field_kind, p.s0 = W.FIELD_UNIFORM, 1.0
    st, h = _create(lib, p)
    assert st == 1 and not h.value


def test_background_nodes_are_passed_x_fastest():
    """Node arrays given shaped dims and indexed [i, j, k] reach the library
    (and the oracle) stored x fastest, as the header specifies."""
    import numpy as np
    import oracle
    from paper_1906_07925_gb300 import background_struct
    nx, ny = 4, 3
    phi = np.add.outer(10.0 * np.arange(nx), np.arange(ny))[:, :, None]  # phi[i, j] = 10 i + j
    bg = W.Background(dims=[nx, ny, 1], lo=[0, 0, 0], hi=[3, 2, 0], phi=phi, spacing=None)
    s, keep = background_struct(bg)
    flat = np.ctypeslib.as_array((C.c_double * (nx * ny)).from_address(s.phi))
    assert list(flat[:5]) == [0.0, 10.0, 20.0, 30.0, 1.0]  # x fastest: (0,0), (1,0), (2,0), (3,0), (0,1)
    p = W.Problem(dim=2, lo=[0, 0, 0], hi=[3, 2, 0], shapes=[W.Shape(W.GRID, True, [0, 0, 0], [1, 0, 0])], bg=bg)
    c = oracle.to_c(p)
    oflat = np.ctypeslib.as_array((C.c_double * (nx * ny)).from_address(c.bg_phi))
    assert np.array_equal(oflat, flat)


def test_missing_library_raises_instead_of_falling_back(monkeypatch, tmp_path):
    """Without libsphmesh.so the package refuses to run: there is no CPU
    implementation to fall back on."""
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "libsphmesh.so"))
    with pytest.raises(RuntimeError, match="missing"):
        B.load()

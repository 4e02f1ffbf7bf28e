"""The allocation-free entry point sph_eval_forces_noalloc.

It serves callers that cannot allocate device memory where they need the
forces (a host framework that owns all device buffers, a real-time loop that
cannot take cudaMalloc's implicit synchronisation): the cell list and pass-A
scratch live in a fixed device array inside the library. The test calls it
through the C ABI, twice in a row on the same inputs (the second call must not
see leftovers of the first), and checks density, acceleration and time steps
against the handle path (sph_set_state + sph_step + sph_get_field) and
against the FP64 oracle, with the parity tolerances of the other GPU tests
(FP32: density 1e-5 relative, force 1e-5 of the oracle's sum of pair-term
magnitudes, time steps 2e-5 relative). A case with more neighbours than the
fixed lists hold must fail with SPH_ERR_CELL_OVERFLOW and leave nothing
behind that changes the next call.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import check_force

pytestmark = pytest.mark.gpu


def _noalloc(lib, p, pos, col, expect=0):
    import torch
    from paper_1906_07925_gb300 import problem_structs
    d, f, q = problem_structs(p, precision="fp32")
    n, dim = pos.shape
    x = torch.from_numpy(pos).cuda()
    c = torch.from_numpy(col).cuda()
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    acc = torch.empty((n, dim), dtype=torch.float64, device="cuda")
    dt = torch.empty(2, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    st = lib.sph_eval_forces_noalloc(C.byref(d), C.byref(f), C.byref(q), n, x.data_ptr(), c.data_ptr(),
                                     rho.data_ptr(), acc.data_ptr(), dt.data_ptr(), C.c_void_p(s.cuda_stream))
    assert st == expect, st
    return rho.cpu().numpy(), acc.cpu().numpy(), dt.cpu().numpy()


@pytest.mark.parametrize("case", ["graded2d", "graded3d"])
def test_noalloc_matches_handle_path_twice(case):
    from paper_1906_07925_gb300 import Relaxation, load_library
    lib = load_library()
    if case == "graded2d":
        p = W.graded_hole_2d(20000, 8)
        pos, col, _ = W.sample_density(p, 20000, 21)
    else:
        p = W.graded_inclusion_3d(30000, 16)
        pos, col, _ = W.sample_density(p, 30000, 22)
    r = Relaxation(p, len(pos), int(col.max()) + 1, precision="fp32", record_fields=True, use_graph=False)
    r.set_state(pos, col)
    r.step(1)
    rho_h, acc_h, st = r.field("rho"), r.field("acc"), r.stats()
    r.close()
    _, info, f = oracle.step(p, pos, col, 0)
    S = f["pair_abs_a"]
    for call in range(2):
        rho, acc, dt = _noalloc(lib, p, pos, col)
        # against the handle path
        assert np.all(np.abs(rho - rho_h) <= 1e-5 * rho_h), call
        assert np.all(np.abs(acc - acc_h).max(axis=1) <= 1e-5 * S), call
        assert abs(dt[0] - st["dt1"]) <= 2e-5 * st["dt1"], call
        assert abs(dt[1] - st["dt2"]) <= 2e-5 * st["dt2"], call
        # against the oracle
        assert np.all(np.abs(rho - f["rho"]) <= 1e-5 * f["rho"]), call
        check_force(p, pos, acc, f, "fp32")
        assert abs(dt[0] - info["dt1"]) <= 2e-5 * info["dt1"], call
        assert abs(dt[1] - info["dt2"]) <= 2e-5 * info["dt2"], call


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    from paper_1906_07925_gb300 import load_library, problem_structs
    lib = load_library()
    p = W.uniform_square_2d(64)
    d, f, q = problem_structs(p, precision="fp32")
    n = 32769
    x = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    c = torch.zeros(n, dtype=torch.uint8, device="cuda")
    o = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    st = lib.sph_eval_forces_noalloc(C.byref(d), C.byref(f), C.byref(q), n, x.data_ptr(), c.data_ptr(),
                                     o.data_ptr(), o.data_ptr(), o.data_ptr(), None)
    assert st == 1


def test_noalloc_list_overflow_is_reported_and_leaves_no_trace():
    """tau = 3 in 3D gives about 113 neighbours inside the support: more than
    the 95 the fixed lists hold. The call reports SPH_ERR_CELL_OVERFLOW (the
    list build stops storing at its capacity); the next call, on a case that
    fits, matches the handle path."""
    from paper_1906_07925_gb300 import Relaxation, load_library
    lib = load_library()
    n = 8000
    big = W.Problem(dim=3, lo=[0, 0, 0], hi=[1, 1, 1], field_kind=W.FIELD_UNIFORM, s0=0.05, rho_scale=1.0,
                    tau=3.0, n_colors=4)
    pos = np.random.default_rng(5).random((n, 3))
    col = (np.arange(n) % 4).astype(np.uint8)
    _noalloc(lib, big, pos, col, expect=6)
    p = W.graded_hole_2d(6000, 8)
    pos2, col2, _ = W.sample_density(p, 6000, 23)
    r = Relaxation(p, len(pos2), int(col2.max()) + 1, precision="fp32", record_fields=True, use_graph=False)
    r.set_state(pos2, col2)
    r.step(1)
    rho_h, acc_h = r.field("rho"), r.field("acc")
    r.close()
    rho, acc, _ = _noalloc(lib, p, pos2, col2)
    _, _, f = oracle.step(p, pos2, col2, 0)
    assert np.all(np.abs(rho - rho_h) <= 1e-5 * rho_h)
    assert np.all(np.abs(acc - acc_h).max(axis=1) <= 1e-5 * f["pair_abs_a"])

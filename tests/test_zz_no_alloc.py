"""The allocation-free entry point sph_eval_forces_noalloc.

It serves callers that cannot allocate device memory where they need the
forces (a host framework that owns all device buffers, a real-time loop that
cannot take cudaMalloc's implicit synchronisation): the cell list and pass-A
scratch live in a fixed device array inside the library. The test calls it
through the C ABI, twice in a row on the same inputs (the second call must not
see leftovers of the first), and checks density, acceleration and time steps
against the handle path (sph_set_state + sph_step + sph_get_field) with the
parity tolerances of the other GPU tests (FP32: density 1e-5 relative, force
1e-5 of the oracle's sum of pair-term magnitudes, time steps 2e-5 relative).

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(lib, p, pos, col):
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
    assert st == 0
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
    _, _, f = oracle.step(p, pos, col, 0)
    S = f["pair_abs_a"]
    for call in range(2):
        rho, acc, dt = _noalloc(lib, p, pos, col)
        assert np.all(np.abs(rho - rho_h) <= 1e-5 * rho_h), call
        assert np.all(np.abs(acc - acc_h).max(axis=1) <= 1e-5 * S), call
        assert abs(dt[0] - st["dt1"]) <= 2e-5 * st["dt1"], call
        assert abs(dt[1] - st["dt2"]) <= 2e-5 * st["dt2"], call


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

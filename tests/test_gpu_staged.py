"""The staged density/force pass (sph_set_tuning stage_views = 1).

Staging changes where pass A reads a neighbour's view (a per-block copy in
shared memory instead of a gather from global memory), never what it
computes: every particle's sums run over its own list in list order. So the
staged handle must give results bit-identical to the unstaged one, over
steps on fresh and on stale lists (a rebuild every few steps), through the
graph and direct launches, and through the reverse pass; a block whose
neighbour set exceeds the stage capacity runs unstaged; the staged step
still matches the oracle at the FP32 parity tolerances.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from parity_util import compare_step, make_gpu

pytestmark = pytest.mark.gpu


def _run(p, n, stage, steps=12, graph=True, seed=3):
    from paper_1906_07925_gb300 import Relaxation
    r = Relaxation(p, n, p.n_colors, precision="fp32", seed=seed, use_graph=graph)
    r.set_tuning(stage_views=stage)
    r.step(steps)
    out = dict(x=r.positions(), st=r.stats(), info=r.stage_info())
    r.close()
    return out


@pytest.mark.parametrize("case", ["3d_graded", "2d_graded", "circle"])
def test_staged_pass_is_bitwise_the_unstaged_pass(case):
    if case == "3d_graded":
        p, n = W.graded_inclusion_3d(200000, 16), 200000
    elif case == "2d_graded":
        p, n = W.graded_hole_2d(300000, 16), 300000
    else:
        p, n = W.circle_2d(), 4289
    off = _run(p, n, 0)
    on = _run(p, n, 1)
    assert off["st"]["list_rebuilds"] == on["st"]["list_rebuilds"] >= 2
    assert np.array_equal(off["x"], on["x"])
    assert off["info"]["staged_blocks"] == 0
    info = on["info"]
    # every block of these workloads fits the stage capacity
    assert info["staged_blocks"] == info["blocks"] == (n + 255) // 256, info
    assert info["staged_views"] > n  # each block stages more neighbours than it has targets


def test_staged_direct_launches_match_the_graph():
    p = W.graded_inclusion_3d(50000, 8)
    a = _run(p, 50000, 1, steps=6, graph=True)
    b = _run(p, 50000, 1, steps=6, graph=False)
    assert np.array_equal(a["x"], b["x"])


def test_blocks_beyond_the_stage_capacity_run_unstaged():
    """tau = 4 in 3D: about 400 list entries per particle, so a block's
    distinct neighbours exceed 2,560 (tau = 3 stages about 1,840 per block)
    and it keeps the global gathers."""
    p = W.Problem(dim=3, lo=[0, 0, 0], hi=[1, 1, 1], field_kind=W.FIELD_UNIFORM, s0=0.05, rho_scale=0.0,
                  tau=4.0, n_colors=4)
    off = _run(p, 20000, 0, steps=4)
    on = _run(p, 20000, 1, steps=4)
    info = on["info"]
    assert info["staged_blocks"] < info["blocks"], info
    assert np.array_equal(off["x"], on["x"])


def test_staged_step_matches_oracle():
    p = W.graded_inclusion_3d(30000, 16)
    pos, col, _ = W.sample_density(p, 30000, 22)
    r = make_gpu(p, pos, col, "fp32")
    r.set_tuning(stage_views=1)
    compare_step(p, pos, col, "fp32", gpu=r)
    assert r.stage_info()["staged_blocks"] == r.stage_info()["blocks"]
    r.close()


def test_staged_reverse_pass_matches_unstaged():
    """The reverse pass re-runs forward segments with the handle's pass A:
    gradients are bit-identical with staging on and off, and match the oracle."""
    p = W.adjoint_poly_2d(n=3000, n_colors=8, seed=3)
    pos, col, _ = W.sample_density(p, 3000, seed=5)
    out = []
    for stage in (0, 1):
        r = make_gpu(p, pos, col, "fp32")
        r.set_tuning(stage_views=stage)
        out.append(r.backward(4, lam=1.0, ckpt_every=2))
        r.close()
    a, b = out
    assert np.array_equal(a["dpos0"], b["dpos0"])
    assert all(a["grads"][k] == b["grads"][k] for k in a["grads"])
    o = oracle.backward(p, pos, col, 4, 1.0)
    scale = np.abs(o["dpos0"]).max()
    assert np.abs(b["dpos0"] - o["dpos0"]).max() <= 1e-4 * scale


def test_staging_is_refused_for_fp64():
    from paper_1906_07925_gb300 import Relaxation, SphError
    p = W.graded_hole_2d(4000, 4)
    r = Relaxation(p, 4000, 4, precision="fp64", seed=1)
    with pytest.raises(SphError):
        r.set_tuning(stage_views=1)
    assert r.tuning()["stage_views"] == 0
    r.close()

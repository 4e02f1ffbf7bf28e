"""Batched instances (sph_batch_*): one CUDA graph per step with concurrent
branches must give, instance by instance, bit-identical results to the same
instances created and stepped on their own (same kernels, same per-instance
order of every sum), whatever the branch count; the autotuner's trial steps
must leave the state untouched."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _instances(k=10, seed=4, n_lo=2000, n_hi=12000):
    inst = W.batch_instances(k, seed=seed, n_lo=n_lo, n_hi=n_hi)
    probs, ns, cols = [], [], []
    for p, n in inst:
        p.rho_scale = 0.0  # the library normalises the field to n particles
        probs.append(p)
        ns.append(n)
        cols.append(p.n_colors)
    return probs, ns, cols


def test_batch_graph_matches_standalone_instances():
    from paper_1906_07925_gb300 import Batch, Relaxation
    probs, ns, cols = _instances()
    seeds = list(range(100, 100 + len(probs)))
    b = Batch(probs, ns, cols, precision="fp32", seeds=seeds, n_branches=4)
    b.step(6)
    b.sync()
    for k, p in enumerate(probs):
        r = Relaxation(p, ns[k], cols[k], precision="fp32", seed=seeds[k], use_graph=True)
        r.step(6)
        assert np.array_equal(b.positions(k), r.positions()), k
        assert np.array_equal(b.colors(k), r.colors())
        assert b.stats(k)["step"] == 6
        r.close()
    b.close()


def test_batch_branch_counts_and_per_instance_graphs_agree():
    from paper_1906_07925_gb300 import Batch
    probs, ns, cols = _instances(k=8, seed=5)
    seeds = list(range(8))
    ref = None
    for mode in ("each", 1, 3, 8):
        b = Batch(probs, ns, cols, precision="fp32", seeds=seeds, n_branches=0 if mode == "each" else mode)
        if mode == "each":
            b.step_each(4)
        else:
            b.step(4)
        b.sync()
        got = [b.positions(k) for k in range(len(probs))]
        if ref is None:
            ref = got
        else:
            for a, c in zip(ref, got):
                assert np.array_equal(a, c)
        b.close()


def test_batch_tune_restores_state_and_picks_a_trial():
    from paper_1906_07925_gb300 import Batch
    probs, ns, cols = _instances(k=12, seed=6)
    b = Batch(probs, ns, cols, precision="fp32", seeds=list(range(12)))
    b.step(2)
    b.sync()
    before = [b.positions(k) for k in range(12)]
    info = b.tune(candidates=(1, 2, 6, 12), steps_each=2)
    trials = info["trials"]
    # the branch counts first, then one trial per other value of each knob
    assert [t["branches"] for t in trials[:4]] == [1, 2, 6, 12]
    assert len(trials) == 4 + 1 + 2 + 1  # the other of (128, 256), two of (0.75, 1, 1.5), staging flipped
    ch = info["chosen"]
    assert info["n_branches"] == ch["branches"] in (1, 2, 6, 12)
    assert ch["ms_per_step"] == min(t["ms_per_step"] for t in trials)
    assert any(all(t[k] == ch[k] for k in ("branches", "pass_threads", "cell_factor", "stage_views")) for t in trials)
    assert trials[-1]["stage_views"] != trials[-2]["stage_views"]
    for k in range(12):
        assert np.abs(b.positions(k) - before[k]).max() <= 1e-14
        assert b.stats(k)["step"] == 2
    b.step(1)
    b.sync()
    b.close()


def test_launch_configuration_leaves_results_unchanged():
    """Threads per block of the pair passes change how the work is spread, not
    what is computed: positions after a few steps are bit-identical (graph
    replay and direct launches); a new cell factor only reorders sums, and the
    step still matches the oracle."""
    from parity_util import compare_step, make_gpu
    p = W.graded_inclusion_3d(20000, 8)
    pos, col, _ = W.sample_density(p, 20000, 5)
    ref = None
    for threads, stage in ((256, 0), (128, 0), (256, 1)):
        for graph in (True, False):
            r = make_gpu(p, pos, col, "fp32", use_graph=graph)
            r.set_tuning(pass_threads=threads, stage_views=stage)
            assert r.tuning()["pass_threads"] == threads
            assert r.tuning()["stage_views"] == stage
            r.step(4)
            x = r.positions()
            if stage:
                info = r.stage_info()
                assert info["staged_blocks"] == info["blocks"] > 0, info
            r.close()
            if ref is None:
                ref = x
            assert np.array_equal(x, ref), (threads, stage, graph)
    r = make_gpu(p, pos, col, "fp32")
    r.set_tuning(cell_factor=1.5)
    assert r.tuning()["cell_factor"] == 1.5
    compare_step(p, pos, col, "fp32", gpu=r)
    r.close()

"""Steps per history synchronisation: the sweeps move the midpoint states between shared memory
and the device history in groups of several steps (one wait per group; the adjoint fetches one
group ahead).  The grouping changes when copies are issued and waited for, never the arithmetic:
every depth must give the one-step results bitwise, over ragged windows (a group cut by a
window's end), tiles over two windows, both kernel families, both solvers and checkpointed
segments (groups cut by a segment's end), and agree with the oracle."""
import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


def run(spec, alpha, W, **kw):
    with msqoc.Problem(spec, **kw) as p:
        return p.eval_gradient(alpha, W), p.steps_per_sync


@pytest.mark.parametrize("layout", [msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_FIBER_LEAN])
@pytest.mark.parametrize("solver", [msqoc.SOLVER_MIXED, msqoc.SOLVER_FP64])
def test_every_depth_matches_one_step_groups_bitwise(layout, solver):
    spec = S.transmon_spec(3, 30.0, 2001, 7, 8)         # ragged windows of 285-286 steps
    alpha, W = S.random_alpha(spec, 71), S.random_W(spec, 71)
    cb = 5                                               # 5 does not divide 8: tiles over two windows
    ref, d1 = run(spec, alpha, W, layout=layout, solver=solver, col_block=cb, steps_per_sync=1)
    assert d1 == 1
    for depth in (2, 3, 4, 8):
        got, d = run(spec, alpha, W, layout=layout, solver=solver, col_block=cb, steps_per_sync=depth)
        assert d == depth
        assert got["P"] == ref["P"]
        np.testing.assert_array_equal(got["grad_alpha"], ref["grad_alpha"])
        np.testing.assert_array_equal(got["grad_W"], ref["grad_W"])
    want = oracle.evaluate(spec, alpha, W)
    assert_objective_close(ref["P"], want["P"])
    assert_grad_close(ref["grad_alpha"], want["grad_alpha"])
    assert_grad_close(ref["grad_W"], want["grad_W"])


@pytest.mark.parametrize("K", [5, 64])
def test_depths_with_checkpointed_segments(K):
    spec = S.transmon_spec(3, 30.0, 2001, 7, 8)
    alpha, W = S.random_alpha(spec, 72), S.random_W(spec, 72)
    ref, _ = run(spec, alpha, W, ckpt_interval=K, steps_per_sync=1)
    for depth in (3, 4):
        got, _ = run(spec, alpha, W, ckpt_interval=K, steps_per_sync=depth)
        assert got["P"] == ref["P"]
        np.testing.assert_array_equal(got["grad_alpha"], ref["grad_alpha"])
        np.testing.assert_array_equal(got["grad_W"], ref["grad_W"])


def test_full_size_4q_benchmark_tiles_with_four_steps_per_sync():
    spec = S.config_4q(M=256)
    alpha, W = S.random_alpha(spec, 73), S.random_W(spec, 73)
    ref, _ = run(spec, alpha, W, layout=msqoc.LAYOUT_FIBER, col_block=9, steps_per_sync=1)
    got, d = run(spec, alpha, W, layout=msqoc.LAYOUT_FIBER, col_block=9, steps_per_sync=4)
    assert d == 4
    assert got["P"] == ref["P"]
    np.testing.assert_array_equal(got["grad_alpha"], ref["grad_alpha"])
    np.testing.assert_array_equal(got["grad_W"], ref["grad_W"])


def test_depth_limits():
    spec = S.config_2q()
    for bad in (-1, 9):
        with pytest.raises(msqoc.MsqocError) as e:
            msqoc.Problem(spec, steps_per_sync=bad)
        assert e.value.status == -1

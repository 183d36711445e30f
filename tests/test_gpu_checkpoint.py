"""Checkpointed adjoint (checkpoint interval K > 1) against the oracle: the forward sweep keeps
the state every K steps of each window, and each K-step segment is recomputed from its
checkpoint before its adjoint sweep.  The gradient must match the oracle to the same bar as
K = 1 (every midpoint kept), including windows whose lengths differ and segments that end
before the window does."""
import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


def evaluate(spec, alpha, W, K, solver=msqoc.SOLVER_DEFAULT, col_block=0, layout=msqoc.LAYOUT_AUTO):
    with msqoc.Problem(spec, ckpt_interval=K, solver=solver, col_block=col_block, layout=layout) as p:
        return p.eval_gradient(alpha, W)


@pytest.mark.parametrize("K", [2, 7, 64])
def test_checkpointed_gradient_matches_oracle_3q(K):
    """Both sweep kernel families, two-window tiles of 5 columns."""
    spec = S.transmon_spec(3, 30.0, 2001, 7, 8)     # windows of 285 and 286 steps
    alpha, W = S.random_alpha(spec, 21), S.random_W(spec, 21)
    want = oracle.evaluate(spec, alpha, W)
    for layout in (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_FIBER_LEAN):
        got = evaluate(spec, alpha, W, K, col_block=5, layout=layout)
        assert_objective_close(got["P"], want["P"])
        assert_grad_close(got["grad_alpha"], want["grad_alpha"], what=f"grad_alpha (layout {layout})")
        assert_grad_close(got["grad_W"], want["grad_W"], what=f"grad_W (layout {layout})")


@pytest.mark.parametrize("K", [1, 16, 512])
def test_checkpoint_intervals_agree_4q(K):
    """4 transmons, 3 windows of 1000 steps: K = 512 leaves a short last segment."""
    spec = S.transmon_spec(4, 18.0, 3000, 3, 6)
    alpha, W = S.random_alpha(spec, 22), S.random_W(spec, 22)
    want = oracle.evaluate(spec, alpha, W)
    got = evaluate(spec, alpha, W, K)
    assert_objective_close(got["P"], want["P"])
    assert_grad_close(got["grad_alpha"], want["grad_alpha"], what="grad_alpha")
    assert_grad_close(got["grad_W"], want["grad_W"], what="grad_W")


def test_checkpoint_single_shooting_fp64_solver():
    spec = S.config_2q(M=1).replace(nsteps=700, T=17.5)
    alpha = S.random_alpha(spec, 23)
    want = oracle.evaluate(spec, alpha, np.zeros(0))
    got = evaluate(spec, alpha, np.zeros(0), 50, solver=msqoc.SOLVER_FP64)
    assert_objective_close(got["P"], want["P"])
    assert_grad_close(got["grad_alpha"], want["grad_alpha"], what="grad_alpha")


def test_checkpointing_shrinks_device_memory():
    spec = S.config_4q(M=64)
    with msqoc.Problem(spec, ckpt_interval=1) as a, msqoc.Problem(spec, ckpt_interval=64) as b:
        assert b.device_bytes < a.device_bytes / 10

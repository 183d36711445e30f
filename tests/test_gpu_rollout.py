"""Roll-out (the paper's initialisation of the window states, Sec. 5) and the roll-out
infidelity estimate (Eq. rollout-infid-est) on the GPU, against the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_objective_close

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", [msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_FIBER_LEAN])
@pytest.mark.parametrize("solver", [msqoc.SOLVER_MIXED, msqoc.SOLVER_FP64])
def test_rollout_matches_oracle_and_zeroes_the_penalties(solver, layout):
    spec = S.transmon_spec(3, 30.0, 2001, 7, 8)            # ragged windows
    alpha = S.random_alpha(spec, 71)
    want = oracle.rollout(spec, alpha)
    with msqoc.Problem(spec, solver=solver, col_block=5, layout=layout) as p:
        W = p.rollout(alpha)
        np.testing.assert_allclose(W, want, rtol=0, atol=1e-12)
        obj = p.eval_objective(alpha, W)
    assert np.all(np.abs(obj["pen"]) < 1e-22)
    single = oracle.evaluate(spec.replace(M=1), alpha, np.zeros(0), grad=False)
    assert_objective_close(obj["J"], single["P"], rtol=1e-11)


@pytest.mark.parametrize("layout", [msqoc.LAYOUT_FIBER, msqoc.LAYOUT_FIBER_LEAN])
def test_rollout_with_the_compensated_state_update(layout):
    # 4 transmons at the benchmark's step (|2 kappa| <= 0.034): the mixed solver keeps the state
    # as an FP64 part plus an FP32 carry, which the roll-out adds up where it stores U(t_m)
    spec = S.transmon_spec(4, 18.0, 3000, 3, 6)
    alpha = S.random_alpha(spec, 74)
    want = oracle.rollout(spec, alpha)
    with msqoc.Problem(spec, solver=msqoc.SOLVER_MIXED, col_block=7, layout=layout) as p:
        W = p.rollout(alpha)
        np.testing.assert_allclose(W, want, rtol=0, atol=1e-12)
        obj = p.eval_objective(alpha, W)
    assert np.all(np.abs(obj["pen"]) < 1e-22)


def test_rollout_estimate_is_the_formula_and_bounds_the_rollout_infidelity():
    spec = S.transmon_spec(2, 16.0, 320, 4, 6)
    alpha = S.random_alpha(spec, 72)
    with msqoc.Problem(spec) as p:
        W = p.rollout(alpha) + 0.05 * S.random_W(spec, 72)     # perturbed boundary states
        obj = p.eval_objective(alpha, W)
        est = p.rollout_estimate()
        g = p.eval_gradient(alpha, W)
        est_g = p.rollout_estimate()
    J, pen, mu, n = obj["J"], obj["pen"], 2.0 / spec.E, spec.E
    S_ = sum(math.sqrt(2 * x / mu) for x in pen)
    want = J + 2 / math.sqrt(n) * math.sqrt(J) * S_ + S_ ** 2 / n
    assert est == pytest.approx(want, rel=1e-13)
    assert est_g == pytest.approx(want, rel=1e-12)
    J_ro = oracle.evaluate(spec.replace(M=1), alpha, np.zeros(0), grad=False)["P"]
    assert J_ro <= est * (1 + 1e-12)
    assert g["P"] == pytest.approx(obj["P"], rel=1e-12)


@pytest.mark.parametrize("layout", [msqoc.LAYOUT_PAIR, msqoc.LAYOUT_QUAD])
def test_rollout_two_level_exchange(layout):
    """The roll-out of the paper's QFT-8 model (exchange coupling) with lane pairs and lane
    quads, ragged windows and tiles over two windows."""
    spec = S.paper_qft_spec(3, M=5, nsteps=601)
    alpha = S.random_alpha(spec, 73)
    want = oracle.rollout(spec, alpha)
    with msqoc.Problem(spec, col_block=5, layout=layout) as p:     # 40 or 80 threads, E = 8
        assert p.layout == layout
        W = p.rollout(alpha)
    np.testing.assert_allclose(W, want, rtol=0, atol=1e-12)

"""Window states of extreme magnitude against the oracle, both step solvers and both kernel
families.

The mixed-precision solver runs its inner sweeps in FP32, whose normal range is 2^-126..2^128.
The state is scaled per column by a power of two taken from the launch's initial state (the
step preserves column norms), so a state of any magnitude FP64 represents is solved relative to
its own column norm.  Window states scaled by 1e-36 and 1e36 would otherwise fall below FP32's
normal range or near its top.  Controls sit at the optimiser's box limit (amplitudes up to
2 pi x 25 MHz, Sec. 5), which also raises the solver's iteration counts.  Each window's penalty
and each window block of dP/dW is compared on its own scale, since the first window starts from
the identity embedding and dominates the totals.  dP/dalpha is compared over windows 2..M (a
shard, whose first window starts from W^1): with W ~ 0 next to U ~ 1 the first window's adjoint
state is proportional to its forward state, so its share of dP/dalpha cancels to round-off and
would hide the other windows' 1e-72-sized shares.
"""
import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc, optimize
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


def box_limit_alpha(spec, seed):
    bound = optimize.paper_settings(spec)["bound"]
    sign = np.where(S.uniform01(seed, 0, S.STREAM_MISC, spec.d) < 0.5, -1.0, 1.0)
    return sign * bound


@pytest.mark.parametrize("solver", [msqoc.SOLVER_MIXED, msqoc.SOLVER_FP64])
@pytest.mark.parametrize("scale", [1e-36, 1e36])
def test_extreme_window_state_magnitudes_match_the_oracle(scale, solver):
    spec = S.transmon_spec(3, 30.0, 2000, 7, 8)
    alpha = box_limit_alpha(spec, 5)
    W = S.random_W(spec, 5) * scale
    want = oracle.evaluate(spec, alpha, W)
    tail = oracle.evaluate(spec, alpha, W, windows=(2, spec.M))       # windows 2..M
    nb = 2 * spec.N * spec.E
    for layout in (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_FIBER_LEAN):
        with msqoc.Problem(spec, solver=solver, layout=layout) as p:
            got = p.eval_gradient(alpha, W)
            obj = p.eval_objective(alpha, W)
        assert_objective_close(got["P"], want["P"])
        assert_objective_close(obj["J"], want["J"])
        for m in range(spec.M - 1):
            assert_objective_close(obj["pen"][m], want["pen"][m])
            assert_grad_close(got["grad_W"][m * nb:(m + 1) * nb], want["grad_W"][m * nb:(m + 1) * nb],
                              what=f"grad_W block {m + 1} (layout {layout}, scale {scale:g})")
        with msqoc.Problem(spec, solver=solver, layout=layout, windows=(2, spec.M)) as p:
            got_t = p.eval_gradient(alpha, W)                          # reads W^1 .. W^{M-1}
        assert_objective_close(got_t["P"], tail["P"])
        assert_grad_close(got_t["grad_alpha"], tail["grad_alpha"], what=f"grad_alpha (layout {layout})")


def test_box_limit_controls_with_unit_states_match_the_oracle():
    spec = S.transmon_spec(4, 1.8, 300, 3, 5)
    alpha = box_limit_alpha(spec, 9)
    W = S.random_W(spec, 9)
    want = oracle.evaluate(spec, alpha, W)
    for solver in (msqoc.SOLVER_MIXED, msqoc.SOLVER_FP64):
        with msqoc.Problem(spec, solver=solver) as p:
            got = p.eval_gradient(alpha, W)
        assert_objective_close(got["P"], want["P"])
        assert_grad_close(got["grad_alpha"], want["grad_alpha"], what="grad_alpha")
        assert_grad_close(got["grad_W"], want["grad_W"], what="grad_W")

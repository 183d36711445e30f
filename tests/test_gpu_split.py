"""The compensated FP32 arithmetic of the mixed solver's gradient products on the device gives
the same bits as the host build of the same source (whose accuracy tests/test_split_cpu.py
pins against exact arithmetic), and the mixed solver's gradients (products in that form)
agree with the FP64 solver's (products in FP64) at full size."""
import numpy as np
import pytest

from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close, grad_mismatch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sh", [0, 9, -9, 700, -700])
def test_device_split_equals_host_split(sh):
    rng = np.random.default_rng(3000 + sh)
    x = rng.standard_normal(20000) * 2.0 ** rng.integers(-130, 3, 20000) * 2.0 ** sh
    x[:8] = [0.0, -0.0, 5e-324, 2.0 ** (sh - 127), 2.0 ** (sh - 75), 2.0 ** (sh - 74),
             np.nextafter(2.0, 0.0) * 2.0 ** sh, -(1.0 + 2.0 ** -24) * 2.0 ** sh]
    hh, lh = msqoc.selftest_split(x, sh, device=False)
    hd, ld = msqoc.selftest_split(x, sh, device=True)
    np.testing.assert_array_equal(hd.view(np.uint32), hh.view(np.uint32))
    np.testing.assert_array_equal(ld.view(np.uint32), lh.view(np.uint32))


def test_device_dot_equals_host_dot():
    rng = np.random.default_rng(31)
    for trial in range(40):
        n = int(rng.integers(0, 80))
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        if n > 1 and trial % 2:
            y[-1] = -np.dot(x[:-1], y[:-1]) / x[-1]
        shx, shy = int(rng.integers(-450, 450)), int(rng.integers(-450, 450))   # finite results
        xs, ys = x * 2.0 ** shx, y * 2.0 ** shy
        h = msqoc.selftest_dot(xs, ys, shx, shy, device=False)
        d = msqoc.selftest_dot(xs, ys, shx, shy, device=True)
        assert np.float64(h).view(np.uint64) == np.float64(d).view(np.uint64), (trial, h, d)


def test_mixed_and_fp64_solver_gradients_agree_at_full_size():
    # the benchmark workload (4 transmons, 100000 steps) at 64 windows, both one-thread builds
    spec = S.config_4q(M=64)
    alpha, W = S.random_alpha(spec, 41), S.random_W(spec, 41)
    with msqoc.Problem(spec, solver=msqoc.SOLVER_FP64) as b:
        rb = b.eval_gradient(alpha, W)
    for layout in (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_FIBER_LEAN):
        with msqoc.Problem(spec, solver=msqoc.SOLVER_MIXED, layout=layout) as a:
            ra = a.eval_gradient(alpha, W)
        assert_objective_close(ra["P"], rb["P"], rtol=1e-13)
        assert_grad_close(ra["grad_alpha"], rb["grad_alpha"], rtol=1e-11, what="grad_alpha")
        assert_grad_close(ra["grad_W"], rb["grad_W"], rtol=1e-11, what="grad_W")
        nbad, worst = grad_mismatch(ra["grad_alpha"], rb["grad_alpha"], rtol=1e-12, floor=1e-14)
        print(f"layout {layout}: grad_alpha worst relative difference {worst:.2e}, {nbad} beyond 1e-12")

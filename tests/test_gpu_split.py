"""The compensated FP32 arithmetic of the mixed solver on the device gives the same bits as the
host build of the same source (whose accuracy tests/test_split_cpu.py pins against exact
arithmetic), and at full size the mixed solver (compensated products and state update) is at
least as close to the oracle as the all-FP64 solver."""
import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

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


def test_device_carry_update_equals_host():
    rng = np.random.default_rng(32)
    for trial in range(12):
        n = int(rng.integers(0, 300))
        mag = rng.uniform(0.05, 1.0)
        u0 = mag * np.exp(1j * rng.uniform(0, 2 * np.pi))
        P = 1.0 / complex(1.0, rng.uniform(-0.022, 0.022))
        d = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1e-3 * mag
        sh = int(rng.integers(-40, 40))
        h = msqoc.selftest_carry(u0 * 2.0 ** sh, P, d * 2.0 ** sh, sh=sh, device=False)
        g = msqoc.selftest_carry(u0 * 2.0 ** sh, P, d * 2.0 ** sh, sh=sh, device=True)
        assert np.array([h]).view(np.uint64).tolist() == np.array([g]).view(np.uint64).tolist(), (trial, h, g)


def test_mixed_solver_at_least_as_close_to_the_oracle_as_fp64_at_full_size():
    # the benchmark workload (4 transmons, 100000 steps) at 64 windows, both one-thread builds.
    # The FP64 solver's state update R u with R = 2P - 1 carries the rounding of P (about 2^-53
    # a step, the same every step); the mixed solver's compensated update u + 2 kappa (Im b,
    # -Re b) carries it times |2 kappa| only, and its own errors do not add up the same way.
    spec = S.config_4q(M=64)
    alpha, W = S.random_alpha(spec, 41), S.random_W(spec, 41)
    want = oracle.evaluate(spec, alpha, W)
    with msqoc.Problem(spec, solver=msqoc.SOLVER_FP64) as b:
        rb = b.eval_gradient(alpha, W)
    err = lambda r, k: np.linalg.norm(np.asarray(r[k]) - want[k]) / np.linalg.norm(want[k])
    eb = {k: err(rb, k) for k in ("grad_alpha", "grad_W")}
    for layout in (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_FIBER_LEAN):
        with msqoc.Problem(spec, solver=msqoc.SOLVER_MIXED, layout=layout) as a:
            ra = a.eval_gradient(alpha, W)
        assert_objective_close(ra["P"], want["P"])
        assert_grad_close(ra["grad_alpha"], want["grad_alpha"], what="grad_alpha")
        assert_grad_close(ra["grad_W"], want["grad_W"], what="grad_W")
        assert abs(ra["P"] - want["P"]) <= abs(rb["P"] - want["P"]) * 1.05 + 1e-16 * abs(want["P"])
        for k in ("grad_alpha", "grad_W"):
            assert err(ra, k) <= eb[k] * 1.05, (layout, k, err(ra, k), eb[k])
        print(f"layout {layout}: relative gradient error against the oracle: mixed "
              f"{err(ra, 'grad_alpha'):.2e}, FP64 {eb['grad_alpha']:.2e}; P mixed "
              f"{abs(ra['P'] - want['P']) / abs(want['P']):.2e}, FP64 {abs(rb['P'] - want['P']) / abs(want['P']):.2e}")


@pytest.mark.parametrize("nsteps", [560, 600])
@pytest.mark.parametrize("layout", [msqoc.LAYOUT_FIBER, msqoc.LAYOUT_FIBER_LEAN])
def test_state_update_forms_on_either_side_of_the_bound(nsteps, layout):
    # 3 transmons over 6 ns, max |D| = 4.22: |2 kappa| = h max|D| is 0.0452 at 560 steps (above
    # 2^-4.5 = 0.0442: the FP64 update R u + 2 d) and 0.0422 at 600 (the compensated update)
    spec = S.transmon_spec(3, 6.0, nsteps, 4, 5)
    alpha, W = S.random_alpha(spec, 43), S.random_W(spec, 43)
    want = oracle.evaluate(spec, alpha, W)
    with msqoc.Problem(spec, solver=msqoc.SOLVER_MIXED, layout=layout) as p:
        got = p.eval_gradient(alpha, W)
    assert_objective_close(got["P"], want["P"])
    assert_grad_close(got["grad_alpha"], want["grad_alpha"], what="grad_alpha")
    assert_grad_close(got["grad_W"], want["grad_W"], what="grad_W")

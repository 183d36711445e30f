"""Failure path of the sweeps, exercised without a GPU fault: the bounded mbarrier wait that the
adjoint sweep uses for its history fetches gives up on a phase that nothing completes and
reports MSQOC_ERR_TIMEOUT through the device status word; the context stays usable (an
evaluation afterwards matches the oracle)."""
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_with_timeout_status_and_the_device_stays_usable():
    with pytest.raises(msqoc.MsqocError) as err:
        msqoc.selftest_bounded_wait(4096)                  # a phase nothing completes
    assert err.value.status == -5
    assert msqoc.selftest_bounded_wait(4096, arrive=True) < 1.0   # completed: returns at once
    spec = S.transmon_spec(2, 10.0, 200, 3, 5)
    alpha, W = S.random_alpha(spec, 51), S.random_W(spec, 51)
    with msqoc.Problem(spec) as p:
        got = p.eval_gradient(alpha, W)
    want = oracle.evaluate(spec, alpha, W)
    assert_objective_close(got["P"], want["P"])
    assert_grad_close(got["grad_alpha"], want["grad_alpha"])


def test_sweep_wait_limit_ends_within_seconds():
    """The sweeps' limit (2^18 polls), timed from a shorter give-up: a stuck fetch ends the
    launch in about a second, not never."""
    spins = 1 << 16
    with pytest.raises(msqoc.MsqocError):
        msqoc.selftest_bounded_wait(spins)
    import time
    t0 = time.perf_counter()
    with pytest.raises(msqoc.MsqocError):
        msqoc.selftest_bounded_wait(spins)
    per_spin = (time.perf_counter() - t0) / spins
    limit_s = per_spin * (1 << 18)
    print(f"bounded wait: {per_spin * 1e9:.1f} ns per poll, sweep limit {limit_s:.3f} s")
    assert limit_s < 5.0

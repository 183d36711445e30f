"""The continuous-batching server: every served result equals the session's own single
evaluation of the same inputs (within the parity tolerance), whatever it was batched with;
admission refuses a session whose memory does not fit the budget."""
import pytest

from paper_2407_13950_gb300 import msqoc, serving
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


def small_sessions():
    return [S.transmon_spec(2, 20.0, 800, 4, 6), S.transmon_spec(2, 15.0, 600, 3, 6),
            S.transmon_spec(3, 6.0, 400, 4, 5), S.transmon_spec(3, 4.5, 300, 2, 5),
            S.transmon_spec(4, 1.2, 200, 2, 4)]


def test_served_results_match_single_evaluations():
    specs = small_sessions()
    srv = serving.Server(device_budget_bytes=64 << 30)
    try:
        for sp in specs:
            srv.admit(sp)
        reqs = serving.poisson_requests(specs, rate=400.0, duration=0.1, seed=5)
        assert len(reqs) > 10
        done = srv.run(reqs)
        assert len(done) == len(reqs)
        for r in done:
            p = srv.sessions[r.session]
            if r.gradient:
                want = p.eval_gradient(r.alpha, r.W)
                assert_objective_close(r.result["P"], want["P"])
                assert_grad_close(r.result["grad_alpha"], want["grad_alpha"], what="grad_alpha")
                if p.spec.M > 1:
                    assert_grad_close(r.result["grad_W"], want["grad_W"], what="grad_W")
            else:
                want = p.eval_objective(r.alpha, r.W)
                assert_objective_close(r.result["P"], want["P"])
                assert_objective_close(r.result["J"], want["J"])
            assert r.arrival <= r.dispatched <= r.done
        lat = serving.latency_summary(done)
        assert lat["from_arrival"]["p99"] >= lat["from_arrival"]["p50"] > 0
    finally:
        srv.close()


def test_admission_by_device_memory():
    srv = serving.Server(device_budget_bytes=1 << 20)   # 1 MiB: nothing fits
    try:
        with pytest.raises(serving.NotAdmitted):
            srv.admit(S.config_3q())
        assert srv.used == 0 and not srv.sessions
    finally:
        srv.close()

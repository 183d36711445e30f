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


def assert_same_as_alone(srv, r):
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


def request(spec, session, gradient, arrival, seed):
    return serving.Request(session=session, gradient=gradient, alpha=S.random_alpha(spec, seed, problem=session),
                           W=S.random_W(spec, seed, problem=session) if spec.M > 1 else None, arrival=arrival)


@pytest.mark.parametrize("policy", ["fifo", "throughput"])
def test_served_results_match_single_evaluations_under_both_policies(policy):
    specs = small_sessions()
    srv = serving.Server(device_budget_bytes=64 << 30, policy=policy, lookahead=8)
    try:
        for sp in specs:
            srv.admit(sp)
        reqs = serving.poisson_requests(specs, rate=400.0, duration=0.1, seed=6)
        done = srv.run(reqs)
        assert len(done) == len(reqs)
        for r in done:
            assert_same_as_alone(srv, r)
    finally:
        srv.close()


def test_dispatches_on_two_slots_overlap_on_the_device():
    # two 4-transmon sessions of 16 windows (32 tiles each: together they fill 64 of the SMs),
    # a gradient and an objective request at t = 0: two classes, so two dispatches on two slots.
    # Run one after the other they take t_g + t_o; overlapped, about max(t_g, t_o).
    import torch
    spec = S.transmon_spec(4, 120.0, 20000, 16, 10)
    srv = serving.Server(device_budget_bytes=64 << 30)
    try:
        srv.admit(spec)
        srv.admit(spec)
        alone = {}
        for grad in (True, False):          # each alone (after a warm-up run), device time
            srv.run([request(spec, 0 if grad else 1, grad, 0.0, 3)])
            r = request(spec, 0 if grad else 1, grad, 0.0, 3)
            srv.run([r], record_events=True)
            alone[grad] = r.events[0].elapsed_time(r.events[1])
        rg, ro = request(spec, 0, True, 0.0, 4), request(spec, 1, False, 0.0, 4)
        done = srv.run([rg, ro], record_events=True)
        assert len(done) == 2 and rg.slot != ro.slot
        base = srv.base_event
        s_g, e_g = base.elapsed_time(rg.events[0]), base.elapsed_time(rg.events[1])
        s_o, e_o = base.elapsed_time(ro.events[0]), base.elapsed_time(ro.events[1])
        # the objective ran inside the gradient's interval, and the pair took clearly less than
        # the two alone back to back
        assert s_g < e_o < e_g, (s_g, e_g, s_o, e_o)
        makespan = max(e_g, e_o) - min(s_g, s_o)
        assert makespan < 0.9 * (alone[True] + alone[False]), (makespan, alone)
        for r in done:
            assert_same_as_alone(srv, r)
        torch.cuda.synchronize()
    finally:
        srv.close()


def test_request_arriving_mid_flight_is_dispatched_before_the_running_subset_completes():
    big = S.transmon_spec(4, 300.0, 50000, 16, 20)          # a gradient of ~0.1 s
    small = S.config_2q()
    srv = serving.Server(device_budget_bytes=64 << 30)
    try:
        srv.admit(big)
        srv.admit(small)
        srv.run([request(big, 0, True, 0.0, 8), request(small, 1, True, 0.0, 8)])   # warm
        r_big = request(big, 0, True, 0.0, 9)
        r_small = request(small, 1, True, 0.02, 9)           # arrives while the big one runs
        done = srv.run([r_big, r_small])
        assert len(done) == 2
        assert r_small.arrival <= r_small.dispatched < r_big.done
        assert r_small.done < r_big.done
        for r in done:
            assert_same_as_alone(srv, r)
    finally:
        srv.close()


def test_served_mix_with_a_checkpointed_5q_session_matches_alone():
    # the serving workload's shapes at full size, the 5-transmon session with checkpoint
    # interval 64 (its history with every midpoint would be 18.7 GB)
    shapes = [(S.config_2q(), 0), (S.config_3q(), 0), (S.config_4q(), 0), (S.config_5q(), 64)]
    srv = serving.Server(device_budget_bytes=200 << 30)
    try:
        for sp, K in shapes:
            srv.admit(sp, ckpt_interval=K)
        assert srv.sessions[3].ckpt_interval == 64
        specs = [sp for sp, _ in shapes]
        reqs = [request(specs[i % 4], i % 4, g, 0.002 * i, 20 + i) for i, g in
                enumerate([True, False, True, True, False, True, False, True])]
        reqs += [request(specs[3], 3, True, 0.03, 40), request(specs[2], 2, False, 0.031, 41)]
        reqs.sort(key=lambda r: r.arrival)
        done = srv.run(reqs)
        assert len(done) == len(reqs)
        assert {srv.sessions[r.session].spec.q for r in done} == {2, 3, 4, 5}
        for r in done:
            assert_same_as_alone(srv, r)
    finally:
        srv.close()

"""The allocation-free objective entry point (msqoc_eval_objective_noalloc) against the regular
one (msqoc_create_problem + msqoc_eval_objective), through the C ABI.

Callers that cannot allocate device memory (a plug-in whose host application owns the device
heap, a process that reserved all device memory up front, a control loop that cannot pay for
cudaMalloc / cudaFree) use the allocation-free entry point: every table and intermediate lives
in one static scratch array of the library.  That array is shared by every call and keeps the
previous call's contents, so the checks below run several calls in a row with different
problem sizes and compare each result with the regular entry point within the objective
tolerance of the parity tests.  This file is collected last: a run that stops at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_objective_close

pytestmark = pytest.mark.gpu


def regular_objective(spec, alpha, W, solver=msqoc.SOLVER_DEFAULT):
    with msqoc.Problem(spec, solver=solver) as p:
        return p.eval_objective(alpha, W)


def assert_same_objective(got, want, M):
    assert_objective_close(got["P"], want["P"])
    assert_objective_close(got["J"], want["J"])
    if M > 1:
        # a penalty whose residual is at round-off ((1e-14)^2) has no relative accuracy
        np.testing.assert_allclose(got["pen"], want["pen"], rtol=1e-12, atol=1e-24)


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    cases = [(S.config_3q(), 1, msqoc.SOLVER_DEFAULT),
             (S.config_2q(), 2, msqoc.SOLVER_FP64),
             (S.transmon_spec(3, 30.0, 2000, 7, 8), 3, msqoc.SOLVER_MIXED),
             (S.config_3q(), 1, msqoc.SOLVER_DEFAULT)]
    first = None
    for spec, seed, solver in cases:
        alpha, W = S.random_alpha(spec, seed), S.random_W(spec, seed)
        want = regular_objective(spec, alpha, W, solver)
        got = msqoc.eval_objective_noalloc(spec, alpha, W, solver=solver)
        assert_same_objective(got, want, spec.M)
        if first is None:
            first = got
    # the last call repeats the first one after other sizes have used the scratch
    assert got["P"] == first["P"] and got["J"] == first["J"]
    np.testing.assert_array_equal(got["pen"], first["pen"])


def test_noalloc_full_size_4q_with_device_arrays_twice():
    import torch
    spec = S.config_4q(M=64)
    alpha, W = S.random_alpha(spec, 7), S.random_W(spec, 7)
    want = regular_objective(spec, alpha, W)
    dev = torch.device("cuda")
    a_d = torch.tensor(alpha, device=dev, dtype=torch.float64)
    W_d = torch.tensor(W, device=dev, dtype=torch.float64)
    for _ in range(2):
        P_d = torch.full((1,), float("nan"), device=dev, dtype=torch.float64)
        J_d = torch.full((1,), float("nan"), device=dev, dtype=torch.float64)
        pen_d = torch.full((spec.M - 1,), float("nan"), device=dev, dtype=torch.float64)
        stream = torch.cuda.current_stream()
        msqoc.eval_objective_noalloc(spec, a_d, W_d, stream=stream, P_out=P_d, J_out=J_d, pen_out=pen_d)
        got = {"P": P_d.item(), "J": J_d.item(), "pen": pen_d.cpu().numpy()}
        assert_same_objective(got, want, spec.M)


def test_noalloc_largest_4q_window_count_fits():
    spec = S.config_4q(M=256)
    alpha, W = S.random_alpha(spec, 11), S.random_W(spec, 11)
    got = msqoc.eval_objective_noalloc(spec, alpha, W)
    assert_same_objective(got, regular_objective(spec, alpha, W), spec.M)


def test_noalloc_rejects_a_problem_beyond_the_scratch_limit():
    spec = S.config_5q()     # 150000 steps, N=243, E=32, M=256: about 76 MB of scratch
    alpha, W = S.random_alpha(spec, 1), S.random_W(spec, 1)
    with pytest.raises(msqoc.MsqocError) as err:
        msqoc.eval_objective_noalloc(spec, alpha, W)
    assert err.value.status == -1
    assert "MSQOC_NOALLOC_SCRATCH_BYTES" in str(err.value)
    # the library is still usable after the rejection
    spec2 = S.config_2q()
    a2, W2 = S.random_alpha(spec2, 5), S.random_W(spec2, 5)
    assert_same_objective(msqoc.eval_objective_noalloc(spec2, a2, W2), regular_objective(spec2, a2, W2), spec2.M)


def test_noalloc_calls_leave_device_free_memory_unchanged():
    # what the entry point is for: calls take no device memory.  One warm call per size first:
    # the CUDA runtime loads each kernel's code onto the device at its first launch, which is
    # device memory the driver takes once, not an allocation of the call
    import torch
    cases = [S.config_2q(), S.config_3q(), S.transmon_spec(3, 30.0, 2000, 7, 8), S.config_4q(M=64)]
    inputs = [(sp, S.random_alpha(sp, 3), S.random_W(sp, 3)) for sp in cases]
    warm = [msqoc.eval_objective_noalloc(sp, a, W) for sp, a, W in inputs]
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    results = [msqoc.eval_objective_noalloc(sp, a, W) for sp, a, W in inputs for _ in range(2)]
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (free_before, free_after)
    # every call on the same inputs gives the same numbers
    for k, w in enumerate(warm):
        assert results[2 * k]["P"] == w["P"] and results[2 * k + 1]["P"] == w["P"]

"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on seeded inputs.

Bar: objective within 1e-12 relative; every gradient component within 1e-10 relative (plus a
round-off floor of 1e-13 of the largest component).  Sizes are small enough for the oracle to
finish in seconds while still spanning several tiles, several warps per tile, ragged windows
and both solvers; the full 4-transmon workload is checked on sampled windows in
test_gpu_fullsize.py.
"""
import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu

SOLVERS = {"mixed": msqoc.SOLVER_MIXED, "fp64": msqoc.SOLVER_FP64}


LAYOUTS = {"fiber": msqoc.LAYOUT_FIBER, "pair": msqoc.LAYOUT_PAIR, "lean": msqoc.LAYOUT_FIBER_LEAN}
# one thread per fiber (255 and 168 registers) and a lane pair per fiber
BOTH = (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_FIBER_LEAN)


def run_gpu(spec, alpha, W, solver, col_block=0, ckpt_interval=0, layout=msqoc.LAYOUT_AUTO):
    with msqoc.Problem(spec, solver=solver, col_block=col_block, ckpt_interval=ckpt_interval, layout=layout) as p:
        if layout != msqoc.LAYOUT_AUTO:
            assert p.layout == layout
        return p.eval_gradient(alpha, W), p.eval_objective(alpha, W)


def check(spec, alpha, W, solver, col_block=0, ckpt_interval=0, layouts=BOTH):
    """The sweep kernel families (one thread per fiber in both register budgets, a lane pair per
    fiber) against one oracle evaluation."""
    want = oracle.evaluate(spec, alpha, W)
    for layout in layouts:
        got, obj = run_gpu(spec, alpha, W, solver, col_block, ckpt_interval, layout)
        assert_objective_close(got["P"], want["P"])
        assert_objective_close(obj["P"], want["P"])
        if spec.M > 1:
            # a penalty whose residual is at round-off ((1e-14)^2) has no relative accuracy
            np.testing.assert_allclose(obj["pen"], want["pen"], rtol=1e-12, atol=1e-24)
        assert_objective_close(obj["J"], want["J"])
        assert_grad_close(got["grad_alpha"], want["grad_alpha"], what=f"grad_alpha (layout {layout})")
        if spec.M > 1:
            assert_grad_close(got["grad_W"], want["grad_W"], what=f"grad_W (layout {layout})")
    return got, want


CASES = {
    "1q": S.transmon_spec(1, 10.0, 200, 4, 5),
    "2q-config": S.config_2q(),
    "3q-ragged": S.transmon_spec(3, 30.0, 2000, 7, 8),
    "4q-short": S.transmon_spec(4, 1.8, 300, 3, 5),
}


@pytest.mark.parametrize("solver", list(SOLVERS))
@pytest.mark.parametrize("case", list(CASES))
def test_parity_small(case, solver):
    spec = CASES[case]
    alpha, W = S.random_alpha(spec, 101), S.random_W(spec, 101)
    check(spec, alpha, W, SOLVERS[solver])


@pytest.mark.parametrize("layout,cb", [("fiber", cb) for cb in (1, 2, 3, 4, 5, 7, 8, 9)] +
                         [("pair", cb) for cb in (1, 2, 3, 4, 5, 6, 7)] +
                         [("lean", cb) for cb in (1, 6, 7, 9, 11, 13, 14)])
def test_parity_column_blocks_4q(layout, cb):
    """Tiles of cb columns run along the window-major column list; widths that do not divide
    E = 16 give tiles covering two windows (3, 5, 6, 7, 9, 11, 13 and 14 here).  9 columns (243
    threads) is the widest one-thread-per-fiber tile of the 255-register build, 14 (378 threads)
    of the 168-register build, 7 (384 threads) the widest lane-pair tile."""
    spec = S.transmon_spec(4, 1.2, 200, 3, 4)
    alpha, W = S.random_alpha(spec, 7), S.random_W(spec, 7)
    check(spec, alpha, W, msqoc.SOLVER_MIXED, col_block=cb, layouts=(LAYOUTS[layout],))


@pytest.mark.parametrize("nsteps,M,d1", [(24, 24, 20), (60, 30, 10), (300, 5, 3), (301, 3, 41)])
def test_parity_window_local_gradient_ranges(nsteps, M, d1):
    """The adjoint keeps each window's alpha-gradient over the splines active in that window
    only: one step per window (24 windows, 20 splines), windows shorter than a spline interval
    (30 windows, 10 splines), the smallest basis (3 splines, all active everywhere) and long
    ragged windows over many splines; also with tiles over two windows (cb = 5, E = 8)."""
    spec = S.transmon_spec(3, 12.0, nsteps, M, d1)
    alpha, W = S.random_alpha(spec, 9), S.random_W(spec, 9)
    check(spec, alpha, W, msqoc.SOLVER_MIXED)
    check(spec, alpha, W, msqoc.SOLVER_FP64, col_block=5)


@pytest.mark.parametrize("solver", list(SOLVERS))
@pytest.mark.parametrize("cb", [5, 7])
def test_parity_tiles_over_ragged_windows_3q(cb, solver):
    """Two-window tiles whose windows differ in length by one step (2001 steps over 7 windows)."""
    spec = S.transmon_spec(3, 30.0, 2001, 7, 8)
    alpha, W = S.random_alpha(spec, 8), S.random_W(spec, 8)
    check(spec, alpha, W, SOLVERS[solver], col_block=cb)


def test_one_warp_tiles_must_not_cover_two_windows():
    spec = S.transmon_spec(3, 3.0, 200, 4, 5)     # 9 fibers a column: 3 columns = one warp
    with pytest.raises(msqoc.MsqocError):
        msqoc.Problem(spec, col_block=3, layout=msqoc.LAYOUT_FIBER)
    spec = S.transmon_spec(2, 3.0, 200, 4, 5)     # 3 fibers (6 threads) a column: 3 columns = one warp
    with pytest.raises(msqoc.MsqocError):
        msqoc.Problem(spec, col_block=3, layout=msqoc.LAYOUT_PAIR)


def test_column_block_beyond_the_tile_limit_is_rejected():
    spec = S.transmon_spec(4, 0.6, 100, 2, 4)
    for cb, layout in ((16, msqoc.LAYOUT_AUTO),     # 16 x 27 fibers > 384 threads, x 2 > 384
                       (10, msqoc.LAYOUT_FIBER),    # 270 > 256
                       (15, msqoc.LAYOUT_FIBER_LEAN),   # 405 > 384
                       (8, msqoc.LAYOUT_PAIR)):     # 432 > 384
        with pytest.raises(msqoc.MsqocError) as err:
            msqoc.Problem(spec, col_block=cb, layout=layout)
        assert err.value.status == -1
    with msqoc.Problem(spec, col_block=8) as p:    # automatic family: only one thread per fiber fits
        assert p.layout in (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_FIBER_LEAN)
    with msqoc.Problem(spec, col_block=12) as p:   # 324 threads: only the 168-register build
        assert p.layout == msqoc.LAYOUT_FIBER_LEAN
    with pytest.raises(msqoc.MsqocError) as err:
        msqoc.Problem(spec, layout=3)
    assert err.value.status == -1


def test_parity_5q_tiny():
    spec = S.transmon_spec(5, 0.12, 20, 2, 4)
    alpha, W = S.random_alpha(spec, 5), S.random_W(spec, 5)
    check(spec, alpha, W, msqoc.SOLVER_MIXED)


def test_single_shooting():
    spec = S.config_2q(M=1).replace(nsteps=500, T=12.5)
    alpha = S.random_alpha(spec, 3)
    check(spec, alpha, np.zeros(0), msqoc.SOLVER_MIXED)


def test_one_step_per_window():
    spec = S.transmon_spec(2, 0.4, 16, 16, 4)
    alpha, W = S.random_alpha(spec, 4), S.random_W(spec, 4)
    check(spec, alpha, W, msqoc.SOLVER_MIXED)
    check(spec, alpha, W, msqoc.SOLVER_FP64)


def test_zero_controls():
    spec = S.transmon_spec(3, 3.0, 200, 4, 5)
    alpha, W = np.zeros(spec.d), S.random_W(spec, 9)
    check(spec, alpha, W, msqoc.SOLVER_MIXED)


@pytest.mark.parametrize("solver", list(SOLVERS))
def test_strong_controls_need_more_iterations(solver):
    """Control amplitudes 25x the workload's: the contraction factor grows to ~1e-2 and the
    step solver must take more sweeps / refinement passes to stay at round-off."""
    spec = S.transmon_spec(2, 20.0, 800, 4, 6)
    alpha, W = S.random_alpha(spec, 12, amp=25 * S.ALPHA_AMP), S.random_W(spec, 12)
    check(spec, alpha, W, SOLVERS[solver])


def test_consistent_windows_have_zero_penalty():
    spec = S.transmon_spec(2, 20.0, 800, 5, 6)
    alpha = S.random_alpha(spec, 13)
    W = oracle.rollout(spec, alpha)
    got, want = check(spec, alpha, W, msqoc.SOLVER_MIXED)
    with msqoc.Problem(spec) as p:
        pen = p.eval_objective(alpha, W)["pen"]
    assert np.all(np.abs(pen) < 1e-24)


def test_solvers_agree_with_each_other():
    spec = S.transmon_spec(3, 30.0, 2000, 6, 8)
    alpha, W = S.random_alpha(spec, 14), S.random_W(spec, 14)
    with msqoc.Problem(spec, solver=msqoc.SOLVER_MIXED) as a, msqoc.Problem(spec, solver=msqoc.SOLVER_FP64) as b:
        ra, rb = a.eval_gradient(alpha, W), b.eval_gradient(alpha, W)
    assert_objective_close(ra["P"], rb["P"], rtol=1e-13)
    assert_grad_close(ra["grad_alpha"], rb["grad_alpha"], rtol=1e-11)
    assert_grad_close(ra["grad_W"], rb["grad_W"], rtol=1e-11)


def test_device_pointers_match_host_pointers():
    torch = pytest.importorskip("torch")
    spec = S.config_2q()
    alpha, W = S.random_alpha(spec, 15), S.random_W(spec, 15)
    with msqoc.Problem(spec) as p:
        host = p.eval_gradient(alpha, W)
        a_d = torch.tensor(alpha, device="cuda", dtype=torch.float64)
        W_d = torch.tensor(W, device="cuda", dtype=torch.float64)
        P_d = torch.zeros(1, device="cuda", dtype=torch.float64)
        ga_d = torch.zeros(p.d, device="cuda", dtype=torch.float64)
        gW_d = torch.zeros(p.nW, device="cuda", dtype=torch.float64)
        s = torch.cuda.current_stream()
        p.eval_gradient_into(a_d, W_d, P_d, ga_d, gW_d, stream=s)
        torch.cuda.synchronize()
    assert P_d.item() == host["P"]
    np.testing.assert_array_equal(ga_d.cpu().numpy(), host["grad_alpha"])
    np.testing.assert_array_equal(gW_d.cpu().numpy(), host["grad_W"])


def test_repeated_calls_are_bitwise_reproducible():
    spec = S.transmon_spec(3, 30.0, 1000, 4, 8)
    alpha, W = S.random_alpha(spec, 16), S.random_W(spec, 16)
    with msqoc.Problem(spec) as p:
        r1 = p.eval_gradient(alpha, W)
        r2 = p.eval_gradient(alpha, W)
    assert r1["P"] == r2["P"]
    np.testing.assert_array_equal(r1["grad_alpha"], r2["grad_alpha"])
    np.testing.assert_array_equal(r1["grad_W"], r2["grad_W"])

"""The autotuner: it times every admissible (kernel family, tile width) pair on a probe of the
problem and returns one of them; a problem built with the returned pair evaluates correctly."""
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


def test_autotune_returns_a_measured_admissible_width():
    spec = S.transmon_spec(3, 30.0, 2001, 7, 8)
    alpha, W = S.random_alpha(spec, 61), S.random_W(spec, 61)
    best, layout, sps, times = msqoc.autotune(spec, alpha=alpha, probe_steps=16)
    assert (layout, best, sps) in times and len(times) >= 6
    assert {lay for lay, _, _ in times} == {msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR,
                                            msqoc.LAYOUT_FIBER_LEAN}        # every family tried
    assert {dp for _, _, dp in times} >= {1, 2, 4}      # steps per synchronisation tried
    assert all(t > 0 for t in times.values())
    assert times[(layout, best, sps)] == min(times.values())
    _, lay1, sps1, times1 = msqoc.autotune(spec, alpha=alpha, probe_steps=16, layout=msqoc.LAYOUT_FIBER,
                                           steps_per_sync=2)
    assert lay1 == msqoc.LAYOUT_FIBER and {lay for lay, _, _ in times1} == {msqoc.LAYOUT_FIBER}
    assert sps1 == 2 and {dp for _, _, dp in times1} == {2}
    with msqoc.Problem(spec, col_block=best, layout=layout, steps_per_sync=sps) as p:
        assert p.steps_per_sync == sps
        got = p.eval_gradient(alpha, W)
    want = oracle.evaluate(spec, alpha, W)
    assert_objective_close(got["P"], want["P"])
    assert_grad_close(got["grad_alpha"], want["grad_alpha"])
    assert_grad_close(got["grad_W"], want["grad_W"])


def test_autotune_tries_lane_quads_on_two_levels():
    spec = S.paper_qft_spec(2, M=4, nsteps=400)
    best, layout, sps, times = msqoc.autotune(spec, probe_steps=16)
    assert {lay for lay, _, _ in times} == {msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_QUAD,
                                            msqoc.LAYOUT_FIBER_LEAN}
    assert times[(layout, best, sps)] == min(times.values())


def test_tile_model_picks_the_measured_fastest_tiles_of_the_benchmark_workload():
    # 4 transmons at 256 and 128 windows: 14-column tiles of the 168-register build, one of 12
    # warps to an SM, the autotuner's choice (probes at 256 windows: 2.78 ms against 2.93 for two
    # 7-column tiles an SM and 3.17 for the 255-register build's best, 9 columns); at 64 windows
    # (1024 columns, half the SMs for 14-column tiles) 8-column tiles of the 255-register build
    # (128 CTAs)
    with msqoc.Problem(S.config_4q(M=256)) as p:
        assert (p.layout, p.col_block, p.tiles) == (msqoc.LAYOUT_FIBER_LEAN, 14, 293)
    with msqoc.Problem(S.config_4q(M=128)) as p:
        assert (p.layout, p.col_block) == (msqoc.LAYOUT_FIBER_LEAN, 14)
    with msqoc.Problem(S.config_4q(M=64)) as p:
        assert (p.layout, p.col_block) == (msqoc.LAYOUT_FIBER, 8)

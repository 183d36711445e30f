"""The paper's own model (Eq. sys-ham, Table 1): 2-level qubits in a linear chain with
detuning and dipole exchange, QFT-4/8/16 targets, the paper's carriers and B-spline spacing.
The exchange is a constant off-diagonal part of the implicit step; parity against the oracle
(whose exchange construction is pinned by a kron-built Hamiltonian and finite differences)."""
import os

import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu

SOLVERS = {"mixed": msqoc.SOLVER_MIXED, "fp64": msqoc.SOLVER_FP64}


def families(spec):
    """The sweep kernel families a problem admits: lane quads need 2 levels and at most 6
    exchange-coupled pairs."""
    pairs = sum(1 for row in (spec.jx or []) for v in row if v != 0.0)
    quad = (msqoc.LAYOUT_QUAD,) if spec.L == 2 and pairs <= 6 else ()
    return (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_FIBER_LEAN) + quad


def check(spec, seed, solver=msqoc.SOLVER_DEFAULT, ckpt_interval=0, col_block=0, layouts=None):
    alpha, W = S.random_alpha(spec, seed), S.random_W(spec, seed)
    want = oracle.evaluate(spec, alpha, W, nthreads=os.cpu_count())
    for layout in layouts or families(spec):     # every sweep kernel family the problem admits
        with msqoc.Problem(spec, solver=solver, ckpt_interval=ckpt_interval, layout=layout,
                           col_block=col_block) as p:
            got = p.eval_gradient(alpha, W)
            obj = p.eval_objective(alpha, W)
        assert_objective_close(got["P"], want["P"])
        assert_objective_close(obj["J"], want["J"])
        assert_grad_close(got["grad_alpha"], want["grad_alpha"], what=f"grad_alpha (layout {layout})")
        if spec.M > 1:
            np.testing.assert_allclose(obj["pen"], want["pen"], rtol=1e-12, atol=1e-24)
            assert_grad_close(got["grad_W"], want["grad_W"], what=f"grad_W (layout {layout})")


@pytest.mark.parametrize("M", [1, 8, 64])
def test_qft4_full_time_grid(M):
    check(S.paper_qft_spec(2, M=M), 81)


def test_qft8_ragged_windows_and_checkpoints():
    spec = S.paper_qft_spec(3, M=13, nsteps=4001)
    check(spec, 82)
    check(spec, 82, ckpt_interval=7)


@pytest.mark.parametrize("solver", list(SOLVERS))
def test_qft16_short(solver):
    check(S.paper_qft_spec(4, M=4, nsteps=2000), 83, solver=SOLVERS[solver])


def test_qft16_tiles_over_two_windows():
    """5-column tiles (E = 16): 40 threads (one thread per fiber), 80 (lane pairs) or 160 (lane
    quads), tiles that cover the end of one window and the start of the next, with exchange
    coupling."""
    check(S.paper_qft_spec(4, M=5, nsteps=1001), 87, col_block=5)


@pytest.mark.parametrize("cb", [1, 2, 3, 4, 5, 6, 7, 8])
def test_qft8_lane_quad_tile_widths(cb):
    """Lane quads at every tile width of QFT-8 (16 threads a column): one-warp tiles (1, 2),
    tiles over two windows (3, 5, 6, 7), a ragged last tile (M E = 56 is not a multiple of 3, 5,
    6), ragged windows and checkpointed segments."""
    spec = S.paper_qft_spec(3, M=7, nsteps=803)
    check(spec, 88 + cb, col_block=cb, layouts=(msqoc.LAYOUT_QUAD,))
    if cb in (3, 8):
        check(spec, 88 + cb, col_block=cb, layouts=(msqoc.LAYOUT_QUAD,), ckpt_interval=9,
              solver=msqoc.SOLVER_FP64)


@pytest.mark.parametrize("q", [1, 2, 5, 6])
def test_two_level_shapes_every_family(q):
    """2-level subsystems at the edges of the compiled shapes: one qubit (one fiber a column, no
    neighbour subsystems), two, and five and six qubits (32 and 64 fibers a column, quads of up to
    256 threads a column); anharmonic transmon-style drift, cross-Kerr, no exchange."""
    spec = S.transmon_spec(q, 6.0, 240, 3, 5, L=2, ness=2)
    check(spec, 95 + q)


def test_lane_quads_rejected_where_not_admitted():
    """Lane quads serve 2-level subsystems with at most 6 exchange-coupled pairs."""
    three_levels = S.transmon_spec(2, 10.0, 100, 2, 5)
    base = S.paper_qft_spec(4, M=2, nsteps=100)
    q = 5
    jx = [[(0.03 if l > k else 0.0) for l in range(q)] for k in range(q)]     # 10 pairs
    omega = [list(base.omega[min(k, len(base.omega) - 1)]) for k in range(q)]
    ten_pairs = base.replace(q=q, xi=[0.0] * q, xi_cross=[[0.0] * q for _ in range(q)], omega=omega,
                             detune=[0.1 * k for k in range(q)], jx=jx)
    for spec in (three_levels, ten_pairs):
        with pytest.raises(msqoc.MsqocError) as err:
            msqoc.Problem(spec, layout=msqoc.LAYOUT_QUAD)
        assert err.value.status == -1
        with msqoc.Problem(spec) as p:                      # the automatic choice avoids them
            assert p.layout in (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_FIBER_LEAN)


@pytest.mark.parametrize("q", [4, 5])
def test_all_to_all_exchange(q):
    """Every pair of qubits coupled, with distinct strengths: 4 qubits give 6 pairs (sources
    precomputed per fiber, pairs with the last subsystem and pairs between fixed subsystems at
    every distance; all three kernel families), 5 qubits give 10 (more than the per-fiber list
    holds: the general form, one thread or a lane pair per fiber)."""
    base = S.paper_qft_spec(min(q, 4), M=3, nsteps=300)
    jx = [[(2 * np.pi * 0.004 * (1 + 0.3 * k + 0.1 * l) if l > k else 0.0) for l in range(q)] for k in range(q)]
    omega = [list(base.omega[min(k, len(base.omega) - 1)]) for k in range(q)]
    spec = base.replace(q=q, xi=[0.0] * q, xi_cross=[[0.0] * q for _ in range(q)], omega=omega,
                        detune=[2 * np.pi * 0.06 * (k - (q - 1) / 2) for k in range(q)], jx=jx, T=8.0)
    check(spec, 85)


def test_qft8_full_time_grid():
    """QFT-8 on the paper's full grid (19806 steps) at 32 windows, every kernel family."""
    spec = S.paper_qft_spec(3, M=32)
    check(spec, 86)


@pytest.mark.parametrize("M", [64, 256])
def test_qft16_full_size_sampled_windows(M):
    """QFT-16 at the paper's full size (106072 steps) over 64 windows and 256 (the paper's
    largest run), the library's choice of tiles: the last two windows against the oracle (J,
    pen_{M-1}, dP/dW^{M-1}), the gradients as a whole by central differences along seeded random
    directions."""
    spec = S.paper_qft_spec(4, M=M)
    alpha, W = S.random_alpha(spec, 84), S.random_W(spec, 84)
    M = spec.M
    with msqoc.Problem(spec) as p:
        got = p.eval_gradient(alpha, W)
        obj = p.eval_objective(alpha, W)
        rng = np.random.default_rng(19)
        va, vw = rng.standard_normal(spec.d), rng.standard_normal(spec.nW)
        ea, ew = 1e-6, 1e-7
        fd_a = (p.eval_objective(alpha + ea * va, W)["P"] - p.eval_objective(alpha - ea * va, W)["P"]) / (2 * ea)
        fd_w = (p.eval_objective(alpha, W + ew * vw)["P"] - p.eval_objective(alpha, W - ew * vw)["P"]) / (2 * ew)
    want = oracle.evaluate(spec, alpha, W, windows=(M - 1, M), nthreads=os.cpu_count())
    assert_objective_close(obj["J"], want["J"])
    np.testing.assert_allclose(obj["pen"][M - 2], want["pen"][M - 2], rtol=1e-12, atol=0)
    ne2 = 2 * spec.N * spec.E
    sl = slice((M - 2) * ne2, (M - 1) * ne2)
    assert_grad_close(got["grad_W"][sl], want["grad_W"][sl], what="grad_W^{M-1}")
    ga_v, gw_v = float(got["grad_alpha"] @ va), float(got["grad_W"] @ vw)
    assert abs(fd_a - ga_v) <= 1e-6 * abs(ga_v) + 16 * np.finfo(float).eps * abs(got["P"]) / ea, (fd_a, ga_v)
    assert abs(fd_w - gw_v) <= 1e-6 * abs(gw_v) + 16 * np.finfo(float).eps * abs(got["P"]) / ew, (fd_w, gw_v)


def test_exchange_on_three_levels_is_rejected():
    spec = S.transmon_spec(2, 10.0, 100, 2, 5).replace(jx=[[0.0, 0.03], [0.0, 0.0]])
    with pytest.raises(msqoc.MsqocError) as err:
        msqoc.Problem(spec)
    assert err.value.status == -6

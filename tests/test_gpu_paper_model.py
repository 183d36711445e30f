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


def check(spec, seed, solver=msqoc.SOLVER_DEFAULT, ckpt_interval=0, col_block=0):
    alpha, W = S.random_alpha(spec, seed), S.random_W(spec, seed)
    want = oracle.evaluate(spec, alpha, W, nthreads=os.cpu_count())
    for layout in (msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR):     # both sweep kernel families
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
    """5-column tiles (E = 16): 40 threads (one thread per fiber) or 80 (lane pairs), tiles that
    cover the end of one window and the start of the next, with exchange coupling."""
    check(S.paper_qft_spec(4, M=5, nsteps=1001), 87, col_block=5)


@pytest.mark.parametrize("q", [4, 5])
def test_all_to_all_exchange(q):
    """Every pair of qubits coupled, with distinct strengths: 4 qubits give 6 pairs (sources
    precomputed per fiber, pairs with the last subsystem and pairs between fixed subsystems at
    every distance), 5 qubits give 10 (more than the per-fiber list holds: the general form)."""
    base = S.paper_qft_spec(min(q, 4), M=3, nsteps=300)
    jx = [[(2 * np.pi * 0.004 * (1 + 0.3 * k + 0.1 * l) if l > k else 0.0) for l in range(q)] for k in range(q)]
    omega = [list(base.omega[min(k, len(base.omega) - 1)]) for k in range(q)]
    spec = base.replace(q=q, xi=[0.0] * q, xi_cross=[[0.0] * q for _ in range(q)], omega=omega,
                        detune=[2 * np.pi * 0.06 * (k - (q - 1) / 2) for k in range(q)], jx=jx, T=8.0)
    check(spec, 85)


def test_qft8_full_time_grid_pair_tiles():
    """QFT-8 on the paper's full grid (19806 steps) at 32 windows, the lane-pair kernels."""
    spec = S.paper_qft_spec(3, M=32)
    with msqoc.Problem(spec) as p:
        assert p.layout == msqoc.LAYOUT_PAIR
    check(spec, 86)


@pytest.mark.parametrize("M", [64, 256])
def test_qft16_full_size_sampled_windows(M):
    """QFT-16 at the paper's full size (106072 steps) over 64 windows (lane-pair tiles) and 256
    (the paper's largest run; one thread per fiber): the last two windows against the oracle (J,
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

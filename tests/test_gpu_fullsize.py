"""Full-size parity on the 4-transmon benchmark workload (N=81, E=16, T=600 ns, 100000 steps,
d=640) in the launch configuration the benchmark times (automatic column block, default
solver).  The oracle evaluates every window on all host cores (about 4 s per window per core),
so every output is compared, not a sample."""
import os

import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


_ORACLE = {}


def oracle_4q(M):
    """The oracle's full evaluation of the 4-transmon workload (seed 1), computed once per M."""
    if M not in _ORACLE:
        spec = S.config_4q(M=M)
        alpha, W = S.random_alpha(spec, 1), S.random_W(spec, 1)
        _ORACLE[M] = (spec, alpha, W, oracle.evaluate(spec, alpha, W, nthreads=os.cpu_count()))
    return _ORACLE[M]


@pytest.mark.parametrize("M,cb,layout", [(64, 0, 0), (256, 0, 0), (256, 9, msqoc.LAYOUT_FIBER),
                                         (256, 7, msqoc.LAYOUT_FIBER_LEAN), (256, 14, msqoc.LAYOUT_FIBER_LEAN)])
def test_fullsize_4q(M, cb, layout):
    """The library's tiles (at 256 windows 7-column tiles of the 168-register build, two to an
    SM: 586 tiles over two windows), 9-column tiles of the 255-register build (456 tiles: three
    waves of 152) and 14-column tiles (378 threads, 12 warps)."""
    spec, alpha, W, want = oracle_4q(M)
    with msqoc.Problem(spec, col_block=cb, layout=layout) as p:
        got = p.eval_gradient(alpha, W)
        obj = p.eval_objective(alpha, W)
    assert_objective_close(got["P"], want["P"])
    assert_objective_close(obj["J"], want["J"])
    np.testing.assert_allclose(obj["pen"], want["pen"], rtol=1e-12, atol=0)
    assert_grad_close(got["grad_alpha"], want["grad_alpha"], what="grad_alpha")
    assert_grad_close(got["grad_W"], want["grad_W"], what="grad_W")


def test_fullsize_4q_fp64_solver():
    """The pure-FP64 fixed-point step solver on the full 4-transmon workload at 64 windows,
    against the complete oracle."""
    spec, alpha, W, want = oracle_4q(64)
    with msqoc.Problem(spec, solver=msqoc.SOLVER_FP64) as p:
        got = p.eval_gradient(alpha, W)
    assert_objective_close(got["P"], want["P"])
    assert_grad_close(got["grad_alpha"], want["grad_alpha"], what="grad_alpha")
    assert_grad_close(got["grad_W"], want["grad_W"], what="grad_W")


def test_fullsize_5q_every_midpoint_kept_equals_checkpointed():
    """The 5-transmon workload with every midpoint state kept (K = 1: an 18.7 GB history) and
    with checkpoint interval 64: the same arithmetic, so the same outputs."""
    spec = S.config_5q()
    alpha, W = S.random_alpha(spec, 3), S.random_W(spec, 3)
    with msqoc.Problem(spec, ckpt_interval=1) as p1:
        assert p1.ckpt_interval == 1
        g1 = p1.eval_gradient(alpha, W)
    with msqoc.Problem(spec, ckpt_interval=64) as p64:
        g64 = p64.eval_gradient(alpha, W)
    assert_objective_close(g1["P"], g64["P"])
    assert_grad_close(g1["grad_alpha"], g64["grad_alpha"], what="grad_alpha (K=1 vs 64)")
    assert_grad_close(g1["grad_W"], g64["grad_W"], what="grad_W (K=1 vs 64)")


def test_fullsize_5q_sampled_windows_and_directional_derivatives():
    """The 5-transmon serving workload at full size (N=243, E=32, T=800 ns, 150000 steps,
    M=256, d=1060) with the forced checkpoint interval 64.  The oracle's cost per step is too
    high for all windows, so it evaluates the last two: J, pen_255 and dP/dW^255 (which needs
    Lambda^256 at t_255) are compared element by element.  The alpha- and W-gradients as a
    whole are checked by the property that holds at any size: central differences of the GPU
    objective along seeded random directions equal the gradient's projections."""
    spec = S.config_5q()
    alpha, W = S.random_alpha(spec, 3), S.random_W(spec, 3)
    M = spec.M
    with msqoc.Problem(spec, ckpt_interval=64) as p:
        got = p.eval_gradient(alpha, W)
        obj = p.eval_objective(alpha, W)
        rng = np.random.default_rng(17)
        va = rng.standard_normal(spec.d)
        vw = rng.standard_normal(spec.nW)
        eps_a, eps_w = 1e-6, 1e-7
        fd_a = (p.eval_objective(alpha + eps_a * va, W)["P"] - p.eval_objective(alpha - eps_a * va, W)["P"]) / (2 * eps_a)
        fd_w = (p.eval_objective(alpha, W + eps_w * vw)["P"] - p.eval_objective(alpha, W - eps_w * vw)["P"]) / (2 * eps_w)
    assert_objective_close(obj["P"], got["P"])
    want = oracle.evaluate(spec, alpha, W, windows=(M - 1, M), nthreads=os.cpu_count())
    assert_objective_close(obj["J"], want["J"])
    np.testing.assert_allclose(obj["pen"][M - 2], want["pen"][M - 2], rtol=1e-12, atol=0)
    ne2 = 2 * spec.N * spec.E
    sl = slice((M - 2) * ne2, (M - 1) * ne2)     # W^{M-1}
    assert_grad_close(got["grad_W"][sl], want["grad_W"][sl], what="grad_W^{M-1}")
    # directional derivatives: round-off of P over the step, plus the truncation bound
    ga_v, gw_v = float(got["grad_alpha"] @ va), float(got["grad_W"] @ vw)
    tol_a = 1e-6 * abs(ga_v) + 16 * np.finfo(float).eps * abs(got["P"]) / eps_a
    tol_w = 1e-6 * abs(gw_v) + 16 * np.finfo(float).eps * abs(got["P"]) / eps_w
    assert abs(fd_a - ga_v) <= tol_a, (fd_a, ga_v)
    assert abs(fd_w - gw_v) <= tol_w, (fd_w, gw_v)


@pytest.mark.parametrize("K", [64, 512])
def test_fullsize_4q_checkpoint_intervals_at_128_windows(K):
    """The 4-transmon workload at 128 windows (781-782 steps each) with checkpoint interval K
    (64: 13 segments per window; 512: a long and a short segment): every output equals the
    K = 1 evaluation (the recomputed segments repeat the same arithmetic), and the last two
    windows match the oracle (J, pen_127, dP/dW^127)."""
    spec = S.config_4q(M=128)
    alpha, W = S.random_alpha(spec, 4), S.random_W(spec, 4)
    M = spec.M
    with msqoc.Problem(spec, ckpt_interval=1) as p1:
        ref = p1.eval_gradient(alpha, W)
    with msqoc.Problem(spec, ckpt_interval=K) as pk:
        assert pk.ckpt_interval == K
        got = pk.eval_gradient(alpha, W)
        obj = pk.eval_objective(alpha, W)
    assert_objective_close(got["P"], ref["P"])
    assert_grad_close(got["grad_alpha"], ref["grad_alpha"], what=f"grad_alpha (K={K} vs 1)")
    assert_grad_close(got["grad_W"], ref["grad_W"], what=f"grad_W (K={K} vs 1)")
    want = oracle.evaluate(spec, alpha, W, windows=(M - 1, M), nthreads=os.cpu_count())
    assert_objective_close(obj["J"], want["J"])
    np.testing.assert_allclose(obj["pen"][M - 2], want["pen"][M - 2], rtol=1e-12, atol=0)
    ne2 = 2 * spec.N * spec.E
    sl = slice((M - 2) * ne2, (M - 1) * ne2)
    assert_grad_close(got["grad_W"][sl], want["grad_W"][sl], what="grad_W^{M-1}")

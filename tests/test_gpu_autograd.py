"""The adjoint kernel through torch.autograd: central finite differences of the GPU objective on
seeded coordinates (3-transmon workload: N=27, E=8, 20000 steps, M=32, step 1e-6) and the
oracle's gradient."""
import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _inputs(spec, seed):
    alpha, W = S.random_alpha(spec, seed), S.random_W(spec, seed)
    a = torch.tensor(alpha, device="cuda", dtype=torch.float64, requires_grad=True)
    w = torch.tensor(W, device="cuda", dtype=torch.float64, requires_grad=True)
    return alpha, W, a, w


def test_autograd_matches_oracle_and_finite_differences():
    from paper_2407_13950_gb300.autograd import ms_objective
    spec = S.config_3q()
    alpha, W, a, w = _inputs(spec, 202)
    with msqoc.Problem(spec) as prob:
        P = ms_objective(prob, a, w)
        (2.5 * P).backward()
        ga = a.grad.detach().cpu().numpy() / 2.5
        gw = w.grad.detach().cpu().numpy() / 2.5
        want = oracle.evaluate(spec, alpha, W)
        assert_objective_close(P.item(), want["P"])
        assert_grad_close(ga, want["grad_alpha"], what="grad_alpha")
        assert_grad_close(gw, want["grad_W"], what="grad_W")

        # central differences of the GPU objective on 50 seeded coordinates of (alpha, W)
        rng = np.random.default_rng(50)
        n_a = 25
        idx_a = rng.choice(spec.d, n_a, replace=False)
        idx_w = rng.choice(spec.nW, 50 - n_a, replace=False)
        eps = 1e-6
        # central differences carry the objective's round-off divided by the step: a few ulps
        # of P (~1e-14 for P ~ 60) over 2 eps; 1e-6 relative covers the truncation error
        fd_floor = 8 * np.finfo(float).eps * abs(P.item()) / eps
        a0 = torch.tensor(alpha, device="cuda", dtype=torch.float64)
        w0 = torch.tensor(W, device="cuda", dtype=torch.float64)

        def P_of(av, wv):
            with torch.no_grad():
                return ms_objective(prob, av, wv).item()

        for l in idx_a:
            ap, am = a0.clone(), a0.clone()
            ap[l] += eps
            am[l] -= eps
            fd = (P_of(ap, w0) - P_of(am, w0)) / (2 * eps)
            assert abs(fd - ga[l]) <= 1e-6 * abs(ga[l]) + fd_floor, (l, fd, ga[l])
        for l in idx_w:
            wp, wm = w0.clone(), w0.clone()
            wp[l] += eps
            wm[l] -= eps
            fd = (P_of(a0, wp) - P_of(a0, wm)) / (2 * eps)
            assert abs(fd - gw[l]) <= 1e-6 * abs(gw[l]) + fd_floor, (l, fd, gw[l])


def test_objective_only_when_no_grad_is_needed():
    from paper_2407_13950_gb300.autograd import ms_objective
    spec = S.config_2q()
    alpha, W = S.random_alpha(spec, 9), S.random_W(spec, 9)
    a = torch.tensor(alpha, device="cuda", dtype=torch.float64)
    w = torch.tensor(W, device="cuda", dtype=torch.float64)
    with msqoc.Problem(spec) as prob:
        P = ms_objective(prob, a, w)
        assert not P.requires_grad
        assert_objective_close(P.item(), oracle.evaluate(spec, alpha, W, grad=False)["P"])

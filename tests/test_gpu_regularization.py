"""Regularization of the optimisation problem (Sec. 5: Tikhonov term and control-pulse energy)
on the GPU against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu

CASES = [
    ("2q-ragged", S.transmon_spec(2, 17.3, 1001, 3, 7)),                  # dtau / h not an integer
    ("3q-few-splines", S.transmon_spec(3, 5.0, 333, 2, 3)),               # d1 = 3: one spline start
    ("QFT-4", S.paper_qft_spec(2, M=4)),                                  # the paper's grid and carriers
    ("QFT-8", S.paper_qft_spec(3, M=8)),
]


@pytest.mark.parametrize("name,spec", CASES, ids=[c[0] for c in CASES])
def test_regularization_matches_oracle(name, spec):
    alpha = S.random_alpha(spec, 31, amp=S.PAPER_ALPHA0_AMP)
    gt, ge = 1e-3 / spec.d, 1e-3
    R_want, g_want = oracle.regularization(spec, alpha, gt, ge)
    with msqoc.Problem(spec) as p:
        got = p.eval_regularization(alpha, gt, ge)
    assert_objective_close(got["R"], R_want)
    assert_grad_close(got["grad_alpha"], g_want, what="dR/dalpha")


def test_regularization_terms_separately_and_device_outputs_bitwise():
    spec = S.paper_qft_spec(2, M=4)
    alpha = S.random_alpha(spec, 32, amp=S.PAPER_ALPHA0_AMP)
    with msqoc.Problem(spec) as p:
        tik = p.eval_regularization(alpha, 0.5, 0.0)
        assert tik["R"] == pytest.approx(0.25 * float(alpha @ alpha), rel=1e-14)
        np.testing.assert_array_equal(tik["grad_alpha"], 0.5 * alpha)
        en = p.eval_regularization(alpha, 0.0, 1.0)
        R_want, g_want = oracle.regularization(spec, alpha, 0.0, 1.0)
        assert_objective_close(en["R"], R_want)
        assert_grad_close(en["grad_alpha"], g_want)
        both = p.eval_regularization(alpha, 0.5, 1.0)
        dev = torch.device("cuda")
        a_d = torch.tensor(alpha, device=dev)
        R_d = torch.full((1,), np.nan, device=dev, dtype=torch.float64)
        g_d = torch.full((spec.d,), np.nan, device=dev, dtype=torch.float64)
        p.eval_regularization_into(a_d, 0.5, 1.0, R_d, g_d, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert R_d.item() == both["R"]                               # fixed-order sums: bitwise
        np.testing.assert_array_equal(g_d.cpu().numpy(), both["grad_alpha"])


def test_regularization_leaves_the_last_evaluation_alone():
    spec = S.transmon_spec(2, 16.0, 320, 4, 6)
    alpha, W = S.random_alpha(spec, 33), S.random_W(spec, 33)
    with msqoc.Problem(spec) as p:
        p.eval_objective(alpha, W)
        est = p.rollout_estimate()
        p.eval_regularization(S.random_alpha(spec, 34), 1.0, 1.0)
        assert p.rollout_estimate() == est
        g1 = p.eval_gradient(alpha, W)
        p.eval_regularization(S.random_alpha(spec, 35), 1.0, 1.0)
        g2 = p.eval_gradient(alpha, W)
    np.testing.assert_array_equal(g1["grad_alpha"], g2["grad_alpha"])


def test_regularization_rejects_negative_or_infinite_weights():
    spec = S.transmon_spec(1, 5.0, 50, 1, 4)
    alpha = S.random_alpha(spec, 1)
    with msqoc.Problem(spec) as p:
        for gt, ge in [(-1.0, 0.0), (0.0, -1e-3), (np.inf, 0.0), (0.0, np.nan)]:
            with pytest.raises(msqoc.MsqocError) as err:
                p.eval_regularization(alpha, gt, ge)
            assert err.value.status == -1

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


@pytest.mark.parametrize("M", [64, 256])
def test_fullsize_4q(M):
    spec = S.config_4q(M=M)
    alpha, W = S.random_alpha(spec, 1), S.random_W(spec, 1)
    with msqoc.Problem(spec) as p:
        got = p.eval_gradient(alpha, W)
        obj = p.eval_objective(alpha, W)
    want = oracle.evaluate(spec, alpha, W, nthreads=os.cpu_count())
    assert_objective_close(got["P"], want["P"])
    assert_objective_close(obj["J"], want["J"])
    np.testing.assert_allclose(obj["pen"], want["pen"], rtol=1e-12, atol=0)
    assert_grad_close(got["grad_alpha"], want["grad_alpha"], what="grad_alpha")
    assert_grad_close(got["grad_W"], want["grad_W"], what="grad_W")

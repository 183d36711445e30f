"""Batched evaluation (msqoc_batch_*): several problems of several shapes, durations, window
counts and checkpoint intervals in shared sweep launches, eagerly and replayed from a CUDA
graph.  Every problem's result must equal its own single evaluation within the parity
tolerance (the tiles of a problem are its own; only their scheduling changes), and a graph
replay must read the inputs staged before it."""
import numpy as np
import pytest

import oracle
from paper_2407_13950_gb300 import msqoc
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


def mixed_specs():
    base2 = S.transmon_spec(2, 20.0, 800, 4, 6)
    base3 = S.transmon_spec(3, 6.0, 400, 4, 5)
    base4 = S.transmon_spec(4, 1.2, 200, 2, 4)
    return [S.perturbed_duration_spec(base2, 0.75, 4), S.perturbed_duration_spec(base2, 1.3, 8),
            S.perturbed_duration_spec(base3, 1.0, 3), S.perturbed_duration_spec(base3, 0.6, 5),
            S.perturbed_duration_spec(base4, 1.0, 2), S.perturbed_duration_spec(base4, 1.5, 3)]


def single(spec, alpha, W, **kw):
    with msqoc.Problem(spec, **kw) as p:
        return p.eval_gradient(alpha, W), p.eval_objective(alpha, W)


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_single_evaluations(graph):
    specs = mixed_specs()
    probs = [msqoc.Problem(sp) for sp in specs]
    try:
        with msqoc.Batch(probs, gradient=True, graph=graph) as b:
            for rep, seed in enumerate((31, 32, 33)):      # graph replays with new inputs
                inputs = [(S.random_alpha(sp, seed, problem=i), S.random_W(sp, seed, problem=i))
                          for i, sp in enumerate(specs)]
                for i, (a, W) in enumerate(inputs):
                    b.set_inputs(i, a, W)
                b.eval_gradient()
                got = [b.get_gradient(i) for i in range(len(specs))]
                b.eval_objective()
                obj = [b.get_objective(i) for i in range(len(specs))]
                for i, sp in enumerate(specs):
                    want_g, want_o = single(sp, *inputs[i])
                    assert_objective_close(got[i]["P"], want_g["P"])
                    assert_grad_close(got[i]["grad_alpha"], want_g["grad_alpha"], what=f"grad_alpha[{i}]")
                    assert_grad_close(got[i]["grad_W"], want_g["grad_W"], what=f"grad_W[{i}]")
                    assert_objective_close(obj[i]["P"], want_o["P"])
                    np.testing.assert_allclose(obj[i]["pen"], want_o["pen"], rtol=1e-12, atol=1e-24)
    finally:
        for p in probs:
            p.close()


def test_batch_against_oracle_with_mixed_checkpoint_intervals():
    base = S.transmon_spec(3, 30.0, 2001, 7, 8)
    specs = [base, S.perturbed_duration_spec(base, 0.8, 5)]
    probs = [msqoc.Problem(specs[0], ckpt_interval=1), msqoc.Problem(specs[1], ckpt_interval=64)]
    try:
        with msqoc.Batch(probs, gradient=True, graph=True) as b:
            inputs = [(S.random_alpha(sp, 41, problem=i), S.random_W(sp, 41, problem=i))
                      for i, sp in enumerate(specs)]
            for i, (a, W) in enumerate(inputs):
                b.set_inputs(i, a, W)
            b.eval_gradient()
            for i, sp in enumerate(specs):
                got = b.get_gradient(i)
                want = oracle.evaluate(sp, *inputs[i])
                assert_objective_close(got["P"], want["P"])
                assert_grad_close(got["grad_alpha"], want["grad_alpha"], what=f"grad_alpha[{i}]")
                assert_grad_close(got["grad_W"], want["grad_W"], what=f"grad_W[{i}]")
    finally:
        for p in probs:
            p.close()


def test_gradient_batch_needs_the_gradient_flag():
    spec = S.transmon_spec(2, 5.0, 100, 2, 4)
    with msqoc.Problem(spec) as p, msqoc.Batch([p], gradient=False) as b:
        b.set_inputs(0, S.random_alpha(spec, 1), S.random_W(spec, 1))
        with pytest.raises(msqoc.MsqocError):
            b.eval_gradient()
        b.eval_objective()
        assert np.isfinite(b.get_objective(0)["P"])


def test_subsets_on_two_streams_match_single_evaluations():
    """Continuous-batching step: two disjoint subsets of one batch evaluated at the same time on
    two streams (different staging slots), then a third subset reusing slot 0."""
    import torch
    specs = mixed_specs()
    probs = [msqoc.Problem(sp) for sp in specs]
    try:
        with msqoc.Batch(probs, gradient=True) as b:
            inputs = [(S.random_alpha(sp, 51, problem=i), S.random_W(sp, 51, problem=i))
                      for i, sp in enumerate(specs)]
            s0, s1 = torch.cuda.Stream(), torch.cuda.Stream()
            for i, (a, W) in enumerate(inputs):
                b.set_inputs(i, a, W, stream=s0 if i % 2 == 0 else s1)
            b.eval_subset([0, 2, 4], gradient=True, slot=0, stream=s0)
            b.eval_subset([1, 3, 5], gradient=False, slot=1, stream=s1)
            torch.cuda.synchronize()
            got = {i: b.get_gradient(i) for i in (0, 2, 4)}
            obj = {i: b.get_objective(i) for i in (1, 3, 5)}
            b.eval_subset([5, 1], gradient=True, slot=0, stream=s0)
            torch.cuda.synchronize()
            got.update({i: b.get_gradient(i) for i in (1, 5)})
            for i, res in got.items():
                want, _ = single(specs[i], *inputs[i])
                assert_objective_close(res["P"], want["P"])
                assert_grad_close(res["grad_alpha"], want["grad_alpha"], what=f"grad_alpha[{i}]")
                assert_grad_close(res["grad_W"], want["grad_W"], what=f"grad_W[{i}]")
            for i, res in obj.items():
                _, want = single(specs[i], *inputs[i])
                assert_objective_close(res["P"], want["P"])
    finally:
        for p in probs:
            p.close()


def test_batch_mixes_kernel_families():
    """Problems of one shape built with different kernel families (one thread, a lane pair and
    a lane quad per fiber) go to separate launch groups of one batch; each equals its single
    evaluation."""
    q8 = S.paper_qft_spec(3, M=4, nsteps=400)
    items = [(q8, msqoc.LAYOUT_QUAD), (q8.replace(M=3), msqoc.LAYOUT_PAIR), (q8.replace(M=5), msqoc.LAYOUT_FIBER),
             (S.paper_qft_spec(2, M=6, nsteps=300), msqoc.LAYOUT_QUAD), (S.transmon_spec(2, 20.0, 800, 4, 6), 0)]
    probs = [msqoc.Problem(sp, layout=lay) for sp, lay in items]
    try:
        assert [p.layout for p in probs[:3]] == [msqoc.LAYOUT_QUAD, msqoc.LAYOUT_PAIR, msqoc.LAYOUT_FIBER]
        inputs = [(S.random_alpha(sp, 41, problem=i), S.random_W(sp, 41, problem=i)) for i, (sp, _) in enumerate(items)]
        with msqoc.Batch(probs, gradient=True) as b:
            for i, (a, W) in enumerate(inputs):
                b.set_inputs(i, a, W)
            b.eval_gradient()
            got = [b.get_gradient(i) for i in range(len(items))]
        for i, (sp, lay) in enumerate(items):
            want, _ = single(sp, *inputs[i], layout=lay)
            assert_objective_close(got[i]["P"], want["P"])
            assert_grad_close(got[i]["grad_alpha"], want["grad_alpha"], what=f"grad_alpha[{i}]")
            assert_grad_close(got[i]["grad_W"], want["grad_W"], what=f"grad_W[{i}]")
    finally:
        for p in probs:
            p.close()


def test_batched_workload_at_full_size_matches_alone_and_the_oracle():
    # the batched workload as benchmarked: 32 x 2q + 32 x 3q + 32 x 4q, durations uniform in
    # [0.5 T, 1.5 T], windows in {8, 32, 64, 128}, one graph-replayed batch
    specs = S.mixed_batch_specs(seed=1, n_per_shape=32, shapes=[S.config_2q(), S.config_3q(), S.config_4q()])
    inputs = [(S.random_alpha(sp, 1, problem=i), S.random_W(sp, 1, problem=i)) for i, sp in enumerate(specs)]
    probs = [msqoc.Problem(sp) for sp in specs]
    try:
        with msqoc.Batch(probs, gradient=True, graph=True) as b:
            for i, (a, W) in enumerate(inputs):
                b.set_inputs(i, a, W)
            b.eval_gradient()
            got = [b.get_gradient(i) for i in range(len(specs))]
        for i, p in enumerate(probs):
            want = p.eval_gradient(*inputs[i])
            assert_objective_close(got[i]["P"], want["P"])
            assert_grad_close(got[i]["grad_alpha"], want["grad_alpha"], what=f"grad_alpha[{i}]")
            assert_grad_close(got[i]["grad_W"], want["grad_W"], what=f"grad_W[{i}]")
    finally:
        for p in probs:
            p.close()
    # a member of each shape against the oracle (the one the oracle finishes first)
    ncores = oracle.default_threads()
    for q in (2, 3, 4):
        i = min((k for k, sp in enumerate(specs) if sp.q == q),
                key=lambda k: specs[k].nsteps / min(specs[k].M, ncores))
        want = oracle.evaluate(specs[i], *inputs[i])
        assert_objective_close(got[i]["P"], want["P"])
        assert_grad_close(got[i]["grad_alpha"], want["grad_alpha"], what=f"oracle grad_alpha[{i}]")
        assert_grad_close(got[i]["grad_W"], want["grad_W"], what=f"oracle grad_W[{i}]")

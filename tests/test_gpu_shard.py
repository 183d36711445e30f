"""Shards (window ranges) of one problem through the C ABI: evaluated one after another on one
GPU and recombined (`shard.combine`), and as two gloo ranks sharing the GPU (the distributed
exchange of `shard.ShardedProblem`; the ranks' kernels never wait on each other, the hand-off
and the reduction go through host memory).  A shard runs the same per-column arithmetic as the
whole problem (same kernel family), so the window end states, adjoint states, penalties and
dP/dW agree bitwise; P and dP/dalpha are sums over tiles and shards, equal up to their order."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2407_13950_gb300 import msqoc, shard
from paper_2407_13950_gb300 import synthetic as S

from gpu_helpers import assert_grad_close, assert_objective_close

pytestmark = pytest.mark.gpu


def whole(spec, alpha, W, **kw):
    with msqoc.Problem(spec, **kw) as p:
        return p.eval_gradient(alpha, W), p.eval_objective(alpha, W)


def shards(spec, alpha, W, world, **kw):
    parts, objs = [], []
    for first, last in shard.partition(spec.M, world):
        lo, hi = shard.w_slice(spec, first, last)
        with msqoc.Problem(spec, windows=(first, last), **kw) as p:
            assert p.nW == hi - lo
            parts.append(((first, last), p.eval_gradient(alpha, W[lo:hi])))
            objs.append(p.eval_objective(alpha, W[lo:hi]))
    return shard.combine(spec, parts), objs


@pytest.mark.parametrize("layout", [msqoc.LAYOUT_FIBER, msqoc.LAYOUT_PAIR])
@pytest.mark.parametrize("world", [2, 3, 7])
def test_shards_on_one_gpu_recombine_to_the_whole_problem_and_the_oracle(world, layout):
    spec = S.transmon_spec(3, 30.0, 2000, 7, 8)
    alpha, W = S.random_alpha(spec, 12), S.random_W(spec, 12)
    want_g, want_o = whole(spec, alpha, W, layout=layout)
    got, objs = shards(spec, alpha, W, world, layout=layout)
    np.testing.assert_array_equal(got["grad_W"], want_g["grad_W"])
    assert_objective_close(got["P"], want_g["P"], rtol=1e-14)
    assert_grad_close(got["grad_alpha"], want_g["grad_alpha"], rtol=1e-13, floor=1e-15)
    np.testing.assert_array_equal(np.concatenate([o["pen"] for o in objs]), want_o["pen"])
    assert objs[-1]["J"] == want_o["J"] and all(o["J"] == 0.0 for o in objs[:-1])
    ref = oracle.evaluate(spec, alpha, W)
    assert_objective_close(got["P"], ref["P"])
    assert_grad_close(got["grad_alpha"], ref["grad_alpha"], what="grad_alpha")
    assert_grad_close(got["grad_W"], ref["grad_W"], what="grad_W")


def test_full_size_4q_in_two_shards_with_checkpointing():
    spec = S.config_4q(M=64)
    alpha, W = S.random_alpha(spec, 13), S.random_W(spec, 13)
    want_g, _ = whole(spec, alpha, W, layout=msqoc.LAYOUT_FIBER, col_block=8, ckpt_interval=64)
    got, _ = shards(spec, alpha, W, 2, layout=msqoc.LAYOUT_FIBER, col_block=8, ckpt_interval=64)
    np.testing.assert_array_equal(got["grad_W"], want_g["grad_W"])
    assert_objective_close(got["P"], want_g["P"], rtol=1e-14)
    assert_grad_close(got["grad_alpha"], want_g["grad_alpha"], rtol=1e-13, floor=1e-15)


def test_shard_arguments_and_whole_problem_only_calls():
    spec = S.transmon_spec(2, 10.0, 400, 4, 6)
    for bad in ((0, 2), (2, 1), (3, 5), (1, 0)):
        with pytest.raises(msqoc.MsqocError) as e:
            msqoc.Problem(spec, windows=bad)
        assert e.value.status == -1
    with msqoc.Problem(spec, windows=(2, 3)) as p:
        assert p.nW == 3 * 2 * spec.N * spec.E and p.npen == 2
        with pytest.raises(msqoc.MsqocError) as e:
            p.rollout(S.random_alpha(spec, 1))
        assert e.value.status == -6
        with pytest.raises(msqoc.MsqocError) as e:
            msqoc.Batch([p])
        assert e.value.status == -6
    with msqoc.Problem(spec, windows=(1, spec.M)) as p:      # the whole range is a whole problem
        assert p.nW == spec.nW
        p.rollout(S.random_alpha(spec, 1))


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = S.transmon_spec(3, 30.0, 2000, 7, 8)
        alpha, W = S.random_alpha(spec, 14), S.random_W(spec, 14)
        sp = shard.ShardedProblem(spec, dist, layout=msqoc.LAYOUT_FIBER)
        g = sp.eval_gradient(alpha, W)
        full = sp.gather_grad_W(g["grad_W_own"])
        sp.close()
        out.put((rank, g["P"], g["grad_alpha"], full))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharing_the_gpu_match_the_whole_problem():
    spec = S.transmon_spec(3, 30.0, 2000, 7, 8)
    alpha, W = S.random_alpha(spec, 14), S.random_W(spec, 14)
    want, _ = whole(spec, alpha, W, layout=msqoc.LAYOUT_FIBER)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, P, ga, gW in res:
        np.testing.assert_array_equal(gW, want["grad_W"])
        assert_objective_close(P, want["P"], rtol=1e-14)
        assert_grad_close(ga, want["grad_alpha"], rtol=1e-13, floor=1e-15)

"""One problem's windows sharded over ranks, on CPU: gloo ranks (127.0.0.1) whose compute is
the oracle on their window range, and the exchange of `shard.ShardedProblem` (the hand-off of
-2 Lambda^{b+1}(t_b) across each rank boundary b, one all-reduce of d + 1 doubles, the gather of
dP/dW).  The result must be the single-process oracle's: dP/dW and every penalty bitwise (the
boundary sum mu (W - U) + (-2 Lambda) is the oracle's own expression), P and dP/dalpha up to
the order of the cross-rank sum."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_2407_13950_gb300 import shard  # noqa: E402
from paper_2407_13950_gb300 import synthetic as S  # noqa: E402


def spec_small():
    return S.transmon_spec(2, 12.0, 480, 7, 6)


def oracle_evaluator(spec, first, last):
    """A rank's compute from the oracle: the library shard's outputs for windows first..last."""
    import oracle
    nb = 2 * spec.N * spec.E
    lo, hi = shard.w_slice(spec, first, last)
    k0, k1 = max(first - 1, 1), min(last, spec.M - 1)
    mu = spec.mu if spec.mu > 0 else 2.0 / spec.E          # the default weight (Sec. 5)

    def evaluate(alpha, W_slice, gradient=True):
        W = np.zeros(spec.nW)
        W[lo:hi] = W_slice
        o = oracle.evaluate(spec, alpha, W, windows=(first, last), per_window=True, nthreads=2)
        if not gradient:
            return {"P": o["P"], "J": o["J"], "pen": o["pen"][first - 1:min(last, spec.M - 1)]}
        gW = np.zeros(max(hi - lo, 0))
        for k in range(k0, k1 + 1):
            blk = slice((k - k0) * nb, (k - k0 + 1) * nb)
            src = slice((k - 1) * nb, k * nb)
            if first <= k and k + 1 <= last:
                gW[blk] = o["grad_W"][src]                      # mu (W - U) - 2 Lambda, both own
            elif first <= k:
                gW[blk] = mu * (W[src] - o["Uend"][src])
            else:
                gW[blk] = -(2.0 * o["Lam0"][k * nb:(k + 1) * nb])
        return {"P": o["P"], "grad_alpha": o["grad_alpha"], "grad_W": gW}

    return evaluate


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = spec_small()
        alpha, W = S.random_alpha(spec, 4), S.random_W(spec, 4)
        first, last = shard.partition(spec.M, world)[rank]
        sp = shard.ShardedProblem(spec, dist, evaluate=oracle_evaluator(spec, first, last))
        g = sp.eval_gradient(alpha, W)
        full = sp.gather_grad_W(g["grad_W_own"])
        o = sp.eval_objective(alpha, W)
        out.put((rank, g["P"], g["grad_alpha"], full, o["P"], o["J"], o["pen_own"]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_is_contiguous_and_balanced():
    for M in (1, 2, 7, 64, 256):
        for world in range(1, min(M, 9) + 1):
            r = shard.partition(M, world)
            assert r[0][0] == 1 and r[-1][1] == M
            assert all(b[0] == a[1] + 1 for a, b in zip(r, r[1:]))
            sizes = [b - a + 1 for a, b in r]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        shard.partition(3, 4)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_evaluation_recombines_to_the_single_process_oracle(world):
    import oracle
    spec = spec_small()
    alpha, W = S.random_alpha(spec, 4), S.random_W(spec, 4)
    want = oracle.evaluate(spec, alpha, W, nthreads=2)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, P, ga, gW, Po, J, pen in res:
        # every rank holds the same reduced values and the same gathered dP/dW
        assert P == res[0][1] and np.array_equal(ga, res[0][2]) and np.array_equal(gW, res[0][3])
        assert abs(P - want["P"]) <= 1e-14 * abs(want["P"])
        np.testing.assert_allclose(ga, want["grad_alpha"], rtol=1e-13, atol=1e-15 * np.max(np.abs(want["grad_alpha"])))
        np.testing.assert_array_equal(gW, want["grad_W"])
        assert abs(Po - want["P"]) <= 1e-14 * abs(want["P"])
        assert J == want["J"]
    pens = np.concatenate([r[6] for r in res])
    np.testing.assert_array_equal(pens, want["pen"])

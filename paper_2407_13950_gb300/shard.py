"""One problem's windows sharded over ranks (one process per GPU).

Sec. 3 makes the windows of the multiple-shooting objective independent once the window states
W^m are given, and Sec. 4 distributes them over processes.  Here rank r owns a contiguous range
of windows first_r..last_r (`partition`) and evaluates it as a library shard (a problem created
with a window range; no exchange happens inside the library).  One evaluation then needs:

* the window states the shard reads, W^max(first-1,1) .. W^min(last,M-1) (every rank holds the
  full W vector of the optimiser; each takes its slice);
* the hand-off across each rank boundary b = last_r: dP/dW^b = mu (W^b - U^b(t_b))
  - 2 Lambda^{b+1}(t_b) joins rank r's penalty term with the adjoint of rank r+1's first window
  at its start (Eq. dP-dW).  Rank r+1 sends its term -2 Lambda^{b+1}(t_b) (the first block of
  its shard's grad_W, N x E complex) to rank r, which adds it to its own last block;
* one all-reduce of d + 1 doubles: P and dP/dalpha are sums over windows (Eqs. penalty-fcn,
  grad-int), so the shards' partial sums are added.  J lives on the last rank.

Every rank ends with the same P and dP/dalpha and the dP/dW blocks of the window states it owns
(W^k for k = first..min(last, M-1)); `gather_grad_W` assembles the full vector on every rank.
The exchange goes through torch.distributed (NCCL between GPUs, gloo on CPU); the compute of a
rank is one `evaluate(first, last, alpha, W_slice)` call, by default the library shard.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Tuple

import numpy as np

from . import msqoc


def partition(M: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous window ranges (first, last), 1-based, of sizes differing by at most one
    (windows differ in length by at most one step, so the work is balanced)."""
    if world < 1 or world > M:
        raise ValueError(f"cannot split {M} windows over {world} ranks")
    out, start = [], 1
    for r in range(world):
        n = M // world + (1 if r < M % world else 0)
        out.append((start, start + n - 1))
        start += n
    return out


def w_slice(spec, first: int, last: int) -> Tuple[int, int]:
    """Offsets (in doubles) of the window states W^max(first-1,1) .. W^min(last,M-1) in the
    full W vector (layout [M-1][E][N] complex)."""
    k0, k1 = msqoc.shard_w_range(spec.M, first, last)
    nb = 2 * spec.N * spec.E
    if k1 < k0:
        return 0, 0
    return (k0 - 1) * nb, k1 * nb


def library_evaluator(spec, first: int, last: int, **problem_kw) -> Callable:
    """The library shard of windows first..last as a rank's compute: returns (evaluate, close)."""
    prob = msqoc.Problem(spec, windows=(first, last), **problem_kw)

    def evaluate(alpha, W_slice, gradient: bool = True) -> dict:
        return prob.eval_gradient(alpha, W_slice) if gradient else prob.eval_objective(alpha, W_slice)

    return evaluate, prob.close


class ShardedProblem:
    """This rank's shard of an M-window problem and the exchange that completes an evaluation.

    dist: torch.distributed (initialised); group: process group or None.  evaluate(alpha,
    W_slice, gradient) -> {"P", "grad_alpha", "grad_W"} (gradient) or {"P", "J", "pen"} computes
    the shard; the default is the library shard on the current GPU."""

    def __init__(self, spec, dist, group=None, evaluate: Optional[Callable] = None, **problem_kw):
        self.spec = spec
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.ranges = partition(spec.M, self.world)
        self.first, self.last = self.ranges[self.rank]
        self._close = None
        if evaluate is None:
            evaluate, self._close = library_evaluator(spec, self.first, self.last, **problem_kw)
        self._evaluate = evaluate
        self.nb = 2 * spec.N * spec.E
        self.lo, self.hi = w_slice(spec, self.first, self.last)

    def close(self):
        if self._close is not None:
            self._close()
            self._close = None

    # ---------------------------------------------------------------- exchange helpers
    def _global_rank(self, r: int) -> int:
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def _allreduce(self, x: np.ndarray) -> np.ndarray:
        import torch
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).clone()
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def _handoff(self, first_block: Optional[np.ndarray]) -> Optional[np.ndarray]:
        """Send this rank's first grad_W block (-2 Lambda of its first window at its start) to
        the previous rank; return the block received from the next rank (or None)."""
        import torch
        nccl = self.dist.get_backend(self.group) == "nccl"
        reqs, recv = [], None
        if self.rank > 0 and self.first >= 2:
            t = torch.from_numpy(np.ascontiguousarray(first_block)).clone()
            t = t.cuda() if nccl else t
            reqs.append(self.dist.isend(t, self._global_rank(self.rank - 1), group=self.group))
        if self.rank + 1 < self.world and self.last < self.spec.M:
            recv = torch.empty(self.nb, dtype=torch.float64, device="cuda" if nccl else "cpu")
            reqs.append(self.dist.irecv(recv, self._global_rank(self.rank + 1), group=self.group))
        for r in reqs:
            r.wait()
        return None if recv is None else recv.cpu().numpy()

    # ---------------------------------------------------------------- evaluations
    def eval_gradient(self, alpha, W) -> dict:
        """P and dP/dalpha (identical on every rank) and the dP/dW blocks this rank owns:
        {"P", "grad_alpha", "grad_W_own", "own": (k_first, k_last)}."""
        W = np.asarray(W, dtype=np.float64)
        loc = self._evaluate(alpha, W[self.lo:self.hi], True)
        gW = np.array(loc["grad_W"], dtype=np.float64, copy=True)
        k0, k1 = msqoc.shard_w_range(self.spec.M, self.first, self.last)
        first_block = gW[:self.nb] if (self.first >= 2 and gW.size) else None
        recv = self._handoff(first_block)
        if recv is not None:
            gW[-self.nb:] = gW[-self.nb:] + recv
        red = self._allreduce(np.concatenate([[loc["P"]], loc["grad_alpha"]]))
        # the blocks this rank owns: W^k with k >= first (the block of W^{first-1} went to the
        # previous rank)
        own_from = 1 if self.first >= 2 else 0
        return {"P": float(red[0]), "grad_alpha": red[1:], "grad_W_own": gW[own_from * self.nb:],
                "own": (max(self.first, 1), k1) if k1 >= max(self.first, 1) else (0, -1)}

    def eval_objective(self, alpha, W) -> dict:
        """P (every rank) and J (the last rank's, sent to all in the same reduction)."""
        W = np.asarray(W, dtype=np.float64)
        loc = self._evaluate(alpha, W[self.lo:self.hi], False)
        J = loc["J"] if self.last == self.spec.M else 0.0
        red = self._allreduce(np.array([loc["P"], J]))
        return {"P": float(red[0]), "J": float(red[1]), "pen_own": np.asarray(loc["pen"])}

    def gather_grad_W(self, grad_W_own: np.ndarray) -> np.ndarray:
        """The full dP/dW vector on every rank from each rank's owned blocks (rank order)."""
        import torch
        M, nb = self.spec.M, self.nb
        sizes = []
        for (a, b) in self.ranges:
            k0, k1 = max(a, 1), min(b, M - 1)
            sizes.append(max(0, k1 - k0 + 1) * nb)
        width = max(sizes) if sizes else 0
        nccl = self.dist.get_backend(self.group) == "nccl"
        mine = torch.zeros(width, dtype=torch.float64)
        mine[:grad_W_own.size] = torch.from_numpy(np.ascontiguousarray(grad_W_own))
        if nccl:
            mine = mine.cuda()
        parts = [torch.empty_like(mine) for _ in range(self.world)]
        self.dist.all_gather(parts, mine, group=self.group)
        return np.concatenate([p.cpu().numpy()[:n] for p, n in zip(parts, sizes)])


def combine(spec, parts) -> dict:
    """Whole-problem P, dP/dalpha and dP/dW from shard results computed anywhere (for example
    one after another on one GPU): parts = [((first, last), eval_gradient result), ...] covering
    windows 1..M.  The arithmetic is the distributed path's: partial sums added in rank order,
    each shard's grad_W blocks added into the full vector (overlapping blocks sum the penalty
    term of one shard and the -2 Lambda term of the next)."""
    nb = 2 * spec.N * spec.E
    P = 0.0
    ga = np.zeros(spec.d)
    gW = np.zeros(spec.nW)
    covered = []
    for (first, last), r in sorted(parts, key=lambda x: x[0][0]):
        covered.extend(range(first, last + 1))
        P += r["P"]
        ga += r["grad_alpha"]
        lo, hi = w_slice(spec, first, last)
        gW[lo:hi] += r["grad_W"]
    if sorted(covered) != list(range(1, spec.M + 1)):
        raise ValueError("the shards do not partition the windows")
    return {"P": P, "grad_alpha": ga, "grad_W": gW}

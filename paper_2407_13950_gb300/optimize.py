"""Multiple-shooting pulse optimisation driven by the GPU objective and gradient.

The optimisation variables are the control coefficients alpha and the window states
W^1..W^{M-1} (Sec. 3: the penalty objective P(alpha, W) is minimised over both).  Following
Sec. 5, the window states start from a roll-out of the initial controls (all continuity
penalties zero), the penalty weight is fixed (mu = 2/E, the problem's default), and the
iteration stops once the estimate of the roll-out infidelity (Eq. rollout-infid-est) falls
below a tolerance.  The minimiser is L-BFGS (two-loop recursion, limited memory) with a
backtracking Armijo line search; optional box bounds on alpha are kept by projection (the
search direction is built from the projected gradient and steps are clipped).

Every objective and gradient comes from the library's kernels through the C ABI; the vectors
of the recursion live on the GPU as torch tensors (FP64) and only scalars cross to the host.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import msqoc


@dataclasses.dataclass
class Result:
    alpha: np.ndarray
    W: np.ndarray
    P: float
    estimate: float                 # roll-out infidelity estimate at the end
    iterations: int
    evaluations: int
    converged: bool
    history: List[dict]             # per iteration: P, J, estimate, step


def optimize(problem: msqoc.Problem, alpha0, W0=None, *, tol: float = 1e-3, max_iter: int = 200,
             memory: int = 10, bound: Optional[float] = None, c1: float = 1e-4, max_backtracks: int = 30,
             stream=None) -> Result:
    """Minimise P(alpha, W) of `problem` from alpha0 (and W0, default: the roll-out of alpha0).
    bound: |alpha_i| <= bound when given.  Stops when the roll-out estimate is below tol."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = problem.spec
    d, nW = problem.d, problem.nW
    a0 = np.asarray(alpha0, dtype=np.float64)
    if bound is not None:
        a0 = np.clip(a0, -bound, bound)
    if W0 is None:
        W0 = problem.rollout(a0) if spec.M > 1 else np.zeros(0)
    x = torch.tensor(np.concatenate([a0, np.asarray(W0, dtype=np.float64)]), device=dev, dtype=torch.float64)
    g = torch.zeros_like(x)
    P = torch.zeros(1, device=dev, dtype=torch.float64)
    nev = 0

    def evaluate(xv, gv, Pv):
        nonlocal nev
        nev += 1
        a, w = xv[:d], xv[d:]
        problem.eval_gradient_into(a, w if spec.M > 1 else None, Pv, gv[:d], gv[d:] if spec.M > 1 else None,
                                   stream=stream)

    def project(xv):
        if bound is not None:
            xv[:d].clamp_(-bound, bound)
        return xv

    def projected_gradient(xv, gv):
        # zero the components that push an alpha at its bound outward
        if bound is None:
            return gv
        pg = gv.clone()
        a, ga = xv[:d], pg[:d]
        ga[(a >= bound) & (ga < 0)] = 0.0
        ga[(a <= -bound) & (ga > 0)] = 0.0
        return pg

    evaluate(x, g, P)
    f = float(P.item())
    est = problem.rollout_estimate()
    S_mem, Y_mem = [], []
    history = [{"P": f, "estimate": est, "step": 0.0}]
    it = 0
    while est >= tol and it < max_iter:
        pg = projected_gradient(x, g)
        # two-loop recursion
        q = pg.clone()
        alphas = []
        for s, y in reversed(list(zip(S_mem, Y_mem))):
            rho = 1.0 / float(torch.dot(y, s))
            a_i = rho * float(torch.dot(s, q))
            q -= a_i * y
            alphas.append((rho, a_i))
        if S_mem:
            s, y = S_mem[-1], Y_mem[-1]
            q *= float(torch.dot(s, y)) / float(torch.dot(y, y))
        else:
            q /= max(float(torch.linalg.norm(q)), 1e-300)      # first step: unit length
        for (s, y), (rho, a_i) in zip(zip(S_mem, Y_mem), reversed(alphas)):
            b = rho * float(torch.dot(y, q))
            q += (a_i - b) * s
        direction = -q
        slope = float(torch.dot(pg, direction))
        if slope >= 0:                                          # not a descent direction: restart
            S_mem.clear()
            Y_mem.clear()
            direction = -pg / max(float(torch.linalg.norm(pg)), 1e-300)
            slope = float(torch.dot(pg, direction))
        # backtracking Armijo line search on the projected path
        t = 1.0
        x_new = torch.empty_like(x)
        g_new = torch.empty_like(g)
        P_new = torch.zeros_like(P)
        accepted = False
        for _ in range(max_backtracks):
            x_new.copy_(x).add_(direction, alpha=t)
            project(x_new)
            evaluate(x_new, g_new, P_new)
            f_new = float(P_new.item())
            if f_new <= f + c1 * float(torch.dot(pg, x_new - x)):
                accepted = True
                break
            t *= 0.5
        if not accepted:
            break
        s_vec, y_vec = x_new - x, g_new - g
        if float(torch.dot(s_vec, y_vec)) > 1e-12 * float(torch.dot(y_vec, y_vec)):
            S_mem.append(s_vec)
            Y_mem.append(y_vec)
            if len(S_mem) > memory:
                S_mem.pop(0)
                Y_mem.pop(0)
        x, g, f = x_new.clone(), g_new.clone(), f_new
        est = problem.rollout_estimate()
        it += 1
        history.append({"P": f, "estimate": est, "step": t})
    xh = x.cpu().numpy()
    return Result(alpha=xh[:d], W=xh[d:], P=f, estimate=est, iterations=it, evaluations=nev,
                  converged=est < tol, history=history)

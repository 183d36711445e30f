"""Multiple-shooting pulse optimisation driven by the GPU objective and gradient.

The optimisation variables are the control coefficients alpha and the window states
W^1..W^{M-1} (Sec. 3: the penalty objective P(alpha, W) is minimised over both).  Following
Sec. 5:
- the window states start from a roll-out of the initial controls (all continuity penalties
  zero);
- the penalty weight is fixed (mu = 2/E, the problem's default);
- the objective may carry the paper's regularization: a Tikhonov term (gamma_tik/2)||alpha||^2
  and the time-averaged control-pulse energy gamma_energy (1/T) int sum_k |d_k|^2 dt
  (msqoc_eval_regularization);
- the window states may enter the optimisation scaled, W~ = sigma W, which balances the
  alpha- and W-parts of the gradient (the paper scans sigma in [0.05, 0.15]);
- box bounds on alpha keep the pulse amplitudes below a limit (`amplitude_bound`);
- the iteration stops once the estimate of the roll-out infidelity (Eq. rollout-infid-est)
  falls below a tolerance.

The minimiser is L-BFGS (two-loop recursion, limited memory) with a backtracking Armijo line
search; the box bounds are kept by projection: an alpha at its bound whose gradient pushes it
outward is held fixed for the iteration (its gradient and search-direction components are
zeroed) and steps are clipped to the box.  Every objective and gradient comes from the
library's kernels through the C ABI, and so do the L-BFGS steps (msqoc_lbfgs_direction, _trial,
_update: one CTA each); the vectors live on the GPU as torch tensors (FP64) and only scalars
cross to the host, a few per iteration.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Union

import numpy as np

from . import msqoc

NATIVE_MAX = 1 << 18   # unknowns up to which the one-CTA L-BFGS kernels are used


@dataclasses.dataclass
class Result:
    alpha: np.ndarray
    W: np.ndarray                   # unscaled window states
    P: float                        # penalty objective at the end (without the regularization)
    F: float                        # minimised objective P + R
    estimate: float                 # roll-out infidelity estimate at the end
    iterations: int
    evaluations: int
    converged: bool
    history: List[dict]             # per iteration: F, P, estimate, step


def amplitude_bound(spec, max_amplitude: float) -> np.ndarray:
    """Per-coefficient box bound b (layout of alpha) such that |alpha1|, |alpha2| <= b keeps
    |d_k(t)| <= max_amplitude (rad/ns) at every t.  The B-splines are non-negative and sum
    to one, so |d_k(t)| <= sum_f max_s |alpha1 + i alpha2|_kfs <= sqrt(2) N_f(k) b_k:
    b_k = max_amplitude / (sqrt(2) N_f(k))."""
    out = []
    for k in range(spec.q):
        nf = len(spec.omega[k])
        out.extend([max_amplitude / (math.sqrt(2.0) * nf)] * (2 * spec.d1 * nf))
    return np.asarray(out, dtype=np.float64)


def paper_settings(spec) -> dict:
    """The optimisation settings of Sec. 5: amplitudes below 2 pi x 25 MHz, gamma_tik = 1e-3/d,
    gamma_energy = 1e-3, roll-out estimate below 1e-3."""
    return {"bound": amplitude_bound(spec, 2 * math.pi * 0.025), "gamma_tik": 1e-3 / spec.d,
            "gamma_energy": 1e-3, "tol": 1e-3}


def optimize(problem: msqoc.Problem, alpha0, W0=None, *, tol: float = 1e-3, max_iter: int = 200,
             memory: int = 10, bound: Union[None, float, np.ndarray] = None, gamma_tik: float = 0.0,
             gamma_energy: float = 0.0, sigma: float = 1.0, c1: float = 1e-4, max_backtracks: int = 30,
             stream=None) -> Result:
    """Minimise P(alpha, W) + R(alpha) of `problem` from alpha0 (and W0, default: the roll-out
    of alpha0).  bound: |alpha_i| <= bound (a scalar or one bound per coefficient).  Stops when
    the roll-out estimate is below tol."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = problem.spec
    d, nW = problem.d, problem.nW
    if not sigma > 0:
        raise ValueError("sigma must be > 0")
    regularized = gamma_tik > 0 or gamma_energy > 0
    a0 = np.asarray(alpha0, dtype=np.float64)
    lim = None
    if bound is not None:
        lim_h = np.broadcast_to(np.asarray(bound, dtype=np.float64), (d,))
        a0 = np.clip(a0, -lim_h, lim_h)
        lim = torch.tensor(lim_h, device=dev, dtype=torch.float64)
    if W0 is None:
        W0 = problem.rollout(a0) if spec.M > 1 else np.zeros(0)
    x = torch.tensor(np.concatenate([a0, sigma * np.asarray(W0, dtype=np.float64)]), device=dev,
                     dtype=torch.float64)
    g = torch.zeros_like(x)
    Pv = torch.zeros(1, device=dev, dtype=torch.float64)
    Rv = torch.zeros(1, device=dev, dtype=torch.float64)
    rg = torch.zeros(d, device=dev, dtype=torch.float64)
    w_unscaled = torch.zeros(nW, device=dev, dtype=torch.float64)
    nev = 0

    def evaluate(xv, gv):
        """P into Pv, R into Rv and the gradient of F = P + R in the optimisation variables into
        gv (asynchronous: nothing is read back here)."""
        nonlocal nev
        nev += 1
        a, wt = xv[:d], xv[d:]
        w = None
        if spec.M > 1:
            w = wt if sigma == 1.0 else torch.div(wt, sigma, out=w_unscaled)
        problem.eval_gradient_into(a, w, Pv, gv[:d], gv[d:] if spec.M > 1 else None, stream=stream)
        if sigma != 1.0 and spec.M > 1:
            gv[d:].div_(sigma)
        if regularized:
            problem.eval_regularization_into(a, gamma_tik, gamma_energy, Rv, rg, stream=stream)
            gv[:d].add_(rg)

    def scalars(*ts):
        """device scalars to host floats in one transfer"""
        return torch.cat([t.reshape(1) for t in ts]).tolist()

    n = d + nW
    nb = d if lim is not None else 0
    cap = max(1, min(int(memory), msqoc.LBFGS_MAXMEM))
    S = torch.zeros((cap, n), device=dev, dtype=torch.float64)     # memory ring: s_j, y_j
    Y = torch.zeros((cap, n), device=dev, dtype=torch.float64)
    rho = torch.zeros(cap, device=dev, dtype=torch.float64)        # 1 / <s_j, y_j>
    yy = torch.zeros(cap, device=dev, dtype=torch.float64)         # <y_j, y_j>
    m = head = 0
    direction = torch.empty_like(x)
    slope = torch.zeros(1, device=dev, dtype=torch.float64)
    dec = torch.zeros(1, device=dev, dtype=torch.float64)
    sy_yy = torch.zeros(2, device=dev, dtype=torch.float64)
    x_new = torch.empty_like(x)
    g_new = torch.empty_like(g)
    # The library's L-BFGS kernels run on one CTA: a few launches an iteration, the right
    # trade for the paper's problem sizes; beyond NATIVE_MAX unknowns the same steps run as
    # whole-GPU vector operations.
    native = n <= NATIVE_MAX

    def lbfgs_direction(mm):
        if native:
            msqoc.lbfgs_direction(n, nb, x, g, lim, S, Y, rho, yy, cap, mm, head, direction, slope, stream=stream)
            return
        act = torch.zeros(n, device=dev, dtype=torch.bool)
        if nb:
            act[:nb] = ((x[:nb] >= lim) & (g[:nb] < 0)) | ((x[:nb] <= -lim) & (g[:nb] > 0))
        pg = g.masked_fill(act, 0.0)
        q = pg.clone()
        slots = [(head - mm + j) % cap for j in range(mm)]
        coef = []
        for k in reversed(slots):
            a_k = rho[k] * torch.dot(S[k], q)
            q.sub_(a_k * Y[k])
            coef.append(a_k)
        if mm:
            q.mul_((1.0 / rho[slots[-1]]) / yy[slots[-1]])
        else:
            q.div_(torch.linalg.norm(q).clamp_min(1e-300))
        for k, a_k in zip(slots, reversed(coef)):
            q.add_((a_k - rho[k] * torch.dot(Y[k], q)) * S[k])
        torch.neg(q, out=direction).masked_fill_(act, 0.0)
        slope.copy_(torch.dot(pg, direction).reshape(1))

    def lbfgs_trial(t):
        if native:
            msqoc.lbfgs_trial(n, nb, x, direction, t, lim, g, x_new, dec, stream=stream)
            return
        x_new.copy_(x).add_(direction, alpha=t)
        if nb:
            torch.minimum(torch.maximum(x_new[:nb], -lim), lim, out=x_new[:nb])
        dec.copy_(torch.dot(g, x_new - x).reshape(1))

    def lbfgs_update():
        if native:
            msqoc.lbfgs_update(n, x, x_new, g, g_new, S[head], Y[head], sy_yy, stream=stream)
            return
        torch.sub(x_new, x, out=S[head])
        torch.sub(g_new, g, out=Y[head])
        sy_yy.copy_(torch.stack([torch.dot(S[head], Y[head]), torch.dot(Y[head], Y[head])]))

    evaluate(x, g)
    P, R = scalars(Pv, Rv)
    f = P + R
    est = problem.rollout_estimate()
    history = [{"F": f, "P": P, "estimate": est, "step": 0.0}]
    it = 0
    while est >= tol and it < max_iter:
        # search direction on the device (two-loop recursion, active set held fixed)
        lbfgs_direction(m)
        if slope.item() >= 0:                                   # not a descent direction: restart
            m = 0
            lbfgs_direction(0)
        # backtracking Armijo line search on the projected path
        t = 1.0
        accepted = False
        for _ in range(max_backtracks):
            lbfgs_trial(t)
            evaluate(x_new, g_new)
            P_new, R_new, decrease = scalars(Pv, Rv, dec)
            f_new = P_new + R_new
            if f_new <= f + c1 * decrease:
                accepted = True
                break
            t *= 0.5
        if not accepted:
            break
        lbfgs_update()
        sy, yyv = sy_yy.tolist()
        if sy > 1e-12 * yyv:                                    # curvature condition: keep the pair
            rho[head] = 1.0 / sy
            yy[head] = yyv
            head = (head + 1) % cap
            m = min(m + 1, cap)
        x, x_new = x_new, x
        g, g_new = g_new, g
        f, P = f_new, P_new
        est = problem.rollout_estimate()
        it += 1
        history.append({"F": f, "P": P, "estimate": est, "step": t})
    xh = x.cpu().numpy()
    return Result(alpha=xh[:d], W=xh[d:] / sigma, P=P, F=f, estimate=est, iterations=it, evaluations=nev,
                  converged=est < tol, history=history)

"""The multiple-shooting optimiser (L-BFGS over alpha and the window states, roll-out start,
roll-out-estimate stopping rule) on the GPU objective and gradient."""
import numpy as np
import pytest

from paper_2407_13950_gb300 import msqoc, optimize
from paper_2407_13950_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def test_optimiser_decreases_the_penalty_objective_and_respects_bounds():
    spec = S.paper_qft_spec(2, M=4)                       # QFT-4, the paper's full time grid
    alpha0 = S.random_alpha(spec, 91)
    bound = 2 * np.pi * 0.02
    with msqoc.Problem(spec) as p:
        res = optimize.optimize(p, alpha0, tol=1e-3, max_iter=40, bound=bound)
        check = p.eval_objective(res.alpha, res.W)
    Ps = [h["P"] for h in res.history]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(Ps, Ps[1:]))     # Armijo: monotone
    assert res.F == res.P                                             # no regularization
    assert res.P < 0.5 * Ps[0]
    assert res.estimate < res.history[0]["estimate"]
    assert np.all(np.abs(res.alpha) <= bound * (1 + 1e-15))
    assert check["P"] == pytest.approx(res.P, rel=1e-12)
    print(f"QFT-4 M=4: P {Ps[0]:.4e} -> {res.P:.4e}, estimate {res.history[0]['estimate']:.3e} -> "
          f"{res.estimate:.3e} in {res.iterations} iterations, {res.evaluations} evaluations")


def test_optimiser_starts_from_the_rollout():
    spec = S.transmon_spec(2, 20.0, 800, 4, 6)
    alpha0 = S.random_alpha(spec, 92)
    with msqoc.Problem(spec) as p:
        res = optimize.optimize(p, alpha0, max_iter=0)
        single = msqoc.Problem(spec.replace(M=1))
        want = single.eval_objective(alpha0)["P"]
        single.close()
    assert res.iterations == 0
    assert res.P == pytest.approx(want, rel=1e-11)          # all penalties zero at the roll-out


def _max_amplitude(spec, alpha, nsamples=400):
    """max_k,t |d_k(t)| on a grid of times, controls evaluated by the oracle"""
    import oracle
    ts = (np.arange(nsamples) + 0.5) * spec.T / nsamples
    return max(float(np.max(np.abs(oracle.controls(spec, alpha, t)))) for t in ts)


@pytest.mark.parametrize("M,sigma", [(8, 0.1), (1, 1.0)])
def test_paper_settings_qft4_converge_and_the_estimate_bounds_the_rollout(M, sigma):
    """Sec. 5 settings (amplitude box 25 MHz, Tikhonov 1e-3/d, energy 1e-3, estimate < 1e-3, window
    states scaled by sigma) on QFT-4 from the paper's random initial guess (+-10 MHz)."""
    spec = S.paper_qft_spec(2, M=M)
    alpha0 = S.random_alpha(spec, 7, amp=S.PAPER_ALPHA0_AMP)
    st = optimize.paper_settings(spec)
    with msqoc.Problem(spec) as p:
        res = optimize.optimize(p, alpha0, tol=st["tol"], max_iter=600, bound=st["bound"],
                                gamma_tik=st["gamma_tik"], gamma_energy=st["gamma_energy"], sigma=sigma)
    assert res.converged, (res.iterations, res.estimate)
    Fs = [h["F"] for h in res.history]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(Fs, Fs[1:]))
    assert np.all(np.abs(res.alpha) <= st["bound"] * (1 + 1e-15))
    assert _max_amplitude(spec, res.alpha) <= 2 * np.pi * 0.025 * (1 + 1e-12)
    with msqoc.Problem(spec.replace(M=1)) as p1:
        J_rollout = p1.eval_objective(res.alpha)["J"]
    assert J_rollout <= res.estimate * (1 + 1e-12) and res.estimate < 1e-3
    print(f"QFT-4 M={M} sigma={sigma}: {res.iterations} iterations, estimate {res.estimate:.3e}, "
          f"roll-out infidelity {J_rollout:.3e}")


def test_native_and_vector_lbfgs_steps_agree(monkeypatch):
    """The one-CTA L-BFGS kernels (small problems) and the whole-GPU vector form (large ones)
    take the same iterates, up to the order of their sums."""
    spec = S.paper_qft_spec(2, M=4)
    alpha0 = S.random_alpha(spec, 93)
    st = optimize.paper_settings(spec)
    runs = []
    for native_max in (1 << 18, 0):
        monkeypatch.setattr(optimize, "NATIVE_MAX", native_max)
        with msqoc.Problem(spec) as p:
            runs.append(optimize.optimize(p, alpha0, tol=0.0, max_iter=6, bound=st["bound"],
                                          gamma_tik=st["gamma_tik"], gamma_energy=st["gamma_energy"], sigma=0.1))
    a, b = runs
    assert a.iterations == b.iterations == 6
    assert [h["step"] for h in a.history] == [h["step"] for h in b.history]
    np.testing.assert_allclose([h["F"] for h in a.history], [h["F"] for h in b.history], rtol=1e-9)
    np.testing.assert_allclose(a.alpha, b.alpha, rtol=1e-7, atol=1e-12)

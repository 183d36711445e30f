"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a library routine (scipy expm/eigh/BSpline), a closed
form, a physical fact, an invariant or brute-force finite differences, chosen so that a
plausible slip (dropped term, wrong sign, swapped index, wrong factor) fails one of them.
All tests here run on the CPU.
"""
import math
import os

import numpy as np
import pytest
import scipy.interpolate
import scipy.linalg

import oracle
from paper_2407_13950_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- helpers
def ladder(L):
    """lowering operator a on L levels: a|l> = sqrt(l)|l-1> (independent numpy build)."""
    return np.diag(np.sqrt(np.arange(1, L)), k=1).astype(complex)


def embed(op, k, q, L):
    """I x ... x op (position k, subsystem 0 leftmost) x ... x I via numpy kron."""
    out = np.array([[1.0 + 0j]])
    for j in range(q):
        out = np.kron(out, op if j == k else np.eye(L))
    return out


def drift_closed_form(spec):
    """diagonal energies D_i = sum_k -(xi_k/2) l_k(l_k-1) - sum_{k<l} xi_kl l_k l_l."""
    q, L = spec.q, spec.L
    D = np.zeros(spec.N)
    for i in range(spec.N):
        lv = [(i // L ** (q - 1 - k)) % L for k in range(q)]
        e = sum(-0.5 * spec.xi[k] * lv[k] * (lv[k] - 1) for k in range(q))
        e -= sum(spec.xi_cross[k][l] * lv[k] * lv[l] for k in range(q) for l in range(k + 1, q))
        D[i] = e
    return D


def kron_hamiltonian(spec, d):
    """BASELINE's written form: sum_k -xi_k/2 a^+a^+aa - sum xi_kl n_k n_l
    + sum_k p_k (a_k + a_k^+) + i q_k (a_k - a_k^+), with d_k = p_k + i q_k."""
    q, L = spec.q, spec.L
    a = ladder(L)
    H = np.zeros((spec.N, spec.N), complex)
    for k in range(q):
        ak = embed(a, k, q, L)
        H += -0.5 * spec.xi[k] * ak.conj().T @ ak.conj().T @ ak @ ak
        H += d[k].real * (ak + ak.conj().T) + 1j * d[k].imag * (ak - ak.conj().T)
        for l in range(k + 1, q):
            al = embed(a, l, q, L)
            H += -spec.xi_cross[k][l] * (ak.conj().T @ ak) @ (al.conj().T @ al)
    if spec.detune is not None:
        for k in range(q):
            ak = embed(a, k, q, L)
            H += spec.detune[k] * ak.conj().T @ ak
    if spec.jx is not None:
        for k in range(q):
            for l in range(k + 1, q):
                ak, al = embed(a, k, q, L), embed(a, l, q, L)
                H += spec.jx[k][l] * (al.conj().T @ ak + al @ ak.conj().T)
    return H


def cayley_power(H, h, nsteps):
    """((I + i h H/2)^{-1} (I - i h H/2))^nsteps by eigendecomposition of Hermitian H."""
    lam, Q = scipy.linalg.eigh(H)
    c = (1 - 0.5j * h * lam) / (1 + 0.5j * h * lam)
    return (Q * c ** nsteps) @ Q.conj().T


def constant_alpha(spec, value):
    """equal coefficients on every spline of carrier 0 (partition of unity -> constant envelope)."""
    a = np.zeros(spec.d)
    off = 0
    for k in range(spec.q):
        base = 2 * spec.d1 * off
        a[base:base + 2 * spec.d1:2] = value[k].real
        a[base + 1:base + 2 * spec.d1:2] = value[k].imag
        off += len(spec.omega[k])
    return a


def Wmat(spec, W, m):
    """W^m (1-based) as an N x E complex matrix from the flat interleaved vector."""
    ne = spec.N * spec.E
    return oracle.f64_to_cplx(W[2 * ne * (m - 1): 2 * ne * m], spec.N)


def rand_state(rng, N, E):
    return (rng.standard_normal((N, E)) + 1j * rng.standard_normal((N, E))) / math.sqrt(2 * N)


# ----------------------------------------------------------------------------- controls
def test_bspline_golden_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "bspline_values.txt"))
    for tau, val in rows:
        assert oracle.bspline(tau) == pytest.approx(val, abs=1e-15)


def test_controls_match_scipy_bspline_basis():
    """Placement: d1 splines on knots k*dtau (dtau = T/(d1-2)), centres (s-1/2)dtau, evaluated
    with scipy's B-spline basis elements; carriers exp(+i Omega t) (Eq. dj-ctrl)."""
    sp = S.transmon_spec(2, 37.0, 100, 1, 7)
    alpha = S.random_alpha(sp, 11)
    dtau = sp.T / (sp.d1 - 2)
    basis = [scipy.interpolate.BSpline.basis_element(np.array([s - 2, s - 1, s, s + 1]) * dtau, extrapolate=False)
             for s in range(sp.d1)]
    for t in np.linspace(0.0, sp.T, 41):
        B = np.array([np.nan_to_num(b(t)) for b in basis])
        assert abs(B.sum() - 1.0) < 1e-13          # partition of unity on [0, T]
        want = []
        off = 0
        for k in range(sp.q):
            dk = 0j
            for f, om in enumerate(sp.omega[k]):
                c = alpha[2 * sp.d1 * (off + f): 2 * sp.d1 * (off + f + 1)]
                dk += np.exp(1j * om * t) * np.sum((c[0::2] + 1j * c[1::2]) * B)
            off += len(sp.omega[k])
            want.append(dk)
        np.testing.assert_allclose(oracle.controls(sp, alpha, t), want, rtol=0, atol=1e-15)


def test_carrier_sign_drives_the_resonant_transition():
    """Physics pin of the carrier sign, drift sign and ladder structure: one 3-level transmon
    driven only on carrier Omega = -xi (resonant with |1> <-> |2> in the rotating frame)
    transfers |1> to |2> (Rabi pi pulse); the opposite sign would be detuned by 2 xi."""
    xi = S.TWO_PI * 0.22
    T = 50.0
    for sign, expect_transfer in ((-1.0, True), (+1.0, False)):
        sp = S.ProblemSpec(q=1, L=3, ness=2, xi=[xi], xi_cross=[[0.0]], omega=[[0.0, sign * xi]], d1=12,
                           T=T, nsteps=4000, M=1)
        # constant envelope on carrier 1: coupling of |1>-|2> is sqrt(2)|d|; pi pulse: sqrt(2)|d| T = pi/2
        amp = math.pi / 2 / (math.sqrt(2) * T)
        a = np.zeros(sp.d)
        a[2 * sp.d1: 4 * sp.d1: 2] = amp
        psi0 = np.zeros((3, 1), complex)
        psi0[1, 0] = 1.0
        psi = oracle.propagate(sp, a, 0, sp.nsteps, psi0)
        p2 = abs(psi[2, 0]) ** 2
        if expect_transfer:
            assert p2 > 0.99
        else:
            assert p2 < 0.01


# ----------------------------------------------------------------------------- model
@pytest.mark.parametrize("q", [1, 2, 3])
def test_hamiltonian_matches_kron_construction(q):
    sp = S.transmon_spec(q, 20.0, 100, 1, 5)
    alpha = S.random_alpha(sp, 3)
    for t in (0.0, 3.3, 17.2):
        d = oracle.controls(sp, alpha, t)
        H = oracle.hamiltonian(sp, alpha, t)
        np.testing.assert_allclose(H, kron_hamiltonian(sp, d), atol=1e-14)
        np.testing.assert_allclose(H, H.conj().T, atol=1e-15)


def test_paper_drift_matches_kron_construction():
    """The paper's own model (Eq. sys-ham): detuning and dipole exchange on 2-level qubits."""
    sp = S.ProblemSpec(q=3, L=2, ness=2, xi=[0.0] * 3, xi_cross=[[0.0] * 3] * 3, omega=[[0.0]] * 3, d1=4,
                       T=10.0, nsteps=10, M=1, detune=[0.37, -0.05, -0.32],
                       jx=[[0, 0.0314, 0], [0, 0, 0.0314], [0, 0, 0]])
    Hs = oracle.system_hamiltonian(sp)
    np.testing.assert_allclose(Hs, kron_hamiltonian(sp, np.zeros(3)), atol=1e-15)


def test_lowering_operator_and_strides():
    sp = S.transmon_spec(3, 1.0, 1, 1, 3)
    for k in range(3):
        np.testing.assert_allclose(oracle.lowering(sp, k), embed(ladder(3), k, 3, 3), atol=0)


# ----------------------------------------------------------------------------- targets
def test_qft_targets():
    sp2 = S.ProblemSpec(q=1, L=2, ness=2, xi=[0.0], xi_cross=[[0.0]], omega=[[0.0]], d1=3, T=1, nsteps=1, M=1)
    np.testing.assert_allclose(oracle.target(sp2), np.array([[1, 1], [1, -1]]) / math.sqrt(2), atol=1e-15)
    sp4 = S.ProblemSpec(q=2, L=2, ness=2, xi=[0.0] * 2, xi_cross=[[0.0] * 2] * 2, omega=[[0.0]] * 2, d1=3, T=1,
                        nsteps=1, M=1)
    V = oracle.target(sp4)
    for r, c, re, im in np.loadtxt(os.path.join(GOLDEN, "qft4.txt")):
        assert V[int(r), int(c)] == pytest.approx(re + 1j * im, abs=1e-15)
    for q in (2, 3, 4):
        sp = S.transmon_spec(q, 1.0, 1, 1, 3)
        V = oracle.target(sp)
        np.testing.assert_allclose(V.conj().T @ V, np.eye(sp.E), atol=1e-14)   # V^+ V = I (Sec. 5)
        # guard rows (any level 2) are zero; essential rows hold QFT_E in binary order
        for i in range(sp.N):
            lv = [(i // 3 ** (q - 1 - k)) % 3 for k in range(q)]
            if max(lv) == 2:
                assert np.all(V[i] == 0)
            else:
                e = int("".join(map(str, lv)), 2)
                np.testing.assert_allclose(V[i], np.exp(2j * np.pi * e * np.arange(sp.E) / sp.E) / math.sqrt(sp.E),
                                           atol=1e-14)


# ----------------------------------------------------------------------------- time stepping
@pytest.mark.parametrize("q,nsteps", [(2, 60), (4, 12), (5, 2)])
def test_zero_controls_closed_form(q, nsteps):
    """alpha = 0: H = diag(D), each row evolves by ((1 - i h D/2)/(1 + i h D/2))^n exactly."""
    sp = S.transmon_spec(q, 0.05 * nsteps, nsteps, 1, 4)
    rng = np.random.default_rng(q)
    W = rand_state(rng, sp.N, 3)
    h = sp.T / sp.nsteps
    D = drift_closed_form(sp)
    want = (((1 - 0.5j * h * D) / (1 + 0.5j * h * D)) ** nsteps)[:, None] * W
    got = oracle.propagate(sp, np.zeros(sp.d), 0, nsteps, W)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_constant_controls_cayley_eigendecomposition(q):
    sp = S.transmon_spec(q, 8.0, 400, 1, 6)
    rng = np.random.default_rng(7 + q)
    val = (rng.uniform(-0.05, 0.05, q) + 1j * rng.uniform(-0.05, 0.05, q))
    alpha = constant_alpha(sp, val)
    W = rand_state(rng, sp.N, sp.E)
    H = kron_hamiltonian(sp, val)
    want = cayley_power(H, sp.T / sp.nsteps, sp.nsteps) @ W
    got = oracle.propagate(sp, alpha, 0, sp.nsteps, W)
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-13)


def test_two_level_second_order_vs_dense_exponential():
    """q=1, L=2, constant control: error vs expm(-iHT) falls ~4x per halving of h (2nd order)."""
    errs = []
    for ns in (50, 100, 200, 400):
        sp = S.ProblemSpec(q=1, L=2, ness=2, xi=[0.0], xi_cross=[[0.0]], omega=[[0.0]], d1=4, T=20.0,
                           nsteps=ns, M=1, detune=[0.3])
        val = np.array([0.11 - 0.07j])
        alpha = constant_alpha(sp, val)
        H = kron_hamiltonian(sp, val)
        W = np.eye(2, dtype=complex)
        exact = scipy.linalg.expm(-1j * H * sp.T) @ W
        got = oracle.propagate(sp, alpha, 0, ns, W)
        errs.append(np.linalg.norm(got - exact))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.9 < r < 4.1 for r in ratios), ratios


def test_norm_preservation_and_isometry():
    sp = S.transmon_spec(2, 50.0, 2000, 1, 10)
    alpha = S.random_alpha(sp, 5, amp=0.05)
    rng = np.random.default_rng(1)
    W = rand_state(rng, sp.N, sp.E) * 3.0          # non-unitary
    U = oracle.propagate(sp, alpha, 0, sp.nsteps, W)
    assert np.linalg.norm(U) == pytest.approx(np.linalg.norm(W), rel=1e-13)
    W0 = oracle.identity_state(sp)                 # isometric embedding stays isometric
    U0 = oracle.propagate(sp, alpha, 0, sp.nsteps, W0)
    np.testing.assert_allclose(U0.conj().T @ U0, np.eye(sp.E), atol=1e-13)


def test_time_reversibility():
    """forward midpoint steps followed by the adjoint steps (C_n^+ = C_n^{-1}) return W."""
    sp = S.transmon_spec(3, 30.0, 500, 1, 8)
    alpha = S.random_alpha(sp, 9, amp=0.05)
    rng = np.random.default_rng(2)
    W = rand_state(rng, sp.N, sp.E)
    U = oracle.propagate(sp, alpha, 100, 400, W)
    back = oracle.propagate_adjoint(sp, alpha, 100, 400, U)
    np.testing.assert_allclose(back, W, atol=1e-13)


def test_window_ranges_cover_the_grid():
    sp = S.config_4q(M=64)
    edges = [oracle.window_range(sp, m) for m in range(1, sp.M + 1)]
    assert edges[0][0] == 0 and edges[-1][1] == sp.nsteps
    for (a0, a1), (b0, b1) in zip(edges, edges[1:]):
        assert a1 == b0
    lens = {b - a for a, b in edges}
    assert lens <= {sp.nsteps // sp.M, sp.nsteps // sp.M + 1}


# ----------------------------------------------------------------------------- infidelity
def test_generalized_infidelity_properties():
    sp = S.transmon_spec(2, 1.0, 1, 1, 3)
    V = oracle.target(sp)
    rng = np.random.default_rng(3)
    for beta in (1.0, 0.3 - 2j, 1e3j):
        assert abs(oracle.infidelity(sp, beta * V)) < 1e-12 * max(1, abs(beta) ** 2)
    for _ in range(20):
        U = rand_state(rng, sp.N, sp.E) * rng.uniform(0.1, 10)
        assert oracle.infidelity(sp, U) >= -1e-15
    # exact quadratic along a random non-unitary direction, with nonnegative curvature
    U, D = rand_state(rng, sp.N, sp.E), rand_state(rng, sp.N, sp.E)
    ts = np.array([-2.0, -1.0, 0.0, 1.0, 2.0])
    vals = np.array([oracle.infidelity(sp, U + t * D) for t in ts])
    coef = np.polyfit(ts, vals, 4)
    assert abs(coef[0]) < 1e-13 and abs(coef[1]) < 1e-13
    assert coef[2] > 0


def test_infidelity_hessian_spectrum():
    """J(U) = <vec U, Q_v vec U>/n with Q_v = I - vec V vec V^+/n: in real coordinates the
    Hessian has eigenvalue 0 twice (V and iV directions) and 2/n otherwise (Eq. gen-infid)."""
    sp = S.ProblemSpec(q=1, L=2, ness=2, xi=[0.0], xi_cross=[[0.0]], omega=[[0.0]], d1=3, T=1, nsteps=1, M=1)
    n = sp.N * sp.E
    dim = 2 * n

    def Jreal(x):
        return oracle.infidelity(sp, oracle.f64_to_cplx(x, sp.N))

    Hm = np.zeros((dim, dim))
    eye = np.eye(dim)
    for i in range(dim):
        for j in range(dim):
            Hm[i, j] = Jreal(eye[i] + eye[j]) - Jreal(eye[i]) - Jreal(eye[j])   # = 2 A_ij for J = x^T A x
    ev = np.sort(np.linalg.eigvalsh(Hm))
    E = sp.E
    np.testing.assert_allclose(ev[:2], 0, atol=1e-14)
    np.testing.assert_allclose(ev[2:], 2.0 / E, atol=1e-14)


def test_infidelity_equals_trace_infidelity_for_isometries():
    sp = S.transmon_spec(2, 1.0, 1, 1, 3)
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((sp.N, sp.N)) + 1j * rng.standard_normal((sp.N, sp.N))
    Q, _ = np.linalg.qr(Z)
    U = Q[:, :sp.E]
    V = oracle.target(sp)
    G = 1 - abs(np.trace(V.conj().T @ U)) ** 2 / sp.E ** 2       # Eq. trace-infid with n := E
    assert oracle.infidelity(sp, U) == pytest.approx(G, abs=1e-14)


# ----------------------------------------------------------------------------- objective
def test_consistent_windows_reduce_to_single_shooting():
    """W = roll-out states: every penalty vanishes and P equals the M=1 objective (bitwise,
    same grid, same arithmetic)."""
    sp = S.transmon_spec(2, 20.0, 400, 5, 6)
    alpha = S.random_alpha(sp, 21)
    W = oracle.rollout(sp, alpha)
    r = oracle.evaluate(sp, alpha, W, grad=False)
    assert np.all(r["pen"] == 0.0)
    r1 = oracle.evaluate(sp.replace(M=1), alpha, np.zeros(0), grad=False)
    assert r["P"] == r1["P"] == r["J"]


def test_objective_terms_match_propagation():
    sp = S.transmon_spec(2, 12.0, 240, 3, 5)
    alpha, W = S.random_alpha(sp, 2), S.random_W(sp, 2)
    r = oracle.evaluate(sp, alpha, W, grad=False, per_window=True)
    mu = 2.0 / sp.E
    prev = oracle.identity_state(sp)
    total = 0.0
    for m in range(1, sp.M + 1):
        n0, n1 = oracle.window_range(sp, m)
        Um = oracle.propagate(sp, alpha, n0, n1, prev)
        if m < sp.M:
            pen = 0.5 * mu * np.linalg.norm(Um - Wmat(sp, W, m)) ** 2
            assert r["pen"][m - 1] == pytest.approx(pen, rel=1e-13)
            total += pen
            prev = Wmat(sp, W, m)
        else:
            V = oracle.target(sp)
            J = np.linalg.norm(Um) ** 2 / sp.E - abs(np.vdot(V, Um)) ** 2 / sp.E ** 2
            assert r["J"] == pytest.approx(J, rel=1e-13)
            total += J
    assert r["P"] == pytest.approx(total, rel=1e-13)


def test_rollout_identity_and_estimate():
    """U_ro = U^M + sum_m (prod S) C^m (Eq. constraint) and the roll-out estimate
    (Eq. rollout-infid-est) bounds J(U_ro)."""
    sp = S.transmon_spec(2, 16.0, 320, 4, 6)
    alpha, W = S.random_alpha(sp, 8), S.random_W(sp, 8) * 0.05
    Wro = oracle.rollout(sp, alpha)
    W = Wro + W                                      # perturbed boundary states
    W0 = oracle.identity_state(sp)
    Uro = oracle.propagate(sp, alpha, 0, sp.nsteps, W0)
    nM0, _ = oracle.window_range(sp, sp.M)
    UM = oracle.propagate(sp, alpha, nM0, sp.nsteps, Wmat(sp, W, sp.M - 1))
    acc = UM.copy()
    cnorm = 0.0
    prev = W0
    for m in range(1, sp.M):
        n0, n1 = oracle.window_range(sp, m)
        Cm = oracle.propagate(sp, alpha, n0, n1, prev) - Wmat(sp, W, m)
        cnorm += np.linalg.norm(Cm)
        acc += oracle.propagate(sp, alpha, n1, sp.nsteps, Cm)
        prev = Wmat(sp, W, m)
    np.testing.assert_allclose(acc, Uro, atol=1e-13)
    JM, Jro = oracle.infidelity(sp, UM), oracle.infidelity(sp, Uro)
    est = JM + 2 / math.sqrt(sp.E) * math.sqrt(JM) * cnorm + cnorm ** 2 / sp.E
    assert Jro <= est * (1 + 1e-12)


# ----------------------------------------------------------------------------- gradient
def _fd_check(sp, alpha, W, idx_alpha, idx_W, eps=1e-6, rtol=2e-6):
    r = oracle.evaluate(sp, alpha, W, nthreads=4)
    ga, gW = r["grad_alpha"], r["grad_W"]
    scale_a = np.max(np.abs(ga))
    scale_w = np.max(np.abs(gW)) if gW.size else 1.0
    for l in idx_alpha:
        ap, am = alpha.copy(), alpha.copy()
        ap[l] += eps
        am[l] -= eps
        fd = (oracle.evaluate(sp, ap, W, grad=False)["P"] - oracle.evaluate(sp, am, W, grad=False)["P"]) / (2 * eps)
        assert abs(fd - ga[l]) <= rtol * max(abs(ga[l]), 1e-3 * scale_a), (l, fd, ga[l])
    for l in idx_W:
        wp, wm = W.copy(), W.copy()
        wp[l] += eps
        wm[l] -= eps
        fd = (oracle.evaluate(sp, alpha, wp, grad=False)["P"] - oracle.evaluate(sp, alpha, wm, grad=False)["P"]) / (2 * eps)
        assert abs(fd - gW[l]) <= rtol * max(abs(gW[l]), 1e-3 * scale_w), (l, fd, gW[l])


def test_gradient_fd_one_transmon_all_components():
    sp = S.transmon_spec(1, 10.0, 120, 3, 5)
    alpha, W = S.random_alpha(sp, 31, amp=0.2), S.random_W(sp, 31)
    _fd_check(sp, alpha, W, range(sp.d), range(sp.nW))


def test_gradient_fd_two_transmons():
    sp = S.transmon_spec(2, 12.0, 160, 4, 5)
    alpha, W = S.random_alpha(sp, 32, amp=0.1), S.random_W(sp, 32)
    rng = np.random.default_rng(0)
    _fd_check(sp, alpha, W, range(sp.d), rng.choice(sp.nW, 60, replace=False))


def test_gradient_fd_single_window_and_paper_model():
    """M = 1 (pure infidelity gradient) on the paper's 2-level model with exchange coupling."""
    sp = S.ProblemSpec(q=2, L=2, ness=2, xi=[0.0] * 2, xi_cross=[[0.0] * 2] * 2,
                       omega=[[-0.19, 0.19], [-0.19, 0.19]], d1=6, T=15.0, nsteps=150, M=1,
                       detune=[0.19, -0.19], jx=[[0, 0.0314], [0, 0]])
    alpha = S.random_alpha(sp, 33, amp=0.1)
    _fd_check(sp, alpha, np.zeros(0), range(sp.d), [])


def test_initial_adjoint_norm_is_terminal_norm():
    """Lambda^m(t_{m-1}) = (S^m)^+ Xi_m is a unitary image of the terminal condition."""
    sp = S.transmon_spec(2, 12.0, 240, 3, 5)
    alpha, W = S.random_alpha(sp, 4), S.random_W(sp, 4)
    r = oracle.evaluate(sp, alpha, W, per_window=True)
    ne2 = 2 * sp.N * sp.E
    mu = 2.0 / sp.E
    V = oracle.target(sp)
    for m in range(1, sp.M + 1):
        Uend = oracle.f64_to_cplx(r["Uend"][ne2 * (m - 1): ne2 * m], sp.N)
        Lam0 = oracle.f64_to_cplx(r["Lam0"][ne2 * (m - 1): ne2 * m], sp.N)
        if m < sp.M:
            xi_norm = 0.5 * mu * np.linalg.norm(Wmat(sp, W, m) - Uend)
        else:
            g = np.vdot(V, Uend)
            xi_norm = np.linalg.norm(g * V - sp.E * Uend) / sp.E ** 2
        assert np.linalg.norm(Lam0) == pytest.approx(xi_norm, rel=1e-12)


# ----------------------------------------------------------------------------- regularization
def _constant_envelope_alpha(spec, coeffs):
    """alpha whose every spline coefficient of carrier (k, f) is coeffs[(k, f)] (complex):
    by the partition of unity the envelope of that carrier is the constant coeffs[(k, f)]."""
    a = np.zeros(spec.d)
    fi = 0
    for k in range(spec.q):
        for f in range(len(spec.omega[k])):
            c = coeffs.get((k, f), 0.0)
            blk = a[2 * spec.d1 * fi: 2 * spec.d1 * (fi + 1)]
            blk[0::2], blk[1::2] = c.real if c else 0.0, c.imag if c else 0.0
            fi += 1
    return a


def test_control_energy_of_constant_envelopes_is_the_amplitude_squared():
    # the time average of a constant |d_k|^2
    sp = S.transmon_spec(2, 12.0, 300, 1, 7)
    c = {(0, 0): 0.3 - 0.2j, (1, 0): -0.1 + 0.05j}          # carrier 0 has Omega = 0
    R, _ = oracle.regularization(sp, _constant_envelope_alpha(sp, c), 0.0, 1.0)
    want = sum(abs(v) ** 2 for v in c.values())
    assert R == pytest.approx(want, rel=1e-13)


def test_control_energy_two_carriers_geometric_sum():
    # |c0 + c1 e^{i D t}|^2 = |c0|^2 + |c1|^2 + 2 Re(conj(c0) c1 e^{i D t}); the midpoint sum of
    # the oscillating term is a geometric series with a closed form
    sp = S.transmon_spec(1, 10.0, 250, 1, 6)
    c0, c1 = 0.4 + 0.1j, -0.2 + 0.3j
    R, _ = oracle.regularization(sp, _constant_envelope_alpha(sp, {(0, 0): c0, (0, 1): c1}), 0.0, 1.0)
    D = sp.omega[0][1] - sp.omega[0][0]
    h, n = sp.T / sp.nsteps, sp.nsteps
    geo = h * np.exp(0.5j * D * h) * (1 - np.exp(1j * D * h * n)) / (1 - np.exp(1j * D * h))
    want = (sp.T * (abs(c0) ** 2 + abs(c1) ** 2) + 2 * (np.conj(c0) * c1 * geo).real) / sp.T
    assert R == pytest.approx(want, rel=1e-12)


def test_tikhonov_term_closed_form():
    sp = S.transmon_spec(2, 8.0, 100, 2, 5)
    a = S.random_alpha(sp, 3)
    R, g = oracle.regularization(sp, a, 0.7, 0.0)
    assert R == pytest.approx(0.35 * float(a @ a), rel=1e-14)
    np.testing.assert_allclose(g, 0.7 * a, rtol=1e-15)


def test_regularization_gradient_central_differences_and_euler_identity():
    # R is a quadratic in alpha: central differences are exact up to rounding, and for the
    # homogeneous energy term alpha . grad E = 2 E
    sp = S.paper_qft_spec(2, nsteps=240).replace(T=20.0, d1=9)
    a = S.random_alpha(sp, 5, amp=2 * np.pi * 0.01)
    gt, ge = 1e-3 / sp.d, 1e-3
    R, g = oracle.regularization(sp, a, gt, ge)
    fd = np.empty(sp.d)
    eps = 1e-3
    for j in range(sp.d):
        e = np.zeros(sp.d)
        e[j] = eps
        fd[j] = (oracle.regularization(sp, a + e, gt, ge)[0] - oracle.regularization(sp, a - e, gt, ge)[0]) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-8, atol=1e-10 * np.max(np.abs(g)))
    E, gE = oracle.regularization(sp, a, 0.0, 1.0)
    assert float(a @ gE) == pytest.approx(2 * E, rel=1e-12)

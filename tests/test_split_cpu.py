"""The compensated FP32 arithmetic of the mixed solver's gradient products, run on the host
(the same source is compiled for the device; tests/test_gpu_split.py checks that the device
gives the same bits).  Pinned against exact rational arithmetic (fractions.Fraction), not
against another floating-point implementation:

* the split x 2^-sh = hi + lo: hi is x 2^-sh rounded to 24 bits (float32 rounding, away from
  zero at ties), |x 2^-sh - hi - lo| <= 2^-48 |x 2^-sh|, and the documented range edges;
* the dot product built from the splits: its error is at most a few 2^-47 of sum |x_i y_i|,
  including sums that cancel to zero or almost;
* the compensated state update of the implicit midpoint rule (Sec. 5), U_{j+1} = R U_j + 2 d_j
  with R = 2P - 1 = 1 - 2 i kappa P: against the same map in 320-bit arithmetic (mpmath) its
  error is a random walk of about 2^-53 |U| a step, and with d = 0 it follows the exact Cayley
  factor (1 - i kappa) / (1 + i kappa) of the diagonal step.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2407_13950_gb300 import msqoc

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _exact_err(x, sh, hi, lo):
    xs = Fr(float(x)) / Fr(2) ** sh
    return abs(xs - Fr(float(hi)) - Fr(float(lo))), abs(xs)


@pytest.mark.parametrize("sh", [0, 7, -7, 600, -600])
def test_split_error_and_leading_part(sh):
    rng = np.random.default_rng(1000 + sh)
    x = rng.standard_normal(3000) * 2.0 ** rng.integers(-70, 10, 3000)
    x = x * 2.0 ** sh
    hi, lo = msqoc.selftest_split(x, sh)
    scaled = x * 2.0 ** -sh
    np.testing.assert_array_equal(hi, scaled.astype(np.float32))   # no exact ties in random data
    for i in range(0, x.size, 5):
        err, mag = _exact_err(x[i], sh, hi[i], lo[i])
        # below 2^-74 (scaled) the remainder is not kept: the leading part's 2^-24 only
        bound = Fr(1, 2 ** 48) if mag >= Fr(1, 2 ** 74) else Fr(1, 2 ** 24)
        assert err <= mag * bound, (x[i], hi[i], lo[i])


def test_split_tie_rounds_away_from_zero():
    # 1 + 2^-24 (a tie at 24 bits) and its negative: hi rounds away from zero, lo = -2^-24
    x = np.array([1.0 + 2.0 ** -24, -(1.0 + 2.0 ** -24), 1.0 + 3 * 2.0 ** -24])
    hi, lo = msqoc.selftest_split(x, 0)
    assert hi[0] == np.float32(1.0 + 2.0 ** -23) and lo[0] == np.float32(-(2.0 ** -24))
    assert hi[1] == -np.float32(1.0 + 2.0 ** -23) and lo[1] == np.float32(2.0 ** -24)
    assert hi[2] == np.float32(1.0 + 2.0 ** -22) and lo[2] == np.float32(-(2.0 ** -24))


def test_split_carry_into_the_exponent():
    # the largest double below 2: hi rounds up to 2, lo is the (negative) remainder
    x = np.array([np.nextafter(2.0, 0.0), -np.nextafter(2.0, 0.0), np.nextafter(0.5, 0.0)])
    hi, lo = msqoc.selftest_split(x, 0)
    for i in range(3):
        err, mag = _exact_err(x[i], 0, hi[i], lo[i])
        assert err == 0 or err <= mag * Fr(1, 2 ** 48)
    assert hi[0] == 2.0 and lo[0] == -(2.0 ** -52) and hi[1] == -2.0 and lo[1] == 2.0 ** -52


def test_split_range_edges():
    tiny = 2.0 ** -127                          # below the FP32 normal range after scaling
    x = np.array([0.0, -0.0, 5e-324, tiny, 2.0 ** -100 * (1 + 2.0 ** -40), 2.0 ** -75 * (1 + 2.0 ** -40),
                  2.0 ** -74 * (1 + 2.0 ** -40)])
    hi, lo = msqoc.selftest_split(x, 0)
    assert list(hi[:4]) == [0.0, 0.0, 0.0, 0.0] and list(lo[:4]) == [0.0, 0.0, 0.0, 0.0]
    assert np.signbit(hi[1]) and np.signbit(lo[1])
    # between 2^-126 and 2^-74: the leading part only
    assert hi[4] == np.float32(x[4]) and lo[4] == 0.0
    assert hi[5] == np.float32(x[5]) and lo[5] == 0.0
    # from 2^-74 on: the remainder too
    err, mag = _exact_err(x[6], 0, hi[6], lo[6])
    assert lo[6] != 0.0 and err <= mag * Fr(1, 2 ** 48)
    # the scale moves the edges with it
    hi2, lo2 = msqoc.selftest_split(x * 2.0 ** 300, 300)
    np.testing.assert_array_equal(hi2[3:], hi[3:])
    np.testing.assert_array_equal(lo2[3:], lo[3:])


def _dot_err(x, y, got):
    ex = sum(Fr(float(a)) * Fr(float(b)) for a, b in zip(x, y))
    mag = sum(abs(Fr(float(a)) * Fr(float(b))) for a, b in zip(x, y))
    return abs(Fr(got) - ex), mag, ex


@pytest.mark.parametrize("shx,shy", [(0, 0), (12, -40), (500, -480), (-700, -300)])
def test_dot_error_bound_with_cancellation(shx, shy):
    rng = np.random.default_rng(1000 + shx)
    for trial in range(20):
        n = int(rng.integers(1, 60))
        x = rng.standard_normal(n)
        y = rng.standard_normal(n)
        if n > 1 and trial % 2 == 0:               # cancel the sum to (almost) zero
            y[-1] = -np.dot(x[:-1], y[:-1]) / x[-1]
        xs, ys = x * 2.0 ** shx, y * 2.0 ** shy
        got = msqoc.selftest_dot(xs, ys, shx, shy)
        err, mag, _ = _dot_err(xs, ys, got)
        assert err <= mag * Fr(8, 2 ** 47), (trial, float(err / mag))


def test_dot_exact_cases():
    # a product that fits 24 bits exactly and a sum of two that cancel exactly
    assert msqoc.selftest_dot([3.0], [5.0]) == 15.0
    assert msqoc.selftest_dot([1.0 + 2.0 ** -30, 1.0 + 2.0 ** -30], [1.0, -1.0]) == 0.0
    # the double x = 1 + 2^-30 squared needs the cross terms: 1 + 2^-29 + 2^-60
    got = msqoc.selftest_dot([1.0 + 2.0 ** -30], [1.0 + 2.0 ** -30])
    assert got == 1.0 + 2.0 ** -29              # the dropped lo*lo term is 2^-60, below the double's ulp
    assert msqoc.selftest_dot([], []) == 0.0


def test_dot_scale_range():
    # scales that move the result beyond the double range saturate instead of wrapping
    assert msqoc.selftest_dot([2.0 ** 1000], [2.0 ** 1000], 1000, 1000) == np.inf
    assert msqoc.selftest_dot([2.0 ** -1000], [2.0 ** -1000], -1000, -1000) == 0.0
    assert msqoc.selftest_dot([2.0 ** 600], [2.0 ** -500], 600, -500) == 2.0 ** 100


def test_selftests_reject_bad_arguments():
    lib = msqoc.load()
    assert lib.msqoc_selftest_split(None, 4, 0, 0, None, None) == -1
    assert lib.msqoc_selftest_split(None, 0, 5000, 0, None, None) == -1
    assert lib.msqoc_selftest_dot(None, None, -1, 0, 0, 0, None) == -1


# ------------------------------------------------------------------ compensated state update
def _carry_map(u0, P, d):
    """u_{j+1} = u_j + k2 (Im(P u_j), -Re(P u_j)) + 2 d_j in 320-bit arithmetic, k2 = -2 Im P / Re P
    rounded to a double as the library forms it (R - 1 = 2 (P - 1) = -2 i kappa P)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 320
    M = mp.mpf
    px, py = M(P.real), M(P.imag)
    k2 = M(-2.0 * P.imag / P.real)
    ur, ui = M(u0.real), M(u0.imag)
    for dj in d:
        br, bi = px * ur - py * ui, px * ui + py * ur
        ur, ui = ur + k2 * bi + 2 * M(dj.real), ui - k2 * br + 2 * M(dj.imag)
    return ur, ui


def _carry_err(got, ref, mag):
    return float(abs((got.real - ref[0]) + 1j * (got.imag - ref[1]))) / mag / 2.0 ** -53


def test_carry_update_one_step():
    rng = np.random.default_rng(2001)
    worst = 0.0
    for _ in range(200):
        mag = rng.uniform(0.05, 1.0)
        u0 = mag * np.exp(1j * rng.uniform(0, 2 * np.pi))
        P = 1.0 / complex(1.0, rng.uniform(-0.022, 0.022))
        d = (rng.standard_normal(1) + 1j * rng.standard_normal(1)) * 1e-3 * mag
        got = msqoc.selftest_carry(u0, P, d, sh=int(rng.integers(-5, 6)))
        worst = max(worst, _carry_err(got, _carry_map(u0, P, d), mag))
    assert worst <= 6.0, worst          # a few units of 2^-53 |U| (measured: about 3)


def test_carry_update_error_is_a_random_walk():
    # 64 steps with corrections: the errors of the steps add like independent roundings
    # (about 0.6 2^-53 |U| rms a step), not like a constant error of P or kappa (the splits of
    # both are exact) nor like a carry that keeps the low parts of every step
    rng = np.random.default_rng(2002)
    n, errs = 64, []
    for _ in range(30):
        mag = rng.uniform(0.3, 1.0)
        u0 = mag * np.exp(1j * rng.uniform(0, 2 * np.pi))
        P = 1.0 / complex(1.0, rng.uniform(-0.022, 0.022))
        d = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1e-3 * mag
        got = msqoc.selftest_carry(u0, P, d)
        errs.append(_carry_err(got, _carry_map(u0, P, d), mag))
    errs = np.array(errs)
    assert np.sqrt(np.mean(errs ** 2)) <= 2.0 * np.sqrt(n), errs
    assert errs.max() <= 6.0 * np.sqrt(n), errs


def test_carry_update_follows_the_cayley_factor():
    # d = 0: the diagonal part of the implicit midpoint step alone, U_n = R^n U_0 with the
    # Cayley factor R = (1 - i kappa) / (1 + i kappa) of kappa = (h/2) D; P = 1 / (1 + i kappa)
    # is rounded to doubles, which moves R by about |kappa| 2^-53 a step in this form (R = 2P - 1
    # formed in FP64 from the rounded P would be off by up to 2^-52 a step: 300-800 units here)
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 320
    rng = np.random.default_rng(2003)
    n = 400
    for kap in (0.0, 3e-4, -0.0083, 0.022):
        u0 = 0.8 * np.exp(1j * rng.uniform(0, 2 * np.pi))
        P = 1.0 / complex(1.0, kap)
        got = msqoc.selftest_carry(u0, P, np.zeros(n, complex))
        k = mp.mpf(kap)
        R = (1 - 1j * k) / (1 + 1j * k)
        want = mp.mpc(u0.real, u0.imag) * R ** n
        err = float(abs(mp.mpc(got.real, got.imag) - want)) / 0.8 / 2.0 ** -53
        assert err <= 3.0 * np.sqrt(n), (kap, err)        # measured: 2-12
    assert msqoc.selftest_carry(0.3 - 0.4j, 1.0, np.zeros(5)) == 0.3 - 0.4j     # kappa = 0: exact


def test_carry_selftest_rejects_bad_arguments():
    with pytest.raises(msqoc.MsqocError):
        msqoc.selftest_carry(1.0, 1.0 / complex(1.0, 0.03), np.zeros(3))     # |2 kappa| > 2^-4.5
    with pytest.raises(msqoc.MsqocError):
        msqoc.selftest_carry(1.0, complex(0.4, 0.0), np.zeros(3))            # Re P outside (1/2, 1]
    with pytest.raises(msqoc.MsqocError):
        msqoc.selftest_carry(1.0, 1.0, np.zeros(3), sh=897)

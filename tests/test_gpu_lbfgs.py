"""L-BFGS steps of the client optimiser on the device (msqoc_lbfgs_direction / _trial / _update)
against a plain numpy statement of the same operations: the projected two-loop recursion over
a ring of stored pairs, the clipped trial point and the memory update."""
import numpy as np
import pytest

from paper_2407_13950_gb300 import msqoc

pytestmark = pytest.mark.gpu


def active_np(x, g, lim, nb):
    act = np.zeros(x.size, dtype=bool)
    if nb:
        a, ga = x[:nb], g[:nb]
        act[:nb] = ((a >= lim) & (ga < 0)) | ((a <= -lim) & (ga > 0))
    return act


def direction_np(x, g, lim, nb, pairs):
    """pairs: [(s, y)] oldest first"""
    act = active_np(x, g, lim, nb)
    pg = np.where(act, 0.0, g)
    q = pg.copy()
    alphas = []
    for s, y in reversed(pairs):
        a = (s @ q) / (s @ y)
        q -= a * y
        alphas.append(a)
    if pairs:
        s, y = pairs[-1]
        q *= (s @ y) / (y @ y)
    else:
        q /= max(np.linalg.norm(q), 1e-300)
    for (s, y), a in zip(pairs, reversed(alphas)):
        q += (a - (y @ q) / (s @ y)) * s
    dvec = np.where(act, 0.0, -q)
    return dvec, pg @ dvec


@pytest.mark.parametrize("n,nb,cap,m,head", [(1000, 300, 5, 3, 1), (3001, 0, 4, 4, 2), (7, 7, 3, 0, 0),
                                             (50000, 640, 10, 10, 0), (2000, 100, 8, 5, 6)])
def test_direction_matches_two_loop_recursion(n, nb, cap, m, head):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(n + cap + m)
    x = rng.uniform(-1, 1, n)
    g = rng.standard_normal(n)
    lim = rng.uniform(0.3, 0.9, nb)
    if nb:
        x[:nb] = np.clip(x[:nb], -lim, lim)          # some entries sit on their bound
    S = rng.standard_normal((cap, n)) * 0.1
    Y = S + 0.05 * rng.standard_normal((cap, n))      # <s, y> > 0
    slots = [(head - m + j) % cap for j in range(m)]  # oldest first
    pairs = [(S[k], Y[k]) for k in slots]
    want_d, want_slope = direction_np(x, g, lim, nb, pairs)
    dev = torch.device("cuda")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev, dtype=torch.float64)
    rho = np.array([1.0 / (S[k] @ Y[k]) for k in range(cap)])
    yy = np.array([Y[k] @ Y[k] for k in range(cap)])
    d_out = torch.full((n,), np.nan, device=dev, dtype=torch.float64)
    slope = torch.zeros(1, device=dev, dtype=torch.float64)
    msqoc.lbfgs_direction(n, nb, T(x), T(g), T(lim) if nb else None, T(S), T(Y), T(rho), T(yy), cap, m, head,
                          d_out, slope)
    got = d_out.cpu().numpy()
    np.testing.assert_allclose(got, want_d, rtol=1e-11, atol=1e-13 * np.max(np.abs(want_d)))
    assert slope.item() == pytest.approx(want_slope, rel=1e-11)
    assert slope.item() < 0
    act = active_np(x, g, lim, nb)
    assert np.all(got[act] == 0.0)


def test_trial_and_update():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    n, nb = 4097, 1000
    x = rng.uniform(-0.5, 0.5, n)
    dvec = rng.standard_normal(n)
    g = rng.standard_normal(n)
    lim = rng.uniform(0.4, 0.6, nb)
    dev = torch.device("cuda")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev, dtype=torch.float64)
    x_new = torch.empty(n, device=dev, dtype=torch.float64)
    dec = torch.zeros(1, device=dev, dtype=torch.float64)
    msqoc.lbfgs_trial(n, nb, T(x), T(dvec), 0.25, T(lim), T(g), x_new, dec)
    want = x + 0.25 * dvec
    want[:nb] = np.clip(want[:nb], -lim, lim)
    np.testing.assert_array_equal(x_new.cpu().numpy(), want)
    assert dec.item() == pytest.approx(g @ (want - x), rel=1e-12)
    g_new = g + rng.standard_normal(n)
    s_out = torch.empty(n, device=dev, dtype=torch.float64)
    y_out = torch.empty(n, device=dev, dtype=torch.float64)
    syy = torch.zeros(2, device=dev, dtype=torch.float64)
    msqoc.lbfgs_update(n, T(x), x_new, T(g), T(g_new), s_out, y_out, syy)
    s, y = want - x, g_new - g
    np.testing.assert_array_equal(s_out.cpu().numpy(), s)
    np.testing.assert_array_equal(y_out.cpu().numpy(), y)
    np.testing.assert_allclose(syy.cpu().numpy(), [s @ y, y @ y], rtol=1e-12)


def test_direction_rejects_bad_memory_and_host_arrays():
    torch = pytest.importorskip("torch")
    n = 16
    dev = torch.device("cuda")
    x = torch.zeros(n, device=dev, dtype=torch.float64)
    g = torch.ones(n, device=dev, dtype=torch.float64)
    d_out = torch.zeros(n, device=dev, dtype=torch.float64)
    slope = torch.zeros(1, device=dev, dtype=torch.float64)
    S = torch.zeros((2, n), device=dev, dtype=torch.float64)
    r = torch.ones(2, device=dev, dtype=torch.float64)
    for cap, m, head in ((2, 3, 0), (msqoc.LBFGS_MAXMEM + 1, 1, 0), (2, 1, 2)):
        with pytest.raises(msqoc.MsqocError) as err:
            msqoc.lbfgs_direction(n, 0, x, g, None, S, S, r, r, cap, m, head, d_out, slope)
        assert err.value.status == -1
    with pytest.raises(msqoc.MsqocError) as err:
        msqoc.lbfgs_direction(n, 0, np.zeros(n), g, None, S, S, r, r, 2, 0, 0, d_out, slope)
    assert err.value.status == -1

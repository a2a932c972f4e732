"""Pins of the oracle's Grunwald coefficients and WSGD weights against what
the paper fixes (Eq. gk and its listed properties, Proposition ww, Eq. fgamma)
and against an independent library routine."""
import numpy as np
import pytest
from scipy.special import binom

from oracle.wsgd import grunwald_g, wsgd_weights, GAMMA0

GAMMAS = [1.1, 1.3, 1.5, 1.6, 1.7, 1.8, 1.9]


@pytest.mark.parametrize("g", GAMMAS)
def test_g_matches_library_binomial(g):
    # Eq. (gk): g_k = (-1)^k binom(gamma, k); scipy evaluates binom through Gamma functions
    K = 300
    ref = (-1.0) ** np.arange(K + 1) * binom(g, np.arange(K + 1))
    np.testing.assert_allclose(grunwald_g(g, K), ref, rtol=1e-11, atol=1e-300)


@pytest.mark.parametrize("g", GAMMAS)
def test_g_properties(g):
    # properties listed after Eq. (gk): g0 = 1, g1 = -gamma, g2 > g3 > ... > 0,
    # partial sums < 0 for n >= 1 and the full sum 0, g_j = O(j^-(gamma+1))
    K = 20000
    gk = grunwald_g(g, K)
    assert gk[0] == 1.0 and gk[1] == -g
    assert np.all(gk[2:] > 0) and np.all(np.diff(gk[2:]) < 0)
    ps = np.cumsum(gk)
    assert np.all(ps[1:] < 0)
    # closed form of the partial sum: sum_{j<=K} g_j = (-1)^K binom(gamma-1, K) -> 0
    np.testing.assert_allclose(ps[[10, 100, 1000]], (-1.0) ** np.array([10, 100, 1000])
                               * binom(g - 1, np.array([10, 100, 1000])), rtol=1e-9)
    j = np.array([1000, 4000, 16000])
    ratio = gk[j] * j ** (g + 1)
    assert np.all(np.abs(np.diff(ratio)) / ratio[0] < 0.01)  # asymptotically a constant


@pytest.mark.parametrize("g", GAMMAS)
def test_w_closed_forms_and_properties(g):
    # Proposition (ww)
    K = 20000
    w = wsgd_weights(g, K, 1, 0)
    np.testing.assert_allclose(w[0], g / 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w[1], (2 - g - g * g) / 2, rtol=1e-14)
    np.testing.assert_allclose(w[2], g * (g * g + g - 4) / 4, rtol=1e-13)
    assert w[1] < 0
    assert 1 >= w[0] >= w[3] and np.all(np.diff(w[3:]) <= 0) and np.all(w[3:] >= 0)
    ps = np.cumsum(w)
    assert np.all(ps[2:] < 0)
    assert abs(ps[-1]) < 5 * K ** (-g)  # partial sums -> 0 like the tail K^-gamma


def test_laplacian_limit():
    # gamma = 2: g = (1, -2, 1, 0, ...) and w = (1, -2, 1, 0, ...): A^2 = tridiag(-1, 2, -1)
    np.testing.assert_array_equal(grunwald_g(2.0, 5), [1, -2, 1, 0, 0, 0])
    np.testing.assert_array_equal(wsgd_weights(2.0, 5), [1, -2, 1, 0, 0, 0])


@pytest.mark.parametrize("g", GAMMAS)
@pytest.mark.parametrize("q", [0, -1])
def test_generating_function(g, q):
    # sum_k w_k z^k = (1 - z)^gamma (lambda_p + lambda_q z^(p-q)) for the WSGD
    # combination (Eq. w at q = 0); checked inside the unit disk where the
    # series converges geometrically
    K = 400
    w = wsgd_weights(g, K, 1, q)
    d = 1 - q
    lp, lq = (g - 2 * q) / (2 * d), (2 - g) / (2 * d)
    for z in [0.5, -0.6, 0.3 + 0.5j, -0.2 - 0.7j]:
        series = np.sum(w * z ** np.arange(K + 1))
        closed = (1 - z) ** g * (lp + lq * z ** d)
        assert abs(series - closed) < 1e-12


def test_second_shift_numbers():
    # (1,-1) at gamma = 1.3: w_0 = (g+2)/4, w_1 = -(g+2) g /4
    w = wsgd_weights(1.3, 10, 1, -1)
    np.testing.assert_allclose(w[:2], [0.825, -1.0725], rtol=1e-14)
    assert abs(np.sum(wsgd_weights(1.3, 200000, 1, -1))) < 1e-5


@pytest.mark.parametrize("g", [1.2, 1.6, 1.8])
def test_symbol_closed_form(g):
    # Eq. (fgamma): -sum_{k>=-1} w_{k+1} e^{ik xi} = -[(2 - g(1 - e^{-i xi}))/2] (1 + e^{i(xi+pi)})^g.
    # The truncated series has tail bounded by sum_{k>K} |w_k| <= C K^-g.
    K = 400000
    w = wsgd_weights(g, K, 1, 0)
    for xi in [0.3, 1.0, 2.5, -1.7]:
        series = -np.sum(w * np.exp(1j * (np.arange(K + 1) - 1) * xi))
        closed = -((2 - g * (1 - np.exp(-1j * xi))) / 2) * (1 + np.exp(1j * (xi + np.pi))) ** g
        assert abs(series - closed) < 3 * K ** (-g)
    # q_gamma = 2 Re f_gamma peaks at xi = pi with value (gamma-1) 2^(gamma+1) (Prop. PaPb)
    fpi = -((2 - g * 2) / 2) * (1 + np.exp(1j * 2 * np.pi)) ** g
    np.testing.assert_allclose(2 * fpi.real, (g - 1) * 2 ** (g + 1), rtol=1e-12)


def test_gamma0():
    # Sec. 2: gamma_0 = (-1 + sqrt 17)/2 is where w_2 = gamma (gamma^2 + gamma - 4)/4 changes sign
    w2 = lambda g: g * (g * g + g - 4) / 4
    assert abs(w2(GAMMA0)) < 1e-14 and w2(GAMMA0 - 1e-6) < 0 < w2(GAMMA0 + 1e-6)

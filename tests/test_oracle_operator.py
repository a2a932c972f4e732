"""Pins of the oracle's operators (Sec. 2: Eq. AN, AxAy, M, system; Sec. 3:
Eq. fgamma, phi): the pointwise shifted-Grunwald scheme written with loops, the
BTTB symbol of the constant-coefficient matrix computed from the closed form,
SPD and M-matrix structure, and two library formulations against each other."""
import numpy as np
import pytest

from oracle.wsgd import wsgd_weights, GAMMA0
from oracle.operator import (toeplitz_A, apply_M, assemble_M, apply_M_fft, rhs, rhs_fft,
                             cn_scalars, toeplitz_rows)

rng = np.random.default_rng(7)


def _pointwise_delta(U, w, coefp, coefm, h, al, dt, axis):
    """delta^{gamma} u of Eq. (CNWSGD) by the sums that define L D^gamma_h and
    R D^gamma_h in Sec. 2 (1-based indices, zero Dirichlet values u_0 = u_{n+1} = 0)."""
    n2, n1 = U.shape
    out = np.zeros_like(U)
    for j in range(1, n2 + 1):
        for i in range(1, n1 + 1):
            def u(ii, jj):
                if axis == 0:
                    return U[jj - 1, ii - 1] if 1 <= ii <= n1 else 0.0
                return U[jj - 1, ii - 1] if 1 <= jj <= n2 else 0.0
            if axis == 0:
                L = sum(w[k] * u(i - k + 1, j) for k in range(0, i + 1))
                R = sum(w[k] * u(i + k - 1, j) for k in range(0, n1 - i + 2))
            else:
                L = sum(w[k] * u(i, j - k + 1) for k in range(0, j + 1))
                R = sum(w[k] * u(i, j + k - 1) for k in range(0, n2 - j + 2))
            out[j - 1, i - 1] = (coefp[j - 1, i - 1] * dt / 2 * L + coefm[j - 1, i - 1] * dt / 2 * R) / h ** al
    return out


@pytest.mark.parametrize("q", [0, -1])
def test_matrix_form_equals_pointwise_scheme(q):
    # Eq. (system) divided by r (Eq. M) must reproduce Eq. (CNWSGD) point by point
    n1, n2, al, be, dt = 6, 5, 1.7, 1.4, 0.03
    hx, hy = 1.0 / (n1 + 1), 2.0 / (n2 + 1)
    wx, wy = wsgd_weights(al, n1 + 1, 1, q), wsgd_weights(be, n2 + 1, 1, q)
    cf = [rng.uniform(0.5, 2, (n2, n1)) for _ in range(4)]
    cf_old = [rng.uniform(0.5, 2, (n2, n1)) for _ in range(4)]
    U = rng.standard_normal((n2, n1))
    V = rng.standard_normal((n2, n1))
    sc = cn_scalars(al, be, hx, hy, dt)
    dx = _pointwise_delta(U, wx, cf[0], cf[1], hx, al, dt, 0)
    dy = _pointwise_delta(U, wy, cf[2], cf[3], hy, be, dt, 1)
    lhs = (U - dx - dy) / sc["r"]
    np.testing.assert_allclose(apply_M(U, wx, wy, sc["c"], sc["sigma"], *cf), lhs, rtol=1e-12, atol=1e-12)
    dxo = _pointwise_delta(U, wx, cf_old[0], cf_old[1], hx, al, dt, 0)
    dyo = _pointwise_delta(U, wy, cf_old[2], cf_old[3], hy, be, dt, 1)
    rh = (U + dxo + dyo + dt * V) / sc["r"]
    np.testing.assert_allclose(rhs(U, wx, wy, sc["c"], sc["sigma"], *cf_old, V, hx, al), rh,
                               rtol=1e-12, atol=1e-12)


def _fourier_coeffs_closed_form(g, kmax, L=1 << 18):
    """f^_k, |k| <= kmax, of f_gamma(xi) = -[(2 - g(1 - e^{-i xi}))/2](1 - e^{i xi})^g (Eq. fgamma)
    by an L-point trapezoidal rule (aliasing error ~ L^-(g+1))."""
    xi = 2 * np.pi * np.arange(L) / L
    f = -((2 - g * (1 - np.exp(-1j * xi))) / 2) * (1 + np.exp(1j * (xi + np.pi))) ** g
    fh = np.fft.fft(f) / L
    return {k: fh[k % L] for k in range(-kmax, kmax + 1)}


def test_constant_coefficients_matrix_is_bttb_of_phi():
    # Corollary after Prop. pro2: M = T_N^(2)(phi), phi = 1/r + d+ f_a(t1) + d- f_a(-t1)
    #   + s/r (e+ f_b(t2) + e- f_b(-t2)); T_N^(2)(f) = [f^_{i-j}] (Definition in Sec. 3)
    n1, n2, al, be = 7, 6, 1.6, 1.8
    dp, dm, ep, em = 1.3, 0.7, 0.4, 2.1
    c, sigma = 0.35, 1.7
    fa = _fourier_coeffs_closed_form(al, n1)
    fb = _fourier_coeffs_closed_form(be, n2)
    N = n1 * n2
    T = np.zeros((N, N), dtype=complex)
    for j in range(n2):
        for i in range(n1):
            for jj in range(n2):
                for ii in range(n1):
                    k1, k2 = i - ii, j - jj
                    v = 0.0
                    if k2 == 0:
                        v += dp * fa[k1] + dm * fa[-k1] + (c if k1 == 0 else 0.0)
                    if k1 == 0:
                        v += sigma * (ep * fb[k2] + em * fb[-k2])
                    T[j * n1 + i, jj * n1 + ii] = v
    assert np.max(np.abs(T.imag)) < 1e-12
    wx, wy = wsgd_weights(al, n1), wsgd_weights(be, n2)
    ones = np.ones((n2, n1))
    M = assemble_M(toeplitz_A(wx, n1), toeplitz_A(wy, n2), c, sigma, dp * ones, dm * ones,
                   ep * ones, em * ones)
    np.testing.assert_allclose(M, T.real, atol=1e-10)


def test_toeplitz_structure():
    # Eq. (AN): -w_0 on the super-diagonal, -w_1 on the diagonal, -w_n bottom-left, zero above
    n, g = 9, 1.7
    w = wsgd_weights(g, n)
    A = toeplitz_A(w, n)
    assert np.all(np.triu(A, 2) == 0)
    np.testing.assert_array_equal(np.diag(A, 1), -w[0])
    np.testing.assert_array_equal(np.diag(A), -w[1])
    assert A[n - 1, 0] == -w[n] and A[1, 0] == -w[2]


def test_equal_constant_coefficients_spd():
    # Sec. 2: d+ = d- = d, e+ = e- = e constant => M symmetric positive definite BTTB
    n1, n2 = 9, 8
    for al, be in [(1.2, 1.9), (1.5, 1.5), (1.8, 1.3)]:
        wx, wy = wsgd_weights(al, n1), wsgd_weights(be, n2)
        ones = np.ones((n2, n1))
        M = assemble_M(toeplitz_A(wx, n1), toeplitz_A(wy, n2), 0.01, 0.8, 2 * ones, 2 * ones,
                       ones, ones)
        np.testing.assert_allclose(M, M.T, atol=1e-14)
        assert np.min(np.linalg.eigvalsh(M)) > 0


def test_m_matrix_for_gamma_above_gamma0():
    # Sec. 2: gamma in [gamma_0, 2) => strictly diagonally dominant M-matrix
    n1, n2 = 10, 9
    for al, be in [(GAMMA0 + 1e-9, 1.9), (1.7, 1.6)]:
        wx, wy = wsgd_weights(al, n1), wsgd_weights(be, n2)
        cf = [rng.uniform(0.5, 2, (n2, n1)) for _ in range(4)]
        M = assemble_M(toeplitz_A(wx, n1), toeplitz_A(wy, n2), 0.05, 1.3, *cf)
        off = M - np.diag(np.diag(M))
        assert np.all(off <= 1e-15)
        assert np.all(np.diag(M) > np.sum(np.abs(off), axis=1))
    # below gamma_0 the w_2 entries are positive, so the sign pattern fails
    wx = wsgd_weights(1.3, n1)
    assert toeplitz_A(wx, n1)[1, 0] > 0


@pytest.mark.parametrize("shape", [(9, 13), (37, 41), (64, 31)])
def test_kron_matmul_fft_agree(shape):
    n2, n1 = shape
    al, be = 1.45, 1.85
    wx, wy = wsgd_weights(al, n1, 1, -1), wsgd_weights(be, n2, 1, 0)
    cf = [rng.uniform(0.5, 2, (n2, n1)) for _ in range(4)]
    X = rng.standard_normal((n2, n1))
    y1 = apply_M(X, wx, wy, 0.2, 1.4, *cf)
    y2 = apply_M_fft(X, wx, wy, 0.2, 1.4, *cf)
    np.testing.assert_allclose(y1, y2, rtol=1e-11, atol=1e-11)
    if n1 * n2 <= 1200:
        M = assemble_M(toeplitz_A(wx, n1), toeplitz_A(wy, n2), 0.2, 1.4, *cf)
        np.testing.assert_allclose((M @ X.ravel()).reshape(n2, n1), y1, rtol=1e-12, atol=1e-12)
    V = rng.standard_normal((n2, n1))
    np.testing.assert_allclose(rhs(X, wx, wy, 0.2, 1.4, *cf, V, 0.1, al),
                               rhs_fft(X, wx, wy, 0.2, 1.4, *cf, V, 0.1, al), rtol=1e-11, atol=1e-11)


def test_toeplitz_rows_against_dense():
    n, g = 50, 1.35
    w = wsgd_weights(g, n)
    X = rng.standard_normal((3, n))
    A = toeplitz_A(w, n)
    np.testing.assert_allclose(toeplitz_rows(X, w), X @ A.T, atol=1e-12)
    np.testing.assert_allclose(toeplitz_rows(X, w, True), X @ A, atol=1e-12)


def _q_closed_form(g, xi):
    # q_gamma(xi) = f_gamma(xi) + f_gamma(-xi) = 2 Re f_gamma(xi), f_gamma of Eq. (fgamma)
    f = -((2 - g * (1 - np.exp(-1j * xi))) / 2) * (1 + np.exp(1j * (xi + np.pi))) ** g
    return 2 * f.real


@pytest.mark.parametrize("al,be", [(1.5, 1.7), (1.2, 1.9)])
def test_eigenvalues_cluster_at_symbol_samples(al, be):
    # Prop. PaPb: with d+- = d, e+- = e constant, {A_x + (s/r) A_y} ~_lambda
    # F = d q_a(t1) + e (s/r) q_b(t2).  For this real even symbol the sorted
    # eigenvalues approach the sorted samples F(j pi/(n1+1), k pi/(n2+1)); the
    # largest gap falls as the grid is refined.  The eigenvalues of a Hermitian
    # Toeplitz matrix lie strictly inside (min F, max F) = (0, d ||q_a|| + e (s/r) ||q_b||),
    # ||q_g||_inf = (g - 1) 2^(g+1).
    d, e, sig = 1.3, 0.6, 0.9
    fmax = d * (al - 1) * 2 ** (al + 1) + sig * e * (be - 1) * 2 ** (be + 1)
    gaps = []
    for n in [15, 31]:
        n1, n2 = n, n + 2
        ones = np.ones((n2, n1))
        M = assemble_M(toeplitz_A(wsgd_weights(al, n1), n1), toeplitz_A(wsgd_weights(be, n2), n2),
                       0.0, sig, d * ones, d * ones, e * ones, e * ones)
        lam = np.sort(np.linalg.eigvalsh(M))
        t1 = np.pi * np.arange(1, n1 + 1) / (n1 + 1)
        t2 = np.pi * np.arange(1, n2 + 1) / (n2 + 1)
        F = np.sort((d * _q_closed_form(al, t1)[None, :]
                     + sig * e * _q_closed_form(be, t2)[:, None]).ravel())
        assert 0 < lam[0] and lam[-1] < fmax
        gaps.append(np.max(np.abs(lam - F)) / fmax)
    assert gaps[1] < 0.011 and gaps[1] < 0.6 * gaps[0], gaps
    # the one-level factor alone on larger sizes: the same O(1/n) clustering
    gaps1 = []
    for n in [63, 127, 255]:
        A = toeplitz_A(wsgd_weights(al, n), n)
        lam = np.sort(np.linalg.eigvalsh(A + A.T))
        F = np.sort(_q_closed_form(al, np.pi * np.arange(1, n + 1) / (n + 1)))
        gaps1.append(np.max(np.abs(lam - F)))
    assert gaps1[2] < 0.6 * gaps1[1] < 0.36 * gaps1[0], gaps1

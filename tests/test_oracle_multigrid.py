"""Pins of the oracle's multigrid (Sec. 4): grid transfer, Galerkin projection of
Toeplitz factors, the TGM iteration matrix against the recursive V-cycle, the
two-grid contraction theorem, the smoothing-parameter bound of Lemma lemsmo,
and the flexible GMRES solve against a dense direct solve."""
import numpy as np
import pytest

from oracle import multigrid as mg
from oracle.wsgd import wsgd_weights
from oracle.operator import toeplitz_A, assemble_M, apply_M
from oracle.krylov import fgmres

rng = np.random.default_rng(11)


def test_prolongation_is_bilinear():
    # Remark after Lemma lemapp: P = T(p) U is (up to scale) linear interpolation
    for n in [7, 15, 31]:
        P = mg.prolongation_1d(n)
        nc = (n - 1) // 2
        xc = (2 * np.arange(nc) + 2) / (n + 1)        # coarse node j <-> fine node 2j+1 (0-based)
        xf = np.arange(1, n + 1) / (n + 1)
        np.testing.assert_allclose((P @ xc)[:-1], xf[:-1], atol=1e-15)
        np.testing.assert_array_equal(P.sum(axis=0), 2.0)   # stencil 1/2, 1, 1/2
    P = mg.prolongation_1d(8)                              # even n: K^k_n picks fine 1, 3, 5, 7
    np.testing.assert_array_equal(np.argmax(P, axis=0), [0, 2, 4, 6])


@pytest.mark.parametrize("n", [7, 15, 31, 63])
def test_galerkin_of_toeplitz_is_q_coarsened_toeplitz(n):
    # P^T T(t) P = T(t^c), t^c_k = sum_m q_m t_{2k+m}, q = (1/4, 1, 3/2, 1, 1/4), for odd n
    P = mg.prolongation_1d(n)
    nc = (n - 1) // 2
    g = 1.37
    w = wsgd_weights(g, n)
    A = toeplitz_A(w, n)
    t = lambda d: A[d, 0] if d >= 0 else A[0, -d]      # Toeplitz generator t_d = A[i, i-d]
    q = {-2: 0.25, -1: 1.0, 0: 1.5, 1: 1.0, 2: 0.25}
    tc = lambda d: sum(qm * (t(2 * d + m) if abs(2 * d + m) < n else 0.0) for m, qm in q.items())
    Ac = P.T @ A @ P
    ref = np.array([[tc(i - j) for j in range(nc)] for i in range(nc)])
    np.testing.assert_allclose(Ac, ref, atol=1e-14)
    B = P.T @ P
    np.testing.assert_allclose(B, 1.5 * np.eye(nc) + 0.25 * (np.eye(nc, k=1) + np.eye(nc, k=-1)),
                               atol=1e-15)


def test_structured_galerkin_equals_exact_galerkin_for_constant_coefficients():
    n = 31
    wx, wy = wsgd_weights(1.6, n), wsgd_weights(1.75, n)
    ones = np.ones((n, n))
    cf = (1.2 * ones, 0.8 * ones, 0.5 * ones, 1.9 * ones)
    h = mg.structured_galerkin(wx, wy, n, n, 0.3, 1.1, cf)
    K0 = assemble_M(toeplitz_A(wx, n), toeplitz_A(wy, n), 0.3, 1.1, *cf)
    he = mg.exact_galerkin(K0, n, n)
    assert len(h.levels) == len(he.levels) == 3
    for l in range(3):
        np.testing.assert_allclose(h.levels[l].dense(), he.levels[l].dense(), atol=1e-11)
        np.testing.assert_allclose(h.levels[l].diag(), he.levels[l].diag(), atol=1e-11)


def test_structured_galerkin_injects_variable_coefficients():
    n = 15
    wx, wy = wsgd_weights(1.6, n), wsgd_weights(1.75, n)
    cf = tuple(rng.uniform(0.5, 2, (n, n)) for _ in range(4))
    h = mg.structured_galerkin(wx, wy, n, n, 0.3, 1.1, cf)
    np.testing.assert_array_equal(h.levels[1].dp, cf[0][1::2, 1::2])
    P = np.kron(mg.prolongation_1d(n), mg.prolongation_1d(n))
    exact = P.T @ h.levels[0].dense() @ P
    sg = h.levels[1].dense()
    # not exact for variable coefficients, but close (smooth coefficients would be closer)
    assert np.linalg.norm(sg - exact) / np.linalg.norm(exact) < 0.5


def test_vcycle_two_level_equals_tgm_matrix():
    # Sec. 4: with exact coarse solve the cycle is TGM(S, P) with one pre- and one
    # post-smoothing step: x = (I - TGM) K^{-1} b
    n = 15
    wx, wy = wsgd_weights(1.7, n), wsgd_weights(1.5, n)
    cf = tuple(rng.uniform(0.5, 2, (n, n)) for _ in range(4))
    K0 = assemble_M(toeplitz_A(wx, n), toeplitz_A(wy, n), 0.2, 0.9, *cf)
    h = mg.exact_galerkin(K0, n, n)
    assert len(h.levels) == 2
    P = np.kron(mg.prolongation_1d(n), mg.prolongation_1d(n))
    T = mg.tgm_matrix(K0, P, 0.7, nu_pre=1, nu_post=1)
    b = rng.standard_normal((n, n))
    x = mg.vcycle(h, b, omega=0.7)
    np.testing.assert_allclose(x.ravel(), (np.eye(n * n) - T) @ np.linalg.solve(K0, b.ravel()),
                               rtol=1e-10, atol=1e-12)


def test_tgm_contraction_below_one_and_flat():
    # Theorem (theorem21bis): ||TGM||_A <= c < 1 independently of N, alpha, beta,
    # for equal constant coefficients, 0 < omega < 2 a_0/||F||_inf, bilinear P
    norms = []
    for n in [7, 15, 31]:
        for al, be in [(1.3, 1.7), (1.8, 1.6)]:
            wx, wy = wsgd_weights(al, n), wsgd_weights(be, n)
            ones = np.ones((n, n))
            K = assemble_M(toeplitz_A(wx, n), toeplitz_A(wy, n), 0.0, 1.0, ones, ones, ones, ones)
            P = np.kron(mg.prolongation_1d(n), mg.prolongation_1d(n))
            T = mg.tgm_matrix(K, P, 0.7, nu_pre=0, nu_post=1)
            ev, Q = np.linalg.eigh(K)
            Kh = Q @ np.diag(np.sqrt(ev)) @ Q.T
            Khi = Q @ np.diag(1 / np.sqrt(ev)) @ Q.T
            norms.append(np.linalg.norm(Kh @ T @ Khi, 2))
    assert max(norms) < 0.95
    assert max(norms) - min(norms) < 0.15


@pytest.mark.parametrize("g", [1.05, 1.3, 1.562, 1.8, 1.99])
def test_omega_admissible(g):
    # Lemma lemsmo: 0 < omega < 2 a_0/||F||_inf with a_0 = -2(d w1^a + (s/r) e w1^b) the
    # zero-order Fourier coefficient of F = d q_a + (s/r) e q_b and
    # ||q_g||_inf = (g - 1) 2^(g+1) (Prop. PaPb); both terms give the ratio (g+2)/2^g
    w1 = wsgd_weights(g, 2)[1]
    ratio = 2 * (-2 * w1) / ((g - 1) * 2 ** (g + 1))
    np.testing.assert_allclose(ratio, (g + 2) / 2 ** g, rtol=1e-13)
    assert 0.7 < ratio and 1.0 <= ratio  # damped (0.7) and classical (1.0) Jacobi admissible


@pytest.mark.parametrize("kind", ["sg", "redisc", "p2"])
def test_fgmres_mg_matches_direct_solve(kind):
    from oracle.timeloop import make_preconditioner
    n = 31
    al, be = 1.5, 1.7
    wx, wy = wsgd_weights(al, n, 1, -1), wsgd_weights(be, n, 1, -1)
    X, Y = np.meshgrid(np.arange(1, n + 1) / (n + 1), np.arange(1, n + 1) / (n + 1))
    cf = (1 + X ** al * Y, 1 + (1 - X) ** al * Y, 1 + Y ** be * X, 1 + (1 - Y) ** be * X)
    sc = {"c": 0.35, "sigma": 1.8}
    prec, _ = make_preconditioner(kind, al, be, wx, wy, n, n, sc, cf)
    A = lambda Z: apply_M(Z, wx, wy, 0.35, 1.8, *cf)
    b = rng.standard_normal((n, n))
    x, its, rel, ok = fgmres(A, b, prec, 30, 1e-10)
    K = assemble_M(toeplitz_A(wx, n), toeplitz_A(wy, n), 0.35, 1.8, *cf)
    xd = np.linalg.solve(K, b.ravel())
    assert ok and rel <= 1e-10
    assert np.linalg.norm(b.ravel() - K @ x.ravel()) <= 1.0001e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x.ravel() - xd) <= np.linalg.cond(K) * 1e-10 * np.linalg.norm(xd)
    assert its < 30


def test_fgmres_identity_and_exact_preconditioner():
    n = 12
    wx, wy = wsgd_weights(1.5, n), wsgd_weights(1.6, n)
    cf = tuple(rng.uniform(0.5, 2, (n, n)) for _ in range(4))
    K = assemble_M(toeplitz_A(wx, n), toeplitz_A(wy, n), 0.1, 1.0, *cf)
    A = lambda Z: (K @ Z.ravel()).reshape(n, n)
    b = rng.standard_normal((n, n))
    x, its, rel, ok = fgmres(A, b, lambda R: np.linalg.solve(K, R.ravel()).reshape(n, n), 5, 1e-12)
    assert ok and its == 1
    x, its, rel, ok = fgmres(A, b, None, n * n, 1e-12)  # full GMRES: at most N steps
    assert ok and its <= n * n


def test_rediscretised_level_is_scheme_on_coarse_grid():
    # Sec. 4.2: the coarse matrix re-discretises the equation on the grid of width
    # 2h; in the scaling of Eq. (M) (times 1/r of the fine grid) level 1 must equal
    # (r_1/r_0) M(2h) with M(2h) = (1/r_1) I + A_x + (s_1/r_1) A_y built by Eq. (M)
    from oracle.operator import cn_scalars
    n, al, be, dt = 15, 1.45, 1.75, 0.01
    h = 1.0 / (n + 1)
    wx, wy = wsgd_weights(al, n), wsgd_weights(be, n)
    cf = tuple(rng.uniform(0.5, 2, (n, n)) for _ in range(4))
    s0 = cn_scalars(al, be, h, h, dt)
    hier = mg.rediscretised(al, be, wx, wy, n, n, s0["c"], s0["sigma"], cf)
    nc = 7
    s1 = cn_scalars(al, be, 2 * h, 2 * h, dt)
    cfc = tuple(f[1::2, 1::2] for f in cf)
    M1 = assemble_M(toeplitz_A(wx, nc), toeplitz_A(wy, nc), s1["c"], s1["sigma"], *cfc)
    np.testing.assert_allclose(hier.levels[1].dense(), (s1["r"] / s0["r"]) * M1, rtol=1e-13, atol=1e-14)
    assert hier.rscale == 0.25


# ----------------------------------------------------------------------------
# P_2 (Sec. 4.3): the band preconditioner and its Galerkin hierarchy

def test_p2_constant_coefficients_spectrum():
    # unit coefficients: P_2 = c I + 2 (I (x) L) + 2 sigma (L (x) I) with L the
    # Dirichlet Laplacian tridiag(-1, 2, -1), eigenvalues 4 sin^2(k pi / (2 (n + 1)))
    n1, n2, c, sigma = 9, 6, 0.37, 1.9
    ones = np.ones((n2, n1))
    K = mg.band_p2_matrix(n1, n2, c, sigma, (ones, ones, ones, ones)).toarray()
    lam = lambda n: 4 * np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2
    ev = (c + 2 * lam(n1)[None, :] + 2 * sigma * lam(n2)[:, None]).ravel()
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(K)), np.sort(ev), rtol=1e-12)
    # five nonzero diagonals (Sec. 4.3), at offsets 0, +-1 and +-n1
    offs = {j - i for i, j in zip(*np.nonzero(K))}
    assert offs == {0, 1, -1, n1, -n1}


def test_p2_galerkin_level_constant_coefficients_closed_form():
    # for linear interpolation P: P^T P = B = tridiag(1/4, 3/2, 1/4) and
    # P^T L P = L / 2 (the coarse Laplacian), so with unit coefficients level 1
    # is c (B (x) B) + (B (x) L) + sigma (L (x) B): a nine-point stencil
    n, c, sigma = 15, 0.41, 1.3
    ones = np.ones((n, n))
    h = mg.band_p2(n, n, c, sigma, (ones, ones, ones, ones))
    nc = 7
    B = 1.5 * np.eye(nc) + 0.25 * (np.eye(nc, k=1) + np.eye(nc, k=-1))
    L = 2 * np.eye(nc) - np.eye(nc, k=1) - np.eye(nc, k=-1)
    K1 = c * np.kron(B, B) + np.kron(B, L) + sigma * np.kron(L, B)
    np.testing.assert_allclose(h.levels[1].dense(), K1, rtol=1e-13, atol=1e-14)
    assert len(h.levels) == 2 and h.rscale == 1.0


def test_p2_galerkin_level_is_nine_point_with_variable_coefficients():
    n = 31
    cf = tuple(rng.uniform(0.5, 2, (n, n)) for _ in range(4))
    h = mg.band_p2(n, n, 0.3, 1.7, cf)
    for lev in h.levels[1:]:
        K = lev.dense()
        r, q = np.nonzero(K)
        dj = q // lev.n1 - r // lev.n1
        di = q % lev.n1 - r % lev.n1
        assert np.abs(dj).max() == 1 and np.abs(di).max() == 1
        assert np.all(np.diag(K) > 0)


@pytest.mark.parametrize("idx", [0, 1])
def test_p2_exact_inverse_counts_table1(idx):
    # Table 1's column for P_2 solved directly (Sec. 5.1): left GMRES(20), tol 1e-7
    import json
    import os
    import scipy.sparse.linalg as spla
    from paper_1706_06844_gb300 import inputs
    from oracle.operator import cn_scalars, rhs
    from oracle.krylov import gmres_left
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    t1 = gold["table1_example1"]
    n = t1["n"][idx]
    pb = inputs.example1()
    X, Y, hx, hy = pb.grid(n, n)
    dt = 1.0 / n
    wx, wy = wsgd_weights(pb.alpha, n), wsgd_weights(pb.beta, n)
    sc = cn_scalars(pb.alpha, pb.beta, hx, hy, dt)
    c, s = sc["c"], sc["sigma"]
    U = pb.exact(X, Y, 0.0)
    its = []
    for m in range(1, n + 1):
        co, cn = pb.coefficients(X, Y, (m - 1) * dt), pb.coefficients(X, Y, m * dt)
        B = rhs(U, wx, wy, c, s, *co, pb.source(X, Y, (m - 0.5) * dt), hx, pb.alpha)
        lu = spla.splu(mg.band_p2_matrix(n, n, c, s, cn).tocsc())
        prec = lambda R: lu.solve(np.asarray(R).ravel()).reshape(n, n)
        U, k, rel, ok = gmres_left(lambda Z: apply_M(Z, wx, wy, c, s, *cn), B, prec, 20, 1e-7)
        its.append(k)
    assert abs(np.mean(its) - t1["p2_exact"][idx]) <= 1.0, its


def test_p2_two_cycles_beat_one():
    # Sec. 5.1: two V-cycles per application of P_2 cut the GMRES count
    from oracle.timeloop import make_preconditioner
    n = 63
    al, be = 1.8, 1.6
    wx, wy = wsgd_weights(al, n), wsgd_weights(be, n)
    X, Y = np.meshgrid(np.arange(1, n + 1) / (n + 1), np.arange(1, n + 1) / (n + 1))
    cf = (1 + X, 2 - X, 1 + Y, 2 - Y)
    sc = {"c": 0.2, "sigma": 1.1}
    A = lambda Z: apply_M(Z, wx, wy, 0.2, 1.1, *cf)
    b = rng.standard_normal((n, n))
    counts = []
    for cycles in (1, 2):
        prec, _ = make_preconditioner("p2", al, be, wx, wy, n, n, sc, cf, omega=1.0, cycles=cycles)
        x, its, rel, ok = fgmres(A, b, prec, 60, 1e-8)
        assert ok
        counts.append(its)
    assert counts[1] < counts[0], counts


# ----------------------------------------------------------------------------
# multigrid as a stand-alone solver; warm starts

def test_mg_solve_error_follows_the_tgm_iteration_matrix():
    # two levels with an exact coarse solve: every cycle multiplies the error by
    # TGM(S, P) (Sec. 4), so after k cycles e_k = T^k e_0 with T built from the
    # matrices (independent of the recursive cycle code)
    from oracle.krylov import mg_solve
    n = 15
    wx, wy = wsgd_weights(1.6, n), wsgd_weights(1.8, n)
    cf = tuple(rng.uniform(0.5, 2, (n, n)) for _ in range(4))
    K0 = assemble_M(toeplitz_A(wx, n), toeplitz_A(wy, n), 0.3, 1.1, *cf)
    h = mg.exact_galerkin(K0, n, n)
    P = np.kron(mg.prolongation_1d(n), mg.prolongation_1d(n))
    T = mg.tgm_matrix(K0, P, 0.7, nu_pre=1, nu_post=1)
    b = rng.standard_normal((n, n))
    xs = np.linalg.solve(K0, b.ravel())
    apply = lambda X: (K0 @ X.ravel()).reshape(n, n)
    for k in (1, 2, 5):
        x, cyc, rel, ok = mg_solve(apply, b, lambda R: mg.vcycle(h, R), rtol=0.0, maxit=k)
        assert cyc == k
        np.testing.assert_allclose(x.ravel() - xs, np.linalg.matrix_power(T, k) @ (-xs),
                                   rtol=1e-9, atol=1e-12)


def test_mg_solve_converges_to_direct_solve():
    from oracle.krylov import mg_solve
    n = 31
    al, be = 1.5, 1.7
    wx, wy = wsgd_weights(al, n, 1, -1), wsgd_weights(be, n, 1, -1)
    X, Y = np.meshgrid(np.arange(1, n + 1) / (n + 1), np.arange(1, n + 1) / (n + 1))
    cf = (1 + X ** al * Y, 1 + (1 - X) ** al * Y, 1 + Y ** be * X, 1 + (1 - Y) ** be * X)
    hier = mg.structured_galerkin(wx, wy, n, n, 0.35, 1.8, cf)
    A = lambda Z: apply_M(Z, wx, wy, 0.35, 1.8, *cf)
    b = rng.standard_normal((n, n))
    x, cyc, rel, ok = mg_solve(A, b, lambda R: mg.vcycle(hier, R), 1e-10, 500)
    K = assemble_M(toeplitz_A(wx, n), toeplitz_A(wy, n), 0.35, 1.8, *cf)
    assert ok and rel <= 1e-10
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(K, b.ravel()), rtol=0, atol=1e-8 * np.abs(x).max())
    # a warm start at the solution needs no cycle; one near it needs fewer
    x2, cyc2, _, ok2 = mg_solve(A, b, lambda R: mg.vcycle(hier, R), 1e-10, 500, x0=x)
    assert ok2 and cyc2 == 0


def test_fgmres_warm_start():
    from oracle.timeloop import make_preconditioner
    n = 31
    wx, wy = wsgd_weights(1.5, n), wsgd_weights(1.7, n)
    cf = tuple(rng.uniform(0.5, 2, (n, n)) for _ in range(4))
    A = lambda Z: apply_M(Z, wx, wy, 0.35, 1.8, *cf)
    prec, _ = make_preconditioner("sg", 1.5, 1.7, wx, wy, n, n, {"c": 0.35, "sigma": 1.8}, cf)
    b = rng.standard_normal((n, n))
    x, its, rel, ok = fgmres(A, b, prec, 30, 1e-10)
    x0 = x + 1e-6 * rng.standard_normal((n, n))
    xw, itsw, relw, okw = fgmres(A, b, prec, 30, 1e-10, x0=x0)
    assert ok and okw and itsw < its
    assert np.linalg.norm(A(xw) - b) <= 1.0001e-10 * np.linalg.norm(b)


def _fgmres_counts(kind, al, be, sizes):
    from oracle.timeloop import make_preconditioner
    from oracle.operator import cn_scalars
    r = np.random.default_rng(3)
    counts = []
    for n in sizes:
        wx, wy = wsgd_weights(al, n, 1, -1), wsgd_weights(be, n, 1, -1)
        h = 1.0 / (n + 1)
        sc = cn_scalars(al, be, h, h, h)
        X, Y = np.meshgrid(np.arange(1, n + 1) * h, np.arange(1, n + 1) * h)
        cf = (1 + X ** al * Y, 1 + (1 - X) ** al * Y, 1 + Y ** be * X, 1 + (1 - Y) ** be * X)
        prec, _ = make_preconditioner(kind, al, be, wx, wy, n, n, sc, cf)
        A = lambda Z: apply_M(Z, wx, wy, sc["c"], sc["sigma"], *cf)
        x, its, rel, ok = fgmres(A, r.standard_normal((n, n)), prec, 60, 1e-8)
        assert ok
        counts.append(its)
    return counts


def _cn_counts(kind, sizes):
    # FGMRES(30) counts of one CN step of the perturbed power-law workload
    # (alpha = 1.5, beta = 1.7, dt = h), rtol 1e-8
    from paper_1706_06844_gb300 import inputs
    from oracle.timeloop import make_preconditioner
    from oracle.operator import cn_scalars, apply_M_fft, rhs_fft
    pb = inputs.perturbed_power_law()
    counts = []
    for n in sizes:
        X, Y, hx, hy = pb.grid(n, n)
        wx, wy = wsgd_weights(pb.alpha, n + 1, 1, pb.qx), wsgd_weights(pb.beta, n + 1, 1, pb.qy)
        sc = cn_scalars(pb.alpha, pb.beta, hx, hy, hx)
        c, s = sc["c"], sc["sigma"]
        c1, c0 = pb.coefficients(X, Y, hx), pb.coefficients(X, Y, 0.0)
        B = rhs_fft(pb.exact(X, Y, 0.0), wx, wy, c, s, *c0, pb.source(X, Y, 0.5 * hx), hx,
                    pb.alpha)
        prec, _ = make_preconditioner(kind, pb.alpha, pb.beta, wx, wy, n, n, sc, c1)
        x, its, rel, ok = fgmres(lambda Z: apply_M_fft(Z, wx, wy, c, s, *c1), B, prec, 30, 1e-8)
        assert ok
        counts.append(its)
    return counts


def test_cn_step_counts_flat_in_n():
    # Sec. 4-5: for a CN step of a smooth problem the multigrid preconditioners'
    # counts do not grow with n (structured Galerkin and rediscretised alike);
    # P_2 needs more iterations at every size when alpha, beta are away from 2
    sizes = [31, 63, 127, 255]
    sg, rd, p2 = (_cn_counts(k, sizes) for k in ("sg", "redisc", "p2"))
    for c in (sg, rd):
        assert 12 <= min(c) and max(c) <= 16 and max(c) - min(c) <= 2, (sg, rd)
    assert all(a > b for a, b in zip(p2, sg)), (p2, sg)


def test_iteration_counts_flat_in_n_for_multigrid_not_for_p2():
    # Sec. 4 / Sec. 5: the V-cycle preconditioner's iteration count is (nearly)
    # independent of n and of alpha, beta; the band preconditioner P_2 is a
    # second-order operator, so its count grows with n when alpha, beta are far
    # from 2 and stays low only near 2 (dt = h, variable coefficients)
    sizes = [15, 31, 63, 127, 255]
    far, near = (1.2, 1.3), (1.9, 1.8)
    sg_far, sg_near = _fgmres_counts("sg", *far, sizes), _fgmres_counts("sg", *near, sizes)
    rd_far, rd_near = _fgmres_counts("redisc", *far, sizes), _fgmres_counts("redisc", *near, sizes)
    p2_far, p2_near = _fgmres_counts("p2", *far, sizes), _fgmres_counts("p2", *near, sizes)
    for c in (sg_far, sg_near, rd_far, rd_near):
        assert max(c) <= 16 and c[-1] - c[0] <= 5, c
    assert abs(sg_far[-1] - sg_near[-1]) <= 2, (sg_far, sg_near)
    assert p2_far[-1] - p2_far[0] >= 2 * (sg_far[-1] - sg_far[0]), (p2_far, sg_far)
    assert p2_far[-1] > p2_near[-1] + 5, (p2_far, p2_near)


def test_grid_transfer_helpers():
    # Sec. 4.1 / 4.2: for odd n = 2k + 1 the coarse nodes are fine nodes (the
    # coarse grid of width 2h sits on every other fine node); the level sizes
    # halve down to the fixed coarsest grid (n = 2047: 9 levels down to 7)
    for n in [7, 15, 63, 2047]:
        k = mg.coarse_size(n)
        assert n == 2 * k + 1
        xf = (mg.coarse_to_fine(n) + 1) / (n + 1)
        xc = np.arange(1, k + 1) / (k + 1)
        np.testing.assert_allclose(xf, xc, rtol=0, atol=1e-15)
    assert mg.level_sizes(2047) == [2047, 1023, 511, 255, 127, 63, 31, 15, 7]
    assert mg.level_sizes(16) == [16, 8]
    # even n: k = n/2 coarse nodes on the odd fine nodes (1-based 1, 3, ...)
    assert list(mg.coarse_to_fine(8)) == [0, 2, 4, 6]


def test_jacobi_sweep_and_fixed_point():
    # Eq. (Sn): from x = 0 one sweep gives omega b / diag(K); the solution of
    # K x = b is a fixed point of the damped iteration
    n = 15
    wx, wy = wsgd_weights(1.6, n), wsgd_weights(1.4, n)
    X, Y = np.meshgrid(np.arange(1, n + 1) / (n + 1), np.arange(1, n + 1) / (n + 1))
    cf = (1 + X * Y, 2 - X, 1 + Y, 1.5 + 0 * X)
    hier = mg.structured_galerkin(wx, wy, n, n, 0.4, 1.3, cf)
    lev = hier.levels[0]
    K = assemble_M(toeplitz_A(wx, n), toeplitz_A(wy, n), 0.4, 1.3, *cf)
    np.testing.assert_allclose(lev.diag().ravel(), np.diag(K), rtol=1e-14)
    b = rng.standard_normal((n, n))
    x1 = mg.jacobi(lev, np.zeros((n, n)), b, 0.7, 1)
    np.testing.assert_allclose(x1.ravel(), 0.7 * b.ravel() / np.diag(K), rtol=1e-14)
    xs = np.linalg.solve(K, b.ravel()).reshape(n, n)
    np.testing.assert_allclose(mg.jacobi(lev, xs, b, 0.7, 3), xs, rtol=0, atol=1e-12)


def test_laplacian_weights_and_shift_choice():
    # gamma = 2 member of Eq. (w): the second difference (1, -2, 1); the shift
    # used by the drawn workloads switches to (1,-1) below gamma_0 (Sec. 2)
    from oracle.wsgd import choose_shift, GAMMA0
    np.testing.assert_array_equal(mg.laplacian_weights(), [1.0, -2.0, 1.0])
    A2 = toeplitz_A(np.r_[mg.laplacian_weights(), np.zeros(4)], 5)
    np.testing.assert_array_equal(A2, 2 * np.eye(5) - np.eye(5, k=1) - np.eye(5, k=-1))
    assert choose_shift(GAMMA0, 1.9) == 0 and choose_shift(1.9, GAMMA0) == 0
    assert choose_shift(GAMMA0 - 1e-9, 1.9) == -1 and choose_shift(1.9, 1.2) == -1


def test_apply_kron_with_mass_factors_equals_dense_kronecker():
    # the coarse-level form c (By (x) Bx) + D+ (By (x) Ax) + ... evaluated by
    # matmuls equals the explicit Kronecker products
    from oracle.operator import apply_kron
    n1, n2 = 6, 5
    Ax, Ay = rng.standard_normal((n1, n1)), rng.standard_normal((n2, n2))
    Bx, By = rng.standard_normal((n1, n1)), rng.standard_normal((n2, n2))
    cf = [rng.uniform(0.5, 2, (n2, n1)) for _ in range(4)]
    X = rng.standard_normal((n2, n1))
    K = assemble_M(Ax, Ay, 0.3, 1.7, *cf, Bx=Bx, By=By)
    np.testing.assert_allclose(apply_kron(X, Ax, Ay, 0.3, 1.7, *cf, Bx, By).ravel(),
                               K @ X.ravel(), rtol=1e-12, atol=1e-12)

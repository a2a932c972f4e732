"""Multigrid of Sec. 4: damped Jacobi (Eq. Sn, Lemma lemsmo), bilinear grid
transfer P = T(p) U (Sec. 4.1, Eq. q), the two-grid method TGM(S, P) and its
recursive V-cycle (Sec. 4 and 4.2), with three ways to build coarse operators:

* ``structured_galerkin``: every Kronecker term of Eq. (AxAy) is projected
  exactly (P^T T P for each 1-D factor), the coefficient diagonals are injected.
  For constant coefficients this equals the exact Galerkin P^T M P.
* ``rediscretised``: the paper's geometric P_MGM (Sec. 4.2): the same weights
  on the coarse grid with h_l = 2^l h, full-weighting restriction (1/4) P^T.
* ``exact_galerkin``: A_k = P^T A_N P as dense matrices (tiny grids; the
  paper's tilde-P_MGM), and ``band_p2``: the preconditioner P_2 of Sec. 4.3
  (alpha = beta = 2 Laplacian factors) with exact sparse Galerkin coarse
  operators.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np
import scipy.sparse as sp

from .operator import toeplitz_A, apply_kron, assemble_M
from .wsgd import wsgd_weights


# ----------------------------------------------------------------------------
# grid transfer (Sec. 4.1)

def coarse_size(n):
    """k = (n - (n mod 2))/2 (Sec. 4.1)."""
    return (n - n % 2) // 2


def coarse_to_fine(n):
    """0-based fine index of each coarse node: [K^k_n]_{ij} = 1 iff
    i = 2j - ((n+1) mod 2) (1-based, Sec. 4.1)."""
    k = coarse_size(n)
    j = np.arange(1, k + 1)
    return 2 * j - ((n + 1) % 2) - 1


def prolongation_1d(n):
    """P_n = T_n(1 + cos theta) K^k_n: the 1-D factor of P_N = T_N(p) U^k_N with
    p(t1, t2) = (1 + cos t1)(1 + cos t2) (Eq. q), i.e. bilinear interpolation.
    T_n(1 + cos) is tridiag(1/2, 1, 1/2) (Fourier coefficients of 1 + cos)."""
    k = coarse_size(n)
    K = np.zeros((n, k))
    K[coarse_to_fine(n), np.arange(k)] = 1.0
    T = np.eye(n) + 0.5 * (np.eye(n, k=1) + np.eye(n, k=-1))
    return T @ K


def inject(F, n1, n2):
    """Coefficient diagonal sampled at the coarse nodes (injection)."""
    return np.asarray(F)[np.ix_(coarse_to_fine(n2), coarse_to_fine(n1))]


# ----------------------------------------------------------------------------
# levels

class KronLevel:
    """K = c (By (x) Bx) + D+ (By (x) Ax) + D- (By (x) Ax^T)
         + sigma [E+ (Ay (x) Bx) + E- (Ay^T (x) Bx)]   on an n2 x n1 grid."""

    def __init__(self, Ax, Ay, Bx, By, c, sigma, dp, dm, ep, em):
        self.Ax, self.Ay, self.Bx, self.By = Ax, Ay, Bx, By
        self.c, self.sigma = c, sigma
        self.dp, self.dm, self.ep, self.em = dp, dm, ep, em
        self.n1, self.n2 = Ax.shape[0], Ay.shape[0]

    def apply(self, X):
        return apply_kron(X, self.Ax, self.Ay, self.c, self.sigma, self.dp, self.dm,
                          self.ep, self.em, self.Bx, self.By)

    def diag(self):
        """True diagonal of K (used by the Jacobi smoother)."""
        bx, by = np.diag(self.Bx), np.diag(self.By)
        ax, ay = np.diag(self.Ax), np.diag(self.Ay)
        return (self.c * np.outer(by, bx) + (self.dp + self.dm) * np.outer(by, ax)
                + self.sigma * (self.ep + self.em) * np.outer(ay, bx))

    def dense(self):
        return assemble_M(self.Ax, self.Ay, self.c, self.sigma, self.dp, self.dm,
                          self.ep, self.em, self.Bx, self.By)


class MatrixLevel:
    """A level given by an explicit (dense or sparse) N x N matrix."""

    def __init__(self, K, n1, n2):
        self.K, self.n1, self.n2 = K, n1, n2

    def apply(self, X):
        return (self.K @ np.asarray(X).ravel()).reshape(self.n2, self.n1)

    def diag(self):
        d = self.K.diagonal() if sp.issparse(self.K) else np.diag(self.K)
        return np.asarray(d).reshape(self.n2, self.n1)

    def dense(self):
        return self.K.toarray() if sp.issparse(self.K) else self.K


class Hierarchy:
    """Levels 0..L, 1-D prolongations between them and the restriction scale
    (R = rscale * P^T)."""

    def __init__(self, levels, Px, Py, rscale):
        self.levels, self.Px, self.Py, self.rscale = levels, Px, Py, rscale

    def restrict(self, l, R):
        """R r = rscale * (Py (x) Px)^T vec(r) = rscale * Py^T r Px."""
        return self.rscale * (self.Py[l].T @ R @ self.Px[l])

    def prolong(self, l, Xc):
        """P x_c = (Py (x) Px) vec(x_c) = Py x_c Px^T."""
        return self.Py[l] @ Xc @ self.Px[l].T


def level_sizes(n, coarsest=8):
    """n_0 = n, n_{l+1} = coarse_size(n_l), stopping at the first n_l <= coarsest
    (the paper fixes the coarsest grid to 8 x 8, Sec. 4.2)."""
    sizes = [n]
    while sizes[-1] > coarsest:
        sizes.append(coarse_size(sizes[-1]))
    return sizes


def structured_galerkin(wx, wy, n1, n2, c, sigma, coef, coarsest=8):
    """Structured Galerkin hierarchy: 1-D factors projected exactly,
    A^{l+1} = P^T A^l P and B^{l+1} = P^T B^l P (B^0 = I), coefficients injected,
    R = P^T (TGM step 2)."""
    s1, s2 = level_sizes(n1, coarsest), level_sizes(n2, coarsest)
    nl = min(len(s1), len(s2))
    Ax, Ay = toeplitz_A(wx, n1), toeplitz_A(wy, n2)
    Bx, By = np.eye(n1), np.eye(n2)
    dp, dm, ep, em = coef
    levels, Px, Py = [], [], []
    for l in range(nl):
        levels.append(KronLevel(Ax, Ay, Bx, By, c, sigma, dp, dm, ep, em))
        if l == nl - 1:
            break
        m1, m2 = Ax.shape[0], Ay.shape[0]
        px, py = prolongation_1d(m1), prolongation_1d(m2)
        Px.append(px)
        Py.append(py)
        Ax, Bx = px.T @ Ax @ px, px.T @ Bx @ px
        Ay, By = py.T @ Ay @ py, py.T @ By @ py
        dp, dm, ep, em = (inject(f, m1, m2) for f in (dp, dm, ep, em))
    return Hierarchy(levels, Px, Py, 1.0)


def rediscretised(alpha, beta, wx, wy, n1, n2, c, sigma, coef, coarsest=8):
    """Geometric P_MGM (Sec. 4.2): level l re-uses the weights on the grid of
    width 2^l h.  Scaled like Eq. (M) (multiplied by 1/r of the finest grid),
    M_l = c I + 2^{-alpha l} A_{x,l} + sigma 2^{-beta l} A_{y,l}; coefficients
    injected; full weighting R = (1/4) P^T."""
    s1, s2 = level_sizes(n1, coarsest), level_sizes(n2, coarsest)
    nl = min(len(s1), len(s2))
    dp, dm, ep, em = coef
    levels, Px, Py = [], [], []
    m1, m2 = n1, n2
    for l in range(nl):
        Ax = 2.0 ** (-alpha * l) * toeplitz_A(wx, m1)
        Ay = 2.0 ** (-beta * l) * toeplitz_A(wy, m2)
        levels.append(KronLevel(Ax, Ay, np.eye(m1), np.eye(m2), c, sigma, dp, dm, ep, em))
        if l == nl - 1:
            break
        Px.append(prolongation_1d(m1))
        Py.append(prolongation_1d(m2))
        dp, dm, ep, em = (inject(f, m1, m2) for f in (dp, dm, ep, em))
        m1, m2 = coarse_size(m1), coarse_size(m2)
    return Hierarchy(levels, Px, Py, 0.25)


def exact_galerkin(K0, n1, n2, coarsest=8):
    """A_{l+1} = P^T A_l P with explicit matrices (TGM step 3 applied at every
    level); dense for small grids."""
    s1, s2 = level_sizes(n1, coarsest), level_sizes(n2, coarsest)
    nl = min(len(s1), len(s2))
    K = K0
    levels, Px, Py = [], [], []
    m1, m2 = n1, n2
    for l in range(nl):
        levels.append(MatrixLevel(K, m1, m2))
        if l == nl - 1:
            break
        px, py = prolongation_1d(m1), prolongation_1d(m2)
        Px.append(px)
        Py.append(py)
        if sp.issparse(K):
            Ps = sp.kron(sp.csr_matrix(py), sp.csr_matrix(px)).tocsr()
            K = (Ps.T @ K @ Ps).tocsr()
        else:
            P = np.kron(py, px)
            K = P.T @ K @ P
        m1, m2 = coarse_size(m1), coarse_size(m2)
    return Hierarchy(levels, Px, Py, 1.0)


def laplacian_weights():
    """gamma = 2 in Eq. (w): w = (1, -2, 1), so A^2 = -[w_{i-j+1}] = tridiag(-1, 2, -1)."""
    return wsgd_weights(2.0, 2)


def band_p2_matrix(n1, n2, c, sigma, coef):
    """P_2 of Sec. 4.3 read as Eq. (M) with A^alpha, A^beta replaced by the
    Laplacian A^2 = tridiag(-1, 2, -1) (the gamma = 2 member of Eq. AN),
    keeping c and sigma: a five-point variable stencil, returned sparse."""
    w2 = np.zeros(max(n1, n2) + 1)
    w2[:3] = laplacian_weights()
    L1 = sp.csr_matrix(toeplitz_A(w2, n1))
    L2 = sp.csr_matrix(toeplitz_A(w2, n2))
    dp, dm, ep, em = (sp.diags(np.asarray(f).ravel()) for f in coef)
    I1, I2 = sp.identity(n1), sp.identity(n2)
    K = (c * sp.identity(n1 * n2) + dp @ sp.kron(I2, L1) + dm @ sp.kron(I2, L1.T)
         + sigma * (ep @ sp.kron(L2, I1) + em @ sp.kron(L2.T, I1)))
    return K.tocsr()


def band_p2(n1, n2, c, sigma, coef, coarsest=8):
    """Galerkin hierarchy of P_2 (Sec. 4.3): exact sparse P^T K P at every level."""
    return exact_galerkin(band_p2_matrix(n1, n2, c, sigma, coef), n1, n2, coarsest)


# ----------------------------------------------------------------------------
# smoother, TGM and V-cycle

def jacobi(level, X, B, omega, sweeps):
    """x <- x + omega D^{-1} (b - K x), D = diag(K) (Eq. Sn with W = D/omega)."""
    d = level.diag()
    for _ in range(sweeps):
        X = X + omega * (B - level.apply(X)) / d
    return X


def vcycle(h, B, omega=0.7, nu_pre=1, nu_post=1, l=0, coarse_solve=None):
    """One V-cycle for K_l x = b from x = 0 (Sec. 4: TGM steps 1-6 with an
    optional pre-smoother, step 4 replaced by recursion, zero initial guess on
    coarse grids; the coarsest system is solved directly)."""
    lev = h.levels[l]
    if l == len(h.levels) - 1:
        if coarse_solve is not None:
            return coarse_solve(B)
        return np.linalg.solve(lev.dense(), np.asarray(B).ravel()).reshape(lev.n2, lev.n1)
    X = np.zeros_like(B)
    X = jacobi(lev, X, B, omega, nu_pre)
    R = B - lev.apply(X)
    Xc = vcycle(h, h.restrict(l, R), omega, nu_pre, nu_post, l + 1, coarse_solve)
    X = X + h.prolong(l, Xc)
    return jacobi(lev, X, B, omega, nu_post)


def tgm_matrix(K, P, omega, nu_pre=0, nu_post=1):
    """Iteration matrix of TGM(S, P) (Sec. 4):
    S^nu_post [I - P (P^T K P)^{-1} P^T K] S^nu_pre,  S = I - omega D^{-1} K."""
    N = K.shape[0]
    S = np.eye(N) - omega * (K / np.diag(K)[:, None])
    CGC = np.eye(N) - P @ np.linalg.solve(P.T @ K @ P, P.T @ K)
    return (np.linalg.matrix_power(S, nu_post) @ CGC @ np.linalg.matrix_power(S, nu_pre))

"""Toeplitz and Kronecker operators of the CN-WSGD scheme (Sec. 2).

Test infrastructure only (see ``oracle/__init__.py``).

Layout: a grid function is an array X[j, i] of shape (n2, n1) with the x index
i fastest, so ``X.ravel()`` is the lexicographic vector of Sec. 2 (x first).
For that ordering (I_{n2} (x) A) vec(X) = vec(X A^T) and
(A (x) I_{n1}) vec(X) = vec(A X).
"""
import numpy as np
from scipy.signal import fftconvolve


def grid(a, b, n):
    """Interior nodes x_i = a + i h, i = 1..n, h = (b - a)/(n + 1) (Sec. 2)."""
    h = (b - a) / (n + 1)
    return a + h * np.arange(1, n + 1, dtype=np.float64), h


def cn_scalars(alpha, beta, hx, hy, dt):
    """r = dt/(2 hx^alpha), s = dt/(2 hy^beta) (Eq. system); the scaled system
    Eq. (M) has c = 1/r on the identity and sigma = s/r on A_y."""
    r = dt / (2.0 * hx ** alpha)
    s = dt / (2.0 * hy ** beta)
    return {"r": r, "s": s, "c": 1.0 / r, "sigma": s / r}


def toeplitz_A(w, n):
    """A^gamma_n = -[w_{i-j+1}]_{i,j=1..n} (Eq. AN): lower Hessenberg, w_0 on the
    super-diagonal, w_n in the bottom-left corner; w_k = 0 for k < 0."""
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    k = i - j + 1
    A = np.zeros((n, n), dtype=np.float64)
    mask = (k >= 0) & (k <= n)
    A[mask] = -np.asarray(w, dtype=np.float64)[k[mask]]
    return A


def apply_kron(X, Ax, Ay, c, sigma, dp, dm, ep, em, Bx=None, By=None):
    """y = c (By (x) Bx) x + D+ (By (x) Ax) x + D- (By (x) Ax^T) x
           + sigma [E+ (Ay (x) Bx) x + E- (Ay^T (x) Bx) x]

    With Bx = By = I this is M x of Eq. (M) with A_x, A_y of Eq. (AxAy).
    The B factors carry the Galerkin mass matrices of coarse levels.  All 1-D
    factors are dense matrices; the products are plain matmuls."""
    X = np.asarray(X, dtype=np.float64)
    if Bx is None and By is None:
        return (c * X + dp * (X @ Ax.T) + dm * (X @ Ax)
                + sigma * (ep * (Ay @ X) + em * (Ay.T @ X)))
    XBx = X @ Bx.T
    ByX = By @ X
    return (c * (By @ XBx) + dp * (ByX @ Ax.T) + dm * (ByX @ Ax)
            + sigma * (ep * (Ay @ XBx) + em * (Ay.T @ XBx)))


def apply_M(X, wx, wy, c, sigma, dp, dm, ep, em):
    """M x (Eq. M) with the Toeplitz factors built densely from the weights."""
    n2, n1 = X.shape
    return apply_kron(X, toeplitz_A(wx, n1), toeplitz_A(wy, n2), c, sigma, dp, dm, ep, em)


def assemble_M(Ax, Ay, c, sigma, dp, dm, ep, em, Bx=None, By=None):
    """Dense N x N matrix of ``apply_kron`` by explicit Kronecker products
    (Eq. AxAy, Eq. M).  For tiny grids only."""
    n1, n2 = Ax.shape[0], Ay.shape[0]
    Bx = np.eye(n1) if Bx is None else Bx
    By = np.eye(n2) if By is None else By
    D = lambda f: np.diag(np.asarray(f, dtype=np.float64).ravel())
    return (c * np.kron(By, Bx)
            + D(dp) @ np.kron(By, Ax) + D(dm) @ np.kron(By, Ax.T)
            + sigma * (D(ep) @ np.kron(Ay, Bx) + D(em) @ np.kron(Ay.T, Bx)))


def rhs(U, wx, wy, c, sigma, dp_old, dm_old, ep_old, em_old, V, hx, alpha):
    """b^(m) = (c I - A_x^(m-1) - sigma A_y^(m-1)) u^(m-1) + 2 hx^alpha v^(m-1/2)
    (Eq. M, second line), coefficients taken at t^(m-1)."""
    n2, n1 = U.shape
    Ax, Ay = toeplitz_A(wx, n1), toeplitz_A(wy, n2)
    return (c * U - (dp_old * (U @ Ax.T) + dm_old * (U @ Ax))
            - sigma * (ep_old * (Ay @ U) + em_old * (Ay.T @ U)) + 2.0 * hx ** alpha * V)


# --- the same Toeplitz products through a library convolution (for large n) ---

def toeplitz_rows(X, w, transpose=False):
    """Rows of X times A^T (A applied to every row) or, with transpose=True,
    times A, where A = -[w_{i-j+1}] (Eq. AN).

    (A x)_i   = -sum_j w_{i-j+1} x_j  = -(w * x)[i+1]        (linear convolution)
    (A^T x)_i = -sum_j w_{j-i+1} x_j  = -(w * rev(x))[n-i]
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[-1]
    wv = np.asarray(w[: n + 1], dtype=np.float64)[None, :]
    if not transpose:
        full = fftconvolve(X, wv, axes=-1)
        return -full[:, 1:n + 1]
    full = fftconvolve(X[:, ::-1], wv, axes=-1)
    return -full[:, n:0:-1]


def apply_M_fft(X, wx, wy, c, sigma, dp, dm, ep, em):
    """M x of Eq. (M) using ``toeplitz_rows`` for the four Toeplitz products."""
    X = np.asarray(X, dtype=np.float64)
    XT = X.T
    return (c * X + dp * toeplitz_rows(X, wx) + dm * toeplitz_rows(X, wx, True)
            + sigma * (ep * toeplitz_rows(XT, wy).T + em * toeplitz_rows(XT, wy, True).T))


def rhs_fft(U, wx, wy, c, sigma, dp_old, dm_old, ep_old, em_old, V, hx, alpha):
    """``rhs`` with the FFT-convolution Toeplitz products."""
    return (2.0 * c * U - apply_M_fft(U, wx, wy, c, sigma, dp_old, dm_old, ep_old, em_old)
            + 2.0 * hx ** alpha * V)

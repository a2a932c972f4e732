"""Restarted GMRES, as used for every linear solve of Sec. 5 (restart length,
relative-residual tolerance, zero initial guess), in its flexible
right-preconditioned form; and multigrid used on its own as the solver
(Sec. 1 and Sec. 4.3 note that the method can run without a Krylov wrapper).

Arnoldi by modified Gram-Schmidt, least squares by Givens rotations, and the
true residual ||b - M x|| recomputed at every restart.  The iteration count is
the total number of inner (Arnoldi) steps.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np


def fgmres(apply_A, b, precond=None, restart=30, rtol=1e-8, maxit=10000, x0=None):
    """Solve A x = b.  ``apply_A`` and ``precond`` map arrays of b's shape to
    arrays of b's shape.  Returns (x, iterations, relative true residual,
    converged)."""
    shape = np.shape(b)
    b = np.asarray(b, dtype=np.float64).ravel()
    A = lambda v: np.asarray(apply_A(v.reshape(shape)), dtype=np.float64).ravel()
    Pinv = (lambda v: v) if precond is None else (
        lambda v: np.asarray(precond(v.reshape(shape)), dtype=np.float64).ravel())
    N = b.size
    bnorm = np.linalg.norm(b)
    x = np.zeros(N) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    if bnorm == 0.0:
        return x.reshape(shape), 0, 0.0, True
    r = b - A(x)
    beta = np.linalg.norm(r)
    its = 0
    while beta > rtol * bnorm and its < maxit:
        m = restart
        V = np.zeros((m + 1, N))
        Z = np.zeros((m, N))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = Pinv(V[j])
            w = A(Z[j])
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                     # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = np.hypot(H[j, j], H[j + 1, j])   # new rotation
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j], H[j + 1, j] = rho, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            if abs(g[j + 1]) <= rtol * bnorm or its >= maxit or H[j, j] == 0.0:
                break
        y = np.zeros(k)                            # back substitution
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        r = b - A(x)
        beta = np.linalg.norm(r)
    return x.reshape(shape), its, beta / bnorm, bool(beta <= rtol * bnorm)


def gmres_left(apply_A, b, precond, restart=20, rtol=1e-7, maxit=10000):
    """Restarted GMRES on the left-preconditioned system P^{-1} A x = P^{-1} b
    from x = 0, stopping on the preconditioned relative residual
    ||P^{-1}(b - A x)|| <= rtol ||P^{-1} b||: the convention of the solver used
    for the tables of Sec. 5.  Returns (x, iterations, relative preconditioned
    residual, converged)."""
    shape = np.shape(b)
    PA = lambda v: np.asarray(precond(np.asarray(apply_A(v.reshape(shape))).reshape(shape)),
                              dtype=np.float64).ravel()
    pb = np.asarray(precond(np.asarray(b, dtype=np.float64).reshape(shape)), dtype=np.float64)
    x, its, rel, ok = fgmres(lambda v: PA(np.asarray(v).ravel()).reshape(shape), pb, None,
                             restart, rtol, maxit)
    return x, its, rel, ok


def mg_solve(apply_A, b, vcycle, rtol=1e-8, maxit=1000, x0=None):
    """Multigrid as a stand-alone solver: the stationary iteration
    x_{k+1} = x_k + V(b - A x_k), V one V-cycle from a zero initial guess, until
    ||b - A x|| <= rtol ||b||.  Returns (x, cycles, relative residual, converged)."""
    b = np.asarray(b, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if bnorm == 0.0:
        return x, 0, 0.0, True
    k = 0
    while True:
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
        if rel <= rtol or k >= maxit:
            return x, k, rel, bool(rel <= rtol)
        x = x + vcycle(r)
        k += 1

"""The CN-WSGD time loop (Eq. CNWSGD): at each t^(m) assemble b^(m) and solve
M^(m) u^(m) = b^(m) (Eq. 2) from a zero initial guess (Sec. 5).

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

from .wsgd import wsgd_weights
from .operator import cn_scalars, apply_M, apply_M_fft, rhs, rhs_fft, toeplitz_A
from . import multigrid as mg
from .krylov import fgmres


def make_preconditioner(kind, alpha, beta, wx, wy, n1, n2, sc, coef, omega=0.7,
                        nu_pre=1, nu_post=1, coarsest=8, cycles=1):
    """kind in {"none", "sg" (structured Galerkin), "redisc" (P_MGM of Sec. 4.2),
    "galerkin" (exact dense Galerkin, tiny grids), "p2" (Sec. 4.3)}."""
    c, sigma = sc["c"], sc["sigma"]
    if kind == "none":
        return None, None
    if kind == "sg":
        h = mg.structured_galerkin(wx, wy, n1, n2, c, sigma, coef, coarsest)
    elif kind == "redisc":
        h = mg.rediscretised(alpha, beta, wx, wy, n1, n2, c, sigma, coef, coarsest)
    elif kind == "galerkin":
        from .operator import assemble_M
        K0 = assemble_M(toeplitz_A(wx, n1), toeplitz_A(wy, n2), c, sigma, *coef)
        h = mg.exact_galerkin(K0, n1, n2, coarsest)
    elif kind == "p2":
        h = mg.band_p2(n1, n2, c, sigma, coef, coarsest)
    else:
        raise ValueError(kind)

    def prec(B):
        X = mg.vcycle(h, B, omega, nu_pre, nu_post)
        for _ in range(cycles - 1):   # further V-cycles as a stationary iteration
            X = X + mg.vcycle(h, B - h.levels[0].apply(X), omega, nu_pre, nu_post)
        return X
    return prec, h


def run(problem, n, steps=None, precond="sg", restart=30, rtol=1e-8, maxit=10000,
        T=1.0, use_fft=None, record=False, **mgopts):
    """Run the time loop on an n x n grid with M = ``steps`` (default n) steps
    over [0, T].  Returns dict(error_inf, iterations per step, U, ...)."""
    n1 = n2 = n
    M = n if steps is None else steps
    dt = T / M
    X, Y, hx, hy = problem.grid(n1, n2)
    al, be = problem.alpha, problem.beta
    wx = wsgd_weights(al, n1, 1, problem.qx)
    wy = wsgd_weights(be, n2, 1, problem.qy)
    sc = cn_scalars(al, be, hx, hy, dt)
    c, sigma = sc["c"], sc["sigma"]
    fft = (n > 255) if use_fft is None else use_fft
    U = problem.exact(X, Y, 0.0)
    its, res, hist = [], [], []
    coef_new = problem.coefficients(X, Y, 0.0)
    prec = None
    for m in range(1, M + 1):
        t_old, t_new = (m - 1) * dt, m * dt
        coef_old = coef_new
        coef_new = problem.coefficients(X, Y, t_new)
        V = problem.source(X, Y, t_old + 0.5 * dt)
        if fft:
            B = rhs_fft(U, wx, wy, c, sigma, *coef_old, V, hx, al)
            A = lambda Z: apply_M_fft(Z, wx, wy, c, sigma, *coef_new)
        else:
            B = rhs(U, wx, wy, c, sigma, *coef_old, V, hx, al)
            Ax, Ay = toeplitz_A(wx, n1), toeplitz_A(wy, n2)
            A = (lambda Z, Ax=Ax, Ay=Ay, cf=coef_new:
                 c * Z + cf[0] * (Z @ Ax.T) + cf[1] * (Z @ Ax)
                 + sigma * (cf[2] * (Ay @ Z) + cf[3] * (Ay.T @ Z)))
        if prec is None or problem.time_dependent:
            prec, _ = make_preconditioner(precond, al, be, wx, wy, n1, n2, sc, coef_new, **mgopts)
        U, k, rel, ok = fgmres(A, B, prec, restart, rtol, maxit)
        its.append(k)
        res.append(rel)
        if record:
            hist.append(U.copy())
    err = np.max(np.abs(problem.exact(X, Y, M * dt) - U))
    return {"error_inf": err, "iterations": its, "mean_iterations": float(np.mean(its)),
            "residuals": res, "U": U, "history": hist, "c": c, "sigma": sigma}

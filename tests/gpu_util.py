"""Helpers shared by the GPU tests: problem set-up on the host (from the
shared input generators), device copies, and an oracle twin of each solver
configuration."""
import numpy as np

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde


def torch_cuda():
    import torch
    return torch


def dev(a):
    torch = torch_cuda()
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


class Case:
    """A problem on an n2 x n1 grid with its CN scalars, weights and the
    arrays of one time step, for both the CUDA path and the oracle."""

    def __init__(self, problem, n1, n2=None, dt=None, m=1, **kw):
        from oracle.wsgd import wsgd_weights
        from oracle.operator import cn_scalars
        n2 = n1 if n2 is None else n2
        self.problem, self.n1, self.n2 = problem, n1, n2
        X, Y, hx, hy = problem.grid(n1, n2)
        self.hx, self.hy = hx, hy
        self.dt = hx if dt is None else dt
        self.sc = cn_scalars(problem.alpha, problem.beta, hx, hy, self.dt)
        self.wx = wsgd_weights(problem.alpha, n1 + 1, 1, problem.qx)
        self.wy = wsgd_weights(problem.beta, n2 + 1, 1, problem.qy)
        self.coef_new = problem.coefficients(X, Y, m * self.dt)
        self.coef_old = problem.coefficients(X, Y, (m - 1) * self.dt)
        self.v = problem.source(X, Y, (m - 0.5) * self.dt)
        self.u0 = problem.exact(X, Y, (m - 1) * self.dt)
        a1, b1, a2, b2 = problem.domain
        self.params = fde.params(alpha=problem.alpha, beta=problem.beta, qx=problem.qx,
                                 qy=problem.qy, a1=a1, b1=b1, a2=a2, b2=b2, n1=n1, n2=n2,
                                 dt=self.dt, **kw)

    def handle(self):
        h = fde.fde_create(self.params)
        self.dnew = [dev(f) for f in self.coef_new]
        self.dold = [dev(f) for f in self.coef_old]
        fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *self.dnew)
        fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *self.dold)
        return h

    def oracle_apply(self, X):
        from oracle.operator import apply_M
        return apply_M(X, self.wx, self.wy, self.sc["c"], self.sc["sigma"], *self.coef_new)

    def oracle_abs_apply(self, X):
        """|c||x| + |D+||A||x| + ... : the elementwise scale of rounding errors of M x."""
        from oracle.operator import apply_kron, toeplitz_A
        Ax, Ay = np.abs(toeplitz_A(self.wx, self.n1)), np.abs(toeplitz_A(self.wy, self.n2))
        cf = [np.abs(f) for f in self.coef_new]
        return apply_kron(np.abs(X), Ax, Ay, abs(self.sc["c"]), abs(self.sc["sigma"]), *cf)

    def oracle_rhs(self):
        from oracle.operator import rhs
        return rhs(self.u0, self.wx, self.wy, self.sc["c"], self.sc["sigma"], *self.coef_old,
                   self.v, self.hx, self.problem.alpha)

    def oracle_hierarchy(self):
        from oracle import multigrid as mg
        p = self.params
        c, s = self.sc["c"], self.sc["sigma"]
        if p.precond == fde.FDE_PRECOND_P2:
            return mg.band_p2(self.n1, self.n2, c, s, self.coef_new, p.coarsest_n)
        if p.precond == fde.FDE_PRECOND_MG_EXACT:
            from oracle.operator import assemble_M, toeplitz_A
            K0 = assemble_M(toeplitz_A(self.wx, self.n1), toeplitz_A(self.wy, self.n2), c, s,
                            *self.coef_new)
            return mg.exact_galerkin(K0, self.n1, self.n2, p.coarsest_n)
        if p.precond == fde.FDE_PRECOND_MG_SG:
            return mg.structured_galerkin(self.wx, self.wy, self.n1, self.n2, c, s,
                                          self.coef_new, p.coarsest_n)
        return mg.rediscretised(self.problem.alpha, self.problem.beta, self.wx, self.wy,
                                self.n1, self.n2, c, s, self.coef_new, p.coarsest_n)


def sampled_apply(Ax, Ay, c, sigma, dp, dm, ep, em, X, rows, cols):
    """Rows `rows` and columns `cols` of K x and of |K||x| for
    K = c I + D+ (I (x) Ax) + D- (I (x) Ax^T) + sigma [E+ (Ay (x) I) + E- (Ay^T (x) I)]
    (Eq. M written with dense 1-D factors), each entry summed on its own:
    O(n^2) per sampled line instead of the whole O(n^3) product.
    Returns (K x rows, |K||x| rows, K x cols, |K||x| cols)."""
    X = np.asarray(X)
    aX, aAx, aAy = np.abs(X), np.abs(Ax), np.abs(Ay)

    def row(j, Z, A1, A2, absolute):
        f = (lambda a: np.abs(a)) if absolute else (lambda a: a)
        return (abs(c) * Z[j] if absolute else c * Z[j]) \
            + f(dp[j]) * (Z[j] @ A1.T) + f(dm[j]) * (Z[j] @ A1) \
            + (abs(sigma) if absolute else sigma) * (
                f(ep[j]) * (A2[j] @ Z) + f(em[j]) * (A2.T[j] @ Z))

    def col(i, Z, A1, A2, absolute):
        f = (lambda a: np.abs(a)) if absolute else (lambda a: a)
        return (abs(c) * Z[:, i] if absolute else c * Z[:, i]) \
            + f(dp[:, i]) * (Z @ A1.T[:, i]) + f(dm[:, i]) * (Z @ A1[:, i]) \
            + (abs(sigma) if absolute else sigma) * (
                f(ep[:, i]) * (A2 @ Z[:, i]) + f(em[:, i]) * (A2.T @ Z[:, i]))

    R = np.array([row(j, X, Ax, Ay, False) for j in rows])
    Ra = np.array([row(j, aX, aAx, aAy, True) for j in rows])
    C = np.array([col(i, X, Ax, Ay, False) for i in cols]).T
    Ca = np.array([col(i, aX, aAx, aAy, True) for i in cols]).T
    return R, Ra, C, Ca


def sample_lines(n, count, rng):
    """`count` line indices of an n-point axis: both ends, the tile edges of
    128 and 256 near the middle, and random interior lines."""
    fixed = [0, 1, n - 2, n - 1, min(n - 1, 127), min(n - 1, 128), min(n - 1, 255),
             min(n - 1, 256)]
    extra = list(rng.choice(n, size=max(0, count - len(fixed)), replace=False))
    return sorted(set(int(v) for v in fixed + extra))

"""Fractional Grunwald coefficients and WSGD weights (Sec. 2, Eq. gk, Eq. w).

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np

GAMMA0 = (-1.0 + np.sqrt(17.0)) / 2.0  # Sec. 2: w_2 >= 0 (M-matrix) for gamma >= gamma_0


def grunwald_g(gamma, K):
    """g_k = (-1)^k binom(gamma, k), k = 0..K (Eq. gk).

    Written as the defining product (-1)^k/k! * gamma(gamma-1)...(gamma-k+1),
    accumulated one factor at a time: g_k = g_{k-1} * (k-1-gamma)/k.
    """
    g = np.empty(K + 1, dtype=np.float64)
    g[0] = 1.0
    for k in range(1, K + 1):
        g[k] = g[k - 1] * ((k - 1) - gamma) / k
    return g


def wsgd_weights(gamma, K, p=1, q=0):
    """WSGD weights w_0..w_K for shifts (p, q).

    (p, q) = (1, 0) is Eq. (w): w_0 = gamma/2 g_0, w_k = gamma/2 g_k + (2-gamma)/2 g_{k-1}.
    The paper defines only (1, 0).  For (1, -1) the general weighted-and-shifted
    Grunwald combination of the paper's reference [39] is used,
        lambda_p A_p + lambda_q A_q,  lambda_p = (gamma-2q)/(2(p-q)),
        lambda_q = (2p-gamma)/(2(p-q)),
    whose shifted sums, re-indexed on u_{i-k+1}, give
        w_k = lambda_p g_k + lambda_q g_{k-(p-q)}   (g_{<0} = 0),
    which reduces to Eq. (w) at (1, 0).  Only p = 1 is meaningful here because
    the matrix A = -[w_{i-j+1}] (Eq. AN) fixes the shift of the first term.
    """
    if p != 1:
        raise ValueError("only p = 1 keeps the structure A = -[w_{i-j+1}] of Eq. (AN)")
    if q not in (0, -1):
        raise ValueError("q must be 0 or -1")
    d = p - q
    lam_p = (gamma - 2.0 * q) / (2.0 * d)
    lam_q = (2.0 * p - gamma) / (2.0 * d)
    g = grunwald_g(gamma, K)
    w = lam_p * g.copy()
    w[d:] += lam_q * g[: K + 1 - d]
    return w


def choose_shift(alpha, beta):
    """Shift choice used by the randomly drawn workloads: (1, 0) is proved
    stable (M-matrix) only for gamma >= gamma_0 (Sec. 2); below it the (1, -1)
    weights are used.  Returns q."""
    return 0 if min(alpha, beta) >= GAMMA0 else -1

"""Seeded synthetic inputs for the CN-WSGD solve: diffusion coefficients,
manufactured exact solutions and their source terms (problem (1) of Sec. 2).

This module holds the continuous problem data only -- no step of the
discretisation or of the solver.  Both the CUDA path and the CPU oracle take
their inputs from here.

Source terms follow from the Riemann-Liouville definitions of Sec. 2: for a
monomial in the distance to the left end, D^a_+ (x-a)^m = G(m+1)/G(m+1-a) (x-a)^(m-a),
and for a monomial in the distance to the right end,
D^a_- (b-x)^m = G(m+1)/G(m+1-a) (b-x)^(m-a).  A bubble (x-a)^p (b-x)^p is
expanded binomially in either distance, so every derivative is a closed form.
"""
from dataclasses import dataclass, field
from math import comb, gamma as G
from typing import Callable, Optional

import numpy as np

# ----------------------------------------------------------------------------
# bubbles and their fractional derivatives


def _bubble_coeffs(p, L):
    """(s)^p (L - s)^p = sum_k coef_k s^(p+k): returns {power: coefficient}."""
    return {p + k: comb(p, k) * L ** (p - k) * (-1) ** k for k in range(p + 1)}


def bubble(x, a, b, p):
    return (x - a) ** p * (b - x) ** p


def bubble_dleft(x, a, b, p, alpha):
    """Left RL derivative of order alpha of (x-a)^p (b-x)^p on [a, x]."""
    s = x - a
    out = np.zeros_like(s)
    for m, cf in _bubble_coeffs(p, b - a).items():
        out = out + cf * G(m + 1) / G(m + 1 - alpha) * s ** (m - alpha)
    return out


def bubble_dright(x, a, b, p, alpha):
    """Right RL derivative of order alpha of (x-a)^p (b-x)^p on [x, b]."""
    t = b - x
    out = np.zeros_like(t)
    for m, cf in _bubble_coeffs(p, b - a).items():
        out = out + cf * G(m + 1) / G(m + 1 - alpha) * t ** (m - alpha)
    return out


# ----------------------------------------------------------------------------
# problem description


Coef = Callable[[np.ndarray, np.ndarray, float], np.ndarray]


@dataclass
class Problem:
    """Problem (1) of Sec. 2 with the manufactured solution
    u = amp * exp(-t) * X(x) * Y(y),  X = bubble(x; a1, b1, p), Y = bubble(y; a2, b2, p)."""
    name: str
    alpha: float
    beta: float
    domain: tuple  # (a1, b1, a2, b2)
    dp: Coef
    dm: Coef
    ep: Coef
    em: Coef
    p: int = 2
    amp: float = 1.0
    qx: int = 0  # WSGD shift q for x (p = 1 always)
    qy: int = 0
    time_dependent: bool = False
    meta: dict = field(default_factory=dict)

    # grid ------------------------------------------------------------------
    def grid(self, n1, n2=None):
        n2 = n1 if n2 is None else n2
        a1, b1, a2, b2 = self.domain
        hx = (b1 - a1) / (n1 + 1)
        hy = (b2 - a2) / (n2 + 1)
        x = a1 + hx * np.arange(1, n1 + 1)
        y = a2 + hy * np.arange(1, n2 + 1)
        X, Y = np.meshgrid(x, y)  # shape (n2, n1), x fastest
        return X, Y, hx, hy

    # fields ----------------------------------------------------------------
    def exact(self, X, Y, t):
        a1, b1, a2, b2 = self.domain
        return self.amp * np.exp(-t) * bubble(X, a1, b1, self.p) * bubble(Y, a2, b2, self.p)

    def coefficients(self, X, Y, t):
        return (np.asarray(self.dp(X, Y, t), dtype=np.float64) + 0 * X,
                np.asarray(self.dm(X, Y, t), dtype=np.float64) + 0 * X,
                np.asarray(self.ep(X, Y, t), dtype=np.float64) + 0 * X,
                np.asarray(self.em(X, Y, t), dtype=np.float64) + 0 * X)

    def source(self, X, Y, t):
        """v = u_t - d+ D^a_+x u - d- D^a_-x u - e+ D^b_+y u - e- D^b_-y u (problem (1))."""
        a1, b1, a2, b2 = self.domain
        p, al, be = self.p, self.alpha, self.beta
        et = self.amp * np.exp(-t)
        g = _axes(X, Y)
        if g is not None:
            # grid input: every factor depends on x or y alone; evaluate it on the
            # axis and broadcast (the same values as on the full grid)
            xs, ys = g
            Xe = lambda f, *a: np.broadcast_to(f(xs, *a)[None, :], X.shape)
            Ye = lambda f, *a: np.broadcast_to(f(ys, *a)[:, None], X.shape)
        else:
            Xe = lambda f, *a: f(X, *a)
            Ye = lambda f, *a: f(Y, *a)
        Xb, Yb = Xe(bubble, a1, b1, p), Ye(bubble, a2, b2, p)
        dp, dm, ep, em = self.coefficients(X, Y, t)
        return (-et * Xb * Yb
                - dp * et * Yb * Xe(bubble_dleft, a1, b1, p, al)
                - dm * et * Yb * Xe(bubble_dright, a1, b1, p, al)
                - ep * et * Xb * Ye(bubble_dleft, a2, b2, p, be)
                - em * et * Xb * Ye(bubble_dright, a2, b2, p, be))


# ----------------------------------------------------------------------------
# the three examples of Sec. 5


def example1():
    """Sec. 5, Example 1: alpha=1.8, beta=1.6 on [0,2]^2,
    u = 16 e^-t x^2 (2-x)^2 y^2 (2-y)^2.  The initial condition is u(., ., 0)
    of that solution (the printed u_0 drops the factor 16)."""
    al, be = 1.8, 1.6
    ga, gb = G(3 - al), G(3 - be)
    return Problem("example1", al, be, (0.0, 2.0, 0.0, 2.0),
                   dp=lambda x, y, t: ga * (1 + x) ** al * (1 + y) ** 2,
                   dm=lambda x, y, t: ga * (3 - x) ** al * (3 - y) ** 2,
                   ep=lambda x, y, t: gb * (1 + x) ** 2 * (1 + y) ** be,
                   em=lambda x, y, t: gb * (3 - x) ** 2 * (3 - y) ** be,
                   p=2, amp=16.0)


def example2():
    """Sec. 5, Example 2: alpha=1.8, beta=1.9 on [0,1]^2, time-dependent
    coefficients, u = e^-t x^3 (1-x)^3 y^3 (1-y)^3."""
    al, be = 1.8, 1.9
    return Problem("example2", al, be, (0.0, 1.0, 0.0, 1.0),
                   dp=lambda x, y, t: 4 * (1 + t) * x ** al * (1 + y),
                   dm=lambda x, y, t: 4 * (1 + t) * (1 - x) ** al * (1 + y),
                   ep=lambda x, y, t: 4 * (1 + t) * (1 + x) * y ** be,
                   em=lambda x, y, t: 4 * (1 + t) * (1 + x) * (1 - y) ** be,
                   p=3, amp=1.0, time_dependent=True)


def example3():
    """Sec. 5, Example 3: alpha=1.8, beta=1.9 on [0,1]^2,
    d+ = 6x^a, d- = 6(1-x)^a, e+ = 6y^b, e- = 6(1-y)^b, u as in Example 2."""
    al, be = 1.8, 1.9
    return Problem("example3", al, be, (0.0, 1.0, 0.0, 1.0),
                   dp=lambda x, y, t: 6 * x ** al + 0 * y,
                   dm=lambda x, y, t: 6 * (1 - x) ** al + 0 * y,
                   ep=lambda x, y, t: 6 * y ** be + 0 * x,
                   em=lambda x, y, t: 6 * (1 - y) ** be + 0 * x,
                   p=3, amp=1.0)


# ----------------------------------------------------------------------------
# synthetic workloads shaped like the examples (bubble solutions, smooth
# positive coefficients, dt ~ h)

_GAMMA0 = (-1.0 + np.sqrt(17.0)) / 2.0


def _axes(X, Y):
    """(x, y) 1-D axes when X, Y are a meshgrid (x along rows, y down columns), else None."""
    X, Y = np.asarray(X), np.asarray(Y)
    if X.ndim != 2 or X.shape != Y.shape:
        return None
    if not (np.all(X == X[:1, :]) and np.all(Y == Y[:, :1])):
        return None
    return X[0, :], Y[:, 0]


def _shift_q(alpha, beta):
    return 0 if min(alpha, beta) >= _GAMMA0 else -1


def constant_unit(alpha=1.8, beta=1.6):
    """d+ = d- = e+ = e- = 1 on [0,1]^2, u = e^-t x^2(1-x)^2 y^2(1-y)^2, WSGD (1,0)."""
    one = lambda x, y, t: 1.0 + 0 * x
    return Problem("constant_unit", alpha, beta, (0.0, 1.0, 0.0, 1.0), one, one, one, one, p=2,
                   qx=0, qy=0)


def power_law(alpha=1.3, beta=1.9, q=-1):
    """d+ = 1 + x^a y, d- = 1 + (1-x)^a y, e+ = 1 + y^b x, e- = 1 + (1-y)^b x."""
    return Problem("power_law", alpha, beta, (0.0, 1.0, 0.0, 1.0),
                   dp=lambda x, y, t: 1 + x ** alpha * y,
                   dm=lambda x, y, t: 1 + (1 - x) ** alpha * y,
                   ep=lambda x, y, t: 1 + y ** beta * x,
                   em=lambda x, y, t: 1 + (1 - y) ** beta * x,
                   p=2, qx=q, qy=q)


def smooth_modes(seed, n_modes=8, kmax=4):
    """A smooth field phi(x, y) = sum_k a_k sin(pi k1 x + th_k) sin(pi k2 y + ps_k),
    k1, k2 in {1..kmax}, drawn from PCG64(seed), normalised so that its maximum
    modulus on a fixed 513 x 513 sample of [0,1]^2 is 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k1 = rng.integers(1, kmax + 1, n_modes)
    k2 = rng.integers(1, kmax + 1, n_modes)
    a = rng.uniform(-1.0, 1.0, n_modes)
    th = rng.uniform(0.0, 2 * np.pi, n_modes)
    ps = rng.uniform(0.0, 2 * np.pi, n_modes)

    def raw(x, y):
        g = _axes(x, y)
        if g is not None:
            # grid input: the same products from the 1-D factors, broadcast
            xs, ys = g
            out = np.zeros(np.broadcast(x, y).shape)
            for i in range(n_modes):
                sx = np.sin(np.pi * k1[i] * xs + th[i])[None, :]
                sy = np.sin(np.pi * k2[i] * ys + ps[i])[:, None]
                out = out + a[i] * sx * sy
            return out
        out = 0.0 * (x + y)
        for i in range(n_modes):
            out = out + a[i] * np.sin(np.pi * k1[i] * x + th[i]) * np.sin(np.pi * k2[i] * y + ps[i])
        return out

    s = np.linspace(0.0, 1.0, 513)
    SX, SY = np.meshgrid(s, s)
    scale = 1.0 / np.max(np.abs(raw(SX, SY)))
    return lambda x, y: scale * raw(x, y)


def perturbed_power_law(alpha=1.5, beta=1.7, seed=1706068, amplitude=0.2):
    """``power_law`` coefficients each multiplied by (1 + amplitude * phi_c),
    phi_c = ``smooth_modes`` of four sub-seeds of ``seed``; every coefficient
    stays >= (1 - amplitude) times its unperturbed value > 0."""
    q = _shift_q(alpha, beta)
    base = power_law(alpha, beta, q)
    subs = np.random.SeedSequence(seed).spawn(4)
    phis = [smooth_modes(int(s.generate_state(1)[0])) for s in subs]
    f = lambda c, ph: (lambda x, y, t: c(x, y, t) * (1 + amplitude * ph(x, y)))
    return Problem("perturbed_power_law", alpha, beta, (0.0, 1.0, 0.0, 1.0),
                   dp=f(base.dp, phis[0]), dm=f(base.dm, phis[1]),
                   ep=f(base.ep, phis[2]), em=f(base.em, phis[3]),
                   p=2, qx=q, qy=q, meta={"seed": seed, "amplitude": amplitude})


def random_batch(count=256, seed=1706069, sizes=(63, 127, 255, 511)):
    """``count`` independent problems: n uniform over ``sizes``, alpha, beta ~
    U(1.1, 1.9), WSGD q drawn from {0, -1} (forced to -1 below gamma_0),
    coefficients exp(ln2 * psi) in [0.5, 2] with psi = ``smooth_modes``.
    Returns a list of (n, Problem)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for idx in range(count):
        n = int(rng.choice(sizes))
        al, be = rng.uniform(1.1, 1.9, 2)
        q = int(rng.choice([0, -1]))
        if min(al, be) < _GAMMA0:
            q = -1
        sub = rng.integers(0, 2 ** 62, 4)
        psis = [smooth_modes(int(s)) for s in sub]
        f = lambda ps: (lambda x, y, t: np.exp(np.log(2.0) * ps(x, y)))
        out.append((n, Problem(f"batch{idx}", float(al), float(be), (0.0, 1.0, 0.0, 1.0),
                               f(psis[0]), f(psis[1]), f(psis[2]), f(psis[3]), p=2, qx=q, qy=q)))
    return out


# ----------------------------------------------------------------------------
# per-step arrays


@dataclass
class StepData:
    """Everything one CN step from t^(m-1) to t^(m) needs (Eq. CNWSGD, Eq. system)."""
    coef_new: tuple   # d+, d-, e+, e- at t^(m)
    coef_old: tuple   # same at t^(m-1)
    v_half: np.ndarray  # source at t^(m-1/2)


def step_data(problem: Problem, n1, n2, m, dt):
    X, Y, hx, hy = problem.grid(n1, n2)
    t_new, t_old = m * dt, (m - 1) * dt
    return StepData(problem.coefficients(X, Y, t_new), problem.coefficients(X, Y, t_old),
                    problem.source(X, Y, t_old + 0.5 * dt))


def initial(problem: Problem, n1, n2=None):
    X, Y, hx, hy = problem.grid(n1, n2)
    return problem.exact(X, Y, 0.0)

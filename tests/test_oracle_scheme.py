"""Whole-scheme pins of the oracle against Sec. 5: the error columns of
Tables 1-3 (a property of the discretisation and the manufactured source),
second-order convergence, the GMRES column of Table 1, and the preconditioned
iteration counts of Tables 1-3 (soft: the V-cycle is under-specified)."""
import json
import os

import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from oracle import timeloop
from oracle.krylov import gmres_left
from oracle.wsgd import wsgd_weights
from oracle.operator import cn_scalars, rhs, apply_M

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
EX = {"table1_example1": inputs.example1, "table2_example2": inputs.example2,
      "table3_example3": inputs.example3}


@pytest.mark.parametrize("table", list(EX))
@pytest.mark.parametrize("idx", [0, 1])
def test_error_column(table, idx):
    # Error = ||u(T) - u^M||_inf at T = 1 with n = M; the printed values carry
    # 5 significant digits and come from a tol-1e-7 GMRES solve, so a 0.3 %
    # band covers both the rounding and that solver error
    n = GOLD[table]["n"][idx]
    ref = GOLD[table]["error"][idx]
    r = timeloop.run(EX[table](), n, precond="sg", restart=30, rtol=1e-11)
    assert abs(r["error_inf"] - ref) <= 3e-3 * ref


@pytest.mark.slow
def test_error_column_n64_example1():
    r = timeloop.run(inputs.example1(), 64, precond="sg", restart=30, rtol=1e-11)
    ref = GOLD["table1_example1"]["error"][2]
    assert abs(r["error_inf"] - ref) <= 3e-3 * ref


def test_second_order():
    # Sec. 2: truncation error O(h^2 + dt^2); with dt ~ h the error ratio tends to 4
    e = [GOLD["table1_example1"]["error"][i] for i in range(2)]
    r = [timeloop.run(inputs.example1(), n, precond="sg", rtol=1e-11)["error_inf"] for n in (16, 32)]
    np.testing.assert_allclose(r[0] / r[1], e[0] / e[1], rtol=5e-3)
    assert 3.5 < r[0] / r[1] < 4.5


@pytest.mark.parametrize("idx", [0, 1])
def test_gmres_column_table1(idx):
    # Table 1's unpreconditioned column is reproduced by GMRES without restarts
    # at tol 1e-7 (a restart after 20 steps gives 49 at n = 16)
    n = GOLD["table1_example1"]["n"][idx]
    r = timeloop.run(inputs.example1(), n, precond="none", restart=400, rtol=1e-7)
    assert abs(r["mean_iterations"] - GOLD["table1_example1"]["gmres"][idx]) <= 0.25


def _left_counts(problem, n, kind, omega):
    X, Y, hx, hy = problem.grid(n, n)
    dt = 1.0 / n
    wx, wy = wsgd_weights(problem.alpha, n), wsgd_weights(problem.beta, n)
    sc = cn_scalars(problem.alpha, problem.beta, hx, hy, dt)
    c, s = sc["c"], sc["sigma"]
    U = problem.exact(X, Y, 0.0)
    its = []
    for m in range(1, n + 1):
        co, cn = problem.coefficients(X, Y, (m - 1) * dt), problem.coefficients(X, Y, m * dt)
        B = rhs(U, wx, wy, c, s, *co, problem.source(X, Y, (m - 0.5) * dt), hx, problem.alpha)
        prec, _ = timeloop.make_preconditioner(kind, problem.alpha, problem.beta, wx, wy, n, n,
                                               sc, cn, omega=omega)
        U, k, rel, ok = gmres_left(lambda Z: apply_M(Z, wx, wy, c, s, *cn), B, prec, 20, 1e-7)
        its.append(k)
    return float(np.mean(its))


@pytest.mark.parametrize("table", list(EX))
@pytest.mark.parametrize("kind,col", [("redisc", "p_mgm"), ("p2", "p2")])
def test_preconditioned_counts_soft(table, kind, col):
    # left preconditioning with a preconditioned-residual test, classical Jacobi
    # (omega = 1), as in Sec. 4.2 / Sec. 5; the V-cycle details the paper leaves
    # open allow a band of +-2.5 iterations
    for idx in (0, 1):
        n = GOLD[table]["n"][idx]
        got = _left_counts(EX[table](), n, kind, 1.0)
        assert abs(got - GOLD[table][col][idx]) <= 2.5, (n, got)

"""The paper's experiments (Sec. 5, Tables 1-3) on the GPU at the paper's own
even grid sizes n = 16, 32 (coarse j on fine 2j - 1, Sec. 4.1's K matrix):
the whole CN time loop, M = n steps to T = 1, every step from a zero initial
guess, Example 2's coefficients re-set (and the hierarchy rebuilt on the
device) at every step.

Pinned two ways:
  * against the paper: the final infinity-norm error equals the Error column
    of Tables 1-3 within the 0.3 % band of the oracle's own pins (the printed
    values carry 5 digits and come from a tol-1e-7 solve); Table 1's
    unpreconditioned GMRES column (37 at n = 16, GMRES without restarts) is
    the GPU's mean iteration count;
  * against the oracle's time loop with the same preconditioner and FGMRES(20):
    iteration counts per step within 1 (CGS2 on the GPU, MGS in the oracle),
    final error equal to the oracle's.
The preconditioners are the paper's geometric P_MGM (rediscretised V-cycle),
its Galerkin tilde-P_MGM (exact P^T A P levels, dense, the GPU's validation
mode) and the band preconditioner P_2 (Sec. 4.3), in FP64."""
import json
import os

import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import Case, dev, host

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
EX = {"table1_example1": inputs.example1, "table2_example2": inputs.example2,
      "table3_example3": inputs.example3}
PRECOND = {"redisc": fde.FDE_PRECOND_MG_REDISC, "p2": fde.FDE_PRECOND_P2,
           "galerkin": fde.FDE_PRECOND_MG_EXACT, "none": fde.FDE_PRECOND_NONE}


def gpu_time_loop(prob, n, precond, restart, rtol):
    """The CN time loop of Sec. 5 through the C ABI; returns (final error,
    iterations per step)."""
    import torch
    dt = 1.0 / n
    case = Case(prob, n, dt=dt, precond=PRECOND[precond], restart=restart, rtol=rtol,
                maxit=5000)
    h = fde.fde_create(case.params)
    try:
        X, Y, hx, hy = prob.grid(n, n)
        ud = dev(prob.exact(X, Y, 0.0))
        un = torch.empty_like(ud)
        its = []
        cnew = None
        for m in range(1, n + 1):
            if m == 1 or prob.time_dependent:
                cold = [dev(f) for f in prob.coefficients(X, Y, (m - 1) * dt)]
                cnew = [dev(f) for f in prob.coefficients(X, Y, m * dt)]
                fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *cold)
                fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *cnew)
            st = fde.fde_step(h, ud, dev(prob.source(X, Y, (m - 0.5) * dt)), un)
            assert st.converged == 1, m
            its.append(st.iterations)
            ud, un = un, ud
        err = float(np.max(np.abs(prob.exact(X, Y, 1.0) - host(ud))))
        return err, its
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precond", ["redisc", "p2", "galerkin"])
@pytest.mark.parametrize("idx", [0, 1])
@pytest.mark.parametrize("table", list(EX))
def test_table_error_column_and_oracle_time_loop(table, idx, precond):
    from oracle import timeloop
    prob = EX[table]()
    n = GOLD[table]["n"][idx]
    rtol = 1e-11
    err, its = gpu_time_loop(prob, n, precond, 20, rtol)
    ref_err = GOLD[table]["error"][idx]
    assert abs(err - ref_err) <= 3e-3 * ref_err, (err, ref_err)
    ref = timeloop.run(prob, n, precond=precond, restart=20, rtol=rtol)
    np.testing.assert_allclose(err, ref["error_inf"], rtol=1e-6)
    assert np.max(np.abs(np.array(its) - np.array(ref["iterations"]))) <= 1, (its,
                                                                            ref["iterations"])


def test_table1_gmres_column_n16():
    # unpreconditioned GMRES without restarts (64 > 37 iterations) at tol 1e-7:
    # Table 1 prints 37.000 at n = 16; this runs the Gram-Schmidt passes for
    # bases longer than 32 vectors
    err, its = gpu_time_loop(inputs.example1(), 16, "none", 64, 1e-7)
    assert abs(np.mean(its) - GOLD["table1_example1"]["gmres"][0]) <= 0.25, its


@pytest.mark.parametrize("idx", [0, 1])
def test_table1_galerkin_column_soft(idx):
    # Table 1's tilde-P_MGM column (10, 11 at n = 16, 32) comes from Matlab's
    # left-preconditioned GMRES(20) with classical Jacobi at tol 1e-7; the GPU
    # runs right-preconditioned FGMRES with damped Jacobi (omega = 0.7) on the
    # true residual, so the mean count is a soft pin (within 2.5, the oracle's
    # own band for the preconditioned columns)
    err, its = gpu_time_loop(inputs.example1(), GOLD["table1_example1"]["n"][idx], "galerkin",
                             20, 1e-7)
    assert abs(np.mean(its) - GOLD["table1_example1"]["p_mgm_galerkin"][idx]) <= 2.5, its

"""Degenerate cases of the CUDA path against the oracle: a zero right-hand
side, the smallest grids, and multigrid hierarchies of a single level (a grid
at or below the coarsest size in either direction, Sec. 4.2), where the
V-cycle is the coarsest-grid solve itself."""
import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import Case, dev, host

pytestmark = pytest.mark.gpu


def _dense(case):
    from oracle.operator import toeplitz_A, assemble_M
    return assemble_M(toeplitz_A(case.wx, case.n1), toeplitz_A(case.wy, case.n2),
                      case.sc["c"], case.sc["sigma"], *case.coef_new)


@pytest.mark.parametrize("solver", [fde.FDE_SOLVER_FGMRES, fde.FDE_SOLVER_MG])
@pytest.mark.parametrize("precond", [fde.FDE_PRECOND_MG_SG, fde.FDE_PRECOND_P2])
def test_zero_rhs_gives_zero_without_iterations(solver, precond):
    # ||b|| = 0: x = 0 meets any relative tolerance before the first iteration
    import torch
    case = Case(inputs.perturbed_power_law(), 63, precond=precond, solver=solver)
    h = case.handle()
    try:
        b = torch.zeros((63, 63), dtype=torch.float64, device="cuda")
        x = torch.full_like(b, 7.0)
        st = fde.fde_solve(h, b, x)
        assert st.converged == 1 and st.iterations == 0
        assert torch.count_nonzero(x).item() == 0
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision", [fde.FDE_PREC_FP64, fde.FDE_PREC_FP32])
@pytest.mark.parametrize("precond", [fde.FDE_PRECOND_MG_SG, fde.FDE_PRECOND_MG_REDISC])
@pytest.mark.parametrize("n1,n2,cycles", [(3, 3, 1), (7, 7, 1), (7, 7, 2), (5, 31, 2)])
def test_one_level_toeplitz_hierarchy_is_a_direct_solve(precision, precond, n1, n2, cycles):
    # one level: the preconditioner is the exact inverse of level 0 = M (its
    # FP64 dense inverse; FP32 rounds the vectors), so FGMRES needs one
    # iteration in FP64 and a few in FP32; the solution is the dense solve's
    # within cond(M) x rtol
    import torch
    rtol = 1e-10
    case = Case(inputs.power_law(), n1, n2, precision=precision, precond=precond, cycles=cycles,
                rtol=rtol)
    h = case.handle()
    try:
        assert fde.fde_levels(h) == [(n1, n2)]
        B = np.random.default_rng(100 * n1 + n2).standard_normal((n2, n1))
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        K = _dense(case)
        xd = np.linalg.solve(K, B.ravel())
        assert st.converged == 1
        assert st.iterations <= (1 if precision == fde.FDE_PREC_FP64 else 4), st.iterations
        err = np.linalg.norm(host(x).ravel() - xd) / np.linalg.norm(xd)
        assert err <= 1.1 * np.linalg.cond(K) * rtol, err
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision", [fde.FDE_PREC_FP64, fde.FDE_PREC_FP32])
@pytest.mark.parametrize("n1,n2,cycles", [(7, 7, 1), (5, 31, 2)])
def test_one_level_p2_hierarchy_is_the_exact_band_preconditioner(precision, n1, n2, cycles):
    # one level of P_2: the preconditioner is P_2^{-1} itself (Sec. 4.3), so the
    # count follows the oracle's FGMRES with a sparse LU of P_2
    import torch
    import scipy.sparse.linalg as spla
    from oracle import multigrid as mg
    from oracle.krylov import fgmres
    rtol = 1e-10
    case = Case(inputs.power_law(), n1, n2, precision=precision, precond=fde.FDE_PRECOND_P2,
                cycles=cycles, rtol=rtol)
    h = case.handle()
    try:
        assert fde.fde_levels(h) == [(n1, n2)]
        B = np.random.default_rng(100 * n1 + n2).standard_normal((n2, n1))
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        c, s = case.sc["c"], case.sc["sigma"]
        lu = spla.splu(mg.band_p2_matrix(n1, n2, c, s, case.coef_new).tocsc())
        prec = lambda R: lu.solve(np.asarray(R).ravel()).reshape(n2, n1)
        xo, its, rel, ok = fgmres(case.oracle_apply, B, prec, 30, rtol)
        assert ok and st.converged == 1
        assert st.iterations <= its + (1 if precision == fde.FDE_PREC_FP64 else 3), (st.iterations, its)
        K = _dense(case)
        xd = np.linalg.solve(K, B.ravel())
        err = np.linalg.norm(host(x).ravel() - xd) / np.linalg.norm(xd)
        assert err <= 1.1 * np.linalg.cond(K) * rtol, err
    finally:
        fde.fde_destroy(h)

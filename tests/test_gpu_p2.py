"""The band preconditioner P_2 of Sec. 4.3 on the GPU (five-point Laplacian
operator with the problem's coefficients, Galerkin V-cycle with nine-point
coarse stencils) against the oracle's sparse exact-Galerkin hierarchy, and
repeated V-cycles per preconditioner application (Sec. 5.1)."""
import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import Case, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    fde.lib()


def _vcycles(hier, R, omega, cycles):
    from oracle import multigrid as mg
    X = mg.vcycle(hier, R, omega, 1, 1)
    for _ in range(cycles - 1):
        X = X + mg.vcycle(hier, R - hier.levels[0].apply(X), omega, 1, 1)
    return X


@pytest.mark.parametrize("n1,n2", [(63, 63), (127, 127), (31, 63), (255, 255), (511, 127),
                                   (64, 64), (32, 48), (100, 36)])
def test_fp64_levels_and_vcycle(n1, n2):
    # stencil levels: the Galerkin products are formed in FP64 from at most 81
    # terms per entry, the applies sum nine products: relative 1e-13 against
    # the oracle's sparse P^T K P; one V-cycle: relative 1e-12
    import torch
    case = Case(inputs.perturbed_power_law(), n1, n2, precond=fde.FDE_PRECOND_P2)
    h = case.handle()
    try:
        hier = case.oracle_hierarchy()
        levels = fde.fde_levels(h)
        assert [(L.n1, L.n2) for L in hier.levels] == levels
        rng = np.random.default_rng(21)
        for l, lev in enumerate(hier.levels):
            Xl = rng.standard_normal((lev.n2, lev.n1))
            yl = torch.empty_like(dev(Xl))
            fde.fde_level_apply(h, l, dev(Xl), yl)
            torch.cuda.synchronize()
            rl = lev.apply(Xl)
            assert np.max(np.abs(host(yl) - rl)) <= 1e-13 * np.max(np.abs(rl)), l
        R = rng.standard_normal((n2, n1))
        z = torch.empty_like(dev(R))
        fde.fde_vcycle(h, dev(R), z)
        torch.cuda.synchronize()
        ref = _vcycles(hier, R, case.params.omega, 1)
        assert np.max(np.abs(host(z) - ref)) <= 1e-12 * np.max(np.abs(ref))
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precond", [fde.FDE_PRECOND_P2, fde.FDE_PRECOND_MG_SG])
@pytest.mark.parametrize("cycles", [2, 3])
def test_repeated_vcycles(precond, cycles):
    # z_{k+1} = z_k + V(r - K_0 z_k): the oracle's stationary iteration
    import torch
    case = Case(inputs.perturbed_power_law(), 127, precond=precond, cycles=cycles)
    h = case.handle()
    try:
        hier = case.oracle_hierarchy()
        R = np.random.default_rng(22).standard_normal((127, 127))
        z = torch.empty_like(dev(R))
        fde.fde_vcycle(h, dev(R), z)
        torch.cuda.synchronize()
        ref = _vcycles(hier, R, case.params.omega, cycles)
        assert np.max(np.abs(host(z) - ref)) <= 1e-11 * np.max(np.abs(ref))
    finally:
        fde.fde_destroy(h)


def test_fp32_vcycle_close_to_oracle():
    import torch
    case = Case(inputs.perturbed_power_law(), 255, precond=fde.FDE_PRECOND_P2,
                precision=fde.FDE_PREC_FP32)
    h = case.handle()
    try:
        hier = case.oracle_hierarchy()
        R = np.random.default_rng(23).standard_normal((255, 255))
        z = torch.empty_like(dev(R))
        fde.fde_vcycle(h, dev(R), z)
        torch.cuda.synchronize()
        ref = _vcycles(hier, R, 0.7, 1)
        assert np.linalg.norm(host(z) - ref) <= 1e-5 * np.linalg.norm(ref)
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision", [fde.FDE_PREC_FP64, fde.FDE_PREC_FP32])
@pytest.mark.parametrize("cycles", [1, 2])
def test_solve_matches_oracle(precision, cycles):
    # FGMRES preconditioned by P_2: true residual below rtol, same solution as
    # the oracle, iteration counts within one (FP64) or two (FP32)
    import torch
    from oracle.krylov import fgmres
    case = Case(inputs.perturbed_power_law(), 127, precond=fde.FDE_PRECOND_P2,
                precision=precision, cycles=cycles, rtol=1e-10)
    h = case.handle()
    try:
        B = case.oracle_rhs()
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        xg = host(x)
        res = np.linalg.norm(B - case.oracle_apply(xg)) / np.linalg.norm(B)
        assert st.converged == 1 and res <= 1.05e-10, res
        hier = case.oracle_hierarchy()
        xo, its, rel, ok = fgmres(case.oracle_apply, B,
                                  lambda R: _vcycles(hier, R, 0.7, cycles), 30, 1e-10)
        assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
        tol = 1 if precision == fde.FDE_PREC_FP64 else 2
        assert abs(st.iterations - its) <= tol, (st.iterations, its)
    finally:
        fde.fde_destroy(h)


def test_level0_full_size_sampled_rows():
    # n = 2047 (the bench grid): level 0 is P_2 itself; compare 256 sampled
    # rows against the oracle's sparse P_2, including the four boundary edges
    import torch
    from oracle import multigrid as mg
    n = 2047
    case = Case(inputs.perturbed_power_law(), n, precond=fde.FDE_PRECOND_P2,
                precision=fde.FDE_PREC_FP32)
    h = case.handle()
    try:
        rng = np.random.default_rng(24)
        X = rng.standard_normal((n, n))
        y = torch.empty_like(dev(X))
        fde.fde_level_apply(h, 0, dev(X), y)
        torch.cuda.synchronize()
        K = mg.band_p2_matrix(n, n, case.sc["c"], case.sc["sigma"], case.coef_new)
        rows = np.concatenate([rng.integers(0, n * n, 248), [0, n - 1, n * (n - 1), n * n - 1,
                                                            n, 2 * n - 1, n * n - n - 1, 5]])
        ref = K[rows] @ X.ravel()
        got = host(y).ravel()[rows]
        # FP32 stencil and vector: |err| <= 2^-22 (|K| |x|)
        absr = abs(K[rows]) @ np.abs(X.ravel())
        assert np.all(np.abs(got - ref) <= 2.0 ** -21 * absr)
    finally:
        fde.fde_destroy(h)


def test_p2_rejects_bad_cycles():
    case = Case(inputs.perturbed_power_law(), 63, precond=fde.FDE_PRECOND_P2, cycles=5)
    with pytest.raises(fde.FDEError):
        fde.fde_create(case.params)

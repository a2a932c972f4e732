"""n = 4095: FFT length 8192, where two complex buffers of 16-byte values no
longer fit in shared memory (one-buffer passes with the forward spectrum parked
in global memory; twiddles of the spectra builds in global memory), and the
tensor-core products of the two finest levels (n = 4095 and 2047), whose
generator windows are streamed per job.  The operator apply and the level-0
tensor-core products are checked element by element against the oracle, and
full solves against the oracle's FP64 true residual."""
import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import Case, dev, host, sampled_apply, sample_lines

pytestmark = pytest.mark.gpu

N = 4095
EPS = np.finfo(np.float64).eps
OUTER_EPS = {fde.FDE_OUTER_FP64: EPS, fde.FDE_OUTER_DF32: 2.0 ** -47}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    fde.lib()


def _problem():
    # the n = 4095 workload: alpha = 1.9, beta = 1.2, perturbed power-law fields
    return inputs.perturbed_power_law(alpha=1.9, beta=1.2)


@pytest.mark.parametrize("outer", [fde.FDE_OUTER_FP64, fde.FDE_OUTER_DF32])
def test_outer_apply_n4095(outer):
    # The rounding error of an FFT-based product grows with the number of
    # stages, log2 L, and is normwise (the error of a floating-point FFT is
    # bounded relative to the 2-norm of its input, not element by element):
    # per element it is at most c u log2(L) (|M||x|_i + rms |M||x|), here with
    # c = 8 (8 x 9 stages = 72 u covers the 64 u bound of the n <= 255 tests)
    import torch
    case = Case(_problem(), N, precond=fde.FDE_PRECOND_NONE, outer=outer)
    h = case.handle()
    try:
        X = np.random.default_rng(41).standard_normal((N, N))
        y = torch.empty_like(dev(X))
        fde.fde_apply(h, dev(X), y)
        torch.cuda.synchronize()
        ref = case.oracle_apply(X)
        absr = case.oracle_abs_apply(X)
        bound = 8 * 13 * OUTER_EPS[outer] * (absr + np.sqrt(np.mean(absr ** 2)))
        err = np.abs(host(y) - ref)
        assert np.all(err <= bound), float(np.max(err / bound))
    finally:
        fde.fde_destroy(h)


def test_gemm_level0_products_n4095():
    # BF16x3 tensor-core products of the 4095 x 4095 level (32 x 16 tiles of
    # 128 x 256, 64 K blocks each) on sampled rows and columns, under the
    # elementwise error model of the smaller sizes
    import torch
    from oracle.operator import toeplitz_A
    case = Case(_problem(), N, precond=fde.FDE_PRECOND_MG_SG, precision=fde.FDE_PREC_BF16X3,
                toeplitz_path=fde.FDE_PATH_GEMM)
    h = case.handle()
    try:
        assert fde.fde_level_path(h, 0) == fde.FDE_PATH_GEMM
        assert fde.fde_level_path(h, 1) == fde.FDE_PATH_GEMM
        rng = np.random.default_rng(4095)
        X = rng.standard_normal((N, N))
        y = torch.empty_like(dev(X))
        fde.fde_level_apply(h, 0, dev(X), y)
        torch.cuda.synchronize()
        yh = host(y)
        Ax, Ay = toeplitz_A(case.wx, N), toeplitz_A(case.wy, N)
        rows, cols = sample_lines(N, 16, rng), sample_lines(N, 16, rng)
        R, Ra, C, Ca = sampled_apply(Ax, Ay, case.sc["c"], case.sc["sigma"], *case.coef_new, X,
                                     rows, cols)
        u = 2 * 2.0 ** -16 + N * 2.0 ** -24 + 2.0 ** -22
        for got, ref, ab in [(yh[rows], R, Ra), (yh[:, cols], C, Ca)]:
            err = np.abs(got - ref)
            assert np.all(err <= u * ab + 1e-30), float(np.max(err / (u * ab + 1e-300)))
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision", [fde.FDE_PREC_FP32, fde.FDE_PREC_BF16X3, fde.FDE_PREC_BF16])
def test_solve_n4095(precision):
    # FGMRES(20) with the structured-Galerkin V-cycle: the oracle recomputes
    # the FP64 true residual of the returned solution
    import torch
    case = Case(_problem(), N, precond=fde.FDE_PRECOND_MG_SG, precision=precision,
                outer=fde.FDE_OUTER_DF32, restart=20, rtol=1e-8)
    h = case.handle()
    try:
        B = case.oracle_rhs()
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        res = np.linalg.norm(B - case.oracle_apply(host(x))) / np.linalg.norm(B)
        assert st.converged == 1 and res <= 1.05e-8, (res, st.iterations)
        # beta = 1.2 is far from 2: the oracle needs 43, 51, 59 iterations at
        # n = 127, 255, 511 (about 8 more per doubling, so ~83 at n = 4095)
        assert st.iterations <= 110, st.iterations
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision,tol", [(fde.FDE_PREC_FP32, 2), (fde.FDE_PREC_BF16X3, 3)])
def test_iterations_match_oracle_n511(precision, tol):
    # the same workload at n = 511, where the oracle's FGMRES(20) runs: the
    # iteration counts agree (CGS2 vs MGS and reduced-precision products)
    import torch
    from oracle.krylov import fgmres
    from oracle import multigrid as mg
    case = Case(_problem(), 511, precond=fde.FDE_PRECOND_MG_SG, precision=precision,
                toeplitz_path=fde.FDE_PATH_GEMM if precision == fde.FDE_PREC_BF16X3
                else fde.FDE_PATH_AUTO, outer=fde.FDE_OUTER_DF32, restart=20, rtol=1e-8)
    h = case.handle()
    try:
        B = case.oracle_rhs()
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        hier = case.oracle_hierarchy()
        xo, its, rel, ok = fgmres(case.oracle_apply, B, lambda R: mg.vcycle(hier, R), 20, 1e-8)
        assert st.converged == 1 and ok
        assert abs(st.iterations - its) <= tol, (st.iterations, its)
    finally:
        fde.fde_destroy(h)


def test_fp64_solver_n4095_vcycle_levels():
    # the plain FP64 solver: FP64 FFT level products at L = 8192 also take the
    # one-buffer pass; its level-0 product matches the oracle's Kronecker form
    import torch
    case = Case(_problem(), N, precond=fde.FDE_PRECOND_MG_SG, precision=fde.FDE_PREC_FP64,
                toeplitz_path=fde.FDE_PATH_FFT)
    h = case.handle()
    try:
        hier = case.oracle_hierarchy()
        X = np.random.default_rng(42).standard_normal((N, N))
        y = torch.empty_like(dev(X))
        fde.fde_level_apply(h, 0, dev(X), y)
        torch.cuda.synchronize()
        ref = hier.levels[0].apply(X)
        assert np.max(np.abs(host(y) - ref)) <= 1e-12 * np.max(np.abs(ref))
    finally:
        fde.fde_destroy(h)

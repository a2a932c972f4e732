"""tcgen05 Toeplitz GEMM levels (BF16/FP16 operands, FP32 accumulation)
against the FP64 oracle's level operators.

Error model: operands are rounded once to 16 bits (relative 2^-9 for BF16,
2^-12 for FP16 incl. the Toeplitz bank), products are exact in FP32 and the
accumulation adds at most K 2^-24 relative; so elementwise
|K x - K~ x| <= (2 u16 + n 2^-24) * (|c||x| + |D||A||x| + ...) plus the FP32
rounding of the coefficient fields (2^-24)."""
import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import Case, dev, host, sampled_apply, sample_lines

pytestmark = pytest.mark.gpu

U16 = {fde.FDE_PREC_BF16: 2.0 ** -8, fde.FDE_PREC_FP16: 2.0 ** -11,
       fde.FDE_PREC_BF16X3: 2.0 ** -16}


def _abs_level(lev, X):
    from oracle.operator import apply_kron
    A = lambda M: None if M is None else np.abs(M)
    return apply_kron(np.abs(X), A(lev.Ax), A(lev.Ay), abs(lev.c), abs(lev.sigma),
                      np.abs(lev.dp), np.abs(lev.dm), np.abs(lev.ep), np.abs(lev.em),
                      A(lev.Bx), A(lev.By))


@pytest.mark.parametrize("precision", [fde.FDE_PREC_BF16, fde.FDE_PREC_FP16, fde.FDE_PREC_BF16X3])
@pytest.mark.parametrize("precond", [fde.FDE_PRECOND_MG_SG, fde.FDE_PRECOND_MG_REDISC])
@pytest.mark.parametrize("n1,n2", [(255, 255), (511, 255), (383, 767), (511, 511), (1023, 1023)])
def test_gemm_level_apply(precision, precond, n1, n2):
    # every level the tensor path serves (n >= 127), incl. ragged tiles (383 = 240+143),
    # the structured-Galerkin mass terms of coarse levels, and split K (tiles
    # of 511 and 1023 leave most SMs idle: 2 and 3 CTAs share a tile's K range)
    import torch
    if (n1 - 1) // 2 % 2 == 0 and n1 > 255:
        pytest.skip("level sizes must stay odd")
    case = Case(inputs.perturbed_power_law(), n1, n2, precond=precond, precision=precision,
                toeplitz_path=fde.FDE_PATH_GEMM)
    # a tensor-core level that cannot be created is a failure, not a skip
    h = case.handle()
    try:
        for l, (m1, m2) in enumerate(fde.fde_levels(h)[:-1]):
            if min(m1, m2) >= 127:
                assert fde.fde_level_path(h, l) == fde.FDE_PATH_GEMM, l
        hier = case.oracle_hierarchy()
        rng = np.random.default_rng(9)
        for l, lev in enumerate(hier.levels):
            if min(lev.n1, lev.n2) < 127:
                break
            X = rng.standard_normal((lev.n2, lev.n1))
            y = torch.empty_like(dev(X))
            fde.fde_level_apply(h, l, dev(X), y)
            torch.cuda.synchronize()
            ref = lev.apply(X)
            bound = (2 * U16[precision] + max(lev.n1, lev.n2) * 2.0 ** -24 + 2.0 ** -22) * _abs_level(lev, X)
            err = np.abs(host(y) - ref)
            assert np.all(err <= bound + 1e-30), (l, float(np.max(err / (bound + 1e-300))))
            # and the products are not trivially inaccurate
            rel = np.linalg.norm(host(y) - ref) / np.linalg.norm(ref)
            assert rel <= 0.05
            # 16-bit operands really were used (an FP32 path would sit near 1e-7)
            assert rel > 1e-6 * (U16[precision] / 2.0 ** -11), rel
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision", [fde.FDE_PREC_BF16X3, fde.FDE_PREC_BF16, fde.FDE_PREC_FP16])
def test_gemm_level0_products_n2047(precision):
    # the bench grid's level-0 products forced onto the tensor cores (no tuner,
    # no fallback), element by element on sampled rows and columns (both ends,
    # the 128/256 tile edges, random lines) against the oracle's level-0
    # operator under the same error model as the smaller sizes
    import torch
    from oracle.operator import toeplitz_A
    n = 2047
    case = Case(inputs.perturbed_power_law(), n, precond=fde.FDE_PRECOND_MG_SG,
                precision=precision, toeplitz_path=fde.FDE_PATH_GEMM)
    h = case.handle()
    try:
        assert fde.fde_level_path(h, 0) == fde.FDE_PATH_GEMM
        rng = np.random.default_rng(2047)
        X = rng.standard_normal((n, n))
        y = torch.empty_like(dev(X))
        fde.fde_level_apply(h, 0, dev(X), y)
        torch.cuda.synchronize()
        yh = host(y)
        Ax, Ay = toeplitz_A(case.wx, n), toeplitz_A(case.wy, n)
        rows, cols = sample_lines(n, 24, rng), sample_lines(n, 24, rng)
        R, Ra, C, Ca = sampled_apply(Ax, Ay, case.sc["c"], case.sc["sigma"], *case.coef_new, X,
                                     rows, cols)
        u = 2 * U16[precision] + n * 2.0 ** -24 + 2.0 ** -22
        for got, ref, ab in [(yh[rows], R, Ra), (yh[:, cols], C, Ca)]:
            err = np.abs(got - ref)
            assert np.all(err <= u * ab + 1e-30), float(np.max(err / (u * ab + 1e-300)))
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel > 1e-6 * (U16[precision] / 2.0 ** -11), rel  # 16-bit operands used
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision", [fde.FDE_PREC_BF16, fde.FDE_PREC_FP16, fde.FDE_PREC_BF16X3])
def test_mixed_solve_converges_to_fp64_residual(precision):
    # the reduced-precision V-cycle only preconditions: the FP64 FGMRES still
    # drives the true residual below rtol, and the solution matches the oracle's
    import torch
    from oracle.krylov import fgmres
    from oracle import multigrid as mg
    case = Case(inputs.perturbed_power_law(), 255, precision=precision, rtol=1e-10,
                toeplitz_path=fde.FDE_PATH_GEMM)
    h = case.handle()
    try:
        B = case.oracle_rhs()
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        xg = host(x)
        res = np.linalg.norm(B - case.oracle_apply(xg)) / np.linalg.norm(B)
        assert st.converged and res <= 1.05e-10
        hier = case.oracle_hierarchy()
        xo, its, rel, ok = fgmres(case.oracle_apply, B, lambda R: mg.vcycle(hier, R), 30, 1e-12)
        assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)
        assert st.iterations <= its + 3, (st.iterations, its)
    finally:
        fde.fde_destroy(h)


def test_tuned_paths_and_vcycle():
    # FDE_PATH_TUNE times each level's candidate paths (tensor cores, FFT,
    # direct) at the first set-up and keeps the fastest; the cycle stays a
    # BF16x3-accurate cycle whatever it picks
    import torch
    from oracle import multigrid as mg
    case = Case(inputs.perturbed_power_law(), 511, precision=fde.FDE_PREC_BF16X3,
                toeplitz_path=fde.FDE_PATH_TUNE)
    h = case.handle()
    try:
        levels = fde.fde_levels(h)
        for l, (n1, n2) in enumerate(levels):
            path = fde.fde_level_path(h, l)
            if l == len(levels) - 1:
                assert path == -1
            elif min(n1, n2) >= 127:
                assert path in (fde.FDE_PATH_GEMM, fde.FDE_PATH_FFT, fde.FDE_PATH_DIRECT), (l, path)
            else:
                assert path in (fde.FDE_PATH_FFT, fde.FDE_PATH_DIRECT), (l, path)
        hier = case.oracle_hierarchy()
        R = np.random.default_rng(31).standard_normal((511, 511))
        z = torch.empty_like(dev(R))
        fde.fde_vcycle(h, dev(R), z)
        torch.cuda.synchronize()
        ref = mg.vcycle(hier, R, 0.7, 1, 1)
        assert np.linalg.norm(host(z) - ref) <= 1e-3 * np.linalg.norm(ref)
    finally:
        fde.fde_destroy(h)


def test_capped_wait_gives_up_and_reports_timeout():
    # failure detection without a fault: the tensor-core kernels' bounded
    # mbarrier wait runs once on a barrier that nothing completes; it gives up
    # after 20 ms and raises the level's device flag, the next solve writes its
    # result as usual and returns FDE_ERR_TIMEOUT, and the flag is cleared: the
    # context stays usable and the following solve is clean
    import time
    import torch
    case = Case(inputs.perturbed_power_law(), 127, precision=fde.FDE_PREC_BF16X3, rtol=1e-10,
                toeplitz_path=fde.FDE_PATH_GEMM)
    h = case.handle()
    try:
        B = case.oracle_rhs()
        b = dev(B)
        x = torch.empty_like(b)
        fde.fde_wait_selftest(h, 1)  # a completed barrier raises nothing
        st = fde.fde_solve(h, b, x)
        assert st.converged
        x_ref = host(x).copy()
        t0 = time.perf_counter()
        fde.fde_wait_selftest(h, 0)
        torch.cuda.synchronize()
        assert time.perf_counter() - t0 < 5.0
        x.zero_()
        with pytest.raises(fde.FDEError) as e:
            fde.fde_solve(h, b, x)
        assert e.value.code == fde.FDE_ERR_TIMEOUT
        assert np.linalg.norm(host(x) - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
        st = fde.fde_solve(h, b, x)
        assert st.converged
        assert np.linalg.norm(host(x) - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
        res = np.linalg.norm(B - case.oracle_apply(host(x))) / np.linalg.norm(B)
        assert res <= 1.05e-10
    finally:
        fde.fde_destroy(h)


def test_wait_selftest_needs_a_tensor_core_level():
    case = Case(inputs.perturbed_power_law(), 63, precision=fde.FDE_PREC_FP32)
    h = case.handle()
    try:
        with pytest.raises(fde.FDEError) as e:
            fde.fde_wait_selftest(h, 0)
        assert e.value.code == fde.FDE_ERR_UNSUPPORTED
        with pytest.raises(fde.FDEError) as e:
            fde.fde_wait_selftest(h, 2)
        assert e.value.code == fde.FDE_ERR_ARG
    finally:
        fde.fde_destroy(h)

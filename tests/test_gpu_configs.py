"""The workload configurations at their full sizes, in the configuration the
bench times: n = 511 with the power-law coefficients (plain FP64 solver), and
n = 2047 with the mixed-precision solver exactly as bench.py runs it (BF16x3
tensor-core level 0 chosen by the autotuner, relaxed matvec), checked through
the oracle's FP64 operator and against the plain FP64 GPU solver's iteration
count."""
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


def _oracle_fft_apply(case):
    from oracle.operator import apply_M_fft
    return lambda X: apply_M_fft(X, case.wx, case.wy, case.sc["c"], case.sc["sigma"],
                                 *case.coef_new)


def test_power_law_n511_fp64_steps_match_oracle():
    # n = 511, alpha = 1.3, beta = 1.9, WSGD (1,-1), dt = h, plain FP64 solver:
    # two CN steps, each within 1e-8 (relative L2) of the oracle's solve to 1e-12
    import torch
    from oracle.krylov import fgmres
    from oracle.operator import rhs_fft
    prob = inputs.power_law()
    n = 511
    case = Case(prob, n, precision=fde.FDE_PREC_FP64, rtol=1e-8)
    h = case.handle()
    try:
        hier = case.oracle_hierarchy()
        from oracle import multigrid as mg
        X, Y, hx, hy = prob.grid(n, n)
        A = _oracle_fft_apply(case)
        U = prob.exact(X, Y, 0.0)
        ud = dev(U)
        un = torch.empty_like(ud)
        for m in (1, 2):
            V = prob.source(X, Y, (m - 0.5) * case.dt)
            st = fde.fde_step(h, ud, dev(V), un)
            B = rhs_fft(U, case.wx, case.wy, case.sc["c"], case.sc["sigma"], *case.coef_old, V,
                        hx, prob.alpha)
            U, its, rel, ok = fgmres(A, B, lambda R: mg.vcycle(hier, R), 30, 1e-12)
            assert np.linalg.norm(host(un) - U) <= 1e-8 * np.linalg.norm(U), m
            ud, un = un, ud
    finally:
        fde.fde_destroy(h)


def test_bench_configuration_n2047():
    # the n = 2047 workload as bench.py runs it; the oracle's FFT operator
    # re-checks the true residual, and the iteration count equals the plain
    # FP64 GPU solver's (target: within one)
    import torch
    prob = inputs.perturbed_power_law()
    n = 2047
    its = {}
    for name, kw in [("mixed", dict(precision=fde.FDE_PREC_BF16X3, toeplitz_path=fde.FDE_PATH_TUNE,
                                    outer=fde.FDE_OUTER_DF32, relax=1)),
                     ("mixed_gemm", dict(precision=fde.FDE_PREC_BF16X3,
                                         toeplitz_path=fde.FDE_PATH_GEMM,
                                         outer=fde.FDE_OUTER_DF32, relax=1)),
                     ("fp64", dict(precision=fde.FDE_PREC_FP64))]:
        case = Case(prob, n, rtol=1e-8, maxit=2000, **kw)
        h = case.handle()
        try:
            from oracle.operator import rhs_fft
            X, Y, hx, hy = prob.grid(n, n)
            B = rhs_fft(case.u0, case.wx, case.wy, case.sc["c"], case.sc["sigma"],
                        *case.coef_old, case.v, hx, prob.alpha)
            x = torch.empty_like(dev(B))
            st = fde.fde_solve(h, dev(B), x)
            res = np.linalg.norm(B - _oracle_fft_apply(case)(host(x))) / np.linalg.norm(B)
            assert st.converged == 1 and res <= 1.05e-8, (name, res)
            its[name] = st.iterations
            if name == "mixed":
                # the tuner's choice for level 0: tensor cores or FFT products
                assert fde.fde_level_path(h, 0) in (fde.FDE_PATH_GEMM, fde.FDE_PATH_FFT)
                assert st.relaxed > 0
            if name == "mixed_gemm":
                # the same solve with level 0 on the tensor cores
                assert fde.fde_level_path(h, 0) == fde.FDE_PATH_GEMM
        finally:
            fde.fde_destroy(h)
    assert abs(its["mixed"] - its["fp64"]) <= 1, its
    assert abs(its["mixed_gemm"] - its["fp64"]) <= 1, its

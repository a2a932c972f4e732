"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Sizes span several FFT lengths, ragged (non-power-of-two) grids,
non-square grids and both WSGD shifts; tolerances come from the arithmetic
and are written next to each check."""
import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import Case, dev, host

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    fde.lib()


def _cases():
    return [
        ("unit_63", lambda: Case(inputs.constant_unit(), 63)),
        ("power_31x63", lambda: Case(inputs.power_law(), 31, 63)),
        ("perturbed_127", lambda: Case(inputs.perturbed_power_law(), 127)),
        ("example1_15", lambda: Case(inputs.example1(), 15)),
    ]


@pytest.mark.parametrize("name,mk", _cases())
def test_weights_on_device(name, mk):
    # Eq. (gk)/(w): same recurrence in FP64 on both sides; the GPU may fuse the
    # final combination into an FMA, so allow a few ulps
    case = mk()
    h = case.handle()
    try:
        w = np.array(fde.fde_weights(h, 0, case.n1 + 1))
        np.testing.assert_allclose(w, case.wx[: case.n1 + 1], rtol=4 * EPS, atol=4 * EPS)
        w = np.array(fde.fde_weights(h, 1, case.n2 + 1))
        np.testing.assert_allclose(w, case.wy[: case.n2 + 1], rtol=4 * EPS, atol=4 * EPS)
    finally:
        fde.fde_destroy(h)


# unit roundoff of the outer apply: FP64, or double-float (two FP32 words, the
# trailing one rounded: 2^-47 per operation)
OUTER_EPS = {fde.FDE_OUTER_FP64: EPS, fde.FDE_OUTER_DF32: 2.0 ** -47}


@pytest.mark.parametrize("outer", [fde.FDE_OUTER_FP64, fde.FDE_OUTER_DF32])
@pytest.mark.parametrize("name,mk", _cases())
def test_outer_apply_and_rhs(name, mk, outer):
    # FFT-embedding product: error ~ u log2(L) times the absolute sums
    # |c||x| + |D||A||x| + ...; 64 u leaves room for log2(L) <= 9 stages
    import torch
    case = mk()
    case.params.outer = outer
    h = case.handle()
    try:
        rng = np.random.default_rng(3)
        X = rng.standard_normal((case.n2, case.n1))
        y = torch.empty_like(dev(X))
        fde.fde_apply(h, dev(X), y)
        torch.cuda.synchronize()
        ref = case.oracle_apply(X)
        bound = 64 * OUTER_EPS[outer] * case.oracle_abs_apply(X)
        assert np.all(np.abs(host(y) - ref) <= bound)
        b = torch.empty_like(y)
        fde.fde_rhs(h, dev(case.u0), dev(case.v), b)
        torch.cuda.synchronize()
        rb = case.oracle_rhs()
        assert np.max(np.abs(host(b) - rb)) <= 1e-12 * np.max(np.abs(rb))
        if outer == fde.FDE_OUTER_DF32:
            # and it is not silently the FP64 path: df32 rounding is visible
            assert np.max(np.abs(host(y) - ref) / (case.oracle_abs_apply(X) + 1e-300)) > 2 * EPS
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precond", [fde.FDE_PRECOND_MG_SG, fde.FDE_PRECOND_MG_REDISC])
@pytest.mark.parametrize("n1,n2", [(63, 63), (127, 127), (31, 63), (255, 255)])
def test_fp64_vcycle_matches_oracle(precond, n1, n2):
    # one V-cycle (Sec. 4) in FP64: same algorithm, rounding-order differences
    # only (FFT vs matmul products): relative 1e-11
    _fp64_vcycle_check(precond, n1, n2)


@pytest.mark.parametrize("n1,n2", [(64, 64), (128, 128), (32, 48), (100, 36), (16, 16)])
def test_fp64_vcycle_even_sizes(n1, n2):
    # even and mixed-parity grids (the paper's n = 16 .. 128): coarse j on fine
    # 2j - 1 and the bilinear stencil truncated at the low end (Sec. 4.1's K
    # matrix), rediscretised coarse operators; the same bars as odd sizes
    _fp64_vcycle_check(fde.FDE_PRECOND_MG_REDISC, n1, n2)


@pytest.mark.parametrize("n1,n2", [(31, 31), (32, 32), (63, 63), (16, 48), (64, 64)])
def test_exact_galerkin_levels_and_vcycle(n1, n2):
    # the exact Galerkin hierarchy (dense P^T A P on the device, FP64) for
    # variable coefficients, either parity: every level operator within 1e-12
    # of the oracle's dense triple products (rounding order only: each entry
    # sums at most 81 products per level), one V-cycle within 1e-11
    _fp64_vcycle_check(fde.FDE_PRECOND_MG_EXACT, n1, n2)


def test_exact_galerkin_differs_from_structured_for_variable_coefficients():
    # Sec. 4.2 calls the exact Galerkin operator of variable coefficients
    # infeasible at scale; the structured reading injects the coefficients
    # instead: on level 1 the two differ by far more than rounding (and agree
    # exactly for constant coefficients, tested separately)
    import torch
    rng = np.random.default_rng(8)
    outs = {}
    for pc in (fde.FDE_PRECOND_MG_SG, fde.FDE_PRECOND_MG_EXACT):
        case = Case(inputs.perturbed_power_law(), 63, precond=pc)
        h = case.handle()
        try:
            X = rng.standard_normal((31, 31)) if not outs else outs["X"]
            y = torch.empty_like(dev(X))
            fde.fde_level_apply(h, 1, dev(X), y)
            torch.cuda.synchronize()
            outs[pc] = host(y)
            outs["X"] = X
        finally:
            fde.fde_destroy(h)
    d = np.linalg.norm(outs[fde.FDE_PRECOND_MG_SG] - outs[fde.FDE_PRECOND_MG_EXACT])
    assert d > 1e-4 * np.linalg.norm(outs[fde.FDE_PRECOND_MG_EXACT])


def test_exact_galerkin_limits():
    case = Case(inputs.perturbed_power_law(), 65, precond=fde.FDE_PRECOND_MG_EXACT)
    with pytest.raises(fde.FDEError) as e:
        fde.fde_create(case.params)  # 65^2 > 4096: dense levels refused
    assert e.value.code == fde.FDE_ERR_UNSUPPORTED
    case = Case(inputs.perturbed_power_law(), 31, precond=fde.FDE_PRECOND_MG_EXACT,
                precision=fde.FDE_PREC_FP32)
    with pytest.raises(fde.FDEError) as e:
        fde.fde_create(case.params)
    assert e.value.code == fde.FDE_ERR_ARG


def test_structured_galerkin_rejects_even_levels():
    # projecting a Toeplitz factor of an even level is no longer Toeplitz
    case = Case(inputs.perturbed_power_law(), 64, precond=fde.FDE_PRECOND_MG_SG)
    with pytest.raises(fde.FDEError) as e:
        fde.fde_create(case.params)
    assert e.value.code == fde.FDE_ERR_UNSUPPORTED


def _fp64_vcycle_check(precond, n1, n2):
    import torch
    from oracle import multigrid as mg
    case = Case(inputs.perturbed_power_law(), n1, n2, precond=precond)
    h = case.handle()
    try:
        hier = case.oracle_hierarchy()
        rng = np.random.default_rng(5)
        R = rng.standard_normal((n2, n1))
        z = torch.empty_like(dev(R))
        fde.fde_vcycle(h, dev(R), z)
        torch.cuda.synchronize()
        ref = mg.vcycle(hier, R, case.params.omega, case.params.nu_pre, case.params.nu_post)
        err = np.max(np.abs(host(z) - ref)) / np.max(np.abs(ref))
        assert err <= 1e-11, err
        # every level operator
        levels = fde.fde_levels(h)
        assert [(L.n1, L.n2) for L in hier.levels] == levels
        for l, lev in enumerate(hier.levels):
            Xl = rng.standard_normal((lev.n2, lev.n1))
            yl = torch.empty_like(dev(Xl))
            fde.fde_level_apply(h, l, dev(Xl), yl)
            torch.cuda.synchronize()
            rl = lev.apply(Xl)
            assert np.max(np.abs(host(yl) - rl)) <= 1e-12 * np.max(np.abs(rl)), l
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precond", [fde.FDE_PRECOND_MG_SG, fde.FDE_PRECOND_MG_REDISC])
def test_fp32_vcycle_close_to_oracle(precond):
    # FP32 V-cycle: the cycle is linear and contractive, so the FP32 result
    # stays within a few hundred FP32 ulps of the FP64 one (relative 1e-4)
    import torch
    from oracle import multigrid as mg
    case = Case(inputs.perturbed_power_law(), 255, precond=precond,
                precision=fde.FDE_PREC_FP32)
    h = case.handle()
    try:
        hier = case.oracle_hierarchy()
        R = np.random.default_rng(6).standard_normal((255, 255))
        z = torch.empty_like(dev(R))
        fde.fde_vcycle(h, dev(R), z)
        torch.cuda.synchronize()
        ref = mg.vcycle(hier, R, 0.7, 1, 1)
        assert np.linalg.norm(host(z) - ref) <= 1e-4 * np.linalg.norm(ref)
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision,outer", [(fde.FDE_PREC_FP64, fde.FDE_OUTER_FP64),
                                             (fde.FDE_PREC_FP32, fde.FDE_OUTER_FP64),
                                             (fde.FDE_PREC_BF16, fde.FDE_OUTER_DF32)])
@pytest.mark.parametrize("name,mk", _cases()[:3])
def test_solve_matches_oracle(name, mk, precision, outer):
    # FGMRES to rtol 1e-10 on both sides: the GPU's true residual (re-checked by
    # the oracle) meets rtol, the solutions agree within the conditioning bound,
    # and iteration counts differ by at most one (CGS2 vs MGS rounding)
    import torch
    from oracle.krylov import fgmres
    from oracle import multigrid as mg
    case = mk()
    case.params.rtol = 1e-10
    case.params.precision = precision
    case.params.outer = outer
    h = case.handle()
    try:
        B = case.oracle_rhs()
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        xg = host(x)
        res = np.linalg.norm(B - case.oracle_apply(xg)) / np.linalg.norm(B)
        assert st.converged == 1 and res <= 1.05e-10, res
        hier = case.oracle_hierarchy()
        xo, its, rel, ok = fgmres(case.oracle_apply, B, lambda R: mg.vcycle(hier, R), 30, 1e-10)
        assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
        if precision == fde.FDE_PREC_FP64:
            assert abs(st.iterations - its) <= 1, (st.iterations, its)
        elif precision == fde.FDE_PREC_FP32:
            assert abs(st.iterations - its) <= 2, (st.iterations, its)
        else:
            assert st.iterations <= its + 4, (st.iterations, its)
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("restart", [5, 40])
def test_restarts_and_long_bases(restart):
    # unpreconditioned FGMRES needs ~100 iterations here: restart 5 runs many
    # restart cycles (true residual recomputed, V_0 rebuilt, the device-side
    # Arnoldi state restarted), restart 40 builds bases longer than the 32
    # vectors of the fused Gram-Schmidt passes (separate passes beyond that);
    # both meet the oracle's FP64 true residual, and the iteration count stays
    # within 2 of the oracle's MGS FGMRES with the same restart length
    import torch
    from oracle.krylov import fgmres
    case = Case(inputs.perturbed_power_law(), 31, precond=fde.FDE_PRECOND_NONE, rtol=1e-8,
                restart=restart, maxit=5000)
    h = case.handle()
    try:
        B = case.oracle_rhs()
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        res = np.linalg.norm(B - case.oracle_apply(host(x))) / np.linalg.norm(B)
        assert st.converged and res <= 1.05e-8, res
        xo, its, rel, ok = fgmres(case.oracle_apply, B, None, restart, 1e-8, maxit=5000)
        assert ok and abs(st.iterations - its) <= 2, (st.iterations, its)
        if restart == 40:
            assert st.iterations > 33  # the separate-pass branch ran
        assert st.restarts >= (st.iterations + restart - 1) // restart
    finally:
        fde.fde_destroy(h)


def test_time_loop_matches_oracle():
    # eight CN steps (Eq. CNWSGD) of the constant-coefficient bubble at n = 63:
    # each step's solution within 1e-8 (relative L2) of the oracle's solve
    import torch
    from oracle.krylov import fgmres
    from oracle import multigrid as mg
    from oracle.operator import rhs, apply_M
    prob = inputs.constant_unit()
    n, steps = 63, 8
    case = Case(prob, n, rtol=1e-10)
    h = case.handle()
    try:
        X, Y, hx, hy = prob.grid(n, n)
        dt = case.dt
        U = prob.exact(X, Y, 0.0)
        ud = dev(U)
        un = torch.empty_like(ud)
        c, s = case.sc["c"], case.sc["sigma"]
        hier = case.oracle_hierarchy()
        for m in range(1, steps + 1):
            V = prob.source(X, Y, (m - 0.5) * dt)
            st = fde.fde_step(h, ud, dev(V), un)
            B = rhs(U, case.wx, case.wy, c, s, *case.coef_old, V, hx, prob.alpha)
            U, its, rel, ok = fgmres(lambda Z: apply_M(Z, case.wx, case.wy, c, s, *case.coef_new),
                                     B, lambda R: mg.vcycle(hier, R), 30, 1e-12)
            ug = host(un)
            assert np.linalg.norm(ug - U) <= 1e-8 * np.linalg.norm(U), m
            ud, un = un, ud
        assert fde.fde_get_state(h) == steps
    finally:
        fde.fde_destroy(h)


def test_step_host_matches_device_step():
    import torch
    case = Case(inputs.perturbed_power_law(), 63)
    h = case.handle()
    try:
        u_next = np.zeros_like(case.u0)
        st1 = fde.fde_step_host(h, np.ascontiguousarray(case.u0), np.ascontiguousarray(case.v), u_next)
        x = torch.empty_like(dev(case.u0))
        st2 = fde.fde_step(h, dev(case.u0), dev(case.v), x)
        assert st1.iterations == st2.iterations
        np.testing.assert_array_equal(u_next, host(x))
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("restart", [30, 4])
def test_step_host_pinned_two_steps_match_device_steps(restart):
    # pinned host arrays: the source's upload overlaps the right-hand side's
    # operator apply and every restart cycle's solution is copied out while
    # its true residual is checked (restart 4: several cycles, so later
    # updates wait for earlier copies); two steps in a row with different
    # sources give the device path's bits
    import torch
    case = Case(inputs.perturbed_power_law(), 127, restart=restart, precision=fde.FDE_PREC_FP32,
                outer=fde.FDE_OUTER_DF32, relax=1)
    X, Y, _, _ = case.problem.grid(127, 127)
    v2 = case.problem.source(X, Y, 1.5 * case.dt)
    h = case.handle()
    try:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        u0, s1, s2 = pin(case.u0), pin(case.v), pin(v2)
        u1, u2 = torch.empty_like(u0).pin_memory(), torch.empty_like(u0).pin_memory()
        fde.fde_step_host(h, u0.data_ptr(), s1.data_ptr(), u1.data_ptr())
        fde.fde_step_host(h, u1.data_ptr(), s2.data_ptr(), u2.data_ptr())
        d0 = dev(case.u0)
        d1, d2 = torch.empty_like(d0), torch.empty_like(d0)
        fde.fde_step(h, d0, dev(case.v), d1)
        fde.fde_step(h, d1, dev(v2), d2)
        np.testing.assert_array_equal(u1.numpy(), host(d1))
        np.testing.assert_array_equal(u2.numpy(), host(d2))
    finally:
        fde.fde_destroy(h)


def test_error_paths():
    # host-side failure injection: bad arguments, non-finite data, too few iterations
    import torch
    with pytest.raises(fde.FDEError) as e:
        fde.fde_create(fde.params(n1=64, n2=64))  # even sizes cannot be coarsened
    assert e.value.code == fde.FDE_ERR_UNSUPPORTED
    case = Case(inputs.perturbed_power_law(), 63, maxit=1)
    h = case.handle()
    try:
        B = dev(case.oracle_rhs())
        x = torch.empty_like(B)
        st = fde.fde_solve(h, B, x, allow_not_converged=True)
        assert st.converged == 0 and st.iterations == 1
        with pytest.raises(fde.FDEError) as e:
            fde.fde_solve(h, B, x)
        assert e.value.code == fde.FDE_ERR_NOT_CONVERGED
        Bn = B.clone()
        Bn[3, 4] = float("nan")
        with pytest.raises(fde.FDEError) as e:
            fde.fde_solve(h, Bn, x)
        assert e.value.code == fde.FDE_ERR_NONFINITE
        with pytest.raises(fde.FDEError) as e:
            fde.fde_apply(h, B, B)
        assert e.value.code == fde.FDE_ERR_ARG
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precond,precision,path", [
    (fde.FDE_PRECOND_MG_SG, fde.FDE_PREC_FP32, fde.FDE_PATH_AUTO),
    (fde.FDE_PRECOND_MG_SG, fde.FDE_PREC_BF16X3, fde.FDE_PATH_GEMM),
    (fde.FDE_PRECOND_MG_REDISC, fde.FDE_PREC_FP64, fde.FDE_PATH_AUTO),
    (fde.FDE_PRECOND_P2, fde.FDE_PREC_FP32, fde.FDE_PATH_AUTO)])
@pytest.mark.parametrize("cycles", [1, 2])
def test_graph_replay_equals_eager_cycle(precond, precision, path, cycles):
    # the V-cycle is captured into a CUDA graph on first use and replayed;
    # with kernel profiling on it runs eagerly: all runs give identical bits
    import torch
    case = Case(inputs.perturbed_power_law(), 255, precond=precond, precision=precision,
                toeplitz_path=path, cycles=cycles)
    h = case.handle()
    try:
        R = dev(np.random.default_rng(9).standard_normal((255, 255)))
        outs = []
        for prof in (0, 0, 1, 0):
            fde.fde_profile_enable(h, prof)
            z = torch.empty_like(R)
            fde.fde_vcycle(h, R, z)
            torch.cuda.synchronize()
            outs.append(host(z))
        for o in outs[1:]:
            np.testing.assert_array_equal(o, outs[0])
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precision,path", [(fde.FDE_PREC_FP32, fde.FDE_PATH_AUTO),
                                            (fde.FDE_PREC_BF16X3, fde.FDE_PATH_GEMM)])
def test_relaxed_matvec_meets_the_same_true_residual(precision, path):
    # with relax = 1 the late Krylov matvecs run in FP32; the oracle's FP64
    # true residual of the result still meets rtol, and the iteration count
    # stays within one of the exact-matvec solve
    import torch
    its = {}
    for relax in (1, 0):
        case = Case(inputs.perturbed_power_law(), 255, precision=precision, toeplitz_path=path,
                    outer=fde.FDE_OUTER_DF32, rtol=1e-10, relax=relax)
        h = case.handle()
        try:
            B = case.oracle_rhs()
            x = torch.empty_like(dev(B))
            st = fde.fde_solve(h, dev(B), x)
            res = np.linalg.norm(B - case.oracle_apply(host(x))) / np.linalg.norm(B)
            assert st.converged == 1 and res <= 1.05e-10, (relax, res)
            its[relax] = st.iterations
            if relax:
                assert st.relaxed > 0
            else:
                assert st.relaxed == 0
        finally:
            fde.fde_destroy(h)
    assert its[1] <= its[0] + 1, its


@pytest.mark.parametrize("precision,tol", [(fde.FDE_PREC_FP64, 1), (fde.FDE_PREC_FP32, 2)])
@pytest.mark.parametrize("precond", [fde.FDE_PRECOND_MG_SG, fde.FDE_PRECOND_P2])
def test_multigrid_solver_matches_oracle(precision, tol, precond):
    # multigrid as the solver: x <- x + V(b - M x) until the true residual meets
    # rtol; the oracle's stationary iteration needs the same number of cycles
    import torch
    from oracle.krylov import mg_solve
    from oracle import multigrid as mg
    case = Case(inputs.perturbed_power_law(), 127, precond=precond, precision=precision,
                solver=fde.FDE_SOLVER_MG, rtol=1e-9, maxit=400)
    h = case.handle()
    try:
        B = case.oracle_rhs()
        x = torch.empty_like(dev(B))
        st = fde.fde_solve(h, dev(B), x)
        res = np.linalg.norm(B - case.oracle_apply(host(x))) / np.linalg.norm(B)
        assert st.converged == 1 and res <= 1.05e-9, res
        hier = case.oracle_hierarchy()
        xo, cyc, rel, ok = mg_solve(case.oracle_apply, B, lambda R: mg.vcycle(hier, R), 1e-9, 400)
        assert ok and abs(st.iterations - cyc) <= tol, (st.iterations, cyc)
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("solver", [fde.FDE_SOLVER_FGMRES, fde.FDE_SOLVER_MG])
def test_warm_start_step(solver):
    # warm = 1 starts each step's solve from u^(m-1): fewer iterations, the
    # same true-residual tolerance (checked by the oracle's FP64 operator)
    import torch
    counts = {}
    for warm in (0, 1):
        case = Case(inputs.perturbed_power_law(), 127, precision=fde.FDE_PREC_FP32,
                    solver=solver, warm=warm, rtol=1e-9, maxit=400)
        h = case.handle()
        try:
            B = case.oracle_rhs()
            u0 = dev(case.u0)
            x = torch.empty_like(u0)
            st = fde.fde_step(h, u0, dev(case.v), x)
            res = np.linalg.norm(B - case.oracle_apply(host(x))) / np.linalg.norm(B)
            assert st.converged == 1 and res <= 1.05e-9, (warm, res)
            counts[warm] = st.iterations
        finally:
            fde.fde_destroy(h)
    assert counts[1] < counts[0], counts


@pytest.mark.parametrize("precision", [fde.FDE_PREC_FP64, fde.FDE_PREC_FP32])
def test_time_dependent_coefficients_example2(precision):
    # Example 2 (Sec. 5.2): coefficients change every step, so every step sets
    # both coefficient levels and rebuilds the multigrid hierarchy on the
    # device; the whole time loop (M = n = 31 steps to T = 1) follows the
    # oracle's time loop step by step, and the final error against the exact
    # solution equals the oracle's
    import torch
    from oracle import timeloop
    prob = inputs.example2()
    n = 31
    ref = timeloop.run(prob, n, precond="sg", rtol=1e-12, record=True)
    case = Case(prob, n, dt=1.0 / n, precision=precision, rtol=1e-10)
    h = fde.fde_create(case.params)
    try:
        X, Y, hx, hy = prob.grid(n, n)
        dt = 1.0 / n
        ud = dev(prob.exact(X, Y, 0.0))
        un = torch.empty_like(ud)
        for m in range(1, n + 1):
            cold = [dev(f) for f in prob.coefficients(X, Y, (m - 1) * dt)]
            cnew = [dev(f) for f in prob.coefficients(X, Y, m * dt)]
            fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *cold)
            fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *cnew)
            st = fde.fde_step(h, ud, dev(prob.source(X, Y, (m - 0.5) * dt)), un)
            assert st.converged == 1
            ug = host(un)
            Uo = ref["history"][m - 1]
            assert np.linalg.norm(ug - Uo) <= 1e-8 * np.linalg.norm(Uo), m
            ud, un = un, ud
        err = np.max(np.abs(prob.exact(X, Y, 1.0) - host(ud)))
        np.testing.assert_allclose(err, ref["error_inf"], rtol=1e-6)
    finally:
        fde.fde_destroy(h)


def test_structured_galerkin_levels_equal_exact_galerkin_for_constant_coefficients():
    # the paper's tilde-P_MGM (exact Galerkin P^T A P at every level): for
    # constant coefficients the structured-Galerkin hierarchy the GPU builds
    # is exactly that, so every GPU level operator matches the oracle's dense
    # triple products
    import torch
    from oracle import multigrid as mg
    from oracle.operator import assemble_M, toeplitz_A
    n = 31
    case = Case(inputs.constant_unit(), n)
    h = case.handle()
    try:
        K0 = assemble_M(toeplitz_A(case.wx, n), toeplitz_A(case.wy, n), case.sc["c"],
                        case.sc["sigma"], *case.coef_new)
        hier = mg.exact_galerkin(K0, n, n)
        assert [(L.n1, L.n2) for L in hier.levels] == fde.fde_levels(h)
        rng = np.random.default_rng(33)
        for l, lev in enumerate(hier.levels):
            Xl = rng.standard_normal((lev.n2, lev.n1))
            yl = torch.empty_like(dev(Xl))
            fde.fde_level_apply(h, l, dev(Xl), yl)
            torch.cuda.synchronize()
            rl = lev.apply(Xl)
            assert np.max(np.abs(host(yl) - rl)) <= 1e-12 * np.max(np.abs(rl)), l
    finally:
        fde.fde_destroy(h)


_POISON_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + '/tests')
from paper_1706_06844_gb300 import fde, inputs
from gpu_util import Case, dev, host
out = []
for kw in (dict(precision=fde.FDE_PREC_FP32), dict(precision=fde.FDE_PREC_BF16X3,
           toeplitz_path=fde.FDE_PATH_GEMM, relax=1, outer=fde.FDE_OUTER_DF32),
           dict(precond=fde.FDE_PRECOND_P2, precision=fde.FDE_PREC_FP32)):
    case = Case(inputs.perturbed_power_law(), 255, rtol=1e-10, **kw)
    h = case.handle()
    B = dev(case.oracle_rhs()); x = torch.empty_like(B)
    fde.fde_solve(h, B, x); fde.fde_destroy(h)
    out.append(host(x))
np.save(sys.argv[2], np.stack(out))
"""


def test_poisoned_workspace_changes_nothing(tmp_path):
    # FDE_POISON=1 fills every workspace buffer with NaN bit patterns when it
    # is allocated: a kernel reading memory that nothing wrote first would turn
    # the solution into NaN or change it; the poisoned solves (in a child
    # process, where the option is read at the first allocation) give the same
    # bits as unpoisoned ones
    import os
    import subprocess
    import sys
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    path = str(tmp_path / "poisoned.npy")
    env = dict(os.environ, FDE_POISON="1")
    r = subprocess.run([sys.executable, "-c", _POISON_CHILD, root, path], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    poisoned = np.load(path)
    assert np.all(np.isfinite(poisoned))
    for k, kw in enumerate((dict(precision=fde.FDE_PREC_FP32),
                            dict(precision=fde.FDE_PREC_BF16X3, toeplitz_path=fde.FDE_PATH_GEMM,
                                 relax=1, outer=fde.FDE_OUTER_DF32),
                            dict(precond=fde.FDE_PRECOND_P2, precision=fde.FDE_PREC_FP32))):
        case = Case(inputs.perturbed_power_law(), 255, rtol=1e-10, **kw)
        h = case.handle()
        try:
            B = dev(case.oracle_rhs())
            x = torch.empty_like(B)
            fde.fde_solve(h, B, x)
            np.testing.assert_array_equal(host(x), poisoned[k])
        finally:
            fde.fde_destroy(h)

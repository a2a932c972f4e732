"""fde_apply_noalloc: the operator apply for callers that cannot allocate
device memory (their device heap belongs to another runtime's pool, so they
cannot create a solver handle).  It must reproduce the handle-based fde_apply
on two calls in a row, since every call reuses the same fixed device array,
and both must agree with the FP64 oracle's Eq. (M) under the outer-apply
parity bound.

Collected last on purpose (file name), so a failure here stops a -x run only
after every other test has run."""
import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import Case, dev, host, sampled_apply, sample_lines

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("n1,n2", [(63, 63), (255, 127)])
def test_noalloc_apply_matches_handle_apply_and_oracle(n1, n2):
    import torch
    case = Case(inputs.perturbed_power_law(), n1, n2)
    h = case.handle()
    try:
        rng = np.random.default_rng(21)
        X = rng.standard_normal((n2, n1))
        xd = dev(X)
        ref = torch.empty_like(xd)
        fde.fde_apply(h, xd, ref)
        torch.cuda.synchronize()
        ref_h = host(ref)
        # same tolerance as the outer-apply parity test: 64 eps times the
        # absolute sums |c||x| + |D||A||x| + ..., against the oracle's Eq. (M)
        # and against the handle's apply
        bound = 64 * EPS * case.oracle_abs_apply(X)
        oracle = case.oracle_apply(X)
        assert np.all(np.abs(ref_h - oracle) <= bound)
        for call in range(2):
            y = torch.full_like(xd, float("nan"))
            fde.fde_apply_noalloc(case.params, *case.dnew, xd, y)
            torch.cuda.synchronize()
            assert np.all(np.abs(host(y) - ref_h) <= bound), call
            assert np.all(np.abs(host(y) - oracle) <= bound), call
    finally:
        fde.fde_destroy(h)


def _check_sampled(case, X, yh, rng):
    """Sampled rows and columns of the oracle's Eq. (M) against yh, with the
    normwise FFT bound c u log2 L (|M||x|_i + rms |M||x|), c = 8 (the n = 4095
    outer-apply test's bound; at n <= 255 the elementwise 64 u bound holds)."""
    from oracle.operator import toeplitz_A
    n1, n2 = case.n1, case.n2
    Ax, Ay = toeplitz_A(case.wx, n1), toeplitz_A(case.wy, n2)
    rows, cols = sample_lines(n2, 16, rng), sample_lines(n1, 16, rng)
    R, Ra, C, Ca = sampled_apply(Ax, Ay, case.sc["c"], case.sc["sigma"], *case.coef_new, X,
                                 rows, cols)
    logL = int(np.ceil(np.log2(2 * max(n1, n2) - 1)))
    rms = np.sqrt(np.mean(np.concatenate([Ra.ravel(), Ca.ravel()]) ** 2))
    for got, ref, ab in [(yh[rows], R, Ra), (yh[:, cols], C, Ca)]:
        bound = 8 * logL * EPS * (ab + rms)
        err = np.abs(got - ref)
        assert np.all(err <= bound), float(np.max(err / bound))


def test_noalloc_alternating_sizes_up_to_the_limit():
    # the largest grids the fixed array serves (2048 points on one axis: FFT
    # length 4096 fills the spectra and twiddle blocks) alternating with a
    # small one, so data left in the shared array by a larger call would show
    import torch
    prob = inputs.perturbed_power_law()
    rng = np.random.default_rng(2048)
    for n1, n2 in [(2048, 2047), (63, 63), (2047, 2048), (63, 63)]:
        case = Case(prob, n1, n2)
        X = rng.standard_normal((n2, n1))
        xd = dev(X)
        cf = [dev(f) for f in case.coef_new]
        y = torch.full_like(xd, float("nan"))
        fde.fde_apply_noalloc(case.params, *cf, xd, y)
        torch.cuda.synchronize()
        yh = host(y)
        assert np.all(np.isfinite(yh))
        if n1 <= 255:
            bound = 64 * EPS * case.oracle_abs_apply(X)
            assert np.all(np.abs(yh - case.oracle_apply(X)) <= bound)
        else:
            _check_sampled(case, X, yh, rng)


def test_noalloc_rejects_oversized_grid_and_overlap():
    import torch
    p = fde.params(n1=2049, n2=63)
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(fde.FDEError) as e:
        fde.fde_apply_noalloc(p, z, z, z, z, z, z[1:])
    assert e.value.code == fde.FDE_ERR_ARG and "2048" in str(e.value)
    # y overlapping an input in part is rejected before any launch
    q = fde.params(n1=7, n2=7)
    buf = torch.zeros(2 * 49, dtype=torch.float64, device="cuda")
    cf = torch.ones(49, dtype=torch.float64, device="cuda")
    with pytest.raises(fde.FDEError) as e:
        fde.fde_apply_noalloc(q, cf, cf, cf, cf, buf[:49], buf[10:59])
    assert e.value.code == fde.FDE_ERR_ARG and "overlap" in str(e.value)

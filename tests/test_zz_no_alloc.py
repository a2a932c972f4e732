"""fde_apply_noalloc: the operator apply for callers that cannot allocate
device memory (their device heap belongs to another runtime's pool, so they
cannot create a solver handle).  It must reproduce the handle-based fde_apply
on two calls in a row, since every call reuses the same fixed device array.

Collected last on purpose (file name), so a failure here stops a -x run only
after every other test has run."""
import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import Case, dev, host

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("n1,n2", [(63, 63), (255, 127)])
def test_noalloc_apply_matches_handle_apply(n1, n2):
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
        # absolute sums |c||x| + |D||A||x| + ...
        bound = 64 * EPS * case.oracle_abs_apply(X)
        for call in range(2):
            y = torch.full_like(xd, float("nan"))
            fde.fde_apply_noalloc(case.params, *case.dnew, xd, y)
            torch.cuda.synchronize()
            assert np.all(np.abs(host(y) - ref_h) <= bound), call
    finally:
        fde.fde_destroy(h)


def test_noalloc_rejects_oversized_grid():
    import torch
    p = fde.params(n1=2049, n2=63)
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(fde.FDEError) as e:
        fde.fde_apply_noalloc(p, z, z, z, z, z, z[1:])
    assert e.value.code == fde.FDE_ERR_ARG and "2048" in str(e.value)

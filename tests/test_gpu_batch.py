"""Batches of independent problems (mixed sizes, orders, WSGD shifts and
coefficient fields) stepped concurrently through fde_batch_step: every
problem's result equals, bit for bit, the same step taken alone on its own
handle, and agrees with the oracle's solve."""
import numpy as np
import pytest

from paper_1706_06844_gb300 import inputs
from paper_1706_06844_gb300 import fde
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    fde.lib()


def _setup(problems, **kw):
    out = []
    for n, pb in problems:
        X, Y, hx, hy = pb.grid(n, n)
        a1, b1, a2, b2 = pb.domain
        p = fde.params(alpha=pb.alpha, beta=pb.beta, qx=pb.qx, qy=pb.qy, a1=a1, b1=b1, a2=a2,
                       b2=b2, n1=n, n2=n, dt=hx, **kw)
        out.append(dict(n=n, pb=pb, X=X, Y=Y, dt=hx, params=p,
                        coef=[dev(f) for f in pb.coefficients(X, Y, 0.0)],
                        u0=dev(pb.exact(X, Y, 0.0))))
    return out


def _source(d, m):
    return dev(d["pb"].source(d["X"], d["Y"], (m - 0.5) * d["dt"]))


def test_batch_equals_single_handles_and_oracle():
    import torch
    probs = _setup(inputs.random_batch(10, sizes=(63, 127, 255)), precision=fde.FDE_PREC_FP32,
                   rtol=1e-10)
    b = fde.fde_batch_create([d["params"] for d in probs])
    singles = []
    try:
        assert fde.fde_batch_size(b) == len(probs)
        for i, d in enumerate(probs):
            h = fde.fde_batch_handle(b, i)
            fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *d["coef"])
            fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *d["coef"])
        u = [d["u0"].clone() for d in probs]
        nxt = [torch.empty_like(x) for x in u]
        for m in (1, 2):
            v = [_source(d, m) for d in probs]
            stats = fde.fde_batch_step(b, u, v, nxt)
            torch.cuda.synchronize()
            assert all(s.converged == 1 for s in stats)
            if m == 1:
                first = [host(x).copy() for x in nxt]
            u, nxt = nxt, u
        # every problem alone on a handle of its own: identical bits
        for i, d in enumerate(probs):
            h = fde.fde_create(d["params"])
            singles.append(h)
            fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *d["coef"])
            fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *d["coef"])
            x = torch.empty_like(d["u0"])
            fde.fde_step(h, d["u0"], _source(d, 1), x)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(host(x), first[i])
        # and the oracle's solve of the first step of two problems
        from oracle.operator import cn_scalars, rhs, apply_M
        from oracle.wsgd import wsgd_weights
        from oracle.krylov import fgmres
        for i in (0, len(probs) - 1):
            d = probs[i]
            n, pb = d["n"], d["pb"]
            wx = wsgd_weights(pb.alpha, n + 1, 1, pb.qx)
            wy = wsgd_weights(pb.beta, n + 1, 1, pb.qy)
            sc = cn_scalars(pb.alpha, pb.beta, d["dt"], d["dt"], d["dt"])
            cf = pb.coefficients(d["X"], d["Y"], 0.0)
            B = rhs(host(d["u0"]), wx, wy, sc["c"], sc["sigma"], *cf,
                    host(_source(d, 1)), d["dt"], pb.alpha)
            A = lambda Z: apply_M(Z, wx, wy, sc["c"], sc["sigma"], *cf)
            res = np.linalg.norm(B - A(first[i])) / np.linalg.norm(B)
            assert res <= 1.05e-10, (i, res)
            from oracle import multigrid as mg
            hier = mg.structured_galerkin(wx, wy, n, n, sc["c"], sc["sigma"], cf, 8)
            xo, its, rel, ok = fgmres(A, B, lambda R: mg.vcycle(hier, R), 30, 1e-12)
            assert np.linalg.norm(first[i] - xo) <= 1e-6 * np.linalg.norm(xo)
    finally:
        for h in singles:
            fde.fde_destroy(h)
        fde.fde_batch_destroy(b)


def test_batch_reports_each_problem_status():
    # one problem capped at a single iteration: it reports NOT_CONVERGED, the
    # others are unaffected and the call returns the first failing status
    import torch
    probs = _setup(inputs.random_batch(4, sizes=(63,)), rtol=1e-10)
    probs[2]["params"].maxit = 1
    b = fde.fde_batch_create([d["params"] for d in probs])
    try:
        for i, d in enumerate(probs):
            h = fde.fde_batch_handle(b, i)
            fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *d["coef"])
            fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *d["coef"])
        u = [d["u0"] for d in probs]
        nxt = [torch.empty_like(x) for x in u]
        v = [_source(d, 1) for d in probs]
        with pytest.raises(fde.FDEError) as e:
            fde.fde_batch_step(b, u, v, nxt)
        assert e.value.code == fde.FDE_ERR_NOT_CONVERGED
        assert "problem 2" in str(e.value)
        st = [fde.fde_batch_status(b, i) for i in range(4)]
        assert st == [fde.FDE_OK, fde.FDE_OK, fde.FDE_ERR_NOT_CONVERGED, fde.FDE_OK]
        stats = fde.fde_batch_step(b, u, v, nxt, allow_not_converged=True)
        assert stats[2].iterations == 1 and stats[0].converged == 1
    finally:
        fde.fde_batch_destroy(b)

"""Batches of independent problems (mixed sizes, orders, WSGD shifts and
coefficient fields) stepped through fde_batch_step.

Worker-thread engine (FDE_BATCH_ENGINE=threads): every problem's result
equals, bit for bit, the same step taken alone on its own handle.  Grouped
engine (the default for FP32 V-cycles): every stage of all problems' solves
is one launch and the FGMRES iterations run in lockstep, so the reductions are
partitioned differently from a lone handle: per problem the iteration count is
within 1 of the lone handle's, the solution within the solve's tolerance of
it, and the oracle's true residual meets rtol.  Both agree with the oracle's
solve."""
import contextlib
import os

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


@contextlib.contextmanager
def _engine(name):
    old = os.environ.get("FDE_BATCH_ENGINE")
    if name is None:
        os.environ.pop("FDE_BATCH_ENGINE", None)
    else:
        os.environ["FDE_BATCH_ENGINE"] = name
    try:
        yield
    finally:
        if old is None:
            os.environ.pop("FDE_BATCH_ENGINE", None)
        else:
            os.environ["FDE_BATCH_ENGINE"] = old


def _oracle_residual(d, u_prev, u_next, m):
    from oracle.operator import cn_scalars, rhs, apply_M
    from oracle.wsgd import wsgd_weights
    n, pb = d["n"], d["pb"]
    wx = wsgd_weights(pb.alpha, n + 1, 1, pb.qx)
    wy = wsgd_weights(pb.beta, n + 1, 1, pb.qy)
    sc = cn_scalars(pb.alpha, pb.beta, d["dt"], d["dt"], d["dt"])
    cf = pb.coefficients(d["X"], d["Y"], 0.0)
    B = rhs(u_prev, wx, wy, sc["c"], sc["sigma"], *cf, host(_source(d, m)), d["dt"], pb.alpha)
    return np.linalg.norm(B - apply_M(u_next, wx, wy, sc["c"], sc["sigma"], *cf)) / \
        np.linalg.norm(B)


def _run_batch(probs, steps, engine):
    """Steps of the batch; returns (engine used, per-step solutions, stats)."""
    import torch
    with _engine(engine):
        b = fde.fde_batch_create([d["params"] for d in probs])
        try:
            for i, d in enumerate(probs):
                h = fde.fde_batch_handle(b, i)
                fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *d["coef"])
                fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *d["coef"])
            u = [d["u0"].clone() for d in probs]
            nxt = [torch.empty_like(x) for x in u]
            sols, stats = [], []
            for m in range(1, steps + 1):
                v = [_source(d, m) for d in probs]
                st = fde.fde_batch_step(b, u, v, nxt, allow_not_converged=True)
                torch.cuda.synchronize()
                sols.append([host(x).copy() for x in nxt])
                stats.append(st)
                u, nxt = nxt, u
            return fde.fde_batch_engine(b), sols, stats
        finally:
            fde.fde_batch_destroy(b)


def _single(d, steps):
    import torch
    h = fde.fde_create(d["params"])
    try:
        fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *d["coef"])
        fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *d["coef"])
        u, x = d["u0"].clone(), torch.empty_like(d["u0"])
        sols, its = [], []
        for m in range(1, steps + 1):
            st = fde.fde_step(h, u, _source(d, m), x)
            torch.cuda.synchronize()
            sols.append(host(x).copy())
            its.append(st.iterations)
            u, x = x, u
        return sols, its
    finally:
        fde.fde_destroy(h)


@pytest.mark.parametrize("precond", [fde.FDE_PRECOND_MG_SG, fde.FDE_PRECOND_MG_REDISC])
@pytest.mark.parametrize("relax", [0, 1])
def test_grouped_engine_matches_single_handles_and_oracle(precond, relax):
    # mixed sizes (odd and, for the rediscretised cycle, even), orders and
    # shifts; two steps of the time loop through the grouped engine
    sizes = (63, 127, 255) if precond == fde.FDE_PRECOND_MG_SG else (63, 64, 128, 255)
    probs = _setup(inputs.random_batch(12, sizes=sizes), precision=fde.FDE_PREC_FP32,
                   outer=fde.FDE_OUTER_DF32, precond=precond, relax=relax, rtol=1e-10)
    eng, sols, stats = _run_batch(probs, 2, None)
    assert eng == 1  # the grouped engine ran
    for i, d in enumerate(probs):
        ref, its = _single(d, 2)
        for m in range(2):
            st = stats[m][i]
            assert st.converged == 1, (i, m)
            assert abs(st.iterations - its[m]) <= 1, (i, m, st.iterations, its[m])
            x = sols[m][i]
            assert np.linalg.norm(x - ref[m]) <= 1e-7 * np.linalg.norm(ref[m]), (i, m)
            prev = host(d["u0"]) if m == 0 else sols[0][i]
            assert _oracle_residual(d, prev, x, m + 1) <= 1.05e-10, (i, m)


def test_grouped_engine_restarts_and_caps():
    # restart length 4: several restart cycles per step (the batch's restart
    # graph replays); one problem capped at 3 iterations reports
    # NOT_CONVERGED with its last iterate while the others converge
    import torch
    probs = _setup(inputs.random_batch(6, sizes=(63, 127)), precision=fde.FDE_PREC_FP32,
                   outer=fde.FDE_OUTER_DF32, restart=4, rtol=1e-9, maxit=500)
    probs[3]["params"].maxit = 3
    eng, sols, stats = _run_batch(probs, 1, None)
    assert eng == 1
    for i, d in enumerate(probs):
        st = stats[0][i]
        if i == 3:
            assert st.converged == 0 and st.iterations == 3
            continue
        assert st.converged == 1 and st.restarts >= 2, (i, st.restarts)
        assert _oracle_residual(d, host(d["u0"]), sols[0][i], 1) <= 1.05e-9
        ref, its = _single(d, 1)
        assert abs(st.iterations - its[0]) <= 1


def test_grouped_engine_is_deterministic():
    # the same batch twice: identical bits (fixed-order reductions)
    probs = _setup(inputs.random_batch(8, sizes=(63, 127, 255)), precision=fde.FDE_PREC_FP32,
                   outer=fde.FDE_OUTER_DF32, relax=1, rtol=1e-10)
    _, a, _ = _run_batch(probs, 1, None)
    _, b, _ = _run_batch(probs, 1, None)
    for x, y in zip(a[0], b[0]):
        np.testing.assert_array_equal(x, y)


def test_grouped_engine_declines_other_configurations():
    # an FP64 V-cycle is not served by the grouped engine: worker threads run it
    probs = _setup(inputs.random_batch(3, sizes=(63,)), precision=fde.FDE_PREC_FP64, rtol=1e-9)
    eng, sols, stats = _run_batch(probs, 1, None)
    assert eng == 2 and all(s.converged for s in stats[0])


def test_batch_equals_single_handles_and_oracle():
    import torch
    probs = _setup(inputs.random_batch(10, sizes=(63, 127, 255)), precision=fde.FDE_PREC_FP32,
                   rtol=1e-10)
    os.environ["FDE_BATCH_ENGINE"] = "threads"
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
        os.environ.pop("FDE_BATCH_ENGINE", None)
        for h in singles:
            fde.fde_destroy(h)
        fde.fde_batch_destroy(b)


@pytest.mark.parametrize("engine", ["threads", None])
def test_batch_reports_each_problem_status(engine):
    # one problem capped at a single iteration: it reports NOT_CONVERGED, the
    # others are unaffected and the call returns the first failing status
    # (both engines; the default configuration here is the grouped one's)
    import torch
    ctx = _engine(engine)
    ctx.__enter__()
    probs = _setup(inputs.random_batch(4, sizes=(63,)), rtol=1e-10, precision=fde.FDE_PREC_FP32,
                   outer=fde.FDE_OUTER_DF32)
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
        ctx.__exit__(None, None, None)

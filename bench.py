"""Benchmark: CN-WSGD time steps per second at n = 2047 (rtol 1e-8).

One bench step is one CN-WSGD time step (Eq. CNWSGD): the right-hand side
b^(m) and the FGMRES(30) solve of M^(m) u^(m) = b^(m) preconditioned by one
structured-Galerkin V-cycle, on the 2047 x 2047 grid of the perturbed
power-law workload (alpha = 1.5, beta = 1.7, WSGD (1,-1), smooth seeded
coefficient perturbation of amplitude 0.2, dt = h, manufactured bubble
solution).  The timed region holds W warm-up steps' successors: K consecutive
steps of the time loop with every input already resident in HBM.

The headline solver is mixed precision: FP64 Krylov vectors with
double-float matvecs until the FGMRES residual estimate is within 1e4 x of
the target, FP32 matvecs after that (the exit test is the double-float true
residual, so the tolerance met is unchanged), and a V-cycle whose level-0
products run on the tensor cores in BF16x3.  Reported beside it: the same
solver with every matvec double-float (`exact_matvec`), the same steps with
the plain FP64 solver, an end-to-end figure
through fde_step_host (host arrays, copies inside the timed region), the
roofline of the dominant kernel (timed with CUDA events on the library's
stream), sampled SM clocks, and the CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun) every rank runs an independent replica of the
workload (the solve does not shard across GPUs); value aggregates all ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 2047
RESTART = 30
RTOL = 1e-8
METRIC = "CN-WSGD time steps/s at n=2047, rtol 1e-8: mixed-precision MG-GMRES vs FP64"
WORKLOAD = ("perturbed power-law coefficients, n=2047, alpha=1.5, beta=1.7, WSGD (1,-1), "
            "dt=h, FGMRES(30) + structured-Galerkin V-cycle, rtol 1e-8")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# FP64 issue rate of GB300: 2 FMA per SM per clock (nominal 1.25 TFLOP/s)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07  # = 1258.6 GFLOP/s at the 2070 MHz maximum clock
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07  # = 80 548 GFLOP/s (FMA = 2 flops)
FP32_ISSUE_TOPS = 152 * 128 * 2.07 / 1e3  # = 40.3 T FP32 instructions/s
TRAFFIC_DF32_PASS = 100.882688e6 + 13.245184e6  # dram__bytes_read.sum + dram__bytes_write.sum


def problem():
    from paper_1706_06844_gb300 import inputs
    return inputs.perturbed_power_law(alpha=1.5, beta=1.7, seed=1706068, amplitude=0.2)


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class Workload:
    """Device-resident inputs of the time loop and one solver handle."""

    def __init__(self, precision, path=None, outer=None, precond=None, cycles=1, relax=0,
                 solver=0, warm=0):
        import torch
        from paper_1706_06844_gb300 import fde
        self.fde, self.torch = fde, torch
        prob = problem()
        n = N_GRID
        X, Y, hx, hy = prob.grid(n, n)
        self.prob, self.X, self.Y, self.dt = prob, X, Y, hx
        a1, b1, a2, b2 = prob.domain
        kw = dict(alpha=prob.alpha, beta=prob.beta, qx=prob.qx, qy=prob.qy, a1=a1, b1=b1,
                  a2=a2, b2=b2, n1=n, n2=n, dt=self.dt, rtol=RTOL, restart=RESTART, maxit=2000,
                  precond=fde.FDE_PRECOND_MG_SG if precond is None else precond,
                  precision=precision, cycles=cycles, relax=relax, solver=solver, warm=warm)
        if path is not None:
            kw["toeplitz_path"] = path
        if outer is not None:
            kw["outer"] = outer
        d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
        coef = [d(f) for f in prob.coefficients(X, Y, 0.0)]  # time-independent coefficients
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.h = fde.fde_create(fde.params(**kw))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        # the NEW coefficients build the multigrid hierarchy (and tune the level paths)
        fde.fde_set_coefficients(self.h, fde.FDE_COEF_NEW, *coef)
        fde.fde_set_coefficients(self.h, fde.FDE_COEF_OLD, *coef)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        self.setup_ms = {"create_ms": round((t1 - t0) * 1e3, 2),
                         "set_coefficients_ms": round((t2 - t1) * 1e3, 2)}
        self.u = [d(prob.exact(X, Y, 0.0)), torch.empty((n, n), dtype=torch.float64, device="cuda")]
        self.vsrc = {}
        self.m = 0
        self.first = None
        self.d = d

    def source(self, m):
        if m not in self.vsrc:
            self.vsrc[m] = self.d(self.prob.source(self.X, self.Y, (m - 0.5) * self.dt))
        return self.vsrc[m]

    def step(self):
        self.m += 1
        st = self.fde.fde_step(self.h, self.u[0], self.source(self.m), self.u[1])
        self.u.reverse()
        if self.m == 1:  # kept for the accuracy check against the oracle
            self.first = self.u[0].cpu().numpy()
        return st

    def close(self):
        self.fde.fde_destroy(self.h)


def time_steps(w, steps, warmup, dist):
    import torch
    for i in range(warmup):
        if i == 0 and w.m == 0:
            # the first step also captures the V-cycle's CUDA graph
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            w.step()
            torch.cuda.synchronize()
            w.setup_ms["first_step_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        else:
            w.step()
    for m in range(w.m + 1, w.m + steps + 1):
        w.source(m)  # sources resident before the timed region
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = w.fde.fde_launch_count(w.h)
    its = []
    ev0.record(stream)
    t0 = time.perf_counter()
    for _ in range(steps):
        its.append(w.step().iterations)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    return ms, wall, its, w.fde.fde_launch_count(w.h) - l0


def e2e_steps(w, steps):
    """Same steps through fde_step_host: pinned host arrays in, host array out."""
    import torch
    n = N_GRID
    u_host = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    u_host.copy_(w.u[0].cpu())
    out = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    srcs = []
    for m in range(w.m + 1, w.m + steps + 1):
        s = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        s.copy_(torch.from_numpy(w.prob.source(w.X, w.Y, (m - 0.5) * w.dt)))
        srcs.append(s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in srcs:
        w.fde.fde_step_host(w.h, u_host.data_ptr(), s.data_ptr(), out.data_ptr())
        u_host, out = out, u_host
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nbytes = n * n * 8
    return steps / dt, 2 * nbytes, nbytes


def fft_pass_work(n, outer):
    """Algorithmic work of one outer-apply pass (all rows or all columns): per
    pair of grid vectors one forward and two inverse complex FFTs of length L
    (radix-2^2: per group of 4 points 3 complex multiplies and 8 complex
    additions per two stages) and two complex spectral products per point.
    FP64: real flops (complex multiply 6, complex add 2).  Double-float: the
    FP32 operations of the double-float formulas used (complex multiply as two
    fused two-product dot products, 2 x 19; complex add as two double-float
    additions, 2 x 11), each operation one FP32 instruction."""
    L = 1 << (2 * n - 2).bit_length()
    logL = L.bit_length() - 1
    cm, ca = (6, 2) if outer == "fp64" else (38, 22)
    groups = (logL // 2) * (L // 4)
    fft = groups * (3 * cm + 8 * ca) + (L // 2 if logL % 2 else 0) * (cm + 2 * ca)
    return ((n + 1) // 2) * (3 * fft + 2 * cm * L)


def roofline(w, steps, outer):
    """Dominant kernel: the FP64-accurate outer Toeplitz apply (one launch = one
    FFT pass over all rows or all columns).  Timed with CUDA events on the
    library's stream over `steps` further time steps."""
    fde = w.fde
    fde.fde_profile_enable(w.h, 1)
    for _ in range(steps):
        w.step()
    res = {}
    for k, name in [(fde.FDE_KCLASS_OUTER_APPLY, "outer_apply"),
                    (fde.FDE_KCLASS_LEVEL_APPLY, "level_apply"),
                    (fde.FDE_KCLASS_KRYLOV, "krylov"), (fde.FDE_KCLASS_MG_OTHER, "mg_other"),
                    (fde.FDE_KCLASS_OUTER_FP32, "outer_apply_fp32")]:
        res[name] = fde.fde_profile_query(w.h, k)
    fde.fde_profile_enable(w.h, 0)
    work = fft_pass_work(N_GRID, outer)
    launches, ms = res["outer_apply"]
    avg_s = ms / max(launches, 1) * 1e-3
    achieved = work / avg_s / 1e12
    if outer == "fp64":
        peak, unit = FP64_PEAK_GFLOPS / 1e3, "TFLOP/s"
        kern = "fft_pass_kernel<double,double,double> (outer FP64 Toeplitz apply)"
        src = "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"
    else:
        peak, unit = FP32_ISSUE_TOPS, "T FP32-op/s"
        kern = "fft_pass_kernel<double,df,df> (outer double-float Toeplitz apply)"
        src = "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz (one instruction = one op)"
    total_ms = sum(v[1] for v in res.values())
    # DRAM bytes (read + write) of one row pass at n = 2047 from the ncu capture
    # summarised in profiles/fft_pass_df32_outer_apply_n2047.md (same kernel code)
    traffic = TRAFFIC_DF32_PASS if (outer == "df32" and N_GRID == 2047) else None
    return {"bound": "alu", "kernel": kern, "achieved": round(achieved, 3), "peak": round(peak, 2),
            "unit": unit, "frac": round(achieved / peak, 4), "peak_source": src,
            "traffic": traffic, "traffic_unit": "bytes per launch",
            "work_per_launch": work, "launches": launches,
            "avg_launch_ms": round(avg_s * 1e3, 4),
            "share_of_profiled_time": {k: round(v[1] / total_ms, 4) for k, v in res.items()}}


class OracleStep:
    """The FP64 oracle's CN step at the bench grid (right-hand side +
    FGMRES(30) with the structured-Galerkin V-cycle to rtol 1e-8), with the
    one-off set-up (weights, coefficients, hierarchy) done once and untimed."""

    def __init__(self):
        from oracle.wsgd import wsgd_weights
        from oracle.operator import cn_scalars, rhs_fft, apply_M_fft
        from oracle import multigrid as mg
        prob = problem()
        n = N_GRID
        X, Y, hx, hy = prob.grid(n, n)
        dt = hx
        wx = wsgd_weights(prob.alpha, n + 1, 1, prob.qx)
        wy = wsgd_weights(prob.beta, n + 1, 1, prob.qy)
        sc = cn_scalars(prob.alpha, prob.beta, hx, hy, dt)
        c, s = sc["c"], sc["sigma"]
        coef = prob.coefficients(X, Y, 0.0)
        hier = mg.structured_galerkin(wx, wy, n, n, c, s, coef)
        U = prob.exact(X, Y, 0.0)
        V = prob.source(X, Y, 0.5 * dt)
        self.rhs = lambda: rhs_fft(U, wx, wy, c, s, *coef, V, hx, prob.alpha)
        self.A = lambda Z: apply_M_fft(Z, wx, wy, c, s, *coef)
        self.prec = lambda R: mg.vcycle(hier, R)
        self.wall_s = 0.0  # timed wall and process CPU seconds (all threads)
        self.cpu_s = 0.0

    def threads_used(self):
        """Effective number of host threads of the timed work: process CPU
        time over wall time, at least 1."""
        return max(1, int(round(self.cpu_s / self.wall_s))) if self.wall_s > 0 else 1

    def full(self):
        """Time one whole step; returns (seconds, iterations, solution, rhs)."""
        from oracle.krylov import fgmres
        c0, t0 = time.process_time(), time.perf_counter()
        B = self.rhs()
        x, its, rel, ok = fgmres(self.A, B, self.prec, RESTART, RTOL)
        t = time.perf_counter() - t0
        self.wall_s += t
        self.cpu_s += time.process_time() - c0
        return t, its, x, B

    def sample(self, iters):
        """Time the right-hand side and the first `iters` FGMRES iterations
        (with the closing true residual); returns (rhs seconds, iteration
        seconds per iteration)."""
        from oracle.krylov import fgmres
        c0, t0 = time.process_time(), time.perf_counter()
        B = self.rhs()
        t1 = time.perf_counter()
        fgmres(self.A, B, self.prec, RESTART, RTOL, maxit=iters)
        t2 = time.perf_counter()
        self.wall_s += t2 - t0
        self.cpu_s += time.process_time() - c0
        return t1 - t0, (t2 - t1) / iters


def cpu_baseline_sample(refine=False):
    """The FP64 oracle as it stands, timed on this host: one whole CN step at
    the bench grid after an untimed set-up.  With refine, the oracle's solution
    is then driven on (untimed) to rtol 1e-12 and returned as the reference
    solution of step 1."""
    from oracle.krylov import fgmres
    o = OracleStep()
    t, its, x, B = o.full()
    threads = o.threads_used()
    if refine:
        xr, _, _, _ = fgmres(o.A, B, o.prec, RESTART, 1e-12, x0=x)
        return t, its, xr, threads
    return t, its, threads


def run_reference(args, rank):
    """The oracle as the reference arm: one whole step measures the step's
    iteration count; then every warm-up and timed step is a bounded sample --
    the right-hand side and the first 3 FGMRES iterations -- scaled to the
    whole step's iteration count, so K + W steps take a few minutes."""
    if rank != 0:
        return
    o = OracleStep()
    t_full, its_full, _, _ = o.full()
    sample_its = 3
    times = []
    for i in range(args.warmup + args.steps):
        t_rhs, t_it = o.sample(sample_its)
        if i >= args.warmup:
            times.append(t_rhs + t_it * its_full)
    total = sum(times)
    v = args.steps / total
    cores = o.threads_used()
    sample = (f"one whole CN step at n=2047 ({its_full} FGMRES iterations, {t_full:.1f} s); "
              f"then each step: the right-hand side + the first {sample_its} FGMRES(30)/SG "
              f"V-cycle iterations of the FP64 numpy oracle, scaled to {its_full} iterations")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_GRID, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": round(v, 5), "unit": "steps/s", "cores": cores,
                             "cores_available": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 5), "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "whole_step_s": round(t_full, 2), "iterations_per_step": [its_full]}
    print(json.dumps(line), flush=True)


def kernel_micro(kind, reps):
    """One kernel class in isolation at the bench grid, for profiler captures:
    gemm / fft32 = level-0 V-cycle products (BF16 tcgen05 GEMM / FP32 FFT),
    fft64 / fftdf = the outer apply (FP64 / double-float FFT)."""
    import torch
    from paper_1706_06844_gb300 import fde
    prec = {"gemm": fde.FDE_PREC_BF16, "gemm3": fde.FDE_PREC_BF16X3, "fft32": fde.FDE_PREC_FP32,
            "fft64": fde.FDE_PREC_FP64, "fftdf": fde.FDE_PREC_FP64}[kind]
    path = {"gemm": fde.FDE_PATH_GEMM, "gemm3": fde.FDE_PATH_GEMM,
            "fft32": fde.FDE_PATH_FFT}.get(kind)
    outer = fde.FDE_OUTER_DF32 if kind == "fftdf" else None
    w = Workload(prec, path=path, outer=outer)
    x = torch.randn((N_GRID, N_GRID), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    call = ((lambda: fde.fde_level_apply(w.h, 0, x, y)) if kind in ("gemm", "gemm3", "fft32")
            else (lambda: fde.fde_apply(w.h, x, y)))
    for _ in range(2):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"kernel": kind, "n": N_GRID, "reps": reps,
                      "ms_per_call": round(e0.elapsed_time(e1) / reps, 4)}))
    w.close()


BATCH_COUNT = 256
BATCH_METRIC = "CN-WSGD problem-steps/s, 256 independent problems (n in {63,127,255,511}), rtol 1e-8"
BATCH_WORKLOAD = ("256 problems, seed 1706069: n uniform over {63,127,255,511}, alpha, beta ~ "
                  "U(1.1,1.9), WSGD q in {0,-1} (-1 below gamma_0), coefficients exp(ln2 psi) in "
                  "[0.5,2] with psi a smooth seeded field, dt=h, FGMRES(30) + structured-Galerkin "
                  "FP32 V-cycle, double-float outer apply (relaxed matvec unless --relax 0), "
                  "rtol 1e-8")


def run_batch(args, rank, world, dist):
    """Every rank steps its share of the 256 problems (no data-path collective);
    value = all problem-steps of all ranks / the slowest rank's time."""
    import torch
    from paper_1706_06844_gb300 import fde, inputs, shard
    probs = inputs.random_batch(BATCH_COUNT)
    mine = shard.shard([shard.problem_cost(n, n) for n, _ in probs], rank, world)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    params, coef, u, base, dts = [], [], [], [], []
    for i in mine:
        n, pb = probs[i]
        X, Y, hx, hy = pb.grid(n, n)
        a1, b1, a2, b2 = pb.domain
        params.append(fde.params(alpha=pb.alpha, beta=pb.beta, qx=pb.qx, qy=pb.qy, a1=a1, b1=b1,
                                 a2=a2, b2=b2, n1=n, n2=n, dt=hx, rtol=RTOL, restart=RESTART,
                                 maxit=2000, precond=fde.FDE_PRECOND_MG_SG,
                                 precision=fde.FDE_PREC_FP32, outer=fde.FDE_OUTER_DF32,
                                 relax=args.relax))
        coef.append([d(f) for f in pb.coefficients(X, Y, 0.0)])
        u.append(d(pb.exact(X, Y, 0.0)))
        # time-independent coefficients: the manufactured source is exp(-t) v(0)
        base.append(d(pb.source(X, Y, 0.0)))
        dts.append(hx)
    b = fde.fde_batch_create(params)
    for k in range(len(mine)):
        h = fde.fde_batch_handle(b, k)
        fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *coef[k])
        fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *coef[k])
    total = args.warmup + args.steps
    src = [[base[k] * float(np.exp(-(m - 0.5) * dts[k])) for k in range(len(mine))]
           for m in range(1, total + 1)]
    nxt = [torch.empty_like(x) for x in u]
    its = []

    def step(m):
        nonlocal u, nxt
        st = fde.fde_batch_step(b, u, src[m - 1], nxt)
        its.append(sum(s.iterations for s in st))
        u, nxt = nxt, u

    for m in range(1, args.warmup + 1):
        step(m)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ev0.record()
        t0 = time.perf_counter()
        for m in range(args.warmup + 1, total + 1):
            step(m)
        ev1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    from paper_1706_06844_gb300 import shard as sh
    ms = sh.max_over_ranks(ev0.elapsed_time(ev1), dist)
    units = sh.sum_over_ranks(len(mine) * args.steps, dist)
    launches = sum(fde.fde_launch_count(fde.fde_batch_handle(b, k)) for k in range(len(mine)))
    fde.fde_batch_destroy(b)
    if rank == 0:
        line = {"metric": BATCH_METRIC, "value": round(units / (ms * 1e-3), 3),
                "unit": "problem-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f64 Krylov + fp32 V-cycle", "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD, "problems": BATCH_COUNT,
                           "relaxed_matvec": bool(args.relax),
                           "workers": os.environ.get("FDE_BATCH_WORKERS", "16"),
                           "parallelism": f"problems sharded over {world} rank(s), 16 host "
                                          f"worker streams per rank",
                           "l2": "inputs larger than L2 (256 problems' Krylov bases)"},
                "inner_iterations_per_batch_step_rank0": its[args.warmup:],
                "wall_s": round(wall, 3), "gpu_launches_rank0_total": int(launches),
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", default=None, choices=["gemm", "gemm3", "fft32", "fft64", "fftdf"],
                    help="time one kernel class alone (for profiler captures)")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16", "fp16", "fp32", "bf16x3"])
    ap.add_argument("--outer", default="df32", choices=["df32", "fp64"])
    ap.add_argument("--precond", default="sg", choices=["sg", "redisc", "p2"],
                    help="structured-Galerkin V-cycle, rediscretised V-cycle (P_MGM) or the "
                         "band preconditioner P_2 with a Galerkin V-cycle")
    ap.add_argument("--cycles", type=int, default=1, help="V-cycles per preconditioner application")
    ap.add_argument("--relax", type=int, default=1, choices=[0, 1],
                    help="1: FP32 Krylov matvecs once the residual estimate is within 1e4 x of "
                         "the target (the exit test stays on the FP64-accurate true residual); "
                         "0: every matvec FP64-accurate")
    ap.add_argument("--path", default="tune", choices=["tune", "auto", "gemm", "fft"],
                    help="level product path: tune = time the tensor-core, FFT and direct "
                         "products of every level at set-up and keep the fastest; auto = fixed "
                         "size rule")
    ap.add_argument("--solver", default="fgmres", choices=["fgmres", "mg"],
                    help="mg: multigrid as the solver (x <- x + V(b - M x)) instead of FGMRES")
    ap.add_argument("--warm", type=int, default=0, choices=[0, 1],
                    help="1: start every step's solve from u^(m-1) (the paper starts from zero)")
    ap.add_argument("--workload", default="n2047", choices=["n2047", "batch256"],
                    help="n2047: the single 2047 x 2047 problem (replicated over ranks); "
                         "batch256: 256 independent problems sharded over ranks")
    args = ap.parse_args()
    if args.kernel:
        kernel_micro(args.kernel, args.reps)
        return
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as td
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        td.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = td
    if args.impl == "reference":
        run_reference(args, rank)
        if dist:
            dist.destroy_process_group()
        return
    import torch
    from paper_1706_06844_gb300 import fde, shard
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.workload == "batch256":
        run_batch(args, rank, world, dist)
        if dist:
            dist.destroy_process_group()
        return
    mixed = {"bf16": fde.FDE_PREC_BF16, "fp16": fde.FDE_PREC_FP16, "fp32": fde.FDE_PREC_FP32,
             "bf16x3": fde.FDE_PREC_BF16X3}[args.precision]
    outer = fde.FDE_OUTER_DF32 if args.outer == "df32" else fde.FDE_OUTER_FP64
    precond = {"sg": fde.FDE_PRECOND_MG_SG, "redisc": fde.FDE_PRECOND_MG_REDISC,
               "p2": fde.FDE_PRECOND_P2}[args.precond]
    solver = fde.FDE_SOLVER_MG if args.solver == "mg" else fde.FDE_SOLVER_FGMRES
    path = {"tune": fde.FDE_PATH_TUNE, "auto": fde.FDE_PATH_AUTO, "gemm": fde.FDE_PATH_GEMM,
            "fft": fde.FDE_PATH_FFT}[args.path]
    if args.precision == "fp32" and path == fde.FDE_PATH_GEMM:
        path = fde.FDE_PATH_AUTO  # no tensor-core path in FP32
    w = Workload(mixed, path=path, outer=outer, precond=precond, cycles=args.cycles,
                 relax=args.relax, solver=solver, warm=args.warm)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms, wall, its, launches = time_steps(w, args.steps, args.warmup, dist)
    setup = dict(w.setup_ms, steady_step_ms=round(ms / args.steps, 3),
                 note="outside value: handle creation, multigrid set-up with path tuning "
                      "(set_coefficients), first step with CUDA-graph capture")
    ms = shard.max_over_ranks(ms, dist)
    value = world * args.steps / (ms * 1e-3)
    e2e_v, h2d, d2h = e2e_steps(w, max(2, min(args.steps, 4)))
    roof = roofline(w, 2, args.outer)
    names = {fde.FDE_PATH_GEMM: "gemm", fde.FDE_PATH_FFT: "fft", fde.FDE_PATH_DIRECT: "direct"}
    level_paths = [names.get(fde.fde_level_path(w.h, l), "dense-inverse")
                   for l in range(len(fde.fde_levels(w.h)))]
    first = w.first
    w.close()
    exact = None
    if args.relax and not args.no_fp64:
        # the same mixed-precision solver with every Krylov matvec FP64-accurate
        wx_ = Workload(mixed, path=path, outer=outer, precond=precond, cycles=args.cycles,
                       relax=0, solver=solver, warm=args.warm)
        kx = max(4, args.steps // 2)
        msx, _, itsx, _ = time_steps(wx_, kx, args.warmup, None)
        exact = {"value": round(kx / (msx * 1e-3), 4), "unit": "steps/s",
                 "ms_per_step": round(msx / kx, 3), "iterations_per_step": itsx,
                 "note": "relax=0: every FGMRES matvec double-float accurate"}
        wx_.close()
    fp64 = None
    if not args.no_fp64:
        w64 = Workload(fde.FDE_PREC_FP64)
        ms64, wall64, its64, _ = time_steps(w64, max(2, args.steps // 4), 1, None)
        k64 = max(2, args.steps // 4)
        fp64 = {"value": round(k64 / (ms64 * 1e-3), 4), "unit": "steps/s",
                "ms_per_step": round(ms64 / k64, 3), "iterations_per_step": its64,
                "note": "plain FP64 GPU solver: same FGMRES(30), FP64 V-cycle with FFT products"}
        w64.close()
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t, k, xref, threads = cpu_baseline_sample(refine=True)
        cpu = {"value": round(1.0 / t, 5), "unit": "steps/s", "cores": threads,
               "cores_available": os.cpu_count(),
               "kind": "oracle", "sample": f"one CN step at n=2047 of the FP64 numpy oracle "
                                           f"({k} FGMRES iterations, {t:.1f} s)"}
        err = float(np.linalg.norm(first - xref) / np.linalg.norm(xref))
        accuracy = {"rel_l2_vs_oracle": err, "step": 1, "gpu_rtol": RTOL,
                    "oracle": "FP64 numpy FGMRES + SG V-cycle driven to rtol 1e-12",
                    "iterations_gpu": its[0] if its else None,
                    "iterations_fp64_gpu": (fp64 or {}).get("iterations_per_step", [None])[0]}
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": f"f64 Krylov + {args.precision} V-cycle products", "data": "synthetic",
                "config": {"workload": WORKLOAD.replace(
                               "structured-Galerkin V-cycle",
                               {"sg": "structured-Galerkin V-cycle",
                                "redisc": "rediscretised V-cycle (P_MGM)",
                                "p2": "band preconditioner P_2 with a Galerkin V-cycle"}[args.precond]),
                           "n": N_GRID, "restart": RESTART, "rtol": RTOL,
                           "precond": {"sg": "MG_SG", "redisc": "MG_REDISC",
                                       "p2": "P2"}[args.precond],
                           "cycles": args.cycles, "relaxed_matvec": bool(args.relax),
                           "solver": args.solver, "warm_start": bool(args.warm),
                           "level_paths": level_paths,
                           "precision": f"{args.precision} V-cycle products (FP32 vectors), "
                                        f"{args.outer} FFT outer apply",
                           "l2": "inputs larger than L2 (Krylov basis 31 x 33.5 MB)",
                           "parallelism": f"replicas x{world}"},
                "iterations_per_step": its, "wall_s": round(wall, 3),
                "e2e": {"value": round(e2e_v, 4), "unit": "steps/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches), "roofline": roof, "clocks": clk.summary(),
                "setup": setup,
                "fp64_gpu": fp64, "exact_matvec": exact, "cpu_baseline": cpu,
                "accuracy": accuracy}
        if fp64:
            line["speedup_vs_fp64_gpu"] = round(value / world / fp64["value"], 3)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

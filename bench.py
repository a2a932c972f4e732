"""Benchmark: CN-WSGD time steps per second at n = 2047 (rtol 1e-8).

One bench step is one CN-WSGD time step (Eq. CNWSGD): the right-hand side
b^(m) and the FGMRES(30) solve of M^(m) u^(m) = b^(m) preconditioned by one
structured-Galerkin V-cycle, on the 2047 x 2047 grid of the perturbed
power-law workload (alpha = 1.5, beta = 1.7, WSGD (1,-1), smooth seeded
coefficient perturbation of amplitude 0.2, dt = h, manufactured bubble
solution).  The timed region holds K consecutive steps of the time loop after
W warm-up steps, with every input already resident in HBM.

The headline solver is mixed precision: FP64 Krylov vectors; double-float
right-hand side, true residuals and Krylov matvecs until the FGMRES residual
estimate is within 1e4 x of the target, FP32 matvecs after that (the exit
test is the double-float true residual, so the tolerance met is unchanged);
a V-cycle whose level-0 products run on the tensor cores in BF16x3.

Reported beside it:
  * roofline of the dominant kernel (the tcgen05 Toeplitz products, one
    direction per launch, 2 n^3 method flops) and of every kernel class in the
    units of the method's own work (flops of the Toeplitz products, bytes of
    the FP64 applies, of CGS2 and of the V-cycle's smoothing and transfers),
    with the step's lower bound T_min against the measured step time;
  * the accuracy of EVERY timed step against the FP64 oracle (true residual
    of the GPU's u^(m) in the oracle's arithmetic, from the GPU's u^(m-1)),
    and the distance to an oracle solve driven to rtol 1e-12 at the first and
    the last timed step;
  * the same solver with every matvec double-float, the plain FP64 GPU
    solver, an end-to-end figure through fde_step_host (host arrays, copies
    inside the timed region), sampled SM clocks, the CPU oracle on one whole
    step, the n = 4095 workload (tensor-core vs FFT level products, plain
    FP64), the 256-problem batch and the per-step multigrid set-up of
    time-dependent coefficients.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun) every rank runs an independent replica of the
workload (the solve does not shard across GPUs); value aggregates all ranks.
"""
import argparse
import hashlib
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
CSRC = os.path.join(ROOT, "paper_1706_06844_gb300", "csrc")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the tensor-core products kernel at n = 2047, from ncu captures of exactly
# the kernel source whose SHA-256 is the key (any edit of the file voids the
# figure: the line then reports traffic null).  Value: (x launch, y launch).
GEMM_TRAFFIC = {
    # ncu --set full, bench.py --kernel gemm3 --reps 1 (n = 2047), 128 x 240 tiles
    "a4c2bd93c638de0d2b8934a3e9a4ad25aa49e597a5b810c2c32ded57d1cc71da": (70.178048e6, 67.753216e6),
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def peak_values():
    """Measured roofline denominators (driver-written), else the fallbacks."""
    p = _peaks()
    if "hbm_gbs" in p and "bf16_tflops" in p:
        return (float(p["hbm_gbs"]), float(p["bf16_tflops"]),
                float(p.get("bf16_tflops_sustained", p["bf16_tflops"])), "measured")
    return 6800.0, 1900.0, 1700.0, "fallback"


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
                 solver=0, warm=0, prob=None, n=N_GRID, restart=RESTART):
        import torch
        from paper_1706_06844_gb300 import fde
        self.fde, self.torch = fde, torch
        prob = problem() if prob is None else prob
        self.n = n
        X, Y, hx, hy = prob.grid(n, n)
        self.prob, self.X, self.Y, self.dt = prob, X, Y, hx
        a1, b1, a2, b2 = prob.domain
        kw = dict(alpha=prob.alpha, beta=prob.beta, qx=prob.qx, qy=prob.qy, a1=a1, b1=b1,
                  a2=a2, b2=b2, n1=n, n2=n, dt=self.dt, rtol=RTOL, restart=restart, maxit=2000,
                  precond=fde.FDE_PRECOND_MG_SG if precond is None else precond,
                  precision=precision, cycles=cycles, relax=relax, solver=solver, warm=warm)
        if path is not None:
            kw["toeplitz_path"] = path
        if outer is not None:
            kw["outer"] = outer
        d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
        self.d = d
        self.coef_host = prob.coefficients(X, Y, 0.0)  # time-independent coefficients
        coef = [d(f) for f in self.coef_host]
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
        self.u = d(prob.exact(X, Y, 0.0))
        self.spare = torch.empty((n, n), dtype=torch.float64, device="cuda")
        self.vsrc, self.vhost = {}, {}
        self.m = 0

    def source(self, m, keep_host=False):
        if m not in self.vsrc:
            v = self.prob.source(self.X, self.Y, (m - 0.5) * self.dt)
            self.vsrc[m] = self.d(v)
            if keep_host:
                self.vhost[m] = v
        return self.vsrc[m]

    def step(self, out=None):
        """One CN step from self.u into `out` (default: the spare buffer, and
        the two buffers swap roles)."""
        self.m += 1
        dst = self.spare if out is None else out
        st = self.fde.fde_step(self.h, self.u, self.source(self.m), dst)
        if out is None:
            self.u, self.spare = dst, self.u
        else:
            self.u = dst
        return st

    def close(self):
        self.fde.fde_destroy(self.h)


def time_steps(w, steps, warmup, dist, keep=False):
    """W warm-up steps, then K timed steps bracketed by a barrier and a device
    synchronisation on both sides, CUDA events on the current stream.  With
    keep, every timed step writes a buffer of its own (allocated before the
    timed region), so each step's input and output stay available for the
    oracle check afterwards."""
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
    m_first = w.m + 1
    for m in range(m_first, m_first + steps):
        w.source(m, keep_host=keep)  # sources resident before the timed region
    outs = None
    if keep:
        outs = [torch.empty((w.n, w.n), dtype=torch.float64, device="cuda") for _ in range(steps)]
        start = w.u.clone()
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
    for s in range(steps):
        its.append(w.step(outs[s] if keep else None).iterations)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    hist = None
    if keep:
        hist = {"m_first": m_first, "u": [start.cpu().numpy()] + [o.cpu().numpy() for o in outs]}
        w.spare = outs[-2] if steps > 1 else start  # any buffer that is not w.u
    return ms, wall, its, w.fde.fde_launch_count(w.h) - l0, hist


def e2e_steps(w, steps, warmup=1):
    """Same steps through fde_step_host: pinned host arrays in, host array out
    (the first `warmup` of them untimed)."""
    import torch
    n = w.n
    u_host = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    u_host.copy_(w.u.cpu())
    out = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    srcs = []
    for m in range(w.m + 1, w.m + warmup + steps + 1):
        s = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        s.copy_(torch.from_numpy(w.prob.source(w.X, w.Y, (m - 0.5) * w.dt)))
        srcs.append(s)
    torch.cuda.synchronize()
    for i, s in enumerate(srcs):
        if i == warmup:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        w.fde.fde_step_host(w.h, u_host.data_ptr(), s.data_ptr(), out.data_ptr())
        u_host, out = out, u_host
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nbytes = n * n * 8
    return steps / dt, 2 * nbytes, nbytes


# ---------------------------------------------------------------------------
# roofline in the method's own units

def level_sizes(n, coarsest=8):
    sizes = [n]
    while sizes[-1] > coarsest:
        sizes.append((sizes[-1] - 1) // 2)
    return sizes


def method_work(n, k, n_outer, n_relaxed):
    """Algorithmic work of one CN step with k FGMRES iterations (one V-cycle
    each) on an n x n grid, N = n^2:
      products   level Toeplitz products: two per level and cycle (residual and
                 post-smoothing; the pre-smoothing sweep from zero needs none),
                 each the four triangular n_l x n_l x n_l products of Eq.
                 (AxAy): 4 n_l^3 flops (the coarsest level is a dense solve);
      outer      FP64-accurate applies (rhs, double-float matvecs, true
                 residuals): read x and four coefficient fields, write y:
                 48 N bytes each;
      relaxed    FP32 Krylov matvecs on 8-byte (double-float) vectors: x
                 (8 N), four FP32 coefficient fields (16 N), y (8 N): 32 N
                 bytes each;
      krylov     CGS2 as the method's reference count: at iteration j (j + 1
                 basis vectors) two projections and two updates read the
                 basis four times: sum 4 (j+1) 8 N = 2 k (k+1) 8 N bytes (the
                 delayed scheme that runs reads it twice and writes two
                 vectors: sum (2 (j+2) + 4) 8 N, about 0.7 of this at k = 13,
                 so a fraction f here is about 0.7 f of HBM in bytes moved);
      mg         the V-cycle's smoothing and transfers (FP32): per level
                 below the coarsest, Jacobi from zero (W, b -> x: 3 N_l),
                 residual (K x, b -> r: 3 N_l), restriction (r -> b_c: 1.25
                 N_l), prolongation and correction (x_c, x -> x: 2.25 N_l),
                 post-smoothing (K x, b, x, W -> x: 5 N_l), 4 bytes each,
                 plus the FP64 <-> FP32 conversions of r and z at level 0
                 (24 N bytes), per cycle."""
    N = n * n
    lv = level_sizes(n)
    prod_flops = k * sum(2 * 4 * m ** 3 for m in lv[:-1])
    return {
        "products": {"work": float(prod_flops), "unit": "flop"},
        "outer": {"work": float(n_outer * 48 * N), "unit": "byte"},
        "relaxed": {"work": float(n_relaxed * 32 * N), "unit": "byte"},
        "krylov": {"work": float(2 * k * (k + 1) * 8 * N), "unit": "byte"},
        "mg": {"work": float(k * (24 * N + sum(14.5 * 4 * m * m for m in lv[:-1]))),
               "unit": "byte"},
    }


def level_paths(w):
    """Product path of every multigrid level of a workload's handle."""
    fde = w.fde
    names = {fde.FDE_PATH_GEMM: "gemm", fde.FDE_PATH_FFT: "fft", fde.FDE_PATH_DIRECT: "direct"}
    return [names.get(fde.fde_level_path(w.h, l), "dense-inverse")
            for l in range(len(fde.fde_levels(w.h)))]


def _sha256(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def profile_step_classes(w, steps):
    """Run `steps` further time steps with the library's kernel-class event
    timing on (CUDA events on the library's stream; the V-cycle then runs
    eagerly instead of from its CUDA graph, with the same kernels); returns
    per class (launches, ms) summed over the steps, and the iterations."""
    fde = w.fde
    fde.fde_profile_enable(w.h, 1)
    its, relaxed = [], []
    for _ in range(steps):
        st = w.step()
        its.append(st.iterations)
        relaxed.append(st.relaxed)
    res = {}
    for k, name in [(fde.FDE_KCLASS_OUTER_APPLY, "outer"),
                    (fde.FDE_KCLASS_LEVEL_APPLY, "products"),
                    (fde.FDE_KCLASS_TC_GEMM, "tc_gemm"),
                    (fde.FDE_KCLASS_KRYLOV, "krylov"), (fde.FDE_KCLASS_MG_OTHER, "mg"),
                    (fde.FDE_KCLASS_OUTER_FP32, "relaxed")]:
        res[name] = fde.fde_profile_query(w.h, k)
    fde.fde_profile_enable(w.h, 0)
    return res, its, relaxed


def roofline(w, prof, its, relaxed, ms_per_step, level_paths):
    """Dominant kernel (the tcgen05 products, one launch per direction) and
    every kernel class against its own bound, in the method's units."""
    hbm, bf16, bf16_s, src = peak_values()
    n = w.n
    steps = len(its)
    k = float(np.mean(its))
    n_relaxed = float(np.mean(relaxed))
    n_outer = prof["outer"][0] / steps
    work = method_work(n, k, n_outer, n_relaxed)
    classes = {}
    t_min = 0.0
    for name in ["products", "outer", "relaxed", "krylov", "mg"]:
        wk = work[name]
        launches, ms = prof[name]
        meas = ms / steps
        if wk["unit"] == "flop":
            bound = wk["work"] / (bf16 * 1e12) * 1e3
            peak, unit, ach = bf16, "TFLOP/s", (wk["work"] / (meas * 1e-3) / 1e12 if meas else None)
        else:
            bound = wk["work"] / (hbm * 1e9) * 1e3
            peak, unit, ach = hbm, "GB/s", (wk["work"] / (meas * 1e-3) / 1e9 if meas else None)
        t_min += bound
        classes[name] = {"work_per_step": wk["work"], "work_unit": wk["unit"],
                         "t_min_ms": round(bound, 4), "measured_ms_per_step": round(meas, 4),
                         "achieved": None if ach is None else round(ach, 2), "peak": peak,
                         "unit": unit, "frac": None if not meas else round(bound / meas, 4),
                         "launches_per_step": round(launches / steps, 1)}
    classes["products"]["note"] = ("all levels' Toeplitz products (tensor-core, FFT and direct "
                                   "paths, operand packing) against the BF16 tensor peak")
    classes["relaxed"]["note"] = "FFT passes in FP32 issue-bound; bytes are the HBM floor"
    prof_total = sum(prof[c][1] for c in ["products", "outer", "relaxed", "krylov", "mg"]) / steps
    # the dominant kernel: tensor-core products, one direction per launch
    gl, gms = prof["tc_gemm"]
    gemm_levels = [l for l, p in enumerate(level_paths) if p == "gemm"]
    roof = None
    if gl > 0 and gemm_levels:
        sizes = level_sizes(n)
        # every tensor-core level runs the same number of launches per cycle
        flops_launch = float(np.mean([2.0 * sizes[l] ** 3 for l in gemm_levels]))
        avg_s = gms / gl * 1e-3
        ach = flops_launch / avg_s / 1e12
        sha = _sha256(os.path.join(CSRC, "tc_gemm.cu"))
        tr = GEMM_TRAFFIC.get(sha)
        roof = {"bound": "tensor",
                "kernel": "tc::toeplitz_gemm_kernel (tcgen05, BF16x3: 3 BF16 products per "
                          "block, FP32 accumulation in TMEM), one direction per launch",
                "achieved": round(ach, 2), "peak": bf16, "unit": "TFLOP/s",
                "frac": round(ach / bf16, 4),
                "peak_kind": f"bf16 dense burst ({src}); frac against the sustained "
                             f"{bf16_s} TFLOP/s: {round(ach / bf16_s, 4)}",
                "traffic": None if tr is None else float(np.mean(tr)),
                "traffic_note": ("dram__bytes_read.sum + dram__bytes_write.sum per launch (mean "
                                 "of the x and y launches) from an ncu capture of this kernel "
                                 "source" if tr is not None else
                                 "null: no ncu capture of the current kernel source"),
                "work_per_launch": flops_launch,
                "work_note": "method flops: the two triangular Toeplitz products of one "
                             "direction, 2 n^3 at n = 2047 (the BF16x3 split executes 3 "
                             "products per block, ~3.5x this on the tensor pipe)",
                "launches": int(gl), "avg_launch_us": round(avg_s * 1e6, 2),
                "share_of_step": round(gms / steps / prof_total, 4) if prof_total else None}
    if roof is None:
        # no tensor-core level in this run (the tuner kept FFT products on every
        # level): the class with the largest measured time stands in
        name = max(classes, key=lambda c: classes[c]["measured_ms_per_step"])
        cl = classes[name]
        roof = {"bound": "tensor" if cl["work_unit"] == "flop" else "hbm",
                "kernel": f"kernel class '{name}' (no tensor-core level in this run)",
                "achieved": cl["achieved"], "peak": cl["peak"], "unit": cl["unit"],
                "frac": None if cl["achieved"] is None else round(cl["achieved"] / cl["peak"], 4),
                "traffic": None, "traffic_note": "null: a class of several kernels",
                "work_per_launch": None, "launches": None, "avg_launch_us": None,
                "share_of_step": (round(cl["measured_ms_per_step"] / prof_total, 4)
                                  if prof_total else None)}
    step = {"t_min_ms": round(t_min, 4), "ms_per_step": round(ms_per_step, 4),
            "frac": round(t_min / ms_per_step, 4),
            "note": "T_min = product flops / BF16 burst peak + all other bytes / HBM copy peak "
                    f"({src}); k = {k:g} iterations, {n_outer:g} FP64-accurate applies, "
                    f"{n_relaxed:g} relaxed matvecs per step"}
    return roof, classes, step


# ---------------------------------------------------------------------------
# the FP64 oracle at the bench grid

class Oracle:
    """The FP64 oracle at the bench grid: weights, CN scalars, the
    structured-Galerkin hierarchy (set up once, untimed), its operator, right-
    hand side and FGMRES solve."""

    def __init__(self, prob=None, n=N_GRID, restart=RESTART):
        from oracle.wsgd import wsgd_weights
        from oracle.operator import cn_scalars, rhs_fft, apply_M_fft
        from oracle import multigrid as mg
        prob = problem() if prob is None else prob
        self.prob, self.n, self.restart = prob, n, restart
        X, Y, hx, hy = prob.grid(n, n)
        self.X, self.Y, self.hx, self.dt = X, Y, hx, hx
        wx = wsgd_weights(prob.alpha, n + 1, 1, prob.qx)
        wy = wsgd_weights(prob.beta, n + 1, 1, prob.qy)
        sc = cn_scalars(prob.alpha, prob.beta, hx, hy, self.dt)
        c, s = sc["c"], sc["sigma"]
        coef = prob.coefficients(X, Y, 0.0)
        self.hier = mg.structured_galerkin(wx, wy, n, n, c, s, coef)
        self.rhs = lambda U, V: rhs_fft(U, wx, wy, c, s, *coef, V, hx, prob.alpha)
        self.A = lambda Z: apply_M_fft(Z, wx, wy, c, s, *coef)
        self.prec = lambda R: mg.vcycle(self.hier, R)
        self.wall_s = 0.0  # timed wall and process CPU seconds (all threads)
        self.cpu_s = 0.0

    def threads_used(self):
        """Effective number of host threads of the timed work: process CPU
        time over wall time, at least 1."""
        return max(1, int(round(self.cpu_s / self.wall_s))) if self.wall_s > 0 else 1

    def source(self, m):
        return self.prob.source(self.X, self.Y, (m - 0.5) * self.dt)

    def step(self, U, V):
        """One whole CN step (right-hand side + FGMRES(30) to rtol 1e-8), timed."""
        from oracle.krylov import fgmres
        c0, t0 = time.process_time(), time.perf_counter()
        B = self.rhs(U, V)
        x, its, rel, ok = fgmres(self.A, B, self.prec, self.restart, RTOL)
        t = time.perf_counter() - t0
        self.wall_s += t
        self.cpu_s += time.process_time() - c0
        return t, its, x, B

    def residual(self, U_prev, V, U):
        """||b - M u|| / ||b|| of a GPU step in FP64, b from the GPU's u^(m-1)."""
        B = self.rhs(U_prev, V)
        return float(np.linalg.norm(B - self.A(U)) / np.linalg.norm(B)), B

    def refined_error(self, B, U):
        """Relative L2 distance of U to the oracle solution of M x = B driven
        to rtol 1e-12 (FGMRES started from U)."""
        from oracle.krylov import fgmres
        x, its, rel, ok = fgmres(self.A, B, self.prec, self.restart, 1e-12, x0=U)
        return float(np.linalg.norm(U - x) / np.linalg.norm(x)), int(its)


def accuracy_check(orc, hist, vhost, its_gpu, its_fp64):
    """Every timed step: the oracle's true residual of the GPU's u^(m) (its
    right-hand side built from the GPU's u^(m-1)); first and last timed step:
    distance to the oracle solution driven to rtol 1e-12."""
    U = hist["u"]
    m0 = hist["m_first"]
    res, errs = [], {}
    K = len(U) - 1
    for s in range(K):
        r, B = orc.residual(U[s], vhost[m0 + s], U[s + 1])
        res.append(r)
        if s == 0 or s == K - 1:
            e, k = orc.refined_error(B, U[s + 1])
            errs[f"step_{m0 + s}"] = {"rel_l2_vs_oracle": e, "oracle_refine_iterations": k}
    return {"oracle": "FP64 numpy: rhs and M from Eq. (M) by FFT embedding; FGMRES(30) + SG "
                      "V-cycle driven to rtol 1e-12 from the GPU's solution",
            "gpu_rtol": RTOL,
            "true_residual_every_step": [float(f"{r:.3e}") for r in res],
            "max_true_residual": max(res), "all_steps_within_rtol": bool(max(res) <= 1.05 * RTOL),
            "rel_l2_first_last": errs,
            "max_rel_l2": max(v["rel_l2_vs_oracle"] for v in errs.values()),
            "target_rel_l2": 1e-8,
            "iterations_gpu": its_gpu, "iterations_fp64_gpu": its_fp64}


def run_reference(args, rank):
    """The oracle as the reference arm: the oracle's own CN time loop at the
    bench grid; every timed step is one whole step (right-hand side and
    FGMRES(30) with the SG V-cycle to rtol 1e-8), sources precomputed like the
    GPU arm's resident inputs; the W warm-up steps are right-hand sides only."""
    if rank != 0:
        return
    o = Oracle()
    U = o.prob.exact(o.X, o.Y, 0.0)
    for i in range(args.warmup):
        o.rhs(U, o.source(1))  # untimed warm-up (page-in, FFT plans)
    srcs = [o.source(m) for m in range(1, args.steps + 1)]
    o.wall_s = o.cpu_s = 0.0
    times, its = [], []
    for m in range(args.steps):
        t, k, U, _ = o.step(U, srcs[m])
        times.append(t)
        its.append(k)
    total = sum(times)
    v = args.steps / total
    cores = o.threads_used()
    sample = (f"{args.steps} whole consecutive CN steps of the FP64 numpy oracle at n=2047 "
              f"(right-hand side + FGMRES(30)/SG V-cycle to rtol 1e-8, FFT products), "
              f"{args.warmup} untimed right-hand sides as warm-up")
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
            "timed_s": round(total, 2), "iterations_per_step": its}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# further workloads reported as sub-objects of the default line

def sub_n4095(reps=3):
    """n = 4095 (alpha = 1.9, beta = 1.2, config-3 coefficients, FGMRES(20)):
    level-0 products on the tensor cores (BF16x3) vs FFT embedding, and the
    plain FP64 solver; steps/s over `reps` steps after one warm-up step, the
    oracle's true residual of the first timed step of the tensor-core run."""
    import torch
    from paper_1706_06844_gb300 import fde, inputs
    prob = inputs.perturbed_power_law(alpha=1.9, beta=1.2, seed=1706068, amplitude=0.2)
    n = 4095
    out = {"workload": "perturbed power-law, n=4095, alpha=1.9, beta=1.2, FGMRES(20), rtol 1e-8",
           "precision": "BF16x3 tensor-core products read as the TF32-class preconditioner"}
    for name, kw in [("gemm", dict(precision=fde.FDE_PREC_BF16X3, path=fde.FDE_PATH_GEMM,
                                   outer=fde.FDE_OUTER_DF32, relax=1)),
                     ("fft", dict(precision=fde.FDE_PREC_BF16X3, path=fde.FDE_PATH_FFT,
                                  outer=fde.FDE_OUTER_DF32, relax=1)),
                     ("fp64", dict(precision=fde.FDE_PREC_FP64))]:
        try:
            w = Workload(kw["precision"], path=kw.get("path"), outer=kw.get("outer"),
                         relax=kw.get("relax", 0), prob=prob, n=n, restart=20)
        except fde.FDEError as e:
            out[name] = {"unavailable": str(e)}
            continue
        try:
            k = 2 if name == "fp64" else reps
            ms, wall, its, launches, hist = time_steps(w, k, 1, None, keep=(name == "gemm"))
            ent = {"value": round(k / (ms * 1e-3), 4), "unit": "steps/s",
                   "ms_per_step": round(ms / k, 3), "iterations_per_step": its,
                   "level_paths": level_paths(w)}
            if name == "gemm":
                prof, pits, prel = profile_step_classes(w, 1)
                gl, gms = prof["tc_gemm"]
                glev = [l for l, p_ in enumerate(ent["level_paths"]) if p_ == "gemm"]
                if gl and glev:
                    # every tensor-core level runs the same number of launches per cycle
                    sizes = level_sizes(n)
                    avg = gms / gl * 1e-3
                    flops = float(np.mean([2.0 * sizes[l] ** 3 for l in glev]))
                    ent["tc_gemm_avg_launch_us"] = round(avg * 1e6, 2)
                    ent["tc_gemm_method_tflops"] = round(flops / avg / 1e12, 2)
                    ent["tc_gemm_note"] = ("launches of all tensor-core levels; method flops "
                                           "2 n_l^3 averaged over those levels")
                orc = Oracle(prob, n, restart=20)
                r, _ = orc.residual(hist["u"][0], w.vhost[hist["m_first"]], hist["u"][1])
                ent["oracle_true_residual_first_step"] = r
            out[name] = ent
        finally:
            w.close()
            torch.cuda.empty_cache()
    return out


def sub_setup_per_step(reps=3):
    """Time-dependent coefficients (Example 2 of Sec. 5, on the bench grid's
    mixed-precision solver): per step the multigrid set-up for the new
    coefficients (fde_set_coefficients of t^(m) and t^(m-1): hierarchy,
    level fields, tensor-core generators, coarsest inverse) against the step."""
    import torch
    from paper_1706_06844_gb300 import fde, inputs
    prob = inputs.example2()
    n = N_GRID
    w = Workload(fde.FDE_PREC_BF16X3, path=fde.FDE_PATH_TUNE, outer=fde.FDE_OUTER_DF32, relax=1,
                 prob=prob, n=n)
    try:
        X, Y = w.X, w.Y
        coefs = [[w.d(f) for f in prob.coefficients(X, Y, m * w.dt)] for m in range(reps + 2)]
        srcs = [w.source(m) for m in range(1, reps + 2)]
        w.step()  # warm-up (captures the cycle's graph)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        setup_ms, step_ms, its = [], [], []
        for m in range(2, reps + 2):
            e[0].record()
            fde.fde_set_coefficients(w.h, fde.FDE_COEF_OLD, *coefs[m - 1])
            fde.fde_set_coefficients(w.h, fde.FDE_COEF_NEW, *coefs[m])
            e[1].record()
            its.append(fde.fde_step(w.h, w.u, srcs[m - 1], w.spare).iterations)
            w.u, w.spare = w.spare, w.u
            e[2].record()
            torch.cuda.synchronize()
            setup_ms.append(e[0].elapsed_time(e[1]))
            step_ms.append(e[1].elapsed_time(e[2]))
        return {"workload": "Example 2 coefficients (1 + t) factors, n=2047, alpha=1.8, "
                            "beta=1.9, BF16x3 V-cycle, FGMRES(30), rtol 1e-8",
                "setup_ms_per_step": round(float(np.mean(setup_ms)), 3),
                "solve_ms_per_step": round(float(np.mean(step_ms)), 3),
                "setup_share": round(float(np.mean(setup_ms)) /
                                     float(np.mean(setup_ms) + np.mean(step_ms)), 4),
                "iterations_per_step": its,
                "note": "set-up = both coefficient uploads' device work: copies, sigma "
                        "scaling, transposes, double-float and FP32 copies, every level's "
                        "generator and fields, tensor-core generator banks, coarsest inverse "
                        "(a device->host status read synchronises once)"}
    finally:
        w.close()
        torch.cuda.empty_cache()


BATCH_COUNT = 256
BATCH_METRIC = "CN-WSGD problem-steps/s, 256 independent problems (n in {63,127,255,511}), rtol 1e-8"
BATCH_WORKLOAD = ("256 problems, seed 1706069: n uniform over {63,127,255,511}, alpha, beta ~ "
                  "U(1.1,1.9), WSGD q in {0,-1} (-1 below gamma_0), coefficients exp(ln2 psi) in "
                  "[0.5,2] with psi a smooth seeded field, dt=h, FGMRES(30) + structured-Galerkin "
                  "FP32 V-cycle, double-float outer apply (relaxed matvec unless --relax 0), "
                  "rtol 1e-8")


class BatchRun:
    """The 256-problem workload (or this rank's share of it) on one batch."""

    def __init__(self, relax, rank=0, world=1):
        import torch
        from paper_1706_06844_gb300 import fde, inputs, shard
        self.fde = fde
        probs = inputs.random_batch(BATCH_COUNT)
        self.mine = shard.shard([shard.problem_cost(n, n) for n, _ in probs], rank, world)
        d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
        params, coef, self.u, self.base, self.dts, self.probs = [], [], [], [], [], []
        for i in self.mine:
            n, pb = probs[i]
            X, Y, hx, hy = pb.grid(n, n)
            a1, b1, a2, b2 = pb.domain
            params.append(fde.params(alpha=pb.alpha, beta=pb.beta, qx=pb.qx, qy=pb.qy, a1=a1,
                                     b1=b1, a2=a2, b2=b2, n1=n, n2=n, dt=hx, rtol=RTOL,
                                     restart=RESTART, maxit=2000,
                                     precond=fde.FDE_PRECOND_MG_SG,
                                     precision=fde.FDE_PREC_FP32, outer=fde.FDE_OUTER_DF32,
                                     relax=relax))
            coef.append([d(f) for f in pb.coefficients(X, Y, 0.0)])
            self.u.append(d(pb.exact(X, Y, 0.0)))
            # time-independent coefficients: the manufactured source is exp(-t) v(0)
            self.base.append(d(pb.source(X, Y, 0.0)))
            self.dts.append(hx)
            self.probs.append((n, pb))
        self.b = fde.fde_batch_create(params)
        for k in range(len(self.mine)):
            h = fde.fde_batch_handle(self.b, k)
            fde.fde_set_coefficients(h, fde.FDE_COEF_NEW, *coef[k])
            fde.fde_set_coefficients(h, fde.FDE_COEF_OLD, *coef[k])
        self.nxt = [torch.empty_like(x) for x in self.u]
        self.m = 0
        self.its = []

    def sources(self, m):
        return [self.base[k] * float(np.exp(-(m - 0.5) * self.dts[k]))
                for k in range(len(self.mine))]

    def step(self, src):
        self.m += 1
        st = self.fde.fde_batch_step(self.b, self.u, src, self.nxt)
        self.its.append(sum(s.iterations for s in st))
        self.u, self.nxt = self.nxt, self.u

    def launches(self):
        return self.fde.fde_batch_launch_count(self.b)

    def engine(self):
        return {1: "grouped: one launch per stage for all problems, restart cycles replayed "
                   "from a CUDA graph", 2: "worker threads"}.get(
            self.fde.fde_batch_engine(self.b), "none") + \
            (f" ({self.fde.fde_batch_engine_note(self.b)})"
             if self.fde.fde_batch_engine_note(self.b) else "")

    def close(self):
        self.fde.fde_batch_destroy(self.b)


def run_batch(args, rank, world, dist):
    """Every rank steps its share of the 256 problems (no data-path collective);
    value = all problem-steps of all ranks / the slowest rank's time."""
    import torch
    from paper_1706_06844_gb300 import shard as sh
    br = BatchRun(args.relax, rank, world)
    total = args.warmup + args.steps
    src = [br.sources(m) for m in range(1, total + 1)]
    for m in range(args.warmup):
        br.step(src[m])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = br.launches()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ev0.record()
        t0 = time.perf_counter()
        for m in range(args.warmup, total):
            br.step(src[m])
        ev1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    ms = sh.max_over_ranks(ev0.elapsed_time(ev1), dist)
    units = sh.sum_over_ranks(len(br.mine) * args.steps, dist)
    launches = br.launches() - l0
    br.close()
    if rank == 0:
        line = {"metric": BATCH_METRIC, "value": round(units / (ms * 1e-3), 3),
                "unit": "problem-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "FP64 Krylov vectors, double-float rhs/true residual/matvecs, FP32 "
                         "relaxed matvecs, FP32 V-cycle", "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD, "problems": BATCH_COUNT,
                           "relaxed_matvec": bool(args.relax),
                           "parallelism": f"problems sharded over {world} rank(s)",
                           "l2": "inputs larger than L2 (256 problems' Krylov bases)"},
                "inner_iterations_per_batch_step_rank0": br.its[args.warmup:],
                "wall_s": round(wall, 3), "gpu_launches": int(launches),
                "engine": br.engine(), "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def sub_batch(reps=3):
    """The 256-problem batch on this GPU: problem-steps/s over `reps` batch
    steps after one warm-up, and the oracle's true residual of 8 problems'
    last step (b from the GPU's u^(m-1))."""
    import torch
    from oracle.wsgd import wsgd_weights
    from oracle.operator import cn_scalars, rhs, apply_M
    br = BatchRun(1)
    try:
        src = [br.sources(m) for m in range(1, reps + 2)]
        br.step(src[0])
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = br.launches()
        ev0.record()
        for m in range(1, reps):
            br.step(src[m])
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = br.launches() - l0
        prev = [x.cpu().numpy() for x in br.u]
        br.step(src[reps])
        cur = [x.cpu().numpy() for x in br.u]
        srch = [s.cpu().numpy() for s in src[reps]]
        res = []
        for k in range(0, len(br.mine), max(1, len(br.mine) // 8)):
            n, pb = br.probs[k]
            X, Y, hx, hy = pb.grid(n, n)
            wx, wy = wsgd_weights(pb.alpha, n + 1, 1, pb.qx), wsgd_weights(pb.beta, n + 1, 1, pb.qy)
            sc = cn_scalars(pb.alpha, pb.beta, hx, hy, hx)
            cf = pb.coefficients(X, Y, 0.0)
            B = rhs(prev[k], wx, wy, sc["c"], sc["sigma"], *cf, srch[k], hx, pb.alpha)
            res.append(float(np.linalg.norm(B - apply_M(cur[k], wx, wy, sc["c"], sc["sigma"],
                                                        *cf)) / np.linalg.norm(B)))
        k = reps - 1
        return {"metric": BATCH_METRIC, "value": round(len(br.mine) * k / (ms * 1e-3), 3),
                "unit": "problem-steps/s", "ms_per_batch_step": round(ms / k, 3),
                "inner_iterations_per_batch_step": br.its[1:reps],
                "gpu_launches_per_batch_step": int(launches / k),
                "engine": br.engine(),
                "oracle_true_residual_sample": [float(f"{r:.3e}") for r in res],
                "workload": BATCH_WORKLOAD}
    finally:
        br.close()
        torch.cuda.empty_cache()


def kernel_micro(kind, reps, n=N_GRID):
    """One kernel class in isolation, for profiler captures:
    gemm / gemm3 = level-0 V-cycle products (BF16 / BF16x3 tcgen05 GEMM),
    fft32 = FP32 FFT level products, fft64 / fftdf = the outer apply
    (FP64 / double-float FFT), step = whole CN steps of the headline solver
    (its Krylov, matvec and V-cycle kernels, e.g. for a capture of the
    Gram-Schmidt passes at a smaller n)."""
    import torch
    from paper_1706_06844_gb300 import fde
    if kind == "step":
        w = Workload(fde.FDE_PREC_BF16X3, outer=fde.FDE_OUTER_DF32, relax=1, n=n)
        its = [w.step().iterations for _ in range(2)]
        for m in range(w.m + 1, w.m + reps + 1):
            w.source(m)  # the sources of the timed steps, sampled on the host beforehand
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            its.append(w.step().iterations)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"kernel": kind, "n": n, "reps": reps, "iterations": its,
                          "level_paths": level_paths(w),
                          "ms_per_call": round(e0.elapsed_time(e1) / reps, 4)}))
        w.close()
        return
    prec = {"gemm": fde.FDE_PREC_BF16, "gemm3": fde.FDE_PREC_BF16X3, "fft32": fde.FDE_PREC_FP32,
            "fft64": fde.FDE_PREC_FP64, "fftdf": fde.FDE_PREC_FP64}[kind]
    path = {"gemm": fde.FDE_PATH_GEMM, "gemm3": fde.FDE_PATH_GEMM,
            "fft32": fde.FDE_PATH_FFT}.get(kind)
    outer = fde.FDE_OUTER_DF32 if kind == "fftdf" else None
    w = Workload(prec, path=path, outer=outer, n=n)
    x = torch.randn((n, n), dtype=torch.float64, device="cuda")
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
    print(json.dumps({"kernel": kind, "n": n, "reps": reps,
                      "ms_per_call": round(e0.elapsed_time(e1) / reps, 4)}))
    w.close()


def dtype_string(args):
    if args.outer == "df32":
        parts = ["double-float (FP32-pair) Krylov vectors with DCGS2 on the FP32 pipes, FP64 "
                 "Hessenberg/Givens/least squares on the device",
                 "FP64 x, b and true residual from double-float FFT matvecs"]
    else:
        parts = ["FP64 Krylov vectors (DCGS2), FP64 Hessenberg/Givens/least squares",
                 "FP64 rhs/true residual/matvecs"]
    if args.relax:
        parts.append("FP32 relaxed matvecs near convergence")
    prec = {"bf16x3": "BF16x3", "bf16": "BF16", "fp16": "FP16", "fp32": "FP32"}[args.precision]
    if args.precision == "fp32":
        parts.append("FP32 V-cycle")
    else:
        parts.append(f"FP32 V-cycle vectors with {prec} tensor-core level products where tuned "
                     f"(FP32 accumulation)")
    return ", ".join(parts)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", default=None,
                    choices=["gemm", "gemm3", "fft32", "fft64", "fftdf", "step"],
                    help="time one kernel class alone (for profiler captures)")
    ap.add_argument("--kernel-n", type=int, default=N_GRID)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle legs (CPU baseline and accuracy checks)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the n = 4095, batch and set-up sub-objects")
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
        kernel_micro(args.kernel, args.reps, args.kernel_n)
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
    oracle_legs = rank == 0 and world == 1 and not args.no_cpu_baseline
    w = Workload(mixed, path=path, outer=outer, precond=precond, cycles=args.cycles,
                 relax=args.relax, solver=solver, warm=args.warm)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms, wall, its, launches, hist = time_steps(w, args.steps, args.warmup, dist,
                                                   keep=oracle_legs)
    setup = dict(w.setup_ms, steady_step_ms=round(ms / args.steps, 3),
                 note="outside value: handle creation, multigrid set-up with path tuning "
                      "(set_coefficients), first step with CUDA-graph capture")
    ms = shard.max_over_ranks(ms, dist)
    value = world * args.steps / (ms * 1e-3)
    e2e_v, h2d, d2h = e2e_steps(w, max(2, min(args.steps, 8)))
    paths = level_paths(w)
    prof, pits, prel = profile_step_classes(w, 3)
    roof, classes, step_roof = roofline(w, prof, pits, prel, ms / args.steps, paths)
    vhost = w.vhost
    w.close()
    exact = None
    if args.relax and not args.no_fp64:
        # the same mixed-precision solver with every Krylov matvec FP64-accurate
        wx_ = Workload(mixed, path=path, outer=outer, precond=precond, cycles=args.cycles,
                       relax=0, solver=solver, warm=args.warm)
        kx = max(4, args.steps // 2)
        msx, _, itsx, _, _ = time_steps(wx_, kx, args.warmup, None)
        exact = {"value": round(kx / (msx * 1e-3), 4), "unit": "steps/s",
                 "ms_per_step": round(msx / kx, 3), "iterations_per_step": itsx,
                 "note": "relax=0: every FGMRES matvec double-float accurate"}
        wx_.close()
    fp64 = None
    if not args.no_fp64:
        w64 = Workload(fde.FDE_PREC_FP64)
        k64 = max(2, args.steps // 4)
        ms64, wall64, its64, _, _ = time_steps(w64, k64, 1, None)
        fp64 = {"value": round(k64 / (ms64 * 1e-3), 4), "unit": "steps/s",
                "ms_per_step": round(ms64 / k64, 3), "iterations_per_step": its64,
                "note": "plain FP64 GPU solver: same FGMRES(30), FP64 V-cycle with FFT products, "
                        "FP64 FFT matvecs"}
        w64.close()
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        for name, fn in [("n4095", sub_n4095), ("batch256", sub_batch),
                         ("setup_per_step", sub_setup_per_step)]:
            try:
                extra[name] = fn()
            except Exception as e:  # reported, never silently dropped
                extra[name] = {"failed": f"{type(e).__name__}: {e}"}
    cpu = None
    accuracy = None
    if oracle_legs:
        orc = Oracle()
        U0 = hist["u"][0]
        t, k, x, B = orc.step(U0, vhost[hist["m_first"]])
        cpu = {"value": round(1.0 / t, 5), "unit": "steps/s", "cores": orc.threads_used(),
               "cores_available": os.cpu_count(), "kind": "oracle",
               "sample": f"one whole CN step at n=2047 of the FP64 numpy oracle (rhs + "
                         f"FGMRES(30)/SG V-cycle to rtol 1e-8: {k} iterations, {t:.1f} s), "
                         f"from the GPU's u at the first timed step"}
        accuracy = accuracy_check(orc, hist, vhost, its,
                                  (fp64 or {}).get("iterations_per_step"))
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": dtype_string(args), "data": "synthetic",
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
                           "level_paths": paths,
                           "precision": f"{args.precision} V-cycle products (FP32 vectors), "
                                        f"{args.outer} FFT outer apply",
                           "l2": "inputs larger than L2 (Krylov basis 31 x 33.5 MB)",
                           "parallelism": f"replicas x{world}"},
                "iterations_per_step": its, "wall_s": round(wall, 3),
                "e2e": {"value": round(e2e_v, 4), "unit": "steps/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches), "roofline": roof,
                "roofline_classes": classes, "step_roofline": step_roof,
                "clocks": clk.summary(), "setup": setup,
                "fp64_gpu": fp64, "exact_matvec": exact, "cpu_baseline": cpu,
                "accuracy": accuracy, **extra}
        if fp64:
            line["speedup_vs_fp64_gpu"] = round(value / world / fp64["value"], 3)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

// libfde host side: the C ABI of include/fde.h, the FP64-accurate outer
// operator (Eq. M) and restarted flexible GMRES (Sec. 5) of one problem; the
// handle and the multigrid hierarchies (Sec. 4) are in solver.cuh.  All
// arithmetic on grid data runs in the kernels of kernels_*.cu; the host only
// sequences launches and reads one small status per Krylov step.
#include "solver.cuh"

namespace {
std::string g_create_error;
}  // namespace

namespace fde {
void set_global_error(const char* msg) { g_create_error = msg; }
}  // namespace fde

// ============================================================================
// FP64-accurate outer operator

// The two passes of an outer apply -- the rows of x (with the c x term) and
// the rows of the transposed grid -- then y += yT^T.  When both FFT lengths
// agree the passes share one launch (the transpose of x goes first).
template <typename T, typename R, typename C>
static int outer_passes(fde_handle* h, const T* x, T* y, T* xT, T* yT, int logLx, int logLy,
                        const cx<R>* S1x, const cx<R>* S2x, const cx<R>* twx, const C* cpx,
                        const C* cmx, const cx<R>* S1y, const cx<R>* S2y, const cx<R>* twy,
                        const C* cpy, const C* cmy, cx<R>* ws, size_t wse) {
  const FftPass<T, R, C> px{x, 1, h->n1, h->n2, h->n1, S1x, S2x, twx, cpx, cmx, x, h->c, y, 0};
  const FftPass<T, R, C> py{xT, 1, h->n2, h->n1, h->n2, S1y, S2y, twy, cpy, cmy, nullptr, 0.0,
                            yT, 0};
  LCHK(launch_transpose<T>(x, h->n2, h->n1, xT, 0, h->st));
  if (logLx == logLy) {
    LCHK((launch_fft_pass2<T, R, C>(px, py, logLx, h->st, ws, wse)));
  } else {
    LCHK((launch_fft_pass<T, R, C>(px.X, px.es, px.vs, px.nvec, px.n, logLx, px.S1, px.S2, px.tw,
                                   px.cp, px.cm, px.M, px.cmass, px.Y, 0, h->st, ws, wse)));
    LCHK((launch_fft_pass<T, R, C>(py.X, py.es, py.vs, py.nvec, py.n, logLy, py.S1, py.S2, py.tw,
                                   py.cp, py.cm, nullptr, 0.0, py.Y, 0, h->st, ws, wse)));
  }
  LCHK(launch_transpose<T>(yT, h->n1, h->n2, y, 1, h->st));
  return FDE_OK;
}

static int outer_apply(fde_handle* h, const double* x, double* y, bool old) {
  NvtxRange range("matvec");
  const int pi = h->pbeg(FDE_KCLASS_OUTER_APPLY);
  if (h->p.outer == FDE_OUTER_DF32) {
    df* const* cf = old ? h->cfO : h->cfN;
    df* const* cfT = old ? h->cfOT : h->cfNT;
    RCHK((outer_passes<double, df, df>(h, x, y, h->xT, h->yT, h->logLx, h->logLy, h->S1xd,
                                       h->S2xd, h->twxd, cf[0], cf[1], h->S1yd, h->S2yd, h->twyd,
                                       cfT[0], cfT[1], reinterpret_cast<cx<df>*>(h->fft_ws),
                                       h->fft_ws_elems)));
  } else {
    RCHK((outer_passes<double, double, double>(
        h, x, y, h->xT, h->yT, h->logLx, h->logLy, h->S1x, h->S2x, h->twx, old ? h->dpO : h->dpN,
        old ? h->dmO : h->dmN, h->S1y, h->S2y, h->twy, old ? h->epOsT : h->epNsT,
        old ? h->emOsT : h->emNsT, h->fft_ws, h->fft_ws_elems)));
  }
  h->pend(pi);
  return FDE_OK;
}

// y = M^(m) x on double-float vectors (x, y: 8-byte hi, lo pairs), the
// double-float outer operator without conversions at its ends
static int outer_apply_df(fde_handle* h, const double* x_, double* y_) {
  NvtxRange range("matvec");
  const int pi = h->pbeg(FDE_KCLASS_OUTER_APPLY);
  RCHK((outer_passes<df, df, df>(h, reinterpret_cast<const df*>(x_), reinterpret_cast<df*>(y_),
                                 reinterpret_cast<df*>(h->xT), reinterpret_cast<df*>(h->yT),
                                 h->logLx, h->logLy, h->S1xd, h->S2xd, h->twxd, h->cfN[0],
                                 h->cfN[1], h->S1yd, h->S2yd, h->twyd, h->cfNT[0], h->cfNT[1],
                                 reinterpret_cast<cx<df>*>(h->fft_ws), h->fft_ws_elems)));
  h->pend(pi);
  return FDE_OK;
}

// the relaxed matvec on double-float vectors (FP32 arithmetic, FP32 result
// widened)
static int outer_apply32_df(fde_handle* h, const double* x_, double* y_) {
  NvtxRange range("matvec_fp32");
  const int pi = h->pbeg(FDE_KCLASS_OUTER_FP32);
  RCHK((outer_passes<df, float, float>(
      h, reinterpret_cast<const df*>(x_), reinterpret_cast<df*>(y_), reinterpret_cast<df*>(h->xT),
      reinterpret_cast<df*>(h->yT), h->logLx, h->logLy, h->S1x32, h->S2x32, h->twx32, h->cf32[0],
      h->cf32[1], h->S1y32, h->S2y32, h->twy32, h->cf32T[0], h->cf32T[1],
      reinterpret_cast<cx<float>*>(h->fft_ws), h->fft_ws_elems * 2)));
  h->pend(pi);
  return FDE_OK;
}

// y = M^(m) x with FP32 arithmetic on FP64 data (relaxed Krylov matvec)
static int outer_apply32(fde_handle* h, const double* x, double* y) {
  NvtxRange range("matvec_fp32");
  const int pi = h->pbeg(FDE_KCLASS_OUTER_FP32);
  RCHK((outer_passes<double, float, float>(
      h, x, y, h->xT, h->yT, h->logLx, h->logLy, h->S1x32, h->S2x32, h->twx32, h->cf32[0],
      h->cf32[1], h->S1y32, h->S2y32, h->twy32, h->cf32T[0], h->cf32T[1],
      reinterpret_cast<cx<float>*>(h->fft_ws), h->fft_ws_elems * 2)));
  h->pend(pi);
  return FDE_OK;
}

static int norm2(fde_handle* h, const double* x, double* dev_out, double* host_out) {
  int pi = h->pbeg(FDE_KCLASS_KRYLOV);
  LCHK(launch_sumsq(x, h->N, h->part, h->nb, h->st));
  LCHK(launch_reduce(h->part, 1, h->nb, dev_out, 2, h->st));
  h->pend(pi);
  if (host_out) {
    CCHK(cudaMemcpyAsync(host_out, dev_out, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CCHK(cudaStreamSynchronize(h->st));
  }
  return FDE_OK;
}

static int precond(fde_handle* h, const double* v, double* z, bool df_io = false) {
  NvtxRange range("vcycle");
  if (!h->mg) {
    CCHK(cudaMemcpyAsync(z, v, h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return FDE_OK;
  }
  return h->mg->vcycle(h, v, z, df_io);
}

// Multigrid as the solver (fde_params.solver = FDE_SOLVER_MG): the stationary
// iteration x <- x + V(b - M x) with the FP64-accurate residual as the test.
static int solve_mg(fde_handle* h, const double* b, double* x, fde_stats* st_out,
                    const double* x0) {
  const fde_params& p = h->p;
  const size_t N = h->N;
  fde_stats st{0, 1, 0, 0.0, 0};
  double bnorm = 0.0;
  RCHK(norm2(h, b, h->hdev, &bnorm));
  if (!std::isfinite(bnorm)) return h->fail(FDE_ERR_NONFINITE, "right-hand side is not finite");
  if (x0) CCHK(cudaMemcpyAsync(x, x0, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  else CCHK(cudaMemsetAsync(x, 0, N * sizeof(double), h->st));
  const double tol = p.rtol * bnorm;
  int status = FDE_ERR_NOT_CONVERGED;
  for (;;) {
    // r = b - M x (r = b while x = 0)
    if (x0 || st.iterations > 0) {
      RCHK(outer_apply(h, x, h->tmp, false));
      LCHK(launch_sub(N, b, h->tmp, h->tmp, h->st));
    } else {
      CCHK(cudaMemcpyAsync(h->tmp, b, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    }
    double rn = 0.0;
    RCHK(norm2(h, h->tmp, h->h2dev, &rn));
    if (!std::isfinite(rn)) return h->fail(FDE_ERR_NONFINITE, "non-finite residual");
    st.rel_residual = bnorm > 0.0 ? rn / bnorm : 0.0;
    if (rn <= tol) {
      status = FDE_OK;
      st.converged = 1;
      break;
    }
    if (st.iterations >= p.maxit) break;
    RCHK(precond(h, h->tmp, h->Z));
    LCHK(launch_lincomb(N, 1.0, x, 1.0, h->Z, 0.0, nullptr, x, h->st));
    st.iterations++;
  }
  if (st_out) *st_out = st;
  if (status == FDE_ERR_NOT_CONVERGED)
    h->fail(FDE_ERR_NOT_CONVERGED, "not converged: %d cycles, relative residual %.3e",
            st.iterations, st.rel_residual);
  return status;
}

static int solve_impl(fde_handle* h, const double* b, double* x, fde_stats* st_out,
                      const double* x0) {
  const fde_params& p = h->p;
  const size_t N = h->N;
  const int m = p.restart;
  fde_stats st{0, 0, 0, 0.0, 0};
  // With the double-float outer operator the Krylov vectors V and Z are kept
  // in double-float (hi, lo FP32 pairs in the same 8 bytes an element): the
  // Gram-Schmidt passes, matvecs and V-cycle ends then run on the FP32 pipes
  // (GB300 issues FP64 at 1/64 of the FP32 rate).  x, b and the true residual
  // stay FP64.
  const bool dfk = p.outer == FDE_OUTER_DF32 && m <= kDcgsMax;
  auto start_basis = [&](const double* r, const double* nrm_dev) {
    return dfk ? launch_scale_inv_df(N, r, nrm_dev, h->V, h->st)
               : launch_scale_inv(N, r, nrm_dev, h->V, h->st);
  };
  double bnorm = 0.0;
  RCHK(norm2(h, b, h->hdev, &bnorm));
  if (!std::isfinite(bnorm)) return h->fail(FDE_ERR_NONFINITE, "right-hand side is not finite");
  if (bnorm == 0.0) {
    CCHK(cudaMemsetAsync(x, 0, N * sizeof(double), h->st));
    st.converged = 1;
    if (st_out) *st_out = st;
    CCHK(cudaStreamSynchronize(h->st));
    return FDE_OK;
  }
  double beta = bnorm;
  if (x0) {
    // warm start: FGMRES on the correction, from r_0 = b - M x_0
    CCHK(cudaMemcpyAsync(x, x0, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    RCHK(outer_apply(h, x, h->tmp, false));
    LCHK(launch_sub(N, b, h->tmp, h->tmp, h->st));
    RCHK(norm2(h, h->tmp, h->h2dev, &beta));
    if (!std::isfinite(beta)) return h->fail(FDE_ERR_NONFINITE, "non-finite residual");
    st.rel_residual = beta / bnorm;
    if (beta <= p.rtol * bnorm) {
      st.converged = 1;
      if (st_out) *st_out = st;
      return FDE_OK;
    }
    LCHK(start_basis(h->tmp, h->h2dev));
  } else {
    CCHK(cudaMemsetAsync(x, 0, N * sizeof(double), h->st));
    // V_0 = b / ||b||
    LCHK(start_basis(b, h->hdev));
  }
  const double tol = p.rtol * bnorm;
  const size_t ldv = h->ldv;
  const size_t Ne = (N + 1) / 2 * 2;  // even length covered by the zero padding
  const double* beta_dev = x0 ? h->h2dev : h->hdev;
  int status = FDE_ERR_NOT_CONVERGED;
  while (st.iterations < p.maxit) {
    st.restarts++;
    // g = (beta, 0, ...) on the device
    LCHK(launch_arnoldi_start(h->ast, beta_dev, h->st));
    double gprev = beta;  // residual estimate before the step (|g_j|)
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* Vj = h->V + (size_t)j * ldv;
      double* Zj = h->Z + (size_t)j * ldv;
      double* w = h->V + (size_t)(j + 1) * ldv;
      RCHK(precond(h, Vj, Zj, dfk));
      // relaxed matvec once the residual estimate is near the target
      if (p.relax && gprev <= FDE_RELAX_FACTOR * tol) {
        RCHK(dfk ? outer_apply32_df(h, Zj, w) : outer_apply32(h, Zj, w));
        st.relaxed++;
      } else {
        RCHK(dfk ? outer_apply_df(h, Zj, w) : outer_apply(h, Zj, w, false));
      }
      NvtxRange arnoldi("cgs2");
      int pi = h->pbeg(FDE_KCLASS_KRYLOV);
      if (m <= kDcgsMax) {
        // two fused passes over V (V_j re-orthogonalised one step late), Givens
        // updates in their last blocks, w /= ||w||
        LCHK(launch_dcgs2(h->V, ldv, j, Ne, h->cgs_part, h->tickets, h->dcgs_coef, h->ast, dfk,
                          h->st));
        h->launches += 2;  // three kernels, one counted by LCHK
      } else if (j + 1 <= 32) {
        // three fused passes over V, Givens update in the last block, w /= ||w||
        LCHK(launch_cgs2(h->V, ldv, j + 1, w, Ne, h->cgs_part, h->tickets, h->hdev, h->h2dev,
                         h->ast, j, h->st));
        h->launches += 3;  // four kernels, one counted by LCHK
      } else {
        // longer bases: separate dot and update passes, then the same column update
        LCHK(launch_dots(h->V, ldv, j + 1, w, N, h->part, h->nb, h->st));
        LCHK(launch_reduce(h->part, j + 1, h->nb, h->hdev, 0, h->st));
        LCHK(launch_axpy_dots(h->V, ldv, j + 1, h->hdev, w, N, h->part, h->nb, 0, h->st));
        LCHK(launch_dots(h->V, ldv, j + 1, w, N, h->part, h->nb, h->st));
        LCHK(launch_reduce(h->part, j + 1, h->nb, h->h2dev, 0, h->st));
        LCHK(launch_axpy_dots(h->V, ldv, j + 1, h->h2dev, w, N, h->part, h->nb, 1, h->st));
        LCHK(launch_reduce(h->part, 1, h->nb, h->ydev, 0, h->st));
        LCHK(launch_arnoldi_column(h->ast, j, h->hdev, h->h2dev, h->ydev, h->st));
        LCHK(launch_scale_by(w, Ne, h->ast.status, h->st));
      }
      h->pend(pi);
      CCHK(cudaMemcpyAsync(h->status_host, h->ast.status, sizeof(ArnoldiStatus),
                           cudaMemcpyDeviceToHost, h->st));
      CCHK(cudaStreamSynchronize(h->st));
      const ArnoldiStatus as = *h->status_host;
      if (as.nonfinite)
        return h->fail(FDE_ERR_NONFINITE, "non-finite Hessenberg entry at iteration %d",
                       st.iterations + 1);
      st.iterations++;
      k = j + 1;
      gprev = as.gabs;
      if (as.gabs <= tol || st.iterations >= p.maxit || as.hnext == 0.0) break;
    }
    // y = R^{-1} g, x += Z y (on the device)
    int pi = h->pbeg(FDE_KCLASS_KRYLOV);
    LCHK(launch_arnoldi_lsq(h->ast, k, h->ydev, h->st));
    // an earlier cycle's copy of x to the host must have read x first
    if (h->early_issued) CCHK(cudaStreamWaitEvent(h->st, h->x_copied, 0));
    LCHK(dfk ? launch_update_df(h->Z, ldv, k, h->ydev, x, N, h->st)
             : launch_update(h->Z, ldv, k, h->ydev, x, N, h->st));
    h->pend(pi);
    if (h->early_out) {
      // fde_step_host: copy this x to the host while the true residual is
      // formed; if the cycle converges it is the result
      CCHK(cudaEventRecord(h->x_ready, h->st));
      CCHK(cudaStreamWaitEvent(h->copy_st, h->x_ready, 0));
      CCHK(cudaMemcpyAsync(h->early_out, x, N * sizeof(double), cudaMemcpyDeviceToHost,
                           h->copy_st));
      CCHK(cudaEventRecord(h->x_copied, h->copy_st));
      h->early_issued = true;
    }
    // true residual in FP64
    RCHK(outer_apply(h, x, h->tmp, false));
    LCHK(launch_sub(N, b, h->tmp, h->tmp, h->st));
    RCHK(norm2(h, h->tmp, h->h2dev, &beta));
    if (!std::isfinite(beta)) return h->fail(FDE_ERR_NONFINITE, "non-finite residual");
    st.rel_residual = beta / bnorm;
    if (beta <= tol) {
      status = FDE_OK;
      st.converged = 1;
      break;
    }
    if (st.iterations >= p.maxit) break;
    LCHK(start_basis(h->tmp, h->h2dev));
    beta_dev = h->h2dev;
  }
  if (st_out) *st_out = st;
  if (status == FDE_ERR_NOT_CONVERGED)
    h->fail(FDE_ERR_NOT_CONVERGED, "not converged: %d iterations, relative residual %.3e",
            st.iterations, st.rel_residual);
  return status;
}

// ============================================================================
// C ABI

extern "C" {

void fde_default_params(fde_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->alpha = 1.5;
  p->beta = 1.5;
  p->qx = p->qy = 0;
  p->a1 = p->a2 = 0.0;
  p->b1 = p->b2 = 1.0;
  p->n1 = p->n2 = 63;
  p->dt = 1.0 / 64.0;
  p->rtol = 1e-8;
  p->restart = 30;
  p->maxit = 1000;
  p->precond = FDE_PRECOND_MG_SG;
  p->nu_pre = 1;
  p->nu_post = 1;
  p->omega = 0.7;
  p->coarsest_n = 8;
  p->precision = FDE_PREC_FP64;
  p->toeplitz_path = FDE_PATH_AUTO;
  p->outer = FDE_OUTER_FP64;
  p->cycles = 1;
}

static int validate(const fde_params* p, std::string& why) {
  char buf[256];
  auto bad = [&](const char* m) { why = m; return FDE_ERR_ARG; };
  if (!(p->alpha > 1.0 && p->alpha < 2.0) || !(p->beta > 1.0 && p->beta < 2.0))
    return bad("alpha and beta must lie in (1, 2)");
  if ((p->qx != 0 && p->qx != -1) || (p->qy != 0 && p->qy != -1)) return bad("q must be 0 or -1");
  if (!(p->b1 > p->a1) || !(p->b2 > p->a2)) return bad("empty domain");
  if (p->n1 < 3 || p->n2 < 3 || p->n1 > 8191 || p->n2 > 8191) return bad("n1, n2 must be in [3, 8191]");
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return bad("dt must be positive");
  if (!(p->rtol > 0.0) || !(p->rtol < 1.0)) return bad("rtol must be in (0, 1)");
  if (p->restart < 1 || p->restart > 64) return bad("restart must be in [1, 64]");
  if (p->maxit < 1) return bad("maxit must be >= 1");
  if (p->precond < FDE_PRECOND_NONE || p->precond > FDE_PRECOND_MG_EXACT)
    return bad("unknown precond");
  if (p->precond == FDE_PRECOND_MG_EXACT && p->precision != FDE_PREC_FP64)
    return bad("the exact-Galerkin validation mode runs in FP64 only");
  if (p->cycles < 0 || p->cycles > 4) return bad("cycles must be in [0, 4]");
  if (p->relax != 0 && p->relax != 1) return bad("relax must be 0 or 1");
  if (p->solver != FDE_SOLVER_FGMRES && p->solver != FDE_SOLVER_MG) return bad("unknown solver");
  if (p->solver == FDE_SOLVER_MG && p->precond == FDE_PRECOND_NONE)
    return bad("the multigrid solver needs a multigrid precond");
  if (p->warm != 0 && p->warm != 1) return bad("warm must be 0 or 1");
  if (p->nu_pre < 0 || p->nu_pre > 4 || p->nu_post < 0 || p->nu_post > 4) return bad("nu in [0, 4]");
  if (!(p->omega > 0.0 && p->omega < 2.0)) return bad("omega must be in (0, 2)");
  if (p->coarsest_n < 1) return bad("coarsest_n must be >= 1");
  if (p->precision < FDE_PREC_FP64 || p->precision > FDE_PREC_BF16X3) return bad("unknown precision");
  if (p->toeplitz_path < FDE_PATH_AUTO || p->toeplitz_path > FDE_PATH_TUNE) return bad("unknown toeplitz_path");
  if (p->outer != FDE_OUTER_FP64 && p->outer != FDE_OUTER_DF32) return bad("unknown outer");
  const int L1 = ceil_log2(2L * p->n1 - 1), L2 = ceil_log2(2L * p->n2 - 1);
  if (L1 > 13 || L2 > 13) {
    snprintf(buf, sizeof(buf), "FP64 FFT apply supports n <= 4096 (got %d x %d)", p->n1, p->n2);
    why = buf;
    return FDE_ERR_UNSUPPORTED;
  }
  return FDE_OK;
}

int fde_create(const fde_params* pin, void* stream, fde_handle** out) {
  if (!out) return FDE_ERR_ARG;
  *out = nullptr;
  if (!pin) {
    g_create_error = "null params";
    return FDE_ERR_ARG;
  }
  std::string why;
  int v = validate(pin, why);
  if (v != FDE_OK) {
    g_create_error = why;
    return v;
  }
  std::unique_ptr<fde_handle> hp(new fde_handle());
  fde_handle* h = hp.get();
  h->p = *pin;
  h->st = (cudaStream_t)stream;
  const fde_params& p = h->p;
  h->n1 = p.n1;
  h->n2 = p.n2;
  h->N = (size_t)p.n1 * p.n2;
  h->hx = (p.b1 - p.a1) / (p.n1 + 1);
  h->hy = (p.b2 - p.a2) / (p.n2 + 1);
  const double r = p.dt / (2.0 * std::pow(h->hx, p.alpha));  // Eq. (system)
  const double s = p.dt / (2.0 * std::pow(h->hy, p.beta));
  h->c = 1.0 / r;
  h->sigma = s / r;
  h->two_h_alpha = 2.0 * std::pow(h->hx, p.alpha);
  const size_t N = h->N;
  int rc = FDE_OK;
  auto setup = [&]() -> int {
    CCHK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    RCHK(h->alloc(&h->wx, p.n1 + 2));
    RCHK(h->alloc(&h->wy, p.n2 + 2));
    RCHK(h->alloc(&h->tx0, p.n1 + 2));
    RCHK(h->alloc(&h->ty0, p.n2 + 2));
    LCHK(launch_wsgd_weights(p.alpha, p.qx, p.n1 + 1, h->wx, h->st));
    LCHK(launch_wsgd_weights(p.beta, p.qy, p.n2 + 1, h->wy, h->st));
    LCHK(launch_generator_from_weights(h->wx, p.n1, 1.0, h->tx0, h->st));
    LCHK(launch_generator_from_weights(h->wy, p.n2, 1.0, h->ty0, h->st));
    h->logLx = ceil_log2(2L * p.n1 - 1);
    h->logLy = ceil_log2(2L * p.n2 - 1);
    {
      const int lmax = std::max(h->logLx, h->logLy);
      if (fft_pass_two_buffer_bytes(lmax, sizeof(cx<double>)) > 227 * 1024) {
        h->fft_ws_elems = (size_t)152 << lmax;  // one CTA per SM, L entries each
        RCHK(h->alloc(&h->fft_ws, h->fft_ws_elems));
      }
    }
    RCHK(h->alloc(&h->S1x, (size_t)1 << h->logLx));
    RCHK(h->alloc(&h->S2x, (size_t)1 << h->logLx));
    RCHK(h->alloc(&h->twx, (size_t)1 << h->logLx));
    RCHK(h->alloc(&h->S1y, (size_t)1 << h->logLy));
    RCHK(h->alloc(&h->S2y, (size_t)1 << h->logLy));
    RCHK(h->alloc(&h->twy, (size_t)1 << h->logLy));
    LCHK(launch_build_spectra<double>(h->tx0, p.n1, h->logLx, 1.0, h->S1x, h->S2x, h->twx, h->st, h->fft_ws));
    LCHK(launch_build_spectra<double>(h->ty0, p.n2, h->logLy, 1.0, h->S1y, h->S2y, h->twy, h->st, h->fft_ws));
    if (p.outer == FDE_OUTER_DF32) {
      RCHK(h->alloc(&h->S1xd, (size_t)1 << h->logLx));
      RCHK(h->alloc(&h->S2xd, (size_t)1 << h->logLx));
      RCHK(h->alloc(&h->twxd, (size_t)1 << h->logLx));
      RCHK(h->alloc(&h->S1yd, (size_t)1 << h->logLy));
      RCHK(h->alloc(&h->S2yd, (size_t)1 << h->logLy));
      RCHK(h->alloc(&h->twyd, (size_t)1 << h->logLy));
      LCHK(launch_build_spectra<df>(h->tx0, p.n1, h->logLx, 1.0, h->S1xd, h->S2xd, h->twxd, h->st, h->fft_ws));
      LCHK(launch_build_spectra<df>(h->ty0, p.n2, h->logLy, 1.0, h->S1yd, h->S2yd, h->twyd, h->st, h->fft_ws));
      for (int k = 0; k < 4; ++k) {
        RCHK(h->alloc(&h->cfN[k], N));
        RCHK(h->alloc(&h->cfO[k], N));
      }
      for (int k = 0; k < 2; ++k) {
        RCHK(h->alloc(&h->cfNT[k], N));
        RCHK(h->alloc(&h->cfOT[k], N));
      }
    }
    if (p.relax) {
      RCHK(h->alloc(&h->S1x32, (size_t)1 << h->logLx));
      RCHK(h->alloc(&h->S2x32, (size_t)1 << h->logLx));
      RCHK(h->alloc(&h->twx32, (size_t)1 << h->logLx));
      RCHK(h->alloc(&h->S1y32, (size_t)1 << h->logLy));
      RCHK(h->alloc(&h->S2y32, (size_t)1 << h->logLy));
      RCHK(h->alloc(&h->twy32, (size_t)1 << h->logLy));
      LCHK(launch_build_spectra<float>(h->tx0, p.n1, h->logLx, 1.0, h->S1x32, h->S2x32, h->twx32,
                                       h->st, h->fft_ws));
      LCHK(launch_build_spectra<float>(h->ty0, p.n2, h->logLy, 1.0, h->S1y32, h->S2y32, h->twy32,
                                       h->st, h->fft_ws));
      for (int k = 0; k < 2; ++k) {
        RCHK(h->alloc(&h->cf32[k], N));
        RCHK(h->alloc(&h->cf32T[k], N));
      }
    }
    double** fields[] = {&h->dpN, &h->dmN, &h->epN, &h->emN, &h->epNs, &h->emNs,
                         &h->dpO, &h->dmO, &h->epOs, &h->emOs, &h->tmp, &h->bwork,
                         &h->hu, &h->hv, &h->hx_out, &h->u_last, &h->epNsT, &h->emNsT,
                         &h->epOsT, &h->emOsT, &h->xT, &h->yT};
    for (double** f : fields) RCHK(h->alloc(f, N));
    h->ldv = (N + 63) / 64 * 64;
    RCHK(h->alloc(&h->V, h->ldv * (size_t)(p.restart + 1)));
    RCHK(h->alloc(&h->Z, h->ldv * (size_t)p.restart));
    // the padding between columns must read as zero in the Gram-Schmidt passes
    CCHK(cudaMemsetAsync(h->V, 0, h->ldv * (size_t)(p.restart + 1) * sizeof(double), h->st));
    CCHK(cudaMemsetAsync(h->Z, 0, h->ldv * (size_t)p.restart * sizeof(double), h->st));
    h->nb = krylov_blocks();
    RCHK(h->alloc(&h->part, (size_t)h->nb * (p.restart + 2)));
    // the first Gram-Schmidt pass writes KMAX + 1 <= 33 sums (projections, ||w||^2)
    RCHK(h->alloc(&h->hdev, std::max(p.restart + 4, 40)));
    RCHK(h->alloc(&h->h2dev, p.restart + 4));
    RCHK(h->alloc(&h->ydev, p.restart + 4));
    RCHK(h->alloc(&h->cgs_part, (size_t)cgs_blocks() * (2 * kDcgsMax + 2) + 8));
    RCHK(h->alloc(&h->dcgs_coef, kDcgsCoef));
    RCHK(h->alloc(&h->tickets, 4));
    CCHK(cudaMemsetAsync(h->tickets, 0, 4 * sizeof(unsigned), h->st));
    {
      const int mm = p.restart;
      double* a = nullptr;
      RCHK(h->alloc(&a, 2 * (size_t)(mm + 1) * mm + 4 * (size_t)mm + 2));
      h->ast.m = mm;
      h->ast.R = a;
      h->ast.cs = a + (size_t)(mm + 1) * mm;
      h->ast.sn = h->ast.cs + mm;
      h->ast.g = h->ast.sn + mm;               // m + 1 entries
      h->ast.H = h->ast.g + mm + 1;            // (m + 1) x m
      h->ast.gpre = h->ast.H + (size_t)(mm + 1) * mm;
      RCHK(h->alloc(&h->ast.status, 1));
      CCHK(cudaMallocHost(&h->status_host, sizeof(ArnoldiStatus)));
    }
    if (p.precond == FDE_PRECOND_MG_EXACT) {
      auto* mg = new DenseMG();
      h->mg.reset(mg);
      RCHK(mg->create(h));
    } else if (p.precond == FDE_PRECOND_P2) {
      if (p.precision == FDE_PREC_FP64) {
        auto* mg = new StencilMG<double>();
        h->mg.reset(mg);
        RCHK(mg->create(h));
      } else {
        auto* mg = new StencilMG<float>();
        h->mg.reset(mg);
        RCHK(mg->create(h));
      }
    } else if (p.precond != FDE_PRECOND_NONE) {
      if (p.precision == FDE_PREC_FP64) {
        auto* mg = new MG<double>();
        h->mg.reset(mg);
        RCHK(mg->create(h));
      } else {
        auto* mg = new MG<float>();
        h->mg.reset(mg);
        RCHK(mg->create(h));
      }
    }
    CCHK(cudaStreamSynchronize(h->st));
    return FDE_OK;
  };
  rc = setup();
  if (rc != FDE_OK) {
    g_create_error = h->err;
    fde_destroy(hp.release());
    return rc;
  }
  *out = hp.release();
  return FDE_OK;
}

void fde_destroy(fde_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  h->mg.reset();
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (h->copy_st) cudaStreamSynchronize(h->copy_st), cudaStreamDestroy(h->copy_st);
  if (h->v_ready) cudaEventDestroy(h->v_ready);
  if (h->x_ready) cudaEventDestroy(h->x_ready);
  if (h->x_copied) cudaEventDestroy(h->x_copied);
  for (void* q : h->allocs) cudaFree(q);
  for (auto& pe : h->pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
  if (h->status_host) cudaFreeHost(h->status_host);
  delete h;
}

const char* fde_last_error(const fde_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

int fde_set_coefficients(fde_handle* h, int which, const double* dp, const double* dm,
                         const double* ep, const double* em) {
  if (!h) return FDE_ERR_ARG;
  if (!dp || !dm || !ep || !em) return h->fail(FDE_ERR_ARG, "null coefficient pointer");
  if (which != FDE_COEF_NEW && which != FDE_COEF_OLD) return h->fail(FDE_ERR_ARG, "bad `which`");
  const size_t N = h->N;
  if (which == FDE_COEF_NEW) {
    CCHK(cudaMemcpyAsync(h->dpN, dp, N * 8, cudaMemcpyDeviceToDevice, h->st));
    CCHK(cudaMemcpyAsync(h->dmN, dm, N * 8, cudaMemcpyDeviceToDevice, h->st));
    CCHK(cudaMemcpyAsync(h->epN, ep, N * 8, cudaMemcpyDeviceToDevice, h->st));
    CCHK(cudaMemcpyAsync(h->emN, em, N * 8, cudaMemcpyDeviceToDevice, h->st));
    LCHK((launch_convert<double, double>(N, ep, h->sigma, h->epNs, h->st)));
    LCHK((launch_convert<double, double>(N, em, h->sigma, h->emNs, h->st)));
    LCHK(launch_transpose<double>(h->epNs, h->n2, h->n1, h->epNsT, 0, h->st));
    LCHK(launch_transpose<double>(h->emNs, h->n2, h->n1, h->emNsT, 0, h->st));
    if (h->p.outer == FDE_OUTER_DF32) {
      LCHK(launch_to_df(N, dp, 1.0, h->cfN[0], h->st));
      LCHK(launch_to_df(N, dm, 1.0, h->cfN[1], h->st));
      LCHK(launch_to_df(N, ep, h->sigma, h->cfN[2], h->st));
      LCHK(launch_to_df(N, em, h->sigma, h->cfN[3], h->st));
      LCHK(launch_to_df(N, h->epNsT, 1.0, h->cfNT[0], h->st));
      LCHK(launch_to_df(N, h->emNsT, 1.0, h->cfNT[1], h->st));
    }
    if (h->p.relax) {
      LCHK((launch_convert<double, float>(N, dp, 1.0, h->cf32[0], h->st)));
      LCHK((launch_convert<double, float>(N, dm, 1.0, h->cf32[1], h->st)));
      LCHK((launch_convert<double, float>(N, h->epNsT, 1.0, h->cf32T[0], h->st)));
      LCHK((launch_convert<double, float>(N, h->emNsT, 1.0, h->cf32T[1], h->st)));
    }
    h->have_new = true;
    if (h->mg) RCHK(h->mg->setup(h));
  } else {
    CCHK(cudaMemcpyAsync(h->dpO, dp, N * 8, cudaMemcpyDeviceToDevice, h->st));
    CCHK(cudaMemcpyAsync(h->dmO, dm, N * 8, cudaMemcpyDeviceToDevice, h->st));
    LCHK((launch_convert<double, double>(N, ep, h->sigma, h->epOs, h->st)));
    LCHK((launch_convert<double, double>(N, em, h->sigma, h->emOs, h->st)));
    LCHK(launch_transpose<double>(h->epOs, h->n2, h->n1, h->epOsT, 0, h->st));
    LCHK(launch_transpose<double>(h->emOs, h->n2, h->n1, h->emOsT, 0, h->st));
    if (h->p.outer == FDE_OUTER_DF32) {
      LCHK(launch_to_df(N, dp, 1.0, h->cfO[0], h->st));
      LCHK(launch_to_df(N, dm, 1.0, h->cfO[1], h->st));
      LCHK(launch_to_df(N, ep, h->sigma, h->cfO[2], h->st));
      LCHK(launch_to_df(N, em, h->sigma, h->cfO[3], h->st));
      LCHK(launch_to_df(N, h->epOsT, 1.0, h->cfOT[0], h->st));
      LCHK(launch_to_df(N, h->emOsT, 1.0, h->cfOT[1], h->st));
    }
    h->have_old = true;
  }
  return FDE_OK;
}

// b = c u - A^(m-1) u + 2 h^a v = 2c u - M^(m-1) u + 2 h^a v; v_ready (may be
// null): an event the stream waits for before v is first read
static int rhs_impl(fde_handle* h, const double* u_prev, const double* v_half, double* b,
                    cudaEvent_t v_ready) {
  if (!h->have_old) return h->fail(FDE_ERR_ARG, "FDE_COEF_OLD coefficients not set");
  RCHK(outer_apply(h, u_prev, h->tmp, true));
  if (v_ready) CCHK(cudaStreamWaitEvent(h->st, v_ready, 0));
  LCHK(launch_lincomb(h->N, 2.0 * h->c, u_prev, -1.0, h->tmp, h->two_h_alpha, v_half, b, h->st));
  return FDE_OK;
}

int fde_rhs(fde_handle* h, const double* u_prev, const double* v_half, double* b) {
  if (!h) return FDE_ERR_ARG;
  if (!u_prev || !v_half || !b) return h->fail(FDE_ERR_ARG, "null pointer");
  return rhs_impl(h, u_prev, v_half, b, nullptr);
}

int fde_apply(fde_handle* h, const double* x, double* y) {
  if (!h) return FDE_ERR_ARG;
  if (!x || !y || x == y) return h->fail(FDE_ERR_ARG, "null or aliased pointer");
  if (!h->have_new) return h->fail(FDE_ERR_ARG, "FDE_COEF_NEW coefficients not set");
  return outer_apply(h, x, y, false);
}

int fde_vcycle(fde_handle* h, const double* r, double* z) {
  if (!h) return FDE_ERR_ARG;
  if (!r || !z) return h->fail(FDE_ERR_ARG, "null pointer");
  if (!h->have_new) return h->fail(FDE_ERR_ARG, "FDE_COEF_NEW coefficients not set");
  return precond(h, r, z);
}

int fde_level_apply(fde_handle* h, int level, const double* x, double* y) {
  if (!h) return FDE_ERR_ARG;
  if (!x || !y) return h->fail(FDE_ERR_ARG, "null pointer");
  if (!h->have_new) return h->fail(FDE_ERR_ARG, "FDE_COEF_NEW coefficients not set");
  if (!h->mg) return h->fail(FDE_ERR_ARG, "no multigrid hierarchy (precond NONE)");
  return h->mg->level_apply(h, level, x, y);
}

int fde_levels(const fde_handle* h, int* levels, int* n1s, int* n2s) {
  if (!h) return FDE_ERR_ARG;
  const int L = h->mg ? (int)h->mg->n1s.size() : 1;
  if (levels) *levels = L;
  for (int l = 0; l < L; ++l) {
    if (n1s) n1s[l] = h->mg ? h->mg->n1s[l] : h->n1;
    if (n2s) n2s[l] = h->mg ? h->mg->n2s[l] : h->n2;
  }
  return FDE_OK;
}

int fde_level_path(const fde_handle* h, int level) {
  if (!h || !h->mg) return -1;
  return h->mg->level_path(level);
}

int fde_weights(const fde_handle* hc, int axis, double* w_host, int count) {
  fde_handle* h = const_cast<fde_handle*>(hc);
  if (!h) return FDE_ERR_ARG;
  const int n = axis == 0 ? h->n1 : h->n2;
  if (!w_host || count < 0 || count > n + 2 || (axis != 0 && axis != 1))
    return h->fail(FDE_ERR_ARG, "bad weights request");
  CCHK(cudaMemcpyAsync(w_host, axis == 0 ? h->wx : h->wy, count * sizeof(double),
                       cudaMemcpyDeviceToHost, h->st));
  CCHK(cudaStreamSynchronize(h->st));
  return FDE_OK;
}

int fde_solve(fde_handle* h, const double* b, double* x, fde_stats* st) {
  if (!h) return FDE_ERR_ARG;
  if (!b || !x || b == x) return h->fail(FDE_ERR_ARG, "null or aliased pointer");
  if (!h->have_new) return h->fail(FDE_ERR_ARG, "FDE_COEF_NEW coefficients not set");
  NvtxRange range("fde_solve");
  int r = h->p.solver == FDE_SOLVER_MG ? solve_mg(h, b, x, st, nullptr)
                                       : solve_impl(h, b, x, st, nullptr);
  h->prof_collect();
  if (h->mg && h->mg->device_error(h))
    return h->fail(FDE_ERR_TIMEOUT, "a capped device-side wait gave up during the solve");
  return r;
}

int fde_conversion_selftest(long long n, long long* mismatches) {
  if (n < 1 || !mismatches) return FDE_ERR_ARG;
  if (conversion_selftest(n, mismatches)) return FDE_ERR_CUDA;
  return FDE_OK;
}

int fde_wait_selftest(fde_handle* h, int complete) {
  if (!h) return FDE_ERR_ARG;
  if (complete != 0 && complete != 1) return h->fail(FDE_ERR_ARG, "complete must be 0 or 1");
  const int r = h->mg ? h->mg->wait_selftest(h, complete) : -1;
  if (r < 0) return h->fail(FDE_ERR_UNSUPPORTED, "the handle has no tensor-core level");
  if (r > 0) return h->fail(FDE_ERR_CUDA, "bounded-wait self-test launch failed");
  return FDE_OK;
}

static int step_impl(fde_handle* h, const double* u_prev, const double* v_half, double* u_next,
                     fde_stats* st, cudaEvent_t v_ready) {
  RCHK(rhs_impl(h, u_prev, v_half, h->bwork, v_ready));
  if (!h->have_new) return h->fail(FDE_ERR_ARG, "FDE_COEF_NEW coefficients not set");
  const double* x0 = h->p.warm ? u_prev : nullptr;
  NvtxRange range("fde_step");
  int r = h->p.solver == FDE_SOLVER_MG ? solve_mg(h, h->bwork, u_next, st, x0)
                                       : solve_impl(h, h->bwork, u_next, st, x0);
  h->prof_collect();
  if (h->mg && h->mg->device_error(h))
    return h->fail(FDE_ERR_TIMEOUT, "a capped device-side wait gave up during the step");
  if (r == FDE_OK || r == FDE_ERR_NOT_CONVERGED) {
    CCHK(cudaMemcpyAsync(h->u_last, u_next, h->N * 8, cudaMemcpyDeviceToDevice, h->st));
    h->m++;
  }
  return r;
}

int fde_step(fde_handle* h, const double* u_prev, const double* v_half, double* u_next,
             fde_stats* st) {
  if (!h) return FDE_ERR_ARG;
  if (!u_prev || !v_half || !u_next || u_prev == u_next)
    return h->fail(FDE_ERR_ARG, "null or aliased pointer");
  return step_impl(h, u_prev, v_half, u_next, st, nullptr);
}

int fde_step_host(fde_handle* h, const double* u_prev_host, const double* v_half_host,
                  double* u_next_host, fde_stats* st) {
  if (!h) return FDE_ERR_ARG;
  if (!u_prev_host || !v_half_host || !u_next_host)
    return h->fail(FDE_ERR_ARG, "null pointer");
  if (!h->copy_st) {
    CCHK(cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking));
    CCHK(cudaEventCreateWithFlags(&h->v_ready, cudaEventDisableTiming));
    CCHK(cudaEventCreateWithFlags(&h->x_ready, cudaEventDisableTiming));
    CCHK(cudaEventCreateWithFlags(&h->x_copied, cudaEventDisableTiming));
  }
  // copies run beside the computation only from page-locked host memory (from
  // pageable memory an asynchronous copy blocks the host until it is done)
  auto pinned = [](const void* p) {
    cudaPointerAttributes a{};
    const bool ok = cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost;
    cudaGetLastError();
    return ok;
  };
  CCHK(cudaMemcpyAsync(h->hu, u_prev_host, h->N * 8, cudaMemcpyHostToDevice, h->st));
  // the source is first read after the right-hand side's operator apply of
  // u: its upload overlaps that apply (the previous call ended with a stream
  // synchronisation, so nothing still reads h->hv)
  cudaEvent_t v_ready = nullptr;
  if (pinned(v_half_host)) {
    CCHK(cudaMemcpyAsync(h->hv, v_half_host, h->N * 8, cudaMemcpyHostToDevice, h->copy_st));
    CCHK(cudaEventRecord(h->v_ready, h->copy_st));
    v_ready = h->v_ready;
  } else {
    CCHK(cudaMemcpyAsync(h->hv, v_half_host, h->N * 8, cudaMemcpyHostToDevice, h->st));
  }
  // the FGMRES solve copies each cycle's x to u_next_host while it checks the
  // true residual; the copy of the last cycle's x is the result
  const bool early = h->p.solver == FDE_SOLVER_FGMRES && pinned(u_next_host);
  h->early_out = early ? u_next_host : nullptr;
  h->early_issued = false;
  int r = step_impl(h, h->hu, h->hv, h->hx_out, st, v_ready);
  h->early_out = nullptr;
  const bool copied = h->early_issued;
  h->early_issued = false;
  if (r != FDE_OK && r != FDE_ERR_NOT_CONVERGED) {
    cudaStreamSynchronize(h->copy_st);
    return r;
  }
  if (copied) CCHK(cudaStreamSynchronize(h->copy_st));
  else CCHK(cudaMemcpyAsync(u_next_host, h->hx_out, h->N * 8, cudaMemcpyDeviceToHost, h->st));
  CCHK(cudaStreamSynchronize(h->st));
  return r;
}

int fde_get_state(const fde_handle* hc, int* m, double* u_out) {
  fde_handle* h = const_cast<fde_handle*>(hc);
  if (!h) return FDE_ERR_ARG;
  if (m) *m = h->m;
  if (u_out)
    CCHK(cudaMemcpyAsync(u_out, h->u_last, h->N * 8, cudaMemcpyDeviceToDevice, h->st));
  return FDE_OK;
}

int fde_set_state(fde_handle* h, int m) {
  if (!h) return FDE_ERR_ARG;
  if (m < 0) return h->fail(FDE_ERR_ARG, "negative step counter");
  h->m = m;
  return FDE_OK;
}

int fde_profile_enable(fde_handle* h, int on) {
  if (!h) return FDE_ERR_ARG;
  h->prof_collect();
  h->prof = on != 0;
  for (int k = 0; k < FDE_KCLASS_COUNT; ++k) {
    h->prof_launches[k] = 0;
    h->prof_ms[k] = 0.0;
  }
  return FDE_OK;
}

int fde_profile_query(fde_handle* h, int kclass, long long* launches, double* ms) {
  if (!h) return FDE_ERR_ARG;
  if (kclass < 0 || kclass >= FDE_KCLASS_COUNT) return h->fail(FDE_ERR_ARG, "bad kernel class");
  h->prof_collect();
  if (launches) *launches = h->prof_launches[kclass];
  if (ms) *ms = h->prof_ms[kclass];
  return FDE_OK;
}

long long fde_launch_count(const fde_handle* h) { return h ? h->launches : 0; }

}  // extern "C"

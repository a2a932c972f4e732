// Private to libfde: the solver handle and the multigrid hierarchies behind
// the C ABI of include/fde.h (Sec. 4: V-cycles with structured-Galerkin,
// rediscretised, exact-Galerkin or P_2 levels), shared by the single-problem
// driver (fde.cu) and the grouped batch engine (fde_group.cu).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "df32.cuh"
#include "tc_gemm.h"
#include "../../include/fde.h"

namespace fde {
// message returned by fde_last_error(NULL) for calls without a handle
void set_global_error(const char* msg);
}  // namespace fde

static inline int ceil_log2(long v) {
  int l = 0;
  while ((1L << l) < v) ++l;
  return l;
}

struct ProfEvent {
  int kclass;
  cudaEvent_t a, b;
};

using namespace fde;

// NVTX range for profilers (no cost without an attached tool)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct MGBase;

struct fde_handle {
  fde_params p{};
  cudaStream_t st = nullptr;
  cudaStream_t cap_st = nullptr;  // private stream on which V-cycles are captured into graphs
  // fde_step_host: the source's upload runs on copy_st, beside the right-hand
  // side's operator apply, and v_ready orders it before its first use
  cudaStream_t copy_st = nullptr;
  cudaEvent_t v_ready = nullptr;
  // ... and each FGMRES cycle's x is copied to early_out (page-locked host
  // memory) beside the true-residual check: x_ready orders the copy after
  // the update, x_copied a later update after the copy
  double* early_out = nullptr;
  bool early_issued = false;
  cudaEvent_t x_ready = nullptr, x_copied = nullptr;
  std::string err;
  long long launches = 0;
  int n1 = 0, n2 = 0;
  size_t N = 0;
  double hx = 0, hy = 0, c = 0, sigma = 0, two_h_alpha = 0;
  std::vector<void*> allocs;

  // weights and the FP64 outer operator (generator t = -w, spectra, coefficients)
  double *wx = nullptr, *wy = nullptr, *tx0 = nullptr, *ty0 = nullptr;
  int logLx = 0, logLy = 0;
  cx<double> *S1x = nullptr, *S2x = nullptr, *S1y = nullptr, *S2y = nullptr;
  cx<double> *twx = nullptr, *twy = nullptr;
  double *dpN = nullptr, *dmN = nullptr, *epN = nullptr, *emN = nullptr;  // unscaled, t^(m)
  double *epNs = nullptr, *emNs = nullptr;                                 // sigma-scaled
  double *dpO = nullptr, *dmO = nullptr, *epOs = nullptr, *emOs = nullptr;  // t^(m-1)
  // double-float copies for the df32 outer apply: {dp, dm, sigma ep, sigma em}
  cx<df> *S1xd = nullptr, *S2xd = nullptr, *S1yd = nullptr, *S2yd = nullptr, *twxd = nullptr,
         *twyd = nullptr;
  df *cfN[4] = {nullptr, nullptr, nullptr, nullptr}, *cfO[4] = {nullptr, nullptr, nullptr, nullptr};
  // transposed (n1 x n2) copies of sigma e+- for the column pass: FP64 and double-float
  double *epNsT = nullptr, *emNsT = nullptr, *epOsT = nullptr, *emOsT = nullptr;
  df *cfNT[2] = {nullptr, nullptr}, *cfOT[2] = {nullptr, nullptr};
  // FP32 copies for the relaxed Krylov matvec (fde_params.relax): spectra and
  // the t^(m) coefficients {dp, dm} and transposed {sigma ep, sigma em}
  cx<float> *S1x32 = nullptr, *S2x32 = nullptr, *S1y32 = nullptr, *S2y32 = nullptr,
            *twx32 = nullptr, *twy32 = nullptr;
  float *cf32[2] = {nullptr, nullptr}, *cf32T[2] = {nullptr, nullptr};
  double *xT = nullptr, *yT = nullptr;  // transposed operand / result of the column pass
  // FFT passes whose two length-L buffers exceed shared memory (L = 8192 with
  // 16-byte complex values) park spectra here; also the twiddle scratch of
  // their spectra builds
  cx<double>* fft_ws = nullptr;
  size_t fft_ws_elems = 0;
  bool have_new = false, have_old = false;

  std::unique_ptr<MGBase> mg;

  // Krylov workspace: basis V (restart + 1 columns) and Z (restart columns)
  // at a column pitch ldv, a multiple of 64 doubles with zero padding, so the
  // fused Gram-Schmidt passes read whole double2 pairs
  double *V = nullptr, *Z = nullptr, *part = nullptr, *hdev = nullptr, *h2dev = nullptr;
  double *ydev = nullptr, *tmp = nullptr, *bwork = nullptr, *hu = nullptr, *hv = nullptr,
         *hx_out = nullptr, *u_last = nullptr;
  size_t ldv = 0;
  int nb = 0;
  int m = 0;
  // Arnoldi state on the device (rotated Hessenberg matrix, rotations, g)
  ArnoldiState ast{};
  double* cgs_part = nullptr;
  double* dcgs_coef = nullptr;  // the delayed scheme's projection coefficients
  unsigned* tickets = nullptr;
  ArnoldiStatus* status_host = nullptr;  // pinned: the status read after each step

  // profiling
  bool prof = false;
  std::vector<ProfEvent> pending;
  std::vector<cudaEvent_t> pool;
  long long prof_launches[FDE_KCLASS_COUNT] = {};
  double prof_ms[FDE_KCLASS_COUNT] = {};

  int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }

  template <typename P>
  int alloc(P** ptr, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(P) + 16);
    if (e != cudaSuccess) return fail(FDE_ERR_CUDA, "cudaMalloc(%zu): %s", count * sizeof(P),
                                      cudaGetErrorString(e));
    // FDE_POISON=1: fill every workspace buffer with NaN bit patterns, so a
    // read of memory that no kernel wrote first shows up in the results
    static const bool poison = [] {
      const char* v = std::getenv("FDE_POISON");
      return v && v[0] == '1';
    }();
    if (poison) cudaMemset(q, 0xFF, count * sizeof(P) + 16);
    allocs.push_back(q);
    *ptr = static_cast<P*>(q);
    return FDE_OK;
  }

  cudaEvent_t ev() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  int pbeg(int k) {
    if (!prof) return -1;
    ProfEvent pe{k, ev(), ev()};
    cudaEventRecord(pe.a, st);
    pending.push_back(pe);
    return (int)pending.size() - 1;
  }
  void pend(int idx) {
    if (idx >= 0) cudaEventRecord(pending[idx].b, st);
  }
  void prof_collect() {
    if (pending.empty()) return;
    cudaStreamSynchronize(st);
    for (auto& pe : pending) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pe.a, pe.b);
      prof_ms[pe.kclass] += ms;
      prof_launches[pe.kclass] += 1;
      pool.push_back(pe.a);
      pool.push_back(pe.b);
    }
    pending.clear();
  }
};

#define LCHK(call)                                                                       \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    h->launches++;                                                                       \
    if (_e != cudaSuccess)                                                               \
      return h->fail(FDE_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(_e));      \
  } while (0)
#define CCHK(call)                                                                       \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess)                                                               \
      return h->fail(FDE_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(_e));      \
  } while (0)
#define RCHK(call)                 \
  do {                             \
    int _r = (call);               \
    if (_r != FDE_OK) return _r;   \
  } while (0)

// ============================================================================
// multigrid hierarchy

// the finest level's right-hand side from the Krylov vector r, and the
// Krylov vector z from the cycle's result (FP64 or double-float vectors)
template <typename T>
inline cudaError_t vcycle_in(bool df_io, size_t N, const double* r, T* b, cudaStream_t st) {
  return df_io ? launch_convert<df, T>(N, reinterpret_cast<const df*>(r), 1.0, b, st)
               : launch_convert<double, T>(N, r, 1.0, b, st);
}
template <typename T>
inline cudaError_t vcycle_out(bool df_io, size_t N, const T* x, double* z, cudaStream_t st) {
  return df_io ? launch_convert<T, df>(N, x, 1.0, reinterpret_cast<df*>(z), st)
               : launch_convert<T, double>(N, x, 1.0, z, st);
}

struct MGBase {
  virtual ~MGBase() {
    if (graph) cudaGraphExecDestroy(graph);
  }
  virtual int setup(fde_handle* h) = 0;  // from h->dpN.. (FP64, unscaled)
  // z = V(r); df_io: r and z hold double-float vectors (8 bytes an element)
  virtual int vcycle(fde_handle* h, const double* r, double* z, bool df_io) = 0;
  virtual int level_apply(fde_handle* h, int l, const double* x, double* y) = 0;
  // one V-cycle on the finest level's (b -> x) buffers: a fixed sequence of
  // launches on fixed buffers, so it can be replayed from a CUDA graph
  virtual int cycle_root(fde_handle* h) = 0;
  virtual int level_path(int l) const { (void)l; return -1; }
  // 1 if a capped device-side wait gave up since the last check
  virtual int device_error(fde_handle* h) { (void)h; return 0; }
  // enqueue the bounded-wait self-test on the first tensor-core level (-1: none)
  virtual int wait_selftest(fde_handle* h, int complete) {
    (void)h;
    (void)complete;
    return -1;
  }
  std::vector<int> n1s, n2s;
  cudaGraphExec_t graph = nullptr;
  long long graph_launches = 0;
  bool graph_off = false;

  // The first call captures the cycle's ~8 launches per level on the handle's
  // private stream and instantiates a graph; every call then launches that
  // graph on the handle's stream (one launch instead of dozens of small ones
  // on the coarse levels). With kernel profiling on, the cycle runs eagerly.
  int run_cycle(fde_handle* h);
};

inline int MGBase::run_cycle(fde_handle* h) {
  if (h->prof || graph_off || !h->cap_st) return cycle_root(h);
  if (!graph) {
    cudaStream_t user = h->st;
    const long long l0 = h->launches;
    CCHK(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
    h->st = h->cap_st;
    const int rc = cycle_root(h);
    h->st = user;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_st, &g);
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei =
        (rc == FDE_OK && e == cudaSuccess) ? cudaGraphInstantiate(&ex, g, 0) : cudaErrorUnknown;
    if (g) cudaGraphDestroy(g);
    const long long captured = h->launches - l0;
    h->launches = l0;
    if (rc != FDE_OK || ei != cudaSuccess) {
      // capture refused (a call that cannot be captured) or the cycle failed:
      // run eagerly from now on, which also reports a genuine error
      cudaGetLastError();
      graph_off = true;
      h->err.clear();
      return cycle_root(h);
    }
    graph = ex;
    graph_launches = captured;
  }
  CCHK(cudaGraphLaunch(graph, h->st));
  h->launches += graph_launches;
  return FDE_OK;
}

template <typename T>
struct MG : MGBase {
  struct Lv {
    int n1, n2;
    size_t N;
    double bx0 = 1, bx1 = 0, by0 = 1, by1 = 0;  // Galerkin mass tridiagonals
    int offx = 0, offy = 0;                      // finest index of level point 0 per axis
    double *tx = nullptr, *ty = nullptr;         // Toeplitz generators (FP64)
    int path = FDE_PATH_DIRECT;                  // FFT, DIRECT or GEMM
    bool tune = false;                           // time the candidates at the first setup
    int cands = 0;                               // candidate paths (bit FDE_PATH_*)
    int logLx = 0, logLy = 0;
    cx<T> *S1x = nullptr, *S2x = nullptr, *S1y = nullptr, *S2y = nullptr, *twx = nullptr,
          *twy = nullptr;
    T *txT = nullptr, *tyT = nullptr;
    T *dp, *dm, *ep, *em, *W;
    T *x, *b, *kx, *xby = nullptr, *xbx = nullptr, *mass = nullptr;
    T *epT = nullptr, *emT = nullptr, *xT = nullptr, *yT = nullptr;  // column pass (FFT levels)
    tc::ToeplitzGemmLevel gemm;
  };
  std::vector<Lv> lv;
  double *inv = nullptr, *cwork = nullptr, *cf[4] = {nullptr, nullptr, nullptr, nullptr};
  int* info = nullptr;
  double rscale = 1.0;
  bool sg = true;
  T *acc_x = nullptr, *acc_b = nullptr;  // further V-cycles: iterate and second rhs buffer
  size_t tail0 = 0;  // first level handled by the one-launch tail of the cycle (== size: none)

  int create(fde_handle* h) {
    const fde_params& p = h->p;
    sg = p.precond == FDE_PRECOND_MG_SG;
    rscale = sg ? 1.0 : 0.25;
    int m1 = h->n1, m2 = h->n2;
    for (;;) {
      Lv L;
      L.n1 = m1;
      L.n2 = m2;
      L.N = (size_t)m1 * m2;
      lv.push_back(L);
      n1s.push_back(m1);
      n2s.push_back(m2);
      if (m1 <= p.coarsest_n || m2 <= p.coarsest_n) break;
      // the structured Galerkin projection keeps a 1-D factor Toeplitz only
      // when the fine size is odd (n = 2 n_c + 1); the rediscretised cycle
      // coarsens either parity (Sec. 4.1's K matrix)
      if (sg && (!(m1 & 1) || !(m2 & 1)))
        return h->fail(FDE_ERR_UNSUPPORTED,
                       "the structured-Galerkin hierarchy needs odd level sizes down to the "
                       "coarsest grid (got %d x %d); use MG_REDISC, MG_EXACT or P2",
                       m1, m2);
      m1 = coarse_n(m1);
      m2 = coarse_n(m2);
    }
    if (lv.back().N > 1024)
      return h->fail(FDE_ERR_UNSUPPORTED, "coarsest grid %d x %d exceeds 1024 unknowns",
                     lv.back().n1, lv.back().n2);
    // injection offsets of every level (finest point of level point (j, i))
    for (size_t l = 1; l < lv.size(); ++l) {
      lv[l].offx = lv[l - 1].offx + ((lv[l - 1].n1 & 1) << (l - 1));
      lv[l].offy = lv[l - 1].offy + ((lv[l - 1].n2 & 1) << (l - 1));
    }
    // mass tridiagonals (structured Galerkin: b^{c}_0 = 3/2 b_0 + 2 b_1, b^{c}_1 = b_0/4 + b_1)
    for (size_t l = 1; l < lv.size(); ++l) {
      if (sg) {
        Lv& a = lv[l - 1];
        lv[l].bx0 = 1.5 * a.bx0 + 2.0 * a.bx1;
        lv[l].bx1 = 0.25 * a.bx0 + a.bx1;
        lv[l].by0 = 1.5 * a.by0 + 2.0 * a.by1;
        lv[l].by1 = 0.25 * a.by0 + a.by1;
      }
    }
    const bool lowp = (p.precision == FDE_PREC_BF16 || p.precision == FDE_PREC_FP16 ||
                       p.precision == FDE_PREC_BF16X3);
    // the small end of the cycle runs as one launch: from the first level with
    // n <= kTailN down to the coarsest (direct-sum products there)
    tail0 = lv.size();
    for (size_t l = 0; l < lv.size(); ++l)
      if (std::max(lv[l].n1, lv[l].n2) <= kTailN) {
        tail0 = l;
        break;
      }
    if (lv.size() - tail0 > (size_t)kTailMaxLevels || tail0 + 1 >= lv.size()) tail0 = lv.size();
    for (size_t l = 0; l < lv.size(); ++l) {
      Lv& L = lv[l];
      const bool last = l + 1 == lv.size();
      RCHK(h->alloc(&L.tx, L.n1 + 2));
      RCHK(h->alloc(&L.ty, L.n2 + 2));
      RCHK(h->alloc(&L.dp, L.N));
      RCHK(h->alloc(&L.dm, L.N));
      RCHK(h->alloc(&L.ep, L.N));
      RCHK(h->alloc(&L.em, L.N));
      RCHK(h->alloc(&L.W, L.N));
      RCHK(h->alloc(&L.x, L.N));
      RCHK(h->alloc(&L.b, L.N));
      RCHK(h->alloc(&L.kx, L.N));
      if (sg && l > 0) {
        RCHK(h->alloc(&L.xby, L.N));
        RCHK(h->alloc(&L.xbx, L.N));
        RCHK(h->alloc(&L.mass, L.N));
      }
      if (last) continue;
      // product path of this level
      int path = p.toeplitz_path;
      const int nmin = std::min(L.n1, L.n2), nmax = std::max(L.n1, L.n2);
      if (l >= tail0) path = FDE_PATH_DIRECT;  // the tail sums directly
      if (path == FDE_PATH_TUNE) {
        // candidates: tensor cores (reduced precision, n >= 127), FFT, and
        // direct summation while its O(n^2) per line stays small (n <= 1023)
        L.cands = (1 << FDE_PATH_FFT) | (nmax <= 1023 ? (1 << FDE_PATH_DIRECT) : 0) |
                  ((lowp && nmin >= tc::kMinGemmN) ? (1 << FDE_PATH_GEMM) : 0);
        L.tune = true;
        path = (L.cands & (1 << FDE_PATH_GEMM)) ? FDE_PATH_GEMM : FDE_PATH_FFT;
      }
      if (path == FDE_PATH_AUTO) {
        if (lowp && nmin >= tc::kAutoGemmN) path = FDE_PATH_GEMM;
        else path = nmin >= 127 ? FDE_PATH_FFT : FDE_PATH_DIRECT;
      }
      if (path == FDE_PATH_GEMM && !lowp)
        return h->fail(FDE_ERR_ARG, "the tensor-core path needs BF16, FP16 or BF16X3 precision");
      if (path == FDE_PATH_GEMM && nmin < tc::kMinGemmN) path = FDE_PATH_FFT;
      L.path = path;
      if (path == FDE_PATH_FFT) {
        L.logLx = ceil_log2(2L * L.n1 - 1);
        L.logLy = ceil_log2(2L * L.n2 - 1);
        const int lmax = std::max(L.logLx, L.logLy);
        if (fft_pass_two_buffer_bytes(lmax, sizeof(cx<T>)) > 227 * 1024 &&
            h->fft_ws_elems < ((size_t)152 << lmax))
          return h->fail(FDE_ERR_UNSUPPORTED, "FFT length too large for shared memory");
        RCHK(h->alloc(&L.S1x, (size_t)1 << L.logLx));
        RCHK(h->alloc(&L.S2x, (size_t)1 << L.logLx));
        RCHK(h->alloc(&L.twx, (size_t)1 << L.logLx));
        RCHK(h->alloc(&L.epT, L.N));
        RCHK(h->alloc(&L.emT, L.N));
        RCHK(h->alloc(&L.xT, L.N));
        RCHK(h->alloc(&L.yT, L.N));
        RCHK(h->alloc(&L.S1y, (size_t)1 << L.logLy));
        RCHK(h->alloc(&L.S2y, (size_t)1 << L.logLy));
        RCHK(h->alloc(&L.twy, (size_t)1 << L.logLy));
      } else if (path == FDE_PATH_DIRECT) {
        RCHK(h->alloc(&L.txT, L.n1 + 2));
        RCHK(h->alloc(&L.tyT, L.n2 + 2));
      } else {
        const int prec = p.precision == FDE_PREC_BF16 ? tc::kBF16
                         : p.precision == FDE_PREC_FP16 ? tc::kFP16 : tc::kBF16X3;
        int r = tc::level_create(&L.gemm, L.n1, L.n2, prec, sg && l > 0);
        if (r == 13 && (p.toeplitz_path == FDE_PATH_AUTO || L.tune)) {
          L.cands &= ~(1 << FDE_PATH_GEMM);
          // the generator copies do not fit beside the pipeline: FFT products
          tc::level_destroy(&L.gemm);
          L.path = FDE_PATH_FFT;
          L.logLx = ceil_log2(2L * L.n1 - 1);
          L.logLy = ceil_log2(2L * L.n2 - 1);
          RCHK(h->alloc(&L.S1x, (size_t)1 << L.logLx));
          RCHK(h->alloc(&L.S2x, (size_t)1 << L.logLx));
          RCHK(h->alloc(&L.twx, (size_t)1 << L.logLx));
          RCHK(h->alloc(&L.epT, L.N));
          RCHK(h->alloc(&L.emT, L.N));
          RCHK(h->alloc(&L.xT, L.N));
          RCHK(h->alloc(&L.yT, L.N));
          RCHK(h->alloc(&L.S1y, (size_t)1 << L.logLy));
          RCHK(h->alloc(&L.S2y, (size_t)1 << L.logLy));
          RCHK(h->alloc(&L.twy, (size_t)1 << L.logLy));
        } else if (r != 0) {
          return h->fail(FDE_ERR_UNSUPPORTED, "tensor-core level allocation failed (%d)", r);
        } else if (L.tune) {
          // the FFT path's data, for the timing at the first setup
          L.logLx = ceil_log2(2L * L.n1 - 1);
          L.logLy = ceil_log2(2L * L.n2 - 1);
          const int lmax = std::max(L.logLx, L.logLy);
          if (fft_pass_two_buffer_bytes(lmax, sizeof(cx<T>)) > 227 * 1024 &&
              h->fft_ws_elems < ((size_t)152 << lmax)) {
            L.cands &= ~(1 << FDE_PATH_FFT);  // FFT impossible here
          } else {
            RCHK(h->alloc(&L.S1x, (size_t)1 << L.logLx));
            RCHK(h->alloc(&L.S2x, (size_t)1 << L.logLx));
            RCHK(h->alloc(&L.twx, (size_t)1 << L.logLx));
            RCHK(h->alloc(&L.epT, L.N));
            RCHK(h->alloc(&L.emT, L.N));
            RCHK(h->alloc(&L.xT, L.N));
            RCHK(h->alloc(&L.yT, L.N));
            RCHK(h->alloc(&L.S1y, (size_t)1 << L.logLy));
            RCHK(h->alloc(&L.S2y, (size_t)1 << L.logLy));
            RCHK(h->alloc(&L.twy, (size_t)1 << L.logLy));
          }
        }
      }
    }
    for (size_t l = 0; l + 1 < lv.size(); ++l) {
      Lv& L = lv[l];
      if (L.tune && (L.cands & (1 << FDE_PATH_DIRECT)) && !L.txT) {
        RCHK(h->alloc(&L.txT, L.n1 + 2));
        RCHK(h->alloc(&L.tyT, L.n2 + 2));
      }
      if (L.tune && __builtin_popcount(L.cands) < 2) L.tune = false;
    }
    const Lv& C = lv.back();
    RCHK(h->alloc(&inv, C.N * C.N));
    RCHK(h->alloc(&cwork, C.N * C.N * 2));
    for (int k = 0; k < 4; ++k) RCHK(h->alloc(&cf[k], C.N));
    RCHK(h->alloc(&info, 4));
    if (p.cycles > 1) {
      RCHK(h->alloc(&acc_x, lv[0].N));
      RCHK(h->alloc(&acc_b, lv[0].N));
    }
    return FDE_OK;
  }

  ~MG() {
    for (auto& L : lv) tc::level_destroy(&L.gemm);
  }

  // generators, coefficient fields, spectra, coarsest inverse
  int setup(fde_handle* h) override {
    const fde_params& p = h->p;
    cudaStream_t st = h->st;
    for (size_t l = 0; l < lv.size(); ++l) {
      Lv& L = lv[l];
      if (l == 0 || !sg) {
        const double sx = std::pow(2.0, -p.alpha * (double)l), sy = std::pow(2.0, -p.beta * (double)l);
        LCHK(launch_generator_from_weights(h->wx, L.n1, sx, L.tx, st));
        LCHK(launch_generator_from_weights(h->wy, L.n2, sy, L.ty, st));
      } else {
        LCHK(launch_coarsen_generator(lv[l - 1].tx, lv[l - 1].n1, L.tx, L.n1, st));
        LCHK(launch_coarsen_generator(lv[l - 1].ty, lv[l - 1].n2, L.ty, L.n2, st));
      }
      const int stride = 1 << l;
      LCHK(launch_level_fields<T>(h->dpN, h->dmN, h->epN, h->emN, h->n1, L.n1, L.n2, stride,
                                  L.offx, L.offy, h->sigma, h->c, L.bx0, L.by0, L.tx, L.ty,
                                  p.omega, L.dp, L.dm, L.ep, L.em, L.W, st));
      if ((L.path == FDE_PATH_FFT || (L.tune && (L.cands & (1 << FDE_PATH_FFT)))) &&
          l + 1 < lv.size()) {
        LCHK(launch_transpose<T>(L.ep, L.n2, L.n1, L.epT, 0, st));
        LCHK(launch_transpose<T>(L.em, L.n2, L.n1, L.emT, 0, st));
        LCHK(launch_build_spectra<T>(L.tx, L.n1, L.logLx, 1.0, L.S1x, L.S2x, L.twx, st, h->fft_ws));
        LCHK(launch_build_spectra<T>(L.ty, L.n2, L.logLy, 1.0, L.S1y, L.S2y, L.twy, st, h->fft_ws));
      }
      if ((L.path == FDE_PATH_DIRECT || (L.tune && (L.cands & (1 << FDE_PATH_DIRECT)))) &&
          l + 1 < lv.size()) {
        LCHK((launch_convert<double, T>(L.n1 + 1, L.tx, 1.0, L.txT, st)));
        LCHK((launch_convert<double, T>(L.n2 + 1, L.ty, 1.0, L.tyT, st)));
      }
      if (L.path == FDE_PATH_GEMM && l + 1 < lv.size()) {
        int r = tc::level_setup(&L.gemm, L.tx, L.ty, st);
        h->launches += 2;
        if (r != 0) return h->fail(FDE_ERR_CUDA, "tensor-core bank setup failed (%d)", r);
      }
    }
    // coarsest: FP64 fields, dense inverse
    Lv& C = lv.back();
    const int stride = 1 << (lv.size() - 1);
    LCHK(launch_level_fields<double>(h->dpN, h->dmN, h->epN, h->emN, h->n1, C.n1, C.n2, stride,
                                     C.offx, C.offy, h->sigma, h->c, C.bx0, C.by0, C.tx, C.ty,
                                     p.omega, cf[0], cf[1], cf[2], cf[3], nullptr, st));
    LCHK(launch_coarse_inverse(C.tx, C.ty, C.n1, C.n2, C.bx0, C.bx1, C.by0, C.by1, h->c, cf[0],
                               cf[1], cf[2], cf[3], cwork, inv, info, st));
    int hinfo = 0;
    CCHK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    CCHK(cudaStreamSynchronize(st));
    if (hinfo != 0) return h->fail(FDE_ERR_NONFINITE, "coarsest-grid matrix is singular");
    RCHK(tune(h));
    return FDE_OK;
  }

  // FDE_PATH_TUNE: time each candidate path's products of a level (one
  // warm-up, five timed runs on the level's own buffers) and keep the fastest;
  // a later candidate (order: tensor cores, FFT, direct sums) must be faster
  // by more than 3 %, so that near-ties, within the timing noise between
  // runs and boxes, resolve the same way every time
  int tune(fde_handle* h) {
    cudaStream_t st = h->st;
    for (size_t l = 0; l + 1 < lv.size(); ++l) {
      Lv& L = lv[l];
      if (!L.tune) continue;
      CCHK(cudaMemsetAsync(L.x, 0, L.N * sizeof(T), st));
      float best = 0.f;
      int best_path = FDE_PATH_GEMM;
      const bool prof = h->prof;
      h->prof = false;
      bool first = true;
      for (int cand : {FDE_PATH_GEMM, FDE_PATH_FFT, FDE_PATH_DIRECT}) {
        if (!(L.cands & (1 << cand))) continue;
        L.path = cand;
        RCHK(products(h, l, L.x, L.kx));
        cudaEvent_t e0 = h->ev(), e1 = h->ev();
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5; ++r) RCHK(products(h, l, L.x, L.kx));
        cudaEventRecord(e1, st);
        CCHK(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        h->pool.push_back(e0);
        h->pool.push_back(e1);
        if (first || ms < 0.97f * best) {
          best = ms;
          best_path = cand;
          first = false;
        }
      }
      h->prof = prof;
      L.path = best_path;
      L.tune = false;
    }
    return FDE_OK;
  }

  int level_path(int l) const override {
    if (l < 0 || l + 1 >= (int)lv.size()) return -1;
    return lv[l].path;
  }

  int device_error(fde_handle* h) override {
    int any = 0;
    for (auto& L : lv)
      if (L.gemm.built && tc::level_error(&L.gemm, h->st) != 0) any = 1;
    return any;
  }

  int wait_selftest(fde_handle* h, int complete) override {
    for (auto& L : lv)
      if (L.gemm.built) return tc::level_wait_selftest(&L.gemm, complete, h->st);
    return -1;
  }

  // kx = K_l x (products + mass term); jacobi_from_zero (structured-Galerkin
  // levels l > 0 only): x is first set to W b in the same pass as the mass terms;
  // smoothed (non-null, x = L.x): on the FFT path the damped-Jacobi update
  // x <- x + W (b - K x) is applied in the products' last pass instead of
  // storing kx, and *smoothed is set
  int products(fde_handle* h, size_t l, const T* x, T* kx, bool jacobi_from_zero = false,
               bool* smoothed = nullptr) {
    Lv& L = lv[l];
    cudaStream_t st = h->st;
    const T *xin_x = x, *xin_y = x, *M = x;
    double cm = h->c;
    // structured-Galerkin level on the two-pass FFT path: the pre-pass writes
    // the column pass's operand already transposed
    const bool xT_ready = sg && l > 0 && L.path == FDE_PATH_FFT && L.logLx == L.logLy;
    if (xT_ready) {
      LCHK(launch_mass_prepass_t<T>(jacobi_from_zero ? L.W : nullptr,
                                    jacobi_from_zero ? L.b : nullptr, L.n1, L.n2, L.bx0, L.bx1,
                                    L.by0, L.by1, h->c, const_cast<T*>(x), L.xby, L.xT, L.mass,
                                    st));
      xin_x = L.xby;
      xin_y = nullptr;
      M = L.mass;
      cm = 1.0;
    } else if (sg && l > 0) {
      if (jacobi_from_zero)
        LCHK(launch_jacobi_mass_prepass<T>(L.W, L.b, L.n1, L.n2, L.bx0, L.bx1, L.by0, L.by1, h->c,
                                           const_cast<T*>(x), L.xby, L.xbx, L.mass, st));
      else
        LCHK(launch_mass_prepass<T>(x, L.n1, L.n2, L.bx0, L.bx1, L.by0, L.by1, h->c, L.xby,
                                    L.xbx, L.mass, st));
      xin_x = L.xby;
      xin_y = L.xbx;
      M = L.mass;
      cm = 1.0;
    }
    const int pi = h->pbeg(FDE_KCLASS_LEVEL_APPLY);
    if (L.path == FDE_PATH_FFT) {
      cx<T>* ws = reinterpret_cast<cx<T>*>(h->fft_ws);
      const size_t wse = h->fft_ws_elems * sizeof(cx<double>) / sizeof(cx<T>);
      if (L.logLx == L.logLy) {
        // both directions' passes in one launch (the y pass on the transposed grid)
        if (!xT_ready) LCHK(launch_transpose<T>(xin_y, L.n2, L.n1, L.xT, 0, st));
        const FftPass<T, T, T> px{xin_x, 1, L.n1, L.n2, L.n1, L.S1x, L.S2x, L.twx, L.dp, L.dm,
                                  M,     cm, kx,   0};
        const FftPass<T, T, T> py{L.xT, 1,   L.n2,    L.n1, L.n2, L.S1y, L.S2y, L.twy, L.epT,
                                  L.emT, nullptr, 0.0, L.yT, 0};
        LCHK((launch_fft_pass2<T, T, T>(px, py, L.logLx, st, ws, wse)));
      } else {
        LCHK((launch_fft_pass<T, T, T>(xin_x, 1, L.n1, L.n2, L.n1, L.logLx, L.S1x, L.S2x, L.twx,
                                       L.dp, L.dm, M, cm, kx, 0, st, ws, wse)));
        LCHK(launch_transpose<T>(xin_y, L.n2, L.n1, L.xT, 0, st));
        LCHK((launch_fft_pass<T, T, T>(L.xT, 1, L.n2, L.n1, L.n2, L.logLy, L.S1y, L.S2y, L.twy,
                                       L.epT, L.emT, nullptr, 0.0, L.yT, 0, st, ws, wse)));
      }
      if (smoothed) {
        LCHK(launch_transpose_smooth<T>(L.yT, L.n1, L.n2, kx, L.b, L.W, L.x, st));
        *smoothed = true;
      } else {
        LCHK(launch_transpose<T>(L.yT, L.n1, L.n2, kx, 1, st));
      }
    } else if (L.path == FDE_PATH_DIRECT) {
      LCHK(launch_direct_pass<T>(xin_x, 1, L.n1, L.n2, L.n1, L.txT, L.dp, L.dm, M, cm, kx, 0, st));
      LCHK(launch_direct_pass<T>(xin_y, L.n1, 1, L.n1, L.n2, L.tyT, L.ep, L.em, nullptr, 0.0, kx,
                                 1, st));
    } else {
      int r = tc::level_pack(&L.gemm, (const float*)xin_x, (const float*)xin_y, st);
      h->launches += (sg && l > 0) ? 2 : 1;
      if (r != 0) return h->fail(FDE_ERR_CUDA, "tensor-core operand packing failed (%d)", r);
      // each direction is one launch, timed on its own (FDE_KCLASS_TC_GEMM)
      int gi = h->pbeg(FDE_KCLASS_TC_GEMM);
      r = tc::level_gemm(&L.gemm, 0, (const float*)M, cm, (const float*)L.dp, (const float*)L.dm,
                         (float*)kx, st);
      h->pend(gi);
      h->launches++;
      if (r != 0) return h->fail(FDE_ERR_CUDA, "tensor-core products failed (%d)", r);
      gi = h->pbeg(FDE_KCLASS_TC_GEMM);
      r = tc::level_gemm(&L.gemm, 1, nullptr, 0.0, (const float*)L.ep, (const float*)L.em,
                         (float*)kx, st);
      h->pend(gi);
      h->launches++;
      if (r != 0) return h->fail(FDE_ERR_CUDA, "tensor-core products failed (%d)", r);
      r = tc::level_finish(&L.gemm, (const float*)M, cm, (float*)kx, st);
      if (L.gemm.splits > 1) h->launches++;
      if (r != 0) return h->fail(FDE_ERR_CUDA, "tensor-core split reduction failed (%d)", r);
    }
    h->pend(pi);
    return FDE_OK;
  }

  int smooth(fde_handle* h, size_t l) {  // x <- x + W (b - K x)
    Lv& L = lv[l];
    bool done = false;
    RCHK(products(h, l, L.x, L.kx, false, &done));
    if (done) return FDE_OK;
    const int pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    LCHK(launch_level_epilogue<T>(2, L.N, L.kx, L.b, L.x, L.W, L.x, h->st));
    h->pend(pi);
    return FDE_OK;
  }

  int cycle(fde_handle* h, size_t l) {
    Lv& L = lv[l];
    const fde_params& p = h->p;
    cudaStream_t st = h->st;
    if (l == tail0) return cycle_tail(h);
    if (l + 1 == lv.size()) {
      const int pi = h->pbeg(FDE_KCLASS_MG_OTHER);
      LCHK(launch_coarse_solve<T>(inv, (int)L.N, L.b, L.x, st));
      h->pend(pi);
      return FDE_OK;
    }
    // pre-smoothing from zero: x = W b (on structured-Galerkin levels l > 0
    // with one sweep, inside the mass-term pass of the residual's products)
    const bool fused_sweep = p.nu_pre == 1 && sg && l > 0;
    int pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    if (p.nu_pre >= 1 && !fused_sweep) LCHK(launch_mul<T>(L.N, L.W, L.b, L.x, st));
    else if (p.nu_pre < 1) CCHK(cudaMemsetAsync(L.x, 0, L.N * sizeof(T), st));
    h->pend(pi);
    for (int s = 1; s < p.nu_pre; ++s) RCHK(smooth(h, l));
    // residual r = b - K x restricted without storing r
    RCHK(products(h, l, L.x, L.kx, fused_sweep));
    pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    LCHK(launch_restrict_residual<T>(L.b, L.kx, L.n1, L.n2, rscale, lv[l + 1].b, st));
    h->pend(pi);
    RCHK(cycle(h, l + 1));
    pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    LCHK(launch_prolong_add<T>(lv[l + 1].x, L.n1, L.n2, L.x, st));
    h->pend(pi);
    for (int s = 0; s < p.nu_post; ++s) RCHK(smooth(h, l));
    return FDE_OK;
  }

  // levels tail0 .. last in one launch (kernels_tail.cu)
  int cycle_tail(fde_handle* h) {
    const TailArgs<T> a = tail_args(h);
    const int pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    LCHK(launch_mg_tail<T>(a, h->st));
    h->pend(pi);
    return FDE_OK;
  }

  // the arguments of the one-launch tail (levels tail0 .. last)
  TailArgs<T> tail_args(fde_handle* h) const {
    TailArgs<T> a{};
    a.nlev = (int)(lv.size() - tail0);
    a.nu_pre = h->p.nu_pre;
    a.nu_post = h->p.nu_post;
    a.c = h->c;
    a.rscale = rscale;
    a.inv = inv;
    for (int k = 0; k < a.nlev; ++k) {
      const Lv& L = lv[tail0 + k];
      TailLevel<T>& t = a.lv[k];
      t.n1 = L.n1;
      t.n2 = L.n2;
      t.x = L.x;
      t.b = L.b;
      t.kx = L.kx;
      t.W = L.W;
      t.dp = L.dp;
      t.dm = L.dm;
      t.ep = L.ep;
      t.em = L.em;
      t.tx = L.txT;
      t.ty = L.tyT;
      const bool mass = sg && tail0 + k > 0;
      t.xby = mass ? L.xby : nullptr;
      t.xbx = mass ? L.xbx : nullptr;
      t.mass = mass ? L.mass : nullptr;
      t.bx0 = T(L.bx0);
      t.bx1 = T(L.bx1);
      t.by0 = T(L.by0);
      t.by1 = T(L.by1);
    }
    return a;
  }

  int cycle_root(fde_handle* h) override { return cycle(h, 0); }

  int vcycle(fde_handle* h, const double* r, double* z, bool df_io) override {
    Lv& L = lv[0];
    LCHK(vcycle_in<T>(df_io, L.N, r, L.b, h->st));
    RCHK(run_cycle(h));
    // a one-level hierarchy is the coarsest-grid solve itself, exact up to
    // rounding: further cycles are skipped (level 0 then has no product path)
    const int cycles = (h->p.cycles > 1 && lv.size() > 1) ? h->p.cycles : 1;
    if (cycles > 1) {
      // stationary iteration z_{k+1} = z_k + V(r - K_0 z_k): r is kept in acc_b,
      // each cycle reads its right-hand side from L.b and leaves z in L.x
      CCHK(cudaMemcpyAsync(acc_b, L.b, L.N * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
      for (int k = 1; k < cycles; ++k) {
        CCHK(cudaMemcpyAsync(acc_x, L.x, L.N * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
        RCHK(products(h, 0, acc_x, L.kx));
        LCHK(launch_level_epilogue<T>(1, L.N, L.kx, acc_b, acc_x, L.W, L.b, h->st));
        RCHK(run_cycle(h));
        LCHK(launch_add<T>(L.N, acc_x, L.x, L.x, h->st));
      }
    }
    LCHK(vcycle_out<T>(df_io, L.N, L.x, z, h->st));
    return FDE_OK;
  }

  int level_apply(fde_handle* h, int l, const double* x, double* y) override {
    if (l < 0 || l >= (int)lv.size()) return h->fail(FDE_ERR_ARG, "level %d out of range", l);
    Lv& L = lv[l];
    if (l + 1 == (int)lv.size()) {
      // coarsest level (the cycle uses its inverse): apply through the direct
      // path, with generators in T allocated on the first request
      LCHK((launch_convert<double, T>(L.N, x, 1.0, L.x, h->st)));
      if (!L.txT) {
        RCHK(h->alloc(&L.txT, L.n1 + 2));
        RCHK(h->alloc(&L.tyT, L.n2 + 2));
      }
      LCHK((launch_convert<double, T>(L.n1 + 1, L.tx, 1.0, L.txT, h->st)));
      LCHK((launch_convert<double, T>(L.n2 + 1, L.ty, 1.0, L.tyT, h->st)));
      const T *xin_x = L.x, *xin_y = L.x, *M = L.x;
      double cm = h->c;
      if (sg && l > 0) {  // mass-term buffers of every SG level l > 0 exist
        LCHK(launch_mass_prepass<T>(L.x, L.n1, L.n2, L.bx0, L.bx1, L.by0, L.by1, h->c, L.xby,
                                    L.xbx, L.mass, h->st));
        xin_x = L.xby;
        xin_y = L.xbx;
        M = L.mass;
        cm = 1.0;
      }
      LCHK(launch_direct_pass<T>(xin_x, 1, L.n1, L.n2, L.n1, L.txT, L.dp, L.dm, M, cm, L.kx, 0,
                                 h->st));
      LCHK(launch_direct_pass<T>(xin_y, L.n1, 1, L.n1, L.n2, L.tyT, L.ep, L.em, nullptr, 0.0, L.kx,
                                 1, h->st));
      LCHK((launch_convert<T, double>(L.N, L.kx, 1.0, y, h->st)));
      return FDE_OK;
    }
    LCHK((launch_convert<double, T>(L.N, x, 1.0, L.x, h->st)));
    RCHK(products(h, l, L.x, L.kx));
    LCHK((launch_convert<T, double>(L.N, L.kx, 1.0, y, h->st)));
    return FDE_OK;
  }
};

// ============================================================================
// P_2 (Sec. 4.3): five-point band operator with a Galerkin V-cycle. Every
// level is a nine-point stencil (kernels_stencil.cu): level 0 is P_2 itself,
// level l + 1 is P^T K_l P computed in FP64, the coarsest is inverted densely.

template <typename T>
struct StencilMG : MGBase {
  struct Lv {
    int n1, n2;
    size_t N;
    double* S64 = nullptr;  // FP64 stencil (Galerkin products, coarsest inverse)
    T *S = nullptr, *W = nullptr, *x = nullptr, *b = nullptr, *kx = nullptr;
  };
  std::vector<Lv> lv;
  double *inv = nullptr, *cwork = nullptr;
  int* info = nullptr;
  T *acc_x = nullptr, *acc_b = nullptr;

  int create(fde_handle* h) {
    const fde_params& p = h->p;
    int m1 = h->n1, m2 = h->n2;
    for (;;) {
      Lv L;
      L.n1 = m1;
      L.n2 = m2;
      L.N = (size_t)m1 * m2;
      lv.push_back(L);
      n1s.push_back(m1);
      n2s.push_back(m2);
      if (m1 <= p.coarsest_n || m2 <= p.coarsest_n) break;
      m1 = coarse_n(m1);  // either parity: Sec. 4.1's transfer
      m2 = coarse_n(m2);
    }
    if (lv.back().N > 1024)
      return h->fail(FDE_ERR_UNSUPPORTED, "coarsest grid %d x %d exceeds 1024 unknowns",
                     lv.back().n1, lv.back().n2);
    for (size_t l = 0; l < lv.size(); ++l) {
      Lv& L = lv[l];
      RCHK(h->alloc(&L.S64, 9 * L.N));
      RCHK(h->alloc(&L.x, L.N));
      RCHK(h->alloc(&L.b, L.N));
      RCHK(h->alloc(&L.kx, L.N));
      RCHK(h->alloc(&L.W, L.N));
      if (std::is_same<T, double>::value) L.S = reinterpret_cast<T*>(L.S64);
      else RCHK(h->alloc(&L.S, 9 * L.N));
    }
    const Lv& C = lv.back();
    RCHK(h->alloc(&inv, C.N * C.N));
    RCHK(h->alloc(&cwork, C.N * C.N * 2));
    RCHK(h->alloc(&info, 4));
    if (p.cycles > 1) {
      RCHK(h->alloc(&acc_x, lv[0].N));
      RCHK(h->alloc(&acc_b, lv[0].N));
    }
    return FDE_OK;
  }

  int setup(fde_handle* h) override {
    cudaStream_t st = h->st;
    LCHK(launch_p2_fields(h->dpN, h->dmN, h->epN, h->emN, h->n1, h->n2, h->c, h->sigma,
                          lv[0].S64, st));
    for (size_t l = 1; l < lv.size(); ++l)
      LCHK(launch_galerkin9(lv[l - 1].S64, lv[l - 1].n1, lv[l - 1].n2, lv[l].S64, lv[l].n1,
                            lv[l].n2, st));
    for (size_t l = 0; l < lv.size(); ++l) {
      Lv& L = lv[l];
      if (std::is_same<T, double>::value) {
        // S aliases S64: only the Jacobi weights
        LCHK((launch_stencil_convert<T>(L.S64, L.N, h->p.omega, nullptr, L.W, st)));
      } else {
        LCHK((launch_stencil_convert<T>(L.S64, L.N, h->p.omega, L.S, L.W, st)));
      }
    }
    Lv& C = lv.back();
    LCHK(launch_stencil_inverse(C.S64, C.n1, C.n2, cwork, inv, info, st));
    int hinfo = 0;
    CCHK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    CCHK(cudaStreamSynchronize(st));
    if (hinfo != 0) return h->fail(FDE_ERR_NONFINITE, "coarsest-grid matrix is singular");
    return FDE_OK;
  }

  int apply(fde_handle* h, size_t l, int mode, const T* x, const T* b, T* y) {
    Lv& L = lv[l];
    const int pi = h->pbeg(FDE_KCLASS_LEVEL_APPLY);
    LCHK(launch_stencil_apply<T>(mode, l == 0, L.S, L.n1, L.n2, x, b, L.W, y, h->st));
    h->pend(pi);
    return FDE_OK;
  }

  // V-cycle on level l from x = 0; *out receives the buffer (x or kx of the
  // level) that holds the result: Jacobi sweeps ping-pong between the two, in
  // the same order on every call
  int cycle(fde_handle* h, size_t l, T** out) {
    Lv& L = lv[l];
    const fde_params& p = h->p;
    cudaStream_t st = h->st;
    T *x = L.x, *t = L.kx;
    if (l + 1 == lv.size()) {
      const int pi = h->pbeg(FDE_KCLASS_MG_OTHER);
      LCHK(launch_coarse_solve<T>(inv, (int)L.N, L.b, x, st));
      h->pend(pi);
      *out = x;
      return FDE_OK;
    }
    int pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    if (p.nu_pre >= 1) LCHK(launch_mul<T>(L.N, L.W, L.b, x, st));
    else CCHK(cudaMemsetAsync(x, 0, L.N * sizeof(T), st));
    h->pend(pi);
    for (int s = 1; s < p.nu_pre; ++s) {
      RCHK(apply(h, l, 2, x, L.b, t));
      std::swap(x, t);
    }
    RCHK(apply(h, l, 1, x, L.b, t));  // r = b - K x
    pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    LCHK(launch_restrict<T>(t, L.n1, L.n2, 1.0, lv[l + 1].b, st));  // R = P^T
    h->pend(pi);
    T* xc = nullptr;
    RCHK(cycle(h, l + 1, &xc));
    pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    LCHK(launch_prolong_add<T>(xc, L.n1, L.n2, x, st));
    h->pend(pi);
    for (int s = 0; s < p.nu_post; ++s) {
      RCHK(apply(h, l, 2, x, L.b, t));
      std::swap(x, t);
    }
    *out = x;
    return FDE_OK;
  }

  T* root_out = nullptr;  // finest-level buffer holding a cycle's result
  int cycle_root(fde_handle* h) override { return cycle(h, 0, &root_out); }

  int vcycle(fde_handle* h, const double* r, double* z, bool df_io) override {
    Lv& L = lv[0];
    LCHK(vcycle_in<T>(df_io, L.N, r, L.b, h->st));
    RCHK(run_cycle(h));
    const int cycles = h->p.cycles > 1 ? h->p.cycles : 1;
    if (cycles > 1) {
      // stationary iteration z_{k+1} = z_k + V(r - K_0 z_k): r is kept in acc_b
      CCHK(cudaMemcpyAsync(acc_b, L.b, L.N * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
      for (int k = 1; k < cycles; ++k) {
        CCHK(cudaMemcpyAsync(acc_x, root_out, L.N * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
        RCHK(apply(h, 0, 1, acc_x, acc_b, L.b));
        RCHK(run_cycle(h));
        LCHK(launch_add<T>(L.N, acc_x, root_out, root_out, h->st));
      }
    }
    LCHK(vcycle_out<T>(df_io, L.N, root_out, z, h->st));
    return FDE_OK;
  }

  int level_apply(fde_handle* h, int l, const double* x, double* y) override {
    if (l < 0 || l >= (int)lv.size()) return h->fail(FDE_ERR_ARG, "level %d out of range", l);
    Lv& L = lv[l];
    if (l + 1 == (int)lv.size()) {
      // the coarsest level applies its FP64 stencil (the cycle uses its inverse)
      LCHK(launch_stencil_apply<double>(0, false, L.S64, L.n1, L.n2, x, nullptr, nullptr, y,
                                        h->st));
      return FDE_OK;
    }
    LCHK((launch_convert<double, T>(L.N, x, 1.0, L.x, h->st)));
    LCHK(launch_stencil_apply<T>(0, l == 0, L.S, L.n1, L.n2, L.x, nullptr, nullptr, L.kx,
                                 h->st));
    LCHK((launch_convert<T, double>(L.N, L.kx, 1.0, y, h->st)));
    return FDE_OK;
  }
};

// ============================================================================
// Exact Galerkin hierarchy with explicit matrices (Sec. 4, TGM step 3 at every
// level; the paper's tilde-P_MGM of Sec. 5.1): level 0 is M of Eq. (M)
// assembled densely, level l + 1 is P^T A_l P, formed on the device in FP64;
// damped Jacobi with the true diagonal, R = P^T, dense coarsest inverse.  A
// validation mode for small variable-coefficient grids (N <= kDenseMaxN),
// where the structured-Galerkin reading and the exact one differ.

constexpr size_t kDenseMaxN = 4096;

struct DenseMG : MGBase {
  struct Lv {
    int n1, n2;
    size_t N;
    double *A = nullptr, *W = nullptr, *x = nullptr, *b = nullptr, *kx = nullptr;
  };
  std::vector<Lv> lv;
  double *AP = nullptr, *inv = nullptr, *cwork = nullptr;
  double *acc_x = nullptr, *acc_b = nullptr;
  int* info = nullptr;

  int create(fde_handle* h) {
    const fde_params& p = h->p;
    if (h->N > kDenseMaxN)
      return h->fail(FDE_ERR_UNSUPPORTED,
                     "the exact-Galerkin hierarchy stores dense levels: N = %zu exceeds %zu",
                     h->N, kDenseMaxN);
    int m1 = h->n1, m2 = h->n2;
    for (;;) {
      Lv L;
      L.n1 = m1;
      L.n2 = m2;
      L.N = (size_t)m1 * m2;
      lv.push_back(L);
      n1s.push_back(m1);
      n2s.push_back(m2);
      if (m1 <= p.coarsest_n || m2 <= p.coarsest_n) break;
      m1 = coarse_n(m1);
      m2 = coarse_n(m2);
    }
    if (lv.back().N > 1024)
      return h->fail(FDE_ERR_UNSUPPORTED, "coarsest grid %d x %d exceeds 1024 unknowns",
                     lv.back().n1, lv.back().n2);
    size_t ap = 0;
    for (size_t l = 0; l < lv.size(); ++l) {
      Lv& L = lv[l];
      RCHK(h->alloc(&L.A, L.N * L.N));
      RCHK(h->alloc(&L.W, L.N));
      RCHK(h->alloc(&L.x, L.N));
      RCHK(h->alloc(&L.b, L.N));
      RCHK(h->alloc(&L.kx, L.N));
      if (l + 1 < lv.size()) ap = std::max(ap, L.N * lv[l + 1].N);
    }
    if (ap) RCHK(h->alloc(&AP, ap));
    const Lv& C = lv.back();
    RCHK(h->alloc(&inv, C.N * C.N));
    RCHK(h->alloc(&cwork, C.N * C.N * 2));
    RCHK(h->alloc(&info, 4));
    if (p.cycles > 1) {
      RCHK(h->alloc(&acc_x, lv[0].N));
      RCHK(h->alloc(&acc_b, lv[0].N));
    }
    return FDE_OK;
  }

  int setup(fde_handle* h) override {
    cudaStream_t st = h->st;
    LCHK(launch_dense_assemble(h->tx0, h->ty0, h->n1, h->n2, h->c, h->sigma, h->dpN, h->dmN,
                               h->epN, h->emN, lv[0].A, st));
    for (size_t l = 0; l + 1 < lv.size(); ++l)
      LCHK(launch_dense_galerkin(lv[l].A, lv[l].n1, lv[l].n2, AP, lv[l + 1].A, st));
    for (auto& L : lv) LCHK(launch_dense_jacobi_weights(L.A, L.N, h->p.omega, L.W, st));
    const Lv& C = lv.back();
    LCHK(launch_dense_inverse(C.A, (int)C.N, cwork, inv, info, st));
    int hinfo = 0;
    CCHK(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    CCHK(cudaStreamSynchronize(st));
    if (hinfo != 0) return h->fail(FDE_ERR_NONFINITE, "coarsest-grid matrix is singular");
    return FDE_OK;
  }

  int apply(fde_handle* h, size_t l, int mode, const double* x, const double* b, double* y) {
    Lv& L = lv[l];
    const int pi = h->pbeg(FDE_KCLASS_LEVEL_APPLY);
    LCHK(launch_dense_apply(mode, L.A, L.N, x, b, L.W, y, h->st));
    h->pend(pi);
    return FDE_OK;
  }

  // V-cycle on level l from x = 0 (ping-pong between x and kx as the P_2
  // hierarchy does); *out receives the buffer holding the result
  int cycle(fde_handle* h, size_t l, double** out) {
    Lv& L = lv[l];
    const fde_params& p = h->p;
    cudaStream_t st = h->st;
    double *x = L.x, *t = L.kx;
    if (l + 1 == lv.size()) {
      const int pi = h->pbeg(FDE_KCLASS_MG_OTHER);
      LCHK(launch_coarse_solve<double>(inv, (int)L.N, L.b, x, st));
      h->pend(pi);
      *out = x;
      return FDE_OK;
    }
    int pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    if (p.nu_pre >= 1) LCHK(launch_mul<double>(L.N, L.W, L.b, x, st));
    else CCHK(cudaMemsetAsync(x, 0, L.N * sizeof(double), st));
    h->pend(pi);
    for (int s = 1; s < p.nu_pre; ++s) {
      RCHK(apply(h, l, 2, x, L.b, t));
      std::swap(x, t);
    }
    RCHK(apply(h, l, 1, x, L.b, t));  // r = b - A x
    pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    LCHK(launch_restrict<double>(t, L.n1, L.n2, 1.0, lv[l + 1].b, st));  // R = P^T
    h->pend(pi);
    double* xc = nullptr;
    RCHK(cycle(h, l + 1, &xc));
    pi = h->pbeg(FDE_KCLASS_MG_OTHER);
    LCHK(launch_prolong_add<double>(xc, L.n1, L.n2, x, st));
    h->pend(pi);
    for (int s = 0; s < p.nu_post; ++s) {
      RCHK(apply(h, l, 2, x, L.b, t));
      std::swap(x, t);
    }
    *out = x;
    return FDE_OK;
  }

  double* root_out = nullptr;
  int cycle_root(fde_handle* h) override { return cycle(h, 0, &root_out); }

  int vcycle(fde_handle* h, const double* r, double* z, bool df_io) override {
    Lv& L = lv[0];
    if (df_io) LCHK(vcycle_in<double>(true, L.N, r, L.b, h->st));
    else CCHK(cudaMemcpyAsync(L.b, r, L.N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    RCHK(run_cycle(h));
    const int cycles = (h->p.cycles > 1 && lv.size() > 1) ? h->p.cycles : 1;
    if (cycles > 1) {
      // stationary iteration z_{k+1} = z_k + V(r - A_0 z_k): r is kept in acc_b
      CCHK(cudaMemcpyAsync(acc_b, L.b, L.N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
      for (int k = 1; k < cycles; ++k) {
        CCHK(cudaMemcpyAsync(acc_x, root_out, L.N * sizeof(double), cudaMemcpyDeviceToDevice,
                             h->st));
        RCHK(apply(h, 0, 1, acc_x, acc_b, L.b));
        RCHK(run_cycle(h));
        LCHK(launch_add<double>(L.N, acc_x, root_out, root_out, h->st));
      }
    }
    if (df_io) LCHK(vcycle_out<double>(true, L.N, root_out, z, h->st));
    else CCHK(cudaMemcpyAsync(z, root_out, L.N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return FDE_OK;
  }

  int level_apply(fde_handle* h, int l, const double* x, double* y) override {
    if (l < 0 || l >= (int)lv.size()) return h->fail(FDE_ERR_ARG, "level %d out of range", l);
    Lv& L = lv[l];
    CCHK(cudaMemcpyAsync(L.x, x, L.N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    LCHK(launch_dense_apply(0, L.A, L.N, L.x, nullptr, nullptr, y, h->st));
    return FDE_OK;
  }
};


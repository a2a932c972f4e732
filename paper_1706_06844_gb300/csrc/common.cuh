// Shared device types and the internal launch interface of libfde.
// Kernels live in kernels_*.cu; the host drivers (handle, V-cycle, FGMRES)
// in fde.cu call them only through the launchers declared here.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace fde {

struct df;  // double-float value (df32.cuh)

// ---------------------------------------------------------------- complex
template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
template <typename R>
__device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}

// ---------------------------------------------------------------- grid transfer
// One axis of the bilinear transfer of Sec. 4.1 (P = T(1 + cos) K): a fine
// axis of n points coarsens to m = (n - n mod 2) / 2 points, coarse point c
// sitting on fine point 2c + (n mod 2) (0-based; the down-sampling matrix K
// puts coarse j on fine 2j for odd n and on fine 2j - 1 for even n, 1-based);
// P's column c holds 1/2, 1, 1/2 at fine 2c + o - 1, 2c + o, 2c + o + 1,
// truncated at the ends of the axis (only even n reaches past fine 0).
__host__ __device__ __forceinline__ int coarse_n(int n) { return (n - (n & 1)) / 2; }
__host__ __device__ __forceinline__ int coarse_at(int n, int c) { return 2 * c + (n & 1); }
// coarse parents of fine point i and P's weights: returns their count (1 or 2)
template <typename T>
__host__ __device__ __forceinline__ int coarse_parents(int n, int i, int* q, T* w) {
  const int m = coarse_n(n), r = i - (n & 1);
  int k = 0;
  if ((r & 1) == 0 && r >= 0) {  // on a coarse point
    if (r / 2 < m) { q[k] = r / 2; w[k] = T(1); ++k; }
    return k;
  }
  const int lo = (r - 1) >> 1;  // between coarse lo and lo + 1
  if (lo >= 0 && lo < m) { q[k] = lo; w[k] = T(0.5); ++k; }
  if (lo + 1 >= 0 && lo + 1 < m) { q[k] = lo + 1; w[k] = T(0.5); ++k; }
  return k;
}

// ---------------------------------------------------------------- launches
// Every launcher returns the cudaError_t of its launch (cudaGetLastError()).

// Raise a kernel's dynamic shared-memory limit to 227 KB on the CURRENT
// device, once per (kernel, device): the attribute belongs to one device, so a
// process that launches on several GPUs sets it on each.  Thread-safe.
cudaError_t ensure_max_smem(const void* kernel);

// Circulant-embedding Toeplitz pass over a set of vectors (rows or columns of a
// grid).  For every vector v (elements x_v[i] = X[v*vs + i*es], i < n):
//   y_v[i] = cmass * M[v*vs + i*es] + cp[.] * (A x_v)_i + cm[.] * (A^T x_v)_i
// written to Y (accumulate = 0) or added to Y (accumulate = 1), where
// A = [t_{i-k}] is the lower-Hessenberg Toeplitz matrix whose spectra S1 (A)
// and S2 (A^T) were built by build_spectra for the same L.  M, cp, cm may be
// null (term omitted; null cp/cm means 1).  T: storage type, R: FFT arithmetic.
// C: storage type of the coefficient fields (T, or df for the double-float path).
// When two padded length-L buffers of cx<R> exceed shared memory (L = 8192 for
// 16-byte complex values) the pass keeps one buffer and parks the forward
// spectrum in `ws` (global memory, ws_elems cx<R> entries, at least L per
// concurrently resident CTA; cudaErrorInvalidValue if too small).
template <typename T, typename R, typename C>
cudaError_t launch_fft_pass(const T* X, int es, int vs, int nvec, int n, int logL,
                            const cx<R>* S1, const cx<R>* S2, const cx<R>* tw,
                            const C* cp, const C* cm, const T* M, double cmass,
                            T* Y, int accumulate, cudaStream_t st, cx<R>* ws = nullptr,
                            size_t ws_elems = 0);
// shared-memory bytes a pass of length 2^logL in cx<R> needs with two buffers
size_t fft_pass_two_buffer_bytes(int logL, size_t cx_bytes);
// the arguments of one pass (as launch_fft_pass's)
template <typename T, typename R, typename C>
struct FftPass {
  const T* X;
  int es, vs, nvec, n;
  const cx<R>*S1, *S2, *tw;
  const C *cp, *cm;
  const T* M;
  double cmass;
  T* Y;
  int accumulate;
};
// two independent passes of the same length 2^logL in one launch (their row
// pairs share the grid, so each pass's latency hides behind the other's);
// results are those of two launch_fft_pass calls.  Falls back to two launches
// where the one-buffer pass would be needed.
template <typename T, typename R, typename C>
cudaError_t launch_fft_pass2(const FftPass<T, R, C>& a, const FftPass<T, R, C>& b, int logL,
                             cudaStream_t st, cx<R>* ws = nullptr, size_t ws_elems = 0);

// Spectra of the circulant embeddings (length L = 2^logL >= 2n - 1) of A and A^T,
// A = [t_{i-k}], generator t_d at t[d+1] for d = -1..n-1, scaled by scale/L and
// stored in bit-reversed order.  Also fills (when tw is non-null) the twiddle
// table of length L - 1: tw[half - 1 + pos] = e^{-2 pi i pos/(2 half)}.
// For L whose twiddles do not fit in shared memory beside the transform
// (L = 8192), `tw_scratch` (L - 1 entries of global memory) holds them.
template <typename R>
cudaError_t launch_build_spectra(const double* t, int n, int logL, double scale, cx<R>* S1,
                                 cx<R>* S2, cx<R>* tw, cudaStream_t st,
                                 cx<double>* tw_scratch = nullptr);

// Direct summation version of launch_fft_pass (same contract), A given by the
// generator t (length n + 1, t_d at t[d+1]).
template <typename T>
cudaError_t launch_direct_pass(const T* X, int es, int vs, int nvec, int n, const T* t,
                               const T* cp, const T* cm, const T* M, double cmass, T* Y,
                               int accumulate, cudaStream_t st);

// Galerkin mass pre-pass of a structured-Galerkin level:
//   XBY = (B_y (x) I) x,  XBX = (I (x) B_x) x,  MASS = c (B_y (x) B_x) x
// with B = tridiag(b1, b0, b1) per axis.
template <typename T>
cudaError_t launch_mass_prepass(const T* X, int n1, int n2, double bx0, double bx1, double by0,
                                double by1, double c, T* XBY, T* XBX, T* MASS, cudaStream_t st);

// Level epilogue on K x (already summed in KX):
//   mode 0: Y = KX;  mode 1: Y = B - KX;  mode 2: Y = X + W (B - KX)
template <typename T>
cudaError_t launch_level_epilogue(int mode, size_t N, const T* KX, const T* B, const T* X,
                                  const T* W, T* Y, cudaStream_t st);

// out[c][r] = in[r][c] (in: rows x cols, out: cols x rows); add = 1: out[c][r] += in[r][c]
template <typename T>
cudaError_t launch_transpose(const T* in, int rows, int cols, T* out, int add, cudaStream_t st);

// Y = W * B (Jacobi sweep from a zero guess)
template <typename T>
cudaError_t launch_mul(size_t N, const T* W, const T* B, T* Y, cudaStream_t st);

// coarse b_c = rscale * P^T r (bilinear P of the transfer above, any fine sizes)
template <typename T>
cudaError_t launch_restrict(const T* R, int n1, int n2, double rscale, T* BC, cudaStream_t st);
// mass-term pre-pass with (I (x) B_x) x written transposed (XBXT, n1 x n2);
// W, B non-null: X = W B first (as launch_jacobi_mass_prepass), else X is read
template <typename T>
cudaError_t launch_mass_prepass_t(const T* W, const T* B, int n1, int n2, double bx0, double bx1,
                                  double by0, double by1, double c, T* X, T* XBY, T* XBXT,
                                  T* MASS, cudaStream_t st);
// out = transpose(in) added to KX, then X <- X + W (B - out) (out not stored)
template <typename T>
cudaError_t launch_transpose_smooth(const T* in, int rows, int cols, const T* KX, const T* B,
                                    const T* W, T* X, cudaStream_t st);
// restriction of the residual B - KX without storing it
template <typename T>
cudaError_t launch_restrict_residual(const T* B, const T* KX, int n1, int n2, double rscale,
                                     T* BC, cudaStream_t st);
// the Jacobi sweep from zero X = W B fused into the mass-term pre-pass of X
template <typename T>
cudaError_t launch_jacobi_mass_prepass(const T* W, const T* B, int n1, int n2, double bx0,
                                       double bx1, double by0, double by1, double c, T* X,
                                       T* XBY, T* XBX, T* MASS, cudaStream_t st);

// X += P x_c
template <typename T>
cudaError_t launch_prolong_add(const T* XC, int n1, int n2, T* X, cudaStream_t st);

// Y[i] = (TO)(scale * X[i])
template <typename TI, typename TO>
cudaError_t launch_convert(size_t N, const TI* X, double scale, TO* Y, cudaStream_t st);

// double -> double-float copy of a field, scaled: Y = scale * X
cudaError_t launch_to_df(size_t N, const double* X, double scale, df* Y, cudaStream_t st);
// Y = A - B (FP64)
cudaError_t launch_sub(size_t N, const double* A, const double* B, double* Y, cudaStream_t st);

// ---- setup
// w_0..w_K of the WSGD family (p = 1, q in {0,-1}) by the Grunwald recurrence, FP64.
cudaError_t launch_wsgd_weights(double gamma, int q, int K, double* w, cudaStream_t st);
// level-0 generator t_d = scale * (-w_{d+1}), d = -1..n-1 (t[d+1])
cudaError_t launch_generator_from_weights(const double* w, int n, double scale, double* t,
                                          cudaStream_t st);
// q-coarsening t^c_d = sum_m q_m t_{2d+m}, q = (1/4, 1, 3/2, 1, 1/4)
cudaError_t launch_coarsen_generator(const double* t, int n, double* tc, int nc,
                                     cudaStream_t st);
// coarse coefficient injection F_c[jc][ic] = F[coarse_at(n2, jc)][coarse_at(n1, ic)]
template <typename T>
cudaError_t launch_inject(const T* F, int n1, int n2, T* FC, cudaStream_t st);
// per-level fields: dp, dm, ep, em (ep, em scaled by sigma), W = omega/diag(K_l)
// from FP64 fine coefficients at the level's nodes: level point (j, i) is
// finest point (stride j + offy, stride i + offx), stride = 2^l, the offsets
// summing the per-level shifts n_t mod 2 of the transfer: off = sum_t 2^t (n_t & 1).
template <typename T>
cudaError_t launch_level_fields(const double* dp, const double* dm, const double* ep,
                                const double* em, int n1f, int n1, int n2, int stride, int offx,
                                int offy, double sigma, double c, double bx0, double by0,
                                const double* tx, const double* ty, double omega, T* odp, T* odm,
                                T* oep, T* oem, T* W, cudaStream_t st);
// out = a X + b Y + c Z (Z may be null when c == 0), FP64
cudaError_t launch_lincomb(size_t N, double a, const double* X, double b, const double* Y,
                           double c, const double* Z, double* out, cudaStream_t st);
// dense coarsest operator (N = n1 n2), LU with partial pivoting, explicit inverse (FP64)
cudaError_t launch_coarse_inverse(const double* tx, const double* ty, int n1, int n2,
                                  double bx0, double bx1, double by0, double by1, double c,
                                  const double* dp, const double* dm, const double* ep,
                                  const double* em, double* work, double* inv, int* info,
                                  cudaStream_t st);
// x = inv * b  (b, x in T; inv FP64)
template <typename T>
cudaError_t launch_coarse_solve(const double* inv, int N, const T* b, T* x, cudaStream_t st);

// ---- the small end of a V-cycle in one launch (kernels_tail.cu): levels with
// n <= kTailN, from the first such level down to the coarsest, all in one CTA
constexpr int kTailN = 31;
constexpr int kTailMaxLevels = 8;
template <typename T>
struct TailLevel {
  int n1, n2;
  T *x, *b, *kx;
  const T *W, *dp, *dm, *ep, *em, *tx, *ty;  // tx, ty: generators t_d at [d + 1], d = -1..n-1
  T *xby, *xbx, *mass;                       // structured-Galerkin mass terms (null: level 0 / none)
  T bx0, bx1, by0, by1;
};
template <typename T>
struct TailArgs {
  TailLevel<T> lv[kTailMaxLevels];  // lv[0] = first tail level, lv[nlev - 1] = coarsest
  int nlev, nu_pre, nu_post;
  double c, rscale;
  const double* inv;  // explicit inverse of the coarsest operator (FP64, row-major)
};
template <typename T>
cudaError_t launch_mg_tail(const TailArgs<T>& a, cudaStream_t st);

// ---- nine-point stencil levels (P_2 of Sec. 4.3; layout S[o * N + j * n1 + i],
// o = 3 (dy + 1) + (dx + 1), coefficients reaching outside the grid are zero)
// level 0: P_2 = c I + (D+ + D-)(I (x) A2) + sigma (E+ + E-)(A2 (x) I), A2 = tridiag(-1, 2, -1)
cudaError_t launch_p2_fields(const double* dp, const double* dm, const double* ep,
                             const double* em, int n1, int n2, double c, double sigma, double* S,
                             cudaStream_t st);
// Galerkin coarse stencil P^T K P (bilinear P), fine n1 x n2 -> coarse m1 x m2 (FP64)
cudaError_t launch_galerkin9(const double* Sf, int n1, int n2, double* Sc, int m1, int m2,
                             cudaStream_t st);
// ST = (T) S (skipped when ST is null), W = omega / diag
template <typename T>
cudaError_t launch_stencil_convert(const double* S, size_t N, double omega, T* ST, T* W,
                                   cudaStream_t st);
// mode 0: Y = K X; 1: Y = B - K X; 2: Y = X + W (B - K X). Y must not alias X.
template <typename T>
cudaError_t launch_stencil_apply(int mode, bool five, const T* S, int n1, int n2, const T* X,
                                 const T* B, const T* W, T* Y, cudaStream_t st);
template <typename T>
cudaError_t launch_add(size_t N, const T* A, const T* B, T* Y, cudaStream_t st);
// explicit inverse of a stencil level's dense operator (N = n1 n2 <= 1024; work 2 N^2)
cudaError_t launch_stencil_inverse(const double* S, int n1, int n2, double* work, double* inv,
                                   int* info, cudaStream_t st);

// ---- dense levels (exact Galerkin validation mode, N_l x N_l row-major FP64)
// level 0: M of Eq. (M) from the generators t_d = -w_{d+1} (t[d + 1]) and the
// unscaled coefficients
cudaError_t launch_dense_assemble(const double* tx, const double* ty, int n1, int n2, double c,
                                  double sigma, const double* dp, const double* dm,
                                  const double* ep, const double* em, double* A, cudaStream_t st);
// Ac = P^T A P for the fine n1 x n2 grid (AP: N_f x N_c scratch)
cudaError_t launch_dense_galerkin(const double* A, int n1, int n2, double* AP, double* Ac,
                                  cudaStream_t st);
cudaError_t launch_dense_jacobi_weights(const double* A, size_t N, double omega, double* W,
                                        cudaStream_t st);
// mode 0: Y = A X; 1: Y = B - A X; 2: Y = X + W (B - A X).  Y must not alias X.
cudaError_t launch_dense_apply(int mode, const double* A, size_t N, const double* X,
                               const double* B, const double* W, double* Y, cudaStream_t st);
// explicit inverse of a dense N x N matrix (N <= 1024; work 2 N^2)
cudaError_t launch_dense_inverse(const double* K, int N, double* work, double* inv, int* info,
                                 cudaStream_t st);

// ---- Krylov (FP64)
// partial dots: part[i * nb + blk] = sum over block chunk of V_i . w  (i < k)
cudaError_t launch_dots(const double* V, size_t ldv, int k, const double* w, size_t N,
                        double* part, int nb, cudaStream_t st);
// w -= sum_i h_i V_i (i < k); mode 1: partial sums of |w_new|^2 into part[blk];
// mode 2 (k <= 16): partial dots V_i . w_new into part[i * nb + blk]
cudaError_t launch_axpy_dots(const double* V, size_t ldv, int k, const double* h, double* w,
                             size_t N, double* part, int nb, int mode, cudaStream_t st);
// out[i] = sum_b part[i * nb + b] (+ out[i] if add), i < k (one block)
cudaError_t launch_reduce(const double* part, int k, int nb, double* out, int add,
                          cudaStream_t st);
// y = x * (1/s[0])
cudaError_t launch_scale_inv(size_t N, const double* x, const double* s, double* y,
                             cudaStream_t st);
// x += sum_i c_i Z_i
cudaError_t launch_update(const double* Z, size_t ldz, int k, const double* c, double* x,
                          size_t N, cudaStream_t st);
// partial sums of squares of x
cudaError_t launch_sumsq(const double* x, size_t N, double* part, int nb, cudaStream_t st);

int krylov_blocks();

// ---- Arnoldi state on the device (FGMRES, Sec. 5): the rotated Hessenberg
// matrix R ((m + 1) x m, column j at R[j (m + 1) ..]), the Givens rotations,
// the rotated right-hand side g, and the status the host reads after a step
struct ArnoldiStatus {
  double gabs;      // |g_{j+1}|: the FGMRES residual estimate after the step
  double hnext;     // ||w|| before normalisation (0: exact breakdown)
  double inv_norm;  // 1 / hnext (scales w into the next basis vector)
  int nonfinite;    // a Hessenberg entry was NaN or Inf
  int pad;
};
struct ArnoldiState {
  static constexpr int kMaxM = 64;
  int m;
  double *R, *cs, *sn, *g;
  ArnoldiStatus* status;
  // delayed re-orthogonalisation (launch_dcgs2): the unrotated Hessenberg
  // columns ((m + 1) x m, column j at H[j (m + 1) ..]) and g_j as it was before
  // rotation j, so that column j - 1 can be corrected and re-rotated one step late
  double* H = nullptr;
  double* gpre = nullptr;
};
// one Arnoldi step j (k = j + 1 basis vectors V_0 .. V_j, w = the new vector):
// CGS2 in three fused passes over V, the Givens update of column j in the
// last block of the third pass, then w /= ||w||.  ldv and N even (the basis is
// zero-padded), k <= 32; part: cgs_blocks() * 32 doubles (cgs_blocks() is the
// largest grid a pass uses: the blocks the GPU holds at once); tickets: 3 counters
// that start at zero (each pass resets its own).
cudaError_t launch_cgs2(const double* V, size_t ldv, int k, double* w, size_t N, double* part,
                        unsigned* tickets, double* h, double* h2, const ArnoldiState& st, int j,
                        cudaStream_t s);
// Arnoldi step j with delayed re-orthogonalisation (DCGS2), two fused passes
// over V_0 .. V_{j-1}: the first projects both the new vector w = V_{j+1} and
// the once-orthogonalised V_j, the second re-orthogonalises V_j, orthogonalises
// w against the corrected basis and takes ||w||; the Givens updates run in the
// last block of each pass (column j - 1 final, column j provisional), then
// w /= ||w||.  df_store: the basis holds double-float vectors (hi, lo FP32
// pairs, 8 bytes an element like FP64) and the passes compute in double-float
// on the FP32 pipes; otherwise FP64 vectors and arithmetic.  j < kDcgsMax;
// ldv and N even; part: cgs_blocks() * (2 kDcgsMax + 2) doubles; coef:
// kDcgsCoef doubles; tickets[0..1] zero at rest.
constexpr int kDcgsMax = 32;
constexpr int kDcgsCoef = 2 * kDcgsMax + 2;
cudaError_t launch_dcgs2(double* V, size_t ldv, int j, size_t N, double* part, unsigned* tickets,
                         double* coef, const ArnoldiState& st, bool df_store, cudaStream_t s);
// y_df = x / *s (FP64 in, double-float out); x += Z_df c (k <= kDcgsMax)
cudaError_t launch_scale_inv_df(size_t N, const double* x, const double* s, double* y_df,
                                cudaStream_t st);
cudaError_t launch_update_df(const double* Z_df, size_t ldz, int k, const double* c, double* x,
                             size_t N, cudaStream_t st);
// k > 32: the same step from separate passes (dots, reduce, axpy); the Givens
// update and the scaling as above
cudaError_t launch_arnoldi_column(const ArnoldiState& st, int j, const double* h,
                                  const double* h2, const double* nrm2, cudaStream_t s);
cudaError_t launch_scale_by(double* w, size_t N, const ArnoldiStatus* status, cudaStream_t s);
// g = (beta, 0, ...), beta read from device memory; status.gabs = beta
cudaError_t launch_arnoldi_start(const ArnoldiState& st, const double* beta_dev, cudaStream_t s);
// y = R^{-1} g for the first k columns
cudaError_t launch_arnoldi_lsq(const ArnoldiState& st, int k, double* y, cudaStream_t s);
int cgs_blocks();
// integer conversions against the CUDA ones (fde_conversion_selftest); 0 on success
int conversion_selftest(long long n, long long* mismatches);

// ---------------------------------------------------------------- grouped launches
// Many independent problems advanced by one launch per stage (the batch
// engine): a launch takes an array of per-call argument records ("entries",
// one per problem, the same arguments the single-problem launcher takes) and
// a work list of (entry, unit) items; a unit is a vector pair of an FFT pass,
// a vector of a direct pass, a 32 x 32 tile of a transpose or a chunk of an
// element-wise stage.  An entry runs only while its problem is active
// (gate.active[prob] != 0) and, when want >= 0, while gate.relax[prob] == want.
struct GGate {
  const int* active;
  const int* relax;
};
struct GItem {
  int e;     // entry index
  int unit;  // unit within the entry
};
__device__ __forceinline__ bool gate_open(const GGate& g, int prob, int want) {
  return g.active[prob] != 0 && (want < 0 || g.relax[prob] == want);
}
constexpr int kGChunk = 2048;  // elements per chunk of an element-wise stage

template <typename T, typename R, typename C>
struct GFftPass {
  const T* X;
  int es, vs, nvec, n, logL;
  const cx<R>*S1, *S2, *tw;
  const C *cp, *cm;
  const T* M;
  double cmass;
  T* Y;
  int accumulate, prob, want;
};
// the largest logL of the entries sets the shared memory (two padded buffers)
template <typename T, typename R, typename C>
cudaError_t launch_g_fft_pass(const GFftPass<T, R, C>* ent, const GItem* items, int nitems,
                              int max_logL, GGate gate, cudaStream_t st);

template <typename T>
struct GDirectPass {
  const T* X;
  int es, vs, nvec, n;
  const T *t, *cp, *cm, *M;
  double cmass;
  T* Y;
  int accumulate, prob, want;
};
template <typename T>
cudaError_t launch_g_direct_pass(const GDirectPass<T>* ent, const GItem* items, int nitems,
                                 int max_n, GGate gate, cudaStream_t st);

template <typename T>
struct GTranspose {
  const T* in;
  int rows, cols;
  T* out;
  int add, prob, want;
};
template <typename T>
cudaError_t launch_g_transpose(const GTranspose<T>* ent, const GItem* items, int nitems,
                               GGate gate, cudaStream_t st);

// element-wise and stencil stages of a V-cycle level, one record per problem
enum GOp : int {
  G_MUL = 0,       // x = W b
  G_RESID = 1,     // kx = b - kx
  G_SMOOTH = 2,    // x = x + W (b - kx)
  G_MASS = 3,      // xby, xbx, mass from x (structured-Galerkin level > 0)
  G_RESTRICT = 4,  // bc = rscale P^T kx (units over the coarse grid)
  G_PROLONG = 5,   // x += P xc
};
template <typename T>
struct GLevelOp {
  int n1, n2;
  T *x, *b, *kx, *W;
  T *xby, *xbx, *mass;
  T bx0, bx1, by0, by1, c;
  T *bc, *xc;  // next level's right-hand side and solution
  T rscale;
  int prob;
};
template <typename T>
cudaError_t launch_g_level_op(int op, const GLevelOp<T>* ent, const GItem* items, int nitems,
                              GGate gate, cudaStream_t st);

// ---- grouped FGMRES (Sec. 5) of many problems in lockstep: iteration j of
// every active problem in one launch per pass; per-problem reductions finish
// in the block that completes a problem's chunks last
constexpr int kGKChunk = 4096;  // double2 pairs per chunk of a Krylov pass
struct GSolveState {
  double bnorm;         // ||b||
  double beta;          // residual norm at the start of the current cycle
  double tol;           // rtol ||b||
  double rel_residual;  // ||b - M x|| / ||b|| of the last true residual
  int its;              // inner iterations of this solve
  int k;                // columns of the current cycle
  int restarts, relaxed, converged, failed;  // failed: a non-finite value was met
};
struct GKrylov {
  double *V, *Z;   // padded bases, column pitch ldv (zero padding)
  size_t ldv, N;   // N: grid points
  double* part;    // this problem's partial sums: nchunk * 32
  unsigned* tickets;  // 4 counters, zero at rest
  double *h, *h2, *y, *scal;  // projections, least-squares solution, scratch scalars
  ArnoldiState st;
  GSolveState* ss;
  double rtol;
  int maxit, relax_on, restart, nchunk, prob;
};
// passes of Arnoldi step j (k = j + 1 <= 32) over the entries' chunks; the
// last one also updates ss (iterations, k), status and the gates: active =
// not (|g_{j+1}| <= tol or its >= maxit or breakdown or non-finite), relax =
// relax_on and |g_{j+1}| <= FDE_RELAX_FACTOR tol
cudaError_t launch_g_cgs2(const GKrylov* ent, const GItem* items, int nitems, int j, GGate gate,
                          int* active, int* relax, cudaStream_t st);
// element-wise vector stages of the grouped solve
enum GVOp : int {
  GV_D2F = 0,        // yf = (float) a
  GV_F2D = 1,        // y = (double) af
  GV_SUB = 2,        // y = a - b
  GV_LINCOMB = 3,    // y = s0 a + s1 b + s2 c
  GV_SCALE_INV = 4,  // y = a / sptr[0]
  GV_ZERO = 5,       // y = 0
  GV_COPY = 6,       // y = a
};
struct GVec {
  const double *a, *b, *c;
  const float* af;
  double* y;
  float* yf;
  double s0, s1, s2;
  const double* sptr;
  size_t N;
  int prob;
};
cudaError_t launch_g_vec(int op, const GVec* ent, const GItem* items, int nitems, GGate gate,
                         cudaStream_t st);
// out[e] = ||a_e|| per entry (deterministic per-problem reduction); ent[e].y
// receives the norm at ent[e].y[0]; uses ticket slot 3 of the problem's
// GKrylov (same index) and its partials
cudaError_t launch_g_norm(const GVec* ent, const GKrylov* kry, const GItem* items, int nitems,
                          GGate gate, cudaStream_t st);
// start of a solve: ss = ||b|| (scal[0]), tol; problems with b = 0 finish at
// once (x = 0 written by the caller); gates active = incycle = (b != 0)
cudaError_t launch_g_solve_start(const GKrylov* ent, int count, int* active, int* incycle,
                                 cudaStream_t st);
// start of a cycle: g = (beta, 0, ...), beta = scal[1] (or ||b|| on the first
// cycle), k = 0, restarts += 1, active = incycle, relax from |g_0| = beta
cudaError_t launch_g_cycle_start(const GKrylov* ent, int count, int first, const int* incycle,
                                 int* active, int* relax, cudaStream_t st);
// end of a cycle: y = R^{-1} g over the problem's k columns
cudaError_t launch_g_lsq(const GKrylov* ent, int count, const int* incycle, cudaStream_t st);
// x += Z y over k columns (items over the grid, x the problem's solution)
cudaError_t launch_g_update(const GKrylov* ent, double* const* x, const GItem* items, int nitems,
                            const int* incycle, cudaStream_t st);
// after the true residual norm (scal[1]): rel_residual, converged; incycle =
// not converged and its < maxit and not failed
cudaError_t launch_g_cycle_end(const GKrylov* ent, int count, int* incycle, cudaStream_t st);

// the one-launch end of every problem's cycle: one CTA per entry
template <typename T>
cudaError_t launch_g_mg_tail(const TailArgs<T>* args, const int* probs, int count, GGate gate,
                             cudaStream_t st);

}  // namespace fde

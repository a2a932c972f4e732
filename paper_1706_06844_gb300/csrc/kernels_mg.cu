// Multigrid kernels (Sec. 4) and device-side setup (Sec. 2 weights, coarse
// operators, coarsest-grid direct solve).  Grid functions are row-major
// n2 x n1 arrays (x fastest).
#include "common.cuh"
#include "df32.cuh"

namespace fde {

static inline int grid_for(size_t N, int threads) {
  size_t g = (N + threads - 1) / threads;
  const size_t cap = 152 * 16;
  return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

// ---------------------------------------------------------------- level ops
// W, B non-null: x is first the Jacobi sweep from zero, x = W b, formed at
// every point it is read and written to X (one pass instead of two; the same
// products, so the same values)
template <typename T>
__global__ void mass_prepass_kernel(T* X, int n1, int n2, T bx0, T bx1, T by0, T by1, T c,
                                    T* __restrict__ XBY, T* __restrict__ XBX,
                                    T* __restrict__ MASS, const T* __restrict__ W,
                                    const T* __restrict__ B) {
  const size_t N = (size_t)n1 * n2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n1), j = (int)(idx / n1);
    auto at = [&](int jj, int ii) -> T {
      if (ii < 0 || ii >= n1 || jj < 0 || jj >= n2) return T(0);
      const size_t k = (size_t)jj * n1 + ii;
      return W ? W[k] * B[k] : X[k];
    };
    // (B_y (x) I) x: tridiagonal along y;  (I (x) B_x) x: along x
    const T xc = at(j, i);
    if (W) X[idx] = xc;
    const T up = at(j - 1, i), dn = at(j + 1, i), lf = at(j, i - 1), rt = at(j, i + 1);
    XBY[idx] = by1 * up + by0 * xc + by1 * dn;
    XBX[idx] = bx1 * lf + bx0 * xc + bx1 * rt;
    const T rowm = bx1 * at(j - 1, i - 1) + bx0 * up + bx1 * at(j - 1, i + 1);
    const T row0 = bx1 * lf + bx0 * xc + bx1 * rt;
    const T rowp = bx1 * at(j + 1, i - 1) + bx0 * dn + bx1 * at(j + 1, i + 1);
    MASS[idx] = c * (by1 * rowm + by0 * row0 + by1 * rowp);
  }
}

// The same pre-pass over 32 x 32 tiles (x and its one-point halo staged in
// shared memory) that writes (I (x) B_x) x TRANSPOSED (n1 x n2, XBXT) for
// the FFT path's column pass, saving that pass's separate transpose.
template <typename T>
__global__ void mass_prepass_t_kernel(T* X, int n1, int n2, T bx0, T bx1, T by0, T by1, T c,
                                      T* __restrict__ XBY, T* __restrict__ XBXT,
                                      T* __restrict__ MASS, const T* __restrict__ W,
                                      const T* __restrict__ B) {
  __shared__ T xs[34][35];
  __shared__ T tb[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int k = tid; k < 34 * 34; k += 32 * blockDim.y) {
    const int jj = j0 - 1 + k / 34, ii = i0 - 1 + k % 34;
    T v = T(0);
    if (ii >= 0 && ii < n1 && jj >= 0 && jj < n2) {
      const size_t q = (size_t)jj * n1 + ii;
      v = W ? W[q] * B[q] : X[q];
    }
    xs[k / 34][k % 34] = v;
  }
  __syncthreads();
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, i = i0 + tx;
    if (i < n1 && j < n2) {
      const size_t idx = (size_t)j * n1 + i;
      const T xc = xs[r + 1][tx + 1];
      const T up = xs[r][tx + 1], dn = xs[r + 2][tx + 1], lf = xs[r + 1][tx],
              rt = xs[r + 1][tx + 2];
      if (W) X[idx] = xc;
      XBY[idx] = by1 * up + by0 * xc + by1 * dn;
      tb[r][tx] = bx1 * lf + bx0 * xc + bx1 * rt;
      const T rowm = bx1 * xs[r][tx] + bx0 * up + bx1 * xs[r][tx + 2];
      const T row0 = bx1 * lf + bx0 * xc + bx1 * rt;
      const T rowp = bx1 * xs[r + 2][tx] + bx0 * dn + bx1 * xs[r + 2][tx + 2];
      MASS[idx] = c * (by1 * rowm + by0 * row0 + by1 * rowp);
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + tx;
    if (i < n1 && j < n2) XBXT[(size_t)i * n2 + j] = tb[tx][r];
  }
}

template <typename T>
cudaError_t launch_mass_prepass_t(const T* W, const T* B, int n1, int n2, double bx0, double bx1,
                                  double by0, double by1, double c, T* X, T* XBY, T* XBXT,
                                  T* MASS, cudaStream_t st) {
  dim3 grid((n1 + 31) / 32, (n2 + 31) / 32), block(32, 8);
  mass_prepass_t_kernel<T><<<grid, block, 0, st>>>(X, n1, n2, T(bx0), T(bx1), T(by0), T(by1),
                                                   T(c), XBY, XBXT, MASS, W, B);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mass_prepass(const T* X, int n1, int n2, double bx0, double bx1, double by0,
                                double by1, double c, T* XBY, T* XBX, T* MASS, cudaStream_t st) {
  const size_t N = (size_t)n1 * n2;
  mass_prepass_kernel<T><<<grid_for(N, 256), 256, 0, st>>>(
      const_cast<T*>(X), n1, n2, T(bx0), T(bx1), T(by0), T(by1), T(c), XBY, XBX, MASS, nullptr,
      nullptr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi_mass_prepass(const T* W, const T* B, int n1, int n2, double bx0,
                                       double bx1, double by0, double by1, double c, T* X,
                                       T* XBY, T* XBX, T* MASS, cudaStream_t st) {
  const size_t N = (size_t)n1 * n2;
  mass_prepass_kernel<T><<<grid_for(N, 256), 256, 0, st>>>(
      X, n1, n2, T(bx0), T(bx1), T(by0), T(by1), T(c), XBY, XBX, MASS, W, B);
  return cudaGetLastError();
}

template <typename T>
__global__ void level_epilogue_kernel(int mode, size_t N, const T* __restrict__ KX,
                                      const T* __restrict__ B, const T* X,
                                      const T* __restrict__ W, T* Y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const T kx = KX[i];
    if (mode == 0) Y[i] = kx;
    else if (mode == 1) Y[i] = B[i] - kx;
    else Y[i] = X[i] + W[i] * (B[i] - kx);
  }
}

template <typename T>
cudaError_t launch_level_epilogue(int mode, size_t N, const T* KX, const T* B, const T* X,
                                  const T* W, T* Y, cudaStream_t st) {
  level_epilogue_kernel<T><<<grid_for(N, 256), 256, 0, st>>>(mode, N, KX, B, X, W, Y);
  return cudaGetLastError();
}

// 32 x 32 tiles through shared memory (padded against bank conflicts); both the
// read of `in` and the write of `out` are row segments
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ in, int rows, int cols, T* out, int add) {
  __shared__ T tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;  // out row c, column r
    if (r < rows && c < cols) {
      const size_t o = (size_t)c * rows + r;
      out[o] = add ? out[o] + tile[threadIdx.x][k] : tile[threadIdx.x][k];
    }
  }
}

// the last step of a level's smoothing sweep on the FFT path: the transposed
// y products are added to the x products KX and the damped-Jacobi update
// X <- X + W (B - KX) is applied in the same pass (KX itself is not stored)
template <typename T>
__global__ void transpose_smooth_kernel(const T* __restrict__ in, int rows, int cols,
                                        const T* __restrict__ KX, const T* __restrict__ B,
                                        const T* __restrict__ W, T* X) {
  __shared__ T tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;  // out row c, column r
    if (r < rows && c < cols) {
      const size_t o = (size_t)c * rows + r;
      const T kx = KX[o] + tile[threadIdx.x][k];
      X[o] = X[o] + W[o] * (B[o] - kx);
    }
  }
}

template <typename T>
cudaError_t launch_transpose_smooth(const T* in, int rows, int cols, const T* KX, const T* B,
                                    const T* W, T* X, cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  transpose_smooth_kernel<T><<<grid, block, 0, st>>>(in, rows, cols, KX, B, W, X);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_transpose(const T* in, int rows, int cols, T* out, int add, cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  transpose_kernel<T><<<grid, block, 0, st>>>(in, rows, cols, out, add);
  return cudaGetLastError();
}

template <typename T>
__global__ void mul_kernel(size_t N, const T* __restrict__ W, const T* __restrict__ B, T* Y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    Y[i] = W[i] * B[i];
}

template <typename T>
cudaError_t launch_mul(size_t N, const T* W, const T* B, T* Y, cudaStream_t st) {
  mul_kernel<T><<<grid_for(N, 256), 256, 0, st>>>(N, W, B, Y);
  return cudaGetLastError();
}

// b_c = rscale * (P_y (x) P_x)^T r, P column stencil (1/2, 1, 1/2) centred on
// fine coarse_at(n, c), truncated at the ends of each axis
// B non-null: restrict the residual B - R, formed at every point it is read
// (the same subtraction as a separate residual pass, so the same values)
template <typename T>
__global__ void restrict_kernel(const T* __restrict__ R, int n1, int n2, T rscale,
                                T* __restrict__ BC, const T* __restrict__ B) {
  const int m1 = coarse_n(n1), m2 = coarse_n(n2);
  const size_t NC = (size_t)m1 * m2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < NC;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int ic = (int)(idx % m1), jc = (int)(idx / m1);
    const int i = coarse_at(n1, ic), j = coarse_at(n2, jc);
    const T h = T(0.5);
    T acc = T(0);
    for (int dj = -1; dj <= 1; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= n2) continue;
      const size_t o = (size_t)jj * n1;
      auto r = [&](int ii) -> T { return B ? B[o + ii] - R[o + ii] : R[o + ii]; };
      T sr = r(i);
      if (i > 0) sr += h * r(i - 1);
      if (i + 1 < n1) sr += h * r(i + 1);
      acc += (dj ? h : T(1)) * sr;
    }
    BC[idx] = rscale * acc;
  }
}

template <typename T>
cudaError_t launch_restrict(const T* R, int n1, int n2, double rscale, T* BC, cudaStream_t st) {
  const size_t NC = (size_t)coarse_n(n1) * coarse_n(n2);
  restrict_kernel<T><<<grid_for(NC, 256), 256, 0, st>>>(R, n1, n2, T(rscale), BC, nullptr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict_residual(const T* B, const T* KX, int n1, int n2, double rscale,
                                     T* BC, cudaStream_t st) {
  const size_t NC = (size_t)coarse_n(n1) * coarse_n(n2);
  restrict_kernel<T><<<grid_for(NC, 256), 256, 0, st>>>(KX, n1, n2, T(rscale), BC, B);
  return cudaGetLastError();
}

// x += (P_y (x) P_x) x_c
template <typename T>
__global__ void prolong_add_kernel(const T* __restrict__ XC, int n1, int n2, T* X) {
  const int m1 = coarse_n(n1);
  const size_t N = (size_t)n1 * n2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n1), j = (int)(idx / n1);
    int ci[2], cj[2];
    T wi[2], wj[2];
    const int ni = coarse_parents<T>(n1, i, ci, wi);
    const int nj = coarse_parents<T>(n2, j, cj, wj);
    T s = T(0);
    for (int b = 0; b < nj; ++b)
      for (int a = 0; a < ni; ++a) s += wj[b] * wi[a] * XC[(size_t)cj[b] * m1 + ci[a]];
    X[idx] += s;
  }
}

template <typename T>
cudaError_t launch_prolong_add(const T* XC, int n1, int n2, T* X, cudaStream_t st) {
  const size_t N = (size_t)n1 * n2;
  prolong_add_kernel<T><<<grid_for(N, 256), 256, 0, st>>>(XC, n1, n2, X);
  return cudaGetLastError();
}

// Y = scale X; at scale 1 (the V-cycle's input and output) FP32 <-> FP64 runs
// through the integer conversions, bit-identical to the FP64 instructions,
// which run at the FP64 rate on GB300
template <typename TI, typename TO>
__global__ void convert_kernel(size_t N, const TI* __restrict__ X, double scale, TO* Y) {
  const bool unit = scale == 1.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    Y[i] = unit ? cvt<TO>(X[i]) : (TO)(scale * (double)X[i]);
}

template <typename TI, typename TO>
cudaError_t launch_convert(size_t N, const TI* X, double scale, TO* Y, cudaStream_t st) {
  convert_kernel<TI, TO><<<grid_for(N, 256), 256, 0, st>>>(N, X, scale, Y);
  return cudaGetLastError();
}

__global__ void to_df_kernel(size_t N, const double* __restrict__ X, double scale, df* Y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const double v = scale * X[i];
    const float h = __double2float_rn(v);
    Y[i] = fast_two_sum(h, __double2float_rn(v - (double)h));
  }
}

cudaError_t launch_to_df(size_t N, const double* X, double scale, df* Y, cudaStream_t st) {
  to_df_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, X, scale, Y);
  return cudaGetLastError();
}

__global__ void sub_kernel(size_t N, const double* __restrict__ A, const double* __restrict__ B,
                           double* Y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    Y[i] = A[i] - B[i];
}

cudaError_t launch_sub(size_t N, const double* A, const double* B, double* Y, cudaStream_t st) {
  sub_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, A, B, Y);
  return cudaGetLastError();
}

__global__ void lincomb_kernel(size_t N, double a, const double* __restrict__ X, double b,
                               const double* __restrict__ Y, double c,
                               const double* __restrict__ Z, double* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = a * X[i] + b * Y[i];
    if (Z) v += c * Z[i];
    out[i] = v;
  }
}

cudaError_t launch_lincomb(size_t N, double a, const double* X, double b, const double* Y,
                           double c, const double* Z, double* out, cudaStream_t st) {
  lincomb_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, a, X, b, Y, c, Z, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- setup
// Eq. (gk) by the recurrence g_k = g_{k-1} (k - 1 - gamma)/k, then the WSGD
// combination w_k = lp g_k + lq g_{k-(p-q)} with lp = (gamma - 2q)/(2(p-q)),
// lq = (2p - gamma)/(2(p-q)), p = 1 (Eq. w for q = 0).  One thread: the
// recurrence is sequential and O(n).
__global__ void wsgd_kernel(double gamma, int q, int K, double* w) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int d = 1 - q;
  const double lp = (gamma - 2.0 * q) / (2.0 * d), lq = (2.0 - gamma) / (2.0 * d);
  double g = 1.0, gm1 = 0.0, gm2 = 0.0;  // g_k, g_{k-1}, g_{k-2}
  for (int k = 0; k <= K; ++k) {
    if (k > 0) {
      gm2 = gm1;
      gm1 = g;
      g = g * ((double)(k - 1) - gamma) / (double)k;
    }
    const double gs = (d == 1) ? gm1 : gm2;  // g_{k-d}
    w[k] = lp * g + lq * (k >= d ? gs : 0.0);
  }
}

cudaError_t launch_wsgd_weights(double gamma, int q, int K, double* w, cudaStream_t st) {
  wsgd_kernel<<<1, 32, 0, st>>>(gamma, q, K, w);
  return cudaGetLastError();
}

__global__ void generator_kernel(const double* __restrict__ w, int n, double scale, double* t) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x - 1; d <= n - 1; d += gridDim.x * blockDim.x)
    t[d + 1] = -scale * w[d + 1];  // A = -[w_{i-j+1}] (Eq. AN): t_d = -w_{d+1}
}

cudaError_t launch_generator_from_weights(const double* w, int n, double scale, double* t,
                                          cudaStream_t st) {
  generator_kernel<<<(n + 256) / 256 + 1, 256, 0, st>>>(w, n, scale, t);
  return cudaGetLastError();
}

// P^T T(t) P = T(t^c) for bilinear P on odd grids n = 2 nc + 1:
// t^c_d = sum_{m=-2..2} q_m t_{2d+m}, q = (1/4, 1, 3/2, 1, 1/4), d = -1..nc-1
__global__ void coarsen_kernel(const double* __restrict__ t, int n, double* tc, int nc) {
  const double q[5] = {0.25, 1.0, 1.5, 1.0, 0.25};
  for (int d = blockIdx.x * blockDim.x + threadIdx.x - 1; d <= nc - 1;
       d += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int m = -2; m <= 2; ++m) {
      const int e = 2 * d + m;
      if (e >= -1 && e <= n - 1) s += q[m + 2] * t[e + 1];
    }
    tc[d + 1] = s;
  }
}

cudaError_t launch_coarsen_generator(const double* t, int n, double* tc, int nc,
                                     cudaStream_t st) {
  coarsen_kernel<<<(nc + 256) / 256 + 1, 256, 0, st>>>(t, n, tc, nc);
  return cudaGetLastError();
}

template <typename T>
__global__ void inject_kernel(const T* __restrict__ F, int n1, int n2, T* FC) {
  const int m1 = coarse_n(n1), m2 = coarse_n(n2);
  const size_t NC = (size_t)m1 * m2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < NC;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int ic = (int)(idx % m1), jc = (int)(idx / m1);
    FC[idx] = F[(size_t)coarse_at(n2, jc) * n1 + coarse_at(n1, ic)];
  }
}

template <typename T>
cudaError_t launch_inject(const T* F, int n1, int n2, T* FC, cudaStream_t st) {
  const size_t NC = (size_t)coarse_n(n1) * coarse_n(n2);
  inject_kernel<T><<<grid_for(NC, 256), 256, 0, st>>>(F, n1, n2, FC);
  return cudaGetLastError();
}

// Level fields by injection from the finest grid: level node (j, i) is fine
// node (s j + offy, s i + offx), s = 2^l (for odd sizes all the way down,
// off = s - 1: node ((j+1) s - 1, (i+1) s - 1)).  diag(K_l) = c by0 bx0
// + (d+ + d-) by0 ax0 + sigma (e+ + e-) ay0 bx0 (ax0, ay0: Toeplitz diagonals,
// bx0, by0: Galerkin mass diagonals); W = omega / diag.
template <typename T>
__global__ void level_fields_kernel(const double* __restrict__ dp, const double* __restrict__ dm,
                                    const double* __restrict__ ep, const double* __restrict__ em,
                                    int n1f, int n1, int n2, int s, int offx, int offy,
                                    double sigma, double c,
                                    double bx0, double by0, const double* __restrict__ tx,
                                    const double* __restrict__ ty, double omega, T* odp, T* odm,
                                    T* oep, T* oem, T* W) {
  const size_t N = (size_t)n1 * n2;
  const double ax0 = tx[1], ay0 = ty[1];  // Toeplitz diagonals t_0
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n1), j = (int)(idx / n1);
    const size_t f = (size_t)(s * j + offy) * n1f + (size_t)(s * i + offx);
    const double a = dp[f], b = dm[f], e = sigma * ep[f], g = sigma * em[f];
    odp[idx] = T(a);
    odm[idx] = T(b);
    oep[idx] = T(e);
    oem[idx] = T(g);
    const double diag = c * by0 * bx0 + (a + b) * by0 * ax0 + (e + g) * ay0 * bx0;
    if (W) W[idx] = T(omega / diag);
  }
}

template <typename T>
cudaError_t launch_level_fields(const double* dp, const double* dm, const double* ep,
                                const double* em, int n1f, int n1, int n2, int stride, int offx,
                                int offy, double sigma, double c, double bx0, double by0,
                                const double* tx, const double* ty, double omega, T* odp, T* odm,
                                T* oep, T* oem, T* W, cudaStream_t st) {
  const size_t N = (size_t)n1 * n2;
  level_fields_kernel<T><<<grid_for(N, 256), 256, 0, st>>>(dp, dm, ep, em, n1f, n1, n2, stride,
                                                           offx, offy, sigma, c, bx0, by0, tx, ty,
                                                           omega, odp, odm, oep, oem, W);
  return cudaGetLastError();
}

// Gauss-Jordan elimination with partial pivoting in FP64 on the augmented
// N x 2N matrix [K | I] held in A (one block of 256 threads; N <= 1024): the
// right half becomes K^{-1}, copied to inv. info = 1 if a pivot is zero.
__device__ void gauss_jordan_block(double* A, int N, double* inv, int* info) {
  const int W2 = 2 * N;
  __shared__ double red_v[256];
  __shared__ int red_i[256];
  __shared__ int piv_s;
  int ok = 1;
  for (int k = 0; k < N; ++k) {
    double best = -1.0;
    int bi = k;
    for (int r = k + threadIdx.x; r < N; r += blockDim.x) {
      const double a = fabs(A[(size_t)r * W2 + k]);
      if (a > best) { best = a; bi = r; }
    }
    red_v[threadIdx.x] = best;
    red_i[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s && red_v[threadIdx.x + s] > red_v[threadIdx.x]) {
        red_v[threadIdx.x] = red_v[threadIdx.x + s];
        red_i[threadIdx.x] = red_i[threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) piv_s = red_i[0];
    if (red_v[0] == 0.0) ok = 0;
    __syncthreads();
    const int p = piv_s;
    if (p != k)
      for (int col = threadIdx.x; col < W2; col += blockDim.x) {
        const double t = A[(size_t)k * W2 + col];
        A[(size_t)k * W2 + col] = A[(size_t)p * W2 + col];
        A[(size_t)p * W2 + col] = t;
      }
    __syncthreads();
    const double inv_p = 1.0 / A[(size_t)k * W2 + k];
    __syncthreads();
    for (int col = threadIdx.x; col < W2; col += blockDim.x) A[(size_t)k * W2 + col] *= inv_p;
    __syncthreads();
    for (int e = threadIdx.x; e < N * W2; e += blockDim.x) {
      const int r = e / W2, col = e % W2;
      if (r == k || col == k) continue;
      A[e] -= A[(size_t)r * W2 + k] * A[(size_t)k * W2 + col];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x)
      if (r != k) A[(size_t)r * W2 + k] = 0.0;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int r = e / N, col = e % N;
    inv[e] = A[(size_t)r * W2 + N + col];
  }
  if (threadIdx.x == 0) *info = ok ? 0 : 1;
}

// Dense coarsest operator
//   K = c (By (x) Bx) + D+ (By (x) Ax) + D- (By (x) Ax^T) + E+ (Ay (x) Bx) + E- (Ay^T (x) Bx)
// (E+- already scaled by sigma), inverted by Gauss-Jordan elimination.
__global__ void coarse_inverse_kernel(const double* __restrict__ tx, const double* __restrict__ ty,
                                      int n1, int n2, double bx0, double bx1, double by0,
                                      double by1, double c, const double* __restrict__ dp,
                                      const double* __restrict__ dm,
                                      const double* __restrict__ ep,
                                      const double* __restrict__ em, double* A, double* inv,
                                      int* info) {
  const int N = n1 * n2, W2 = 2 * N;
  auto T1 = [](const double* t, int n, int a, int b) -> double {  // Toeplitz entry (a, b)
    const int d = a - b;
    return (d >= -1 && d <= n - 1) ? t[d + 1] : 0.0;
  };
  auto B1 = [](double b0, double b1, int a, int b) -> double {
    return a == b ? b0 : ((a - b == 1 || b - a == 1) ? b1 : 0.0);
  };
  for (int e = threadIdx.x; e < N * W2; e += blockDim.x) {
    const int r = e / W2, col = e % W2;
    double v;
    if (col < N) {
      const int j = r / n1, i = r % n1, jj = col / n1, ii = col % n1;
      const double byv = B1(by0, by1, j, jj), bxv = B1(bx0, bx1, i, ii);
      v = c * byv * bxv + dp[r] * byv * T1(tx, n1, i, ii) + dm[r] * byv * T1(tx, n1, ii, i) +
          ep[r] * T1(ty, n2, j, jj) * bxv + em[r] * T1(ty, n2, jj, j) * bxv;
    } else {
      v = (col - N == r) ? 1.0 : 0.0;
    }
    A[e] = v;
  }
  __syncthreads();
  gauss_jordan_block(A, N, inv, info);
}

cudaError_t launch_coarse_inverse(const double* tx, const double* ty, int n1, int n2,
                                  double bx0, double bx1, double by0, double by1, double c,
                                  const double* dp, const double* dm, const double* ep,
                                  const double* em, double* work, double* inv, int* info,
                                  cudaStream_t st) {
  coarse_inverse_kernel<<<1, 256, 0, st>>>(tx, ty, n1, n2, bx0, bx1, by0, by1, c, dp, dm, ep, em,
                                           work, inv, info);
  return cudaGetLastError();
}

// inverse of the dense N x N operator of a nine-point stencil level (stored by
// rows, see kernels_stencil.cu): assemble [K | I], then Gauss-Jordan
__global__ void stencil_inverse_kernel(const double* __restrict__ S, int n1, int n2, double* A,
                                       double* inv, int* info) {
  const int N = n1 * n2, W2 = 2 * N;
  for (int e = threadIdx.x; e < N * W2; e += blockDim.x) {
    const int r = e / W2, col = e % W2;
    double v;
    if (col < N) {
      const int dj = col / n1 - r / n1, di = col % n1 - r % n1;
      v = (dj >= -1 && dj <= 1 && di >= -1 && di <= 1)
              ? S[(size_t)((dj + 1) * 3 + di + 1) * N + r]
              : 0.0;
    } else {
      v = (col - N == r) ? 1.0 : 0.0;
    }
    A[e] = v;
  }
  __syncthreads();
  gauss_jordan_block(A, N, inv, info);
}

cudaError_t launch_stencil_inverse(const double* S, int n1, int n2, double* work, double* inv,
                                   int* info, cudaStream_t st) {
  stencil_inverse_kernel<<<1, 256, 0, st>>>(S, n1, n2, work, inv, info);
  return cudaGetLastError();
}

// explicit inverse of a dense N x N matrix (row-major, N <= 1024)
__global__ void dense_inverse_kernel(const double* __restrict__ K, int N, double* A, double* inv,
                                     int* info) {
  const int W2 = 2 * N;
  for (int e = threadIdx.x; e < N * W2; e += blockDim.x) {
    const int r = e / W2, col = e % W2;
    A[e] = col < N ? K[(size_t)r * N + col] : (col - N == r ? 1.0 : 0.0);
  }
  __syncthreads();
  gauss_jordan_block(A, N, inv, info);
}

cudaError_t launch_dense_inverse(const double* K, int N, double* work, double* inv, int* info,
                                 cudaStream_t st) {
  if (N > 1024) return cudaErrorInvalidValue;
  dense_inverse_kernel<<<1, 256, 0, st>>>(K, N, work, inv, info);
  return cudaGetLastError();
}

template <typename T>
__global__ void coarse_solve_kernel(const double* __restrict__ inv, int N, const T* __restrict__ b,
                                    T* x) {
  extern __shared__ double bs[];
  for (int k = threadIdx.x; k < N; k += blockDim.x) bs[k] = (double)b[k];
  __syncthreads();
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    double s = 0.0;
    const double* row = inv + (size_t)r * N;
    for (int k = 0; k < N; ++k) s += row[k] * bs[k];
    x[r] = T(s);
  }
}

template <typename T>
cudaError_t launch_coarse_solve(const double* inv, int N, const T* b, T* x, cudaStream_t st) {
  coarse_solve_kernel<T><<<1, 256, N * sizeof(double), st>>>(inv, N, b, x);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- instantiations
// ============================================================================
// grouped stages (many problems per launch; see GItem / GGate)

template <typename T>
__global__ void g_transpose_kernel(const GTranspose<T>* __restrict__ ent,
                                   const GItem* __restrict__ items, int nitems, GGate gate) {
  __shared__ T tile[32][33];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GTranspose<T> e = ent[g.e];
    if (!gate_open(gate, e.prob, e.want)) continue;
    const int tc = (e.cols + 31) / 32;
    const int c0 = (g.unit % tc) * 32, r0 = (g.unit / tc) * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
      const int r = r0 + k, c = c0 + threadIdx.x;
      if (r < e.rows && c < e.cols) tile[k][threadIdx.x] = e.in[(size_t)r * e.cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
      const int c = c0 + k, r = r0 + threadIdx.x;
      if (r < e.rows && c < e.cols) {
        const size_t o = (size_t)c * e.rows + r;
        e.out[o] = e.add ? e.out[o] + tile[threadIdx.x][k] : tile[threadIdx.x][k];
      }
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_g_transpose(const GTranspose<T>* ent, const GItem* items, int nitems,
                               GGate gate, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const int grid = nitems < 152 * 16 ? nitems : 152 * 16;
  g_transpose_kernel<T><<<grid, dim3(32, 8), 0, st>>>(ent, items, nitems, gate);
  return cudaGetLastError();
}

// one chunk (kGChunk points of the fine grid, or of the coarse grid for the
// restriction) of a level stage, the same arithmetic as the single-problem
// kernels above
template <typename T>
__global__ void g_level_op_kernel(int op, const GLevelOp<T>* __restrict__ ent,
                                  const GItem* __restrict__ items, int nitems, GGate gate) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GLevelOp<T>& e = ent[g.e];
    if (!gate_open(gate, e.prob, -1)) continue;
    if (op == G_MASS && !e.xby) continue;  // no mass terms on this problem's level
    const int n1 = e.n1, n2 = e.n2;
    const size_t N = op == G_RESTRICT ? (size_t)coarse_n(n1) * coarse_n(n2) : (size_t)n1 * n2;
    const size_t lo = (size_t)g.unit * kGChunk;
    const size_t hi = lo + kGChunk < N ? lo + kGChunk : N;
    for (size_t idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) {
      if (op == G_MUL) {
        e.x[idx] = e.W[idx] * e.b[idx];
      } else if (op == G_RESID) {
        e.kx[idx] = e.b[idx] - e.kx[idx];
      } else if (op == G_SMOOTH) {
        e.x[idx] = e.x[idx] + e.W[idx] * (e.b[idx] - e.kx[idx]);
      } else if (op == G_MASS) {
        const int i = (int)(idx % n1), j = (int)(idx / n1);
        const T* X = e.x;
        auto at = [&](int jj, int ii) -> T {
          return (ii >= 0 && ii < n1 && jj >= 0 && jj < n2) ? X[(size_t)jj * n1 + ii] : T(0);
        };
        const T xc = X[idx];
        const T up = at(j - 1, i), dn = at(j + 1, i), lf = at(j, i - 1), rt = at(j, i + 1);
        e.xby[idx] = e.by1 * up + e.by0 * xc + e.by1 * dn;
        e.xbx[idx] = e.bx1 * lf + e.bx0 * xc + e.bx1 * rt;
        const T rowm = e.bx1 * at(j - 1, i - 1) + e.bx0 * up + e.bx1 * at(j - 1, i + 1);
        const T row0 = e.bx1 * lf + e.bx0 * xc + e.bx1 * rt;
        const T rowp = e.bx1 * at(j + 1, i - 1) + e.bx0 * dn + e.bx1 * at(j + 1, i + 1);
        e.mass[idx] = e.c * (e.by1 * rowm + e.by0 * row0 + e.by1 * rowp);
      } else if (op == G_RESTRICT) {
        const int m1 = coarse_n(n1);
        const int ic = (int)(idx % m1), jc = (int)(idx / m1);
        const int i = coarse_at(n1, ic), j = coarse_at(n2, jc);
        const T h = T(0.5);
        T acc = T(0);
        for (int dj = -1; dj <= 1; ++dj) {
          const int jj = j + dj;
          if (jj < 0 || jj >= n2) continue;
          const T* r = e.kx + (size_t)jj * n1;
          T sr = r[i];
          if (i > 0) sr += h * r[i - 1];
          if (i + 1 < n1) sr += h * r[i + 1];
          acc += (dj ? h : T(1)) * sr;
        }
        e.bc[idx] = e.rscale * acc;
      } else {  // G_PROLONG
        const int m1 = coarse_n(n1);
        const int i = (int)(idx % n1), j = (int)(idx / n1);
        int ci[2], cj[2];
        T wi[2], wj[2];
        const int ni = coarse_parents<T>(n1, i, ci, wi);
        const int nj = coarse_parents<T>(n2, j, cj, wj);
        T sum = T(0);
        for (int bb = 0; bb < nj; ++bb)
          for (int a = 0; a < ni; ++a) sum += wj[bb] * wi[a] * e.xc[(size_t)cj[bb] * m1 + ci[a]];
        e.x[idx] += sum;
      }
    }
  }
}

template <typename T>
cudaError_t launch_g_level_op(int op, const GLevelOp<T>* ent, const GItem* items, int nitems,
                              GGate gate, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (op < G_MUL || op > G_PROLONG) return cudaErrorInvalidValue;
  const int grid = nitems < 152 * 16 ? nitems : 152 * 16;
  g_level_op_kernel<T><<<grid, 256, 0, st>>>(op, ent, items, nitems, gate);
  return cudaGetLastError();
}

template cudaError_t launch_g_transpose<float>(const GTranspose<float>*, const GItem*, int, GGate,
                                               cudaStream_t);
template cudaError_t launch_g_transpose<double>(const GTranspose<double>*, const GItem*, int,
                                                GGate, cudaStream_t);
template cudaError_t launch_g_level_op<float>(int, const GLevelOp<float>*, const GItem*, int,
                                              GGate, cudaStream_t);

#define INST_T(T)                                                                               \
  template cudaError_t launch_mass_prepass<T>(const T*, int, int, double, double, double, double, \
                                              double, T*, T*, T*, cudaStream_t);                  \
  template cudaError_t launch_level_epilogue<T>(int, size_t, const T*, const T*, const T*,        \
                                                const T*, T*, cudaStream_t);                      \
  template cudaError_t launch_mul<T>(size_t, const T*, const T*, T*, cudaStream_t);               \
  template cudaError_t launch_restrict<T>(const T*, int, int, double, T*, cudaStream_t);          \
  template cudaError_t launch_mass_prepass_t<T>(const T*, const T*, int, int, double, double,     \
                                                double, double, double, T*, T*, T*, T*,           \
                                                cudaStream_t);                                    \
  template cudaError_t launch_transpose_smooth<T>(const T*, int, int, const T*, const T*,         \
                                                  const T*, T*, cudaStream_t);                    \
  template cudaError_t launch_restrict_residual<T>(const T*, const T*, int, int, double, T*,      \
                                                   cudaStream_t);                                 \
  template cudaError_t launch_jacobi_mass_prepass<T>(const T*, const T*, int, int, double, double,\
                                                     double, double, double, T*, T*, T*, T*,      \
                                                     cudaStream_t);                               \
  template cudaError_t launch_prolong_add<T>(const T*, int, int, T*, cudaStream_t);               \
  template cudaError_t launch_inject<T>(const T*, int, int, T*, cudaStream_t);                    \
  template cudaError_t launch_level_fields<T>(const double*, const double*, const double*,        \
                                              const double*, int, int, int, int, int, int,        \
                                              double, double,                                     \
                                              double, double, const double*, const double*,       \
                                              double, T*, T*, T*, T*, T*, cudaStream_t);          \
  template cudaError_t launch_coarse_solve<T>(const double*, int, const T*, T*, cudaStream_t); \
  template cudaError_t launch_transpose<T>(const T*, int, int, T*, int, cudaStream_t);
INST_T(double)
INST_T(float)
template cudaError_t launch_transpose<df>(const df*, int, int, df*, int, cudaStream_t);
// ---------------------------------------------------------------- conversion self-test
// input i: 64 bits of splitmix64 (Steele, Lea and Flood 2014) of seed + i,
// shaped by i mod 4 into a raw bit pattern, a value with exponent in
// [-160, 160], a round-to-nearest tie of the FP32 significand, or a value
// with exponent in [-100, 100] for the double-float split
__global__ void conversion_selftest_kernel(unsigned long long seed, long long n,
                                           unsigned long long* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const int mode = (int)(i & 3);
    const unsigned long long sign = z & (1ull << 63);
    unsigned long long mant = z & 0xFFFFFFFFFFFFFull;
    long long ex;
    if (mode == 0) ex = (long long)((z >> 52) & 0x7FF);
    else if (mode == 3) ex = 1023 + (long long)((z >> 52) % 201) - 100;
    else ex = 1023 + (long long)((z >> 52) % 321) - 160;
    if (mode == 2) mant = (mant & ~0x1FFFFFFFull) | (1ull << 28);  // exact tie
    if (i < 16) {  // zeros, infinities, NaN, extreme subnormal / normal doubles
      const unsigned long long sp[8] = {0ull, 0x7FFull << 52, (0x7FFull << 52) | 1ull, 1ull,
                                        0xFFFFFFFFFFFFFull, 1ull << 52, 0x7FEFFFFFFFFFFFFFull,
                                        0x3810000000000000ull};
      ex = -1;
      z = sp[i & 7] | ((i & 8) ? (1ull << 63) : 0ull);
    }
    const double x = ex < 0 ? __longlong_as_double((long long)z)
                            : __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) | mant));
    unsigned long long nbad = 0;
    const float a = d2f_bits(x), b = __double2float_rn(x);
    if (!((isnan(a) && isnan(b)) || __float_as_uint(a) == __float_as_uint(b))) ++nbad;
    const float f = __uint_as_float((unsigned)(z >> 32));
    const double c = f2d_bits(f), d = (double)f;
    if (!((isnan(c) && isnan(d)) ||
          __double_as_longlong(c) == __double_as_longlong(d)))
      ++nbad;
    const double ax = fabs(x);
    if (ax <= 0x1p100) {
      const df s = df_from_bits(x);
      const double err = fabs(((double)s.hi + (double)s.lo) - x);
      if (!(err <= (ax >= 0x1p-73 ? 0x1p-47 * ax : 0x1p-97))) ++nbad;
    }
    if (nbad) atomicAdd(bad, nbad);
  }
}

int conversion_selftest(long long n, long long* mismatches) {
  unsigned long long* bad = nullptr;
  if (cudaMalloc(&bad, sizeof(unsigned long long)) != cudaSuccess) return 1;
  cudaMemset(bad, 0, sizeof(unsigned long long));
  conversion_selftest_kernel<<<152 * 8, 256>>>(0x243F6A8885A308D3ull, n, bad);
  unsigned long long h = 0;
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(bad);
  if (e1 != cudaSuccess || e2 != cudaSuccess) return 1;
  *mismatches = (long long)h;
  return 0;
}

template cudaError_t launch_convert<df, float>(size_t, const df*, double, float*, cudaStream_t);
template cudaError_t launch_convert<float, df>(size_t, const float*, double, df*, cudaStream_t);
template cudaError_t launch_convert<df, double>(size_t, const df*, double, double*, cudaStream_t);
template cudaError_t launch_convert<double, df>(size_t, const double*, double, df*, cudaStream_t);
template cudaError_t launch_convert<double, float>(size_t, const double*, double, float*,
                                                   cudaStream_t);
template cudaError_t launch_convert<float, double>(size_t, const float*, double, double*,
                                                   cudaStream_t);
template cudaError_t launch_convert<double, double>(size_t, const double*, double, double*,
                                                    cudaStream_t);

}  // namespace fde

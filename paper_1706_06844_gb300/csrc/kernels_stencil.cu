// Nine-point stencil levels: the band preconditioner P_2 of Sec. 4.3 and its
// Galerkin multigrid hierarchy.
//
// P_2 = c I + D+ (I (x) A2) + D- (I (x) A2^T) + sigma [E+ (A2 (x) I) + E- (A2^T (x) I)]
// with A2 = tridiag(-1, 2, -1) (the gamma = 2 member of Eq. AN) is a five-point
// variable stencil; every Galerkin product P^T K P with the bilinear P of
// Sec. 4.1 is a nine-point stencil. A level stores its operator "by rows" in
// structure-of-arrays form: coefficient o = 3 (dy + 1) + (dx + 1) of grid row
// (j, i) multiplies x[j + dy][i + dx], at S[o * N + j * n1 + i]. Coefficients
// that would reach outside the grid are stored as zero.
#include <cuda_runtime.h>

#include "common.cuh"

namespace fde {

namespace {
inline int blocks_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}
}  // namespace

// level 0: row (j, i) of P_2 (Sec. 4.3). A2 is symmetric, so D+ A2 + D- A2^T
// acts with the summed coefficient (d+ + d-) on the three-point Laplacian.
__global__ void p2_fields_kernel(const double* __restrict__ dp, const double* __restrict__ dm,
                                 const double* __restrict__ ep, const double* __restrict__ em,
                                 int n1, int n2, double c, double sigma, double* S) {
  const size_t N = (size_t)n1 * n2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / n1), i = (int)(idx % n1);
    const double a = dp[idx] + dm[idx];
    const double b = sigma * (ep[idx] + em[idx]);
    S[0 * N + idx] = 0.0;
    S[1 * N + idx] = j > 0 ? -b : 0.0;
    S[2 * N + idx] = 0.0;
    S[3 * N + idx] = i > 0 ? -a : 0.0;
    S[4 * N + idx] = c + 2.0 * a + 2.0 * b;
    S[5 * N + idx] = i < n1 - 1 ? -a : 0.0;
    S[6 * N + idx] = 0.0;
    S[7 * N + idx] = j < n2 - 1 ? -b : 0.0;
    S[8 * N + idx] = 0.0;
  }
}

cudaError_t launch_p2_fields(const double* dp, const double* dm, const double* ep,
                             const double* em, int n1, int n2, double c, double sigma, double* S,
                             cudaStream_t st) {
  p2_fields_kernel<<<blocks_for((size_t)n1 * n2, 256), 256, 0, st>>>(dp, dm, ep, em, n1, n2, c,
                                                                       sigma, S);
  return cudaGetLastError();
}

// Galerkin coarse operator K_c = P^T K P (TGM step 3, Sec. 4) for the bilinear
// P = P_y (x) P_x: coarse node J of an axis sits on fine node 2J + 1 and
// interpolates to fine 2J, 2J + 1, 2J + 2 with weights 1/2, 1, 1/2.
//   K_c(I, J) = sum_a sum_b P(a, I) K(a, b) P(b, J)
// One thread owns coarse row I: it visits the 3 x 3 fine rows a around I and
// their nine stencil entries b, and scatters P(a, I) K(a, b) onto the (one,
// two or four) coarse parents J of b, which all lie within one coarse step of I.
__global__ void galerkin9_kernel(const double* __restrict__ Sf, int n1, int n2,
                                 double* __restrict__ Sc, int m1, int m2) {
  const size_t Nf = (size_t)n1 * n2, Nc = (size_t)m1 * m2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < Nc;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int J = (int)(idx / m1), I = (int)(idx % m1);
    double acc[9];
#pragma unroll
    for (int o = 0; o < 9; ++o) acc[o] = 0.0;
#pragma unroll
    for (int ay = -1; ay <= 1; ++ay) {
#pragma unroll
      for (int ax = -1; ax <= 1; ++ax) {
        // the fine points of P's column (J, I); for even sizes the first
        // column is truncated at the low end
        const int fy = coarse_at(n2, J) + ay, fx = coarse_at(n1, I) + ax;
        if (fy < 0 || fy >= n2 || fx < 0 || fx >= n1) continue;
        const double pa = (ay ? 0.5 : 1.0) * (ax ? 0.5 : 1.0);
        const size_t frow = (size_t)fy * n1 + fx;
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy) {
#pragma unroll
          for (int ox = -1; ox <= 1; ++ox) {
            const int by = fy + oy, bx = fx + ox;
            if (by < 0 || by >= n2 || bx < 0 || bx >= n1) continue;
            const double v = pa * Sf[(size_t)((oy + 1) * 3 + ox + 1) * Nf + frow];
            // coarse parents of fine node b along each axis
            int qy[2], qx[2];
            double wy[2], wx[2];
            const int ny = coarse_parents<double>(n2, by, qy, wy);
            const int nx = coarse_parents<double>(n1, bx, qx, wx);
            for (int u = 0; u < ny; ++u)
              for (int t = 0; t < nx; ++t)
                acc[(qy[u] - J + 1) * 3 + (qx[t] - I + 1)] += v * wy[u] * wx[t];
          }
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 9; ++o) Sc[(size_t)o * Nc + idx] = acc[o];
  }
}

cudaError_t launch_galerkin9(const double* Sf, int n1, int n2, double* Sc, int m1, int m2,
                             cudaStream_t st) {
  galerkin9_kernel<<<blocks_for((size_t)m1 * m2, 128), 128, 0, st>>>(Sf, n1, n2, Sc, m1, m2);
  return cudaGetLastError();
}

// stencil arrays in the cycle's precision and the damped-Jacobi weights
// W = omega / diag(K) (Eq. Sn with the true diagonal)
template <typename T>
__global__ void stencil_convert_kernel(const double* __restrict__ S, size_t N, double omega,
                                       T* __restrict__ ST, T* __restrict__ W) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (ST) {
#pragma unroll
      for (int o = 0; o < 9; ++o) ST[(size_t)o * N + idx] = (T)S[(size_t)o * N + idx];
    }
    W[idx] = (T)(omega / S[4 * N + idx]);
  }
}

template <typename T>
cudaError_t launch_stencil_convert(const double* S, size_t N, double omega, T* ST, T* W,
                                   cudaStream_t st) {
  stencil_convert_kernel<T><<<blocks_for(N, 256), 256, 0, st>>>(S, N, omega, ST, W);
  return cudaGetLastError();
}

// y = K x (mode 0), y = b - K x (mode 1), y = x + W (b - K x) (mode 2, one
// damped-Jacobi sweep). FIVE skips the four corner coefficients (level 0 of
// P_2, where they are zero). y must not alias x.
template <typename T, bool FIVE>
__global__ void __launch_bounds__(256) stencil_apply_kernel(int mode, const T* __restrict__ S,
                                                            int n1, int n2,
                                                            const T* __restrict__ X,
                                                            const T* __restrict__ B,
                                                            const T* __restrict__ W,
                                                            T* __restrict__ Y) {
  const size_t N = (size_t)n1 * n2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n1) return;
  // a thread walks down a column of rows, keeping three rows of x in registers
  const int rows = (n2 + gridDim.y - 1) / gridDim.y;
  const int j0 = blockIdx.y * rows, j1 = min(n2, j0 + rows);
  if (j0 >= j1) return;
  const bool hl = i > 0, hr = i < n1 - 1;
  auto ld = [&](int j, T* v) {
    if (j < 0 || j >= n2) {
      v[0] = v[1] = v[2] = T(0);
      return;
    }
    const T* r = X + (size_t)j * n1 + i;
    v[0] = hl ? r[-1] : T(0);
    v[1] = r[0];
    v[2] = hr ? r[1] : T(0);
  };
  T up[3], mid[3], dn[3];
  ld(j0 - 1, up);
  ld(j0, mid);
  for (int j = j0; j < j1; ++j) {
    ld(j + 1, dn);
    const size_t idx = (size_t)j * n1 + i;
    T acc = S[4 * N + idx] * mid[1];
    acc += S[3 * N + idx] * mid[0];
    acc += S[5 * N + idx] * mid[2];
    acc += S[1 * N + idx] * up[1];
    acc += S[7 * N + idx] * dn[1];
    if (!FIVE) {
      acc += S[0 * N + idx] * up[0];
      acc += S[2 * N + idx] * up[2];
      acc += S[6 * N + idx] * dn[0];
      acc += S[8 * N + idx] * dn[2];
    }
    T out;
    if (mode == 0) out = acc;
    else if (mode == 1) out = B[idx] - acc;
    else out = mid[1] + W[idx] * (B[idx] - acc);
    Y[idx] = out;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      up[k] = mid[k];
      mid[k] = dn[k];
    }
  }
}

template <typename T>
cudaError_t launch_stencil_apply(int mode, bool five, const T* S, int n1, int n2, const T* X,
                                 const T* B, const T* W, T* Y, cudaStream_t st) {
  // 128-wide column strips; enough row chunks for about 8 CTAs per SM
  const int bx = (n1 + 127) / 128;
  int by = (152 * 8 + bx - 1) / bx;
  const int min_rows = 16;
  if (by > (n2 + min_rows - 1) / min_rows) by = (n2 + min_rows - 1) / min_rows;
  if (by < 1) by = 1;
  dim3 grid(bx, by);
  if (five)
    stencil_apply_kernel<T, true><<<grid, 128, 0, st>>>(mode, S, n1, n2, X, B, W, Y);
  else
    stencil_apply_kernel<T, false><<<grid, 128, 0, st>>>(mode, S, n1, n2, X, B, W, Y);
  return cudaGetLastError();
}

template <typename T>
__global__ void add_kernel(size_t N, const T* A, const T* B, T* Y) {  // Y may alias A or B
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    Y[i] = A[i] + B[i];
}

template <typename T>
cudaError_t launch_add(size_t N, const T* A, const T* B, T* Y, cudaStream_t st) {
  add_kernel<T><<<blocks_for(N, 256), 256, 0, st>>>(N, A, B, Y);
  return cudaGetLastError();
}

#define FDE_STENCIL_INST(T)                                                                   \
  template cudaError_t launch_stencil_convert<T>(const double*, size_t, double, T*, T*,      \
                                                 cudaStream_t);                              \
  template cudaError_t launch_stencil_apply<T>(int, bool, const T*, int, int, const T*,      \
                                               const T*, const T*, T*, cudaStream_t);        \
  template cudaError_t launch_add<T>(size_t, const T*, const T*, T*, cudaStream_t);
FDE_STENCIL_INST(float)
FDE_STENCIL_INST(double)
#undef FDE_STENCIL_INST

// ============================================================================
// Dense levels: the exact Galerkin hierarchy A_{l+1} = P^T A_l P of Sec. 4
// (TGM step 3 at every level; the paper's tilde-P_MGM of Sec. 5.1) with
// explicit N_l x N_l matrices, for small grids.  Row-major, FP64.

// level 0: M of Eq. (M) assembled entry by entry; generators t_d at t[d + 1]
// (d = -1 .. n - 1), A_gamma[i][k] = t_{i - k}
__global__ void dense_assemble_kernel(const double* __restrict__ tx, const double* __restrict__ ty,
                                      int n1, int n2, double c, double sigma,
                                      const double* __restrict__ dp, const double* __restrict__ dm,
                                      const double* __restrict__ ep, const double* __restrict__ em,
                                      double* __restrict__ A) {
  const size_t N = (size_t)n1 * n2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N * N;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / N, col = e % N;
    const int i = (int)(r % n1), j = (int)(r / n1);
    const int k = (int)(col % n1), l = (int)(col / n1);
    double v = 0.0;
    if (l == j) {  // x direction within grid row j
      const int d = i - k;
      if (d >= -1 && d <= n1 - 1) v += dp[r] * tx[d + 1];   // D+ (I (x) A_alpha)
      if (-d >= -1 && -d <= n1 - 1) v += dm[r] * tx[-d + 1];  // D- (I (x) A_alpha^T)
      if (k == i) v += c;
    }
    if (k == i) {  // y direction within grid column i
      const int d = j - l;
      if (d >= -1 && d <= n2 - 1) v += sigma * ep[r] * ty[d + 1];
      if (-d >= -1 && -d <= n2 - 1) v += sigma * em[r] * ty[-d + 1];
    }
    A[e] = v;
  }
}

cudaError_t launch_dense_assemble(const double* tx, const double* ty, int n1, int n2, double c,
                                  double sigma, const double* dp, const double* dm,
                                  const double* ep, const double* em, double* A, cudaStream_t st) {
  const size_t N = (size_t)n1 * n2;
  dense_assemble_kernel<<<blocks_for(N * N, 256), 256, 0, st>>>(tx, ty, n1, n2, c, sigma, dp, dm,
                                                               ep, em, A);
  return cudaGetLastError();
}

// AP = A P (N_f x N_c) and A_c = P^T AP (N_c x N_c), P the bilinear transfer
// of the fine n1 x n2 grid; each column of P has at most nine entries
__global__ void dense_times_p_kernel(const double* __restrict__ A, int n1, int n2,
                                     double* __restrict__ AP) {
  const int m1 = coarse_n(n1), m2 = coarse_n(n2);
  const size_t Nf = (size_t)n1 * n2, Nc = (size_t)m1 * m2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < Nf * Nc;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / Nc, cc = e % Nc;
    const int cx = (int)(cc % m1), cy = (int)(cc / m1);
    double s = 0.0;
    for (int dy = -1; dy <= 1; ++dy) {
      const int fy = coarse_at(n2, cy) + dy;
      if (fy < 0 || fy >= n2) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int fx = coarse_at(n1, cx) + dx;
        if (fx < 0 || fx >= n1) continue;
        s += (dy ? 0.5 : 1.0) * (dx ? 0.5 : 1.0) * A[r * Nf + (size_t)fy * n1 + fx];
      }
    }
    AP[e] = s;
  }
}

__global__ void dense_pt_times_kernel(const double* __restrict__ AP, int n1, int n2,
                                      double* __restrict__ Ac) {
  const int m1 = coarse_n(n1), m2 = coarse_n(n2);
  const size_t Nc = (size_t)m1 * m2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < Nc * Nc;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t rc = e / Nc, cc = e % Nc;
    const int cx = (int)(rc % m1), cy = (int)(rc / m1);
    double s = 0.0;
    for (int dy = -1; dy <= 1; ++dy) {
      const int fy = coarse_at(n2, cy) + dy;
      if (fy < 0 || fy >= n2) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int fx = coarse_at(n1, cx) + dx;
        if (fx < 0 || fx >= n1) continue;
        s += (dy ? 0.5 : 1.0) * (dx ? 0.5 : 1.0) * AP[((size_t)fy * n1 + fx) * Nc + cc];
      }
    }
    Ac[e] = s;
  }
}

cudaError_t launch_dense_galerkin(const double* A, int n1, int n2, double* AP, double* Ac,
                                  cudaStream_t st) {
  const size_t Nf = (size_t)n1 * n2, Nc = (size_t)coarse_n(n1) * coarse_n(n2);
  dense_times_p_kernel<<<blocks_for(Nf * Nc, 256), 256, 0, st>>>(A, n1, n2, AP);
  dense_pt_times_kernel<<<blocks_for(Nc * Nc, 256), 256, 0, st>>>(AP, n1, n2, Ac);
  return cudaGetLastError();
}

// W = omega / diag(A)
__global__ void dense_jacobi_weights_kernel(const double* __restrict__ A, size_t N, double omega,
                                            double* W) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    W[i] = omega / A[i * N + i];
}

cudaError_t launch_dense_jacobi_weights(const double* A, size_t N, double omega, double* W,
                                        cudaStream_t st) {
  dense_jacobi_weights_kernel<<<blocks_for(N, 256), 256, 0, st>>>(A, N, omega, W);
  return cudaGetLastError();
}

// mode 0: y = A x; 1: y = b - A x; 2: y = x + W (b - A x).  One warp per row
// (coalesced along the row), fixed-order warp reduction.  y must not alias x.
__global__ void dense_apply_kernel(int mode, const double* __restrict__ A, size_t N,
                                   const double* __restrict__ X, const double* __restrict__ B,
                                   const double* __restrict__ W, double* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const size_t warps = (size_t)gridDim.x * (blockDim.x / 32);
  for (size_t r = blockIdx.x * (size_t)(blockDim.x / 32) + (threadIdx.x >> 5); r < N;
       r += warps) {
    double s = 0.0;
    for (size_t k = lane; k < N; k += 32) s += A[r * N + k] * X[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (mode == 0) Y[r] = s;
      else if (mode == 1) Y[r] = B[r] - s;
      else Y[r] = X[r] + W[r] * (B[r] - s);
    }
  }
}

cudaError_t launch_dense_apply(int mode, const double* A, size_t N, const double* X,
                               const double* B, const double* W, double* Y, cudaStream_t st) {
  dense_apply_kernel<<<blocks_for(N * 32, 256), 256, 0, st>>>(mode, A, N, X, B, W, Y);
  return cudaGetLastError();
}

}  // namespace fde

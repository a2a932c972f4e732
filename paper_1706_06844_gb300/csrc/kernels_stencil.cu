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
        const int fy = 2 * J + 1 + ay, fx = 2 * I + 1 + ax;  // always inside the fine grid
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
            int ny = 0, nx = 0;
            if (by & 1) {
              qy[0] = (by - 1) >> 1; wy[0] = 1.0; ny = 1;
            } else {
              if (by / 2 - 1 >= 0) { qy[ny] = by / 2 - 1; wy[ny] = 0.5; ++ny; }
              if (by / 2 < m2) { qy[ny] = by / 2; wy[ny] = 0.5; ++ny; }
            }
            if (bx & 1) {
              qx[0] = (bx - 1) >> 1; wx[0] = 1.0; nx = 1;
            } else {
              if (bx / 2 - 1 >= 0) { qx[nx] = bx / 2 - 1; wx[nx] = 0.5; ++nx; }
              if (bx / 2 < m1) { qx[nx] = bx / 2; wx[nx] = 0.5; ++nx; }
            }
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

}  // namespace fde

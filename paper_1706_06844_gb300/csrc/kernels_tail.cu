// The small end of a V-cycle in one launch.  On the coarse levels (n <= 31,
// at most 961 unknowns) every step of the cycle -- damped Jacobi, the
// level's Toeplitz products by direct summation, residual, restriction, the
// coarsest-grid solve, prolongation -- is a few microseconds of work, and as
// separate launches each costs more in latency than in execution.  One CTA of
// 1024 threads runs the whole sub-cycle with block barriers between the
// dependent steps, on the levels' own buffers (Sec. 4: TGM steps 1-6, step 4
// by recursion, the coarsest system by its explicit inverse).  The arithmetic
// of every step is that of the separate kernels (kernels_mg.cu,
// kernels_toeplitz.cu: direct_pass).
#include "common.cuh"

namespace fde {

namespace {

template <typename T>
__device__ void blk_mul(size_t N, const T* W, const T* B, T* Y) {
  for (size_t i = threadIdx.x; i < N; i += blockDim.x) Y[i] = W[i] * B[i];
}

// structured-Galerkin mass terms of level l > 0: XBY = (B_y (x) I) x,
// XBX = (I (x) B_x) x, MASS = c (B_y (x) B_x) x
template <typename T>
__device__ void blk_mass(const T* X, int n1, int n2, T bx0, T bx1, T by0, T by1, T c, T* XBY,
                         T* XBX, T* MASS) {
  const size_t N = (size_t)n1 * n2;
  for (size_t idx = threadIdx.x; idx < N; idx += blockDim.x) {
    const int i = (int)(idx % n1), j = (int)(idx / n1);
    auto at = [&](int jj, int ii) -> T {
      return (ii >= 0 && ii < n1 && jj >= 0 && jj < n2) ? X[(size_t)jj * n1 + ii] : T(0);
    };
    const T xc = X[idx];
    const T up = at(j - 1, i), dn = at(j + 1, i), lf = at(j, i - 1), rt = at(j, i + 1);
    XBY[idx] = by1 * up + by0 * xc + by1 * dn;
    XBX[idx] = bx1 * lf + bx0 * xc + bx1 * rt;
    const T rowm = bx1 * at(j - 1, i - 1) + bx0 * up + bx1 * at(j - 1, i + 1);
    const T row0 = bx1 * lf + bx0 * xc + bx1 * rt;
    const T rowp = bx1 * at(j + 1, i - 1) + bx0 * dn + bx1 * at(j + 1, i + 1);
    MASS[idx] = c * (by1 * rowm + by0 * row0 + by1 * rowp);
  }
}

// one direction of the level's Toeplitz products by direct summation over
// the nvec vectors x_v[k] = X[v vs + k es]: y = cp (A x) + cm (A^T x)
// (+ cmass M) (+ Y), A = [t_{i-k}], t_d at t[d + 1]
template <typename T>
__device__ void blk_direct(const T* X, int es, int vs, int nvec, int n, const T* t, const T* cp,
                           const T* cm, const T* M, T cmass, T* Y, bool accumulate, T* xs,
                           T* ts) {
  const int total = nvec * n;  // <= kTailN^2: the vectors and t are staged in shared memory
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int v = e / n, k = e % n;
    xs[e] = X[(size_t)v * vs + (size_t)k * es];
  }
  for (int k = threadIdx.x; k <= n; k += blockDim.x) ts[k] = t[k];
  __syncthreads();
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int v = e / n, i = e % n;
    const T* x = xs + v * n;
    T s1 = T(0), s2 = T(0);
    const int k1 = (i + 1 < n - 1) ? i + 1 : n - 1;
    for (int k = 0; k <= k1; ++k) s1 += ts[i - k + 1] * x[k];
    for (int k = (i > 0 ? i - 1 : 0); k < n; ++k) s2 += ts[k - i + 1] * x[k];
    const size_t ia = (size_t)v * vs + (size_t)i * es;
    T y = s1 * cp[ia] + s2 * cm[ia];
    if (M) y += cmass * M[ia];
    if (accumulate) y += Y[ia];
    Y[ia] = y;
  }
  __syncthreads();  // the staging buffers are reused by the next call
}

// kx = K_l x (products + mass term)
template <typename T>
__device__ void blk_products(const TailLevel<T>& L, const T* x, T c, T* xs, T* ts) {
  const T *xin_x = x, *xin_y = x, *M = x;
  T cm = c;
  if (L.xby) {
    blk_mass<T>(x, L.n1, L.n2, L.bx0, L.bx1, L.by0, L.by1, c, L.xby, L.xbx, L.mass);
    __syncthreads();
    xin_x = L.xby;
    xin_y = L.xbx;
    M = L.mass;
    cm = T(1);
  }
  blk_direct<T>(xin_x, 1, L.n1, L.n2, L.n1, L.tx, L.dp, L.dm, M, cm, L.kx, false, xs, ts);
  blk_direct<T>(xin_y, L.n1, 1, L.n1, L.n2, L.ty, L.ep, L.em, nullptr, T(0), L.kx, true, xs, ts);
}

// x <- x + W (b - K x)
template <typename T>
__device__ void blk_smooth(const TailLevel<T>& L, T c, T* xs, T* ts) {
  blk_products<T>(L, L.x, c, xs, ts);
  const size_t N = (size_t)L.n1 * L.n2;
  for (size_t i = threadIdx.x; i < N; i += blockDim.x)
    L.x[i] = L.x[i] + L.W[i] * (L.b[i] - L.kx[i]);
  __syncthreads();
}

template <typename T>
__device__ void blk_restrict(const T* R, int n1, int n2, T rscale, T* BC) {
  const int m1 = coarse_n(n1), m2 = coarse_n(n2);
  const size_t NC = (size_t)m1 * m2;
  for (size_t idx = threadIdx.x; idx < NC; idx += blockDim.x) {
    const int ic = (int)(idx % m1), jc = (int)(idx / m1);
    const int i = coarse_at(n1, ic), j = coarse_at(n2, jc);
    const T h = T(0.5);
    T acc = T(0);
    for (int dj = -1; dj <= 1; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= n2) continue;
      const T* r = R + (size_t)jj * n1;
      T sr = r[i];
      if (i > 0) sr += h * r[i - 1];
      if (i + 1 < n1) sr += h * r[i + 1];
      acc += (dj ? h : T(1)) * sr;
    }
    BC[idx] = rscale * acc;
  }
}

template <typename T>
__device__ void blk_prolong_add(const T* XC, int n1, int n2, T* X) {
  const int m1 = coarse_n(n1);
  const size_t N = (size_t)n1 * n2;
  for (size_t idx = threadIdx.x; idx < N; idx += blockDim.x) {
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
__device__ __forceinline__ void mg_tail_body(const TailArgs<T>& a, double* bs, T* xs, T* ts) {
  const int last = a.nlev - 1;
  const T c = T(a.c);
  // down: pre-smoothing, residual, restriction
  for (int l = 0; l < last; ++l) {
    const TailLevel<T>& L = a.lv[l];
    const size_t N = (size_t)L.n1 * L.n2;
    if (a.nu_pre >= 1) blk_mul<T>(N, L.W, L.b, L.x);
    else
      for (size_t i = threadIdx.x; i < N; i += blockDim.x) L.x[i] = T(0);
    __syncthreads();
    for (int s = 1; s < a.nu_pre; ++s) blk_smooth<T>(L, c, xs, ts);
    blk_products<T>(L, L.x, c, xs, ts);
    for (size_t i = threadIdx.x; i < N; i += blockDim.x) L.kx[i] = L.b[i] - L.kx[i];
    __syncthreads();
    blk_restrict<T>(L.kx, L.n1, L.n2, T(a.rscale), a.lv[l + 1].b);
    __syncthreads();
  }
  // coarsest: x = K^{-1} b with the explicit FP64 inverse
  {
    const TailLevel<T>& C = a.lv[last];
    const int N = C.n1 * C.n2;
    for (int k = threadIdx.x; k < N; k += blockDim.x) bs[k] = (double)C.b[k];
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      double s = 0.0;
      const double* row = a.inv + (size_t)r * N;
      for (int k = 0; k < N; ++k) s += row[k] * bs[k];
      C.x[r] = T(s);
    }
    __syncthreads();
  }
  // up: prolongation, post-smoothing
  for (int l = last - 1; l >= 0; --l) {
    const TailLevel<T>& L = a.lv[l];
    blk_prolong_add<T>(a.lv[l + 1].x, L.n1, L.n2, L.x);
    __syncthreads();
    for (int s = 0; s < a.nu_post; ++s) blk_smooth<T>(L, c, xs, ts);
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) mg_tail_kernel(const TailArgs<T> a) {
  __shared__ double bs[1024];
  __shared__ T xs[kTailN * kTailN];
  __shared__ T ts[kTailN + 2];
  mg_tail_body<T>(a, bs, xs, ts);
}

// grouped: one CTA per problem, each running its own tail from device memory
template <typename T>
__global__ void __launch_bounds__(1024) g_mg_tail_kernel(const TailArgs<T>* __restrict__ args,
                                                         const int* __restrict__ probs, int count,
                                                         GGate gate) {
  __shared__ double bs[1024];
  __shared__ T xs[kTailN * kTailN];
  __shared__ T ts[kTailN + 2];
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    if (!gate_open(gate, probs[k], -1)) continue;
    mg_tail_body<T>(args[k], bs, xs, ts);
    __syncthreads();
  }
}

}  // namespace

template <typename T>
cudaError_t launch_g_mg_tail(const TailArgs<T>* args, const int* probs, int count, GGate gate,
                             cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  g_mg_tail_kernel<T><<<count, 1024, 0, st>>>(args, probs, count, gate);
  return cudaGetLastError();
}
template cudaError_t launch_g_mg_tail<float>(const TailArgs<float>*, const int*, int, GGate,
                                             cudaStream_t);

template <typename T>
cudaError_t launch_mg_tail(const TailArgs<T>& a, cudaStream_t st) {
  if (a.nlev < 1 || a.nlev > kTailMaxLevels) return cudaErrorInvalidValue;
  mg_tail_kernel<T><<<1, 1024, 0, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_mg_tail<float>(const TailArgs<float>&, cudaStream_t);
template cudaError_t launch_mg_tail<double>(const TailArgs<double>&, cudaStream_t);

}  // namespace fde

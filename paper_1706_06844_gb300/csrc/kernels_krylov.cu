// FP64 kernels of the flexible GMRES iteration: block-partial dot products
// for classical Gram-Schmidt with re-orthogonalisation (CGS2), the combined
// basis update w -= V h, norms, and the solution update x += Z y.
// Reductions are two-pass (per-block partials, then one block sums them in a
// fixed order), so results are deterministic run to run.
#include "common.cuh"

namespace fde {

static constexpr int KT = 256;   // threads per block
static constexpr int KG = 8;     // vectors per pass in the dot kernel

int krylov_blocks() { return 152 * 4; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum `acc[0..cnt)` over the block; thread 0 ends with the totals in red[]
__device__ __forceinline__ void block_sums(double* acc, int cnt, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int g = 0; g < cnt; ++g) {
    const double v = warp_sum(acc[g]);
    if (lane == 0) red[g * (KT / 32) + wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int w = 0; w < KT / 32; ++w) s += red[threadIdx.x * (KT / 32) + w];
    red[KG * (KT / 32) + threadIdx.x] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(KT) dots_kernel(const double* __restrict__ V, size_t ldv, int k,
                                                  const double* __restrict__ w, size_t N,
                                                  double* part, int nb) {
  __shared__ double red[KG * (KT / 32) + KG];
  const size_t chunk = (N + nb - 1) / nb;
  const size_t lo = blockIdx.x * chunk, hi = lo + chunk < N ? lo + chunk : N;
  for (int g0 = 0; g0 < k; g0 += KG) {
    const int cnt = (k - g0) < KG ? (k - g0) : KG;
    double acc[KG];
#pragma unroll
    for (int g = 0; g < KG; ++g) acc[g] = 0.0;
    for (size_t e = lo + threadIdx.x; e < hi; e += KT) {
      const double we = w[e];
#pragma unroll
      for (int g = 0; g < KG; ++g)
        if (g < cnt) acc[g] += V[(size_t)(g0 + g) * ldv + e] * we;
    }
    block_sums(acc, cnt, red);
    if (threadIdx.x < cnt) part[(size_t)(g0 + threadIdx.x) * nb + blockIdx.x] = red[KG * (KT / 32) + threadIdx.x];
    __syncthreads();
  }
}

cudaError_t launch_dots(const double* V, size_t ldv, int k, const double* w, size_t N,
                        double* part, int nb, cudaStream_t st) {
  dots_kernel<<<nb, KT, 0, st>>>(V, ldv, k, w, N, part, nb);
  return cudaGetLastError();
}

// w -= sum_{i<k} h_i V_i ; with_norm: also partial sums of w_new . w_new into part[blk]
__global__ void __launch_bounds__(KT) axpy_kernel(const double* __restrict__ V, size_t ldv, int k,
                                                  const double* __restrict__ h, double* w,
                                                  size_t N, double* part, int nb, int with_norm) {
  __shared__ double hs[128];
  __shared__ double red[KG * (KT / 32) + KG];
  for (int i = threadIdx.x; i < k; i += KT) hs[i] = h[i];
  __syncthreads();
  const size_t chunk = (N + nb - 1) / nb;
  const size_t lo = blockIdx.x * chunk, hi = lo + chunk < N ? lo + chunk : N;
  double acc[1] = {0.0};
  for (size_t e = lo + threadIdx.x; e < hi; e += KT) {
    double we = w[e];
    for (int i = 0; i < k; ++i) we -= hs[i] * V[(size_t)i * ldv + e];
    w[e] = we;
    acc[0] += we * we;
  }
  if (with_norm) {
    block_sums(acc, 1, red);
    if (threadIdx.x == 0) part[blockIdx.x] = red[KG * (KT / 32)];
  }
}

// w <- w - sum_{i<k} h_i V_i, then partial dots V_i . w_new (k <= KMAX): the
// k values V_i[e] are loaded once into registers and used by both steps, so
// the subtraction of the first Gram-Schmidt pass and the projection of the
// second read V from memory once.
template <int KMAX>
__global__ void __launch_bounds__(KT) axpy_proj_kernel(const double* __restrict__ V, size_t ldv,
                                                       int k, const double* __restrict__ h,
                                                       double* w, size_t N, double* part, int nb) {
  __shared__ double hs[KMAX];
  __shared__ double red[KMAX * (KT / 32) + KMAX];
  for (int i = threadIdx.x; i < KMAX; i += KT) hs[i] = i < k ? h[i] : 0.0;
  __syncthreads();
  const size_t chunk = (N + nb - 1) / nb;
  const size_t lo = blockIdx.x * chunk, hi = lo + chunk < N ? lo + chunk : N;
  double acc[KMAX];
#pragma unroll
  for (int g = 0; g < KMAX; ++g) acc[g] = 0.0;
  for (size_t e = lo + threadIdx.x; e < hi; e += KT) {
    double v[KMAX];
#pragma unroll
    for (int g = 0; g < KMAX; ++g) v[g] = g < k ? V[(size_t)g * ldv + e] : 0.0;
    double we = w[e];
#pragma unroll
    for (int g = 0; g < KMAX; ++g) we -= hs[g] * v[g];
    w[e] = we;
#pragma unroll
    for (int g = 0; g < KMAX; ++g) acc[g] += v[g] * we;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < KMAX; ++g) {
    const double t = warp_sum(acc[g]);
    if (lane == 0) red[g * (KT / 32) + wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double t = 0.0;
    for (int q = 0; q < KT / 32; ++q) t += red[threadIdx.x * (KT / 32) + q];
    part[(size_t)threadIdx.x * nb + blockIdx.x] = t;
  }
}

cudaError_t launch_axpy_dots(const double* V, size_t ldv, int k, const double* h, double* w,
                             size_t N, double* part, int nb, int mode, cudaStream_t st) {
  if (k > 128 || (mode == 2 && k > 16)) return cudaErrorInvalidValue;
  if (mode == 2) {
    axpy_proj_kernel<16><<<nb, KT, 0, st>>>(V, ldv, k, h, w, N, part, nb);
  } else {
    axpy_kernel<<<nb, KT, 0, st>>>(V, ldv, k, h, w, N, part, nb, mode);
  }
  return cudaGetLastError();
}

// mode 0: out = sum; 1: out += sum; 2: out = sqrt(sum).  One block per sum
// (block i reduces part[i * nb .. i * nb + nb) in a fixed order), so the k
// sums run side by side and every result is the same from run to run.
__global__ void reduce_kernel(const double* __restrict__ part, int k, int nb, double* out,
                              int mode) {
  __shared__ double red[KT];
  const int i = blockIdx.x;
  if (i >= k) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += KT) s += part[(size_t)i * nb + b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = KT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double t = red[0];
    out[i] = mode == 0 ? t : (mode == 1 ? out[i] + t : sqrt(t));
  }
}

cudaError_t launch_reduce(const double* part, int k, int nb, double* out, int mode,
                          cudaStream_t st) {
  if (k < 1) return cudaSuccess;
  reduce_kernel<<<k, KT, 0, st>>>(part, k, nb, out, mode);
  return cudaGetLastError();
}

__global__ void scale_inv_kernel(size_t N, const double* __restrict__ x,
                                 const double* __restrict__ s, double* y) {
  const double inv = 1.0 / s[0];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}

cudaError_t launch_scale_inv(size_t N, const double* x, const double* s, double* y,
                             cudaStream_t st) {
  scale_inv_kernel<<<krylov_blocks(), KT, 0, st>>>(N, x, s, y);
  return cudaGetLastError();
}

__global__ void update_kernel(const double* __restrict__ Z, size_t ldz, int k,
                              const double* __restrict__ c, double* x, size_t N) {
  __shared__ double cs[128];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N;
       e += (size_t)gridDim.x * blockDim.x) {
    double s = x[e];
    for (int i = 0; i < k; ++i) s += cs[i] * Z[(size_t)i * ldz + e];
    x[e] = s;
  }
}

cudaError_t launch_update(const double* Z, size_t ldz, int k, const double* c, double* x,
                          size_t N, cudaStream_t st) {
  if (k > 128) return cudaErrorInvalidValue;
  update_kernel<<<krylov_blocks(), KT, 0, st>>>(Z, ldz, k, c, x, N);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(KT) sumsq_kernel(const double* __restrict__ x, size_t N,
                                                   double* part, int nb) {
  __shared__ double red[KG * (KT / 32) + KG];
  const size_t chunk = (N + nb - 1) / nb;
  const size_t lo = blockIdx.x * chunk, hi = lo + chunk < N ? lo + chunk : N;
  double acc[1] = {0.0};
  for (size_t e = lo + threadIdx.x; e < hi; e += KT) acc[0] += x[e] * x[e];
  block_sums(acc, 1, red);
  if (threadIdx.x == 0) part[blockIdx.x] = red[KG * (KT / 32)];
}

cudaError_t launch_sumsq(const double* x, size_t N, double* part, int nb, cudaStream_t st) {
  sumsq_kernel<<<nb, KT, 0, st>>>(x, N, part, nb);
  return cudaGetLastError();
}

}  // namespace fde

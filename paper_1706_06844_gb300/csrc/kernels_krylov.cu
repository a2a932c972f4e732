// FP64 kernels of the flexible GMRES iteration: block-partial dot products
// for classical Gram-Schmidt with re-orthogonalisation (CGS2), the combined
// basis update w -= V h, norms, and the solution update x += Z y.
// Reductions are two-pass (per-block partials, then one block sums them in a
// fixed order), so results are deterministic run to run.
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "df32.cuh"
#include "../../include/fde.h"

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

// ============================================================================
// Fused classical Gram-Schmidt with re-orthogonalisation (CGS2) for one
// Arnoldi step of FGMRES (Sec. 5), three passes over the basis:
//   project            h  = V^T w
//   subtract_project   w -= V h,  h2 = V^T w          (one read of V: the
//                      values of V a thread subtracts stay in its registers
//                      for the second projection)
//   subtract_norm      w -= V h2, ||w||, and in the last block the Hessenberg
//                      column h + h2 | ||w||, the Givens rotations and the
//                      residual estimate |g_{j+1}|
// then w is scaled by 1/||w||.  Each pass reduces its per-block partial sums
// in the block that finishes last (a ticket counter), in a fixed block order,
// so results are the same from run to run and no separate reduction launch is
// needed.  Vectors are the columns of the padded basis (ldv a multiple of 64
// doubles, zero padding) and are read as double2.

namespace {

constexpr int CT = 256;  // threads per block of the fused passes

// block-wide sum of acc[0..cnt) into red[g] (thread 0 reads it back after the barrier)
template <int KMAX>
__device__ __forceinline__ void block_reduce_vec(const double* acc, int cnt, double* sred) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < KMAX; ++g) {
    if (g < cnt) {
      const double v = warp_sum(acc[g]);
      if (lane == 0) sred[g * (CT / 32) + wid] = v;
    }
  }
  __syncthreads();
}

// write this block's partial sums, take a ticket; true in the block that
// finishes last, which then sums part[i * nb + b] over b = 0 .. nb - 1 in order
__device__ __forceinline__ bool publish_partials(const double* sred, int cnt, double* part, int nb,
                                                 unsigned* ticket) {
  __shared__ unsigned last;
  if ((int)threadIdx.x < cnt) {
    double t = 0.0;
    for (int w = 0; w < CT / 32; ++w) t += sred[threadIdx.x * (CT / 32) + w];
    part[(size_t)threadIdx.x * nb + blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == (unsigned)(nb - 1)) ? 1u : 0u;
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

// the last block: out[i] = sum_b part[i * nb + b], the whole block on each
// sum (thread t adds b = t, t + CT, ... with L2 loads that bypass L1, then a
// fixed-order warp and block reduction), so the result is the same every run
__device__ __forceinline__ void final_sums(const double* part, int cnt, int nb, double* out) {
  __shared__ double wsum[CT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < cnt; ++i) {
    const double* p = part + (size_t)i * nb;
    double s = 0.0;
#pragma unroll 4
    for (int b = threadIdx.x; b < nb; b += CT) s += __ldcg(p + b);
    s = warp_sum(s);
    if (lane == 0) wsum[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < CT / 32; ++w) t += wsum[w];
      out[i] = t;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double2 ld2(const double* p, size_t q) {
  return reinterpret_cast<const double2*>(p)[q];
}

// Re-orthogonalise only when the first projection removed most of w: with
// h = V^T w and an orthonormal V, ||w - V h||^2 = ||w||^2 - ||h||^2; when that
// keeps more than half of ||w||^2 (the classical "twice is enough" test with
// the factor 1/sqrt(2)) one projection leaves w orthogonal to working
// accuracy and the second pass is skipped.  ww = ||w||^2; the verdict goes to
// status->pad (1: project twice).
__device__ __forceinline__ int needs_second_projection(const double* h, int k, double ww) {
  double hh = 0.0;
  for (int i = 0; i < k; ++i) hh = fma(h[i], h[i], hh);
  return (ww - hh > 0.5 * ww) ? 0 : 1;
}

template <int KMAX>
__global__ void __launch_bounds__(CT) cgs_project_kernel(const double* __restrict__ V, size_t ldv,
                                                         int k, const double* __restrict__ w,
                                                         size_t n2, double* part, int nb,
                                                         unsigned* ticket, double* h,
                                                         ArnoldiStatus* status) {
  __shared__ double sred[(KMAX + 1) * (CT / 32)];
  double acc[KMAX + 1];
#pragma unroll
  for (int g = 0; g <= KMAX; ++g) acc[g] = 0.0;
  for (size_t q = blockIdx.x * (size_t)CT + threadIdx.x; q < n2; q += (size_t)nb * CT) {
    const double2 wv = ld2(w, q);
#pragma unroll
    for (int g = 0; g < KMAX; ++g)
      if (g < k) {
        const double2 v = ld2(V + (size_t)g * ldv, q);
        acc[g] = fma(v.x, wv.x, fma(v.y, wv.y, acc[g]));
      }
    acc[KMAX] = fma(wv.x, wv.x, fma(wv.y, wv.y, acc[KMAX]));
  }
  // the KMAX + 1 sums (unused projections are zero, ||w||^2 last) in h[0 .. KMAX]
  block_reduce_vec<KMAX + 1>(acc, KMAX + 1, sred);
  if (publish_partials(sred, KMAX + 1, part, nb, ticket)) {
    final_sums(part, KMAX + 1, nb, h);
    if (threadIdx.x == 0) {
      *ticket = 0u;
      status->pad = needs_second_projection(h, k, h[KMAX]);
    }
  }
}

// k in 17 .. 32: the same pass over scalar elements, so the KMAX values a
// thread keeps for the second projection fit its registers
__device__ void arnoldi_column(const ArnoldiState& st, int j, const double* h, const double* h2,
                               double nrm2);

// w -= V h, then either h2 = V^T w (second projection) or, when the first
// projection sufficed, ||w||^2 and the Givens update of column j in the last block
template <int KMAX>
__global__ void __launch_bounds__(CT) cgs_subtract_project1_kernel(
    const double* __restrict__ V, size_t ldv, int k, const double* __restrict__ h, double* w,
    size_t n, double* part, int nb, unsigned* ticket, double* h2, ArnoldiState st, int j) {
  __shared__ double sred[KMAX * (CT / 32)];
  __shared__ double hs[KMAX];
  __shared__ double nrm2;
  if ((int)threadIdx.x < KMAX) hs[threadIdx.x] = (int)threadIdx.x < k ? h[threadIdx.x] : 0.0;
  __syncthreads();
  if (!st.status->pad) {
    double a1[1] = {0.0};
    for (size_t q = blockIdx.x * (size_t)CT + threadIdx.x; q < n; q += (size_t)nb * CT) {
      double wv = w[q];
#pragma unroll
      for (int g = 0; g < KMAX; ++g)
        if (g < k) wv = fma(-hs[g], V[(size_t)g * ldv + q], wv);
      w[q] = wv;
      a1[0] = fma(wv, wv, a1[0]);
    }
    block_reduce_vec<1>(a1, 1, sred);
    if (publish_partials(sred, 1, part, nb, ticket)) {
      final_sums(part, 1, nb, &nrm2);
      __syncthreads();
      if (threadIdx.x == 0) {
        *ticket = 0u;
        arnoldi_column(st, j, h, nullptr, nrm2);
      }
    }
    return;
  }
  double acc[KMAX];
#pragma unroll
  for (int g = 0; g < KMAX; ++g) acc[g] = 0.0;
  for (size_t q = blockIdx.x * (size_t)CT + threadIdx.x; q < n; q += (size_t)nb * CT) {
    double v[KMAX];
#pragma unroll
    for (int g = 0; g < KMAX; ++g) v[g] = g < k ? V[(size_t)g * ldv + q] : 0.0;
    double wv = w[q];
#pragma unroll
    for (int g = 0; g < KMAX; ++g) wv = fma(-hs[g], v[g], wv);
    w[q] = wv;
#pragma unroll
    for (int g = 0; g < KMAX; ++g) acc[g] = fma(v[g], wv, acc[g]);
  }
  block_reduce_vec<KMAX>(acc, k, sred);
  if (publish_partials(sred, k, part, nb, ticket)) {
    final_sums(part, k, nb, h2);
    if (threadIdx.x == 0) *ticket = 0u;
  }
}

template <int KMAX>
__global__ void __launch_bounds__(CT) cgs_subtract_project_kernel(
    const double* __restrict__ V, size_t ldv, int k, const double* __restrict__ h, double* w,
    size_t n2, double* part, int nb, unsigned* ticket, double* h2, ArnoldiState st, int j) {
  __shared__ double sred[KMAX * (CT / 32)];
  __shared__ double hs[KMAX];
  __shared__ double nrm2;
  if ((int)threadIdx.x < KMAX) hs[threadIdx.x] = (int)threadIdx.x < k ? h[threadIdx.x] : 0.0;
  __syncthreads();
  double2* w2 = reinterpret_cast<double2*>(w);
  if (!st.status->pad) {
    double a1[1] = {0.0};
    for (size_t q = blockIdx.x * (size_t)CT + threadIdx.x; q < n2; q += (size_t)nb * CT) {
      double2 wv = w2[q];
#pragma unroll
      for (int g = 0; g < KMAX; ++g)
        if (g < k) {
          const double2 v = ld2(V + (size_t)g * ldv, q);
          wv.x = fma(-hs[g], v.x, wv.x);
          wv.y = fma(-hs[g], v.y, wv.y);
        }
      w2[q] = wv;
      a1[0] = fma(wv.x, wv.x, fma(wv.y, wv.y, a1[0]));
    }
    block_reduce_vec<1>(a1, 1, sred);
    if (publish_partials(sred, 1, part, nb, ticket)) {
      final_sums(part, 1, nb, &nrm2);
      __syncthreads();
      if (threadIdx.x == 0) {
        *ticket = 0u;
        arnoldi_column(st, j, h, nullptr, nrm2);
      }
    }
    return;
  }
  double acc[KMAX];
#pragma unroll
  for (int g = 0; g < KMAX; ++g) acc[g] = 0.0;
  for (size_t q = blockIdx.x * (size_t)CT + threadIdx.x; q < n2; q += (size_t)nb * CT) {
    double2 v[KMAX];
#pragma unroll
    for (int g = 0; g < KMAX; ++g)
      v[g] = g < k ? ld2(V + (size_t)g * ldv, q) : make_double2(0.0, 0.0);
    double2 wv = w2[q];
#pragma unroll
    for (int g = 0; g < KMAX; ++g) {
      wv.x = fma(-hs[g], v[g].x, wv.x);
      wv.y = fma(-hs[g], v[g].y, wv.y);
    }
    w2[q] = wv;
#pragma unroll
    for (int g = 0; g < KMAX; ++g) acc[g] = fma(v[g].x, wv.x, fma(v[g].y, wv.y, acc[g]));
  }
  block_reduce_vec<KMAX>(acc, k, sred);
  if (publish_partials(sred, k, part, nb, ticket)) {
    final_sums(part, k, nb, h2);
    if (threadIdx.x == 0) *ticket = 0u;
  }
}

// Hessenberg column of Arnoldi step j (h + h2 above the diagonal, ||w||
// below), the previous rotations applied to it, the new rotation, the rotated
// right-hand side g and the status (one thread)
__device__ void arnoldi_column(const ArnoldiState& st, int j, const double* h, const double* h2,
                               double nrm2) {
  const int m = st.m;
  double col[ArnoldiState::kMaxM + 1];
  int bad = 0;
  for (int i = 0; i <= j; ++i) {
    col[i] = h2 ? h[i] + h2[i] : h[i];
    if (!isfinite(col[i])) bad = 1;
  }
  const double hnext = sqrt(nrm2);
  col[j + 1] = hnext;
  if (!isfinite(hnext)) bad = 1;
  for (int i = 0; i < j; ++i) {
    const double t = st.cs[i] * col[i] + st.sn[i] * col[i + 1];
    col[i + 1] = -st.sn[i] * col[i] + st.cs[i] * col[i + 1];
    col[i] = t;
  }
  const double rho = hypot(col[j], col[j + 1]);
  st.cs[j] = col[j] / rho;
  st.sn[j] = col[j + 1] / rho;
  col[j] = rho;
  for (int i = 0; i <= j; ++i) st.R[(size_t)j * (m + 1) + i] = col[i];
  const double gj = st.g[j];
  st.g[j + 1] = -st.sn[j] * gj;
  st.g[j] = st.cs[j] * gj;
  st.status->gabs = fabs(st.g[j + 1]);
  st.status->hnext = hnext;
  st.status->inv_norm = 1.0 / hnext;
  st.status->nonfinite = bad;
}

template <int KMAX>
__global__ void __launch_bounds__(CT) cgs_subtract_norm_kernel(
    const double* __restrict__ V, size_t ldv, int k, const double* __restrict__ h,
    const double* __restrict__ h2, double* w, size_t n2, double* part, int nb, unsigned* ticket,
    ArnoldiState st, int j) {
  __shared__ double sred[CT / 32];
  __shared__ double hs[KMAX];
  __shared__ double nrm2;
  if (!st.status->pad) return;  // one projection sufficed: the previous pass closed the step
  if ((int)threadIdx.x < KMAX) hs[threadIdx.x] = (int)threadIdx.x < k ? h2[threadIdx.x] : 0.0;
  __syncthreads();
  double acc[1] = {0.0};
  double2* w2 = reinterpret_cast<double2*>(w);
  for (size_t q = blockIdx.x * (size_t)CT + threadIdx.x; q < n2; q += (size_t)nb * CT) {
    double2 wv = w2[q];
#pragma unroll
    for (int g = 0; g < KMAX; ++g)
      if (g < k) {
        const double2 v = ld2(V + (size_t)g * ldv, q);
        wv.x = fma(-hs[g], v.x, wv.x);
        wv.y = fma(-hs[g], v.y, wv.y);
      }
    w2[q] = wv;
    acc[0] = fma(wv.x, wv.x, fma(wv.y, wv.y, acc[0]));
  }
  block_reduce_vec<1>(acc, 1, sred);
  if (publish_partials(sred, 1, part, nb, ticket)) {
    final_sums(part, 1, nb, &nrm2);
    __syncthreads();
    if (threadIdx.x == 0) {
      *ticket = 0u;
      arnoldi_column(st, j, h, h2, nrm2);
    }
  }
}

__global__ void arnoldi_column_kernel(ArnoldiState st, int j, const double* h, const double* h2,
                                      const double* nrm2) {
  if (threadIdx.x == 0) arnoldi_column(st, j, h, h2, *nrm2);
}

__global__ void scale_by_kernel(double* w, size_t n2, const ArnoldiStatus* s) {
  const double inv = s->inv_norm;
  double2* w2 = reinterpret_cast<double2*>(w);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n2;
       q += (size_t)gridDim.x * blockDim.x) {
    double2 v = w2[q];
    v.x *= inv;
    v.y *= inv;
    w2[q] = v;
  }
}

// g = (beta, 0, ..., 0) with beta = *beta_dev
__global__ void arnoldi_start_kernel(ArnoldiState st, const double* beta_dev) {
  for (int i = threadIdx.x; i <= st.m; i += blockDim.x) st.g[i] = i == 0 ? *beta_dev : 0.0;
  if (threadIdx.x == 0) st.status->gabs = *beta_dev;
}

// y = R^{-1} g over the first k columns (back substitution, one thread)
__global__ void arnoldi_lsq_kernel(ArnoldiState st, int k, double* y) {
  if (threadIdx.x != 0) return;
  const int m = st.m;
  for (int i = k - 1; i >= 0; --i) {
    double s = st.g[i];
    for (int l = i + 1; l < k; ++l) s -= st.R[(size_t)l * (m + 1) + i] * y[l];
    y[i] = s / st.R[(size_t)i * (m + 1) + i];
  }
}

}  // namespace

// blocks of a fused pass: every block the GPU holds at once (occupancy x SMs),
// at most kMaxCgsBlocks, so the loads in flight saturate HBM whatever k is
constexpr int kMaxCgsBlocks = 2048;
int cgs_blocks() { return kMaxCgsBlocks; }

static int resident_blocks(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({kernel, dev});
  if (it != cache.end()) return it->second;
  int per_sm = 1, sms = 152;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, CT, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int nb = (per_sm < 1 ? 1 : per_sm) * sms;
  if (nb > kMaxCgsBlocks) nb = kMaxCgsBlocks;
  cache[{kernel, dev}] = nb;
  return nb;
}

cudaError_t launch_cgs2(const double* V, size_t ldv, int k, double* w, size_t N, double* part,
                        unsigned* tickets, double* h, double* h2, const ArnoldiState& st, int j,
                        cudaStream_t s) {
  if (k < 1 || k > ArnoldiState::kMaxM || (ldv & 1) || (N & 1)) return cudaErrorInvalidValue;
  const size_t n2 = N / 2;
#define CGS_LAUNCH(KM, SP, SPN)                                                                \
  {                                                                                           \
    const int b1 = resident_blocks((const void*)cgs_project_kernel<KM>);                      \
    const int b2 = resident_blocks((const void*)SP<KM>);                                      \
    const int b3 = resident_blocks((const void*)cgs_subtract_norm_kernel<KM>);                \
    cgs_project_kernel<KM><<<b1, CT, 0, s>>>(V, ldv, k, w, n2, part, b1, tickets, h,          \
                                             st.status);                                      \
    SP<KM><<<b2, CT, 0, s>>>(V, ldv, k, h, w, SPN, part, b2, tickets + 1, h2, st, j);         \
    cgs_subtract_norm_kernel<KM><<<b3, CT, 0, s>>>(V, ldv, k, h, h2, w, n2, part, b3,         \
                                                   tickets + 2, st, j);                       \
  }
  if (k <= 4) {
    CGS_LAUNCH(4, cgs_subtract_project_kernel, n2)
  } else if (k <= 8) {
    CGS_LAUNCH(8, cgs_subtract_project_kernel, n2)
  } else if (k <= 16) {
    CGS_LAUNCH(16, cgs_subtract_project_kernel, n2)
  } else if (k <= 32) {
    CGS_LAUNCH(32, cgs_subtract_project1_kernel, N)
  } else {
    return cudaErrorInvalidValue;
  }
#undef CGS_LAUNCH
  scale_by_kernel<<<152 * 4, 256, 0, s>>>(w, n2, st.status);
  return cudaGetLastError();
}

cudaError_t launch_arnoldi_column(const ArnoldiState& st, int j, const double* h,
                                  const double* h2, const double* nrm2, cudaStream_t s) {
  arnoldi_column_kernel<<<1, 32, 0, s>>>(st, j, h, h2, nrm2);
  return cudaGetLastError();
}

cudaError_t launch_scale_by(double* w, size_t N, const ArnoldiStatus* status, cudaStream_t s) {
  if (N & 1) return cudaErrorInvalidValue;
  scale_by_kernel<<<152 * 4, 256, 0, s>>>(w, N / 2, status);
  return cudaGetLastError();
}

cudaError_t launch_arnoldi_start(const ArnoldiState& st, const double* beta_dev, cudaStream_t s) {
  arnoldi_start_kernel<<<1, 64, 0, s>>>(st, beta_dev);
  return cudaGetLastError();
}

cudaError_t launch_arnoldi_lsq(const ArnoldiState& st, int k, double* y, cudaStream_t s) {
  arnoldi_lsq_kernel<<<1, 32, 0, s>>>(st, k, y);
  return cudaGetLastError();
}

// ============================================================================
// Delayed classical Gram-Schmidt with re-orthogonalisation (DCGS2; Bielich,
// Langou, Thomas, Swirydowicz, Yamazaki and Boman, Parallel Computing 2022)
// for the Arnoldi steps of FGMRES (Sec. 5).  CGS2 reads the basis three times
// per step; here the second projection of basis vector v_j is taken one step
// late, in the same read of V as the first projection of the new vector
// w = M^(m) z_j, so a step reads V_0 .. V_{j-1} twice:
//   dots    s = V_{<j}^T v_j, alpha = v_j.v_j, a = V_{<j}^T w, b = v_j.w;
//           last block: r = sqrt(alpha - s.s) (the norm of v_j - V s),
//           c = (b - s.a) / r (the projection of w on the corrected v_j),
//           Hessenberg column j - 1 corrected for v_j's re-orthogonalisation
//           (h_{i,j-1} += eta s_i, h_{j,j-1} = eta r, eta its old subdiagonal)
//           and its rotation redone from the unrotated column
//   update  v_j <- (v_j - V_{<j} s) / r, w <- w - V_{<j} a - c v_j, ||w||^2;
//           last block: column j = (a, c, ||w||) rotated, the residual
//           estimate |g_{j+1}| (final once column j is corrected next step)
// then w /= ||w||.  FGMRES keeps z_j = M^{-1} v_j from before v_j's
// correction: A Z = V H holds for the corrected H whatever the z_j are.
// v_0 = r_0 / ||r_0|| is taken as final (r = 1, no correction at j = 0).
// Cost: both schemes take four FP64 FMAs per basis element and step, and on
// this GPU (FP64 at 1/64 of the FP32 rate, ~0.5 T FP64 instructions/s) those
// FMAs, not the bytes, bound the passes; the delayed scheme saves one read of
// the basis and one serial reduction tail per step.
namespace {

__host__ __device__ __forceinline__ int dcgs_slot(int t, int j) {
  // the 2j + 2 sums a step uses, in the slot layout s | a | alpha, b
  return t < j ? t : t < 2 * j ? kDcgsMax + (t - j) : 2 * kDcgsMax + (t - 2 * j);
}

// the last block: out[slot] = sum_b part[slot * nb + b] for the step's sums;
// warp w takes sums w, w + 8, ..., lane l adds b = l, l + 32, ... in order,
// then a fixed butterfly: the same result every run
__device__ __forceinline__ void dcgs_final_sums(const double* part, int nb, int j, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int cnt = 2 * j + 2;
  for (int t = wid; t < cnt; t += CT / 32) {
    const int slot = dcgs_slot(t, j);
    const double* p = part + (size_t)slot * nb;
    double s = 0.0;
#pragma unroll 8
    for (int b = lane; b < nb; b += 32) s += __ldcg(p + b);
    s = warp_sum(s);
    if (lane == 0) out[slot] = s;
  }
  __syncthreads();
}

// rotations 0 .. j-1 applied to the unrotated column j of H, rotation j
// computed from it, R's column j stored; g_j (as it was before rotation j) is
// saved and rotated.  Returns |g_{j+1}|.
__device__ double dcgs_rotate_column(const ArnoldiState& st, int j) {
  const int m = st.m;
  double col[ArnoldiState::kMaxM + 1];
  for (int i = 0; i <= j + 1; ++i) col[i] = st.H[(size_t)j * (m + 1) + i];
  for (int i = 0; i < j; ++i) {
    const double t = st.cs[i] * col[i] + st.sn[i] * col[i + 1];
    col[i + 1] = -st.sn[i] * col[i] + st.cs[i] * col[i + 1];
    col[i] = t;
  }
  const double rho = hypot(col[j], col[j + 1]);
  st.cs[j] = col[j] / rho;
  st.sn[j] = col[j + 1] / rho;
  col[j] = rho;
  for (int i = 0; i <= j; ++i) st.R[(size_t)j * (m + 1) + i] = col[i];
  const double gj = st.gpre[j];
  st.g[j + 1] = -st.sn[j] * gj;
  st.g[j] = st.cs[j] * gj;
  return fabs(st.g[j + 1]);
}

// the dots pass's scalar work (one thread): d holds the slots of the step's sums
__device__ void dcgs_correct(const ArnoldiState& st, int j, const double* d, double* coef) {
  constexpr int kmax = kDcgsMax;
  const int m = st.m;
  int bad = 0;
  double r = 1.0, c = d[2 * kmax + 1];
  if (j > 0) {
    double ss = 0.0, sa = 0.0;
    for (int i = 0; i < j; ++i) {
      ss = fma(d[i], d[i], ss);
      sa = fma(d[i], d[kmax + i], sa);
    }
    const double rr = d[2 * kmax] - ss;
    if (!(rr > 0.0)) bad = 1;  // v_j numerically inside span(V_{<j}), or not finite
    r = sqrt(rr);
    c = (d[2 * kmax + 1] - sa) / r;
    // column j - 1: v_j^old = r v_j^new + V_{<j} s
    double* hc = st.H + (size_t)(j - 1) * (m + 1);
    const double eta = hc[j];
    for (int i = 0; i < j; ++i) hc[i] = fma(eta, d[i], hc[i]);
    hc[j] = eta * r;
    // redo rotation j - 1 from g_{j-1} as it was before it
    dcgs_rotate_column(st, j - 1);
  }
  double* hj = st.H + (size_t)j * (m + 1);
  for (int i = 0; i < j; ++i) {
    coef[i] = d[i] / r;  // v_j / r - sum_i (s_i / r) V_i
    coef[kDcgsMax + i] = d[kmax + i];
    hj[i] = d[kmax + i];
    if (!isfinite(d[i]) || !isfinite(d[kmax + i])) bad = 1;
  }
  hj[j] = c;
  if (!isfinite(c) || !isfinite(r)) bad = 1;
  coef[2 * kDcgsMax] = 1.0 / r;
  coef[2 * kDcgsMax + 1] = c;
  st.status->nonfinite = bad;
}

// Storage and arithmetic of the passes: FP64 vectors, or double-float vectors
// (hi, lo FP32 pairs, ~2^-48, 8 bytes an element like FP64) computed on the
// FP32 pipes.  Two elements per 16-byte load either way.
template <typename S>
struct Store;
template <>
struct Store<double> {
  using A = double;
  static __device__ __forceinline__ void ld(const double* p, size_t q, A& a0, A& a1) {
    const double2 v = reinterpret_cast<const double2*>(p)[q];
    a0 = v.x;
    a1 = v.y;
  }
  static __device__ __forceinline__ void st(double* p, size_t q, A a0, A a1) {
    reinterpret_cast<double2*>(p)[q] = make_double2(a0, a1);
  }
  static __device__ __forceinline__ A from(double x) { return x; }
  static __device__ __forceinline__ A zero() { return 0.0; }
  static __device__ __forceinline__ A fma(A a, A b, A c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ A mul(A a, A b) { return a * b; }
  static __device__ __forceinline__ A neg(A a) { return -a; }
  // warp sum (every lane gets it)
  static __device__ __forceinline__ double wsum(A a) { return warp_sum(a); }
};
template <>
struct Store<df> {
  using A = df;
  static __device__ __forceinline__ void ld(const double* p, size_t q, A& a0, A& a1) {
    const float4 v = reinterpret_cast<const float4*>(p)[q];
    a0 = df(v.x, v.y);
    a1 = df(v.z, v.w);
  }
  static __device__ __forceinline__ void st(double* p, size_t q, A a0, A a1) {
    reinterpret_cast<float4*>(p)[q] = make_float4(a0.hi, a0.lo, a1.hi, a1.lo);
  }
  static __device__ __forceinline__ A from(double x) { return df_from_bits(x); }
  static __device__ __forceinline__ A zero() { return df(0.f, 0.f); }
  static __device__ __forceinline__ A fma(A a, A b, A c) { return df_fma(a, b, c); }
  static __device__ __forceinline__ A mul(A a, A b) { return a * b; }
  static __device__ __forceinline__ A neg(A a) { return -a; }
  static __device__ __forceinline__ double wsum(A a) {
    for (int o = 16; o > 0; o >>= 1) {
      const df b(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
      a = a + b;
    }
    return (double)a;
  }
};

// J = j exactly (one instantiation per basis length): no predicated loads of
// unused vectors
template <int J, typename S>
__global__ void __launch_bounds__(CT) dcgs_dots_kernel(const double* __restrict__ V, size_t ldv,
                                                       size_t n2, double* part, int nb,
                                                       unsigned* ticket, double* coef,
                                                       ArnoldiState st) {
  using K = Store<S>;
  using A = typename K::A;
  constexpr int NS = 2 * kDcgsMax + 2;
  constexpr int JA = J > 0 ? J : 1;
  __shared__ double sred[(2 * J + 2) * (CT / 32)];
  __shared__ double d[NS];
  __shared__ unsigned last;
  const double* __restrict__ vj = V + (size_t)J * ldv;
  const double* __restrict__ w = V + (size_t)(J + 1) * ldv;
  A as[JA], aw[JA], al = K::zero(), bw = K::zero();
#pragma unroll
  for (int g = 0; g < JA; ++g) as[g] = aw[g] = K::zero();
  for (size_t q = blockIdx.x * (size_t)CT + threadIdx.x; q < n2; q += (size_t)nb * CT) {
    A v0, v1, w0, w1;
    K::ld(vj, q, v0, v1);
    K::ld(w, q, w0, w1);
#pragma unroll
    for (int g = 0; g < J; ++g) {
      A x0, x1;
      K::ld(V + (size_t)g * ldv, q, x0, x1);
      as[g] = K::fma(x1, v1, K::fma(x0, v0, as[g]));
      aw[g] = K::fma(x1, w1, K::fma(x0, w0, aw[g]));
    }
    al = K::fma(v1, v1, K::fma(v0, v0, al));
    bw = K::fma(v1, w1, K::fma(v0, w0, bw));
  }
  // block sums in compact order (s_0 .. s_{J-1}, a_0 .. a_{J-1}, alpha, b)
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < J; ++g) {
      const double x = K::wsum(as[g]), y = K::wsum(aw[g]);
      if (lane == 0) {
        sred[g * (CT / 32) + wid] = x;
        sred[(J + g) * (CT / 32) + wid] = y;
      }
    }
    const double x = K::wsum(al), y = K::wsum(bw);
    if (lane == 0) {
      sred[2 * J * (CT / 32) + wid] = x;
      sred[(2 * J + 1) * (CT / 32) + wid] = y;
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < 2 * J + 2) {
    const int t = threadIdx.x;
    double v = 0.0;
    for (int ww = 0; ww < CT / 32; ++ww) v += sred[t * (CT / 32) + ww];
    part[(size_t)dcgs_slot(t, J) * nb + blockIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == (unsigned)(nb - 1)) ? 1u : 0u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  dcgs_final_sums(part, nb, J, d);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    dcgs_correct(st, J, d, coef);
  }
}

// v_j <- v_j / r - sum_g (s_g / r) V_g and w <- w - sum_g a_g V_g - c v_j
// (two FMAs per basis element), j = J unrolled so that a thread's loads of
// all J basis vectors are in flight together
template <int J, typename S>
__global__ void __launch_bounds__(CT) dcgs_update_kernel(double* V, size_t ldv, size_t n2,
                                                         double* part, int nb, unsigned* ticket,
                                                         const double* __restrict__ coef,
                                                         ArnoldiState st) {
  constexpr int j = J;
  using K = Store<S>;
  using A = typename K::A;
  __shared__ A cs_[kDcgsMax], ca_[kDcgsMax];
  __shared__ double sred[CT / 32];
  __shared__ double nrm2;
  if ((int)threadIdx.x < kDcgsMax) {
    const int g = threadIdx.x;
    cs_[g] = K::neg(K::from(g < j ? coef[g] : 0.0));
    ca_[g] = K::neg(K::from(g < j ? coef[kDcgsMax + g] : 0.0));
  }
  __syncthreads();
  const A rinv = K::from(coef[2 * kDcgsMax]), mc = K::neg(K::from(coef[2 * kDcgsMax + 1]));
  double* vj = V + (size_t)j * ldv;
  double* w = V + (size_t)(j + 1) * ldv;
  A acc = K::zero();
  for (size_t q = blockIdx.x * (size_t)CT + threadIdx.x; q < n2; q += (size_t)nb * CT) {
    A v0, v1, w0, w1;
    K::ld(vj, q, v0, v1);
    K::ld(w, q, w0, w1);
    if (j > 0) {
      v0 = K::mul(v0, rinv);
      v1 = K::mul(v1, rinv);
#pragma unroll
      for (int g = 0; g < J; ++g) {
        A x0, x1;
        K::ld(V + (size_t)g * ldv, q, x0, x1);
        v0 = K::fma(cs_[g], x0, v0);
        v1 = K::fma(cs_[g], x1, v1);
        w0 = K::fma(ca_[g], x0, w0);
        w1 = K::fma(ca_[g], x1, w1);
      }
      K::st(vj, q, v0, v1);
    }
    w0 = K::fma(mc, v0, w0);
    w1 = K::fma(mc, v1, w1);
    K::st(w, q, w0, w1);
    acc = K::fma(w1, w1, K::fma(w0, w0, acc));
  }
  {
    const double x = K::wsum(acc);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = x;
    __syncthreads();
  }
  if (publish_partials(sred, 1, part, nb, ticket)) {
    final_sums(part, 1, nb, &nrm2);
    __syncthreads();
    if (threadIdx.x == 0) {
      *ticket = 0u;
      const int m = st.m;
      const double hnext = sqrt(nrm2);
      st.H[(size_t)j * (m + 1) + j + 1] = hnext;
      st.gpre[j] = st.g[j];
      st.status->gabs = dcgs_rotate_column(st, j);
      st.status->hnext = hnext;
      st.status->inv_norm = 1.0 / hnext;
      if (!isfinite(hnext)) st.status->nonfinite = 1;
    }
  }
}

// w <- w / ||w|| for double-float vectors
__global__ void scale_by_df_kernel(double* w, size_t n2, const ArnoldiStatus* s) {
  const df inv = df_from_bits(s->inv_norm);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n2;
       q += (size_t)gridDim.x * blockDim.x) {
    df a0, a1;
    Store<df>::ld(w, q, a0, a1);
    Store<df>::st(w, q, a0 * inv, a1 * inv);
  }
}

template <int J, typename S>
void launch_dcgs_pair(double* V, size_t ldv, size_t n2, double* part, unsigned* tickets,
                      double* coef, const ArnoldiState& st, cudaStream_t s) {
  const int nb = resident_blocks((const void*)dcgs_dots_kernel<J, S>);
  dcgs_dots_kernel<J, S><<<nb, CT, 0, s>>>(V, ldv, n2, part, nb, tickets, coef, st);
  const int nb2 = resident_blocks((const void*)dcgs_update_kernel<J, S>);
  dcgs_update_kernel<J, S><<<nb2, CT, 0, s>>>(V, ldv, n2, part, nb2, tickets + 1, coef, st);
}

template <typename S>
void launch_dcgs_step(double* V, size_t ldv, int j, size_t n2, double* part, unsigned* tickets,
                      double* coef, const ArnoldiState& st, cudaStream_t s) {
  using Pair = void (*)(double*, size_t, size_t, double*, unsigned*, double*,
                        const ArnoldiState&, cudaStream_t);
  static const Pair pairs[kDcgsMax] = {
      launch_dcgs_pair<0, S>,  launch_dcgs_pair<1, S>,  launch_dcgs_pair<2, S>,
      launch_dcgs_pair<3, S>,  launch_dcgs_pair<4, S>,  launch_dcgs_pair<5, S>,
      launch_dcgs_pair<6, S>,  launch_dcgs_pair<7, S>,  launch_dcgs_pair<8, S>,
      launch_dcgs_pair<9, S>,  launch_dcgs_pair<10, S>, launch_dcgs_pair<11, S>,
      launch_dcgs_pair<12, S>, launch_dcgs_pair<13, S>, launch_dcgs_pair<14, S>,
      launch_dcgs_pair<15, S>, launch_dcgs_pair<16, S>, launch_dcgs_pair<17, S>,
      launch_dcgs_pair<18, S>, launch_dcgs_pair<19, S>, launch_dcgs_pair<20, S>,
      launch_dcgs_pair<21, S>, launch_dcgs_pair<22, S>, launch_dcgs_pair<23, S>,
      launch_dcgs_pair<24, S>, launch_dcgs_pair<25, S>, launch_dcgs_pair<26, S>,
      launch_dcgs_pair<27, S>, launch_dcgs_pair<28, S>, launch_dcgs_pair<29, S>,
      launch_dcgs_pair<30, S>, launch_dcgs_pair<31, S>};
  static_assert(kDcgsMax == 32, "one instantiation per basis length");
  pairs[j](V, ldv, n2, part, tickets, coef, st, s);
}

// y = x / *s as double-float (the first basis vector of a restart cycle)
__global__ void scale_inv_df_kernel(size_t N, const double* __restrict__ x,
                                    const double* __restrict__ s, df* y) {
  const double inv = 1.0 / s[0];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = df_from_bits(x[i] * inv);
}

// x += Z c with double-float Z: the combination in double-float, one FP64 add
__global__ void update_df_kernel(const df* __restrict__ Z, size_t ldz, int k,
                                 const double* __restrict__ c, double* x, size_t N) {
  __shared__ df cs[kDcgsMax];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = df_from_bits(c[i]);
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N;
       e += (size_t)gridDim.x * blockDim.x) {
    df s(0.f, 0.f);
    for (int i = 0; i < k; ++i) s = df_fma(cs[i], Z[(size_t)i * ldz + e], s);
    x[e] = x[e] + (double)s;
  }
}

}  // namespace

cudaError_t launch_dcgs2(double* V, size_t ldv, int j, size_t N, double* part, unsigned* tickets,
                         double* coef, const ArnoldiState& st, bool df_store, cudaStream_t s) {
  if (j < 0 || j >= kDcgsMax || j >= st.m || !st.H || !st.gpre || (ldv & 1) || (N & 1))
    return cudaErrorInvalidValue;
  const size_t n2 = N / 2;
  double* w = V + (size_t)(j + 1) * ldv;
  if (df_store) {
    launch_dcgs_step<df>(V, ldv, j, n2, part, tickets, coef, st, s);
    scale_by_df_kernel<<<152 * 4, 256, 0, s>>>(w, n2, st.status);
  } else {
    launch_dcgs_step<double>(V, ldv, j, n2, part, tickets, coef, st, s);
    scale_by_kernel<<<152 * 4, 256, 0, s>>>(w, n2, st.status);
  }
  return cudaGetLastError();
}

cudaError_t launch_scale_inv_df(size_t N, const double* x, const double* s, double* y_df,
                                cudaStream_t st) {
  scale_inv_df_kernel<<<krylov_blocks(), KT, 0, st>>>(N, x, s, reinterpret_cast<df*>(y_df));
  return cudaGetLastError();
}

cudaError_t launch_update_df(const double* Z_df, size_t ldz, int k, const double* c, double* x,
                             size_t N, cudaStream_t st) {
  if (k > kDcgsMax) return cudaErrorInvalidValue;
  update_df_kernel<<<krylov_blocks(), KT, 0, st>>>(reinterpret_cast<const df*>(Z_df), ldz, k, c,
                                                   x, N);
  return cudaGetLastError();
}

// ============================================================================
// grouped FGMRES (many problems in lockstep): the passes above over items
// (problem entry, chunk of kGKChunk double2 pairs); each problem reduces its
// partials in the block that finishes its last chunk, in chunk order

namespace {

__device__ __forceinline__ bool publish_partials_at(const double* sred, int cnt, double* part,
                                                    int nb, int slot, unsigned* ticket) {
  __shared__ unsigned last;
  if ((int)threadIdx.x < cnt) {
    double t = 0.0;
    for (int w = 0; w < CT / 32; ++w) t += sred[threadIdx.x * (CT / 32) + w];
    part[(size_t)threadIdx.x * nb + slot] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == (unsigned)(nb - 1)) ? 1u : 0u;
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

__device__ __forceinline__ void chunk_range(const GKrylov& e, int chunk, size_t& lo, size_t& hi) {
  const size_t n2 = (e.N + 1) / 2;
  lo = (size_t)chunk * kGKChunk;
  hi = lo + kGKChunk < n2 ? lo + kGKChunk : n2;
}

template <int KMAX>
__global__ void __launch_bounds__(CT) g_cgs_project_kernel(const GKrylov* __restrict__ ent,
                                                           const GItem* __restrict__ items,
                                                           int nitems, int j, GGate gate) {
  __shared__ double sred[(KMAX + 1) * (CT / 32)];
  const int k = j + 1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GKrylov& e = ent[g.e];
    if (!gate_open(gate, e.prob, -1)) continue;
    size_t lo, hi;
    chunk_range(e, g.unit, lo, hi);
    const double* w = e.V + (size_t)(j + 1) * e.ldv;
    double acc[KMAX + 1];
#pragma unroll
    for (int q = 0; q <= KMAX; ++q) acc[q] = 0.0;
    for (size_t q = lo + threadIdx.x; q < hi; q += CT) {
      const double2 wv = ld2(w, q);
#pragma unroll
      for (int gg = 0; gg < KMAX; ++gg)
        if (gg < k) {
          const double2 v = ld2(e.V + (size_t)gg * e.ldv, q);
          acc[gg] = fma(v.x, wv.x, fma(v.y, wv.y, acc[gg]));
        }
      acc[KMAX] = fma(wv.x, wv.x, fma(wv.y, wv.y, acc[KMAX]));
    }
    block_reduce_vec<KMAX + 1>(acc, KMAX + 1, sred);
    if (publish_partials_at(sred, KMAX + 1, e.part, e.nchunk, g.unit, e.tickets)) {
      final_sums(e.part, KMAX + 1, e.nchunk, e.h);
      if (threadIdx.x == 0) {
        e.tickets[0] = 0u;
        e.st.status->pad = needs_second_projection(e.h, k, e.h[KMAX]);
      }
    }
    __syncthreads();
  }
}

// close Arnoldi step j of problem e (one thread): Givens update, iteration
// count, gates for the next step
__device__ void grouped_close_step(const GKrylov& e, int j, const double* h2, double nrm2,
                                   int* active, int* relax) {
  const int k = j + 1;
  arnoldi_column(e.st, j, e.h, h2, nrm2);
  GSolveState& ss = *e.ss;
  const ArnoldiStatus as = *e.st.status;
  ss.its += 1;
  ss.k = k;
  if (as.nonfinite) ss.failed = 1;
  const bool stop = as.gabs <= ss.tol || ss.its >= e.maxit || as.hnext == 0.0 || as.nonfinite ||
                    k >= e.restart;
  if (relax[e.prob]) ss.relaxed += 1;  // this step's matvec ran in FP32
  active[e.prob] = stop ? 0 : 1;
  relax[e.prob] = (e.relax_on && as.gabs <= FDE_RELAX_FACTOR * ss.tol) ? 1 : 0;
}

template <int KMAX>
__global__ void __launch_bounds__(CT) g_cgs_subproj_kernel(const GKrylov* __restrict__ ent,
                                                           const GItem* __restrict__ items,
                                                           int nitems, int j, GGate gate,
                                                           int* active, int* relax) {
  __shared__ double sred[KMAX * (CT / 32)];
  __shared__ double hs[KMAX];
  __shared__ double nrm2;
  const int k = j + 1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GKrylov& e = ent[g.e];
    if (!gate_open(gate, e.prob, -1)) continue;
    if ((int)threadIdx.x < KMAX) hs[threadIdx.x] = (int)threadIdx.x < k ? e.h[threadIdx.x] : 0.0;
    __syncthreads();
    size_t lo, hi;
    chunk_range(e, g.unit, lo, hi);
    double* w = e.V + (size_t)(j + 1) * e.ldv;
    if (!e.st.status->pad) {
      // one projection sufficed: w -= V h, ||w||^2, and this pass closes the step
      double a1[1] = {0.0};
      for (size_t q = 2 * lo + threadIdx.x; q < 2 * hi; q += CT) {
        double wv = w[q];
#pragma unroll
        for (int gg = 0; gg < KMAX; ++gg)
          if (gg < k) wv = fma(-hs[gg], e.V[(size_t)gg * e.ldv + q], wv);
        w[q] = wv;
        a1[0] = fma(wv, wv, a1[0]);
      }
      block_reduce_vec<1>(a1, 1, sred);
      if (publish_partials_at(sred, 1, e.part, e.nchunk, g.unit, e.tickets + 1)) {
        final_sums(e.part, 1, e.nchunk, &nrm2);
        __syncthreads();
        if (threadIdx.x == 0) {
          e.tickets[1] = 0u;
          grouped_close_step(e, j, nullptr, nrm2, active, relax);
        }
      }
      __syncthreads();
      continue;
    }
    double acc[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) acc[q] = 0.0;
    for (size_t q = 2 * lo + threadIdx.x; q < 2 * hi; q += CT) {  // scalar elements
      double v[KMAX];
#pragma unroll
      for (int gg = 0; gg < KMAX; ++gg) v[gg] = gg < k ? e.V[(size_t)gg * e.ldv + q] : 0.0;
      double wv = w[q];
#pragma unroll
      for (int gg = 0; gg < KMAX; ++gg) wv = fma(-hs[gg], v[gg], wv);
      w[q] = wv;
#pragma unroll
      for (int gg = 0; gg < KMAX; ++gg) acc[gg] = fma(v[gg], wv, acc[gg]);
    }
    block_reduce_vec<KMAX>(acc, k, sred);
    if (publish_partials_at(sred, k, e.part, e.nchunk, g.unit, e.tickets + 1)) {
      final_sums(e.part, k, e.nchunk, e.h2);
      if (threadIdx.x == 0) e.tickets[1] = 0u;
    }
    __syncthreads();
  }
}

template <int KMAX>
__global__ void __launch_bounds__(CT) g_cgs_subnorm_kernel(const GKrylov* __restrict__ ent,
                                                           const GItem* __restrict__ items,
                                                           int nitems, int j, GGate gate,
                                                           int* active, int* relax) {
  __shared__ double sred[CT / 32];
  __shared__ double hs[KMAX];
  __shared__ double nrm2;
  const int k = j + 1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GKrylov& e = ent[g.e];
    if (!gate_open(gate, e.prob, -1)) continue;
    // a problem whose first projection sufficed closed its step in the previous pass
    if (!e.st.status->pad) continue;
    if ((int)threadIdx.x < KMAX) hs[threadIdx.x] = (int)threadIdx.x < k ? e.h2[threadIdx.x] : 0.0;
    __syncthreads();
    size_t lo, hi;
    chunk_range(e, g.unit, lo, hi);
    double2* w2 = reinterpret_cast<double2*>(e.V + (size_t)(j + 1) * e.ldv);
    double acc[1] = {0.0};
    for (size_t q = lo + threadIdx.x; q < hi; q += CT) {
      double2 wv = w2[q];
#pragma unroll
      for (int gg = 0; gg < KMAX; ++gg)
        if (gg < k) {
          const double2 v = ld2(e.V + (size_t)gg * e.ldv, q);
          wv.x = fma(-hs[gg], v.x, wv.x);
          wv.y = fma(-hs[gg], v.y, wv.y);
        }
      w2[q] = wv;
      acc[0] = fma(wv.x, wv.x, fma(wv.y, wv.y, acc[0]));
    }
    block_reduce_vec<1>(acc, 1, sred);
    if (publish_partials_at(sred, 1, e.part, e.nchunk, g.unit, e.tickets + 2)) {
      final_sums(e.part, 1, e.nchunk, &nrm2);
      __syncthreads();
      if (threadIdx.x == 0) {
        e.tickets[2] = 0u;
        grouped_close_step(e, j, e.h2, nrm2, active, relax);
      }
    }
    __syncthreads();
  }
}

__global__ void g_scale_kernel(const GKrylov* __restrict__ ent, const GItem* __restrict__ items,
                               int nitems, int j, GGate gate) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GKrylov& e = ent[g.e];
    // the step's last pass closed the gate of a problem that stopped: its
    // newest vector is not used, so leaving it unscaled is harmless
    if (gate.active[e.prob] == 0 && e.ss->k != j + 1) continue;
    size_t lo, hi;
    chunk_range(e, g.unit, lo, hi);
    const double inv = e.st.status->inv_norm;
    double2* w2 = reinterpret_cast<double2*>(e.V + (size_t)(j + 1) * e.ldv);
    for (size_t q = lo + threadIdx.x; q < hi; q += CT) {
      double2 v = w2[q];
      v.x *= inv;
      v.y *= inv;
      w2[q] = v;
    }
  }
}

__global__ void g_vec_kernel(int op, const GVec* __restrict__ ent, const GItem* __restrict__ items,
                             int nitems, GGate gate) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GVec& e = ent[g.e];
    if (!gate_open(gate, e.prob, -1)) continue;
    const size_t lo = (size_t)g.unit * kGChunk;
    const size_t hi = lo + kGChunk < e.N ? lo + kGChunk : e.N;
    for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      switch (op) {
        case GV_D2F: e.yf[i] = (float)e.a[i]; break;
        case GV_F2D: e.y[i] = (double)e.af[i]; break;
        case GV_SUB: e.y[i] = e.a[i] - e.b[i]; break;
        case GV_LINCOMB: e.y[i] = e.s0 * e.a[i] + e.s1 * e.b[i] + e.s2 * e.c[i]; break;
        case GV_SCALE_INV: e.y[i] = e.a[i] * (1.0 / e.sptr[0]); break;
        case GV_ZERO: e.y[i] = 0.0; break;
        default: e.y[i] = e.a[i]; break;
      }
    }
  }
}

__global__ void __launch_bounds__(CT) g_norm_kernel(const GVec* __restrict__ ent,
                                                    const GKrylov* __restrict__ kry,
                                                    const GItem* __restrict__ items, int nitems,
                                                    GGate gate) {
  __shared__ double sred[CT / 32];
  __shared__ double tot;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GVec& e = ent[g.e];
    const GKrylov& kk = kry[g.e];
    if (!gate_open(gate, e.prob, -1)) continue;
    const int nb = (int)((e.N + kGChunk - 1) / kGChunk);
    const size_t lo = (size_t)g.unit * kGChunk;
    const size_t hi = lo + kGChunk < e.N ? lo + kGChunk : e.N;
    double acc[1] = {0.0};
    for (size_t i = lo + threadIdx.x; i < hi; i += CT) acc[0] = fma(e.a[i], e.a[i], acc[0]);
    block_reduce_vec<1>(acc, 1, sred);
    if (publish_partials_at(sred, 1, kk.part, nb, g.unit, kk.tickets + 3)) {
      final_sums(kk.part, 1, nb, &tot);
      __syncthreads();
      if (threadIdx.x == 0) {
        kk.tickets[3] = 0u;
        e.y[0] = sqrt(tot);
      }
    }
    __syncthreads();
  }
}

__global__ void g_solve_start_kernel(const GKrylov* __restrict__ ent, int count, int* active,
                                     int* incycle) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
    const GKrylov& e = ent[q];
    GSolveState& ss = *e.ss;
    ss.bnorm = e.scal[0];
    ss.tol = e.rtol * ss.bnorm;
    ss.beta = ss.bnorm;
    ss.its = ss.k = ss.restarts = ss.relaxed = 0;
    ss.failed = isfinite(ss.bnorm) ? 0 : 1;
    ss.converged = (ss.bnorm == 0.0) ? 1 : 0;
    ss.rel_residual = 0.0;
    const int go = (!ss.converged && !ss.failed) ? 1 : 0;
    active[e.prob] = go;
    incycle[e.prob] = go;
  }
}

__global__ void g_cycle_start_kernel(const GKrylov* __restrict__ ent, int count, int first,
                                     const int* incycle, int* active, int* relax) {
  const int p = blockIdx.x;
  if (p >= count) return;
  const GKrylov& e = ent[p];
  if (!incycle[e.prob]) return;
  GSolveState& ss = *e.ss;
  const double beta = first ? ss.bnorm : e.scal[1];
  for (int i = threadIdx.x; i <= e.st.m; i += blockDim.x) e.st.g[i] = i == 0 ? beta : 0.0;
  if (threadIdx.x == 0) {
    e.st.status->gabs = beta;
    ss.beta = beta;
    ss.k = 0;
    ss.restarts += 1;
    active[e.prob] = 1;
    // the first matvec's precision follows the residual estimate |g_0| = beta
    relax[e.prob] = (e.relax_on && beta <= FDE_RELAX_FACTOR * ss.tol) ? 1 : 0;
  }
}

__global__ void g_lsq_kernel(const GKrylov* __restrict__ ent, int count, const int* incycle) {
  const int p = blockIdx.x;
  if (p >= count || threadIdx.x != 0) return;
  const GKrylov& e = ent[p];
  if (!incycle[e.prob]) return;
  const int k = e.ss->k, m = e.st.m;
  for (int i = k - 1; i >= 0; --i) {
    double s = e.st.g[i];
    for (int l = i + 1; l < k; ++l) s -= e.st.R[(size_t)l * (m + 1) + i] * e.y[l];
    e.y[i] = s / e.st.R[(size_t)i * (m + 1) + i];
  }
}

__global__ void g_update_kernel(const GKrylov* __restrict__ ent, double* const* __restrict__ xs,
                                const GItem* __restrict__ items, int nitems, const int* incycle) {
  __shared__ double cs[ArnoldiState::kMaxM];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GKrylov& e = ent[g.e];
    if (!incycle[e.prob]) continue;
    const int k = e.ss->k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = e.y[i];
    __syncthreads();
    double* x = xs[g.e];
    const size_t lo = (size_t)g.unit * kGChunk;
    const size_t hi = lo + kGChunk < e.N ? lo + kGChunk : e.N;
    for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      double s = x[i];
      for (int q = 0; q < k; ++q) s += cs[q] * e.Z[(size_t)q * e.ldv + i];
      x[i] = s;
    }
    __syncthreads();
  }
}

__global__ void g_cycle_end_kernel(const GKrylov* __restrict__ ent, int count, int* incycle) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
    const GKrylov& e = ent[q];
    if (!incycle[e.prob]) continue;
    GSolveState& ss = *e.ss;
    const double beta = e.scal[1];
    if (!isfinite(beta)) ss.failed = 1;
    ss.rel_residual = ss.bnorm > 0.0 ? beta / ss.bnorm : 0.0;
    ss.converged = beta <= ss.tol ? 1 : 0;
    incycle[e.prob] = (!ss.converged && !ss.failed && ss.its < e.maxit) ? 1 : 0;
  }
}

int g_grid(int nitems, const void* kernel) {
  const int nb = resident_blocks(kernel);
  return nitems < nb ? nitems : nb;
}

}  // namespace

cudaError_t launch_g_cgs2(const GKrylov* ent, const GItem* items, int nitems, int j, GGate gate,
                          int* active, int* relax, cudaStream_t st) {
  const int k = j + 1;
  if (nitems <= 0) return cudaSuccess;
  if (k < 1 || k > 32) return cudaErrorInvalidValue;
#define G_CGS(KM)                                                                               \
  {                                                                                            \
    g_cgs_project_kernel<KM><<<g_grid(nitems, (const void*)g_cgs_project_kernel<KM>), CT, 0,  \
                               st>>>(ent, items, nitems, j, gate);                            \
    g_cgs_subproj_kernel<KM><<<g_grid(nitems, (const void*)g_cgs_subproj_kernel<KM>), CT, 0,  \
                               st>>>(ent, items, nitems, j, gate, active, relax);             \
    g_cgs_subnorm_kernel<KM><<<g_grid(nitems, (const void*)g_cgs_subnorm_kernel<KM>), CT, 0,  \
                               st>>>(ent, items, nitems, j, gate, active, relax);             \
  }
  if (k <= 4) G_CGS(4)
  else if (k <= 8) G_CGS(8)
  else if (k <= 16) G_CGS(16)
  else G_CGS(32)
#undef G_CGS
  g_scale_kernel<<<g_grid(nitems, (const void*)g_scale_kernel), CT, 0, st>>>(ent, items, nitems, j,
                                                                            gate);
  return cudaGetLastError();
}

cudaError_t launch_g_vec(int op, const GVec* ent, const GItem* items, int nitems, GGate gate,
                         cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const int grid = nitems < 152 * 16 ? nitems : 152 * 16;
  g_vec_kernel<<<grid, 256, 0, st>>>(op, ent, items, nitems, gate);
  return cudaGetLastError();
}

cudaError_t launch_g_norm(const GVec* ent, const GKrylov* kry, const GItem* items, int nitems,
                          GGate gate, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  g_norm_kernel<<<g_grid(nitems, (const void*)g_norm_kernel), CT, 0, st>>>(ent, kry, items,
                                                                            nitems, gate);
  return cudaGetLastError();
}

cudaError_t launch_g_solve_start(const GKrylov* ent, int count, int* active, int* incycle,
                                 cudaStream_t st) {
  g_solve_start_kernel<<<(count + 127) / 128, 128, 0, st>>>(ent, count, active, incycle);
  return cudaGetLastError();
}

cudaError_t launch_g_cycle_start(const GKrylov* ent, int count, int first, const int* incycle,
                                 int* active, int* relax, cudaStream_t st) {
  g_cycle_start_kernel<<<count, 64, 0, st>>>(ent, count, first, incycle, active, relax);
  return cudaGetLastError();
}

cudaError_t launch_g_lsq(const GKrylov* ent, int count, const int* incycle, cudaStream_t st) {
  g_lsq_kernel<<<count, 32, 0, st>>>(ent, count, incycle);
  return cudaGetLastError();
}

cudaError_t launch_g_update(const GKrylov* ent, double* const* x, const GItem* items, int nitems,
                            const int* incycle, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const int grid = nitems < 152 * 8 ? nitems : 152 * 8;
  g_update_kernel<<<grid, 256, 0, st>>>(ent, x, items, nitems, incycle);
  return cudaGetLastError();
}

cudaError_t launch_g_cycle_end(const GKrylov* ent, int count, int* incycle, cudaStream_t st) {
  g_cycle_end_kernel<<<(count + 127) / 128, 128, 0, st>>>(ent, count, incycle);
  return cudaGetLastError();
}

}  // namespace fde

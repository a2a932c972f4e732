// Toeplitz products of the CN-WSGD operator on CUDA cores.
//
// The operator of Eq. (M)/(AxAy) applies, along every grid row (x) and every
// grid column (y), a lower-Hessenberg Toeplitz matrix A = [t_{i-k}] (level 0:
// t_d = -w_{d+1}, Eq. AN) and its transpose, each scaled point-wise by a
// coefficient field.  Two evaluations live here:
//
//  * fft_pass: the circulant embedding of size L = 2^logL >= 2n - 1 that makes
//    the product O(n log n) (the fast matrix-vector product noted in Sec. 1).
//    Two real vectors are packed as one complex vector; a forward radix-2 DIF
//    transform (natural order in, bit-reversed out) is multiplied point-wise by
//    the bit-reversed spectra of A and A^T and two inverse DIT transforms
//    (bit-reversed in, natural out) give A x and A^T x of both vectors at once
//    -- no bit-reversal permutation is ever performed.
//  * direct_pass: plain O(n^2) summation for small levels.
#include <mutex>
#include <set>
#include <utility>

#include "common.cuh"
#include "df32.cuh"

namespace fde {

cudaError_t ensure_max_smem(const void* kernel) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kernel, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) done.insert({kernel, dev});
  return e;
}

__device__ __forceinline__ int bitrev(int x, int bits) {
  return (int)(__brev((unsigned)x) >> (32 - bits));
}

template <typename R>
__device__ __forceinline__ cx<R> to_cx(cx<double> z) {
  return {R(z.re), R(z.im)};
}
template <typename R, typename C>
__device__ __forceinline__ R coef(const C* p, size_t i) {
  return p ? R(p[i]) : R(1);
}
template <>
__device__ __forceinline__ df coef<df, df>(const df* p, size_t i) {
  return p ? p[i] : df(1.f, 0.f);
}

// Twiddle table layout: for a butterfly of span `half` (sub-transform length
// 2 half) the factors omega_{2 half}^pos, pos < half, are stored contiguously
// at T[half - 1 + pos] (L - 1 entries in all), so the threads of a warp,
// which handle consecutive `pos`, read consecutive words.
//
// Shared-memory layout: element i lives at pad(i) = i + i/16, so that the
// stride-16 accesses of the last fused pass fall into different banks.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int L) { return L + (L >> 4); }

// One fused decimation-in-frequency pass: stages s .. s+q-1 (Q = 2^q points per
// thread group, held in registers).  Group g covers the points
// i0 + m h, m < Q, with h = L >> (s+q) the span of the last stage.
// With h = 1 (UNIT: the last forward / first inverse pass) the twiddles of
// spans 1 and 2, and half of those of span 4, are exactly 1 or -i: those
// butterflies skip the multiply (multiplying by -i swaps and negates).
template <typename R>
__device__ __forceinline__ cx<R> mul_neg_i(cx<R> a) { return {a.im, -a.re}; }  // a * (-i)
template <typename R>
__device__ __forceinline__ cx<R> mul_i(cx<R> a) { return {-a.im, a.re}; }      // a * i
// The double-float passes already use every register the 512-thread block
// allows; a second specialised copy of the butterflies pushes them into local
// memory and costs more than the skipped multiplies save (measured), so they
// keep the general path.
template <typename R>
constexpr bool kUnitPass = true;
template <>
constexpr bool kUnitPass<df> = false;

template <int Q, bool UNIT, typename R>
__device__ __forceinline__ void dif_group(cx<R>* a, int i0, int h, int pos,
                                          const cx<R>* __restrict__ tw) {
  cx<R> v[Q];
#pragma unroll
  for (int m = 0; m < Q; ++m) v[m] = a[pad(i0 + m * h)];
#pragma unroll
  for (int sm = Q / 2; sm >= 1; sm >>= 1) {  // span in units of h
    const int span = sm * h;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      if (m & sm) continue;
      const cx<R> u = v[m], x = v[m + sm];
      v[m] = cadd(u, x);
      const int k = m & (sm - 1);  // twiddle exponent within the span (pos = 0 when UNIT)
      if (UNIT && (sm == 1 || k == 0)) {
        v[m + sm] = csub(u, x);  // w = 1
      } else if (UNIT && 2 * k == sm) {
        v[m + sm] = mul_neg_i(csub(u, x));  // w = -i
      } else {
        const cx<R> w = tw[span - 1 + pos + k * h];
        v[m + sm] = cmul(csub(u, x), w);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < Q; ++m) a[pad(i0 + m * h)] = v[m];
}

// One fused decimation-in-time inverse pass: stages s .. s+q-1 (spans h .. 2^(q-1) h,
// h = 2^s), conjugated twiddles.
template <int Q, bool UNIT, typename R>
__device__ __forceinline__ void dit_group(cx<R>* a, int i0, int h, int pos,
                                          const cx<R>* __restrict__ tw) {
  cx<R> v[Q];
#pragma unroll
  for (int m = 0; m < Q; ++m) v[m] = a[pad(i0 + m * h)];
#pragma unroll
  for (int sm = 1; sm < Q; sm <<= 1) {
    const int span = sm * h;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      if (m & sm) continue;
      const int k = m & (sm - 1);
      cx<R> t;
      if (UNIT && (sm == 1 || k == 0)) {
        t = v[m + sm];  // conj(1) = 1
      } else if (UNIT && 2 * k == sm) {
        t = mul_i(v[m + sm]);  // conj(-i) = i
      } else {
        const cx<R> w = tw[span - 1 + pos + k * h];
        t = cmulc(v[m + sm], w);
      }
      const cx<R> u = v[m];
      v[m] = cadd(u, t);
      v[m + sm] = csub(u, t);
    }
  }
#pragma unroll
  for (int m = 0; m < Q; ++m) a[pad(i0 + m * h)] = v[m];
}

// forward transform, in place, natural order -> bit-reversed order
template <typename R>
__device__ void fft_dif(cx<R>* a, int logL, const cx<R>* __restrict__ tw) {
  int s = 0;
  while (s < logL) {
    const int rem = logL - s;
    const int q = rem >= 4 ? 4 : (rem >= 2 ? 2 : 1);
    const int lh = logL - s - q;  // log2 h
    const int h = 1 << lh;
    const int ngroups = 1 << (logL - q);
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
      const int pos = g & (h - 1);
      const int i0 = ((g >> lh) << (lh + q)) + pos;
      if (h == 1 && kUnitPass<R>) {
        if (q == 4) dif_group<16, true>(a, i0, h, pos, tw);
        else if (q == 2) dif_group<4, true>(a, i0, h, pos, tw);
        else dif_group<2, true>(a, i0, h, pos, tw);
      } else {
        if (q == 4) dif_group<16, false>(a, i0, h, pos, tw);
        else if (q == 2) dif_group<4, false>(a, i0, h, pos, tw);
        else dif_group<2, false>(a, i0, h, pos, tw);
      }
    }
    __syncthreads();
    s += q;
  }
}

// inverse transform (unnormalised) of two arrays (or of `a` alone when c is
// null), in place, bit-reversed order -> natural order
template <typename R>
__device__ void fft_dit_inv2(cx<R>* a, cx<R>* c, int logL, const cx<R>* __restrict__ tw) {
  int s = 0;
  while (s < logL) {
    const int rem = logL - s;
    const int q = rem >= 4 ? 4 : (rem >= 2 ? 2 : 1);
    const int h = 1 << s;
    const int ngroups = 1 << (logL - q);
    const int total = c ? 2 * ngroups : ngroups;  // c may be null: one array
    for (int gg = threadIdx.x; gg < total; gg += blockDim.x) {
      cx<R>* arr = gg < ngroups ? a : c;
      const int g = gg < ngroups ? gg : gg - ngroups;
      const int pos = g & (h - 1);
      const int i0 = ((g >> s) << (s + q)) + pos;
      if (h == 1 && kUnitPass<R>) {
        if (q == 4) dit_group<16, true>(arr, i0, h, pos, tw);
        else if (q == 2) dit_group<4, true>(arr, i0, h, pos, tw);
        else dit_group<2, true>(arr, i0, h, pos, tw);
      } else {
        if (q == 4) dit_group<16, false>(arr, i0, h, pos, tw);
        else if (q == 2) dit_group<4, false>(arr, i0, h, pos, tw);
        else dit_group<2, false>(arr, i0, h, pos, tw);
      }
    }
    __syncthreads();
    s += q;
  }
}

// one vector pair of a pass: x_va + i x_vb transformed, multiplied by the
// spectra of A and A^T, transformed back, scaled and written (two buffers a, c
// of padded_len(L) in shared memory)
template <typename T, typename R, typename C>
__device__ __forceinline__ void fft_pass_pair(const T* __restrict__ X, int es, int vs, int nvec,
                                              int n, int logL, const cx<R>* __restrict__ S1,
                                              const cx<R>* __restrict__ S2,
                                              const cx<R>* __restrict__ tw,
                                              const C* __restrict__ cp, const C* __restrict__ cm,
                                              const T* __restrict__ M, R cmass, T* Y,
                                              int accumulate, int pair, cx<R>* a, cx<R>* c) {
  const int L = 1 << logL;
  const int va = 2 * pair;
  const bool hasb = va + 1 < nvec;
  const size_t oa = (size_t)va * vs, ob = oa + vs;
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    cx<R> z = {R(0), R(0)};
    if (i < n) {  // x_v[i] packed as re (vector va) + i im (vector va + 1)
      z.re = cvt<R>(X[oa + (size_t)i * es]);
      if (hasb) z.im = cvt<R>(X[ob + (size_t)i * es]);
    }
    a[pad(i)] = z;
  }
  __syncthreads();
  fft_dif(a, logL, tw);
  for (int p = threadIdx.x; p < L; p += blockDim.x) {
    const cx<R> z = a[pad(p)];
    c[pad(p)] = cmul(z, S2[p]);
    a[pad(p)] = cmul(z, S1[p]);
  }
  __syncthreads();
  fft_dit_inv2(a, c, logL, tw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const size_t ia = oa + (size_t)i * es;
    const cx<R> ya_ = a[pad(i)], yc_ = c[pad(i)];
    R y = ya_.re * coef<R, C>(cp, ia) + yc_.re * coef<R, C>(cm, ia);
    if (M) y += cmass * cvt<R>(M[ia]);
    if (accumulate) y += cvt<R>(Y[ia]);
    Y[ia] = cvt<T>(y);
    if (hasb) {
      const size_t ib = ob + (size_t)i * es;
      R yb = ya_.im * coef<R, C>(cp, ib) + yc_.im * coef<R, C>(cm, ib);
      if (M) yb += cmass * cvt<R>(M[ib]);
      if (accumulate) yb += cvt<R>(Y[ib]);
      Y[ib] = cvt<T>(yb);
    }
  }
  __syncthreads();
}

// Block size of the two-buffer pass.  FP32: 256 threads with registers capped
// for three blocks an SM (the shared-memory limit at L = 4096), so a pass
// keeps three vector pairs in flight; measured 11-12 % faster than 512
// threads at L = 2048 and 4096.  FP64 and double-float: 512 threads (their
// registers allow one block an SM either way; 256 measured slower).
template <typename R>
struct FftBlock {
  static constexpr int threads = 512, min_blocks = 1;
};
template <>
struct FftBlock<float> {
  static constexpr int threads = 256, min_blocks = 3;
};

template <typename T, typename R, typename C>
__global__ void __launch_bounds__(FftBlock<R>::threads, FftBlock<R>::min_blocks)
fft_pass_kernel(const T* __restrict__ X, int es, int vs, int nvec, int n, int logL,
                const cx<R>* __restrict__ S1, const cx<R>* __restrict__ S2,
                const cx<R>* __restrict__ tw, const C* __restrict__ cp,
                const C* __restrict__ cm, const T* __restrict__ M, double cmass_d, T* Y,
                int accumulate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << logL;
  cx<R>* a = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* c = a + padded_len(L);
  const int npairs = (nvec + 1) >> 1;
  for (int pair = blockIdx.x; pair < npairs; pair += gridDim.x)
    fft_pass_pair<T, R, C>(X, es, vs, nvec, n, logL, S1, S2, tw, cp, cm, M, R(cmass_d), Y,
                           accumulate, pair, a, c);
}

// two passes of the same length in one launch: pairs 0 .. npa-1 of a, then b's
template <typename T, typename R, typename C>
__global__ void __launch_bounds__(FftBlock<R>::threads, FftBlock<R>::min_blocks)
fft_pass2_kernel(const FftPass<T, R, C> pa, const FftPass<T, R, C> pb, int logL) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << logL;
  cx<R>* a = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* c = a + padded_len(L);
  const int npa = (pa.nvec + 1) >> 1, npb = (pb.nvec + 1) >> 1;
  for (int pair = blockIdx.x; pair < npa + npb; pair += gridDim.x) {
    if (pair < npa)
      fft_pass_pair<T, R, C>(pa.X, pa.es, pa.vs, pa.nvec, pa.n, logL, pa.S1, pa.S2, pa.tw, pa.cp,
                             pa.cm, pa.M, R(pa.cmass), pa.Y, pa.accumulate, pair, a, c);
    else
      fft_pass_pair<T, R, C>(pb.X, pb.es, pb.vs, pb.nvec, pb.n, logL, pb.S1, pb.S2, pb.tw, pb.cp,
                             pb.cm, pb.M, R(pb.cmass), pb.Y, pb.accumulate, pair - npa, a, c);
  }
}

// grouped: item (entry, pair) of many problems' passes in one launch
template <typename T, typename R, typename C>
__global__ void __launch_bounds__(256)
g_fft_pass_kernel(const GFftPass<T, R, C>* __restrict__ ent, const GItem* __restrict__ items,
                  int nitems, GGate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GFftPass<T, R, C> e = ent[g.e];
    if (!gate_open(gate, e.prob, e.want)) continue;
    cx<R>* a = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* c = a + padded_len(1 << e.logL);
    fft_pass_pair<T, R, C>(e.X, e.es, e.vs, e.nvec, e.n, e.logL, e.S1, e.S2, e.tw, e.cp, e.cm,
                           e.M, R(e.cmass), e.Y, e.accumulate, g.unit, a, c);
  }
}

template <typename T, typename R, typename C>
cudaError_t launch_g_fft_pass(const GFftPass<T, R, C>* ent, const GItem* items, int nitems,
                              int max_logL, GGate gate, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = fft_pass_two_buffer_bytes(max_logL, sizeof(cx<R>));
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_max_smem((const void*)g_fft_pass_kernel<T, R, C>);
    if (e != cudaSuccess) return e;
  }
  const int per_sm = (int)((227 * 1024) / (smem + 1024));
  int grid = 152 * (per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm));
  if (grid > nitems) grid = nitems;
  g_fft_pass_kernel<T, R, C><<<grid, 256, smem, st>>>(ent, items, nitems, gate);
  return cudaGetLastError();
}

// The same pass with one shared buffer: the forward spectrum of a pair is
// parked in this CTA's slice of `ws`, the A-product is transformed back and
// written, then the A^T-product is formed from the parked spectrum and added.
template <typename T, typename R, typename C>
__global__ void __launch_bounds__(512)
fft_pass_seq_kernel(const T* __restrict__ X, int es, int vs, int nvec, int n, int logL,
                    const cx<R>* __restrict__ S1, const cx<R>* __restrict__ S2,
                    const cx<R>* __restrict__ tw, const C* __restrict__ cp,
                    const C* __restrict__ cm, const T* __restrict__ M, double cmass_d, T* Y,
                    int accumulate, cx<R>* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << logL;
  const R cmass = R(cmass_d);
  cx<R>* a = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* spec = ws + (size_t)blockIdx.x * L;
  const int npairs = (nvec + 1) >> 1;
  for (int pair = blockIdx.x; pair < npairs; pair += gridDim.x) {
    const int va = 2 * pair;
    const bool hasb = va + 1 < nvec;
    const size_t oa = (size_t)va * vs, ob = oa + vs;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      cx<R> z = {R(0), R(0)};
      if (i < n) {
        z.re = cvt<R>(X[oa + (size_t)i * es]);
        if (hasb) z.im = cvt<R>(X[ob + (size_t)i * es]);
      }
      a[pad(i)] = z;
    }
    __syncthreads();
    fft_dif(a, logL, tw);
    for (int p = threadIdx.x; p < L; p += blockDim.x) {
      const cx<R> z = a[pad(p)];
      spec[p] = z;
      a[pad(p)] = cmul(z, S1[p]);
    }
    __syncthreads();
    fft_dit_inv2<R>(a, nullptr, logL, tw);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const size_t ia = oa + (size_t)i * es;
      const cx<R> ya_ = a[pad(i)];
      R y = ya_.re * coef<R, C>(cp, ia);
      if (M) y += cmass * cvt<R>(M[ia]);
      if (accumulate) y += cvt<R>(Y[ia]);
      Y[ia] = cvt<T>(y);
      if (hasb) {
        const size_t ib = ob + (size_t)i * es;
        R yb = ya_.im * coef<R, C>(cp, ib);
        if (M) yb += cmass * cvt<R>(M[ib]);
        if (accumulate) yb += cvt<R>(Y[ib]);
        Y[ib] = cvt<T>(yb);
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < L; p += blockDim.x) a[pad(p)] = cmul(spec[p], S2[p]);
    __syncthreads();
    fft_dit_inv2<R>(a, nullptr, logL, tw);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const size_t ia = oa + (size_t)i * es;
      const cx<R> yc_ = a[pad(i)];
      Y[ia] = cvt<T>(cvt<R>(Y[ia]) + yc_.re * coef<R, C>(cm, ia));
      if (hasb) {
        const size_t ib = ob + (size_t)i * es;
        Y[ib] = cvt<T>(cvt<R>(Y[ib]) + yc_.im * coef<R, C>(cm, ib));
      }
    }
    __syncthreads();
  }
}

size_t fft_pass_two_buffer_bytes(int logL, size_t cx_bytes) {
  return 2 * (size_t)padded_len(1 << logL) * cx_bytes;
}

template <typename T, typename R, typename C>
cudaError_t launch_fft_pass(const T* X, int es, int vs, int nvec, int n, int logL,
                            const cx<R>* S1, const cx<R>* S2, const cx<R>* tw, const C* cp,
                            const C* cm, const T* M, double cmass, T* Y, int accumulate,
                            cudaStream_t st, cx<R>* ws, size_t ws_elems) {
  const int L = 1 << logL;
  const int threads = L / 2 < 512 ? L / 2 : 512;  // the one-buffer pass
  const int npairs = (nvec + 1) / 2;
  if (fft_pass_two_buffer_bytes(logL, sizeof(cx<R>)) > 227 * 1024) {
    const size_t smem1 = (size_t)padded_len(L) * sizeof(cx<R>);
    if (smem1 > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = ensure_max_smem((const void*)fft_pass_seq_kernel<T, R, C>);
    if (e != cudaSuccess) return e;
    const int per_sm = (int)((227 * 1024) / (smem1 + 1024));
    int grid = 152 * (per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm));
    if (grid > npairs) grid = npairs;
    if (!ws || ws_elems / (size_t)L < 1) return cudaErrorInvalidValue;
    if ((size_t)grid > ws_elems / (size_t)L) grid = (int)(ws_elems / (size_t)L);
    fft_pass_seq_kernel<T, R, C><<<grid, threads, smem1, st>>>(
        X, es, vs, nvec, n, logL, S1, S2, tw, cp, cm, M, cmass, Y, accumulate, ws);
    return cudaGetLastError();
  }
  const size_t smem = 2 * (size_t)padded_len(L) * sizeof(cx<R>);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_max_smem((const void*)fft_pass_kernel<T, R, C>);
    if (e != cudaSuccess) return e;
  }
  const int per_sm = (int)((227 * 1024) / (smem + 1024));
  int grid = 152 * (per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm));
  if (grid > npairs) grid = npairs;
  const int threads2 = L / 2 < FftBlock<R>::threads ? L / 2 : FftBlock<R>::threads;
  fft_pass_kernel<T, R, C><<<grid, threads2, smem, st>>>(X, es, vs, nvec, n, logL, S1, S2, tw,
                                                         cp, cm, M, cmass, Y, accumulate);
  return cudaGetLastError();
}

template <typename T, typename R, typename C>
cudaError_t launch_fft_pass2(const FftPass<T, R, C>& a, const FftPass<T, R, C>& b, int logL,
                             cudaStream_t st, cx<R>* ws, size_t ws_elems) {
  const int L = 1 << logL;
  const size_t smem = 2 * (size_t)padded_len(L) * sizeof(cx<R>);
  if (smem > 227 * 1024) {
    cudaError_t e = launch_fft_pass<T, R, C>(a.X, a.es, a.vs, a.nvec, a.n, logL, a.S1, a.S2, a.tw,
                                             a.cp, a.cm, a.M, a.cmass, a.Y, a.accumulate, st, ws,
                                             ws_elems);
    if (e != cudaSuccess) return e;
    return launch_fft_pass<T, R, C>(b.X, b.es, b.vs, b.nvec, b.n, logL, b.S1, b.S2, b.tw, b.cp,
                                    b.cm, b.M, b.cmass, b.Y, b.accumulate, st, ws, ws_elems);
  }
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_max_smem((const void*)fft_pass2_kernel<T, R, C>);
    if (e != cudaSuccess) return e;
  }
  const int npairs = (a.nvec + 1) / 2 + (b.nvec + 1) / 2;
  const int per_sm = (int)((227 * 1024) / (smem + 1024));
  int grid = 152 * (per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm));
  if (grid > npairs) grid = npairs;
  const int threads = L / 2 < FftBlock<R>::threads ? L / 2 : FftBlock<R>::threads;
  fft_pass2_kernel<T, R, C><<<grid, threads, smem, st>>>(a, b, logL);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- spectra
template <typename R>
__global__ void __launch_bounds__(512)
build_spectra_kernel(const double* __restrict__ t, int n, int logL, double scale,
                                     cx<R>* S1, cx<R>* S2, cx<R>* twout, cx<double>* tw_global) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << logL;
  cx<double>* a = reinterpret_cast<cx<double>*>(smem_raw);
  // tw_global (when set) was filled by twiddle_kernel in an earlier launch: a
  // table written and read within one launch could meet stale read-only-cache lines
  cx<double>* tw = tw_global ? tw_global : a + padded_len(L);
  // tw[half - 1 + pos] = exp(-2 pi i pos / (2 half)), half = 1, 2, 4, ..., L/2
  for (int k = threadIdx.x; k < L - 1 && !tw_global; k += blockDim.x) {
    const int lh = 31 - __clz(k + 1);  // half = 2^lh <= k + 1 < 2 half
    const int half = 1 << lh, pos = k + 1 - half;
    double s, c;
    sincospi(-(double)pos / (double)half, &s, &c);
    tw[k] = {c, s};
    if (twout) twout[k] = to_cx<R>(tw[k]);
  }
  if (tw_global && twout)
    for (int k = threadIdx.x; k < L - 1; k += blockDim.x) twout[k] = to_cx<R>(tw[k]);
  // z = h1 + i h2: h1 embeds A (h1[d mod L] = t_d, d = -1..n-1) and h2 embeds
  // A^T (h2[m mod L] = t_{-m}, m = -(n-1)..1); L >= 2n - 1 keeps them apart.
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    const int d1 = (m <= n - 1) ? m : m - L;
    const double h1 = (d1 >= -1 && d1 <= n - 1) ? t[d1 + 1] : 0.0;
    const int m2 = (m <= 1) ? m : m - L;
    const double h2 = (m2 >= -(n - 1) && m2 <= 1) ? t[-m2 + 1] : 0.0;
    a[pad(m)] = {h1, h2};
  }
  __syncthreads();
  fft_dif(a, logL, tw);
  const double sc = scale / (double)L;
  for (int p = threadIdx.x; p < L; p += blockDim.x) {
    const int f = bitrev(p, logL);
    const int pp = bitrev((L - f) & (L - 1), logL);
    const cx<double> z = a[pad(p)], zc = {a[pad(pp)].re, -a[pad(pp)].im};
    const cx<double> h1 = {0.5 * (z.re + zc.re) * sc, 0.5 * (z.im + zc.im) * sc};
    // (z - zc) / (2i)
    const cx<double> h2 = {0.5 * (z.im - zc.im) * sc, -0.5 * (z.re - zc.re) * sc};
    S1[p] = to_cx<R>(h1);
    S2[p] = to_cx<R>(h2);
  }
}

__global__ void twiddle_kernel(int L, cx<double>* tw) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L - 1; k += gridDim.x * blockDim.x) {
    const int lh = 31 - __clz(k + 1);
    const int half = 1 << lh, pos = k + 1 - half;
    double s, c;
    sincospi(-(double)pos / (double)half, &s, &c);
    tw[k] = {c, s};
  }
}

template <typename R>
cudaError_t launch_build_spectra(const double* t, int n, int logL, double scale, cx<R>* S1,
                                 cx<R>* S2, cx<R>* tw, cudaStream_t st, cx<double>* tw_scratch) {
  const int L = 1 << logL;
  size_t smem = (size_t)(padded_len(L) + L) * sizeof(cx<double>);
  cx<double>* twg = nullptr;
  if (smem > 227 * 1024) {  // twiddles in global memory
    if (!tw_scratch) return cudaErrorInvalidValue;
    twg = tw_scratch;
    smem = (size_t)padded_len(L) * sizeof(cx<double>);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    twiddle_kernel<<<(L + 255) / 256, 256, 0, st>>>(L, twg);
  }
  cudaError_t e = cudaFuncSetAttribute(build_spectra_kernel<R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  build_spectra_kernel<R><<<1, 512, smem, st>>>(t, n, logL, scale, S1, S2, tw, twg);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- direct
template <typename T>
__device__ __forceinline__ void direct_pass_vector(const T* __restrict__ X, int es, int vs, int n,
                                                   const T* ts, const T* __restrict__ cp,
                                                   const T* __restrict__ cm,
                                                   const T* __restrict__ M, T cmass, T* Y,
                                                   int accumulate, int v, T* xs) {
  const size_t o = (size_t)v * vs;
  for (int k = threadIdx.x; k < n; k += blockDim.x) xs[k] = X[o + (size_t)k * es];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T s1 = T(0), s2 = T(0);
    const int k1 = (i + 1 < n - 1) ? i + 1 : n - 1;
    for (int k = 0; k <= k1; ++k) s1 += ts[i - k + 1] * xs[k];  // (A x)_i, t_{i-k}
    for (int k = (i > 0 ? i - 1 : 0); k < n; ++k) s2 += ts[k - i + 1] * xs[k];  // (A^T x)_i
    const size_t ia = o + (size_t)i * es;
    T y = s1 * (cp ? cp[ia] : T(1)) + s2 * (cm ? cm[ia] : T(1));
    if (M) y += cmass * M[ia];
    if (accumulate) y += Y[ia];
    Y[ia] = y;
  }
  __syncthreads();
}

template <typename T>
__global__ void direct_pass_kernel(const T* __restrict__ X, int es, int vs, int nvec, int n,
                                   const T* __restrict__ t, const T* __restrict__ cp,
                                   const T* __restrict__ cm, const T* __restrict__ M, T cmass,
                                   T* Y, int accumulate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ts = reinterpret_cast<T*>(smem_raw);  // t_d at ts[d+1], d = -1..n-1
  T* xs = ts + (n + 1);
  for (int k = threadIdx.x; k <= n; k += blockDim.x) ts[k] = t[k];
  for (int v = blockIdx.x; v < nvec; v += gridDim.x)
    direct_pass_vector<T>(X, es, vs, n, ts, cp, cm, M, cmass, Y, accumulate, v, xs);
}

// grouped: item (entry, vector); the generator is staged per item
template <typename T>
__global__ void g_direct_pass_kernel(const GDirectPass<T>* __restrict__ ent,
                                     const GItem* __restrict__ items, int nitems, int max_n,
                                     GGate gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ts = reinterpret_cast<T*>(smem_raw);
  T* xs = ts + (max_n + 1);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GItem g = items[it];
    const GDirectPass<T> e = ent[g.e];
    if (!gate_open(gate, e.prob, e.want)) continue;
    for (int k = threadIdx.x; k <= e.n; k += blockDim.x) ts[k] = e.t[k];
    direct_pass_vector<T>(e.X, e.es, e.vs, e.n, ts, e.cp, e.cm, e.M, T(e.cmass), e.Y,
                          e.accumulate, g.unit, xs);
  }
}

template <typename T>
cudaError_t launch_g_direct_pass(const GDirectPass<T>* ent, const GItem* items, int nitems,
                                 int max_n, GGate gate, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = (size_t)(2 * max_n + 1) * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_max_smem((const void*)g_direct_pass_kernel<T>);
    if (e != cudaSuccess) return e;
  }
  int grid = nitems < 152 * 8 ? nitems : 152 * 8;
  g_direct_pass_kernel<T><<<grid, 128, smem, st>>>(ent, items, nitems, max_n, gate);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_direct_pass(const T* X, int es, int vs, int nvec, int n, const T* t,
                               const T* cp, const T* cm, const T* M, double cmass, T* Y,
                               int accumulate, cudaStream_t st) {
  const size_t smem = (size_t)(2 * n + 1) * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(direct_pass_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  int grid = nvec < 1216 ? nvec : 1216;
  direct_pass_kernel<T><<<grid, 128, smem, st>>>(X, es, vs, nvec, n, t, cp, cm, M, T(cmass), Y,
                                                 accumulate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- instantiations
template cudaError_t launch_fft_pass<double, double, double>(
    const double*, int, int, int, int, int, const cx<double>*, const cx<double>*,
    const cx<double>*, const double*, const double*, const double*, double, double*, int,
    cudaStream_t, cx<double>*, size_t);
template cudaError_t launch_fft_pass<float, float, float>(const float*, int, int, int, int, int,
                                                          const cx<float>*, const cx<float>*,
                                                          const cx<float>*, const float*,
                                                          const float*, const float*, double,
                                                          float*, int, cudaStream_t, cx<float>*,
                                                          size_t);
template cudaError_t launch_fft_pass<double, float, float>(
    const double*, int, int, int, int, int, const cx<float>*, const cx<float>*, const cx<float>*,
    const float*, const float*, const double*, double, double*, int, cudaStream_t, cx<float>*,
    size_t);
template cudaError_t launch_fft_pass<double, df, df>(const double*, int, int, int, int, int,
                                                     const cx<df>*, const cx<df>*,
                                                     const cx<df>*, const df*, const df*,
                                                     const double*, double, double*, int,
                                                     cudaStream_t, cx<df>*, size_t);
template cudaError_t launch_fft_pass2<float, float, float>(const FftPass<float, float, float>&,
                                                           const FftPass<float, float, float>&,
                                                           int, cudaStream_t, cx<float>*, size_t);
template cudaError_t launch_fft_pass2<double, double, double>(
    const FftPass<double, double, double>&, const FftPass<double, double, double>&, int,
    cudaStream_t, cx<double>*, size_t);
template cudaError_t launch_fft_pass2<df, float, float>(const FftPass<df, float, float>&,
                                                       const FftPass<df, float, float>&, int,
                                                       cudaStream_t, cx<float>*, size_t);
template cudaError_t launch_fft_pass2<df, df, df>(const FftPass<df, df, df>&,
                                                 const FftPass<df, df, df>&, int, cudaStream_t,
                                                 cx<df>*, size_t);
template cudaError_t launch_fft_pass2<double, float, float>(const FftPass<double, float, float>&,
                                                            const FftPass<double, float, float>&,
                                                            int, cudaStream_t, cx<float>*, size_t);
template cudaError_t launch_fft_pass2<double, df, df>(const FftPass<double, df, df>&,
                                                     const FftPass<double, df, df>&, int,
                                                     cudaStream_t, cx<df>*, size_t);
template cudaError_t launch_fft_pass<df, float, float>(
    const df*, int, int, int, int, int, const cx<float>*, const cx<float>*, const cx<float>*,
    const float*, const float*, const df*, double, df*, int, cudaStream_t, cx<float>*, size_t);
template cudaError_t launch_fft_pass<df, df, df>(const df*, int, int, int, int, int,
                                                     const cx<df>*, const cx<df>*,
                                                     const cx<df>*, const df*, const df*,
                                                     const df*, double, df*, int,
                                                     cudaStream_t, cx<df>*, size_t);
template cudaError_t launch_build_spectra<df>(const double*, int, int, double, cx<df>*, cx<df>*,
                                              cx<df>*, cudaStream_t, cx<double>*);
template cudaError_t launch_build_spectra<double>(const double*, int, int, double, cx<double>*,
                                                  cx<double>*, cx<double>*, cudaStream_t,
                                                  cx<double>*);
template cudaError_t launch_build_spectra<float>(const double*, int, int, double, cx<float>*,
                                                 cx<float>*, cx<float>*, cudaStream_t,
                                                 cx<double>*);
template cudaError_t launch_g_fft_pass<float, float, float>(const GFftPass<float, float, float>*,
                                                            const GItem*, int, int, GGate,
                                                            cudaStream_t);
template cudaError_t launch_g_fft_pass<double, float, float>(
    const GFftPass<double, float, float>*, const GItem*, int, int, GGate, cudaStream_t);
template cudaError_t launch_g_fft_pass<double, df, df>(const GFftPass<double, df, df>*,
                                                       const GItem*, int, int, GGate,
                                                       cudaStream_t);
template cudaError_t launch_g_direct_pass<float>(const GDirectPass<float>*, const GItem*, int,
                                                 int, GGate, cudaStream_t);
template cudaError_t launch_direct_pass<double>(const double*, int, int, int, int, const double*,
                                                const double*, const double*, const double*,
                                                double, double*, int, cudaStream_t);
template cudaError_t launch_direct_pass<float>(const float*, int, int, int, int, const float*,
                                               const float*, const float*, const float*, double,
                                               float*, int, cudaStream_t);

}  // namespace fde

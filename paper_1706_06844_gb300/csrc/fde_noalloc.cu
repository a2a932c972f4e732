// fde_apply_noalloc: y = M x without a handle and without any device
// allocation, for callers that cannot allocate GPU memory -- code running
// while another runtime owns the device heap (a fixed memory pool or a
// framework allocator that forbids driver allocations), or an embedding that
// must not change the process's device-memory footprint after start-up.
// Such callers cannot call fde_create (which allocates the solver's workspace),
// so this entry point computes the FP64 operator apply from the parameters
// and coefficient arrays alone.
//
// Its working data -- WSGD weights, Toeplitz generators, the spectra of the
// circulant embeddings and the FFT twiddles of both axes -- lives in one
// file-scope device array (NOALLOC_BYTES, about 450 KB), which every GPU that
// loads the library holds until the process exits.  Every call shares that
// array and rewrites all of it before use; two calls that overlap on the GPU
// (different streams, or different host threads) race on it.  The array's
// device address is looked up once per device and kept, so the device must
// not be reset (cudaDeviceReset) between calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "../../include/fde.h"

namespace fde {
void set_global_error(const char* msg);
}

namespace {

using fde::cx;

constexpr int kMaxN = 2048;                 // per axis: FFT length L <= 4096
constexpr int kMaxL = 4096;
constexpr size_t kVec = ((kMaxN + 2) * sizeof(double) + 255) / 256 * 256;  // weights, generators
constexpr size_t kSpec = (size_t)kMaxL * sizeof(cx<double>);               // spectra, twiddles
constexpr size_t NOALLOC_BYTES = 4 * kVec + 6 * kSpec;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// device address of g_noalloc_scratch per device, fetched once per device
constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {nullptr};
std::mutex g_mu;

int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    fde::set_global_error("fde_apply_noalloc: no current CUDA device");
    return FDE_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      char buf[256];
      snprintf(buf, sizeof(buf), "fde_apply_noalloc: cudaGetSymbolAddress failed: %s",
               cudaGetErrorString(e));
      fde::set_global_error(buf);
      return FDE_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return FDE_OK;
}

int ceil_log2(long v) {
  int l = 0;
  while ((1L << l) < v) ++l;
  return l;
}

int fail(int code, const char* msg) {
  fde::set_global_error(msg);
  return code;
}

// true if the byte ranges [a, a + na) and [b, b + nb) share a byte
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return a0 < b0 + nb && b0 < a0 + na;
}

}  // namespace

extern "C" int fde_apply_noalloc(const fde_params* p, const double* dp, const double* dm,
                                 const double* ep, const double* em, const double* x, double* y,
                                 void* stream) {
  if (!p) return fail(FDE_ERR_ARG, "fde_apply_noalloc: null params");
  if (!dp || !dm || !ep || !em || !x || !y || x == y)
    return fail(FDE_ERR_ARG, "fde_apply_noalloc: null or aliased pointer");
  if (!(p->alpha > 1.0 && p->alpha < 2.0) || !(p->beta > 1.0 && p->beta < 2.0))
    return fail(FDE_ERR_ARG, "fde_apply_noalloc: alpha and beta must lie in (1, 2)");
  if ((p->qx != 0 && p->qx != -1) || (p->qy != 0 && p->qy != -1))
    return fail(FDE_ERR_ARG, "fde_apply_noalloc: q must be 0 or -1");
  if (!(p->b1 > p->a1) || !(p->b2 > p->a2) || !(p->dt > 0.0))
    return fail(FDE_ERR_ARG, "fde_apply_noalloc: empty domain or non-positive dt");
  if (p->n1 < 3 || p->n2 < 3) return fail(FDE_ERR_ARG, "fde_apply_noalloc: n1, n2 must be >= 3");
  if (p->n1 > kMaxN || p->n2 > kMaxN) {
    char buf[200];
    snprintf(buf, sizeof(buf),
             "fde_apply_noalloc: grid %d x %d exceeds the fixed scratch limit of %d points per "
             "axis (use fde_create / fde_apply)",
             p->n1, p->n2, kMaxN);
    return fail(FDE_ERR_ARG, buf);
  }
  // y is written while other CTAs still read x and the coefficients: no
  // byte of y may belong to any input
  const size_t nbytes = (size_t)p->n1 * p->n2 * sizeof(double);
  for (const double* in : {x, dp, dm, ep, em})
    if (overlaps(y, nbytes, in, nbytes))
      return fail(FDE_ERR_ARG, "fde_apply_noalloc: y overlaps an input array");
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != FDE_OK) return rc;
  unsigned char* s = static_cast<unsigned char*>(base);
  double* wx = reinterpret_cast<double*>(s);
  double* wy = reinterpret_cast<double*>(s + kVec);
  double* tx = reinterpret_cast<double*>(s + 2 * kVec);
  double* ty = reinterpret_cast<double*>(s + 3 * kVec);
  cx<double>* S1x = reinterpret_cast<cx<double>*>(s + 4 * kVec);
  cx<double>* S2x = reinterpret_cast<cx<double>*>(s + 4 * kVec + kSpec);
  cx<double>* S1y = reinterpret_cast<cx<double>*>(s + 4 * kVec + 2 * kSpec);
  cx<double>* S2y = reinterpret_cast<cx<double>*>(s + 4 * kVec + 3 * kSpec);
  cx<double>* twx = reinterpret_cast<cx<double>*>(s + 4 * kVec + 4 * kSpec);
  cx<double>* twy = reinterpret_cast<cx<double>*>(s + 4 * kVec + 5 * kSpec);

  const int n1 = p->n1, n2 = p->n2;
  const double hx = (p->b1 - p->a1) / (n1 + 1), hy = (p->b2 - p->a2) / (n2 + 1);
  const double r = p->dt / (2.0 * std::pow(hx, p->alpha));  // Eq. (system)
  const double sy = p->dt / (2.0 * std::pow(hy, p->beta));
  const double c = 1.0 / r, sigma = sy / r;
  const int logLx = ceil_log2(2L * n1 - 1), logLy = ceil_log2(2L * n2 - 1);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
#define NA_CHK(call)                                                              \
  do {                                                                            \
    e = (call);                                                                   \
    if (e != cudaSuccess) {                                                       \
      char buf[256];                                                              \
      snprintf(buf, sizeof(buf), "fde_apply_noalloc: %s", cudaGetErrorString(e)); \
      return fail(FDE_ERR_CUDA, buf);                                             \
    }                                                                             \
  } while (0)
  // weights (Eq. gk, w) and generators t_d = -w_{d+1} (Eq. AN); sigma is folded
  // into the y-axis spectra so the coefficient arrays are used as given
  NA_CHK(fde::launch_wsgd_weights(p->alpha, p->qx, n1 + 1, wx, st));
  NA_CHK(fde::launch_wsgd_weights(p->beta, p->qy, n2 + 1, wy, st));
  NA_CHK(fde::launch_generator_from_weights(wx, n1, 1.0, tx, st));
  NA_CHK(fde::launch_generator_from_weights(wy, n2, 1.0, ty, st));
  NA_CHK(fde::launch_build_spectra<double>(tx, n1, logLx, 1.0, S1x, S2x, twx, st));
  NA_CHK(fde::launch_build_spectra<double>(ty, n2, logLy, sigma, S1y, S2y, twy, st));
  // y = c x + D+ (x A_x^T) + D- (x A_x)   (rows), then += sigma [E+ A_y x + E- A_y^T x]
  NA_CHK((fde::launch_fft_pass<double, double, double>(x, 1, n1, n2, n1, logLx, S1x, S2x, twx, dp,
                                                       dm, x, c, y, 0, st)));
  NA_CHK((fde::launch_fft_pass<double, double, double>(x, n1, 1, n1, n2, logLy, S1y, S2y, twy, ep,
                                                       em, nullptr, 0.0, y, 1, st)));
#undef NA_CHK
  return FDE_OK;
}

// Tensor-core (tcgen05) evaluation of the Toeplitz products of one multigrid
// level: the four dense products X A_x^T, X A_x, A_y X, A_y^T X of Eq. (AxAy)
// as BF16/FP16 GEMMs with FP32 accumulation in tensor memory, the coefficient
// scaling and the mass term fused in the epilogue.
#pragma once
#include <cuda_runtime.h>

namespace fde {
namespace tc {

constexpr int kBF16 = 0;
constexpr int kFP16 = 1;
constexpr int kBF16X3 = 2;      // hi/lo BF16 split, three products
constexpr int kMinGemmN = 127;  // smaller levels stay on CUDA cores
// FDE_PATH_AUTO picks the tensor path only from this size up: one CTA owns a
// 128 x 256 output tile, so n = 1023 launches 32 CTAs on 152 SMs and the FFT
// path is faster there; n = 2047 launches 128.
constexpr int kAutoGemmN = 1536;

struct ToeplitzGemmLevel {
  int n1 = 0, n2 = 0, prec = kBF16;
  bool built = false;
  int ld = 0;            // pitch (elements) of the 16-bit operand copies
  void* xa = nullptr;     // 16-bit copy of the x-product operand, n2 rows x ld
  void* xa_lo = nullptr;  // its low part (split precision)
  void* xb = nullptr;     // 16-bit copy of the y-product operand (structured-Galerkin levels)
  void* xb_lo = nullptr;
  void* maps = nullptr;   // tensor maps, generator copies, error flag
  int splits = 1;         // CTAs sharing a tile's K range (small levels)
  float* ws = nullptr;    // their partial products: 2 * splits * n1 * n2
};

// returns 0 on success
int level_create(ToeplitzGemmLevel* L, int n1, int n2, int prec, bool mass);
int level_setup(ToeplitzGemmLevel* L, const double* tx, const double* ty, cudaStream_t st);
// kx = cm * M + dp (.) (X A_x^T) + dm (.) (X A_x) + ep (.) (A_y Y) + em (.) (A_y^T Y)
// with X = xin_x, Y = xin_y (FP32, n2 x n1, unpadded); two kernel launches plus
// one or two operand-packing launches
int level_products(ToeplitzGemmLevel* L, const float* xin_x, const float* xin_y, const float* M,
                   double cm, const float* dp, const float* dm, const float* ep, const float* em,
                   float* kx, cudaStream_t st);
// the same in its three steps, for callers that time the launches one by one:
// level_pack writes the 16-bit operand copies of xin_x (and xin_y on
// structured-Galerkin levels); level_gemm launches one direction, dir 0:
// kx = cm * M + c0 (.) (X A_x^T) + c1 (.) (X A_x), dir 1: kx += c0 (.) (A_y Y)
// + c1 (.) (A_y^T Y) (M ignored)
int level_pack(ToeplitzGemmLevel* L, const float* xin_x, const float* xin_y, cudaStream_t st);
int level_gemm(ToeplitzGemmLevel* L, int dir, const float* M, double cm, const float* c0,
               const float* c1, float* kx, cudaStream_t st);
// after both directions: with split K, kx = cm * M + the partial products of
// every split (fixed order); nothing otherwise
int level_finish(ToeplitzGemmLevel* L, const float* M, double cm, float* kx, cudaStream_t st);
// 1 if a capped wait of the level's kernels gave up since the last call (the flag
// is then cleared), 0 if not, -1 if the flag could not be read; syncs `st`
int level_error(ToeplitzGemmLevel* L, cudaStream_t st);
// enqueue on `st` one run of the kernels' bounded wait on a barrier that is
// completed (complete = 1) or never completed (complete = 0: the wait gives up
// after 20 ms and raises the level's error flag); 0 on success, -1 if the level
// is not built, 31 on a launch error
int level_wait_selftest(ToeplitzGemmLevel* L, int complete, cudaStream_t st);
void level_destroy(ToeplitzGemmLevel* L);

}  // namespace tc
}  // namespace fde

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
constexpr int kMinGemmN = 127;  // smaller levels stay on CUDA cores

struct ToeplitzGemmLevel {
  int n1 = 0, n2 = 0, prec = kBF16;
  bool built = false;
  int ld = 0;            // pitch (elements) of the 16-bit operand copies
  void* xa = nullptr;    // 16-bit copy of the x-pass operand, n2 rows x ld
  void* xb = nullptr;    // 16-bit copy of the y-pass operand, n2 rows x ld
  void* bank = nullptr;  // Toeplitz tile banks (x lower, x upper, y lower, y upper)
  int tiles_x = 0, tiles_y = 0;
  void* maps = nullptr;  // device copy of the tensor maps
};

// returns 0 on success
int level_create(ToeplitzGemmLevel* L, int n1, int n2, int prec, bool mass);
int level_setup(ToeplitzGemmLevel* L, const double* tx, const double* ty, cudaStream_t st);
// kx = cm * M + dp (.) (X A_x^T) + dm (.) (X A_x) + ep (.) (A_y Y) + em (.) (A_y^T Y)
// with X = xin_x, Y = xin_y (FP32, n2 x n1, unpadded)
int level_products(ToeplitzGemmLevel* L, const float* xin_x, const float* xin_y, const float* M,
                   double cm, const float* dp, const float* dm, const float* ep, const float* em,
                   float* kx, cudaStream_t st);
// device error flag of the level's kernels (1 = a bounded wait gave up); reading it synchronises
int level_error(ToeplitzGemmLevel* L);
void level_destroy(ToeplitzGemmLevel* L);

}  // namespace tc
}  // namespace fde

// placeholder until the tcgen05 kernel lands
#include "tc_gemm.h"
namespace fde {
namespace tc {
int level_create(ToeplitzGemmLevel*, int, int, int, bool) { return -1; }
int level_setup(ToeplitzGemmLevel*, const double*, const double*, cudaStream_t) { return -1; }
int level_products(ToeplitzGemmLevel*, const float*, const float*, const float*, double,
                   const float*, const float*, const float*, const float*, float*, cudaStream_t) {
  return -1;
}
void level_destroy(ToeplitzGemmLevel*) {}
}  // namespace tc
}  // namespace fde

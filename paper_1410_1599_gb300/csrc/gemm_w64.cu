// gemm_w64.cu -- elementwise and GEMM kernels, 64-word (2048-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_GEMM(64)
}  // namespace mpg

// gemm_w8.cu -- elementwise and GEMM kernels, 8-word (256-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_GEMM(8)
}  // namespace mpg

// gemm_w16.cu -- elementwise and GEMM kernels, 16-word (512-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_GEMM(16)
}  // namespace mpg

// gemm_w272.cu -- elementwise and GEMM kernels, 272-word (8704-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_GEMM(BIG_W)
}  // namespace mpg

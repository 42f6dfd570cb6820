// gemm_w4.cu -- elementwise and GEMM kernels, 4-word (128-bit) capacity class.
#include "mp_warp.cuh"

namespace mpg {
MPG_INSTANTIATE_GEMM(4)
MPG_INSTANTIATE_WARP(4)
}  // namespace mpg

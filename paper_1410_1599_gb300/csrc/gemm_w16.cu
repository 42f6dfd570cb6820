// gemm_w16.cu -- elementwise and GEMM kernels, 16-word (512-bit) capacity class.
#include "mp_warp.cuh"

namespace mpg {
MPG_INSTANTIATE_GEMM(16)
MPG_INSTANTIATE_WARP(16)
}  // namespace mpg

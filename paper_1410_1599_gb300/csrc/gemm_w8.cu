// gemm_w8.cu -- elementwise and GEMM kernels, 8-word (256-bit) capacity class.
#include "mp_warp.cuh"

namespace mpg {
MPG_INSTANTIATE_GEMM(8)
MPG_INSTANTIATE_WARP(8)
}  // namespace mpg

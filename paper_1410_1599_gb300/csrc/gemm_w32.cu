// gemm_w32.cu -- elementwise and GEMM kernels, 32-word (1024-bit) capacity class.
#include "mp_warp.cuh"

namespace mpg {
MPG_INSTANTIATE_GEMM(32)
MPG_INSTANTIATE_WARP(32)
}  // namespace mpg

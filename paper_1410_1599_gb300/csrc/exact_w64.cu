// exact_w64.cu -- exact-dot GEMM kernel, 64-word (2048-bit) capacity class.
#include "mp_exact.cuh"

namespace mpg {
MPG_INSTANTIATE_EXACT(64)
}  // namespace mpg

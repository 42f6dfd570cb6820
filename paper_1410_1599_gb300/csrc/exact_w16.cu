// exact_w16.cu -- exact-dot GEMM kernel, 16-word (512-bit) capacity class.
#include "mp_exact.cuh"

namespace mpg {
MPG_INSTANTIATE_EXACT(16)
}  // namespace mpg

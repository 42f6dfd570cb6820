// exact_w4.cu -- exact-dot GEMM kernel, 4-word (128-bit) capacity class.
#include "mp_exact.cuh"

namespace mpg {
MPG_INSTANTIATE_EXACT(4)
}  // namespace mpg

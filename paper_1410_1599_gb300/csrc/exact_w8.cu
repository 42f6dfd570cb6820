// exact_w8.cu -- exact-dot GEMM kernel, 8-word (256-bit) capacity class.
#include "mp_exact.cuh"

namespace mpg {
MPG_INSTANTIATE_EXACT(8)
}  // namespace mpg

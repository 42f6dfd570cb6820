// exact_w32.cu -- exact-dot GEMM kernel, 32-word (1024-bit) capacity class.
#include "mp_exact.cuh"

namespace mpg {
MPG_INSTANTIATE_EXACT(32)
}  // namespace mpg

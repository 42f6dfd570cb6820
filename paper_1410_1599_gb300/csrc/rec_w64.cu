// rec_w64.cu -- Strassen/Winograd recursion kernels, 64-word (2048-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_REC(64)
}  // namespace mpg

// rec_w32.cu -- Strassen/Winograd recursion kernels, 32-word (1024-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_REC(32)
}  // namespace mpg

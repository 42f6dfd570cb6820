// rec_w8.cu -- Strassen/Winograd recursion kernels, 8-word (256-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_REC(8)
}  // namespace mpg

// rec_w4.cu -- Strassen/Winograd recursion kernels, 4-word (128-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_REC(4)
}  // namespace mpg

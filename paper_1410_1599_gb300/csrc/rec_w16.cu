// rec_w16.cu -- Strassen/Winograd recursion kernels, 16-word (512-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_REC(16)
}  // namespace mpg

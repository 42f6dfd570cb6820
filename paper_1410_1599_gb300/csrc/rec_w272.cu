// rec_w272.cu -- Strassen/Winograd recursion kernels, 272-word (8704-bit) capacity class.
#include "mp_kernels.cuh"

namespace mpg {
MPG_INSTANTIATE_REC(BIG_W)
}  // namespace mpg

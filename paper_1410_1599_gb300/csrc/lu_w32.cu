// lu_w32.cu -- LU kernels, 32-word (1024-bit) capacity class.
#include "mp_lu.cuh"

namespace mpg {
MPG_INSTANTIATE_LU(32)
}  // namespace mpg

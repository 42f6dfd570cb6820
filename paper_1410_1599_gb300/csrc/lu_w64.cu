// lu_w64.cu -- LU kernels, 64-word (2048-bit) capacity class.
#include "mp_lu.cuh"

namespace mpg {
MPG_INSTANTIATE_LU(64)
}  // namespace mpg

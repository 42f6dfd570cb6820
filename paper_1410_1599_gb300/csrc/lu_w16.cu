// lu_w16.cu -- LU kernels, 16-word (512-bit) capacity class.
#include "mp_lu.cuh"

namespace mpg {
MPG_INSTANTIATE_LU(16)
}  // namespace mpg

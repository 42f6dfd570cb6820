// lu_w8.cu -- LU kernels, 8-word (256-bit) capacity class.
#include "mp_lu.cuh"

namespace mpg {
MPG_INSTANTIATE_LU(8)
}  // namespace mpg

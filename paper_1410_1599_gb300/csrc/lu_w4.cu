// lu_w4.cu -- LU kernels, 4-word (128-bit) capacity class.
#include "mp_lu.cuh"

namespace mpg {
MPG_INSTANTIATE_LU(4)
}  // namespace mpg

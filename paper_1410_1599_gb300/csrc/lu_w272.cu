// lu_w272.cu -- LU kernels, 272-word (8704-bit) capacity class.
#include "mp_lu.cuh"

namespace mpg {
MPG_INSTANTIATE_LU(BIG_W)
}  // namespace mpg

// split_w16.cu -- split-form alignment and recombination kernels, 16-word class.
#include "mp_split.cuh"

namespace mpg {
MPG_INSTANTIATE_SPLIT(16)
}  // namespace mpg

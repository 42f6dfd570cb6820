// split_w32.cu -- split-form alignment and recombination kernels, 32-word class.
#include "mp_split.cuh"

namespace mpg {
MPG_INSTANTIATE_SPLIT(32)
}  // namespace mpg

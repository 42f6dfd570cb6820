// split_w64.cu -- split-form alignment and recombination kernels, 64-word class.
#include "mp_split.cuh"

namespace mpg {
MPG_INSTANTIATE_SPLIT(64)
}  // namespace mpg

// split_w8.cu -- split-form alignment and recombination kernels, 8-word class.
#include "mp_split.cuh"

namespace mpg {
MPG_INSTANTIATE_SPLIT(8)
}  // namespace mpg

// split_w4.cu -- split-form alignment and recombination kernels, 4-word class.
#include "mp_split.cuh"

namespace mpg {
MPG_INSTANTIATE_SPLIT(4)
}  // namespace mpg

// Explicit instantiations of the row-pass and spectrum kernels for FFT lengths 3072.
#include "sf_kernels.cuh"
namespace sf {
SF_INSTANTIATE_LENGTH(3072)
}  // namespace sf

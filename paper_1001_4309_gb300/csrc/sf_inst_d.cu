// Explicit instantiations of the row-pass and spectrum kernels for FFT lengths 8192.
#include "sf_kernels.cuh"
namespace sf {
SF_INSTANTIATE_LENGTH(8192)
}  // namespace sf

// Explicit instantiations of the row-pass and spectrum kernels for FFT lengths 4096.
#include "sf_kernels.cuh"
namespace sf {
SF_INSTANTIATE_LENGTH(4096)
}  // namespace sf

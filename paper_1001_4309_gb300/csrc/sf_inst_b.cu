// Explicit instantiations of the row-pass and spectrum kernels for FFT lengths 1024 2048.
#include "sf_kernels.cuh"
namespace sf {
SF_INSTANTIATE_LENGTH(1024)
SF_INSTANTIATE_LENGTH(2048)
}  // namespace sf

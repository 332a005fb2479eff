// Explicit instantiations of the row-pass and spectrum kernels for FFT lengths 1536 2304.
#include "sf_kernels.cuh"
namespace sf {
SF_INSTANTIATE_LENGTH(1536)
SF_INSTANTIATE_LENGTH(2304)
}  // namespace sf

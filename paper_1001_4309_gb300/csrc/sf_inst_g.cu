// Explicit instantiations of the row-pass and spectrum kernels for FFT lengths 4608 6144.
#include "sf_kernels.cuh"
namespace sf {
SF_INSTANTIATE_LENGTH(4608)
SF_INSTANTIATE_LENGTH(6144)
}  // namespace sf

// Explicit instantiations of the row-pass and spectrum kernels for FFT lengths 64 128 256 512.
#include "sf_kernels.cuh"
namespace sf {
SF_INSTANTIATE_LENGTH(64)
SF_INSTANTIATE_LENGTH(128)
SF_INSTANTIATE_LENGTH(256)
SF_INSTANTIATE_LENGTH(512)
}  // namespace sf

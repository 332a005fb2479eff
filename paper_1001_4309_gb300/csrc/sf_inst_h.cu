// Explicit instantiations of the row pass's alternative CTA sizes (the
// autotuner's rows-per-CTA axis) for FFT lengths 1024, 2048 and 4096.
#include "sf_kernels.cuh"
namespace sf {
static_assert(pass_cta_variant(1024, 1) == 128 && pass_cta_variant(1024, 2) == 512, "1024 variants");
static_assert(pass_cta_variant(2048, 1) == 128 && pass_cta_variant(2048, 2) == 512, "2048 variants");
static_assert(pass_cta_variant(4096, 1) == 256 && pass_cta_variant(4096, 2) == 0, "4096 variants");
SF_INSTANTIATE_VARIANT(1024, 128)
SF_INSTANTIATE_VARIANT(1024, 512)
SF_INSTANTIATE_VARIANT(2048, 128)
SF_INSTANTIATE_VARIANT(2048, 512)
SF_INSTANTIATE_VARIANT(4096, 256)
}  // namespace sf

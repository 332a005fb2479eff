// sf_batch_one.cu -- the persistent batch kernel specialised to one
// power-of-two FFT length on every pass, with the pruned network (every pass
// has n0, n1 <= L / 2, the paper's 2N padding).  Same work loop and
// dependencies as the general kernel (sf_batch.cuh); the kernel holds only
// this length's x and y tiles, so its code stays small and no tile
// dispatches on the length.
#include "sf_batch.cuh"

namespace sf {
namespace {

template <int KIND_X, int L>
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_one(const __grid_constant__ BatchArgs a) {
  extern __shared__ float2 smem[];
  using Sh = BatchShape<L>;
  static_assert(Sh::THREADS == kBatchThreads, "one-length batch tiles fill the batch CTA");
  const float4* tw = a.tw[fft_length_slot_of<L>()];
  batch_loop(a, [&](const PassDesc& d, int phase, int, int tile) {
    if (phase == 0) row_tile<L, KIND_X, false, false, batch_cta(L), true>(d, tile * Sh::G, smem, tw);
    else row_tile<L, PASS_Y, true, false, batch_cta(L), true>(d, tile * Sh::G, smem, tw);
  });
}

template <int L>
const void* one_kernel(PassKind kind_x) {
  return kind_x == PASS_X_CPLX ? (const void*)k_batch_one<PASS_X_CPLX, L> : (const void*)k_batch_one<PASS_X_REAL, L>;
}

}  // namespace

const void* batch_kernel_one(PassKind kind_x, int L) {
  switch (L) {
    case 512: return one_kernel<512>(kind_x);
    case 1024: return one_kernel<1024>(kind_x);
    case 2048: return one_kernel<2048>(kind_x);
    case 4096: return one_kernel<4096>(kind_x);
    default: return nullptr;
  }
}

size_t batch_smem_bytes_one(int L) {
  switch (L) {
    case 512: return BatchShape<512>::SMEM;
    case 1024: return BatchShape<1024>::SMEM;
    case 2048: return BatchShape<2048>::SMEM;
    case 4096: return BatchShape<4096>::SMEM;
    default: return 0;
  }
}

}  // namespace sf

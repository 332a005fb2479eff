// sf_batch.cu -- the persistent batch kernel for any mix of FFT lengths
// (the work loop and its dependencies are in sf_batch.cuh): each row tile
// dispatches on its group's length.
#include "sf_batch.cuh"

namespace sf {
namespace {

// One tile of a length with a factor 3 (24 values per thread).  Not inlined:
// under the batch kernel's 128-register budget these tiles spill a little,
// and a separate function keeps that spill code out of the power-of-two paths.
template <int LL, int KIND_X>
__device__ __noinline__ void mixed_tile(const PassDesc& d, int phase, int tile, float2* smem, const float4* tw) {
  using Sh = BatchShape<LL>;
  constexpr bool spare = Sh::THREADS < kBatchThreads;
  if (phase == 0) row_tile<LL, KIND_X, false, spare, batch_cta(LL)>(d, tile * Sh::G, smem, tw);
  else row_tile<LL, PASS_Y, true, spare, batch_cta(LL)>(d, tile * Sh::G, smem, tw);
}

template <int KIND_X>
__device__ __forceinline__ void run_item(const PassDesc& d, int phase, int L, int tile, float2* smem,
                                         const float4* const* tw) {
  // a tile of G T <= kBatchThreads threads; the rest of the CTA idles through it
#define SF_BATCH_CASE(LL)                                                                              \
  static_assert(BatchShape<LL>::THREADS <= kBatchThreads, "batch tiles must fit the batch CTA");       \
  case LL: {                                                                                           \
    constexpr bool spare = BatchShape<LL>::THREADS < kBatchThreads;                                    \
    const float4* t = tw[fft_length_slot_of<LL>()];                                                    \
    if (phase == 0) row_tile<LL, KIND_X, false, spare, batch_cta(LL)>(d, tile * BatchShape<LL>::G, smem, t); \
    else row_tile<LL, PASS_Y, true, spare, batch_cta(LL)>(d, tile * BatchShape<LL>::G, smem, t);     \
    break;                                                                                             \
  }
#define SF_BATCH_MIXED_CASE(LL)                                                                        \
  static_assert(BatchShape<LL>::THREADS <= kBatchThreads, "batch tiles must fit the batch CTA");       \
  case LL: mixed_tile<LL, KIND_X>(d, phase, tile, smem, tw[fft_length_slot_of<LL>()]); break;
  switch (L) {
    SF_BATCH_CASE(64)
    SF_BATCH_CASE(128)
    SF_BATCH_CASE(256)
    SF_BATCH_CASE(512)
    SF_BATCH_CASE(1024)
    SF_BATCH_MIXED_CASE(1536)
    SF_BATCH_CASE(2048)
    SF_BATCH_MIXED_CASE(2304)
    SF_BATCH_MIXED_CASE(3072)
    SF_BATCH_CASE(4096)
    SF_BATCH_MIXED_CASE(4608)
    SF_BATCH_MIXED_CASE(6144)
    default: break;
  }
#undef SF_BATCH_CASE
#undef SF_BATCH_MIXED_CASE
}

template <int KIND_X>
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch(const __grid_constant__ BatchArgs a) {
  extern __shared__ float2 smem[];
  batch_loop(a, [&](const PassDesc& d, int phase, int L, int tile) { run_item<KIND_X>(d, phase, L, tile, smem, a.tw); });
}

}  // namespace

bool batch_length_supported(int L) { return fft_length_supported(L) && L <= 6144; }

int batch_tile_rows(int L) {
  switch (L) {
#define SF_BATCH_ROWS(LL) case LL: return BatchShape<LL>::G;
    SF_BATCH_ROWS(64) SF_BATCH_ROWS(128) SF_BATCH_ROWS(256) SF_BATCH_ROWS(512) SF_BATCH_ROWS(1024)
    SF_BATCH_ROWS(1536) SF_BATCH_ROWS(2048) SF_BATCH_ROWS(2304) SF_BATCH_ROWS(3072) SF_BATCH_ROWS(4096)
    SF_BATCH_ROWS(4608) SF_BATCH_ROWS(6144)
#undef SF_BATCH_ROWS
    default: return 0;
  }
}

// Tiles per work item: items carry at least 8 rows so the dequeue, dependency
// check and completion count are amortised over several tiles.
int batch_item_tiles(int L) {
  const int g = batch_tile_rows(L);
  return g >= 8 ? 1 : 8 / g;
}

size_t batch_smem_bytes() {
  size_t m = 0;
  for (size_t b : {BatchShape<64>::SMEM, BatchShape<128>::SMEM, BatchShape<256>::SMEM, BatchShape<512>::SMEM,
                   BatchShape<1024>::SMEM, BatchShape<1536>::SMEM, BatchShape<2048>::SMEM, BatchShape<2304>::SMEM,
                   BatchShape<3072>::SMEM, BatchShape<4096>::SMEM, BatchShape<4608>::SMEM, BatchShape<6144>::SMEM})
    m = std::max(m, b);
  return m;
}

const void* batch_kernel(PassKind kind_x) {
  return kind_x == PASS_X_CPLX ? (const void*)k_batch<PASS_X_CPLX> : (const void*)k_batch<PASS_X_REAL>;
}

}  // namespace sf

// sf_batch.cu -- persistent kernel for a batch of ragged views over a stream
// of holograms (the paper's real-time loop, Section 2.2, repeated over frames,
// with every view and frame in one launch).
//
// Work items are (hologram h, group g, tile): group g < V is the x pass of
// view g, group V + v the y pass of view v; within a hologram all x items
// precede all y items, and holograms follow one another.  A CTA takes the
// next item from a global counter, so items start in index order.
// Dependencies, each a wait on a per-(hologram, group) completion counter:
//   - a y item of (h, v) waits until every x tile of (h, v) is done;
//   - an x item of (h, v), h >= 2, waits until every y tile of (h - 2, v) is
//     done, because the x pass of h writes the intermediate slot h % 2 that
//     the y pass of h - 2 read.
// Every awaited item has a smaller index, was therefore taken earlier by a
// running CTA, and itself only waits on smaller indices: the lowest
// unfinished item never waits, so the launch always progresses, whatever
// the number of resident CTAs.  (A CTA takes its next item while working on
// the current one; the next one is larger, so the argument still holds.)  Waits are still bounded (spin_limit sleeps);
// on expiry a CTA sets the error word and leaves, which unblocks nobody but
// ends every other wait by its own limit, so the launch always returns.
#include "sf_kernels.cuh"

namespace sf {
namespace {

// Row tiles of the batch kernel: the pass kernel's tile shape, capped at the
// batch CTA size.
constexpr int batch_cta(int L) { return pass_cta_target(L) < kBatchThreads ? pass_cta_target(L) : kBatchThreads; }
template <int L>
using BatchShape = PassShape<L, batch_cta(L)>;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

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
  __shared__ int s_item, s_group, s_stop;
  if (threadIdx.x == 0) s_item = atomicAdd(a.next, 1);
  for (;;) {
    __syncthreads();
    int nxt = 0;
    if (threadIdx.x == 0) {
      const int item = s_item;
      // Take the following item now; its value is only needed at the end of
      // this one, so the round trip overlaps the work (items stay in order).
      nxt = atomicAdd(a.next, 1);
      int stop = item >= a.total_items || ld_acquire(a.error) != 0;
      int g = 0;
      if (!stop) {
        const int h = item / a.items_per_holo, r = item - h * a.items_per_holo;
        int lo = 0, hi = a.n_groups - 1;  // last group with first_item <= r
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (a.groups[mid].first_item <= r) lo = mid; else hi = mid - 1;
        }
        g = lo;
        // dependency of this item, if any
        const int* cnt = nullptr;
        int target = 0;
        if (g >= a.n_views) {
          cnt = a.done + (size_t)h * a.n_groups + (g - a.n_views);
          target = a.groups[g - a.n_views].items;
        } else if (h >= 2) {
          cnt = a.done + (size_t)(h - 2) * a.n_groups + (g + a.n_views);
          target = a.groups[g + a.n_views].items;
        }
        if (g == a.poison_group) target = 0x7fffffff;  // host-injected never-satisfied dependency (tests)
        if (cnt) {
          long long spins = 0;
          while (ld_acquire(cnt) < target) {
            if (++spins > a.spin_limit || ld_acquire(a.error) != 0) {
              atomicExch(a.error, 1);
              stop = 1;
              break;
            }
            __nanosleep(256);
          }
        }
      }
      s_group = g;
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) return;
    const int item = s_item, g = s_group;
    const int h = item / a.items_per_holo;
    const BatchGroup gi = a.groups[g];
    const PassDesc& d = a.descs[(size_t)h * a.n_groups + g];
    const int t0 = (item - h * a.items_per_holo - gi.first_item) * gi.chunk;
    const int t1 = min(t0 + gi.chunk, gi.tiles);
    for (int tile = t0; tile < t1; ++tile) {
      run_item<KIND_X>(d, gi.phase, gi.L, tile, smem, a.tw);
      __syncthreads();  // the next tile reuses the shared tile buffer
    }
    // The barrier orders every thread's stores before thread 0's device-scope
    // fence and count (the pattern of a grid-wide barrier).
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.done + (size_t)h * a.n_groups + g, 1);
      s_item = nxt;
    }
  }
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

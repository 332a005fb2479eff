// sf_batch.cuh -- work loop of the persistent batch kernels (a batch of
// ragged views over a stream of holograms: the paper's real-time loop,
// Section 2.2, repeated over frames, with every view and frame in one
// launch).
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
// the current one; the next one is larger, so the argument still holds.)
// Waits are still bounded (spin_limit sleeps); on expiry a CTA sets the
// error word and leaves, which unblocks nobody but ends every other wait by
// its own limit, so the launch always returns.
#pragma once

#include "sf_kernels.cuh"

namespace sf {

// Row tiles of the batch kernels: the pass kernel's tile shape, capped at the
// batch CTA size.
constexpr int batch_cta(int L) { return pass_cta_target(L) < kBatchThreads ? pass_cta_target(L) : kBatchThreads; }
template <int L>
using BatchShape = PassShape<L, batch_cta(L)>;

__device__ __forceinline__ int batch_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The persistent loop.  run(d, phase, L, tile) transforms one row tile of
// pass descriptor d; every thread of the CTA calls it.
template <typename Run>
__device__ __forceinline__ void batch_loop(const BatchArgs& a, Run&& run) {
  __shared__ int s_item, s_group, s_stop;
  // the item's pass descriptor, staged once per item: the row tile reads its
  // fields after every barrier, and shared memory answers those re-reads
  // faster than the global table would
  __shared__ PassDesc s_desc;
  if (threadIdx.x == 0) s_item = atomicAdd(a.next, 1);
  for (;;) {
    __syncthreads();
    int nxt = 0;
    if (threadIdx.x == 0) {
      const int item = s_item;
      // Take the following item now; its value is only needed at the end of
      // this one, so the round trip overlaps the work (items stay in order).
      nxt = atomicAdd(a.next, 1);
      int stop = item >= a.total_items || batch_ld_acquire(a.error) != 0;
      int g = 0;
      if (!stop) {
        const int h = item / a.items_per_holo, r = item - h * a.items_per_holo;
        g = a.item_group[r];
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
          while (batch_ld_acquire(cnt) < target) {
            if (++spins > a.spin_limit || batch_ld_acquire(a.error) != 0) {
              atomicExch(a.error, 1);
              stop = 1;
              break;
            }
            __nanosleep(256);
          }
        }
        if (!stop) s_desc = a.descs[(size_t)h * a.n_groups + g];
      }
      s_group = g;
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) return;
    const int item = s_item, g = s_group;
    const int h = item / a.items_per_holo;
    const BatchGroup gi = a.groups[g];
    const int t0 = (item - h * a.items_per_holo - gi.first_item) * gi.chunk;
    const int t1 = min(t0 + gi.chunk, gi.tiles);
    for (int tile = t0; tile < t1; ++tile) {
      run(s_desc, gi.phase, gi.L, tile);
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

}  // namespace sf

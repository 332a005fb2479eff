// sf_persist.cu -- persistent row pass with TMA prefetch of the next tile.
//
// Same arithmetic as k_pass (row_tile_src), but each CTA loops over row tiles
// (tile = blockIdx.x + i * gridDim.x) and, while it transforms tile i, the
// bulk-copy engine (cp.async.bulk, completion on an mbarrier) already moves
// the rows of tile i + 1 into the other half of a two-stage shared-memory
// buffer.  The view's input chirp, output chirp and kernel spectrum are
// copied to shared memory when the tile's view changes, so the FFT network
// reads only shared memory and the twiddle tables.  Requirements (checked by
// the host before choosing this kernel): 16-byte aligned rows and row
// lengths, FFT length <= 4096.  Waits on the mbarriers are bounded; on expiry
// a CTA sets the plan's device error word and carries on, so the launch
// always ends.
#include <cstring>

#include "sf_kernels.cuh"

namespace sf {
namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the given phase of an mbarrier; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, unsigned parity, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try_wait(m, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(m))
               : "memory");
}

template <int L>
__device__ __forceinline__ void decode(const PersistArgs& pa, int tile, int& k, int& row0) {
  k = 0;
  while (tile >= pa.tile_off[k + 1]) ++k;
  row0 = (tile - pa.tile_off[k]) * PassShape<L>::G;
}

template <int L, int KIND, bool PRUNE>
__global__ void __launch_bounds__(PassShape<L>::THREADS, PassShape<L>::MIN_BLOCKS)
k_pass_tma(const __grid_constant__ PassBatch b, const float4* __restrict__ tw, const __grid_constant__ PersistArgs pa,
           const __grid_constant__ OutMaps om) {
  using Sh = PassShape<L>;
  constexpr int G = Sh::G;
  constexpr unsigned ELEM = KIND == PASS_X_REAL ? 4u : 8u;
  extern __shared__ __align__(128) unsigned char sm[];
  float2* exch = reinterpret_cast<float2*>(sm);
  float2* cin_s = reinterpret_cast<float2*>(sm + pa.off_cin);
  float2* cout_s = reinterpret_cast<float2*>(sm + pa.off_cout);
  float2* h_s = reinterpret_cast<float2*>(sm + pa.off_h);
  unsigned char* rows = sm + pa.off_rows;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + pa.off_mbar);
  const int tid = threadIdx.x;

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // thread 0: start the copies of the rows of `tile` into stage buffer `st`
  auto issue = [&](int tile, int st) {
    int k, row0;
    decode<L>(pa, tile, k, row0);
    const PassDesc& d = b.d[k];
    const int nrows = min(G, d.rows - row0);
    const unsigned bytes = (unsigned)d.n0 * ELEM;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&mbar[st], bytes * (unsigned)nrows);
    const unsigned char* src = static_cast<const unsigned char*>(d.src);
    for (int g = 0; g < nrows; ++g)
      tma_load_1d(rows + (size_t)(st * G + g) * pa.row_bytes, src + ((size_t)(row0 + g) * d.src_ld) * ELEM, bytes,
                  &mbar[st]);
  };

  int tile = blockIdx.x;
  if (tile < pa.total_tiles && tid == 0) issue(tile, 0);
  int cur = -1;
  bool failed = false;
  for (int i = 0; tile < pa.total_tiles; ++i, tile += gridDim.x) {
    int k, row0;
    decode<L>(pa, tile, k, row0);
    const PassDesc& d = b.d[k];
    const int nxt = tile + gridDim.x;
    if (nxt < pa.total_tiles && tid == 0) issue(nxt, (i + 1) & 1);
    if (k != cur) {  // this tile belongs to another view: stage its vectors
      __syncthreads();
      for (int p = tid; p < d.n0; p += Sh::THREADS) cin_s[p] = __ldg(d.cin + p);
      for (int p = tid; p < d.n1; p += Sh::THREADS) cout_s[p] = __ldg(d.cout + p);
      for (int p = tid; p < L; p += Sh::THREADS) h_s[p] = __ldg(d.H + p);
      __syncthreads();
      cur = k;
    }
    if (!mbar_wait(&mbar[i & 1], (unsigned)((i >> 1) & 1), pa.spin_limit)) {
      failed = true;
      atomicExch(pa.err, 1);
    }
    const StagedSrc<KIND> src{cin_s, h_s, cout_s, rows + (size_t)((i & 1) * G) * pa.row_bytes, pa.row_bytes};
    // output tiles by tensor stores where the pass allows (thread 0 waits for their shared-memory reads)
    row_tile_src<L, KIND, StagedSrc<KIND>, false, pass_cta_target(L), PRUNE>(d, row0, exch, tw, src,
                                                                           om.use[k] ? &om.map[k] : nullptr);
    __syncthreads();  // stage (i & 1) is free for the copy issued in the next iteration
  }
  if (failed) {
    // a wait gave up: give the copies still in flight one more bounded wait before leaving
    const int n = (pa.total_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // tiles of this CTA
    for (int st = 0; st < 2; ++st) {
      const int uses = (n - st + 1) / 2;  // issues into stage st
      if (uses > 0) mbar_wait(&mbar[st], (unsigned)((uses - 1) & 1), pa.spin_limit);
    }
  }
}

template <int L, int KIND>
cudaError_t launch_tma_t(const PassBatch& b, const float4* tw, const PersistArgs& pa, int grid, size_t smem,
                         cudaStream_t s) {
  auto kern = pass_prunable<L>(b) ? k_pass_tma<L, KIND, true> : k_pass_tma<L, KIND, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  OutMaps om;
  for (int k = 0; k < kMaxPassBatch; ++k)
    om.use[k] = k < b.count && PassShape<L>::G % 2 == 0 &&
                        output_tensor_map((PassKind)KIND, b.d[k], PassShape<L>::G, &om.map[k])
                    ? 1
                    : 0;
  kern<<<grid, PassShape<L>::THREADS, smem, s>>>(b, tw, pa, om);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_tma_kind(PassKind kind, const PassBatch& b, const float4* tw, const PersistArgs& pa, int grid,
                            size_t smem, cudaStream_t s) {
  switch (kind) {
    case PASS_X_REAL: return launch_tma_t<L, PASS_X_REAL>(b, tw, pa, grid, smem, s);
    case PASS_X_CPLX: return launch_tma_t<L, PASS_X_CPLX>(b, tw, pa, grid, smem, s);
    case PASS_Y: return launch_tma_t<L, PASS_Y>(b, tw, pa, grid, smem, s);
  }
  return cudaErrorInvalidValue;
}

template <int L, int KIND>
int occupancy_t(size_t smem) {
  int n = 0;
  auto kern = k_pass_tma<L, KIND, false>;  // the pruned variant has the same resources
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, PassShape<L>::THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

bool tma_length_supported(int L) { return L >= 256 && L <= 4096 && (L & (L - 1)) == 0; }

// Shared-memory layout of one launch; returns the total bytes.
size_t tma_layout(int L, PassKind kind, int n0max, int n1max, PersistArgs& pa) {
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const int G = pass_rows_per_cta(L);
  const size_t elem = kind == PASS_X_REAL ? 4 : 8;
  size_t off = al(sizeof(float2) * (size_t)G * buf_elems(L));
  pa.off_cin = (int)off;
  off = al(off + sizeof(float2) * n0max);
  pa.off_cout = (int)off;
  off = al(off + sizeof(float2) * n1max);
  pa.off_h = (int)off;
  off = al(off + sizeof(float2) * L);
  pa.row_bytes = (int)al(elem * n0max);
  pa.off_rows = (int)off;
  off = al(off + (size_t)2 * G * pa.row_bytes);
  pa.off_mbar = (int)off;
  return off + 16;
}

int tma_occupancy(int L, PassKind kind, size_t smem) {
#define SF_TMA_OCC(LL)                                                    \
  case LL:                                                                \
    return kind == PASS_X_REAL   ? occupancy_t<LL, PASS_X_REAL>(smem)     \
           : kind == PASS_X_CPLX ? occupancy_t<LL, PASS_X_CPLX>(smem)     \
                                 : occupancy_t<LL, PASS_Y>(smem);
  switch (L) {
    SF_TMA_OCC(256)
    SF_TMA_OCC(512)
    SF_TMA_OCC(1024)
    SF_TMA_OCC(2048)
    SF_TMA_OCC(4096)
    default: return 0;
  }
#undef SF_TMA_OCC
}

cudaError_t launch_pass_persistent(int L, PassKind kind, const PassBatch& b, const float4* tw, int* err, int sms,
                                   cudaStream_t s) {
  // bulk copies move whole rows: addresses, strides and row lengths must be multiples of 16 bytes
  const size_t elem = kind == PASS_X_REAL ? sizeof(float) : sizeof(float2);
  if (!tma_length_supported(L)) return cudaErrorInvalidValue;
  for (int k = 0; k < b.count; ++k)
    if (reinterpret_cast<uintptr_t>(b.d[k].src) % 16 || (b.d[k].src_ld * elem) % 16 || (b.d[k].n0 * elem) % 16)
      return cudaErrorInvalidValue;
  PersistArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  const int G = pass_rows_per_cta(L);
  int n0max = 1, n1max = 1, tiles = 0, max_rows = 0;
  for (int k = 0; k < b.count; ++k) {
    pa.tile_off[k] = tiles;
    tiles += (b.d[k].rows + G - 1) / G;
    n0max = std::max(n0max, b.d[k].n0);
    n1max = std::max(n1max, b.d[k].n1);
    max_rows = std::max(max_rows, b.d[k].rows);
  }
  for (int k = b.count; k <= kMaxPassBatch; ++k) pa.tile_off[k] = tiles;
  pa.total_tiles = tiles;
  pa.spin_limit = 1ll << 22;
  pa.err = err;
  const size_t smem = tma_layout(L, kind, n0max, n1max, pa);
  const int occ = tma_occupancy(L, kind, smem);
  if (occ < 1) return launch_pass(L, kind, b, (max_rows + G - 1) / G, tw, s);  // does not fit: grid kernel
  return launch_pass_tma(L, kind, b, tw, pa, std::min(tiles, occ * sms), smem, s);
}

cudaError_t launch_pass_tma(int L, PassKind kind, const PassBatch& b, const float4* tw, const PersistArgs& pa, int grid,
                            size_t smem, cudaStream_t s) {
  switch (L) {
    case 256: return launch_tma_kind<256>(kind, b, tw, pa, grid, smem, s);
    case 512: return launch_tma_kind<512>(kind, b, tw, pa, grid, smem, s);
    case 1024: return launch_tma_kind<1024>(kind, b, tw, pa, grid, smem, s);
    case 2048: return launch_tma_kind<2048>(kind, b, tw, pa, grid, smem, s);
    case 4096: return launch_tma_kind<4096>(kind, b, tw, pa, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sf

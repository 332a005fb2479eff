// sf_kernels.cuh -- fused Bluestein row-pass kernel and the plan-time kernels.
//
// One launch of k_pass runs Section 2.2 steps 2-4 and 7-9 (and, on the y
// pass, step 10 with Eq. 5) for every row of up to kMaxPassBatch
// (view, axis) passes:
//
//   load row (implicit zero padding to L)  x  input chirp of Eq. 3   (steps 2-3)
//   forward length-L FFT network                                     (step 4)
//   x kernel spectrum FFT(h) of Eq. 4, cached at plan time           (steps 5-7)
//   adjoint (inverse) FFT network                                    (step 8)
//   crop to n1 outputs  x  output chirp of Eq. 2 (and 1/L)           (step 9)
//   y pass only: complex view, |u1|^2 (Eq. 5) and phase              (step 10)
//
// The x pass reads hologram rows and writes the intermediate transposed,
// [nx1][ny0]; the y pass then reads those rows (hologram columns) and writes
// the view [ny1][nx1] transposed back.  Both passes load contiguous rows.
// A CTA holds G groups of T = L / E threads (E = 16 for power-of-two lengths,
// 24 for the lengths with a factor 3; G from pass_cta_target); group g
// handles row blockIdx.x * G + g of pass blockIdx.y.  When every pass of a
// launch has n0, n1 <= L / 2 (the paper's 2N padding) the pruned variant
// skips the zero half of the first forward stage and the cropped half of the
// last inverse stage.
#pragma once

#include <climits>

#include "sf_fft.cuh"
#include "sf_internal.h"
#include "sf_umma.cuh"

// CTA size and resident warps per SM the power-of-two row passes are built for
constexpr int kPassCtaThreads = 256;
constexpr int kPassMinWarps = 16;

namespace sf {

// complex values per thread of the FFT network of length L
constexpr int fft_e(int L) { return is_pow2(L) ? kE : 24; }

// CTA size a row pass aims for: 256 threads for powers of two (512 at 4096,
// where a 256-thread CTA holds a single row and two rows per CTA measured 9 %
// faster per row), 192 for the lengths with a factor 3 (24 values per thread).
constexpr int pass_cta_target(int L) {
  return !is_pow2(L) ? 192 : (L == 4096 ? 2 * kPassCtaThreads : kPassCtaThreads);
}

// Alternative CTA sizes of the one-tile-per-CTA row pass that the autotuner
// may choose per (L, kind): variant 1 holds half the default rows per CTA,
// variant 2 twice as many; 0 where a variant does not exist (powers of two
// from 1024 to 4096 only, at least one row and at most 512 threads, so the
// 128-register budget holds).
constexpr int pass_cta_variant(int L, int v) {
  if (v == 0) return pass_cta_target(L);
  if (!is_pow2(L) || L < 1024 || L > 4096 || (v != 1 && v != 2)) return 0;
  const int c = v == 1 ? pass_cta_target(L) / 2 : pass_cta_target(L) * 2;
  return (c < L / kE || c > 512) ? 0 : c;
}

// G rows of T = L / E threads per CTA.  Registers: powers of two for 16 warps
// per SM (128 per thread), the lengths with a factor 3 for 12 (up to 168).
template <int L, int CTA = pass_cta_target(L)>
struct PassShape {
  static constexpr int T = L / fft_e(L);
  static constexpr int MIN_WARPS = is_pow2(L) ? kPassMinWarps : 12;
  static constexpr int G = (CTA / T) > 0 ? (CTA / T) : 1;
  static constexpr int THREADS = G * T;
  // CTAs per SM the register budget is set for
  static constexpr int MIN_BLOCKS = MIN_WARPS / (THREADS / 32) > 0 ? MIN_WARPS / (THREADS / 32) : 1;
  static constexpr size_t SMEM = sizeof(float2) * (size_t)G * buf_elems(L);
  // group g synchronises on named barrier 1 + g when its T threads are whole
  // warps; hardware barrier ids are 0..15
  static_assert(T < 32 || T % 32 != 0 || G <= 15, "row groups need named barrier ids 1..15");
};

// exp(i pi ph / 2^63) from a 64-bit fixed-point phase (full scale 2^64 = 2 pi).
__device__ __forceinline__ float2 expi_fx(uint64_t ph) {
  const double a = (double)(int64_t)ph * 0x1p-63;  // in [-1, 1): units of pi
  double s, c;
  sincospi(a, &s, &c);
  return make_float2((float)c, (float)s);
}

__device__ __forceinline__ float phase_of(float2 u) {
  float p = atan2f(u.y, u.x);
  return p <= -3.14159265358979f ? 3.14159265358979f : p;  // (-pi, pi]
}

// Where a row tile reads its chirp-multiplied input, kernel spectrum and output
// chirp from: global memory (rows through L1, or through L2 only when
// COHERENT, for data written earlier in the same launch) ...
template <int KIND, bool COHERENT>
struct GlobalSrc {
  const PassDesc& d;
  __device__ __forceinline__ float2 in(int g, int row, int p) const {
    const float2 c = __ldg(d.cin + p);
    if constexpr (KIND == PASS_X_REAL) {
      return cscale(c, __ldg(static_cast<const float*>(d.src) + (size_t)row * d.src_ld + p));
    } else {
      const float2* sp = static_cast<const float2*>(d.src) + (size_t)row * d.src_ld + p;
      return cmul(COHERENT ? __ldcg(sp) : __ldg(sp), c);
    }
  }
  __device__ __forceinline__ float2 h(int i) const { return __ldg(d.H + i); }
  __device__ __forceinline__ float2 co(int p) const { return __ldg(d.cout + p); }
};

// ... or shared memory: the view's vectors and the tile's rows staged there
// (row g of the tile at rows + g * row_bytes).
template <int KIND>
struct StagedSrc {
  const float2* cin;
  const float2* H;
  const float2* cout;
  const unsigned char* rows;
  int row_bytes;
  __device__ __forceinline__ float2 in(int g, int, int p) const {
    const float2 c = cin[p];
    if constexpr (KIND == PASS_X_REAL) return cscale(c, reinterpret_cast<const float*>(rows + g * row_bytes)[p]);
    else return cmul(reinterpret_cast<const float2*>(rows + g * row_bytes)[p], c);
  }
  __device__ __forceinline__ float2 h(int i) const { return H[i]; }
  __device__ __forceinline__ float2 co(int p) const { return cout[p]; }
};

// One tile of a pass: group g of the CTA transforms source row r = row0 + g
// (input positions p < n0, zero-padded to L), and the n1 outputs are written
// transposed (dst[p * dst_ld + r]) through a shared-memory tile so the G rows
// of the tile leave as G-element contiguous runs.  With SPARE, the CTA may
// have more threads than the tile's G T (a CTA sized for another length):
// those only join the CTA barriers and the final store loop.  With out_map
// (G even, no SPARE), thread 0 sends the tile out by 2D tensor stores instead
// and waits only until they have read shared memory.
template <int L, int KIND, typename Src, bool SPARE = false, int CTA = pass_cta_target(L), bool PRUNE = false>
__device__ __forceinline__ void row_tile_src(const PassDesc& d, int row0, float2* smem, const float4* __restrict__ tw,
                                             const Src& src, const CUtensorMap* out_map = nullptr) {
  using Sh = PassShape<L, CTA>;
  constexpr int T = Sh::T, G = Sh::G, E = fft_e(L);
  // PRUNE (caller-checked: n0 <= L / 2 and n1 <= L / 2, E = 16): positions
  // t + T j with j >= E / 2 are zero on input and unused on output
  static_assert(!PRUNE || E == 16, "pruning is defined for the radix-16 network");
  constexpr int J_IN = PRUNE ? E / 2 : E;
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  const int row = row0 + g;
  const bool active = !SPARE || threadIdx.x < Sh::THREADS;
  const bool valid = row < d.rows;
  float2* buf = smem + g * buf_elems(L);
  const int n1 = d.n1;

  if (active) {
    float2 v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int p = t + T * j;
      v[j] = (j < J_IN && valid && p < d.n0) ? src.in(g, row, p) : make_float2(0.f, 0.f);
    }

    fft_forward<L, E, 0, PRUNE>(v, t, g, buf, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmul(v[e], src.h(e * T + t));
    fft_inverse<L, E, stage_count(L, E) - 1, PRUNE>(v, t, g, buf, tw);

    // output chirp, then the transposed store through the tile [n1][G]
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J_IN; ++j) {
      const int p = t + T * j;
      if (p < n1) smem[p * G + g] = cmul(v[j], src.co(p));
    }
  } else {
    __syncthreads();
  }
  if constexpr (!SPARE && G % 2 == 0) {
    if (out_map) {
      umma::fence_smem_to_async();  // the tile's shared-memory writes, to the tensor stores
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int j = 0; j * kOutBoxN < n1; ++j)
          umma::tma_store_2d(out_map, smem + j * kOutBoxN * G, 2 * row0, j * kOutBoxN);
        umma::bulk_commit();
        umma::bulk_wait_read();
      }
      return;
    }
  }
  __syncthreads();
  // descriptor fields in registers: a descriptor in global memory (batch
  // kernel) would otherwise be re-read after every store
  const int rows_here = min(G, d.rows - row0);
  const int stride = SPARE ? (int)blockDim.x : Sh::THREADS;
  float2* const dst = d.dst;
  float* const inten = d.inten;
  float* const phase = d.phase;
  const size_t dst_ld = (size_t)d.dst_ld;
  const bool acc = d.accumulate != 0;
  for (int i = threadIdx.x; i < n1 * G; i += stride) {
    const int p = i / G, gg = i - p * G;
    if (gg < rows_here) {
      const float2 u = smem[i];
      const size_t o = (size_t)p * dst_ld + row0 + gg;
      if constexpr (KIND != PASS_Y) {
        dst[o] = u;
      } else {
        if (dst) dst[o] = acc ? cadd(dst[o], u) : u;
        if (inten) inten[o] = fmaf(u.x, u.x, u.y * u.y);
        if (phase) phase[o] = phase_of(u);
      }
    }
  }
}

template <int L, int KIND, bool COHERENT, bool SPARE = false, int CTA = pass_cta_target(L), bool PRUNE = false>
__device__ __forceinline__ void row_tile(const PassDesc& d, int row0, float2* smem, const float4* __restrict__ tw,
                                         const CUtensorMap* out_map = nullptr) {
  row_tile_src<L, KIND, GlobalSrc<KIND, COHERENT>, SPARE, CTA, PRUNE>(d, row0, smem, tw,
                                                                      GlobalSrc<KIND, COHERENT>{d}, out_map);
}

// Row pass: tile blockIdx.x of pass blockIdx.y.  PRUNE: every pass of the
// launch has n0 <= L / 2 and n1 <= L / 2 (the paper's 2N padding).
template <int L, int KIND, bool PRUNE, int CTA = pass_cta_target(L)>
__global__ void __launch_bounds__(PassShape<L, CTA>::THREADS, PassShape<L, CTA>::MIN_BLOCKS)
k_pass(const __grid_constant__ PassBatch b, const float4* __restrict__ tw, const __grid_constant__ OutMaps om) {
  extern __shared__ __align__(128) float2 smem[];
  const PassDesc& d = b.d[blockIdx.y];
  const int row0 = blockIdx.x * PassShape<L, CTA>::G;
  if (row0 >= d.rows) return;  // whole CTA past this pass's rows
  row_tile<L, KIND, false, false, CTA, PRUNE>(d, row0, smem, tw, om.use[blockIdx.y] ? &om.map[blockIdx.y] : nullptr);
}

// The pruned network applies to the radix-16 (power-of-two) lengths.
template <int L>
bool pass_prunable(const PassBatch& b) {
  if (!is_pow2(L) || fft_e(L) != 16) return false;
  for (int k = 0; k < b.count; ++k)
    if (2 * b.d[k].n0 > L || 2 * b.d[k].n1 > L) return false;
  return true;
}

// Kernel spectrum of Eq. 4 (steps 5-6), one thread group per axis, run once
// at plan time: h[p] = exp(i pi S d^2) with d = p for p < n1, d = p - L for
// p > L - n0, 0 elsewhere; pushed through the same forward network so it
// lands in register order.
template <int L>
__global__ void __launch_bounds__(L / fft_e(L)) k_hspec(const AxisCoef* __restrict__ axes,
                                                        const float4* __restrict__ tw) {
  constexpr int T = L / fft_e(L), E = fft_e(L);
  extern __shared__ float2 smem[];
  const AxisCoef a = axes[blockIdx.x];
  const int t = threadIdx.x;
  float2 v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int p = t + T * j;
    int dd = INT_MIN;
    if (p < a.n1) dd = p;
    else if (p > L - a.n0) dd = p - L;
    v[j] = dd == INT_MIN ? make_float2(0.f, 0.f) : expi_fx(a.h2 * (uint64_t)((int64_t)dd * dd));
  }
  fft_forward<L, E>(v, t, 0, smem, tw);
#pragma unroll
  for (int e = 0; e < E; ++e) a.H[e * T + t] = v[e];
}

// The one-tile-per-CTA row pass with CTA threads (pass_cta_variant(L, v)).
template <int L, int CTA>
cudaError_t launch_pass_cta(PassKind kind, const PassBatch& b, int grid_x, const float4* tw, cudaStream_t s) {
  using Sh = PassShape<L, CTA>;
  const dim3 grid(grid_x, b.count), block(Sh::THREADS);
  OutMaps om;
  for (int k = 0; k < kMaxPassBatch; ++k)
    om.use[k] = k < b.count && Sh::G % 2 == 0 && output_tensor_map(kind, b.d[k], Sh::G, &om.map[k]) ? 1 : 0;
  auto go = [&](auto kern) {
    if (Sh::SMEM > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, block, Sh::SMEM, s>>>(b, tw, om);
    return cudaGetLastError();
  };
  if constexpr (is_pow2(L)) {
    if (pass_prunable<L>(b)) {
      switch (kind) {
        case PASS_X_REAL: return go(k_pass<L, PASS_X_REAL, true, CTA>);
        case PASS_X_CPLX: return go(k_pass<L, PASS_X_CPLX, true, CTA>);
        case PASS_Y: return go(k_pass<L, PASS_Y, true, CTA>);
      }
    }
  }
  switch (kind) {
    case PASS_X_REAL: return go(k_pass<L, PASS_X_REAL, false, CTA>);
    case PASS_X_CPLX: return go(k_pass<L, PASS_X_CPLX, false, CTA>);
    case PASS_Y: return go(k_pass<L, PASS_Y, false, CTA>);
  }
  return cudaErrorInvalidValue;
}

template <int L>
cudaError_t launch_pass_t(PassKind kind, const PassBatch& b, int grid_x, const float4* tw, cudaStream_t s);

template <int L>
cudaError_t launch_hspec_t(const AxisCoef* axes_dev, int n_axes, const float4* tw, cudaStream_t s) {
  constexpr size_t smem = sizeof(float2) * (size_t)buf_elems(L);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_hspec<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_hspec<L><<<n_axes, L / fft_e(L), smem, s>>>(axes_dev, tw);
  return cudaGetLastError();
}

// launch_pass_t<L>: the default CTA size (the variants are instantiated on
// their own, SF_INSTANTIATE_VARIANT, and reached through launch_pass_variant).
template <int L>
cudaError_t launch_pass_t(PassKind kind, const PassBatch& b, int grid_x, const float4* tw, cudaStream_t s) {
  return launch_pass_cta<L, pass_cta_target(L)>(kind, b, grid_x, tw, s);
}

#define SF_INSTANTIATE_LENGTH(LL)                                                                      \
  template cudaError_t launch_pass_t<LL>(PassKind, const PassBatch&, int, const float4*, cudaStream_t); \
  template cudaError_t launch_hspec_t<LL>(const AxisCoef*, int, const float4*, cudaStream_t);

#define SF_DECLARE_LENGTH(LL)                                                                                 \
  extern template cudaError_t launch_pass_t<LL>(PassKind, const PassBatch&, int, const float4*, cudaStream_t); \
  extern template cudaError_t launch_hspec_t<LL>(const AxisCoef*, int, const float4*, cudaStream_t);

#define SF_INSTANTIATE_VARIANT(LL, CC) \
  template cudaError_t launch_pass_cta<LL, CC>(PassKind, const PassBatch&, int, const float4*, cudaStream_t);
#define SF_DECLARE_VARIANT(LL, CC) \
  extern template cudaError_t launch_pass_cta<LL, CC>(PassKind, const PassBatch&, int, const float4*, cudaStream_t);

}  // namespace sf

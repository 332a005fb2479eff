// sf_tcgen05.cu -- mixed-precision row pass on the sm_100-family tensor
// cores: the length-L convolution of Section 2.2 steps 4-8 as four dense DFT
// matrix products issued with tcgen05.mma (FP16 or BF16 operands in shared
// memory, FP32 accumulators in tensor memory), chirps, twiddles and kernel
// spectrum applied in FP32 between them.
//
// Four-step split of the FFT of length L = R1 * R2 (R2 = 32, R1 = L / 32;
// built for L = 2048, 1024 and 512):
//   n = R2 n1 + n2,  k = k1 + R1 k2
//   X[k1 + R1 k2] = sum_n2 W_R2^{n2 k2} W_L^{n2 k1} sum_n1 x[R2 n1 + n2] W_R1^{n1 k1}
// and the inverse in the mirrored order, each inverse DFT taken as
// conj(DFT(conj(.))) so that one DFT matrix serves both directions.  With the
// paper's 2N padding (n0, n1 <= L / 2, required here) only n1 < R1 / 2 is
// nonzero on input and only n1 < R1 / 2 survives the crop, which halves the
// first and the last product.
//
// Every product is the real GEMM D (128 x N) = A (128 x K) B (K x N) of the
// block form [Re | Im] [[Fr, Fi], [-Fi, Fr]] of a unitary-scaled DFT matrix
// F; a CTA holds kGroups independent groups of eight warps, and a group
// transforms a tile of TR = 4 rows at a time (8 at L = 512, see Shape):
//
//   stage A   rows (r, n2), K = (re, im) of n1 < R1/2, N = (re, im) of k1
//   twiddle   W_L^{n2 k1} (FP32), to the stage-B operand (transpose via
//             an MN-major operand layout)
//   stage B   rows (r, k1), K = n2, N = k2; R1 / 32 products of 128 rows
//   spectrum  x FFT(h) / sqrt(L) (natural order), conjugated into the
//             stage-B^H operand (K-major)
//   stage B^H rows (r, k1), K = k2, N = n2
//   twiddle   W_L^{n2 k1} again (the conjugations cancel), to the stage-A^H
//             operand (MN-major)
//   stage A^H rows (r, n2), K = k1, N = n1 < R1/2
//   output    conj, undo the scales, x output chirp, staged [n][row] and
//             sent out by 2D tensor stores (TMA), or by a store loop
//
// Warps w and w + 4 of a group read tensor-memory lanes 32 (w mod 4) + l, each
// taking half of every epilogue's columns, so a thread always holds complete
// complex values; every operand store is a 16-byte chunk of 8 consecutive K
// (K-major) or M (MN-major) elements.  Rows are
// normalised by a power of two from their largest input component before the
// first conversion (exact), which keeps FP16 in range.  The x3 precisions
// split each operand into hi + lo parts and accumulate hi*hi + hi*lo + lo*hi.
//
// The kernels are persistent (one CTA per SM): four groups for FP16 / BF16
// (1024 threads, all 512 tensor-memory columns, 128 per group), two for the
// x3 precisions, whose doubled operand buffers leave room for no more.  The
// constant image (DFT matrices, twiddles) arrives by one bulk copy that
// overlaps the first tile's loads; groups start 1 us apart so that their
// products do not reach the tensor core together; the spectrum and
// output-chirp loads are issued before the waits for the products they
// follow; one store thread per group issues the tensor stores and waits for
// them.  k_pass_t5 runs one pass (tiles round-robin over the groups, spread
// over every SM when there are fewer tiles than groups); k_views_t5 runs both
// passes of two to eight views, tiles claimed in order from a global counter,
// each view's y tiles after its x tiles.  Every wait
// (MMA completion, constant image, a y tile's dependency) is bounded; on
// expiry the group sets the plan's device error word, waits once more
// (bounded) where a copy may be in flight, leaves its tile loop and the CTA
// frees its tensor memory.
//
// Measured on the paper-scale step (four 1024^2 views, L = 2048 both axes):
// FP16 and BF16 68.5-69.3 us fused (73.4 us with one launch per pass),
// FP16x3 100.5 us, against 76.1 us for the FP32 pass.  The tensor pipe is ~10 %
// busy: the pass is bound by the latency of a tile's chain (loads, four
// product round trips, FP32 epilogues, output staging; 14-17 us per tile)
// at 16 rows in flight per SM, the number that tensor memory allows.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "sf_kernels.cuh"
#include "sf_umma.cuh"

namespace sf {
namespace t5 {

constexpr int kR2 = 32;        // inner radix: the lanes of a warp
constexpr int kGroupWarps = 8;  // warps per group: two per tensor-memory lane quarter
constexpr int kGroupThreads = 32 * kGroupWarps;
// lane 0 of a group's last warp issues the group's tensor stores, waits for them and (fused launch)
// releases finished x tiles, so that thread 0 (products, claims, dependency waits) never waits on them
constexpr int kStoreTq = kGroupThreads - 32;
// MMA completion waits: tries of at most kSuspendNs each (the waiting thread
// sleeps in hardware instead of spinning), kSpin tries (about 1 s) in all
constexpr uint32_t kSuspendNs = 20000;
constexpr long long kSpin = 50000;
constexpr unsigned kStaggerNs = 1000;  // start offset between a CTA's groups
// waits of a fused launch's y tiles for their view's x tiles: kDepSpin polls kDepSleepNs apart (about 1 s)
constexpr long long kDepSpin = 4000000;
constexpr unsigned kDepSleepNs = 256;

template <int PREC>
struct Prec {
  static constexpr bool kBf16 = PREC == SF_PREC_BF16TC || PREC == SF_PREC_BF16X3TC;
  static constexpr bool kSplit = PREC == SF_PREC_FP16X3TC || PREC == SF_PREC_BF16X3TC;
  static constexpr int kGroups = kSplit ? 2 : 4;
  static constexpr int kThreads = kGroupThreads * kGroups;
};

template <int L>
struct Shape {
  static constexpr int R1 = L / kR2;
  static constexpr int KA = R1 / 2;  // nonzero n1 on input
  static constexpr int NA = R1 / 2;  // kept n1 on output
  static_assert(R1 == 16 || R1 == 32 || R1 == 64,
                "tcgen05 row pass lengths: 512 (16 x 32), 1024 (32 x 32) and 2048 (64 x 32)");
  // rows per tile: 4 (the first product's 128 rows are 4 rows x 32 n2), 8 at R1 = 16 so that a
  // middle-stage product still has 128 rows (8 rows x 16 k1); the first and last stages then take
  // QA = 2 products of 128 rows
  static constexpr int TR = R1 >= 32 ? 4 : 128 / R1;
  static constexpr int QA = TR / 4;
  // real GEMM shapes (M = 128 throughout)
  static constexpr int A_K = 2 * KA, A_N = 2 * R1;    // stage A
  static constexpr int B_K = 2 * kR2, B_N = 2 * kR2;  // stages B and B^H
  static constexpr int H_K = 2 * R1, H_N = 2 * NA;    // stage A^H
  static constexpr int QB = TR * R1 / 128;            // products per middle stage
  static constexpr int RP = 128 / R1;                 // rows of a middle-stage product
  // a K-major operand row holds 64 K elements (128 bytes) per column, whatever K it uses
  static constexpr int kmaj_bytes(int rows, int k) { return rows * 128 * ((k + 63) / 64); }
  // constant image: the three DFT matrices (K-major B operands), hi then lo, then the twiddles
  static constexpr int BA_BYTES = kmaj_bytes(A_N, A_K), BB_BYTES = kmaj_bytes(B_N, B_K),
                       BH_BYTES = kmaj_bytes(H_N, H_K);
  static_assert(H_K <= 64 || H_N == 64, "a second K column starts 8 KiB (64 rows) in");
  static_assert(A_K <= 64 && B_K <= 64, "single-column K-major operands");
  static constexpr int MAT_BYTES = BA_BYTES + BB_BYTES + BH_BYTES;
  static constexpr int TW_LD = kR2 + 1;  // padded row of the twiddle table T[k1][n2] (float2)
  static constexpr int TW_BYTES = R1 * TW_LD * 8;
  // operand bytes of one first-stage / last-stage product (K-major / MN-major, 128 rows)
  static constexpr int A_PROD_BYTES = kmaj_bytes(128, A_K), AH_PROD_BYTES = 128 * H_K * 2;
  static constexpr int cmax(int a, int b) { return a > b ? a : b; }
  // per-group operand buffer: the largest stage operand, also the output staging tile
  static constexpr int OP_BYTES = cmax(cmax(QA * A_PROD_BYTES, QA * AH_PROD_BYTES),
                                       cmax(QB * kmaj_bytes(128, B_K), cmax(QB * 128 * B_K * 2, TR * (L / 2) * 8)));
  static_assert(OP_BYTES % 1024 == 0 && A_PROD_BYTES % 1024 == 0 && AH_PROD_BYTES % 1024 == 0, "1 KiB atoms");
  static constexpr int align(int b) { return (b + 1023) & ~1023; }
  static constexpr int const_bytes(bool split) { return (split ? 2 : 1) * MAT_BYTES + TW_BYTES; }
  static constexpr int op_offset(bool split) { return align(const_bytes(split)); }
  static constexpr int group_bytes(bool split) { return (split ? 2 : 1) * OP_BYTES; }
  static constexpr int misc_offset(bool split) { return op_offset(split) + (split ? 2 : 4) * group_bytes(split); }
  // misc: one MMA mbarrier per group (from byte 0), the constant-image mbarrier (32), the
  // tensor-memory base (48), per-warp row maxima (64 .. 191), per-group tile claims (192 .. 207)
  static constexpr int smem_bytes(bool split) { return misc_offset(split) + 256; }
};

// Operand layouts, 128-byte swizzle (16-bit elements; every operand starts on
// a 1 KiB boundary).  K-major: each row's 64 K elements are 128 bytes, rows
// in 1 KiB groups of 8, 16-byte chunk c of row m stored at chunk c ^ (m mod 8);
// K beyond 64 continues in a further column (only the 64-row stage-A^H
// matrix, 8 KiB per column).  MN-major (M = 128): each K row holds 64 M
// elements with the same XOR, 8 K rows per 1 KiB group, the two 64-wide M
// halves KX / 8 KiB apart.
__host__ __device__ constexpr int kmaj_off(int mn, int kk) {
  return (kk >> 6) * 8192 + (mn >> 3) * 1024 + (mn & 7) * 128 + ((((kk & 63) >> 3) ^ (mn & 7)) << 4) + (kk & 7) * 2;
}
__host__ __device__ constexpr int mnmaj_off(int m, int kk, int KX) {
  return (m >> 6) * (KX >> 3) * 1024 + (kk >> 3) * 1024 + (kk & 7) * 128 + ((((m & 63) >> 3) ^ (kk & 7)) << 4) +
         (m & 7) * 2;
}
__device__ __forceinline__ uint64_t desc_sw(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return umma::sdesc(saddr, lbo, sbo) | ((uint64_t)2 << 61);
}

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b, float& ra, float& rb) {
  if constexpr (BF) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 f = __bfloat1622float2(h);
    ra = a - f.x;
    rb = b - f.y;
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    ra = a - f.x;
    rb = b - f.y;
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}

// Store 8 values as one 16-byte chunk (hi) and, for the split precisions, the
// chunk of their rounding remainders (lo) at the same offset of the lo buffer.
template <int L, int PREC>
__device__ __forceinline__ void store8(unsigned char* hi, int off, const float (&v)[8]) {
  constexpr bool BF = Prec<PREC>::kBf16;
  float r[8];
  uint4 h;
  h.x = pack2<BF>(v[0], v[1], r[0], r[1]);
  h.y = pack2<BF>(v[2], v[3], r[2], r[3]);
  h.z = pack2<BF>(v[4], v[5], r[4], r[5]);
  h.w = pack2<BF>(v[6], v[7], r[6], r[7]);
  *reinterpret_cast<uint4*>(hi + off) = h;
  if constexpr (Prec<PREC>::kSplit) {
    float t[8];
    uint4 lo;
    lo.x = pack2<BF>(r[0], r[1], t[0], t[1]);
    lo.y = pack2<BF>(r[2], r[3], t[2], t[3]);
    lo.z = pack2<BF>(r[4], r[5], t[4], t[5]);
    lo.w = pack2<BF>(r[6], r[7], t[6], t[7]);
    *reinterpret_cast<uint4*>(hi + Shape<L>::OP_BYTES + off) = lo;
  }
}

__device__ __forceinline__ void group_bar(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(kGroupThreads) : "memory");
}
// Group barrier that also ANDs a flag over the group's threads.
__device__ __forceinline__ bool group_bar_and(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbarrier.cta.red.and.pred po, %2, %3, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + g), "n"(kGroupThreads)
      : "memory");
  return r != 0;
}

template <bool SPLIT, bool A_MN>
__device__ __forceinline__ void gemm(uint32_t d, uint32_t a, uint32_t a_lo, int a_kx, uint32_t bm, uint32_t bm_lo,
                                     int b_rows, int ksteps, uint32_t idesc) {
  for (int k = 0; k < ksteps; ++k) {
    uint32_t aoff, albo;
    if constexpr (A_MN) {
      aoff = k * 2048;
      albo = (uint32_t)(a_kx >> 3) * 1024;
    } else {
      aoff = (k & 3) * 32 + (k >> 2) * 16 * 1024;
      albo = 16;
    }
    const uint32_t boff = (k & 3) * 32 + (k >> 2) * (b_rows >> 3) * 1024;
    const uint64_t ad = desc_sw(a + aoff, albo, 1024), bd = desc_sw(bm + boff, 16, 1024);
    umma::mma(d, ad, bd, idesc, k > 0);
    if constexpr (SPLIT) {
      umma::mma(d, ad, desc_sw(bm_lo + boff, 16, 1024), idesc, 1);
      umma::mma(d, desc_sw(a_lo + aoff, albo, 1024), bd, idesc, 1);
    }
  }
}


struct Args {
  const uint4* consts;  // constant image (Shape::const_bytes)
  int* err;             // device error word
  int total_tiles;
  int tile_off[kMaxPassBatch + 1];
  int tma_store[kMaxPassBatch];  // pass k stores through out_map[k] (else plain stores)
  // pass k's output as a 2D float tensor {2 rows, n1} with row pitch dst_ld complex values
  CUtensorMap out_map[kMaxPassBatch];
};

// Source loads: read-only path, or through L2 only (COHERENT) for data that
// other CTAs of the same launch wrote.
template <bool COHERENT, typename T>
__device__ __forceinline__ T ld_src(const T* p) {
  if constexpr (COHERENT) return __ldcg(p);
  else return __ldg(p);
}

// One group's shared-memory regions, tensor-memory columns and wait state.
template <int L, int PREC>
struct GroupCtx {
  int g, tq, gw, wq, hh, l;  // group; thread in group; warp gw = (lane quarter wq, column half hh); lane
  unsigned char* op;         // operand / staging buffer
  uint64_t* bars;            // MMA completion mbarriers (one per group)
  uint64_t* cbar;            // constant-image mbarrier
  float* rowmax;             // this group's per-warp row maxima
  const float2* tw;          // twiddle table
  uint32_t tm, lanes;        // tensor-memory columns of the group, lanes of the warp
  uint32_t parity;           // phase of bars[g] to wait for next
  bool consts_ready;         // the constant image has been waited for
};

// Shared-memory layout, mbarriers, tensor memory, the constant-image copy and
// the group stagger, at kernel entry.
template <int L, int PREC>
__device__ __forceinline__ GroupCtx<L, PREC> group_setup(unsigned char* sm, const uint4* consts) {
  using S = Shape<L>;
  constexpr bool SPLIT = Prec<PREC>::kSplit;
  constexpr int kGroups = Prec<PREC>::kGroups;
  GroupCtx<L, PREC> c;
  c.g = threadIdx.x / kGroupThreads;
  c.tq = threadIdx.x % kGroupThreads;
  c.gw = c.tq >> 5;
  c.wq = c.gw & 3;
  c.hh = c.gw >> 2;
  c.l = c.tq & 31;
  c.op = sm + S::op_offset(SPLIT) + c.g * S::group_bytes(SPLIT);
  unsigned char* const misc = sm + S::misc_offset(SPLIT);
  c.bars = reinterpret_cast<uint64_t*>(misc);
  c.cbar = reinterpret_cast<uint64_t*>(misc + 32);
  uint32_t* const tbase = reinterpret_cast<uint32_t*>(misc + 48);
  c.rowmax = reinterpret_cast<float*>(misc + 64) + kGroupWarps * c.g;
  c.tw = reinterpret_cast<const float2*>(sm + (SPLIT ? 2 : 1) * S::MAT_BYTES);
  if (c.tq == 0) umma::mbar_init(c.bars + c.g, 1);
  if (threadIdx.x == 0) umma::mbar_init(c.cbar, 1);
  if (threadIdx.x < 32) umma::tmem_alloc(tbase, 128 * kGroups);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  // the constant image arrives by one bulk copy while the first tile's inputs load
  if (threadIdx.x == 0) {
    umma::mbar_arrive_expect_tx(c.cbar, S::const_bytes(SPLIT));
    umma::bulk_g2s(sm, consts, S::const_bytes(SPLIT), c.cbar);
  }
  c.consts_ready = false;
  c.parity = 0;
  c.tm = *tbase + 128u * c.g;
  c.lanes = (uint32_t)(32 * c.wq) << 16;
  // Groups start kStaggerNs apart: their products then reach the SM's tensor core at
  // different times instead of queueing behind one another, and their loads and stores
  // spread out in time.
  if (kStaggerNs > 0 && c.g > 0) __nanosleep(kStaggerNs * c.g);
  return c;
}

// This group's tensor stores complete, the constant-image copy has landed
// (a CTA whose groups got no tile never waited for it), then the CTA frees
// its tensor memory.
template <int L, int PREC>
__device__ __forceinline__ void group_teardown(unsigned char* sm, const GroupCtx<L, PREC>& c) {
  using S = Shape<L>;
  if (c.tq == kStoreTq) umma::bulk_wait();
  if (threadIdx.x == 0) umma::mbar_wait(c.cbar, 0, kSpin, kSuspendNs);
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32)
    umma::tmem_dealloc(*reinterpret_cast<uint32_t*>(sm + S::misc_offset(Prec<PREC>::kSplit) + 48),
                       128 * Prec<PREC>::kGroups);
}

// Output staging tile: output n of row r at float2 index TR n + r.  With 4
// rows (32 bytes per n) the tensor map's 32-byte swizzle applies (16-byte
// chunk r / 2 XOR bit 2 of n), so a warp writing 32 consecutive n of one row
// spreads over twice as many banks as the plain layout; 8-row tiles are plain.
template <int TR>
__device__ __forceinline__ int stage_idx(int n, int r) {
  if constexpr (TR == 4) return 4 * n + ((((r >> 1) ^ (n >> 2)) & 1) << 1) + (r & 1);
  else return TR * n + r;
}

// Release of a finished x tile of a fused launch (the group's store thread):
// its tensor stores complete, then the view's count goes up.
__device__ __forceinline__ void signal_tile(int* ctr) {
  umma::bulk_wait();
  umma::fence_async_to_global();
  __threadfence();
  atomicAdd(ctr, 1);
}

// One tile: rows row0 .. row0 + TR - 1 of pass d, steps 2-9 along the
// pass's axis.  out_map: the pass's output tensor map (tensor stores), else
// plain stores.  signal (fused launch, x passes): the counter on which the
// store thread releases the group's previous x tile, once this tile's input
// loads are in flight.  False when an MMA or constant-image wait gave up (err
// set).
template <int L, int KIND, int PREC, bool COHERENT>
__device__ __forceinline__ bool tile_t5(GroupCtx<L, PREC>& ctx, const unsigned char* sm, const PassDesc& d, int row0,
                                        const CUtensorMap* out_map, int* err, int* signal = nullptr) {
  using S = Shape<L>;
  constexpr bool SPLIT = Prec<PREC>::kSplit, BF = Prec<PREC>::kBf16;
  constexpr int R1 = S::R1, KA = S::KA, NA = S::NA;
  constexpr int TR = S::TR;
  // 4-row tiles: warp (wq, hh) takes row wq and half hh of n1 (in and out); 8-row tiles: warp gw takes
  // row gw = 4 hh + wq, all of n1, and hh is the first / last stage's product holding it
  constexpr bool kHalfN1 = TR == 4;
  constexpr int KH = kHalfN1 ? KA / 2 : KA, NH = kHalfN1 ? NA / 2 : NA, CH = kR2 / 2;
  const int g = ctx.g, tq = ctx.tq, gw = ctx.gw, wq = ctx.wq, hh = ctx.hh, l = ctx.l;
  unsigned char* const op = ctx.op;
  uint64_t* const bars = ctx.bars;
  uint64_t* const cbar = ctx.cbar;
  float* const rowmax = ctx.rowmax;
  const float2* const tw = ctx.tw;
  const uint32_t tm = ctx.tm, lanes = ctx.lanes;
  uint32_t& parity = ctx.parity;
  bool& consts_ready = ctx.consts_ready;
  const uint32_t s_op = umma::smem_u32(op), s_lo = s_op + S::OP_BYTES;
  const uint32_t s_ba = umma::smem_u32(sm), s_bb = s_ba + S::BA_BYTES, s_bh = s_bb + S::BB_BYTES;
  constexpr uint32_t LO = SPLIT ? S::MAT_BYTES : 0;
  bool ok = true;

  // wait for the group's last commit (one poller), then agree on the outcome
  auto await = [&]() {
    bool w = true;
    if (tq == 0) {
      w = umma::mbar_wait(bars + g, parity, kSpin, kSuspendNs);
      if (!w) {
        atomicExch(err, 1);
        umma::mbar_wait(bars + g, parity, kSpin, kSuspendNs);
      }
    }
    parity ^= 1;
    ok = group_bar_and(g, w);
    umma::fence_after_sync();
  };
  // operands written -> visible to the tensor core; earlier tensor-memory reads ordered before the next MMA
  auto publish = [&]() {
    umma::fence_smem_to_async();
    umma::fence_before_sync();
    group_bar(g);
  };
  const int n0 = d.n0, n1 = d.n1;

  const int rr = kHalfN1 ? wq : gw;      // this warp's row in the tile (first and last stage)
  const int n1w = kHalfN1 ? KH * hh : 0;  // its first n1 on input (NH hh on output)
  const int pa = kHalfN1 ? 0 : hh;        // its first / last stage product

  // ---- input x chirp (steps 2-3), row normalisation, stage-A operand (K-major).
  // With 4-row tiles a row's maximum is combined with the other half's
  // through shared memory.
  float inv_scale;
  {
    const int row = row0 + rr;
    const bool valid = row < d.rows;
    float2 x[KH];
    float mx = 0.f;
    if constexpr (KIND == PASS_X_REAL) {
      // loads first; the store thread releases the previous x tile while they are in flight
      float u[KH];
#pragma unroll
      for (int i = 0; i < KH; ++i) {
        const int n = kR2 * (n1w + i) + l;
        const bool in = valid && n < n0;
        x[i] = in ? __ldg(d.cin + n) : make_float2(0.f, 0.f);
        u[i] = in ? ld_src<COHERENT>(static_cast<const float*>(d.src) + (size_t)row * d.src_ld + n) : 0.f;
      }
      if (signal && tq == kStoreTq) signal_tile(signal);
#pragma unroll
      for (int i = 0; i < KH; ++i) {
        x[i] = cscale(x[i], u[i]);
        mx = fmaxf(mx, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
      }
    } else {
#pragma unroll
      for (int i = 0; i < KH; ++i) {
        const int n = kR2 * (n1w + i) + l;
        float2 v = make_float2(0.f, 0.f);
        if (valid && n < n0) {
          const float2 c = __ldg(d.cin + n);
          v = cmul(ld_src<COHERENT>(static_cast<const float2*>(d.src) + (size_t)row * d.src_ld + n), c);
        }
        x[i] = v;
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
      if (signal && tq == kStoreTq) signal_tile(signal);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (l == 0) rowmax[gw] = mx;
    // the previous tile's tensor stores have read the buffer (a release above waited for all of them)
    if (tq == kStoreTq && !signal) umma::bulk_wait_read();
    group_bar(g);
    if constexpr (kHalfN1) mx = fmaxf(mx, rowmax[gw ^ 4]);
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    const float s = ldexpf(1.f, -e);  // max * s in [0.5, 1)
    inv_scale = ldexpf(1.f, e);
    const int m = 32 * wq + l;
#pragma unroll
    for (int c = 0; c < KH / 8; ++c) {
      float re[8], im[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        re[j] = x[8 * c + j].x * s;
        im[j] = x[8 * c + j].y * s;
      }
      store8<L, PREC>(op + pa * S::A_PROD_BYTES, kmaj_off(m, n1w + 8 * c), re);
      store8<L, PREC>(op + pa * S::A_PROD_BYTES, kmaj_off(m, KA + n1w + 8 * c), im);
    }
  }
  if (!consts_ready) {  // first tile: every thread sees the constant image before using it
    bool w = umma::mbar_wait(cbar, 0, kSpin, kSuspendNs);
    if (!w && threadIdx.x == 0) {
      atomicExch(err, 1);
      umma::mbar_wait(cbar, 0, kSpin, kSuspendNs);
    }
    consts_ready = true;
    ok = group_bar_and(g, w);
    if (!ok) return false;
  }
  publish();
  if (tq == 0) {
    umma::fence_after_sync();
#pragma unroll
    for (int a = 0; a < S::QA; ++a)
      gemm<SPLIT, false>(tm + 64 * a, s_op + a * S::A_PROD_BYTES, s_lo + a * S::A_PROD_BYTES, S::A_K, s_ba,
                         s_ba + LO, S::A_N, S::A_K / 16, umma::idesc_f16(128, S::A_N, BF, false, false));
    umma::commit(bars + g);
  }
  await();
  if (!ok) return false;

  // ---- twiddle W_L^{n2 k1}; stage-B operand rows (r', k1), K = n2 (MN-major).
  // Lane (r = rr, n2 = l) of first-stage product pa; with 4-row tiles warp half hh
  // takes k1 in [R1/2 hh, R1/2 hh + R1/2), with 8-row tiles every k1.
  {
    constexpr int JW = kHalfN1 ? R1 / 32 : R1 / 16;  // 16-column chunks per warp
    const int q = rr / S::RP, rp = rr % S::RP;        // middle-stage product and row in it
    unsigned char* opq = op + q * 128 * S::B_K * 2;
    const uint32_t ta = tm + 64 * pa;
#pragma unroll
    for (int jj = 0; jj < JW; ++jj) {
      const int j = (kHalfN1 ? JW * hh : 0) + jj;
      float re[16], im[16];
      umma::tmem_ld16(ta + lanes + 16 * j, re);
      umma::tmem_ld16(ta + lanes + R1 + 16 * j, im);
      umma::tmem_wait_ld();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float yr[8], yi[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k1 = 16 * j + 8 * h + i;
          const float2 y = cmul(make_float2(re[8 * h + i], im[8 * h + i]), tw[k1 * S::TW_LD + l]);
          yr[i] = y.x;
          yi[i] = y.y;
        }
        const int m = R1 * rp + 16 * j + 8 * h;
        store8<L, PREC>(opq, mnmaj_off(m, l, S::B_K), yr);
        store8<L, PREC>(opq, mnmaj_off(m, kR2 + l, S::B_K), yi);
      }
    }
  }
  publish();
  if (tq == 0) {
    umma::fence_after_sync();
#pragma unroll
    for (int q = 0; q < S::QB; ++q)
      gemm<SPLIT, true>(tm + 64 * q, s_op + q * 128 * S::B_K * 2, s_lo + q * 128 * S::B_K * 2, S::B_K, s_bb,
                        s_bb + LO, S::B_N, S::B_K / 16, umma::idesc_f16(128, S::B_N, BF, true, false));
    umma::commit(bars + g);
  }
  // the spectrum loads overlap the products: this thread's k1, k2 in [CH hh, CH hh + CH)
  float2 hsp[CH];
  {
    const int k1 = (32 * wq + l) % R1;  // lane (rp, k1) of a middle-stage product
#pragma unroll
    for (int i = 0; i < CH; ++i) hsp[i] = __ldg(d.H + k1 + R1 * (CH * hh + i));
  }
  await();
  if (!ok) return false;

  // ---- x kernel spectrum (step 7), conjugated: stage-B^H operand rows (r', k1), K = k2 (K-major).
  // Warp half hh takes k2 in [CH hh, CH hh + CH).
  {
    const int m = 32 * wq + l;
    const int c = hh;
#pragma unroll
    for (int q = 0; q < S::QB; ++q) {
      float re[16], im[16];
      umma::tmem_ld16(tm + lanes + 64 * q + 16 * c, re);
      umma::tmem_ld16(tm + lanes + 64 * q + kR2 + 16 * c, im);
      umma::tmem_wait_ld();
      unsigned char* opq = op + q * 128 * S::B_K * 2;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float yr[8], yi[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float2 y = cmul(make_float2(re[8 * h + i], im[8 * h + i]), hsp[8 * h + i]);
          yr[i] = y.x;
          yi[i] = -y.y;
        }
        store8<L, PREC>(opq, kmaj_off(m, 16 * c + 8 * h), yr);
        store8<L, PREC>(opq, kmaj_off(m, kR2 + 16 * c + 8 * h), yi);
      }
    }
  }
  publish();
  if (tq == 0) {
    umma::fence_after_sync();
#pragma unroll
    for (int q = 0; q < S::QB; ++q)
      gemm<SPLIT, false>(tm + 64 * q, s_op + q * 128 * S::B_K * 2, s_lo + q * 128 * S::B_K * 2, S::B_K, s_bb,
                         s_bb + LO, S::B_N, S::B_K / 16, umma::idesc_f16(128, S::B_N, BF, false, false));
    umma::commit(bars + g);
  }
  await();
  if (!ok) return false;

  // ---- twiddle W_L^{n2 k1}: stage-A^H operand rows (r, n2), K = k1 (MN-major).
  // Lane (r', k1); warp half hh takes n2 in [CH hh, CH hh + CH).
  {
    const int k1 = (32 * wq + l) % R1;  // lane (rp, k1) of product q: row r = RP q + rp
    const int c = hh;
#pragma unroll
    for (int q = 0; q < S::QB; ++q) {
      const int r = S::RP * q + (32 * wq + l) / R1;
      float re[16], im[16];
      umma::tmem_ld16(tm + lanes + 64 * q + 16 * c, re);
      umma::tmem_ld16(tm + lanes + 64 * q + kR2 + 16 * c, im);
      umma::tmem_wait_ld();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float yr[8], yi[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int n2 = 16 * c + 8 * h + i;
          const float2 y = cmul(make_float2(re[8 * h + i], im[8 * h + i]), tw[k1 * S::TW_LD + n2]);
          yr[i] = y.x;
          yi[i] = y.y;
        }
        // row r of the tile sits in last-stage product r / 4 (one product for 4-row tiles)
        unsigned char* const oph = op + (r / 4) * S::AH_PROD_BYTES;
        const int m = kR2 * (r % 4) + 16 * c + 8 * h;
        store8<L, PREC>(oph, mnmaj_off(m, k1, S::H_K), yr);
        store8<L, PREC>(oph, mnmaj_off(m, R1 + k1, S::H_K), yi);
      }
    }
  }
  publish();
  if (tq == 0) {
    umma::fence_after_sync();
#pragma unroll
    for (int a = 0; a < S::QA; ++a)
      gemm<SPLIT, true>(tm + 64 * a, s_op + a * S::AH_PROD_BYTES, s_lo + a * S::AH_PROD_BYTES, S::H_K, s_bh,
                        s_bh + LO, S::H_N, S::H_K / 16, umma::idesc_f16(128, S::H_N, BF, true, false));
    umma::commit(bars + g);
  }
  // the output-chirp loads overlap the product: this thread's n1 in [n1w', n1w' + NH)
  const int n1o = kHalfN1 ? NH * hh : 0;
  float2 co[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    const int n = kR2 * (n1o + i) + l;
    co[i] = n < n1 ? __ldg(d.cout + n) : make_float2(0.f, 0.f);
  }
  await();
  if (!ok) return false;

  // ---- conj, undo the scales, x output chirp (step 9): staged as [n][r] float2 (the tensor-store box)
  {
    // the three 1/sqrt(L) stage scales (the output chirp carries the transform's 1/L)
    const float sc = inv_scale * (float)L * sqrtf((float)L);
    float2* stage = reinterpret_cast<float2*>(op);
    const uint32_t ta = tm + 64 * pa;  // this warp's last-stage product
#pragma unroll
    for (int c = 0; c < NH / 8; ++c) {
      float re[8], im[8];
      umma::tmem_ld8(ta + lanes + n1o + 8 * c, re);
      umma::tmem_ld8(ta + lanes + NA + n1o + 8 * c, im);
      umma::tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = kR2 * (n1o + 8 * c + i) + l;
        if (n < n1) stage[stage_idx<TR>(n, rr)] = cmul(make_float2(re[i] * sc, -im[i] * sc), co[8 * c + i]);
      }
    }
  }
  umma::fence_smem_to_async();
  umma::fence_before_sync();
  group_bar(g);
  // ---- transposed store: output n of row r to dst[n * dst_ld + row0 + r]
  if (out_map) {
    // tensor stores of kOutBoxN outputs x TR rows, clipped to the pass's rows and n1; they
    // complete in the background, and the buffer is next written after the wait above
    if (tq == kStoreTq) {
      for (int j = 0; j * kOutBoxN < n1; ++j)
        umma::tma_store_2d(out_map, op + j * kOutBoxN * TR * 8, 2 * row0, j * kOutBoxN);
      umma::bulk_commit();
    }
  } else {
    const float2* stage = reinterpret_cast<const float2*>(op);
    const int rows_here = min(TR, d.rows - row0);
    float2* const dst = d.dst;
    float* const inten = d.inten;
    float* const phase = d.phase;
    const size_t ld = (size_t)d.dst_ld;
    const bool acc = d.accumulate != 0;
    for (int i = tq; i < n1 * TR; i += kGroupThreads) {
      const int n = i / TR, r = i % TR;
      if (r < rows_here) {
        const float2 u = stage[stage_idx<TR>(n, r)];
        const size_t o = (size_t)n * ld + row0 + r;
        if constexpr (KIND != PASS_Y) {
          dst[o] = u;
        } else {
          if (dst) dst[o] = acc ? cadd(dst[o], u) : u;
          if (inten) inten[o] = fmaf(u.x, u.x, u.y * u.y);
          if (phase) phase[o] = phase_of(u);
        }
      }
    }
    group_bar(g);  // the staging tile is the next tile's operand buffer
  }
  return true;
}

template <int L, int KIND, int PREC>
__global__ void __launch_bounds__(Prec<PREC>::kThreads, 1)
k_pass_t5(const __grid_constant__ PassBatch b, const __grid_constant__ Args a) {
  constexpr int kGroups = Prec<PREC>::kGroups;
  extern __shared__ __align__(1024) unsigned char sm[];
  GroupCtx<L, PREC> c = group_setup<L, PREC>(sm, reinterpret_cast<const uint4*>(a.consts));
  // tiles CTA-major (a CTA's groups on neighbouring rows) when every group has one, else group-major, so
  // that a launch with fewer tiles than groups spreads them over every SM
  const bool full = a.total_tiles >= (int)gridDim.x * kGroups;
  for (int tile = full ? blockIdx.x * kGroups + c.g : c.g * gridDim.x + blockIdx.x; tile < a.total_tiles;
       tile += gridDim.x * kGroups) {
    int p = 0;
    while (tile >= a.tile_off[p + 1]) ++p;
    if (!tile_t5<L, KIND, PREC, false>(c, sm, b.d[p], (tile - a.tile_off[p]) * Shape<L>::TR,
                                       a.tma_store[p] ? &a.out_map[p] : nullptr, a.err))
      break;
  }
  group_teardown<L, PREC>(sm, c);
}

// Both passes of up to kMaxPassBatch / 2 views in one persistent launch.
// Passes 0 .. nx - 1 are the views' x passes, nx .. 2 nx - 1 their y passes
// (same view order).  Groups claim tiles in order from a global counter, so
// every x tile is claimed before any y tile; a y tile of view v waits
// (bounded) until all x tiles of view v have signalled that their part of the
// intermediate is written.  x tiles never wait, so the claims cannot
// deadlock even when not every CTA of the grid is resident.
struct FuseArgs {
  int* sched;            // [0]: next tile to claim, [1 + v]: completed x tiles of view v; zero at launch
  int nx;                // views
  int poison_view;       // -1; a view index makes its y tiles' dependency unsatisfiable (tests)
  long long spin_limit;  // polls of a y tile's dependency wait before it gives up
};

// Bounded wait until *ctr >= need (acquire at GPU scope); false (err set) when it gives up.
__device__ __forceinline__ bool wait_count(const int* ctr, int need, int* err, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= need) return true;
    __nanosleep(kDepSleepNs);
  }
  atomicExch(err, 1);
  return false;
}

template <int L, int KIND_X, int PREC>
__global__ void __launch_bounds__(Prec<PREC>::kThreads, 1)
k_views_t5(const __grid_constant__ PassBatch b, const __grid_constant__ Args a, const FuseArgs f) {
  extern __shared__ __align__(1024) unsigned char sm[];
  GroupCtx<L, PREC> c = group_setup<L, PREC>(sm, reinterpret_cast<const uint4*>(a.consts));
  int* const claim = reinterpret_cast<int*>(sm + Shape<L>::misc_offset(Prec<PREC>::kSplit) + 192);
  int* pending = nullptr;  // the group's last x tile, released by its store thread at the next tile
  for (;;) {
    if (c.tq == 0) claim[c.g] = atomicAdd(f.sched, 1);
    group_bar(c.g);  // every thread reads the claim before the tile's next barrier
    const int tile = claim[c.g];
    if (tile >= a.total_tiles) break;
    int p = 0;
    while (tile >= a.tile_off[p + 1]) ++p;
    const int row0 = (tile - a.tile_off[p]) * Shape<L>::TR;
    const CUtensorMap* om = a.tma_store[p] ? &a.out_map[p] : nullptr;
    if (p < f.nx) {
      int* const prev = pending;  // released inside the tile, once its input loads are in flight
      pending = nullptr;
      if (!tile_t5<L, KIND_X, PREC, false>(c, sm, b.d[p], row0, om, a.err, prev)) break;
      pending = f.sched + 1 + p;
    } else {
      const int v = p - f.nx;
      bool w = true;
      // the pending release first: this group may hold one of the tiles waited for
      if (c.tq == kStoreTq && pending) signal_tile(pending);
      pending = nullptr;
      if (c.tq == 0) {
        const int need = v == f.poison_view ? 0x7fffffff : a.tile_off[v + 1] - a.tile_off[v];
        w = wait_count(f.sched + 1 + v, need, a.err, f.spin_limit);
      }
      if (!group_bar_and(c.g, w)) break;
      if (!tile_t5<L, PASS_Y, PREC, true>(c, sm, b.d[p], row0, om, a.err)) break;
    }
  }
  if (c.tq == kStoreTq && pending) signal_tile(pending);
  group_teardown<L, PREC>(sm, c);
}

// Natural-order kernel spectrum scaled by 1/sqrt(L), from the FP32 network's
// register order: position p of that network holds frequency
// f(p) = sum_s k_s R_0 ... R_{s-1} with k_s = (p / M_s) mod R_s (its radix-16
// decimation-in-frequency digits, least significant first).
template <int L>
__global__ void k_hnat(const float2* __restrict__ Hreg, float2* __restrict__ Hn) {
  constexpr int T = L / kE;
  const float hs = rsqrtf((float)L);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const int p = last_pos<L, kE>(t, e);
    int f = 0, w = 1, M = L;
    while (M > 1) {  // stages of radix min(M', 16)
      const int R = M > kE ? kE : M;
      M /= R;
      f += ((p / M) % R) * w;
      w *= R;
    }
    const float2 h = Hreg[e * T + t];
    Hn[f] = make_float2(h.x * hs, h.y * hs);
  }
}

template <int L, int PREC>
cudaError_t launch_t(PassKind kind, const PassBatch& b, const Args& a, int grid, cudaStream_t s) {
  constexpr int smem = Shape<L>::smem_bytes(Prec<PREC>::kSplit);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, Prec<PREC>::kThreads, smem, s>>>(b, a);
    return cudaGetLastError();
  };
  switch (kind) {
    case PASS_X_REAL: return go(k_pass_t5<L, PASS_X_REAL, PREC>);
    case PASS_X_CPLX: return go(k_pass_t5<L, PASS_X_CPLX, PREC>);
    case PASS_Y: return go(k_pass_t5<L, PASS_Y, PREC>);
  }
  return cudaErrorInvalidValue;
}

template <int L, int PREC>
cudaError_t launch_fused_t(PassKind kind_x, const PassBatch& b, const Args& a, const FuseArgs& f, int grid,
                           cudaStream_t s) {
  constexpr int smem = Shape<L>::smem_bytes(Prec<PREC>::kSplit);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, Prec<PREC>::kThreads, smem, s>>>(b, a, f);
    return cudaGetLastError();
  };
  if (kind_x == PASS_X_REAL) return go(k_views_t5<L, PASS_X_REAL, PREC>);
  if (kind_x == PASS_X_CPLX) return go(k_views_t5<L, PASS_X_CPLX, PREC>);
  return cudaErrorInvalidValue;
}

// host: 16-bit value of v (round to nearest even) and the remainder v - value
uint16_t to16(double v, bool bf16, double& rem) {
  if (bf16) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
    rem = v - (double)__bfloat162float(h);
    uint16_t r;
    std::memcpy(&r, &h, 2);
    return r;
  }
  const __half h = __float2half_rn((float)v);
  rem = v - (double)__half2float(h);
  uint16_t r;
  std::memcpy(&r, &h, 2);
  return r;
}

// Real block form of the unitary DFT of size R restricted to kin inputs and
// nout outputs, as a K-major B operand image (N = 2 nout rows of K = 2 kin):
// B[(s, i)][(t, o)], s, t in {re, im}: [re][re] = [im][im] = cos, [re][im] =
// -sin, [im][re] = sin of 2 pi i o / R, all over sqrt(R).
void dft_operand(int R, int kin, int nout, bool bf16, uint16_t* hi, uint16_t* lo) {
  const double sc = 1.0 / std::sqrt((double)R);
  for (int t = 0; t < 2; ++t)
    for (int o = 0; o < nout; ++o)
      for (int s = 0; s < 2; ++s)
        for (int i = 0; i < kin; ++i) {
          const double ang = 2.0 * M_PI * (double)(((long long)i * o) % R) / R;
          const double c = std::cos(ang) * sc, sn = -std::sin(ang) * sc;  // W_R^{i o} = c + i sn
          const double v = (s == t) ? c : (s == 0 ? sn : -sn);
          const int n = t * nout + o, kk = s * kin + i;
          double rem, rem2;
          const int off = kmaj_off(n, kk) / 2;
          hi[off] = to16(v, bf16, rem);
          if (lo) lo[off] = to16(rem, bf16, rem2);
        }
}

}  // namespace t5

bool t5_length_supported(int L) { return L == 512 || L == 1024 || L == 2048; }

namespace {
int t5_tile_rows(int L) { return L == 512 ? t5::Shape<512>::TR : 4; }
}  // namespace
bool t5_precision(int prec) {
  return prec == SF_PREC_FP16TC || prec == SF_PREC_BF16TC || prec == SF_PREC_FP16X3TC || prec == SF_PREC_BF16X3TC;
}

namespace {
template <int L>
void build_consts_t(int prec, unsigned char* base) {
  using S = t5::Shape<L>;
  const bool split = prec == SF_PREC_FP16X3TC || prec == SF_PREC_BF16X3TC;
  const bool bf16 = prec == SF_PREC_BF16TC || prec == SF_PREC_BF16X3TC;
  std::memset(base, 0, S::const_bytes(split));
  uint16_t* hi = reinterpret_cast<uint16_t*>(base);
  uint16_t* lo = split ? reinterpret_cast<uint16_t*>(base + S::MAT_BYTES) : nullptr;
  const int o1 = S::BA_BYTES / 2, o2 = (S::BA_BYTES + S::BB_BYTES) / 2;
  t5::dft_operand(S::R1, S::KA, S::R1, bf16, hi, lo);                               // stage A
  t5::dft_operand(t5::kR2, t5::kR2, t5::kR2, bf16, hi + o1, lo ? lo + o1 : nullptr);  // stages B, B^H
  t5::dft_operand(S::R1, S::R1, S::NA, bf16, hi + o2, lo ? lo + o2 : nullptr);       // stage A^H
  float2* tw = reinterpret_cast<float2*>(base + (split ? 2 : 1) * S::MAT_BYTES);
  for (int k1 = 0; k1 < S::R1; ++k1)
    for (int n2 = 0; n2 < t5::kR2; ++n2) {
      const double ang = -2.0 * M_PI * (double)(k1 * n2) / (double)L;
      tw[k1 * S::TW_LD + n2] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
}
}  // namespace

size_t t5_const_bytes(int L, int prec) {
  const bool split = prec == SF_PREC_FP16X3TC || prec == SF_PREC_BF16X3TC;
  if (L == 512) return (size_t)t5::Shape<512>::const_bytes(split);
  if (L == 1024) return (size_t)t5::Shape<1024>::const_bytes(split);
  if (L == 2048) return (size_t)t5::Shape<2048>::const_bytes(split);
  return 0;
}

void t5_build_consts(int L, int prec, void* host) {
  if (L == 512) build_consts_t<512>(prec, static_cast<unsigned char*>(host));
  if (L == 1024) build_consts_t<1024>(prec, static_cast<unsigned char*>(host));
  if (L == 2048) build_consts_t<2048>(prec, static_cast<unsigned char*>(host));
}

cudaError_t launch_hnat(int L, const float2* Hreg, float2* Hn, cudaStream_t s) {
  if (L == 512) t5::k_hnat<512><<<1, 512 / kE, 0, s>>>(Hreg, Hn);
  else if (L == 1024) t5::k_hnat<1024><<<1, 1024 / kE, 0, s>>>(Hreg, Hn);
  else if (L == 2048) t5::k_hnat<2048><<<1, 2048 / kE, 0, s>>>(Hreg, Hn);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_pass_t5(int L, int prec, PassKind kind, const PassBatch& b, const void* consts, int* err, int sms,
                           cudaStream_t s) {
  if (!t5_length_supported(L)) return cudaErrorInvalidValue;
  t5::Args a{};
  a.consts = static_cast<const uint4*>(consts);
  a.err = err;
  a.tile_off[0] = 0;
  const int TR = t5_tile_rows(L);
  for (int k = 0; k < b.count; ++k) a.tile_off[k + 1] = a.tile_off[k] + (b.d[k].rows + TR - 1) / TR;
  for (int k = b.count; k < kMaxPassBatch; ++k) a.tile_off[k + 1] = a.tile_off[k];
  a.total_tiles = a.tile_off[b.count];
  for (int k = 0; k < b.count; ++k)
    a.tma_store[k] = output_tensor_map(kind, b.d[k], TR, &a.out_map[k], TR == 4) ? 1 : 0;
  if (a.total_tiles == 0) return cudaSuccess;
  const int grid = std::min(sms, a.total_tiles);  // every SM that can have a tile gets one
#define SF_T5_PREC_CASES(LL)                                                                  \
  switch (prec) {                                                                              \
    case SF_PREC_FP16TC: return t5::launch_t<LL, SF_PREC_FP16TC>(kind, b, a, grid, s);         \
    case SF_PREC_BF16TC: return t5::launch_t<LL, SF_PREC_BF16TC>(kind, b, a, grid, s);         \
    case SF_PREC_FP16X3TC: return t5::launch_t<LL, SF_PREC_FP16X3TC>(kind, b, a, grid, s);     \
    case SF_PREC_BF16X3TC: return t5::launch_t<LL, SF_PREC_BF16X3TC>(kind, b, a, grid, s);     \
  }
  if (L == 512) SF_T5_PREC_CASES(512)
  if (L == 1024) SF_T5_PREC_CASES(1024)
  if (L == 2048) SF_T5_PREC_CASES(2048)
#undef SF_T5_PREC_CASES
  return cudaErrorInvalidValue;
}

cudaError_t launch_views_t5(int L, int prec, PassKind kind_x, const PassBatch& b, int nx, const void* consts, int* err,
                            int* sched, int sms, cudaStream_t s) {
  if (!t5_length_supported(L) || nx <= 0 || 2 * nx != b.count || kind_x == PASS_Y) return cudaErrorInvalidValue;
  t5::Args a{};
  a.consts = static_cast<const uint4*>(consts);
  a.err = err;
  a.tile_off[0] = 0;
  const int TR = t5_tile_rows(L);
  for (int k = 0; k < b.count; ++k) a.tile_off[k + 1] = a.tile_off[k] + (b.d[k].rows + TR - 1) / TR;
  for (int k = b.count; k < kMaxPassBatch; ++k) a.tile_off[k + 1] = a.tile_off[k];
  a.total_tiles = a.tile_off[b.count];
  for (int k = 0; k < b.count; ++k)
    a.tma_store[k] = output_tensor_map(k < nx ? kind_x : PASS_Y, b.d[k], TR, &a.out_map[k], TR == 4) ? 1 : 0;
  if (a.total_tiles == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(sched, 0, sizeof(int) * (1 + nx), s);
  if (e != cudaSuccess) return e;
  // SF_T5_POISON_VIEW / SF_T5_SPIN_LIMIT: an unsatisfiable dependency and a short wait (tests)
  const char* pv = std::getenv("SF_T5_POISON_VIEW");
  const char* sl = std::getenv("SF_T5_SPIN_LIMIT");
  const t5::FuseArgs f{sched, nx, pv && *pv ? std::atoi(pv) : -1, sl && *sl ? std::atoll(sl) : t5::kDepSpin};
  const int grid = std::min(sms, a.total_tiles);  // every SM that can have a tile gets one
  // FP16 / BF16 only (the x3 precisions run one launch per pass)
  switch (prec) {
    case SF_PREC_FP16TC:
      return L == 512    ? t5::launch_fused_t<512, SF_PREC_FP16TC>(kind_x, b, a, f, grid, s)
             : L == 1024 ? t5::launch_fused_t<1024, SF_PREC_FP16TC>(kind_x, b, a, f, grid, s)
                         : t5::launch_fused_t<2048, SF_PREC_FP16TC>(kind_x, b, a, f, grid, s);
    case SF_PREC_BF16TC:
      return L == 512    ? t5::launch_fused_t<512, SF_PREC_BF16TC>(kind_x, b, a, f, grid, s)
             : L == 1024 ? t5::launch_fused_t<1024, SF_PREC_BF16TC>(kind_x, b, a, f, grid, s)
                         : t5::launch_fused_t<2048, SF_PREC_BF16TC>(kind_x, b, a, f, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sf

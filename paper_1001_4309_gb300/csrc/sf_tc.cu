// sf_tc.cu -- mixed-precision row pass: the radix-16 / radix-8 DFT stages of
// the FFT network as half-precision tensor-core matrix products
// (mma.sync m16n8k16, FP16 or BF16 operands, FP32 accumulation).
//
// Same positions, stages and twiddles as the FP32 network (sf_fft.cuh); only
// the radix-R DFTs move to the tensor cores.  Stage s is the real GEMM
//
//   C (2R x L/R) = A_R (2R x 2R) * B (2R x L/R)
//
// with A_R the real block [[Wr, -Wi], [Wi, Wr]] / sqrt(R) of the radix-R DFT
// matrix (its conjugate for the inverse; the unitary scale keeps values in
// half-precision range) and column b of B the 2R real inputs of butterfly b
// (re of elements 0..R-1, then im).
//
// Shared-memory layout: per row, a real plane and an imaginary plane of L
// halves indexed by network position p (the same positions as the FP32
// network), with 16-byte chunks XOR-swizzled (swz) so that every access
// below is free of bank conflicts.  Butterfly b of stage s reads element j
// at p = (b / M) M' + b % M + j M.  When M >= 8, eight consecutive
// butterflies read eight consecutive positions for each j, so the B operand
// of an 8-butterfly tile is eight 16-byte rows indexed by j: ldmatrix.trans.
// When M = 1 (the last stage) a butterfly's R elements are consecutive:
// plain ldmatrix with rows indexed by butterfly.  The accumulator of a lane
// holds outputs (k, b) and (k, b + 1): for M >= 2 these sit at consecutive
// positions, so the epilogue (FP32 twiddle, conversion) stores one 4-byte
// pair per plane.
//
// Epilogues: forward stage s multiplies by its twiddle W_{M'}^{n k}; the last
// forward stage multiplies by the kernel spectrum in position order (scaled
// by 1/sqrt(L)); inverse stage s (conjugate DFT) multiplies by the conjugated
// twiddle of stage s - 1, since the adjoint network applies it before that
// stage's DFT; the last inverse stage undoes the three 1/sqrt(L) scales and
// the row normalisation, applies the output chirp and stores the row.  Rows
// are normalised by their largest input component before the first
// conversion to half precision.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sf_kernels.cuh"

namespace sf {
namespace tc {

constexpr int kThreads = 256;  // 8 warps
// unroll of the per-warp tile loop (measured best at 2048 within the
// register budget of three CTAs per SM; 4096 spills beyond 2)
template <int L>
__host__ __device__ constexpr int unroll_of() { return L == 2048 ? 4 : 2; }
// rows per CTA: 64 KiB of half-precision buffers per CTA at either length
template <int L>
__host__ __device__ constexpr int rows_of() { return L == 4096 ? 2 : 4; }
// CTAs per SM the register budget is set for (shared memory allows three)
template <int L>
__host__ __device__ constexpr int ctas_of() { return 3; }

// swizzled half index of position p within a plane (bijective on 0..L-1)
__host__ __device__ constexpr int swz(int p) {
  return (((p >> 3) ^ (((p >> 6) ^ (p >> 9)) & 7)) << 3) | (p & 7);
}

template <int L>
struct TcShape {
  static constexpr int kRows = rows_of<L>();
  static constexpr int BUF = 2 * kRows * L;  // halves per buffer: re and im planes of kRows rows
  static constexpr size_t SMEM = sizeof(uint16_t) * 2 * (size_t)BUF + 16 * kRows;
  // the output tile [n1][kRows] (float2) is staged in the free buffer when it fits
  static constexpr int TILE_N1 = (int)(sizeof(uint16_t) * BUF / (sizeof(float2) * kRows));
};

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (PREC == SF_PREC_BF16TC) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

template <int PREC>
__device__ __forceinline__ uint16_t pack1(float v) {
  if constexpr (PREC == SF_PREC_BF16TC) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
  } else {
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
  }
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (PREC == SF_PREC_BF16TC) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

template <bool TRANS>
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const uint16_t* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  if constexpr (TRANS)
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
  else
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

template <bool TRANS>
__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[4], const uint16_t* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  if constexpr (TRANS)
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
  else
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

template <int L, int S>
__device__ __forceinline__ int pos_of(int b, int k) {
  using St = Stage<L, kTcE, S>;
  return (b / St::M) * St::MP + (b % St::M) + k * St::M;
}

// Twiddle tables of the tensor-core network, stage s (with M > 1) as
// [k][n] = W_{M'}^{n k}, n < M, k < R, complex FP32; stages concatenated.
template <int L>
__host__ __device__ constexpr int tw_offset(int S) {
  int o = 0;
  for (int i = 0; i < S; ++i)
    o += (stage_mprev(L, kTcE, i) / stage_radix(L, kTcE, i)) > 1 ? stage_mprev(L, kTcE, i) : 0;
  return o;
}
template <int L>
__host__ __device__ constexpr int tw_entries() { return tw_offset<L>(stage_count(L, kTcE)); }

// Per-lane A fragments: [dir][mt][kt][q][lane] for radix 16, then for radix 8.
__host__ __device__ constexpr int frag_words(int R) { return 2 * (R / 8) * (R / 8) * 4 * 32; }

__device__ __forceinline__ uint16_t* plane(uint16_t* buf, int L, int row, int im) {
  return buf + (row * 2 + im) * L;
}

// Store butterflies b, b + 1 of one output element at positions p, p + 1
// (p even): X = their real parts, Y = their imaginary parts.
template <int L, int PREC>
__device__ __forceinline__ void put_pair(uint16_t* buf, int row, int p, float2 X, float2 Y) {
  const int a = swz(p);
  *reinterpret_cast<uint32_t*>(plane(buf, L, row, 0) + a) = pack2<PREC>(X.x, X.y);
  *reinterpret_cast<uint32_t*>(plane(buf, L, row, 1) + a) = pack2<PREC>(Y.x, Y.y);
}

template <int L, int PREC>
__device__ __forceinline__ void put_one(uint16_t* buf, int row, int p, float2 v) {
  const int a = swz(p);
  plane(buf, L, row, 0)[a] = pack1<PREC>(v.x);
  plane(buf, L, row, 1)[a] = pack1<PREC>(v.y);
}

// (X + i Y) * (WX + i WY) for two values at once (packed f32x2 arithmetic);
// CONJ multiplies by the conjugate.  The results overwrite X and Y.
template <bool CONJ>
__device__ __forceinline__ void cmul_pair(float2& X, float2& Y, float2 WX, float2 WY) {
  const float2 nwy = __fmul2_rn(WY, make_float2(-1.f, -1.f));
  float2 re, im;
  if constexpr (!CONJ) {
    re = __ffma2_rn(Y, nwy, __fmul2_rn(X, WX));  // X WX - Y WY
    im = __ffma2_rn(X, WY, __fmul2_rn(Y, WX));   // X WY + Y WX
  } else {
    re = __ffma2_rn(Y, WY, __fmul2_rn(X, WX));   // X WX + Y WY
    im = __ffma2_rn(X, nwy, __fmul2_rn(Y, WX));  // Y WX - X WY
  }
  X = re;
  Y = im;
}

// One stage's GEMM over all rows of the CTA.  Warp w takes n-tiles
// nt = 8 q + w of every row (q < NT / 8), so a tile's row and first
// butterfly are compile-time functions of the unrolled step.  Epilogue:
// epi(row, b, k, X, Y) with X / Y the real / imaginary parts of output k of
// butterflies b and b + 1.
template <int L, int S, int PREC, bool INV, typename Epi>
__device__ __forceinline__ void stage_gemm(uint16_t* in, const uint32_t* __restrict__ frags, Epi&& epi) {
  using St = Stage<L, kTcE, S>;
  constexpr int R = St::R, M = St::M;
  static_assert(R == 16 || R == 8, "tensor-core stages need radix 8 or 16");
  static_assert(M >= 8 || M == 1, "operand tiles need M >= 8 or M = 1");
  constexpr int NT = L / R / 8;   // n-tiles (8 butterflies) per row
  constexpr int Q = NT / 8;       // n-tiles per warp and row
  static_assert(NT % 8 == 0, "every warp takes the same number of tiles");
  constexpr int T2 = 2 * R / 16;  // m-tiles = k-steps of the real block
  constexpr bool TRANS = M >= 8;
  constexpr int kRows = rows_of<L>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const uint32_t* fp = frags + (R == 16 ? 0 : frag_words(16)) + (INV ? frag_words(R) / 2 : 0);
  uint32_t a[T2][T2][4];
#pragma unroll
  for (int mt = 0; mt < T2; ++mt)
#pragma unroll
    for (int kt = 0; kt < T2; ++kt)
#pragma unroll
      for (int q = 0; q < 4; ++q) a[mt][kt][q] = __ldg(fp + ((mt * T2 + kt) * 4 + q) * 32 + lane);
  // this lane's ldmatrix row: matrix m = lane / 8 (R = 16: re j 0-7, re j 8-15, im j 0-7, im j 8-15;
  // R = 8: re j 0-7, im j 0-7), row rr = lane % 8 (element j0 + rr, or butterfly b0 + rr when M = 1)
  const int m = (lane >> 3) & (R == 16 ? 3 : 1), rr = lane & 7;
  const int im = R == 16 ? (m >> 1) : m, j0 = R == 16 ? (m & 1) * 8 : 0;
#pragma unroll(unroll_of<L>())
  for (int i = 0; i < kRows * Q; ++i) {
    const int row = i / Q, b0 = 64 * (i % Q) + 8 * warp;
    const int p = TRANS ? pos_of<L, S>(b0, j0 + rr) : pos_of<L, S>(b0 + rr, j0);
    const uint16_t* src = plane(in, L, row, im) + swz(p);
    uint32_t bf[4];
    if constexpr (R == 16) ldsm_x4<TRANS>(bf, src);
    else ldsm_x2<TRANS>(bf, src);
    float c[T2][4];
#pragma unroll
    for (int mt = 0; mt < T2; ++mt) c[mt][0] = c[mt][1] = c[mt][2] = c[mt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < T2; ++kt)
#pragma unroll
      for (int mt = 0; mt < T2; ++mt) mma16816<PREC>(c[mt], a[mt][kt], bf[2 * kt], bf[2 * kt + 1]);
    const int bi = b0 + 2 * tig;
    if constexpr (R == 16) {
      // tile 0: re of elements 0..15, tile 1: im; rows g and g + 8, columns bi, bi + 1
      epi(row, bi, g, make_float2(c[0][0], c[0][1]), make_float2(c[1][0], c[1][1]));
      epi(row, bi, g + 8, make_float2(c[0][2], c[0][3]), make_float2(c[1][2], c[1][3]));
    } else {
      // one tile: row g = re of element g, row g + 8 = im of element g
      epi(row, bi, g, make_float2(c[0][0], c[0][1]), make_float2(c[0][2], c[0][3]));
    }
  }
}

// Forward stages S.. of the network; returns the buffer holding the last
// stage's positions after the spectrum multiply.  Twiddle tables hold, per
// (k, even n), the float4 (Re W_n, Re W_n+1, Im W_n, Im W_n+1).
template <int L, int S, int PREC>
__device__ __forceinline__ uint16_t* forward(uint16_t* cur, uint16_t* oth, const uint32_t* frags,
                                             const float2* __restrict__ tw, const float2* __restrict__ Hpos) {
  using St = Stage<L, kTcE, S>;
  constexpr int NS = stage_count(L, kTcE);
  if constexpr (S + 1 < NS) {
    static_assert(St::M >= 2, "twiddled stages pair adjacent butterflies");
    const float2* t = tw + tw_offset<L>(S);
    stage_gemm<L, S, PREC, false>(cur, frags, [&](int row, int b, int k, float2 X, float2 Y) {
      const float4 w = __ldg(reinterpret_cast<const float4*>(t + k * St::M + b % St::M));
      cmul_pair<false>(X, Y, make_float2(w.x, w.y), make_float2(w.z, w.w));
      put_pair<L, PREC>(oth, row, pos_of<L, S>(b, k), X, Y);
    });
    __syncthreads();
    return forward<L, S + 1, PREC>(oth, cur, frags, tw, Hpos);
  } else {
    static_assert(St::M == 1, "the last stage has unit stride");
    stage_gemm<L, S, PREC, false>(cur, frags, [&](int row, int b, int k, float2 X, float2 Y) {
      const int p0 = b * St::R + k, p1 = p0 + St::R;
      put_one<L, PREC>(oth, row, p0, cmul(make_float2(X.x, Y.x), __ldg(Hpos + p0)));
      put_one<L, PREC>(oth, row, p1, cmul(make_float2(X.y, Y.y), __ldg(Hpos + p1)));
    });
    __syncthreads();
    return oth;
  }
}

// Twiddle W of stage S at position p (any parity), from the paired table.
template <int L, int S>
__device__ __forceinline__ float2 twiddle_at(const float2* __restrict__ t, int p) {
  using St = Stage<L, kTcE, S>;
  const int idx = ((p % St::MP) / St::M) * St::M + p % St::M;
  const float4 w = __ldg(reinterpret_cast<const float4*>(t + (idx & ~1)));
  return (idx & 1) ? make_float2(w.y, w.w) : make_float2(w.x, w.z);
}

// Inverse stages S..0; the last one hands (row, position p, X, Y) for the
// natural, even position p and p + 1 to `out`.
template <int L, int S, int PREC, typename Out>
__device__ __forceinline__ void inverse(uint16_t* cur, uint16_t* oth, const uint32_t* frags,
                                        const float2* __restrict__ tw, Out&& out) {
  using St = Stage<L, kTcE, S>;
  if constexpr (S > 0) {
    using Sp = Stage<L, kTcE, S - 1>;
    const float2* t = tw + tw_offset<L>(S - 1);
    stage_gemm<L, S, PREC, true>(cur, frags, [&](int row, int b, int j, float2 X, float2 Y) {
      if constexpr (St::M >= 2) {
        // positions p, p + 1 of stage S - 1: n = p mod M, k = (p mod M') / M there
        const int p = pos_of<L, S>(b, j);
        const int n = p % Sp::M, k = (p % Sp::MP) / Sp::M;
        const float4 w = __ldg(reinterpret_cast<const float4*>(t + k * Sp::M + n));
        cmul_pair<true>(X, Y, make_float2(w.x, w.y), make_float2(w.z, w.w));
        put_pair<L, PREC>(oth, row, p, X, Y);
      } else {
        const int p0 = b * St::R + j, p1 = p0 + St::R;
        put_one<L, PREC>(oth, row, p0, cmulc(make_float2(X.x, Y.x), twiddle_at<L, S - 1>(t, p0)));
        put_one<L, PREC>(oth, row, p1, cmulc(make_float2(X.y, Y.y), twiddle_at<L, S - 1>(t, p1)));
      }
    });
    __syncthreads();
    inverse<L, S - 1, PREC>(oth, cur, frags, tw, out);
  } else {
    static_assert(St::M >= 2, "the first stage pairs adjacent positions");
    stage_gemm<L, 0, PREC, true>(cur, frags, [&](int row, int b, int j, float2 X, float2 Y) {
      out(row, pos_of<L, 0>(b, j), X, Y);
    });
  }
}

template <int L, int KIND, int PREC>
__global__ void __launch_bounds__(kThreads, ctas_of<L>())
k_pass_tc(const __grid_constant__ PassBatch pb, const float2* __restrict__ tw, const uint32_t* __restrict__ frags) {
  constexpr int kRows = rows_of<L>();
  extern __shared__ __align__(16) uint16_t sm[];
  constexpr int BUF = TcShape<L>::BUF;
  uint16_t* buf0 = sm;
  uint16_t* buf1 = sm + BUF;
  unsigned* rowmax = reinterpret_cast<unsigned*>(sm + 2 * BUF);
  const PassDesc& d = pb.d[blockIdx.y];
  const int row0 = blockIdx.x * kRows;
  if (row0 >= d.rows) return;
  const int tid = threadIdx.x, lane = tid & 31;

  auto load = [&](int row, int p) -> float2 {
    const float2 c = __ldg(reinterpret_cast<const float2*>(d.cin) + p);
    if constexpr (KIND == PASS_X_REAL) {
      const float x = __ldg(static_cast<const float*>(d.src) + (size_t)row * d.src_ld + p);
      return make_float2(c.x * x, c.y * x);
    } else {
      const float2 x = __ldg(static_cast<const float2*>(d.src) + (size_t)row * d.src_ld + p);
      return cmul(x, c);
    }
  };

  // 1. largest input component of each row
  if (tid < kRows) rowmax[tid] = 0u;
  __syncthreads();
  for (int r = 0; r < kRows; ++r) {
    const int row = row0 + r;
    float m = 0.f;
    if (row < d.rows)
      for (int p = tid; p < d.n0; p += kThreads) {
        const float2 v = load(row, p);
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m > 0.f) atomicMax(rowmax + r, __float_as_uint(m));
  }
  __syncthreads();
  // 2. normalised input at natural positions (stage 0's layout), pairs of positions, zero padding
  for (int r = 0; r < kRows; ++r) {
    const int row = row0 + r;
    const float mx = __uint_as_float(rowmax[r]);
    const float s0 = mx > 0.f ? 1.0f / mx : 0.f;
    for (int p = 2 * tid; p < L; p += 2 * kThreads) {
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (row < d.rows) {
        if (p < d.n0) v0 = load(row, p);
        if (p + 1 < d.n0) v1 = load(row, p + 1);
      }
      put_pair<L, PREC>(buf0, r, p, make_float2(v0.x * s0, v1.x * s0), make_float2(v0.y * s0, v1.y * s0));
    }
  }
  __syncthreads();

  // 3. forward network and spectrum, 4. inverse network and output
  uint16_t* spec = forward<L, 0, PREC>(buf0, buf1, frags, tw, reinterpret_cast<const float2*>(d.H));
  uint16_t* other = spec == buf0 ? buf1 : buf0;
  const float undo = (float)L * sqrtf((float)L);  // the three 1/sqrt(L) scales
  const int n1 = d.n1;
  const bool staged = n1 <= TcShape<L>::TILE_N1;
  float2* tile = reinterpret_cast<float2*>(other);  // free during the last inverse stage
  auto emit = [&](int r, int p, float2 v) {
    const int row = row0 + r;
    const float s = undo * __uint_as_float(rowmax[r]);
    const float2 u = cmul(make_float2(v.x * s, v.y * s), __ldg(reinterpret_cast<const float2*>(d.cout) + p));
    if (staged) {
      tile[p * kRows + r] = u;
      return;
    }
    if (row >= d.rows) return;
    const size_t o = (size_t)p * d.dst_ld + row;
    if constexpr (KIND != PASS_Y) {
      d.dst[o] = u;
    } else {
      if (d.dst) d.dst[o] = d.accumulate ? cadd(d.dst[o], u) : u;
      if (d.inten) d.inten[o] = fmaf(u.x, u.x, u.y * u.y);
      if (d.phase) d.phase[o] = phase_of(u);
    }
  };
  inverse<L, stage_count(L, kTcE) - 1, PREC>(spec, other, frags, tw, [&](int r, int p, float2 X, float2 Y) {
    if (p < n1) emit(r, p, make_float2(X.x, Y.x));
    if (p + 1 < n1) emit(r, p + 1, make_float2(X.y, Y.y));
  });
  if (!staged) return;
  __syncthreads();
  // 5. the staged tile [n1][kRows] leaves as kRows-element runs of the transposed output
  float2* const dst = d.dst;
  float* const inten = d.inten;
  float* const phase = d.phase;
  const size_t dst_ld = (size_t)d.dst_ld;
  const bool acc = d.accumulate != 0;
  const int rows_here = min(kRows, d.rows - row0);
  for (int i = tid; i < n1 * kRows; i += kThreads) {
    const int p = i / kRows, r = i - p * kRows;
    if (r >= rows_here) continue;
    const float2 u = tile[i];
    const size_t o = (size_t)p * dst_ld + row0 + r;
    if constexpr (KIND != PASS_Y) {
      dst[o] = u;
    } else {
      if (dst) dst[o] = acc ? cadd(dst[o], u) : u;
      if (inten) inten[o] = fmaf(u.x, u.x, u.y * u.y);
      if (phase) phase[o] = phase_of(u);
    }
  }
}

// Per-lane A fragments of the real-block DFT matrices with the unitary scale
// 1/sqrt(R), built once per precision: for R = 16 then R = 8, forward then
// inverse, [mt][kt][q][lane].
template <int PREC>
__global__ void k_tc_frags(uint32_t* out) {
  const int lane = threadIdx.x;
  const int g = lane >> 2, tig = lane & 3;
  int base = 0;
  for (int R = 16; R >= 8; R /= 2) {
    const int T2 = 2 * R / 16;
    const double scale = 1.0 / sqrt((double)R);
    for (int inv = 0; inv < 2; ++inv) {
      auto A = [&](int r, int c) -> float {
        const int k = r % R, j = c % R;
        double s, co;
        sincospi((inv ? 2.0 : -2.0) * (double)((j * k) % R) / (double)R, &s, &co);
        const bool rre = r < R, cre = c < R;
        if (rre && cre) return (float)(scale * co);
        if (rre && !cre) return (float)(-scale * s);
        if (!rre && cre) return (float)(scale * s);
        return (float)(scale * co);
      };
      for (int mt = 0; mt < T2; ++mt)
        for (int kt = 0; kt < T2; ++kt) {
          const int r0 = mt * 16 + g, c0 = kt * 16 + 2 * tig;
          const float v[4][2] = {{A(r0, c0), A(r0, c0 + 1)},
                                 {A(r0 + 8, c0), A(r0 + 8, c0 + 1)},
                                 {A(r0, c0 + 8), A(r0, c0 + 9)},
                                 {A(r0 + 8, c0 + 8), A(r0 + 8, c0 + 9)}};
          for (int q = 0; q < 4; ++q) out[base + ((mt * T2 + kt) * 4 + q) * 32 + lane] = pack2<PREC>(v[q][0], v[q][1]);
        }
      base += frag_words(R) / 2;
    }
  }
}

// Twiddle tables of one length: per stage with M > 1, entry k M + n (n even)
// and its successor hold the float4 (Re W_n, Re W_n+1, Im W_n, Im W_n+1) of
// W_n = W_{M'}^{n k}; double-precision sincospi rounded to float, one thread
// per (k, even n).
template <int L>
__global__ void k_tc_twiddles(float2* tab) {
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= tw_entries<L>()) return;
  int s = 0;
  while (tw_offset<L>(s + 1) <= i) ++s;
  const int MP = stage_mprev(L, kTcE, s), R = stage_radix(L, kTcE, s), M = MP / R;
  const int local = i - tw_offset<L>(s), k = local / M, n = local - k * M;
  double s0, c0, s1, c1;
  sincospi(-2.0 * (double)(((long long)n * k) % MP) / (double)MP, &s0, &c0);
  sincospi(-2.0 * (double)(((long long)(n + 1) * k) % MP) / (double)MP, &s1, &c1);
  reinterpret_cast<float4*>(tab)[i / 2] = make_float4((float)c0, (float)c1, (float)s0, (float)s1);
}

// Kernel spectrum from register order (FP32 network) to position order,
// scaled by 1/sqrt(L) (the unitary scale of the spectrum multiply).
template <int L>
__global__ void k_hpos(const float2* __restrict__ Hreg, float2* __restrict__ Hpos) {
  constexpr int T = L / kE;
  const float hs = rsqrtf((float)L);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const float2 h = Hreg[e * T + t];
    Hpos[last_pos<L, kE>(t, e)] = make_float2(h.x * hs, h.y * hs);
  }
}

template <int L, int PREC>
cudaError_t launch_tc_t(PassKind kind, const PassBatch& b, int grid_x, const uint32_t* tables, cudaStream_t s) {
  const dim3 grid(grid_x, b.count), block(kThreads);
  constexpr size_t smem = TcShape<L>::SMEM;
  const float2* tw = reinterpret_cast<const float2*>(tables + frag_words(16) + frag_words(8)) +
                     (L == 4096 ? tw_entries<2048>() : 0);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, s>>>(b, tw, tables);
    return cudaGetLastError();
  };
  switch (kind) {
    case PASS_X_REAL: return go(k_pass_tc<L, PASS_X_REAL, PREC>);
    case PASS_X_CPLX: return go(k_pass_tc<L, PASS_X_CPLX, PREC>);
    case PASS_Y: return go(k_pass_tc<L, PASS_Y, PREC>);
  }
  return cudaErrorInvalidValue;
}

}  // namespace tc

// The spectrum is converted from the FP32 network's register order, so both
// networks must share their radix plan.
bool tc_length_supported(int L) { return kE == kTcE && (L == 2048 || L == 4096); }
int tc_rows_per_cta(int L) { return L == 4096 ? tc::rows_of<4096>() : tc::rows_of<2048>(); }
// A fragments, then the twiddle tables of 2048 and 4096 (float2)
size_t tc_table_words() {
  return (size_t)tc::frag_words(16) + tc::frag_words(8) + 2 * (tc::tw_entries<2048>() + tc::tw_entries<4096>());
}

cudaError_t launch_tc_tables(uint32_t* out, int prec, cudaStream_t s) {
  if (prec == SF_PREC_BF16TC) tc::k_tc_frags<SF_PREC_BF16TC><<<1, 32, 0, s>>>(out);
  else tc::k_tc_frags<SF_PREC_FP16TC><<<1, 32, 0, s>>>(out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float2* tw = reinterpret_cast<float2*>(out + tc::frag_words(16) + tc::frag_words(8));
  tc::k_tc_twiddles<2048><<<(tc::tw_entries<2048>() / 2 + 255) / 256, 256, 0, s>>>(tw);
  tc::k_tc_twiddles<4096><<<(tc::tw_entries<4096>() / 2 + 255) / 256, 256, 0, s>>>(tw + tc::tw_entries<2048>());
  return cudaGetLastError();
}

cudaError_t launch_hpos(int L, const float2* Hreg, float2* Hpos, cudaStream_t s) {
  switch (L) {
    case 2048: tc::k_hpos<2048><<<1, 2048 / kE, 0, s>>>(Hreg, Hpos); break;
    case 4096: tc::k_hpos<4096><<<1, 4096 / kE, 0, s>>>(Hreg, Hpos); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pass_tc(int L, int prec, PassKind kind, const PassBatch& b, int grid_x, const uint32_t* frags,
                           cudaStream_t s) {
  if (prec == SF_PREC_BF16TC) {
    if (L == 2048) return tc::launch_tc_t<2048, SF_PREC_BF16TC>(kind, b, grid_x, frags, s);
    if (L == 4096) return tc::launch_tc_t<4096, SF_PREC_BF16TC>(kind, b, grid_x, frags, s);
  } else {
    if (L == 2048) return tc::launch_tc_t<2048, SF_PREC_FP16TC>(kind, b, grid_x, frags, s);
    if (L == 4096) return tc::launch_tc_t<4096, SF_PREC_FP16TC>(kind, b, grid_x, frags, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sf

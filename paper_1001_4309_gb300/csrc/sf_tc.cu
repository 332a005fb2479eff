// sf_tc.cu -- mixed-precision row pass: the radix-16 / radix-8 DFT stages of
// the FFT network as half-precision tensor-core matrix products
// (mma.sync m16n8k16, FP16 or BF16 operands, FP32 accumulation).
//
// Same positions, stages and twiddles as the FP32 network (sf_fft.cuh); only
// the radix-R DFTs move to the tensor cores.  Stage s is the real GEMM
//
//   C (2R x L/R) = A_R (2R x 2R) * B (2R x L/R)
//
// with A_R the real block [[Wr, -Wi], [Wi, Wr]] of the radix-R DFT matrix
// (its conjugate for the inverse) and column b of B the 2R real inputs of
// butterfly b (re of elements 0..R-1, then im).  B lives in shared memory as
// [b][2R + 8] halves (inputs contiguous, rows padded by 16 bytes so ldmatrix
// is conflict-free).  Each stage epilogue works in FP32 on the accumulator
// fragments: it applies the stage's twiddle (forward) or the next stage's
// conjugated twiddle (inverse), a 1/sqrt(R) scale that keeps values in
// half-precision range, and scatters the values into the next stage's
// layout.  The last forward epilogue multiplies by the kernel spectrum (in
// position order, scaled by 1/sqrt(L)) and keeps the layout for the first
// inverse stage; the last inverse epilogue undoes the scales, applies the
// output chirp and stores the row.  Rows are normalised by their largest
// input magnitude before the first conversion to half precision.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sf_kernels.cuh"

namespace sf {
namespace tc {

constexpr int kRows = 4;       // rows per CTA
constexpr int kThreads = 256;  // 8 warps

template <int R>
__host__ __device__ constexpr int bstride() { return 2 * R + 8; }  // halves per butterfly row

template <int L>
__host__ __device__ constexpr int buf_halves() {
  return (L / 16) * bstride<16>() > (L / 8) * bstride<8>() ? (L / 16) * bstride<16>() : (L / 8) * bstride<8>();
}

template <int L>
struct TcShape {
  static constexpr int BUF = buf_halves<L>();
  static constexpr size_t SMEM = sizeof(uint16_t) * 2 * kRows * (size_t)BUF + 16 * kRows;
};

template <int PREC>
__device__ __forceinline__ void st_half(uint16_t* p, float v) {
  v = fminf(fmaxf(v, -65504.f), 65504.f);
  if constexpr (PREC == SF_PREC_BF16TC) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    *p = *reinterpret_cast<uint16_t*>(&h);
  } else {
    __half h = __float2half_rn(v);
    *p = *reinterpret_cast<uint16_t*>(&h);
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

__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const uint16_t* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a));
}

// W_{M'}^{n k} of stage S (conjugated when CONJ), from the FP32 network's table.
template <int L, int S, bool CONJ>
__device__ __forceinline__ float2 twiddle(const float4* __restrict__ tw, int n, int k) {
  using St = Stage<L, kTcE, S>;
  const float4 w = __ldg(tw + stage_tw_offset(L, kTcE, S) + (k >> 1) * St::M + n);
  const float2 v = (k & 1) ? make_float2(w.z, w.w) : make_float2(w.x, w.y);
  return CONJ ? make_float2(v.x, -v.y) : v;
}

template <int L, int S>
__device__ __forceinline__ int pos_of(int b, int k) {
  using St = Stage<L, kTcE, S>;
  return (b / St::M) * St::MP + (b % St::M) + k * St::M;
}

template <int L, int S>
__device__ __forceinline__ void bk_of(int p, int& b, int& k) {
  using St = Stage<L, kTcE, S>;
  const int K = p / St::MP, rem = p - K * St::MP;
  const int n = rem % St::M;
  k = rem / St::M;
  b = K * St::M + n;
}

// Store one complex value at position p of row `row` in stage S's input layout.
template <int L, int S, int PREC>
__device__ __forceinline__ void put(uint16_t* buf, int row, int p, float2 v) {
  constexpr int R = Stage<L, kTcE, S>::R;
  int b, k;
  bk_of<L, S>(p, b, k);
  uint16_t* q = buf + row * TcShape<L>::BUF + b * bstride<R>();
  st_half<PREC>(q + k, v.x);
  st_half<PREC>(q + R + k, v.y);
}

// Per-lane A fragments: [dir][mt][kt][q][lane] for radix 16, then for radix 8.
__host__ __device__ constexpr int frag_words(int R) { return 2 * (R / 8) * (R / 8) * 4 * 32; }

// One stage's GEMM over all rows of the CTA; epi(row, butterfly, element, value).
template <int L, int S, int PREC, bool INV, typename Epi>
__device__ __forceinline__ void stage_gemm(const uint16_t* in, const uint32_t* __restrict__ frags, Epi&& epi) {
  using St = Stage<L, kTcE, S>;
  constexpr int R = St::R;
  static_assert(R == 16 || R == 8, "tensor-core stages need radix 8 or 16");
  constexpr int NT = L / R / 8;   // n-tiles (8 butterflies) per row
  constexpr int T2 = 2 * R / 16;  // m-tiles = k-steps of the real block
  constexpr int BS = bstride<R>();
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
  for (int unit = warp; unit < kRows * NT; unit += kThreads / 32) {
    const int row = unit / NT, nt = unit - row * NT;
    const uint16_t* bb = in + row * TcShape<L>::BUF + (nt * 8 + (lane & 7)) * BS + ((lane >> 3) & 1) * 8;
    float c[T2][4];
#pragma unroll
    for (int mt = 0; mt < T2; ++mt) c[mt][0] = c[mt][1] = c[mt][2] = c[mt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < T2; ++kt) {
      uint32_t b0, b1;
      ldsm_x2(b0, b1, bb + kt * 16);
#pragma unroll
      for (int mt = 0; mt < T2; ++mt) mma16816<PREC>(c[mt], a[mt][kt], b0, b1);
    }
    const int bi = nt * 8 + 2 * tig;
    if constexpr (R == 16) {
      // tile 0: re of elements 0..15, tile 1: im; rows g and g + 8, columns bi, bi + 1
      epi(row, bi, g, make_float2(c[0][0], c[1][0]));
      epi(row, bi + 1, g, make_float2(c[0][1], c[1][1]));
      epi(row, bi, g + 8, make_float2(c[0][2], c[1][2]));
      epi(row, bi + 1, g + 8, make_float2(c[0][3], c[1][3]));
    } else {
      // one tile: row g = re of element g, row g + 8 = im of element g
      epi(row, bi, g, make_float2(c[0][0], c[0][2]));
      epi(row, bi + 1, g, make_float2(c[0][1], c[0][3]));
    }
  }
}

template <int R>
__device__ __forceinline__ constexpr float inv_sqrt_radix() {
  return R == 16 ? 0.25f : (R == 8 ? 0.35355339059327373f : 1.0f);
}

// Forward stages S.. of the network; returns the buffer holding the layout of
// the last stage after the spectrum multiply.
template <int L, int S, int PREC>
__device__ __forceinline__ uint16_t* forward(uint16_t* cur, uint16_t* oth, const uint32_t* frags,
                                             const float4* __restrict__ tw, const float2* __restrict__ Hpos,
                                             float hs) {
  using St = Stage<L, kTcE, S>;
  constexpr int NS = stage_count(L, kTcE);
  constexpr float f = inv_sqrt_radix<St::R>();
  if constexpr (S + 1 < NS) {
    stage_gemm<L, S, PREC, false>(cur, frags, [&](int row, int b, int k, float2 v) {
      const float2 w = twiddle<L, S, false>(tw, b % St::M, k);
      put<L, S + 1, PREC>(oth, row, pos_of<L, S>(b, k),
                          make_float2(f * (v.x * w.x - v.y * w.y), f * (v.x * w.y + v.y * w.x)));
    });
    __syncthreads();
    return forward<L, S + 1, PREC>(oth, cur, frags, tw, Hpos, hs);
  } else {
    const float sc = f * hs;
    stage_gemm<L, S, PREC, false>(cur, frags, [&](int row, int b, int k, float2 v) {
      const int p = pos_of<L, S>(b, k);
      const float2 h = __ldg(Hpos + p);
      put<L, S, PREC>(oth, row, p, make_float2(sc * (v.x * h.x - v.y * h.y), sc * (v.x * h.y + v.y * h.x)));
    });
    __syncthreads();
    return oth;
  }
}

// Inverse stages S..0; the last one hands (row, natural position, value) to `out`.
template <int L, int S, int PREC, typename Out>
__device__ __forceinline__ void inverse(uint16_t* cur, uint16_t* oth, const uint32_t* frags,
                                        const float4* __restrict__ tw, Out&& out) {
  using St = Stage<L, kTcE, S>;
  constexpr float f = inv_sqrt_radix<St::R>();
  if constexpr (S > 0) {
    using Sp = Stage<L, kTcE, S - 1>;
    stage_gemm<L, S, PREC, true>(cur, frags, [&](int row, int b, int k, float2 v) {
      const int p = pos_of<L, S>(b, k);
      int bp, kp;
      bk_of<L, S - 1>(p, bp, kp);
      const float2 w = twiddle<L, S - 1, true>(tw, bp % Sp::M, kp);
      put<L, S - 1, PREC>(oth, row, p, make_float2(f * (v.x * w.x - v.y * w.y), f * (v.x * w.y + v.y * w.x)));
    });
    __syncthreads();
    inverse<L, S - 1, PREC>(oth, cur, frags, tw, out);
  } else {
    stage_gemm<L, 0, PREC, true>(cur, frags, [&](int row, int b, int k, float2 v) {
      out(row, pos_of<L, 0>(b, k), make_float2(f * v.x, f * v.y));
    });
  }
}

template <int L, int KIND, int PREC>
__global__ void __launch_bounds__(kThreads, 1)
k_pass_tc(const __grid_constant__ PassBatch pb, const float4* __restrict__ tw, const uint32_t* __restrict__ frags) {
  extern __shared__ __align__(16) uint16_t sm[];
  constexpr int BUF = TcShape<L>::BUF;
  uint16_t* buf0 = sm;
  uint16_t* buf1 = sm + kRows * BUF;
  unsigned* rowmax = reinterpret_cast<unsigned*>(sm + 2 * kRows * BUF);
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

  // 1. largest input magnitude of each row
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
  // 2. normalised input in the layout of stage 0 (implicit zero padding)
  for (int r = 0; r < kRows; ++r) {
    const int row = row0 + r;
    const float mx = __uint_as_float(rowmax[r]);
    const float s0 = mx > 0.f ? 1.0f / mx : 0.f;
    for (int p = tid; p < L; p += kThreads) {
      float2 v = make_float2(0.f, 0.f);
      if (row < d.rows && p < d.n0) {
        v = load(row, p);
        v = make_float2(v.x * s0, v.y * s0);
      }
      put<L, 0, PREC>(buf0, r, p, v);
    }
  }
  __syncthreads();

  // 3. forward network and spectrum, 4. inverse network and output
  const float hs = rsqrtf((float)L);
  uint16_t* spec = forward<L, 0, PREC>(buf0, buf1, frags, tw, reinterpret_cast<const float2*>(d.H), hs);
  uint16_t* other = spec == buf0 ? buf1 : buf0;
  const float undo = (float)L * sqrtf((float)L);  // the three 1/sqrt(L) scales
  inverse<L, stage_count(L, kTcE) - 1, PREC>(spec, other, frags, tw, [&](int r, int p, float2 v) {
    const int row = row0 + r;
    if (row >= d.rows || p >= d.n1) return;
    const float s = undo * __uint_as_float(rowmax[r]);
    const float2 u = cmul(make_float2(v.x * s, v.y * s), __ldg(reinterpret_cast<const float2*>(d.cout) + p));
    const size_t o = (size_t)p * d.dst_ld + row;
    if constexpr (KIND != PASS_Y) {
      d.dst[o] = u;
    } else {
      if (d.dst) d.dst[o] = d.accumulate ? cadd(d.dst[o], u) : u;
      if (d.inten) d.inten[o] = fmaf(u.x, u.x, u.y * u.y);
      if (d.phase) d.phase[o] = phase_of(u);
    }
  });
}

// Per-lane A fragments of the real-block DFT matrices, built once per
// precision: for R = 16 then R = 8, forward then inverse, [mt][kt][q][lane].
template <int PREC>
__global__ void k_tc_frags(uint32_t* out) {
  const int lane = threadIdx.x;
  const int g = lane >> 2, tig = lane & 3;
  int base = 0;
  for (int R = 16; R >= 8; R /= 2) {
    const int T2 = 2 * R / 16;
    for (int inv = 0; inv < 2; ++inv) {
      auto A = [&](int r, int c) -> float {
        const int k = r % R, j = c % R;
        double s, co;
        sincospi((inv ? 2.0 : -2.0) * (double)((j * k) % R) / (double)R, &s, &co);
        const bool rre = r < R, cre = c < R;
        if (rre && cre) return (float)co;
        if (rre && !cre) return (float)-s;
        if (!rre && cre) return (float)s;
        return (float)co;
      };
      for (int mt = 0; mt < T2; ++mt)
        for (int kt = 0; kt < T2; ++kt) {
          const int r0 = mt * 16 + g, c0 = kt * 16 + 2 * tig;
          const float v[4][2] = {{A(r0, c0), A(r0, c0 + 1)},
                                 {A(r0 + 8, c0), A(r0 + 8, c0 + 1)},
                                 {A(r0, c0 + 8), A(r0, c0 + 9)},
                                 {A(r0 + 8, c0 + 8), A(r0 + 8, c0 + 9)}};
          for (int q = 0; q < 4; ++q) {
            uint32_t w;
            if (PREC == SF_PREC_BF16TC) {
              __nv_bfloat162 h = __floats2bfloat162_rn(v[q][0], v[q][1]);
              w = *reinterpret_cast<uint32_t*>(&h);
            } else {
              __half2 h = __floats2half2_rn(v[q][0], v[q][1]);
              w = *reinterpret_cast<uint32_t*>(&h);
            }
            out[base + ((mt * T2 + kt) * 4 + q) * 32 + lane] = w;
          }
        }
      base += frag_words(R) / 2;
    }
  }
}

// Kernel spectrum from register order (FP32 network) to position order.
template <int L>
__global__ void k_hpos(const float2* __restrict__ Hreg, float2* __restrict__ Hpos) {
  constexpr int T = L / kE;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
#pragma unroll
  for (int e = 0; e < kE; ++e) Hpos[last_pos<L, kE>(t, e)] = Hreg[e * T + t];
}

template <int L, int PREC>
cudaError_t launch_tc_t(PassKind kind, const PassBatch& b, int grid_x, const float4* tw, const uint32_t* frags,
                        cudaStream_t s) {
  const dim3 grid(grid_x, b.count), block(kThreads);
  constexpr size_t smem = TcShape<L>::SMEM;
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, block, smem, s>>>(b, tw, frags);
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
int tc_rows_per_cta() { return tc::kRows; }
size_t tc_frag_words() { return (size_t)tc::frag_words(16) + tc::frag_words(8); }

cudaError_t launch_tc_frags(uint32_t* out, int prec, cudaStream_t s) {
  if (prec == SF_PREC_BF16TC) tc::k_tc_frags<SF_PREC_BF16TC><<<1, 32, 0, s>>>(out);
  else tc::k_tc_frags<SF_PREC_FP16TC><<<1, 32, 0, s>>>(out);
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

cudaError_t launch_pass_tc(int L, int prec, PassKind kind, const PassBatch& b, int grid_x, const float4* tw,
                           const uint32_t* frags, cudaStream_t s) {
  if (prec == SF_PREC_BF16TC) {
    if (L == 2048) return tc::launch_tc_t<2048, SF_PREC_BF16TC>(kind, b, grid_x, tw, frags, s);
    if (L == 4096) return tc::launch_tc_t<4096, SF_PREC_BF16TC>(kind, b, grid_x, tw, frags, s);
  } else {
    if (L == 2048) return tc::launch_tc_t<2048, SF_PREC_FP16TC>(kind, b, grid_x, tw, frags, s);
    if (L == 4096) return tc::launch_tc_t<4096, SF_PREC_FP16TC>(kind, b, grid_x, tw, frags, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sf

// sf_fft.cuh -- in-register / shared-memory FFT building blocks for sm_103a.
//
// The zero-padded FFT convolution of Eq. 1 (Section 2.1) is done per row
// by one thread group of T = L / E threads, each holding E complex values in
// registers.  The length-L transform is an in-place decimation-in-frequency
// network of radix-E stages (the last stage takes the remaining factor):
//
//   stage s, sub-length M' = L / (R_0 ... R_{s-1}), radix R = R_s, M = M' / R:
//   for every butterfly (K, n), K < L / M', n < M, the R values at positions
//   K M' + n + j M (j < R) are replaced by  y_k = W_{M'}^{n k} sum_j x_j W_R^{j k}
//   at positions K M' + n + k M.
//
// Power-of-two lengths use E = 16 (radix-16 stages, the last one taking the
// remaining factor).  Lengths with a factor 3 (1536, 2304, 3072, 4608, 6144)
// use E = 24 and an explicit radix sequence whose first radix (24) holds the
// factor 3, so every later sub-length is a power of two.
//
// After the last stage position p holds frequency f(p), the mixed-radix digit
// reversal of p.  The convolution never needs natural frequency order: the
// kernel spectrum is produced by the same network (so it sits in the same
// positions), multiplied in registers, and the exact adjoint network (stages
// in reverse order, conjugated twiddles applied before an inverse radix-R DFT)
// returns L times the circular convolution in natural order.
//
// Between stages the values move through a shared-memory row buffer padded
// by one slot every 16 positions, which keeps the 8-byte accesses of each
// half warp on distinct bank pairs for every stage pattern at L >= 256.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace sf {

// ---------------------------------------------------------------- complex ops
// Complex add and subtract are one packed f32x2 instruction each (sm_100+);
// products by +-i are folded into scalar adds (add_w4 / sub_w4) instead of
// being formed as lane-swapped operands.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 ta, tb, tr;\n\tmov.b64 ta, {%2, %3};\n\tmov.b64 tb, {%4, %5};\n\t"
      "sub.rn.f32x2 tr, ta, tb;\n\tmov.b64 {%0, %1}, tr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// a + W_4 b and a - W_4 b with W_4 = -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 add_w4(float2 a, float2 b) {
  return INV ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
}
template <bool INV>
__device__ __forceinline__ float2 sub_w4(float2 a, float2 b) {
  return INV ? make_float2(a.x + b.y, a.y - b.x) : make_float2(a.x - b.y, a.y + b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Multiplication by W_4 = exp(-+ 2 pi i / 4): -i for the forward transform, +i for the inverse.
template <bool INV>
__device__ __forceinline__ float2 mul_w4(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Twiddle constants W_16^e = exp(-2 pi i e / 16) (conjugated for the inverse).
constexpr float kC1 = 0.92387953251128676f;  // cos(pi/8)
constexpr float kS1 = 0.38268343236508977f;  // sin(pi/8)
constexpr float kR2 = 0.70710678118654752f;  // cos(pi/4)

template <bool INV, int E16>
__device__ __forceinline__ float2 mul_w16(float2 a) {
  constexpr int e = E16 & 15;
  if constexpr (e == 0) return a;
  else if constexpr (e == 4) return mul_w4<INV>(a);
  else if constexpr (e == 8) return make_float2(-a.x, -a.y);
  else if constexpr (e == 12) return mul_w4<!INV>(a);
  else if constexpr (e == 2 || e == 6 || e == 10 || e == 14) {
    // (+-c, +-c) with c = cos(pi/4): two adds and two multiplies
    constexpr float wr = (e == 2 || e == 14) ? kR2 : -kR2;
    constexpr float wi0 = (e == 2 || e == 6) ? -kR2 : kR2;
    constexpr float wi = INV ? -wi0 : wi0;
    return make_float2(wr * a.x - wi * a.y, wr * a.y + wi * a.x);
  } else {
    constexpr float cs[16] = {1.f, kC1, kR2, kS1, 0.f, -kS1, -kR2, -kC1, -1.f, -kC1, -kR2, -kS1, 0.f, kS1, kR2, kC1};
    constexpr float wr = cs[e];
    constexpr float wi0 = -cs[(e + 12) & 15];  // -sin(2 pi e / 16)
    constexpr float wi = INV ? -wi0 : wi0;
    return make_float2(fmaf(wr, a.x, -wi * a.y), fmaf(wr, a.y, wi * a.x));
  }
}

// ------------------------------------------------------------- radix-R DFTs
// In place, natural order in and out: x[k] <- sum_j x[j] W_R^{j k}
// (W_R = exp(-2 pi i / R); exp(+2 pi i / R) for INV, no 1/R scaling).

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s0 = cadd(a0, a2), d0 = csub(a0, a2);
  const float2 s1 = cadd(a1, a3), e1 = csub(a1, a3);
  a0 = cadd(s0, s1);
  a2 = csub(s0, s1);
  a1 = add_w4<INV>(d0, e1);
  a3 = sub_w4<INV>(d0, e1);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* x) {
  // even / odd halves, then combine with W_8^k = W_16^{2k}
  float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = mul_w16<INV, 2>(o1);
  o3 = mul_w16<INV, 6>(o3);
  x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
  x[2] = add_w4<INV>(e2, o2); x[6] = sub_w4<INV>(e2, o2);  // o2 carries W_8^2 = W_4
  x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

// Radix 16 as 4 x 4.  ZIN: inputs 8..15 are known zero (the first forward
// stage of a row with at most L/2 nonzeros), so the first-layer butterflies
// see two inputs.  ZOUT: only outputs 0..7 are used (the last inverse stage of
// a row with at most L/2 outputs), so the second layer forms half of them.
template <bool INV, bool ZIN = false, bool ZOUT = false>
__device__ __forceinline__ void dft16(float2* x) {
  // 4 x 4: j = 4 j1 + j2, k = k1 + 4 k2
  float2 b[16];
#pragma unroll
  for (int j2 = 0; j2 < 4; ++j2) {
    float2 a0 = x[j2], a1 = x[4 + j2], a2, a3;
    if constexpr (ZIN) {
      a2 = csub(a0, a1);
      a3 = sub_w4<INV>(a0, a1);
      a1 = add_w4<INV>(a0, a1);
      a0 = cadd(a0, x[4 + j2]);
    } else {
      a2 = x[8 + j2];
      a3 = x[12 + j2];
      dft4<INV>(a0, a1, a2, a3);  // over j1 -> k1
    }
    b[4 * j2 + 0] = a0; b[4 * j2 + 1] = a1; b[4 * j2 + 2] = a2; b[4 * j2 + 3] = a3;
  }
  // twiddle W_16^{j2 k1}
  b[4 * 1 + 1] = mul_w16<INV, 1>(b[4 * 1 + 1]);
  b[4 * 1 + 2] = mul_w16<INV, 2>(b[4 * 1 + 2]);
  b[4 * 1 + 3] = mul_w16<INV, 3>(b[4 * 1 + 3]);
  b[4 * 2 + 1] = mul_w16<INV, 2>(b[4 * 2 + 1]);
  b[4 * 2 + 3] = mul_w16<INV, 6>(b[4 * 2 + 3]);
  b[4 * 3 + 1] = mul_w16<INV, 3>(b[4 * 3 + 1]);
  b[4 * 3 + 2] = mul_w16<INV, 6>(b[4 * 3 + 2]);
  b[4 * 3 + 3] = mul_w16<INV, 9>(b[4 * 3 + 3]);
  // b[4 * 2 + 2] carries W_16^4 = W_4, folded into the k1 = 2 butterfly below
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 a0 = b[k1], a1 = b[4 + k1], a2 = b[8 + k1], a3 = b[12 + k1];
    float2 s0, d0;
    if (k1 == 2) {
      s0 = add_w4<INV>(a0, a2);
      d0 = sub_w4<INV>(a0, a2);
    } else {
      s0 = cadd(a0, a2);
      d0 = csub(a0, a2);
    }
    const float2 s1 = cadd(a1, a3), e1 = csub(a1, a3);
    x[k1 + 0] = cadd(s0, s1);              // k2 = 0
    x[k1 + 4] = add_w4<INV>(d0, e1);       // k2 = 1
    if constexpr (!ZOUT) {
      x[k1 + 8] = csub(s0, s1);            // k2 = 2
      x[k1 + 12] = sub_w4<INV>(d0, e1);    // k2 = 3
    }
  }
}

// cos(2 pi e / 24), e = 0..23 (multiples of 15 degrees)
constexpr float kCos24[24] = {1.f, 0.96592582628906829f, 0.86602540378443865f, 0.70710678118654752f,
                              0.5f, 0.25881904510252076f, 0.f, -0.25881904510252076f,
                              -0.5f, -0.70710678118654752f, -0.86602540378443865f, -0.96592582628906829f,
                              -1.f, -0.96592582628906829f, -0.86602540378443865f, -0.70710678118654752f,
                              -0.5f, -0.25881904510252076f, 0.f, 0.25881904510252076f,
                              0.5f, 0.70710678118654752f, 0.86602540378443865f, 0.96592582628906829f};

// a * W_24^E24 with W_24 = exp(-2 pi i / 24) (conjugated for the inverse);
// multiples of 45 degrees go through mul_w16.
template <bool INV, int E24>
__device__ __forceinline__ float2 mul_w24(float2 a) {
  constexpr int e = ((E24 % 24) + 24) % 24;
  if constexpr (e % 3 == 0) {
    return mul_w16<INV, 2 * e / 3>(a);
  } else {
    constexpr float wr = kCos24[e];
    constexpr float wi0 = -kCos24[(e + 18) % 24];  // -sin(2 pi e / 24)
    constexpr float wi = INV ? -wi0 : wi0;
    return make_float2(fmaf(wr, a.x, -wi * a.y), fmaf(wr, a.y, wi * a.x));
  }
}

// Radix 3: with s = x1 + x2, d = x1 - x2 and m = x0 - s / 2,
// X0 = x0 + s, X1 = m -+ i (sqrt(3) / 2) d, X2 = m +- i (sqrt(3) / 2) d.
template <bool INV>
__device__ __forceinline__ void dft3(float2& a0, float2& a1, float2& a2) {
  constexpr float kS3 = 0.86602540378443865f;  // sin(pi / 3)
  const float2 s = cadd(a1, a2), d = csub(a1, a2);
  const float2 m = make_float2(fmaf(-0.5f, s.x, a0.x), fmaf(-0.5f, s.y, a0.y));
  a0 = cadd(a0, s);
  const float2 r = INV ? make_float2(-kS3 * d.y, kS3 * d.x) : make_float2(kS3 * d.y, -kS3 * d.x);
  a1 = cadd(m, r);
  a2 = csub(m, r);
}

template <int R, bool INV, bool ZIN = false, bool ZOUT = false>
__device__ __forceinline__ void dft(float2* x);

// Twiddles W_R^{j2 k1} of a Cooley-Tukey split, element I = R1 j2 + k1.
template <bool INV, int R, int R1, int... I>
__device__ __forceinline__ void ct_twiddle(float2* a, std::integer_sequence<int, I...>) {
  static_assert(24 % R == 0, "constant twiddles are multiples of 15 degrees");
  ((a[I] = mul_w24<INV, (24 / R) * ((I / R1) * (I % R1))>(a[I])), ...);
}

// Radix R = R1 R2 by one Cooley-Tukey split: j = R2 j1 + j2, k = k1 + R1 k2,
// X[k] = sum_j2 W_R2^{j2 k2} [W_R^{j2 k1} sum_j1 x[j] W_R1^{j1 k1}].
template <int R1, int R2, bool INV>
__device__ __forceinline__ void dft_ct(float2* x) {
  constexpr int R = R1 * R2;
  float2 a[R];
#pragma unroll
  for (int j2 = 0; j2 < R2; ++j2) {
    float2 c[R1];
#pragma unroll
    for (int j1 = 0; j1 < R1; ++j1) c[j1] = x[R2 * j1 + j2];
    dft<R1, INV>(c);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[R1 * j2 + k1] = c[k1];
  }
  ct_twiddle<INV, R, R1>(a, std::make_integer_sequence<int, R>{});
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    float2 c[R2];
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) c[j2] = a[R1 * j2 + k1];
    dft<R2, INV>(c);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = c[k2];
  }
}

template <int R, bool INV, bool ZIN, bool ZOUT>
__device__ __forceinline__ void dft(float2* x) {
  static_assert(R == 16 || !(ZIN || ZOUT), "pruned butterflies exist for radix 16");
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<INV>(x[0], x[1]);
  } else if constexpr (R == 3) {
    dft3<INV>(x[0], x[1], x[2]);
  } else if constexpr (R == 4) {
    dft4<INV>(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 6) {
    dft_ct<3, 2, INV>(x);
  } else if constexpr (R == 8) {
    dft8<INV>(x);
  } else if constexpr (R == 12) {
    dft_ct<3, 4, INV>(x);
  } else if constexpr (R == 16) {
    dft16<INV, ZIN, ZOUT>(x);
  } else if constexpr (R == 24) {
    dft_ct<3, 8, INV>(x);
  } else {
    static_assert(R == 16, "unsupported radix");
  }
}

// ------------------------------------------------------------- stage layout
constexpr bool is_pow2(int L) { return L > 0 && (L & (L - 1)) == 0; }

// Radix sequences of the lengths with a factor 3 (E = 24); 1 past the last stage.
constexpr int mixed_radix(int L, int s) {
  return L == 1536   ? (s == 0 ? 24 : s < 3 ? 8 : 1)
         : L == 2304 ? (s == 0 ? 24 : s == 1 ? 12 : s == 2 ? 8 : 1)
         : L == 3072 ? (s == 0 ? 24 : s < 3 ? 8 : s == 3 ? 2 : 1)
         : L == 4608 ? (s < 2 ? 24 : s == 2 ? 8 : 1)
         : L == 6144 ? (s == 0 ? 24 : s < 3 ? 8 : s == 3 ? 4 : 1)
                     : 1;
}

// radix of stage s (1 past the last stage)
constexpr int stage_radix(int L, int E, int s) {
  if (!is_pow2(L)) return mixed_radix(L, s);
  int M = L;
  for (int i = 0; i < s; ++i) M /= (M > E ? E : M);
  return M > E ? E : M;
}
// sub-length M' entering stage s
constexpr int stage_mprev(int L, int E, int s) {
  int M = L;
  for (int i = 0; i < s; ++i) M /= stage_radix(L, E, i);
  return M;
}
constexpr int stage_count(int L, int E) {
  int s = 0;
  while (stage_mprev(L, E, s) > 1) ++s;
  return s;
}

// Shared-memory address of a row position (8-byte elements): one pad slot
// every 16 positions.  A stage position is base + k M; for the radix
// sequences used here the two terms never carry across a multiple of 16, so
// phys is additive over them (Stage checks this at compile time) and every
// access is a per-thread base plus a compile-time offset.
__host__ __device__ constexpr int phys(int p) { return p + (p >> 4); }
__host__ __device__ constexpr int buf_elems(int L) { return phys(L - 1) + 1; }

// phys(base + k M) == phys(base) + phys(k M) for every position of stage s
constexpr bool stage_phys_additive(int L, int E, int s) {
  const int T = L / E, MP = stage_mprev(L, E, s), R = stage_radix(L, E, s), M = MP / R;
  for (int b = 0; b < T * (E / R); ++b) {
    const int base = (b / M) * MP + b % M;
    for (int k = 0; k < R; ++k)
      if (phys(base + k * M) != phys(base) + phys(k * M)) return false;
  }
  return true;
}

// Butterfly u (u < E / R) of thread t in stage s.  Power-of-two networks give
// a thread consecutive butterflies (t NB + u), so a stage's butterflies stay
// with the warp that produced their inputs whenever the previous stage's
// stride is at most 32 (warp_local_exchange); the lengths with a factor 3
// interleave them (t + T u).
constexpr int stage_butterfly(int L, int E, int s, int t, int u) {
  return is_pow2(L) ? t * (E / stage_radix(L, E, s)) + u : t + (L / E) * u;
}

// Thread that owns position p in stage s.
constexpr int stage_owner(int L, int E, int s, int p) {
  const int MP = stage_mprev(L, E, s), R = stage_radix(L, E, s), M = MP / R, NB = E / R, T = L / E;
  const int b = (p / MP) * M + (p % MP) % M;
  return is_pow2(L) ? b / NB : b % T;
}

// The exchange between stages s and s + 1 stays inside each warp: every
// position a thread loads for stage s + 1 was stored by a thread of its own
// warp.  Row groups must be whole warps (T a multiple of 32).
constexpr bool warp_local_exchange(int L, int E, int s) {
  const int T = L / E;
  if (T % 32 != 0) return false;
  for (int t = 0; t < T; ++t)
    for (int u = 0; u < E / stage_radix(L, E, s + 1); ++u) {
      const int b = stage_butterfly(L, E, s + 1, t, u);
      const int MP = stage_mprev(L, E, s + 1), M = MP / stage_radix(L, E, s + 1);
      const int base = (b / M) * MP + b % M;
      for (int k = 0; k < stage_radix(L, E, s + 1); ++k)
        if (stage_owner(L, E, s, base + k * M) / 32 != t / 32) return false;
    }
  return true;
}

// Position of element j of butterfly u (u < E / R) of thread t in stage s.
template <int L, int E, int S>
struct Stage {
  static constexpr int T = L / E;
  static constexpr int MP = stage_mprev(L, E, S);
  static constexpr int R = stage_radix(L, E, S);
  static constexpr int M = MP / R;
  static constexpr int NB = E / R;
  static_assert(E % R == 0, "radix must divide the per-thread element count");
  static_assert(stage_phys_additive(L, E, S), "padded addresses must split into base + offset");
  __device__ __forceinline__ static int base(int t, int u) {
    const int b = stage_butterfly(L, E, S, t, u);
    return (b / M) * MP + (b % M);
  }
  __device__ __forceinline__ static int nidx(int t, int u) { return stage_butterfly(L, E, S, t, u) % M; }
};

// Per-stage twiddle tables.  Stage s (with M > 1) owns M * R / 2 float4
// entries: entry q * M + n holds (W_{M'}^{n 2q}, W_{M'}^{n (2q+1)}), so a thread
// fetches the R twiddles of butterfly n with R/2 16-byte loads that are
// coalesced across consecutive n.  Stages are concatenated in order.
constexpr int stage_tw_entries(int L, int E, int s) {
  return (stage_mprev(L, E, s) / stage_radix(L, E, s)) > 1
             ? (stage_mprev(L, E, s) / stage_radix(L, E, s)) * stage_radix(L, E, s) / 2
             : 0;
}
constexpr int stage_tw_offset(int L, int E, int s) {
  int o = 0;
  for (int i = 0; i < s; ++i) o += stage_tw_entries(L, E, i);
  return o;
}
constexpr int tw_table_entries(int L, int E) { return stage_tw_offset(L, E, stage_count(L, E)); }

// Forward stage s on registers (values enter at the stage's read positions
// and leave at the same positions with k in place of j).
template <int L, int E, int S, bool ZIN = false>
__device__ __forceinline__ void stage_fwd(float2* v, int t, const float4* __restrict__ tw) {
  using St = Stage<L, E, S>;
#pragma unroll
  for (int u = 0; u < St::NB; ++u) {
    dft<St::R, false, ZIN>(v + u * St::R);
    if constexpr (St::M > 1) {
      const float4* tp = tw + stage_tw_offset(L, E, S) + St::nidx(t, u);
#pragma unroll
      for (int q = 0; q < St::R / 2; ++q) {
        const float4 w = __ldg(tp + q * St::M);
        if (q > 0) v[u * St::R + 2 * q] = cmul(v[u * St::R + 2 * q], make_float2(w.x, w.y));
        v[u * St::R + 2 * q + 1] = cmul(v[u * St::R + 2 * q + 1], make_float2(w.z, w.w));
      }
    }
  }
}

// Adjoint of stage_fwd: conjugate twiddles, then the inverse radix-R DFT.
template <int L, int E, int S, bool ZOUT = false>
__device__ __forceinline__ void stage_inv(float2* v, int t, const float4* __restrict__ tw) {
  using St = Stage<L, E, S>;
#pragma unroll
  for (int u = 0; u < St::NB; ++u) {
    if constexpr (St::M > 1) {
      const float4* tp = tw + stage_tw_offset(L, E, S) + St::nidx(t, u);
#pragma unroll
      for (int q = 0; q < St::R / 2; ++q) {
        const float4 w = __ldg(tp + q * St::M);
        if (q > 0) v[u * St::R + 2 * q] = cmulc(v[u * St::R + 2 * q], make_float2(w.x, w.y));
        v[u * St::R + 2 * q + 1] = cmulc(v[u * St::R + 2 * q + 1], make_float2(w.z, w.w));
      }
    }
    dft<St::R, true, false, ZOUT>(v + u * St::R);
  }
}

template <int L, int E, int S>
__device__ __forceinline__ void stage_store(const float2* v, int t, float2* buf) {
  using St = Stage<L, E, S>;
#pragma unroll
  for (int u = 0; u < St::NB; ++u) {
    const int b0 = phys(St::base(t, u));
#pragma unroll
    for (int k = 0; k < St::R; ++k) buf[b0 + phys(k * St::M)] = v[u * St::R + k];
  }
}

template <int L, int E, int S>
__device__ __forceinline__ void stage_load(float2* v, int t, const float2* buf) {
  using St = Stage<L, E, S>;
#pragma unroll
  for (int u = 0; u < St::NB; ++u) {
    const int b0 = phys(St::base(t, u));
#pragma unroll
    for (int k = 0; k < St::R; ++k) v[u * St::R + k] = buf[b0 + phys(k * St::M)];
  }
}

// Barrier over the T threads that share one row buffer: a named barrier per
// thread group when the group is whole warps (so the groups of a CTA do not
// wait for each other), the CTA barrier otherwise.  Every thread of the
// group calls it the same number of times.
template <int T>
__device__ __forceinline__ void group_sync(int g) {
  // callers keep 1 + g <= 15 (checked where the group count is fixed)
  if constexpr (T >= 32 && T % 32 == 0) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(T) : "memory");
  } else {
    __syncthreads();
  }
}

// Makes the stores of the exchange between stages s and s + 1 visible to
// the loads of the other side: a warp barrier when the exchange stays inside
// each warp, the row group's barrier otherwise.
template <int L, int E, int S>
__device__ __forceinline__ void exchange_sync(int g) {
  if constexpr (warp_local_exchange(L, E, S)) __syncwarp();
  else group_sync<L / E>(g);
}

// Full forward network.  Input: v[j] = x[t + T j] (stage 0 layout).
// Output: the last stage's positions.  buf: this group's row buffer
// (buf_elems(L) elements); g: the group's index in the CTA.  PRUNE: v[j] is
// zero for j >= E / 2 (a row of at most L / 2 nonzeros, E = 16 networks).
//
// Only the first store needs a barrier in front (earlier users of buf may
// still read any position): every later store of a stage's positions goes to
// exactly the positions the same thread loaded for that stage, so no other
// thread still needs their old contents.
template <int L, int E, int S = 0, bool PRUNE = false>
__device__ __forceinline__ void fft_forward(float2* v, int t, int g, float2* buf, const float4* __restrict__ tw) {
  constexpr int NS = stage_count(L, E);
  stage_fwd<L, E, S, PRUNE && S == 0>(v, t, tw);
  if constexpr (S + 1 < NS) {
    if constexpr (S == 0) group_sync<L / E>(g);  // previous readers of buf are done
    stage_store<L, E, S>(v, t, buf);
    exchange_sync<L, E, S>(g);
    stage_load<L, E, S + 1>(v, t, buf);
    fft_forward<L, E, S + 1, PRUNE>(v, t, g, buf, tw);
  }
}

// Adjoint network: from the last stage's positions back to v[j] = x[t + T j].
// PRUNE: only v[j], j < E / 2, are used afterwards (at most L / 2 outputs).
// Runs on the buffer fft_forward left (each thread last accessed its own
// last-stage positions there), so its stores need no barrier in front.
template <int L, int E, int S = stage_count(L, E) - 1, bool PRUNE = false>
__device__ __forceinline__ void fft_inverse(float2* v, int t, int g, float2* buf, const float4* __restrict__ tw) {
  stage_inv<L, E, S, PRUNE && S == 0>(v, t, tw);
  if constexpr (S > 0) {
    stage_store<L, E, S>(v, t, buf);
    exchange_sync<L, E, S - 1>(g);
    stage_load<L, E, S - 1>(v, t, buf);
    fft_inverse<L, E, S - 1, PRUNE>(v, t, g, buf, tw);
  }
}

// Register e of thread t after fft_forward sits at position last_pos(t, e).
template <int L, int E>
__device__ __forceinline__ int last_pos(int t, int e) {
  using St = Stage<L, E, stage_count(L, E) - 1>;
  const int u = e / St::R, k = e % St::R;
  return St::base(t, u) + k * St::M;
}

}  // namespace sf

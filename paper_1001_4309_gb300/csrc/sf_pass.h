// sf_pass.h -- what the row-pass kernels take: the supported FFT lengths
// and the per-pass descriptors (one separable half of one view).
#pragma once

#include <cuda_runtime.h>
#include <cudaTypedefs.h>

namespace sf {

constexpr int kMaxPassBatch = 16;  // (view, axis) passes per launch
constexpr int kE = 16;             // complex values per thread in the power-of-two FP32 FFT network
constexpr int kTcE = 16;           // radix of the tensor-core network's stages

enum PassKind : int { PASS_X_REAL = 0, PASS_X_CPLX = 1, PASS_Y = 2 };

// Supported FFT lengths: powers of two (radix-16 network) and 3 x powers of
// two / 9 x 256 (radix-24 first stage), ascending.
constexpr int kNumFftLengths = 13;
constexpr int kFftLengths[kNumFftLengths] = {64, 128, 256, 512, 1024, 1536, 2048, 2304, 3072, 4096, 4608, 6144, 8192};
template <int L>
constexpr int fft_length_slot_of() {
  int i = 0;
  while (i < kNumFftLengths && kFftLengths[i] != L) ++i;
  return i;
}

// One separable half of one view (Section 2.2, steps 2-9 along one axis).
// Row r is read from src[r * src_ld + p] (p < n0); output p of row r goes to
// dst[p * dst_ld + r] (p < n1).
//   X pass: src = hologram [rows = ny0][src_ld = nx0], dst = workspace [nx1][dst_ld = ny0]
//   Y pass: src = workspace [rows = nx1][src_ld = ny0], dst = view [ny1][dst_ld = nx1]
struct PassDesc {
  const void* src;
  float2* dst;        // complex output (Y: may be null)
  float* inten;       // Y only, may be null
  float* phase;       // Y only, may be null
  const float2* cin;  // input chirp, n0 entries
  const float2* cout; // output chirp (with 1/L and, on Y, the constant of Eq. 2), n1 entries
  const float2* H;    // kernel spectrum in register order, L entries
  int n0, n1;         // convolution input / output lengths along this axis
  int rows;           // independent rows of this pass
  int src_ld, dst_ld;
  int accumulate;     // Y only: add into dst instead of overwriting it
};

struct PassBatch {
  PassDesc d[kMaxPassBatch];
  int count;
};

// Outputs of a row tile leaving by 2D tensor stores (TMA): pass k's output is
// the float tensor {2 rows, n1} with row pitch dst_ld complex values, written
// in boxes of (all the tile's rows) x kOutBoxN outputs from a [n][row] tile.
constexpr int kOutBoxN = 256;
struct OutMaps {
  int use[kMaxPassBatch];  // pass k stores through map[k] (else plain stores)
  CUtensorMap map[kMaxPassBatch];
};

// Encodes pass d's output tensor map for tiles of box_rows rows; swizzle32:
// the box in shared memory is in the 32-byte swizzle (16-byte chunk index
// XOR bit 7 of the offset; box_rows = 4).  False (plain stores) when the pass
// also writes intensity or phase, accumulates, is not in plain device memory,
// has rows that do not start on 16-byte boundaries, or the driver's encoder is
// unavailable.
bool output_tensor_map(PassKind kind, const PassDesc& d, int box_rows, CUtensorMap* map, bool swizzle32 = false);

}  // namespace sf

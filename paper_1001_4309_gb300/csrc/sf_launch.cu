// sf_launch.cu -- launch dispatch by FFT length, and the plan-time chirp and
// twiddle kernels.
#include <cmath>

#include "sf_kernels.cuh"

namespace sf {

SF_DECLARE_LENGTH(64)
SF_DECLARE_LENGTH(128)
SF_DECLARE_LENGTH(256)
SF_DECLARE_LENGTH(512)
SF_DECLARE_LENGTH(1024)
SF_DECLARE_LENGTH(2048)
SF_DECLARE_LENGTH(4096)
SF_DECLARE_LENGTH(8192)
SF_DECLARE_LENGTH(1536)
SF_DECLARE_LENGTH(2304)
SF_DECLARE_LENGTH(3072)
SF_DECLARE_LENGTH(4608)
SF_DECLARE_LENGTH(6144)
SF_DECLARE_VARIANT(1024, 128)
SF_DECLARE_VARIANT(1024, 512)
SF_DECLARE_VARIANT(2048, 128)
SF_DECLARE_VARIANT(2048, 512)
SF_DECLARE_VARIANT(4096, 256)

int fft_length_slot(int L) {
  for (int i = 0; i < kNumFftLengths; ++i)
    if (kFftLengths[i] == L) return i;
  return -1;
}

bool fft_length_supported(int L) { return fft_length_slot(L) >= 0; }

namespace {
// cuTensorMapEncodeTiled from the driver (null when it cannot be reached)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}
}  // namespace

bool output_tensor_map(PassKind kind, const PassDesc& d, int box_rows, CUtensorMap* map, bool swizzle32) {
  if (!d.dst || d.rows <= 0 || d.n1 <= 0 || box_rows <= 0 || (box_rows & 1) != 0) return false;
  if (swizzle32 && box_rows != 4) return false;
  if (kind == PASS_Y && (d.inten || d.phase || d.accumulate)) return false;
  if ((reinterpret_cast<uintptr_t>(d.dst) & 15) != 0 || (d.dst_ld & 1) != 0) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, d.dst) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeDevice) return false;
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return false;
  const cuuint64_t dims[2] = {2 * (cuuint64_t)d.rows, (cuuint64_t)d.n1};
  const cuuint64_t strides[1] = {(cuuint64_t)d.dst_ld * 8};
  const cuuint32_t box[2] = {2 * (cuuint32_t)box_rows, (cuuint32_t)kOutBoxN};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d.dst, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                swizzle32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

#define SF_LENGTH_SWITCH(L, CALL)                 \
  switch (L) {                                    \
    case 64: { constexpr int LL = 64; CALL; }     \
    case 128: { constexpr int LL = 128; CALL; }   \
    case 256: { constexpr int LL = 256; CALL; }   \
    case 512: { constexpr int LL = 512; CALL; }   \
    case 1024: { constexpr int LL = 1024; CALL; } \
    case 2048: { constexpr int LL = 2048; CALL; } \
    case 4096: { constexpr int LL = 4096; CALL; } \
    case 8192: { constexpr int LL = 8192; CALL; } \
    case 1536: { constexpr int LL = 1536; CALL; } \
    case 2304: { constexpr int LL = 2304; CALL; } \
    case 3072: { constexpr int LL = 3072; CALL; } \
    case 4608: { constexpr int LL = 4608; CALL; } \
    case 6144: { constexpr int LL = 6144; CALL; } \
    default: break;                               \
  }

cudaError_t launch_pass(int L, PassKind kind, const PassBatch& b, int grid_x, const float4* tw, cudaStream_t s,
                        int variant) {
  if (variant != 0) {
    switch (L * 4 + variant) {
      case 1024 * 4 + 1: return launch_pass_cta<1024, pass_cta_variant(1024, 1)>(kind, b, grid_x, tw, s);
      case 1024 * 4 + 2: return launch_pass_cta<1024, pass_cta_variant(1024, 2)>(kind, b, grid_x, tw, s);
      case 2048 * 4 + 1: return launch_pass_cta<2048, pass_cta_variant(2048, 1)>(kind, b, grid_x, tw, s);
      case 2048 * 4 + 2: return launch_pass_cta<2048, pass_cta_variant(2048, 2)>(kind, b, grid_x, tw, s);
      case 4096 * 4 + 1: return launch_pass_cta<4096, pass_cta_variant(4096, 1)>(kind, b, grid_x, tw, s);
      default: return cudaErrorInvalidValue;
    }
  }
  SF_LENGTH_SWITCH(L, return launch_pass_t<LL>(kind, b, grid_x, tw, s))
  return cudaErrorInvalidValue;
}

cudaError_t launch_hspec(int L, const AxisCoef* axes_dev, int n_axes, const float4* tw, cudaStream_t s) {
  SF_LENGTH_SWITCH(L, return launch_hspec_t<LL>(axes_dev, n_axes, tw, s))
  return cudaErrorInvalidValue;
}

namespace {
template <int L>
int variant_rows(int variant) {
  constexpr int c1 = pass_cta_variant(L, 1), c2 = pass_cta_variant(L, 2);
  if (variant == 1) return c1 ? PassShape<L, c1 ? c1 : pass_cta_target(L)>::G : 0;
  if (variant == 2) return c2 ? PassShape<L, c2 ? c2 : pass_cta_target(L)>::G : 0;
  return PassShape<L>::G;
}
}  // namespace

int pass_rows_per_cta(int L, int variant) {
  SF_LENGTH_SWITCH(L, return variant_rows<LL>(variant))
  return 0;
}

// Input and output chirp vectors of every (view, axis): blockIdx.y = axis,
// blockIdx.z = 0 for exp(i pi psi_in(m0)), 1 for out_scale exp(i pi psi_out(m1)).
__global__ void k_chirps(const AxisCoef* __restrict__ axes) {
  const AxisCoef& a = axes[blockIdx.y];
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t mm = (uint64_t)m * (uint64_t)m;
  if (blockIdx.z == 0) {
    if (m < a.n0) a.cin[m] = expi_fx(a.in2 * mm + a.in1 * (uint64_t)m + a.in0);
  } else if (m < a.n1) {
    const uint64_t ph = a.out2 * mm + a.out1 * (uint64_t)m + a.out0;
    const double ang = (double)(int64_t)ph * 0x1p-63;
    double s, c;
    sincospi(ang, &s, &c);
    a.cout[m] = make_float2((float)(a.out_scale * c), (float)(a.out_scale * s));
  }
}

cudaError_t launch_chirps(const AxisCoef* axes_dev, int n_axes, int max_n, cudaStream_t s) {
  const dim3 grid((max_n + 255) / 256, n_axes, 2);
  k_chirps<<<grid, 256, 0, s>>>(axes_dev);
  return cudaGetLastError();
}

size_t twiddle_entries(int L) { return (size_t)tw_table_entries(L, fft_e(L)); }

// Per-stage twiddle tables (layout described at stage_tw_entries), built in
// double precision on the host and rounded to float.
void build_twiddles(int L, float4* tab) {
  const double two_pi = 6.283185307179586476925286766559;
  auto w = [&](long e, float& re, float& im) {
    const double a = two_pi * (double)(e % L) / (double)L;
    re = (float)std::cos(a);
    im = (float)-std::sin(a);
  };
  const int E = fft_e(L);
  for (int st = 0; st < stage_count(L, E); ++st) {
    const int MP = stage_mprev(L, E, st), R = stage_radix(L, E, st), M = MP / R;
    if (M <= 1) continue;
    float4* base = tab + stage_tw_offset(L, E, st);
    for (int q = 0; q < R / 2; ++q)
      for (int n = 0; n < M; ++n) {
        float4 f;
        w((long)n * (2 * q) * (L / MP), f.x, f.y);
        w((long)n * (2 * q + 1) * (L / MP), f.z, f.w);
        base[q * M + n] = f;
      }
  }
}

}  // namespace sf

// sf_static.cu -- allocation-free single-view reconstruction.
//
// Some callers cannot allocate device memory once they are running: a plugin
// inside a host application that owns every device allocation, or an
// acquisition loop whose memory budget is fixed before the first frame.
// They cannot create a plan, because shifted_fresnel_plan calls cudaMalloc.
// shifted_fresnel_execute_static serves them: everything a plan would own
// (twiddle tables, chirp vectors, kernel spectra, the intermediate field)
// lives in one fixed file-scope device array, and each call rebuilds the
// per-view vectors there before running the same two row-pass kernels as
// shifted_fresnel_execute.  No path here calls cudaMalloc, cudaFree or any
// allocating library routine.
//
// Consequences a caller must know:
//   - every GPU that loads this library holds SF_STATIC_SCRATCH_BYTES of
//     device memory for the array until the process exits;
//   - the array is shared by every call on a device and keeps the previous
//     call's contents; every region a call reads is rewritten by that call
//     first, so nothing needs clearing, but calls that overlap on the GPU
//     (different streams, or host threads racing on one device) corrupt
//     each other's results;
//   - the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress, which may load the module), so make that first
//     call before any stream capture; the address is kept per device and
//     CUDA context, so the first call after a device reset (a new context)
//     looks it up again and must also come before any capture.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "sf_kernels.cuh"

// The scratch array.  Host code must not use this name as a device address
// (on the host it is only a stand-in symbol); the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char sf_static_scratch[SF_STATIC_SCRATCH_BYTES];

namespace sf {
namespace {

constexpr size_t kTwBytes = 32u << 10;   // one per-stage twiddle table, L <= 2048
constexpr size_t kVecBytes = 16u << 10;  // one chirp vector or kernel spectrum, <= 2048 complex
constexpr size_t kOffTwX = 0, kOffTwY = kTwBytes, kOffVec = 2 * kTwBytes;
constexpr size_t kOffWork = kOffVec + 6 * kVecBytes;
static_assert(kOffWork + sizeof(float2) * (size_t)SF_STATIC_MAX_WORKSPACE_ELEMS <= SF_STATIC_SCRATCH_BYTES,
              "scratch layout exceeds the declared size");
static_assert(sizeof(float4) * tw_table_entries(SF_STATIC_MAX_FFT_LENGTH, fft_e(SF_STATIC_MAX_FFT_LENGTH)) <= kTwBytes &&
                  sizeof(float4) * tw_table_entries(1536, fft_e(1536)) <= kTwBytes,
              "twiddle table slot too small");
static_assert(sizeof(float2) * SF_STATIC_MAX_FFT_LENGTH <= kVecBytes, "vector slot too small");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  void* addr = nullptr;  // device address of the array ...
  void* ctx = nullptr;   // ... in this context (a device reset makes a new one)
};
ScratchAddr g_scratch[kMaxDevices];

// The calling thread's current CUDA context (driver cuCtxGetCurrent, reached
// through the runtime's entry-point query); nullptr if unavailable.
void* current_context() {
  using Fn = int (*)(void**);
  static const Fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (Fn) nullptr;
    }
    return reinterpret_cast<Fn>(f);
  }();
  void* c = nullptr;
  if (!fn || fn(&c) != 0) return nullptr;
  return c;
}

// Device address of the scratch array on the current device `dev`, looked up
// once per device and context (again after a device reset).
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return SF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchAddr& sa = g_scratch[dev];
  void* ctx = current_context();
  if (!sa.addr || !ctx || ctx != sa.ctx) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, sf_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return SF_ERR_CUDA;
    }
    sa.addr = p;
    sa.ctx = current_context();  // the lookup has made the context current if it was not
  }
  *out = sa.addr;
  return SF_OK;
}

// SF_OK for device (or managed) memory of `dev`; host memory cannot be staged
// without allocating, so it is rejected.
int check_device_pointer(const void* p, int dev) {
  if (!p) return SF_OK;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_INVALID_ARG;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return SF_ERR_INVALID_ARG;
  return at.device == dev ? SF_OK : SF_ERR_DEVICE_MISMATCH;
}

// Per-stage twiddle table of length L (same layout as the plan's), one
// thread per float4 entry, from double-precision sincospi.
__global__ void k_static_twiddles(float4* tab, int L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int E = fft_e(L);
  const int ns = stage_count(L, E);
  if (i >= stage_tw_offset(L, E, ns)) return;
  int st = 0;
  while (st + 1 < ns && i >= stage_tw_offset(L, E, st + 1)) ++st;
  const int MP = stage_mprev(L, E, st), R = stage_radix(L, E, st), M = MP / R;
  const int local = i - stage_tw_offset(L, E, st), q = local / M, n = local - q * M;
  double s0, c0, s1, c1;
  sincospi(-2.0 * (double)(((long long)n * (2 * q) * (L / MP)) % L) / (double)L, &s0, &c0);
  sincospi(-2.0 * (double)(((long long)n * (2 * q + 1) * (L / MP)) % L) / (double)L, &s1, &c1);
  tab[i] = make_float4((float)c0, (float)s0, (float)c1, (float)s1);
}

// Chirp vectors of both axes from coefficients passed by value:
// blockIdx.y = axis, blockIdx.z = 0 (input chirp) or 1 (output chirp).
__global__ void k_static_chirps(AxisCoef ax, AxisCoef ay) {
  const AxisCoef& a = blockIdx.y == 0 ? ax : ay;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t mm = (uint64_t)m * (uint64_t)m;
  if (blockIdx.z == 0) {
    if (m < a.n0) a.cin[m] = expi_fx(a.in2 * mm + a.in1 * (uint64_t)m + a.in0);
  } else if (m < a.n1) {
    const double ang = (double)(int64_t)(a.out2 * mm + a.out1 * (uint64_t)m + a.out0) * 0x1p-63;
    double s, c;
    sincospi(ang, &s, &c);
    a.cout[m] = make_float2((float)(a.out_scale * c), (float)(a.out_scale * s));
  }
}

// Kernel spectrum of one axis (coefficients by value), register order.
template <int L>
__global__ void __launch_bounds__(L / fft_e(L)) k_static_hspec(AxisCoef a, const float4* __restrict__ tw) {
  constexpr int T = L / fft_e(L), E = fft_e(L);
  extern __shared__ float2 smem[];
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

cudaError_t launch_static_hspec(const AxisCoef& a, const float4* tw, cudaStream_t s) {
  switch (a.L) {
#define SF_STATIC_HSPEC_CASE(LL) \
  case LL: k_static_hspec<LL><<<1, LL / fft_e(LL), sizeof(float2) * buf_elems(LL), s>>>(a, tw); return cudaGetLastError();
    SF_STATIC_HSPEC_CASE(64)
    SF_STATIC_HSPEC_CASE(128)
    SF_STATIC_HSPEC_CASE(256)
    SF_STATIC_HSPEC_CASE(512)
    SF_STATIC_HSPEC_CASE(1024)
    SF_STATIC_HSPEC_CASE(1536)
    SF_STATIC_HSPEC_CASE(2048)
#undef SF_STATIC_HSPEC_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace sf

using namespace sf;

extern "C" int shifted_fresnel_execute_static(const sf_view* view, const void* holo, void* view_out,
                                              float* intensity, float* phase, void* stream) {
  if (!view || !holo) return SF_ERR_INVALID_ARG;
  int rc = validate_view(*view);
  if (rc) return rc;
  if (!view_out && !intensity && !phase) return SF_ERR_INVALID_ARG;
  AxisCoef ax[2];
  axis_coefficients(*view, 0, ax[0]);
  axis_coefficients(*view, 1, ax[1]);
  if (ax[0].L > SF_STATIC_MAX_FFT_LENGTH || ax[1].L > SF_STATIC_MAX_FFT_LENGTH ||
      (size_t)view->nx1 * (size_t)view->ny0 > (size_t)SF_STATIC_MAX_WORKSPACE_ELEMS)
    return SF_ERR_UNSUPPORTED_SIZE;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  for (const void* p : {holo, (const void*)view_out, (const void*)intensity, (const void*)phase}) {
    rc = check_device_pointer(p, dev);
    if (rc) return rc;
  }
  void* base = nullptr;
  rc = scratch_address(dev, &base);
  if (rc) return rc;

  char* b = static_cast<char*>(base);
  float4* twx = reinterpret_cast<float4*>(b + kOffTwX);
  float4* twy = ax[1].L == ax[0].L ? twx : reinterpret_cast<float4*>(b + kOffTwY);
  for (int a = 0; a < 2; ++a) {
    ax[a].cin = reinterpret_cast<float2*>(b + kOffVec + (3 * a + 0) * kVecBytes);
    ax[a].cout = reinterpret_cast<float2*>(b + kOffVec + (3 * a + 1) * kVecBytes);
    ax[a].H = reinterpret_cast<float2*>(b + kOffVec + (3 * a + 2) * kVecBytes);
  }
  float2* work = reinterpret_cast<float2*>(b + kOffWork);  // [nx1][ny0]
  cudaStream_t s = (cudaStream_t)stream;

  uint64_t launches = 0;
  cudaError_t e = cudaSuccess;
  const int n_tw_x = (int)twiddle_entries(ax[0].L), n_tw_y = (int)twiddle_entries(ax[1].L);
  k_static_twiddles<<<(n_tw_x + 255) / 256, 256, 0, s>>>(twx, ax[0].L);
  ++launches;
  e = cudaGetLastError();
  if (e == cudaSuccess && twy != twx) {
    k_static_twiddles<<<(n_tw_y + 255) / 256, 256, 0, s>>>(twy, ax[1].L);
    ++launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int max_n = std::max(std::max(ax[0].n0, ax[0].n1), std::max(ax[1].n0, ax[1].n1));
    k_static_chirps<<<dim3((max_n + 255) / 256, 2, 2), 256, 0, s>>>(ax[0], ax[1]);
    ++launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) { e = launch_static_hspec(ax[0], twx, s); ++launches; }
  if (e == cudaSuccess) { e = launch_static_hspec(ax[1], twy, s); ++launches; }

  // the same two row passes as shifted_fresnel_execute, on the scratch workspace
  const bool cplx = (view->flags & SF_IN_COMPLEX) != 0;
  for (int a = 0; a < 2 && e == cudaSuccess; ++a) {
    PassBatch pb;
    std::memset(&pb, 0, sizeof(pb));
    pb.count = 1;
    PassDesc& d = pb.d[0];
    d.cin = ax[a].cin;
    d.cout = ax[a].cout;
    d.H = ax[a].H;
    d.n0 = ax[a].n0;
    d.n1 = ax[a].n1;
    if (a == 0) {
      d.src = holo;
      d.dst = work;
      d.rows = view->ny0;
      d.src_ld = view->nx0;
      d.dst_ld = view->ny0;
    } else {
      d.src = work;
      d.dst = static_cast<float2*>(view_out);
      d.inten = intensity;
      d.phase = phase;
      d.rows = view->nx1;
      d.src_ld = view->ny0;
      d.dst_ld = view->nx1;
    }
    const int G = pass_rows_per_cta(ax[a].L);
    const PassKind kind = a == 1 ? PASS_Y : (cplx ? PASS_X_CPLX : PASS_X_REAL);
    e = launch_pass(ax[a].L, kind, pb, (d.rows + G - 1) / G, a == 0 ? twx : twy, s);
    ++launches;
  }
  count_launches(launches);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

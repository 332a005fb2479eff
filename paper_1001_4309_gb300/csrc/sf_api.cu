// sf_api.cu -- host side of the C ABI declared in include/shifted_fresnel.h.
//
// Plan: per view and axis, the phase polynomials of Eqs. 2-4 (Section 2.1)
// are reduced modulo 2 pi into 64-bit fixed point on the host, and device
// kernels turn them into the input chirp, the output chirp and the kernel
// spectrum FFT(h) (Section 2.2, steps 5-6) once.  Execute: one x-pass launch
// and one y-pass launch per group of views sharing FFT lengths.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <map>
#include <string>
#include <new>
#include <vector>

#include "shifted_fresnel.h"
#include "sf_internal.h"

using namespace sf;

namespace {

std::atomic<uint64_t> g_launches{0};

constexpr uint32_t kKnownFlags = SF_OUT_INTENSITY | SF_OUT_PHASE | SF_NO_PREFACTOR | SF_IN_COMPLEX;
constexpr int kMaxViews = 4096;
constexpr int kMinFFT = 64;

struct ViewState {
  sf_view v;
  AxisCoef ax[2];          // [0] = x, [1] = y; device pointers into the arena
  AxisCoef adj[2];         // adjoint passes: [0] along x (nx1 -> nx0), [1] along y (ny1 -> ny0)
  float2* hpos[2] = {nullptr, nullptr};  // kernel spectra in position order (mma.sync tensor-core axes)
  float2* hnat[2] = {nullptr, nullptr};  // kernel spectra in natural order / sqrt(L) (tcgen05 axes)
  float2* work = nullptr;  // [nx1][ny0] intermediate after the x pass (transposed)
  float2* st_out = nullptr;  // host-I/O staging (lazily allocated)
  float* st_int = nullptr;
  float* st_ph = nullptr;
};

// Resources of shifted_fresnel_execute_batch, built by its first call.
struct BatchState {
  bool init = false;
  int n_holos = 0;                       // hologram count the graphs are built for
  std::vector<BatchGroup> groups;
  int items_per_holo = 0, grid = 0;
  const void* kfunc = nullptr;           // persistent kernel: general, or specialised to one length
  size_t ksmem = 0;                      // its dynamic shared memory
  std::vector<float2*> slot1;            // second intermediate slot per view
  // two-stream batch: holograms per row-pass launch (sk) and their
  // intermediate slots sslot[(group * sk + j) * n_views + v], group = chunk parity
  int sk = 0;
  std::vector<float2*> sslot;
  void* d_sslot = nullptr;
  BatchGroup* d_groups = nullptr;
  int* d_item_group = nullptr;           // group of each item within a hologram
  int* d_error = nullptr;
  void* d_fixed = nullptr;               // slot1 workspaces + groups + error word
  void* d_sized = nullptr;               // descriptors + counters for n_holos
  PassDesc* d_descs = nullptr;
  int* d_done = nullptr;                 // n_holos * n_groups completion counters, then the item counter
  PassDesc* h_descs[2] = {nullptr, nullptr};  // pinned, alternated between calls
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int flip = 0;
  // the per-length kernels on two streams (even / odd holograms, one slot each)
  cudaStream_t st[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  // those launches captured as a CUDA graph, replayed while calls pass the same buffers
  cudaGraphExec_t sgraph = nullptr;
  std::vector<const void*> skey;         // hologram count and every buffer pointer of the captured call
  uint64_t sgraph_kernels = 0;           // kernels in the graph
  cudaStream_t cap = nullptr;            // the graph is captured and launched on this plan stream
  cudaEvent_t pre = nullptr, post = nullptr;  // caller's stream -> cap -> caller's stream
  std::map<int, int> choice;             // hologram count -> BATCH_PERSISTENT / BATCH_STREAMS (autotuned)
};
enum { BATCH_PERSISTENT = 0, BATCH_STREAMS = 1 };

}  // namespace

constexpr int kSchedInts = 1 + sf::kMaxPassBatch;  // one fused launch's schedule buffer

struct sf_plan_s {
  int device = 0;
  int nx0 = 0, ny0 = 0;
  bool in_complex = false;
  std::vector<ViewState> views;
  std::map<int, float4*> tw;  // per-stage twiddle tables per FFT length
  int precision = SF_PREC_FP32;
  uint32_t* tc_frags = nullptr;  // per-lane DFT fragments and twiddle tables of the tensor-core pass
  // DFT operands and twiddles of the tcgen05 row pass, FFT length 512 / 1024 / 2048
  void* t5_consts[3] = {nullptr, nullptr, nullptr};
  // schedule buffers of fused tcgen05 launches (tile counter, per-view x-tile counts): execute's,
  // then one per batch stream, kSchedInts each
  int* t5_sched = nullptr;
  int* dev_err = nullptr;        // device error word of the persistent kernels (bounded waits)
  AxisCoef* axes_dev = nullptr;  // coefficient table read by the chirp and spectrum kernels
  // row-pass kernel per (length slot, kind): 0 grid, 1 persistent TMA, 2 / 3 grid with half / twice the rows per CTA
  int impl[kNumFftLengths][3] = {};
  int sms = 0;
  void* arena = nullptr;
  void* st_holo = nullptr;
  std::vector<void*> staging;
  cudaEvent_t prof[3] = {nullptr, nullptr, nullptr};
  // adjoint scratch, allocated by the first shifted_fresnel_adjoint call
  float2* adj_work = nullptr;   // 3 x max(nx0 * ny1): x-pass intermediates of g, x1 g, y1 g
  float2* adj_G = nullptr;      // 3 x nx0 * ny0: A^H g, A^H (x1 g), A^H (y1 g)
  float2* adj_u1 = nullptr;     // max(nx1 * ny1): recomputed view field
  float2* adj_xy = nullptr;     // 2 x max(nx1 * ny1): x1 g and y1 g
  float2* adj_gst = nullptr;    // max(nx1 * ny1): staging of a host gradient
  float2* adj_out = nullptr;    // nx0 * ny0: staging of a host grad_holo
  double2* adj_part = nullptr;  // kZGradBlocks x 5 partial sums
  double* adj_z = nullptr;      // n_views dL/dz values
  double* loss_part = nullptr;  // kZGradBlocks block partials of shifted_fresnel_intensity_loss
  BatchState batch;
  // host-output overlap, created on first use: a copy stream, one event per
  // view, and the pipeline's x-pass stream (lowest priority) and y-pass
  // stream (highest), with their fork / join and per-view x-pass events
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> view_done;
  cudaEvent_t copies_done = nullptr;
  cudaStream_t pipe_x = nullptr, pipe_y = nullptr;
  std::vector<cudaEvent_t> x_done;
  cudaEvent_t pipe_fork = nullptr, pipe_join = nullptr, holo_half = nullptr, y_half = nullptr;
  // execute's second compute stream (half of the views), created on first use
  cudaStream_t split_stream = nullptr;
  cudaEvent_t split_fork = nullptr, split_join = nullptr;
};

namespace sf {
namespace {
// the tcgen05 constants of FFT length L, or null (no tcgen05 pass at L in this plan)
void* t5_consts_for(const sf_plan_s* p, int L) {
  return L == 512 ? p->t5_consts[0] : L == 1024 ? p->t5_consts[1] : L == 2048 ? p->t5_consts[2] : nullptr;
}
}  // namespace
}  // namespace sf

namespace sf {

bool finite_pos(double x) { return std::isfinite(x) && x > 0; }

// Reduce a phase coefficient (units of pi) modulo 2 into 64-bit fixed point.
uint64_t to_fx(double c) {
  double r = std::fmod(c, 2.0);
  if (r < 0) r += 2.0;
  const double s = std::ldexp(r, 63);
  if (!(s < 18446744073709551616.0)) return 0;
  return (uint64_t)s;
}

int next_fft_length(int need, bool allow_mixed) {
  for (int i = 0; i < kNumFftLengths; ++i) {
    const int L = kFftLengths[i];
    if (L >= std::max(need, kMinFFT) && (allow_mixed || (L & (L - 1)) == 0)) return L;
  }
  return 0;
}

int validate_view(const sf_view& v) {
  if (!finite_pos(v.wavelength) || !std::isfinite(v.z) || v.z == 0.0) return SF_ERR_INVALID_ARG;
  if (!finite_pos(v.px0) || !finite_pos(v.py0) || !finite_pos(v.px1) || !finite_pos(v.py1)) return SF_ERR_INVALID_ARG;
  if (!std::isfinite(v.ox0) || !std::isfinite(v.oy0) || !std::isfinite(v.ox1) || !std::isfinite(v.oy1))
    return SF_ERR_INVALID_ARG;
  if (v.nx0 <= 0 || v.ny0 <= 0 || v.nx1 <= 0 || v.ny1 <= 0) return SF_ERR_INVALID_ARG;
  if (v.flags & ~kKnownFlags) return SF_ERR_INVALID_ARG;
  if ((int64_t)v.nx0 + v.nx1 - 1 > SF_MAX_CONV_LENGTH || (int64_t)v.ny0 + v.ny1 - 1 > SF_MAX_CONV_LENGTH)
    return SF_ERR_UNSUPPORTED_SIZE;
  return SF_OK;
}

// Phase polynomials of one axis (units of pi).  With beta = 1/(lambda z),
// a = o - floor(n/2) p, D = a1 - a0 and S = p0 p1 beta (the S of Eqs. 2-4):
//   beta (x1 - x0)^2 = S (m1 - m0)^2 + psi_in(m0) + psi_out(m1)
//   psi_in(m0)  = (beta p0^2 - S) m0^2 - 2 beta p0 D m0
//   psi_out(m1) = (beta p1^2 - S) m1^2 + 2 beta p1 D m1 + beta D^2
void axis_coefficients(const sf_view& v, int axis, AxisCoef& a, int L) {
  const double lam = v.wavelength, z = v.z, beta = 1.0 / (lam * z);
  const int n0 = axis == 0 ? v.nx0 : v.ny0, n1 = axis == 0 ? v.nx1 : v.ny1;
  const double p0 = axis == 0 ? v.px0 : v.py0, p1 = axis == 0 ? v.px1 : v.py1;
  const double o0 = axis == 0 ? v.ox0 : v.oy0, o1 = axis == 0 ? v.ox1 : v.oy1;
  const double a0 = o0 - (double)(n0 / 2) * p0, a1 = o1 - (double)(n1 / 2) * p1;
  const double D = a1 - a0, S = p0 * p1 * beta;
  a.n0 = n0;
  a.n1 = n1;
  a.L = L > 0 ? L : next_fft_length(n0 + n1 - 1, true);
  a.in2 = to_fx(beta * p0 * p0 - S);
  a.in1 = to_fx(-2.0 * beta * p0 * D);
  a.in0 = 0;
  a.out2 = to_fx(beta * p1 * p1 - S);
  a.out1 = to_fx(2.0 * beta * p1 * D);
  double c0 = beta * D * D;
  a.out_scale = 1.0 / (double)a.L;
  if (axis == 1 && !(v.flags & SF_NO_PREFACTOR)) {
    // exp(i k z) / (i lambda z) = exp(i pi (2 z / lambda - 1/2)) / (lambda z)
    c0 = std::fmod(c0, 2.0) + std::fmod(2.0 * (z / lam), 2.0) - 0.5;
    a.out_scale /= lam * z;
  }
  a.out0 = to_fx(c0);
  a.h2 = to_fx(S);
}

// Adjoint of one axis, A^H = D_in^H T^H D_out^H: a Bluestein pass from n1 to
// n0 samples whose input chirp is the conjugate of the forward output chirp
// (including the constant of Eq. 2), whose kernel is conj(h) (h is even, so
// T^H is the Toeplitz operator of conj(h) with the lengths swapped) and whose
// output chirp is the conjugate of the forward input chirp, with the same
// real scale (1/L, and 1/(lambda z) on y).
void adjoint_axis_coefficients(const sf_view& v, int axis, AxisCoef& a, int L) {
  AxisCoef f;
  axis_coefficients(v, axis, f, L);
  a = f;
  a.n0 = f.n1;
  a.n1 = f.n0;
  a.in2 = 0 - f.out2;
  a.in1 = 0 - f.out1;
  a.in0 = 0 - f.out0;
  a.out2 = 0 - f.in2;
  a.out1 = 0 - f.in1;
  a.out0 = 0 - f.in0;
  a.h2 = 0 - f.h2;
}

void count_launches(uint64_t n) { g_launches += n; }

}  // namespace sf

namespace {

// Intermediate of one view: nx1 columns of ny0 rows.
size_t work_elems(const sf_view& v) { return (size_t)v.ny0 * v.nx1; }

struct Arena {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

enum PtrKind { PTR_DEVICE, PTR_HOST, PTR_OTHER_DEVICE };

PtrKind classify(const void* p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
    return at.device == device ? PTR_DEVICE : PTR_OTHER_DEVICE;
  return PTR_HOST;
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void free_batch_sized(BatchState& b) {
  for (int k = 0; k < 2; ++k) {
    if (b.exec[k]) cudaGraphExecDestroy(b.exec[k]);
    if (b.graph[k]) cudaGraphDestroy(b.graph[k]);
    if (b.h_descs[k]) cudaFreeHost(b.h_descs[k]);
    b.exec[k] = nullptr;
    b.graph[k] = nullptr;
    b.h_descs[k] = nullptr;
  }
  if (b.d_sized) cudaFree(b.d_sized);
  b.d_sized = nullptr;
  b.n_holos = 0;
}

void free_plan(sf_plan p) {
  if (!p) return;
  for (cudaEvent_t e : p->view_done) cudaEventDestroy(e);
  if (p->copies_done) cudaEventDestroy(p->copies_done);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  for (cudaEvent_t e : p->x_done) cudaEventDestroy(e);
  for (cudaEvent_t e : {p->pipe_fork, p->pipe_join, p->holo_half, p->y_half})
    if (e) cudaEventDestroy(e);
  if (p->pipe_x) cudaStreamDestroy(p->pipe_x);
  if (p->pipe_y) cudaStreamDestroy(p->pipe_y);
  if (p->split_fork) cudaEventDestroy(p->split_fork);
  if (p->split_join) cudaEventDestroy(p->split_join);
  if (p->split_stream) cudaStreamDestroy(p->split_stream);
  free_batch_sized(p->batch);
  for (int k = 0; k < 2; ++k) {
    if (p->batch.ev[k]) cudaEventDestroy(p->batch.ev[k]);
    if (p->batch.join[k]) cudaEventDestroy(p->batch.join[k]);
    if (p->batch.st[k]) cudaStreamDestroy(p->batch.st[k]);
  }
  if (p->batch.fork) cudaEventDestroy(p->batch.fork);
  if (p->batch.sgraph) cudaGraphExecDestroy(p->batch.sgraph);
  if (p->batch.pre) cudaEventDestroy(p->batch.pre);
  if (p->batch.post) cudaEventDestroy(p->batch.post);
  if (p->batch.cap) cudaStreamDestroy(p->batch.cap);
  if (p->batch.d_fixed) cudaFree(p->batch.d_fixed);
  if (p->batch.d_sslot) cudaFree(p->batch.d_sslot);
  for (void* s : p->staging) cudaFree(s);
  if (p->arena) cudaFree(p->arena);
  delete p;
}

// Second compute stream and its fork / join events.
int ensure_split_resources(sf_plan p) {
  if (p->split_stream) return SF_OK;
  cudaStream_t st = nullptr;
  cudaEvent_t f = nullptr, j = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&f, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (f) cudaEventDestroy(f);
    if (j) cudaEventDestroy(j);
    if (st) cudaStreamDestroy(st);
    return SF_ERR_CUDA;
  }
  p->split_stream = st;
  p->split_fork = f;
  p->split_join = j;
  return SF_OK;
}

// Copy stream and events for overlapping device-to-host copies with compute.
int ensure_copy_resources(sf_plan p) {
  if (p->copy_stream) return SF_OK;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  std::vector<cudaEvent_t> ev(p->views.size(), nullptr);
  cudaEvent_t done = nullptr;
  bool ok = cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess;
  for (size_t i = 0; ok && i < ev.size(); ++i) ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    if (done) cudaEventDestroy(done);
    cudaStreamDestroy(cs);
    return SF_ERR_CUDA;
  }
  p->copy_stream = cs;
  p->view_done = ev;
  p->copies_done = done;
  return SF_OK;
}

// Copy stream and events, plus the two pipeline streams of the host-output
// path: x passes at the lowest stream priority, y passes at the highest, so a
// view's y pass takes the SMs ahead of the next views' x passes and the
// x passes fill the y pass's launch tail.
int ensure_pipeline_resources(sf_plan p) {
  int rc = ensure_copy_resources(p);
  if (rc || p->pipe_x) return rc;
  int least = 0, greatest = 0;
  cudaStream_t xs = nullptr, ys = nullptr;
  std::vector<cudaEvent_t> ev(p->views.size(), nullptr);
  cudaEvent_t f = nullptr, j = nullptr, h = nullptr, yh = nullptr;
  bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
            cudaStreamCreateWithPriority(&xs, cudaStreamNonBlocking, least) == cudaSuccess &&
            cudaStreamCreateWithPriority(&ys, cudaStreamNonBlocking, greatest) == cudaSuccess &&
            cudaEventCreateWithFlags(&f, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&h, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&yh, cudaEventDisableTiming) == cudaSuccess;
  for (size_t i = 0; ok && i < ev.size(); ++i) ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    for (cudaEvent_t x : {f, j, h, yh})
      if (x) cudaEventDestroy(x);
    if (xs) cudaStreamDestroy(xs);
    if (ys) cudaStreamDestroy(ys);
    return SF_ERR_CUDA;
  }
  p->pipe_x = xs;
  p->pipe_y = ys;
  p->x_done = ev;
  p->pipe_fork = f;
  p->pipe_join = j;
  p->holo_half = h;
  p->y_half = yh;
  return SF_OK;
}

int stage_alloc(sf_plan p, void** out, size_t bytes) {
  if (*out) return SF_OK;
  if (cudaMalloc(out, bytes) != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return SF_ERR_OOM;
  }
  p->staging.push_back(*out);
  return SF_OK;
}


// Adjoint scratch, one cudaMalloc on the first shifted_fresnel_adjoint call.
int alloc_adjoint_scratch(sf_plan p) {
  if (p->adj_work) return SF_OK;
  size_t w = 1, v1 = 1;
  const size_t h0 = (size_t)p->nx0 * p->ny0;
  for (const ViewState& vs : p->views) {
    w = std::max(w, (size_t)vs.v.nx0 * vs.v.ny1);
    v1 = std::max(v1, (size_t)vs.v.nx1 * vs.v.ny1);
  }
  Arena ar;
  const size_t o_work = ar.take(sizeof(float2) * 3 * w), o_G = ar.take(sizeof(float2) * 3 * h0);
  const size_t o_u1 = ar.take(sizeof(float2) * v1), o_xy = ar.take(sizeof(float2) * 2 * v1);
  const size_t o_gst = ar.take(sizeof(float2) * v1), o_out = ar.take(sizeof(float2) * h0);
  const size_t o_part = ar.take(sizeof(double2) * 5 * kZGradBlocks), o_z = ar.take(sizeof(double) * p->views.size());
  void* base = nullptr;
  if (cudaMalloc(&base, ar.off) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_OOM;
  }
  p->staging.push_back(base);
  char* b = static_cast<char*>(base);
  p->adj_work = reinterpret_cast<float2*>(b + o_work);
  p->adj_G = reinterpret_cast<float2*>(b + o_G);
  p->adj_u1 = reinterpret_cast<float2*>(b + o_u1);
  p->adj_xy = reinterpret_cast<float2*>(b + o_xy);
  p->adj_gst = reinterpret_cast<float2*>(b + o_gst);
  p->adj_out = reinterpret_cast<float2*>(b + o_out);
  p->adj_part = reinterpret_cast<double2*>(b + o_part);
  p->adj_z = reinterpret_cast<double*>(b + o_z);
  return SF_OK;
}

// Launch one pass over up to kMaxPassBatch descriptors of one FFT length.
cudaError_t run_pass(sf_plan p, int L, PassKind kind, const PassDesc* descs, int n, cudaStream_t s) {
  PassBatch b;
  std::memset(&b, 0, sizeof(b));
  int max_rows = 0;
  for (int i = 0; i < n; ++i) {
    b.d[i] = descs[i];
    max_rows = std::max(max_rows, descs[i].rows);
  }
  b.count = n;
  const int G = pass_rows_per_cta(L);
  ++g_launches;
  return launch_pass(L, kind, b, (max_rows + G - 1) / G, p->tw[L], s);
}

bool env_is(const char* name, const char* value) {
  const char* v = std::getenv(name);
  return v && std::strcmp(v, value) == 0;
}

long long env_ll(const char* name, long long dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoll(v) : dflt;
}

// Build (or rebuild for a new hologram count) the batch graph:
// memcpy(descriptors <- pinned table), memset(counters), persistent kernel.
// Every FFT length of the plan fits the persistent batch kernel.
bool batch_persistent_supported(sf_plan p) {
  if (p->precision != SF_PREC_FP32) return false;  // its tiles are the FP32 network only
  for (const ViewState& vs : p->views)
    for (int ph = 0; ph < 2; ++ph)
      if (!batch_length_supported(vs.ax[ph].L)) return false;
  return true;
}

int batch_prepare(sf_plan p, int n_holos, bool persistent) {
  BatchState& b = p->batch;
  const int nv = (int)p->views.size();
  if (persistent && !batch_persistent_supported(p)) return SF_ERR_UNSUPPORTED_SIZE;
  if (!b.init) {
    b.groups.clear();
    int first = 0;
    for (int ph = 0; ph < 2; ++ph)
      for (int v = 0; v < nv; ++v) {
        const ViewState& vs = p->views[v];
        const int L = vs.ax[ph].L;
        const int G = std::max(1, batch_tile_rows(L)), chunk = std::max(1, batch_item_tiles(L));
        const int rows = ph == 0 ? vs.v.ny0 : vs.v.nx1;
        const int tiles = (rows + G - 1) / G, items = (tiles + chunk - 1) / chunk;
        b.groups.push_back({first, items, tiles, chunk, L, ph});
        first += items;
      }
    b.items_per_holo = first;
    Arena ar;
    std::vector<size_t> off(nv);
    for (int v = 0; v < nv; ++v) off[v] = ar.take(sizeof(float2) * work_elems(p->views[v].v));
    const size_t o_groups = ar.take(sizeof(BatchGroup) * b.groups.size());
    const size_t o_item_group = ar.take(sizeof(int) * b.items_per_holo);
    if (cudaMalloc(&b.d_fixed, ar.off) != cudaSuccess) {
      cudaGetLastError();
      return SF_ERR_OOM;
    }
    char* base = static_cast<char*>(b.d_fixed);
    b.slot1.resize(nv);
    for (int v = 0; v < nv; ++v) b.slot1[v] = reinterpret_cast<float2*>(base + off[v]);
    b.d_groups = reinterpret_cast<BatchGroup*>(base + o_groups);
    b.d_error = p->dev_err;
    if (cudaMemcpy(b.d_groups, b.groups.data(), sizeof(BatchGroup) * b.groups.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return SF_ERR_CUDA;
    std::vector<int> item_group(b.items_per_holo);
    for (int g = 0; g < (int)b.groups.size(); ++g)
      for (int i = 0; i < b.groups[g].items; ++i) item_group[b.groups[g].first_item + i] = g;
    b.d_item_group = reinterpret_cast<int*>(base + o_item_group);
    if (cudaMemcpy(b.d_item_group, item_group.data(), sizeof(int) * item_group.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return SF_ERR_CUDA;
    // One power-of-two length on every pass of every view, all prunable: the
    // specialised kernel (SF_BATCH_GENERAL=1 keeps the general one).
    const PassKind kx = p->in_complex ? PASS_X_CPLX : PASS_X_REAL;
    const int L1 = p->views[0].ax[0].L;
    bool one = !env_is("SF_BATCH_GENERAL", "1") && batch_kernel_one(kx, L1) != nullptr;
    for (const ViewState& vs : p->views)
      for (int ph = 0; ph < 2 && one; ++ph)
        one = vs.ax[ph].L == L1 && 2 * vs.ax[ph].n0 <= L1 && 2 * vs.ax[ph].n1 <= L1;
    b.kfunc = one ? batch_kernel_one(kx, L1) : batch_kernel(kx);
    b.ksmem = one ? batch_smem_bytes_one(L1) : batch_smem_bytes();
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    cudaFuncSetAttribute(b.kfunc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.ksmem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b.kfunc, kBatchThreads, b.ksmem) != cudaSuccess ||
        per_sm < 1)
      return SF_ERR_CUDA;
    b.grid = sms * per_sm;
    for (int k = 0; k < 2; ++k)
      if (cudaEventCreateWithFlags(&b.ev[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&b.join[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaStreamCreateWithFlags(&b.st[k], cudaStreamNonBlocking) != cudaSuccess)
        return SF_ERR_CUDA;
    if (cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.pre, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.post, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b.cap, cudaStreamNonBlocking) != cudaSuccess)
      return SF_ERR_CUDA;
    b.init = true;
  }
  if (!persistent || b.n_holos == n_holos) return SF_OK;
  free_batch_sized(b);
  const int ng = (int)b.groups.size();
  const size_t n_desc = (size_t)n_holos * ng, n_cnt = n_desc + 1;
  Arena ar;
  const size_t o_desc = ar.take(sizeof(PassDesc) * n_desc), o_done = ar.take(sizeof(int) * n_cnt);
  if (cudaMalloc(&b.d_sized, ar.off) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_OOM;
  }
  b.d_descs = reinterpret_cast<PassDesc*>(static_cast<char*>(b.d_sized) + o_desc);
  b.d_done = reinterpret_cast<int*>(static_cast<char*>(b.d_sized) + o_done);
  BatchArgs args;
  std::memset(&args, 0, sizeof(args));
  args.descs = b.d_descs;
  args.groups = b.d_groups;
  args.item_group = b.d_item_group;
  args.done = b.d_done;
  args.next = b.d_done + n_desc;
  args.error = b.d_error;
  for (auto& kv : p->tw) {
    const int slot = fft_length_slot(kv.first);
    if (slot >= 0) args.tw[slot] = kv.second;
  }
  args.n_holos = n_holos;
  args.n_groups = ng;
  args.n_views = nv;
  args.items_per_holo = b.items_per_holo;
  args.total_items = n_holos * b.items_per_holo;
  args.poison_group = (int)env_ll("SF_BATCH_POISON_GROUP", -1);
  args.spin_limit = env_ll("SF_BATCH_SPIN_LIMIT", 1ll << 22);
  for (int k = 0; k < 2; ++k) {
    if (cudaHostAlloc(&b.h_descs[k], sizeof(PassDesc) * n_desc, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      free_batch_sized(b);
      return SF_ERR_OOM;
    }
    std::memset(b.h_descs[k], 0, sizeof(PassDesc) * n_desc);
    cudaGraphNode_t cp, ms, kn;
    cudaError_t e = cudaGraphCreate(&b.graph[k], 0);
    if (e == cudaSuccess)
      e = cudaGraphAddMemcpyNode1D(&cp, b.graph[k], nullptr, 0, b.d_descs, b.h_descs[k], sizeof(PassDesc) * n_desc,
                                   cudaMemcpyHostToDevice);
    cudaMemsetParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.dst = b.d_done;
    mp.value = 0;
    mp.elementSize = sizeof(int);
    mp.width = n_cnt;
    mp.height = 1;
    mp.pitch = sizeof(int) * n_cnt;
    if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&ms, b.graph[k], nullptr, 0, &mp);
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    void* kargs[] = {&args};
    kp.func = const_cast<void*>(b.kfunc);
    kp.gridDim = dim3(b.grid);
    kp.blockDim = dim3(kBatchThreads);
    kp.sharedMemBytes = (unsigned)b.ksmem;
    kp.kernelParams = kargs;
    cudaGraphNode_t deps[2] = {cp, ms};
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&kn, b.graph[k], deps, 2, &kp);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b.exec[k], b.graph[k], 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_batch_sized(b);
      return SF_ERR_CUDA;
    }
  }
  b.n_holos = n_holos;
  return SF_OK;
}

// The persistent TMA pass: chosen for (L, kind) at plan time, and it needs
// 16-byte aligned rows, row strides and row lengths.
bool persistent_eligible(sf_plan p, int L, PassKind kind, const PassBatch& b) {
  const int slot = fft_length_slot(L);
  if (slot < 0 || p->impl[slot][kind] != 1 || !tma_length_supported(L)) return false;
  const size_t elem = kind == PASS_X_REAL ? 4 : 8;
  for (int k = 0; k < b.count; ++k) {
    const PassDesc& d = b.d[k];
    if (reinterpret_cast<uintptr_t>(d.src) % 16 || (d.src_ld * elem) % 16 || (d.n0 * elem) % 16) return false;
  }
  return true;
}

// One launch of the row pass over the descriptors of b (all FFT length L;
// view_of[k] is descriptor k's view): on reduced-precision plans the tcgen05
// pass where its length and the 2N padding allow, else the mma.sync pass
// (FP16 / BF16 plans); the persistent bulk-copy pass where the plan chose it
// and the rows allow it, else the one-tile-per-CTA pass.  max_rows: the most rows of any
// descriptor.
cudaError_t launch_row_pass(sf_plan plan, int axis, int L, PassBatch& b, const int* view_of, int max_rows,
                            cudaStream_t s) {
  const PassKind kind = axis == 1 ? PASS_Y : (plan->in_complex ? PASS_X_CPLX : PASS_X_REAL);
  cudaError_t e;
  void* const t5c = t5_consts_for(plan, L);
  bool t5 = t5c != nullptr;
  for (int k = 0; k < b.count && t5; ++k) t5 = 2 * b.d[k].n0 <= L && 2 * b.d[k].n1 <= L;
  if (t5) {
    for (int k = 0; k < b.count; ++k) b.d[k].H = plan->views[view_of[k]].hnat[axis];
    e = launch_pass_t5(L, plan->precision, kind, b, t5c, plan->dev_err, plan->sms, s);
  } else if (plan->tc_frags && tc_length_supported(L)) {
    for (int k = 0; k < b.count; ++k) b.d[k].H = plan->views[view_of[k]].hpos[axis];
    const int G = tc_rows_per_cta(L);
    e = launch_pass_tc(L, plan->precision, kind, b, (max_rows + G - 1) / G, plan->tc_frags, s);
  } else if (persistent_eligible(plan, L, kind, b)) {
    e = launch_pass_persistent(L, kind, b, plan->tw[L], plan->dev_err, plan->sms, s);
  } else {
    const int slot = fft_length_slot(L);
    const int impl = slot >= 0 ? plan->impl[slot][kind] : 0;
    const int variant = impl >= 2 ? impl - 1 : 0;  // rows per CTA: default, half, double
    const int G = pass_rows_per_cta(L, variant);
    e = launch_pass(L, kind, b, (max_rows + G - 1) / G, plan->tw[L], s, variant);
  }
  ++g_launches;
  return e;
}

// Every view's pass along one axis (0: x, 1: y), launched in groups of views
// with equal FFT length (at most max_per_launch views per launch).  Pass
// sources: x reads `src` (the hologram) into work[v]; y reads work[v] into the
// view outputs dout/dint/dph[v].  after(views, n) runs after each launch.
// Rows [row0, row1) of each pass only (row1 < 0: to the end): hologram rows
// on the x pass, view columns on the y pass.
template <typename After>
cudaError_t launch_axis(sf_plan plan, int axis, const void* src, float2* const* work, float2* const* dout,
                        float* const* dint, float* const* dph, int max_per_launch, cudaStream_t s, After&& after,
                        const std::vector<int>* subset = nullptr, int row0 = 0, int row1 = -1) {
  std::vector<int> order;
  if (subset) {
    order = *subset;
  } else {
    for (int i = 0; i < (int)plan->views.size(); ++i) order.push_back(i);
  }
  const int nv = (int)order.size();
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return plan->views[a].ax[axis].L < plan->views[b].ax[axis].L; });
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < nv && e == cudaSuccess;) {
    const int L = plan->views[order[i]].ax[axis].L;
    PassBatch b;
    std::memset(&b, 0, sizeof(b));
    int max_rows = 0;
    int batch_view[kMaxPassBatch];
    while (i < nv && b.count < std::min(max_per_launch, kMaxPassBatch) && plan->views[order[i]].ax[axis].L == L) {
      const int vi = order[i++];
      batch_view[b.count] = vi;
      ViewState& vs = plan->views[vi];
      const AxisCoef& c = vs.ax[axis];
      PassDesc& d = b.d[b.count++];
      d.cin = c.cin;
      d.cout = c.cout;
      d.H = c.H;
      d.n0 = c.n0;
      d.n1 = c.n1;
      if (axis == 0) {
        const int r0 = std::min(row0, vs.v.ny0), r1 = row1 < 0 ? vs.v.ny0 : std::min(row1, vs.v.ny0);
        const size_t elem = plan->in_complex ? sizeof(float2) : sizeof(float);
        d.src = static_cast<const char*>(src) + elem * (size_t)r0 * vs.v.nx0;
        d.dst = work[vi] + r0;
        d.rows = std::max(r1 - r0, 0);
        d.src_ld = vs.v.nx0;
        d.dst_ld = vs.v.ny0;
      } else {
        // y-pass row r is column r of the view
        const int r0 = std::min(row0, vs.v.nx1), r1 = row1 < 0 ? vs.v.nx1 : std::min(row1, vs.v.nx1);
        d.src = work[vi] + (size_t)r0 * vs.v.ny0;
        d.dst = dout[vi] ? dout[vi] + r0 : nullptr;
        d.inten = dint[vi] ? dint[vi] + r0 : nullptr;
        d.phase = dph[vi] ? dph[vi] + r0 : nullptr;
        d.rows = std::max(r1 - r0, 0);
        d.src_ld = vs.v.ny0;
        d.dst_ld = vs.v.nx1;
      }
      max_rows = std::max(max_rows, d.rows);
    }
    e = launch_row_pass(plan, axis, L, b, batch_view, max_rows, s);
    if (e == cudaSuccess) e = after(batch_view, b.count);
  }
  return e;
}

// FFT length per (view, axis) and row-pass kernel per (length, kind).
//   default: the smallest supported length (SF_FFT_LENGTHS=pow2 keeps powers
//            of two only); the persistent kernel at 4096, the one-tile-per-CTA
//            kernel with its default rows per CTA elsewhere (SF_PASS_IMPL=
//            grid|tma forces one; half|double: the one-tile-per-CTA kernel with
//            half or twice the rows per CTA where that variant exists);
//   SF_AUTOTUNE=1: per axis the cheaper of the two candidate lengths, per
//            (length, kind) the cheapest of the kernels and rows-per-CTA
//            variants, by measured time per row.
// Tensor-core plans keep the power of two where the tensor-core pass takes it.
struct PlanChoices {
  std::vector<int> L;  // [2 * view + axis]
  int impl[kNumFftLengths][3] = {};
};

PlanChoices plan_choices(sf_plan p, const sf_view* views, int n_views, int precision, cudaStream_t s) {
  PlanChoices c;
  c.L.resize(2 * n_views);
  const char* lens = std::getenv("SF_FFT_LENGTHS");
  const bool allow_mixed = !(lens && std::string(lens) == "pow2");
  // row-pass kernel without tuning: the persistent kernel at 4096 (512-thread
  // CTAs, one per SM: its prefetch overlaps loads and arithmetic, 14 % less
  // time per row measured), one tile per CTA elsewhere; SF_PASS_IMPL=grid|tma
  // forces one where the persistent kernel applies
  const char* impl_env = std::getenv("SF_PASS_IMPL");
  const bool force_grid = impl_env && std::string(impl_env) == "grid";
  const bool force_tma = impl_env && std::string(impl_env) == "tma";
  const int force_variant = impl_env && std::string(impl_env) == "half"     ? 1
                            : impl_env && std::string(impl_env) == "double" ? 2
                                                                             : 0;
  auto impl_default = [&](int L) {
    if (force_variant) return pass_rows_per_cta(L, force_variant) > 0 ? 1 + force_variant : 0;
    if (!tma_length_supported(L)) return 0;
    return force_tma ? 1 : force_grid ? 0 : (L == 4096 ? 1 : 0);
  };
  const bool tune = autotune_mode() == 1;
  auto kind_of = [&](int axis) {
    return axis == 1 ? PASS_Y : (p->in_complex ? PASS_X_CPLX : PASS_X_REAL);
  };
  // best measured cost of (L, kind, prunable) over the kernels, remembering the kernel
  auto best = [&](int L, PassKind kind, bool prune, int* impl) {
    double b = -1;
    for (int k = 0; k < 4; ++k) {
      const double ns = row_cost_ns(p->device, L, kind, k, prune, p->sms, s);
      if (ns > 0 && (b < 0 || ns < b)) {
        b = ns;
        if (impl) *impl = k;
      }
    }
    return b;
  };
  // does axis a of view i run the pruned network at length L
  auto prunable = [&](int i, int a, int L) {
    const int n0 = a == 0 ? views[i].nx0 : views[i].ny0, n1 = a == 0 ? views[i].nx1 : views[i].ny1;
    return (L & (L - 1)) == 0 && 2 * n0 <= L && 2 * n1 <= L;
  };
  for (int i = 0; i < n_views; ++i)
    for (int a = 0; a < 2; ++a) {
      const int need = a == 0 ? views[i].nx0 + views[i].nx1 - 1 : views[i].ny0 + views[i].ny1 - 1;
      const int P = next_fft_length(need, false), Q = allow_mixed ? next_fft_length(need, true) : P;
      int L = Q;
      if (precision != SF_PREC_FP32 && (tc_length_supported(P) || t5_length_supported(P))) {
        L = P;
      } else if (tune && Q != P) {
        const double cp = best(P, kind_of(a), prunable(i, a, P), nullptr);
        const double cq = best(Q, kind_of(a), prunable(i, a, Q), nullptr);
        if (cp > 0 && cq > 0 && cp < cq) L = P;
      }
      c.L[2 * i + a] = L;
    }
  for (int slot = 0; slot < kNumFftLengths; ++slot)
    for (int k = 0; k < 3; ++k) {
      const int L = kFftLengths[slot];
      c.impl[slot][k] = impl_default(L);
      if (!tune) continue;
      bool used = false, all_prunable = true;
      for (int i = 0; i < n_views; ++i)
        for (int a = 0; a < 2; ++a)
          if (c.L[2 * i + a] == L && (kind_of(a) == k || (a == 0 && k == PASS_X_CPLX))) {  // adjoint x: complex
            used = true;
            all_prunable = all_prunable && prunable(i, a, L);
          }
      if (used) best(L, (PassKind)k, all_prunable, &c.impl[slot][k]);
    }
  return c;
}

// The persistent kernel: one graph launch for the whole batch.
int run_batch_persistent(sf_plan plan, const void* const* holos, int n_holos, void* const* view_out,
                         float* const* intensity, float* const* phase, cudaStream_t s) {
  const int nv = (int)plan->views.size();
  int rc = batch_prepare(plan, n_holos, true);
  if (rc) return rc;
  BatchState& b = plan->batch;
  const int k = b.flip;
  if (cudaEventSynchronize(b.ev[k]) != cudaSuccess) {  // the call two back has finished reading this table
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  const int ng = (int)b.groups.size();
  for (int h = 0; h < n_holos; ++h)
    for (int g = 0; g < ng; ++g) {
      const int v = g % nv, ph = g / nv;
      ViewState& vs = plan->views[v];
      float2* slot = (h & 1) ? b.slot1[v] : vs.work;
      const AxisCoef& c = vs.ax[ph];
      PassDesc& d = b.h_descs[k][(size_t)h * ng + g];
      std::memset(&d, 0, sizeof(d));
      d.cin = c.cin; d.cout = c.cout; d.H = c.H; d.n0 = c.n0; d.n1 = c.n1;
      if (ph == 0) {
        d.src = holos[h]; d.dst = slot; d.rows = vs.v.ny0; d.src_ld = vs.v.nx0; d.dst_ld = vs.v.ny0;
      } else {
        const size_t i = (size_t)h * nv + v;
        d.src = slot;
        d.dst = view_out ? static_cast<float2*>(view_out[i]) : nullptr;
        d.inten = intensity ? intensity[i] : nullptr;
        d.phase = phase ? phase[i] : nullptr;
        d.rows = vs.v.nx1; d.src_ld = vs.v.ny0; d.dst_ld = vs.v.nx1;
      }
    }
  cudaError_t e = cudaGraphLaunch(b.exec[k], s);
  if (e == cudaSuccess) e = cudaEventRecord(b.ev[k], s);
  ++g_launches;
  b.flip ^= 1;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}


// The per-length row-pass kernels, holograms alternating between two streams
// (and two intermediate slots), so one hologram's passes overlap the next's.
// Enqueue the per-length launches of a batch on the plan's two streams,
// forked from and joined back into s.
// Holograms per row-pass launch of the two-stream batch.  When one
// hologram's x pass is too small to fill the GPU (fewer CTAs than two waves
// of two per SM), K holograms share each launch (K x n_views <= kMaxPassBatch
// descriptors), each with its own intermediate slot; the two streams then
// alternate chunks of K holograms, so 2 K slots per view are needed, the
// extra ones within 512 MiB.  Sets b.sk and b.sslot.
int ensure_stream_slots(sf_plan p) {
  BatchState& b = p->batch;
  if (b.sk) return SF_OK;
  const int nv = (int)p->views.size();
  long long ctas = 0;
  size_t ws = 0;
  for (const ViewState& vs : p->views) {
    ctas += (vs.v.ny0 + pass_rows_per_cta(vs.ax[0].L) - 1) / std::max(1, pass_rows_per_cta(vs.ax[0].L));
    ws += sizeof(float2) * work_elems(vs.v);
  }
  const long long target = 2LL * 2 * std::max(1, p->sms);
  int K = (int)std::min<long long>(kMaxPassBatch / nv, (target + ctas - 1) / std::max(1LL, ctas));
  K = std::max(K, 1);
  while (K > 1 && (size_t)(2 * K - 2) * ws > ((size_t)512 << 20)) --K;
  std::vector<float2*> slots((size_t)2 * K * nv, nullptr);
  for (int v = 0; v < nv; ++v) {
    slots[(size_t)0 * nv + v] = p->views[v].work;
    slots[(size_t)K * nv + v] = b.slot1[v];
  }
  if (K > 1) {
    Arena ar;
    std::vector<size_t> off(slots.size(), SIZE_MAX);
    for (int grp = 0; grp < 2; ++grp)
      for (int j = 1; j < K; ++j)
        for (int v = 0; v < nv; ++v)
          off[(size_t)(grp * K + j) * nv + v] = ar.take(sizeof(float2) * work_elems(p->views[v].v));
    if (cudaMalloc(&b.d_sslot, ar.off) != cudaSuccess) {
      cudaGetLastError();
      b.d_sslot = nullptr;
      K = 1;  // fall back to one hologram per launch
    } else {
      for (size_t i = 0; i < slots.size(); ++i)
        if (off[i] != SIZE_MAX) slots[i] = reinterpret_cast<float2*>(static_cast<char*>(b.d_sslot) + off[i]);
    }
  }
  if (K == 1) {
    slots.resize((size_t)2 * nv);
    for (int v = 0; v < nv; ++v) {
      slots[v] = p->views[v].work;
      slots[(size_t)nv + v] = b.slot1[v];
    }
  }
  b.sslot = slots;
  b.sk = K;
  return SF_OK;
}

// An FP16 or BF16 plan (the x3 precisions, two groups per SM, measure
// faster with one launch per pass) of two to kMaxPassBatch / 2 views (one
// view measures faster with one launch per pass) that all run both axes on
// the tcgen05 pass at one FFT length (2048, 1024 or 512, with the 2N padding).
bool fused_t5_eligible(sf_plan p) {
  const int nv = (int)p->views.size();
  if (p->precision != SF_PREC_FP16TC && p->precision != SF_PREC_BF16TC) return false;
  if (!p->t5_sched || nv < 2 || nv > kMaxPassBatch / 2) return false;
  const int L = p->views[0].ax[0].L;  // one FFT length on every axis of every view
  if (!t5_consts_for(p, L)) return false;
  for (const ViewState& vs : p->views)
    for (int a = 0; a < 2; ++a) {
      const AxisCoef& c = vs.ax[a];
      if (c.L != L || 2 * c.n0 > c.L || 2 * c.n1 > c.L || !vs.hnat[a]) return false;
    }
  return true;
}

// Both passes of every view of a fused_t5_eligible plan as one persistent
// tcgen05 launch: x passes read the hologram src into work[v], y passes write
// dout / dint / dph[v] (null where not wanted); sched: this launch's schedule
// buffer (launches that may overlap take different ones).
cudaError_t launch_fused_views(sf_plan plan, const void* src, float2* const* work, float2* const* dout,
                               float* const* dint, float* const* dph, int* sched, cudaStream_t s) {
  const int nv = (int)plan->views.size();
  const int L = plan->views[0].ax[0].L;
  PassBatch b;
  std::memset(&b, 0, sizeof(b));
  for (int axis = 0; axis < 2; ++axis)
    for (int vi = 0; vi < nv; ++vi) {
      const ViewState& vs = plan->views[vi];
      const AxisCoef& c = vs.ax[axis];
      PassDesc& d = b.d[b.count++];
      d.cin = c.cin;
      d.cout = c.cout;
      d.H = vs.hnat[axis];
      d.n0 = c.n0;
      d.n1 = c.n1;
      if (axis == 0) {
        d.src = src;
        d.dst = work[vi];
        d.rows = vs.v.ny0;
        d.src_ld = vs.v.nx0;
        d.dst_ld = vs.v.ny0;
      } else {
        d.src = work[vi];
        d.dst = dout[vi];
        d.inten = dint[vi];
        d.phase = dph[vi];
        d.rows = vs.v.nx1;
        d.src_ld = vs.v.ny0;
        d.dst_ld = vs.v.nx1;
      }
    }
  const PassKind kx = plan->in_complex ? PASS_X_CPLX : PASS_X_REAL;
  const cudaError_t e =
      launch_views_t5(L, plan->precision, kx, b, nv, t5_consts_for(plan, L), plan->dev_err, sched, plan->sms, s);
  ++g_launches;
  return e;
}

cudaError_t enqueue_batch_streams(sf_plan plan, const void* const* holos, int n_holos, void* const* view_out,
                                  float* const* intensity, float* const* phase, cudaStream_t s) {
  BatchState& b = plan->batch;
  const int nv = (int)plan->views.size();
  cudaError_t e = cudaEventRecord(b.fork, s);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b.st[k], b.fork, 0);
  if (b.sk > 1) {
    // chunks of K holograms, alternating streams; every (hologram, view) pass
    // of a chunk and axis in launches of up to kMaxPassBatch descriptors of
    // one FFT length
    const int K = b.sk;
    for (int c = 0; c * K < n_holos && e == cudaSuccess; ++c) {
      const int h0 = c * K, h1 = std::min(n_holos, h0 + K), grp = c & 1;
      for (int axis = 0; axis < 2 && e == cudaSuccess; ++axis) {
        std::vector<int> order(nv);
        for (int v = 0; v < nv; ++v) order[v] = v;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return plan->views[x].ax[axis].L < plan->views[y].ax[axis].L; });
        std::vector<std::pair<int, int>> items;  // (hologram, view), grouped by FFT length
        for (int v : order)
          for (int h = h0; h < h1; ++h) items.emplace_back(h, v);
        for (size_t i = 0; i < items.size() && e == cudaSuccess;) {
          const int L = plan->views[items[i].second].ax[axis].L;
          PassBatch pb;
          std::memset(&pb, 0, sizeof(pb));
          int view_of[kMaxPassBatch];
          int max_rows = 0;
          while (i < items.size() && pb.count < kMaxPassBatch && plan->views[items[i].second].ax[axis].L == L) {
            const int h = items[i].first, v = items[i].second;
            const ViewState& vs = plan->views[v];
            const AxisCoef& co = vs.ax[axis];
            float2* slot = b.sslot[(size_t)(grp * K + (h - h0)) * nv + v];
            PassDesc& d = pb.d[pb.count];
            view_of[pb.count++] = v;
            d.cin = co.cin;
            d.cout = co.cout;
            d.H = co.H;
            d.n0 = co.n0;
            d.n1 = co.n1;
            if (axis == 0) {
              d.src = holos[h];
              d.dst = slot;
              d.rows = vs.v.ny0;
              d.src_ld = vs.v.nx0;
              d.dst_ld = vs.v.ny0;
            } else {
              const size_t o = (size_t)h * nv + v;
              d.src = slot;
              d.dst = view_out ? static_cast<float2*>(view_out[o]) : nullptr;
              d.inten = intensity ? intensity[o] : nullptr;
              d.phase = phase ? phase[o] : nullptr;
              d.rows = vs.v.nx1;
              d.src_ld = vs.v.ny0;
              d.dst_ld = vs.v.nx1;
            }
            max_rows = std::max(max_rows, d.rows);
            ++i;
          }
          e = launch_row_pass(plan, axis, L, pb, view_of, max_rows, b.st[grp]);
        }
      }
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventRecord(b.join[k], b.st[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b.join[k], 0);
    }
    return e;
  }
  std::vector<float2*> work(nv), dout(nv);
  std::vector<float*> dint(nv), dph(nv);
  auto none = [](const int*, int) { return cudaSuccess; };
  const bool fused = fused_t5_eligible(plan) && !env_is("SF_T5_FUSED", "0");
  for (int h = 0; h < n_holos && e == cudaSuccess; ++h) {
    for (int v = 0; v < nv; ++v) {
      const size_t i = (size_t)h * nv + v;
      work[v] = (h & 1) ? b.slot1[v] : plan->views[v].work;
      dout[v] = view_out ? static_cast<float2*>(view_out[i]) : nullptr;
      dint[v] = intensity ? intensity[i] : nullptr;
      dph[v] = phase ? phase[i] : nullptr;
    }
    if (fused) {  // one launch per hologram; the two streams' launches keep separate schedule buffers
      e = launch_fused_views(plan, holos[h], work.data(), dout.data(), dint.data(), dph.data(),
                             plan->t5_sched + (1 + (h & 1)) * kSchedInts, b.st[h & 1]);
      continue;
    }
    for (int axis = 0; axis < 2 && e == cudaSuccess; ++axis)
      e = launch_axis(plan, axis, holos[h], work.data(), dout.data(), dint.data(), dph.data(), kMaxPassBatch,
                      b.st[h & 1], none);
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b.join[k], b.st[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b.join[k], 0);
  }
  return e;
}

// The per-length row-pass kernels, holograms alternating between two streams
// (and two intermediate slots), so one hologram's passes overlap the next's.
// The launches are captured once as a CUDA graph and the graph is replayed
// while calls pass the same hologram count and buffers (a frame loop over
// fixed buffers pays one graph launch per call); other calls capture anew.
int run_batch_streams(sf_plan plan, const void* const* holos, int n_holos, void* const* view_out,
                      float* const* intensity, float* const* phase, cudaStream_t s) {
  int rc = batch_prepare(plan, n_holos, false);
  if (rc) return rc;
  if ((rc = ensure_stream_slots(plan))) return rc;
  BatchState& b = plan->batch;
  const size_t n = (size_t)n_holos * plan->views.size();
  std::vector<const void*> key;
  key.reserve(1 + n_holos + 3 * n);
  key.push_back(reinterpret_cast<const void*>((uintptr_t)n_holos));
  for (int h = 0; h < n_holos; ++h) key.push_back(holos[h]);
  for (size_t i = 0; i < n; ++i) {
    key.push_back(view_out ? view_out[i] : nullptr);
    key.push_back(intensity ? intensity[i] : nullptr);
    key.push_back(phase ? phase[i] : nullptr);
  }
  cudaError_t e = cudaSuccess;
  const bool replay = b.sgraph && key == b.skey;
  if (!replay) {
    if (b.sgraph) cudaGraphExecDestroy(b.sgraph);
    b.sgraph = nullptr;
    b.skey.clear();
    const uint64_t before = g_launches.load();
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t ee = enqueue_batch_streams(plan, holos, n_holos, view_out, intensity, phase, b.cap);
      e = cudaStreamEndCapture(b.cap, &graph);
      if (ee != cudaSuccess) e = ee;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      return SF_ERR_CUDA;
    }
    b.sgraph = exec;
    b.skey = key;
    b.sgraph_kernels = g_launches.load() - before;  // counted while capturing
  }
  // ordered after the caller's earlier work, and the caller's stream after the graph
  e = cudaEventRecord(b.pre, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b.cap, b.pre, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(b.sgraph, b.cap);
  if (e == cudaSuccess) e = cudaEventRecord(b.post, b.cap);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b.post, 0);
  if (replay) g_launches += b.sgraph_kernels;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

int run_batch(sf_plan plan, int impl, const void* const* holos, int n_holos, void* const* view_out,
              float* const* intensity, float* const* phase, cudaStream_t s) {
  return impl == BATCH_PERSISTENT ? run_batch_persistent(plan, holos, n_holos, view_out, intensity, phase, s)
                                  : run_batch_streams(plan, holos, n_holos, view_out, intensity, phase, s);
}

// Batch implementation for this plan and hologram count; -1: measure (autotuner).
//   SF_BATCH_IMPL=persistent|streams forces one; SF_AUTOTUNE=1 measures both
//   once per hologram count; otherwise the per-length kernels on two streams,
//   which measured faster than the persistent kernel on every workload tried
//   (paper-scale views, ragged 2048^2 views, 256^2 single views).
int batch_choice(sf_plan p, int n_holos) {
  const char* env = std::getenv("SF_BATCH_IMPL");
  if (env && std::string(env) == "persistent") return BATCH_PERSISTENT;
  if (env && std::string(env) == "streams") return BATCH_STREAMS;
  if (!batch_persistent_supported(p)) return BATCH_STREAMS;
  if (autotune_mode() == 1) {
    auto it = p->batch.choice.find(n_holos);
    return it == p->batch.choice.end() ? -1 : it->second;
  }
  return BATCH_STREAMS;
}

}  // namespace

extern "C" {

int32_t shifted_fresnel_fft_length(int32_t need, int32_t allow_mixed) {
  if (need < 1) return SF_ERR_INVALID_ARG;
  if (need > SF_MAX_CONV_LENGTH) return SF_ERR_UNSUPPORTED_SIZE;
  return next_fft_length(need, allow_mixed != 0);
}

const char* shifted_fresnel_strerror(int status) {
  switch (status) {
    case SF_OK: return "success";
    case SF_ERR_INVALID_ARG: return "invalid argument";
    case SF_ERR_UNSUPPORTED_SIZE: return "unsupported size: n0 + n1 - 1 exceeds the longest supported convolution";
    case SF_ERR_CUDA: return "CUDA runtime error";
    case SF_ERR_OOM: return "out of memory";
    case SF_ERR_TIMEOUT: return "device-side wait timed out";
    case SF_ERR_DEVICE_MISMATCH: return "buffer belongs to another device than the plan";
    default: return "unknown status";
  }
}

uint64_t shifted_fresnel_kernel_launches(void) { return g_launches.load(); }

namespace {

// Input / output chirps and kernel spectra of every view and axis (forward
// and adjoint) from the coefficients in p->views, on stream s: the
// coefficient table goes to the device, then one chirp launch and one
// spectrum launch per FFT length, then (tensor-core plans) the spectra in
// position order.  The device pointers in the coefficients are the plan's.
cudaError_t build_view_vectors(sf_plan p, cudaStream_t s) {
  std::vector<AxisCoef> axes;
  axes.reserve(4 * p->views.size());
  int max_n = 1;
  for (const ViewState& vs : p->views)
    for (int a = 0; a < 2; ++a) {
      axes.push_back(vs.ax[a]);
      axes.push_back(vs.adj[a]);
      max_n = std::max(max_n, std::max(vs.ax[a].n0, vs.ax[a].n1));
    }
  // sorted by FFT length so each length's spectra are built by one launch
  std::stable_sort(axes.begin(), axes.end(), [](const AxisCoef& x, const AxisCoef& y) { return x.L < y.L; });
  // pageable source: the call returns once the table is staged
  cudaError_t e =
      cudaMemcpyAsync(p->axes_dev, axes.data(), sizeof(AxisCoef) * axes.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    e = launch_chirps(p->axes_dev, (int)axes.size(), max_n, s);
    ++g_launches;
  }
  for (size_t i = 0; i < axes.size() && e == cudaSuccess;) {
    size_t j = i;
    while (j < axes.size() && axes[j].L == axes[i].L) ++j;
    e = launch_hspec(axes[i].L, p->axes_dev + i, (int)(j - i), p->tw[axes[i].L], s);
    ++g_launches;
    i = j;
  }
  for (ViewState& vs : p->views)
    for (int a = 0; a < 2 && e == cudaSuccess; ++a)
      {
        if (vs.hpos[a] && e == cudaSuccess) {
          e = launch_hpos(vs.ax[a].L, vs.ax[a].H, vs.hpos[a], s);
          ++g_launches;
        }
        if (vs.hnat[a] && e == cudaSuccess) {
          e = launch_hnat(vs.ax[a].L, vs.ax[a].H, vs.hnat[a], s);
          ++g_launches;
        }
      }
  return e;
}

}  // namespace

int shifted_fresnel_plan(sf_plan* out, const sf_view* views, int n_views, int precision, int device,
                         void* stream) {
  if (!out) return SF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!views || n_views < 1 || n_views > kMaxViews) return SF_ERR_INVALID_ARG;
  if (precision != SF_PREC_FP32 && !t5_precision(precision)) return SF_ERR_INVALID_ARG;
  for (int i = 0; i < n_views; ++i) {
    int rc = validate_view(views[i]);
    if (rc) return rc;
    if (views[i].nx0 != views[0].nx0 || views[i].ny0 != views[0].ny0 ||
        (views[i].flags & SF_IN_COMPLEX) != (views[0].flags & SF_IN_COMPLEX))
      return SF_ERR_INVALID_ARG;
  }
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess) { cudaGetLastError(); return SF_ERR_CUDA; }
  if (device < 0 || device >= n_dev) return SF_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return SF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;

  sf_plan p = new (std::nothrow) sf_plan_s();
  if (!p) return SF_ERR_OOM;
  p->device = device;
  p->nx0 = views[0].nx0;
  p->ny0 = views[0].ny0;
  p->in_complex = (views[0].flags & SF_IN_COMPLEX) != 0;
  p->precision = precision;
  p->views.resize(n_views);

  p->sms = 0;
  cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, device);
  const PlanChoices ch = plan_choices(p, views, n_views, precision, s);
  for (int i = 0; i < kNumFftLengths; ++i)
    for (int k = 0; k < 3; ++k) p->impl[i][k] = ch.impl[i][k];

  // coefficients and arena layout
  Arena ar;
  std::map<int, size_t> tw_off;
  std::vector<size_t> off_cin(4 * n_views), off_cout(4 * n_views), off_H(4 * n_views), off_work(n_views);
  std::vector<size_t> off_hpos(2 * n_views, SIZE_MAX), off_hnat(2 * n_views, SIZE_MAX);
  const bool mma_sync_tables = precision == SF_PREC_FP16TC || precision == SF_PREC_BF16TC;
  bool any_t5 = false, t5_len[3] = {false, false, false};  // FFT lengths 512, 1024, 2048
  for (int i = 0; i < n_views; ++i) {
    ViewState& vs = p->views[i];
    vs.v = views[i];
    for (int a = 0; a < 2; ++a) {
      axis_coefficients(vs.v, a, vs.ax[a], ch.L[2 * i + a]);
      const AxisCoef& c = vs.ax[a];
      if (!tw_off.count(c.L)) tw_off[c.L] = ar.take(sizeof(float4) * twiddle_entries(c.L));
      off_cin[2 * i + a] = ar.take(sizeof(float2) * c.n0);
      off_cout[2 * i + a] = ar.take(sizeof(float2) * c.n1);
      off_H[2 * i + a] = ar.take(sizeof(float2) * c.L);
      adjoint_axis_coefficients(vs.v, a, vs.adj[a], ch.L[2 * i + a]);
      const AxisCoef& ca = vs.adj[a];
      off_cin[2 * n_views + 2 * i + a] = ar.take(sizeof(float2) * ca.n0);
      off_cout[2 * n_views + 2 * i + a] = ar.take(sizeof(float2) * ca.n1);
      off_H[2 * n_views + 2 * i + a] = ar.take(sizeof(float2) * ca.L);
    }
    off_work[i] = ar.take(sizeof(float2) * work_elems(vs.v));
    for (int a = 0; a < 2; ++a) {
      off_hpos[2 * i + a] = (mma_sync_tables && tc_length_supported(vs.ax[a].L))
                                ? ar.take(sizeof(float2) * vs.ax[a].L) : SIZE_MAX;
      if (precision != SF_PREC_FP32 && t5_length_supported(vs.ax[a].L)) {
        off_hnat[2 * i + a] = ar.take(sizeof(float2) * vs.ax[a].L);
        any_t5 = true;
        t5_len[vs.ax[a].L == 2048 ? 2 : vs.ax[a].L == 1024 ? 1 : 0] = true;
      }
    }
  }
  const size_t off_frags = mma_sync_tables ? ar.take(sizeof(uint32_t) * tc_table_words()) : SIZE_MAX;
  size_t off_t5[3];
  for (int k = 0; k < 3; ++k) off_t5[k] = t5_len[k] ? ar.take(t5_const_bytes(512 << k, precision)) : SIZE_MAX;
  const size_t off_sched = any_t5 ? ar.take(sizeof(int) * 3 * kSchedInts) : SIZE_MAX;
  const size_t off_err = ar.take(sizeof(int));
  const size_t off_axes = ar.take(sizeof(AxisCoef) * 4 * n_views);
  if (cudaMalloc(&p->arena, ar.off) != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    return SF_ERR_OOM;
  }
  char* base = static_cast<char*>(p->arena);
  for (auto& kv : tw_off) p->tw[kv.first] = reinterpret_cast<float4*>(base + kv.second);

  for (int i = 0; i < n_views; ++i) {
    ViewState& vs = p->views[i];
    vs.work = reinterpret_cast<float2*>(base + off_work[i]);
    for (int a = 0; a < 2; ++a) {
      if (off_hpos[2 * i + a] != SIZE_MAX) vs.hpos[a] = reinterpret_cast<float2*>(base + off_hpos[2 * i + a]);
      if (off_hnat[2 * i + a] != SIZE_MAX) vs.hnat[a] = reinterpret_cast<float2*>(base + off_hnat[2 * i + a]);
    }
    for (int a = 0; a < 2; ++a) {
      AxisCoef& c = vs.ax[a];
      c.cin = reinterpret_cast<float2*>(base + off_cin[2 * i + a]);
      c.cout = reinterpret_cast<float2*>(base + off_cout[2 * i + a]);
      c.H = reinterpret_cast<float2*>(base + off_H[2 * i + a]);
      AxisCoef& ca = vs.adj[a];
      ca.cin = reinterpret_cast<float2*>(base + off_cin[2 * n_views + 2 * i + a]);
      ca.cout = reinterpret_cast<float2*>(base + off_cout[2 * n_views + 2 * i + a]);
      ca.H = reinterpret_cast<float2*>(base + off_H[2 * n_views + 2 * i + a]);
    }
  }
  p->axes_dev = reinterpret_cast<AxisCoef*>(base + off_axes);

  cudaError_t e = cudaSuccess;
  std::vector<std::vector<float4>> tw_host;  // kept alive until the stream is synchronised below
  for (auto& kv : p->tw) {
    tw_host.emplace_back(twiddle_entries(kv.first));
    build_twiddles(kv.first, tw_host.back().data());
    if (e == cudaSuccess && !tw_host.back().empty())
      e = cudaMemcpyAsync(kv.second, tw_host.back().data(), sizeof(float4) * tw_host.back().size(),
                          cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = build_view_vectors(p, s);
  p->dev_err = reinterpret_cast<int*>(base + off_err);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->dev_err, 0, sizeof(int), s);
  if (off_frags != SIZE_MAX && e == cudaSuccess) {
    p->tc_frags = reinterpret_cast<uint32_t*>(base + off_frags);
    e = launch_tc_tables(p->tc_frags, precision, s);
    g_launches += 3;  // fragments and the twiddle tables of both lengths
  }
  if (off_sched != SIZE_MAX) p->t5_sched = reinterpret_cast<int*>(base + off_sched);
  std::vector<unsigned char> t5_host[3];  // kept alive until the stream is synchronised below
  for (int k = 0; k < 3; ++k)
    if (off_t5[k] != SIZE_MAX && e == cudaSuccess) {
      p->t5_consts[k] = base + off_t5[k];
      t5_host[k].resize(t5_const_bytes(512 << k, precision));
      t5_build_consts(512 << k, precision, t5_host[k].data());
      e = cudaMemcpyAsync(p->t5_consts[k], t5_host[k].data(), t5_host[k].size(), cudaMemcpyHostToDevice, s);
    }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    return e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA;
  }
  *out = p;
  return SF_OK;
}

int shifted_fresnel_plan_update(sf_plan plan, const sf_view* views, int n_views, void* stream) {
  if (!plan || !views || n_views != (int)plan->views.size()) return SF_ERR_INVALID_ARG;
  for (int i = 0; i < n_views; ++i) {
    int rc = validate_view(views[i]);
    if (rc) return rc;
    const sf_view& o = plan->views[i].v;
    if (views[i].nx0 != o.nx0 || views[i].ny0 != o.ny0 || views[i].nx1 != o.nx1 || views[i].ny1 != o.ny1 ||
        (views[i].flags & SF_IN_COMPLEX) != (o.flags & SF_IN_COMPLEX))
      return SF_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  if (!guard.ok) return SF_ERR_CUDA;
  // new coefficients on the same FFT lengths and device vectors
  for (int i = 0; i < n_views; ++i) {
    ViewState& vs = plan->views[i];
    vs.v = views[i];
    for (int a = 0; a < 2; ++a) {
      const AxisCoef f = vs.ax[a], g = vs.adj[a];
      axis_coefficients(vs.v, a, vs.ax[a], f.L);
      adjoint_axis_coefficients(vs.v, a, vs.adj[a], g.L);
      vs.ax[a].cin = f.cin;
      vs.ax[a].cout = f.cout;
      vs.ax[a].H = f.H;
      vs.adj[a].cin = g.cin;
      vs.adj[a].cout = g.cout;
      vs.adj[a].H = g.H;
    }
  }
  if (build_view_vectors(plan, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

int shifted_fresnel_plan_query(sf_plan plan, int view, int32_t* lx, int32_t* ly, size_t* workspace_bytes) {
  if (!plan || view < 0 || view >= (int)plan->views.size()) return SF_ERR_INVALID_ARG;
  const ViewState& vs = plan->views[view];
  if (lx) *lx = vs.ax[0].L;
  if (ly) *ly = vs.ax[1].L;
  if (workspace_bytes) *workspace_bytes = sizeof(float2) * work_elems(vs.v);
  return SF_OK;
}

namespace sf {
namespace {
// After a failed enqueue: make `s` wait for whatever the call already put on
// plan-owned stream `other`, so later work on `s` stays ordered after it
// (best effort; errors here are cleared).
void join_after_error(cudaStream_t s, cudaStream_t other, cudaEvent_t ev) {
  cudaGetLastError();
  if (other && ev && cudaEventRecord(ev, other) == cudaSuccess) cudaStreamWaitEvent(s, ev, 0);
  cudaGetLastError();
}
}  // namespace
}  // namespace sf

namespace {

// Buffers of one execute call once host memory is resolved to staging.
struct ExecBuffers {
  struct Copy { void* dst; const void* src; size_t bytes; int view; size_t elem; };
  const void* src = nullptr;               // hologram on the device
  std::vector<float2*> work, dout;         // per view: intermediate, complex output (or null)
  std::vector<float*> dint, dph;           // per view: intensity, phase (or null)
  std::vector<Copy> d2h;                   // staged host outputs, copied back per view
};

// Device outputs, two or more views: the views are split into two halves of
// about equal work, each run (x pass, then y pass) on its own stream, so one
// half's y pass overlaps the other's x pass.
cudaError_t execute_split_halves(sf_plan plan, const ExecBuffers& io, cudaStream_t s) {
  const int nv = (int)plan->views.size();
  std::vector<int> order(nv), half[2];
  double load[2] = {0, 0};
  for (int i = 0; i < nv; ++i) order[i] = i;
  auto cost = [&](int v) {
    const ViewState& vs = plan->views[v];
    return (double)vs.v.ny0 * vs.ax[0].L + (double)vs.v.nx1 * vs.ax[1].L;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  for (int v : order) {
    const int k = load[1] < load[0] ? 1 : 0;
    half[k].push_back(v);
    load[k] += cost(v);
  }
  for (int k = 0; k < 2; ++k) std::sort(half[k].begin(), half[k].end());
  auto none = [](const int*, int) { return cudaSuccess; };
  cudaError_t e = cudaEventRecord(plan->split_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->split_stream, plan->split_fork, 0);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    cudaStream_t cs = k == 0 ? s : plan->split_stream;
    for (int axis = 0; axis < 2 && e == cudaSuccess; ++axis)
      e = launch_axis(plan, axis, io.src, io.work.data(), io.dout.data(), io.dint.data(), io.dph.data(),
                      kMaxPassBatch, cs, none, &half[k]);
  }
  if (e == cudaSuccess) e = cudaEventRecord(plan->split_join, plan->split_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->split_join, 0);
  if (e != cudaSuccess) join_after_error(s, plan->split_stream, plan->split_join);
  return e;
}

// Host outputs: view by view, each view's copies to the host starting on the
// copy stream as soon as its y pass is done, so the copies (the bound of this
// path) start after the first view instead of after every view's x pass.
// Pipelined (default): the x passes run in view order on the low-priority
// stream, the first one split at row split_row of the hologram when that is
// nonzero (its first half starts while the second half is still being
// copied); each y pass waits for its view's x pass on the high-priority
// stream, the first and the last view's in two column halves.  Otherwise both
// passes of every view run in turn on `s`.  `s` ends after the last copy.
cudaError_t execute_host_outputs(sf_plan plan, const ExecBuffers& io, bool pipeline, int split_row,
                                 cudaStream_t s) {
  const int nv = (int)plan->views.size();
  auto none = [](const int*, int) { return cudaSuccess; };
  cudaStream_t ys = pipeline ? plan->pipe_y : s;
  auto copies = [&](const int* views, int) -> cudaError_t {
    const int vi = views[0];
    cudaError_t r = cudaEventRecord(plan->view_done[vi], ys);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(plan->copy_stream, plan->view_done[vi], 0);
    for (const ExecBuffers::Copy& c : io.d2h)
      if (r == cudaSuccess && c.view == vi)
        r = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, plan->copy_stream);
    return r;
  };
  // Columns [c0, c1) of view vi's host outputs, once the y pass so far is
  // done (one 2-D copy per output: ny1 rows of (c1 - c0) elements).
  auto column_copies = [&](int vi, int c0, int c1, cudaEvent_t ev) -> cudaError_t {
    const size_t ld = (size_t)plan->views[vi].v.nx1;
    cudaError_t r = cudaEventRecord(ev, ys);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(plan->copy_stream, ev, 0);
    for (const ExecBuffers::Copy& c : io.d2h)
      if (r == cudaSuccess && c.view == vi)
        r = cudaMemcpy2DAsync(static_cast<char*>(c.dst) + c.elem * c0, c.elem * ld,
                              static_cast<const char*>(c.src) + c.elem * c0, c.elem * ld, c.elem * (c1 - c0),
                              (size_t)plan->views[vi].v.ny1, cudaMemcpyDeviceToHost, plan->copy_stream);
    return r;
  };
  auto x_pass = [&](int vi, cudaStream_t st, int r0, int r1) {
    const std::vector<int> one{vi};
    return launch_axis(plan, 0, io.src, io.work.data(), io.dout.data(), io.dint.data(), io.dph.data(), 1, st, none,
                       &one, r0, r1);
  };
  auto y_pass = [&](int vi, int r0, int r1, bool with_copies) {
    const std::vector<int> one{vi};
    return with_copies ? launch_axis(plan, 1, io.src, io.work.data(), io.dout.data(), io.dint.data(),
                                     io.dph.data(), 1, ys, copies, &one, r0, r1)
                       : launch_axis(plan, 1, io.src, io.work.data(), io.dout.data(), io.dint.data(),
                                     io.dph.data(), 1, ys, none, &one, r0, r1);
  };
  cudaError_t e = cudaSuccess;
  if (pipeline) {
    cudaStream_t xs = plan->pipe_x;
    e = cudaEventRecord(plan->pipe_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(xs, split_row ? plan->holo_half : plan->pipe_fork, 0);
    for (int vi = 0; vi < nv && e == cudaSuccess; ++vi) {
      if (vi == 0 && split_row) {
        e = x_pass(vi, xs, 0, split_row);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(xs, plan->pipe_fork, 0);
        if (e == cudaSuccess) e = x_pass(vi, xs, split_row, -1);
      } else {
        e = x_pass(vi, xs, 0, -1);
      }
      if (e == cudaSuccess) e = cudaEventRecord(plan->x_done[vi], xs);
    }
    // The first and the last view's y pass run in two column halves, each
    // followed by its copies (FP32 plans, views of >= 256 columns; the split
    // column keeps rows of the intermediate 16-byte aligned).
    for (int vi = 0; vi < nv && e == cudaSuccess; ++vi) {
      const int nx1 = plan->views[vi].v.nx1;
      const int half =
          (vi == 0 || vi == nv - 1) && plan->precision == SF_PREC_FP32 && nx1 >= 256 ? (nx1 / 2) & ~15 : 0;
      e = cudaStreamWaitEvent(ys, plan->x_done[vi], 0);
      if (e == cudaSuccess && half) {
        e = y_pass(vi, 0, half, false);
        if (e == cudaSuccess) e = column_copies(vi, 0, half, plan->y_half);
        if (e == cudaSuccess) e = y_pass(vi, half, -1, false);
        if (e == cudaSuccess) e = column_copies(vi, half, nx1, plan->view_done[vi]);
      } else if (e == cudaSuccess) {
        e = y_pass(vi, 0, -1, true);
      }
    }
    // every x pass precedes some y pass, so the y stream's end covers both
    if (e == cudaSuccess) e = cudaEventRecord(plan->pipe_join, ys);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->pipe_join, 0);
  } else {
    for (int vi = 0; vi < nv && e == cudaSuccess; ++vi) {
      e = x_pass(vi, s, 0, -1);
      if (e == cudaSuccess) e = y_pass(vi, 0, -1, true);
    }
  }
  // the caller's stream resumes after the last copy
  if (e == cudaSuccess) e = cudaEventRecord(plan->copies_done, plan->copy_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->copies_done, 0);
  if (e != cudaSuccess) {
    if (pipeline) {
      join_after_error(s, plan->pipe_x, plan->pipe_fork);
      join_after_error(s, plan->pipe_y, plan->pipe_join);
    }
    join_after_error(s, plan->copy_stream, plan->copies_done);
  }
  return e;
}

// Device outputs on `s` alone: every view's x pass, then every y pass, each
// grouped by FFT length; profiling events (when attached) bracket the passes.
// Device outputs of a plan that fused_t5_eligible accepts: the x and y passes
// of every view in one persistent tcgen05 launch on the plan's first schedule
// buffer, each view's y tiles starting as soon as its x tiles are done.
cudaError_t execute_fused_t5(sf_plan plan, const ExecBuffers& io, cudaStream_t s) {
  return launch_fused_views(plan, io.src, io.work.data(), io.dout.data(), io.dint.data(), io.dph.data(),
                            plan->t5_sched, s);
}

cudaError_t execute_single_stream(sf_plan plan, const ExecBuffers& io, cudaStream_t s) {
  auto none = [](const int*, int) { return cudaSuccess; };
  cudaError_t e = cudaSuccess;
  if (plan->prof[0]) e = cudaEventRecord(plan->prof[0], s);
  for (int axis = 0; axis < 2 && e == cudaSuccess; ++axis) {
    if (axis == 1 && plan->prof[1]) e = cudaEventRecord(plan->prof[1], s);
    if (e == cudaSuccess)
      e = launch_axis(plan, axis, io.src, io.work.data(), io.dout.data(), io.dint.data(), io.dph.data(),
                      kMaxPassBatch, s, none);
  }
  if (e == cudaSuccess && plan->prof[2]) e = cudaEventRecord(plan->prof[2], s);
  return e;
}

}  // namespace

int shifted_fresnel_execute(sf_plan plan, const void* holo, void* const* view_out, float* const* intensity,
                            float* const* phase, void* stream) {
  if (!plan || !holo) return SF_ERR_INVALID_ARG;
  const int nv = (int)plan->views.size();
  for (int i = 0; i < nv; ++i) {
    const bool any = (view_out && view_out[i]) || (intensity && intensity[i]) || (phase && phase[i]);
    if (!any) return SF_ERR_INVALID_ARG;
  }
  DeviceGuard guard(plan->device);
  if (!guard.ok) return SF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  ExecBuffers io;

  // hologram: device pointer used in place, host memory staged (the copy is
  // issued below, once the output placement fixes the schedule)
  const size_t holo_elem = plan->in_complex ? sizeof(float2) : sizeof(float);
  const size_t holo_bytes = holo_elem * (size_t)plan->nx0 * plan->ny0;
  io.src = holo;
  bool holo_host = false;
  switch (classify(holo, plan->device)) {
    case PTR_OTHER_DEVICE: return SF_ERR_DEVICE_MISMATCH;
    case PTR_HOST: {
      int rc = stage_alloc(plan, &plan->st_holo, holo_bytes);
      if (rc) return rc;
      io.src = plan->st_holo;
      holo_host = true;
      break;
    }
    default: break;
  }

  // outputs: resolve staging for host buffers
  io.dout.assign(nv, nullptr);
  io.dint.assign(nv, nullptr);
  io.dph.assign(nv, nullptr);
  io.work.resize(nv);
  for (int i = 0; i < nv; ++i) {
    ViewState& vs = plan->views[i];
    io.work[i] = vs.work;
    const size_t npx = (size_t)vs.v.nx1 * vs.v.ny1;
    auto resolve = [&](void* user, void** stage, size_t bytes, void** dev) -> int {
      if (!user) return SF_OK;
      switch (classify(user, plan->device)) {
        case PTR_OTHER_DEVICE: return SF_ERR_DEVICE_MISMATCH;
        case PTR_HOST: {
          int rc = stage_alloc(plan, stage, bytes);
          if (rc) return rc;
          io.d2h.push_back({user, *stage, bytes, i, bytes / npx});
          *dev = *stage;
          return SF_OK;
        }
        default: *dev = user; return SF_OK;
      }
    };
    int rc = resolve(view_out ? view_out[i] : nullptr, (void**)&vs.st_out, sizeof(float2) * npx,
                     (void**)&io.dout[i]);
    if (!rc)
      rc = resolve(intensity ? (void*)intensity[i] : nullptr, (void**)&vs.st_int, sizeof(float) * npx,
                   (void**)&io.dint[i]);
    if (!rc)
      rc = resolve(phase ? (void*)phase[i] : nullptr, (void**)&vs.st_ph, sizeof(float) * npx, (void**)&io.dph[i]);
    if (rc) return rc;
  }

  // Schedule: host outputs -> execute_host_outputs (pipelined unless
  // SF_EXECUTE_SINGLE_STREAM=1); device outputs without profiling events ->
  // execute_fused_t5 where every axis runs the tcgen05 pass, else
  // execute_split_halves for two or more views (neither with
  // SF_EXECUTE_SINGLE_STREAM=1); otherwise execute_single_stream.
  const bool host_out = !io.d2h.empty();
  const bool single = env_is("SF_EXECUTE_SINGLE_STREAM", "1");
  const bool pipeline = host_out && !single;
  // SF_T5_FUSED=0 / =1: one launch per pass / the fused launch wherever eligible
  const bool fused = !host_out && !plan->prof[0] && !single && fused_t5_eligible(plan) &&
                     !env_is("SF_T5_FUSED", "0");
  const bool split = !fused && !host_out && !plan->prof[0] && nv >= 2 && !single;
  if (host_out || split) {
    int rc = pipeline ? ensure_pipeline_resources(plan)
             : host_out ? ensure_copy_resources(plan)
                        : ensure_split_resources(plan);
    if (rc) return rc;
  }
  // The staged hologram goes in two halves when the pipeline can start the
  // first view's x pass on the first half (FP32 passes; the split row keeps
  // the second half's rows 16-byte aligned).
  int split_row = 0;
  if (holo_host && pipeline && plan->precision == SF_PREC_FP32 && plan->ny0 >= 256 && holo_bytes >= ((size_t)1 << 20))
    split_row = (plan->ny0 / 2) & ~15;
  cudaError_t e = cudaSuccess;
  if (holo_host) {
    const size_t b0 = split_row ? holo_elem * (size_t)split_row * plan->nx0 : holo_bytes;
    e = cudaMemcpyAsync(plan->st_holo, holo, b0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && split_row) e = cudaEventRecord(plan->holo_half, s);
    if (e == cudaSuccess && split_row)
      e = cudaMemcpyAsync(static_cast<char*>(plan->st_holo) + b0, static_cast<const char*>(holo) + b0,
                          holo_bytes - b0, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) {
    e = host_out ? execute_host_outputs(plan, io, pipeline, split_row, s)
        : fused  ? execute_fused_t5(plan, io, s)
        : split  ? execute_split_halves(plan, io, s)
                 : execute_single_stream(plan, io, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

int shifted_fresnel_adjoint(sf_plan plan, const void* holo, const void* const* grad_view, void* grad_holo,
                            double* grad_z, void* stream) {
  if (!plan || !grad_view || (!grad_holo && !grad_z)) return SF_ERR_INVALID_ARG;
  if (grad_z && !holo) return SF_ERR_INVALID_ARG;
  DeviceGuard guard(plan->device);
  if (!guard.ok) return SF_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = alloc_adjoint_scratch(plan);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  const int nv = (int)plan->views.size();
  const size_t h0 = (size_t)plan->nx0 * plan->ny0;

  // hologram (only for dL/dz): device pointer used in place, host memory staged
  const void* u0 = holo;
  if (grad_z) {
    const size_t hb = (plan->in_complex ? sizeof(float2) : sizeof(float)) * h0;
    switch (classify(holo, plan->device)) {
      case PTR_OTHER_DEVICE: return SF_ERR_DEVICE_MISMATCH;
      case PTR_HOST:
        if ((rc = stage_alloc(plan, &plan->st_holo, hb))) return rc;
        if (cudaMemcpyAsync(plan->st_holo, holo, hb, cudaMemcpyHostToDevice, s) != cudaSuccess) {
          cudaGetLastError();
          return SF_ERR_CUDA;
        }
        u0 = plan->st_holo;
        break;
      default: break;
    }
  }
  // grad_holo: device pointer written in place, host memory staged
  float2* gout = nullptr;
  bool gout_host = false;
  if (grad_holo) {
    switch (classify(grad_holo, plan->device)) {
      case PTR_OTHER_DEVICE: return SF_ERR_DEVICE_MISMATCH;
      case PTR_HOST: gout = plan->adj_out; gout_host = true; break;
      default: gout = static_cast<float2*>(grad_holo); break;
    }
  }
  if (grad_z && cudaMemsetAsync(plan->adj_z, 0, sizeof(double) * nv, s) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }

  size_t wmax = 1;
  for (const ViewState& vs : plan->views) wmax = std::max(wmax, (size_t)vs.v.nx0 * vs.v.ny1);
  bool first = true;
  for (int vi = 0; vi < nv && e == cudaSuccess; ++vi) {
    if (!grad_view[vi]) continue;
    ViewState& vs = plan->views[vi];
    const sf_view& v = vs.v;
    const size_t n1px = (size_t)v.nx1 * v.ny1;
    const float2* g = static_cast<const float2*>(grad_view[vi]);
    switch (classify(g, plan->device)) {
      case PTR_OTHER_DEVICE: return SF_ERR_DEVICE_MISMATCH;
      case PTR_HOST:
        e = cudaMemcpyAsync(plan->adj_gst, g, sizeof(float2) * n1px, cudaMemcpyHostToDevice, s);
        g = plan->adj_gst;
        break;
      default: break;
    }
    const bool zg = grad_z != nullptr;
    float2* xg = plan->adj_xy;
    float2* yg = plan->adj_xy + n1px;
    if (zg && e == cudaSuccess) {
      // recompute this view's field u1 = A u0 (no stored forward state is needed)
      PassDesc d;
      std::memset(&d, 0, sizeof(d));
      d.cin = vs.ax[0].cin; d.cout = vs.ax[0].cout; d.H = vs.ax[0].H;
      d.n0 = vs.ax[0].n0; d.n1 = vs.ax[0].n1;
      d.src = u0; d.dst = vs.work; d.rows = v.ny0; d.src_ld = v.nx0; d.dst_ld = v.ny0;
      e = run_pass(plan, vs.ax[0].L, plan->in_complex ? PASS_X_CPLX : PASS_X_REAL, &d, 1, s);
      if (e == cudaSuccess) {
        std::memset(&d, 0, sizeof(d));
        d.cin = vs.ax[1].cin; d.cout = vs.ax[1].cout; d.H = vs.ax[1].H;
        d.n0 = vs.ax[1].n0; d.n1 = vs.ax[1].n1;
        d.src = vs.work; d.dst = plan->adj_u1; d.rows = v.nx1; d.src_ld = v.ny0; d.dst_ld = v.nx1;
        e = run_pass(plan, vs.ax[1].L, PASS_Y, &d, 1, s);
      }
      if (e == cudaSuccess) {
        e = launch_weight_xy(g, xg, yg, v.nx1, v.ny1, v.px1, v.py1, v.ox1, v.oy1, s);
        ++g_launches;
      }
    }
    // adjoint along x: rows of g (length nx1) -> nx0 outputs, intermediate [nx0][ny1]
    const float2* ins[3] = {g, xg, yg};
    const int nin = zg ? 3 : 1;
    PassDesc dx[3], dy[3];
    for (int k = 0; k < nin; ++k) {
      std::memset(&dx[k], 0, sizeof(PassDesc));
      dx[k].cin = vs.adj[0].cin; dx[k].cout = vs.adj[0].cout; dx[k].H = vs.adj[0].H;
      dx[k].n0 = vs.adj[0].n0; dx[k].n1 = vs.adj[0].n1;
      dx[k].src = ins[k]; dx[k].dst = plan->adj_work + k * wmax;
      dx[k].rows = v.ny1; dx[k].src_ld = v.nx1; dx[k].dst_ld = v.ny1;
      std::memset(&dy[k], 0, sizeof(PassDesc));
      dy[k].cin = vs.adj[1].cin; dy[k].cout = vs.adj[1].cout; dy[k].H = vs.adj[1].H;
      dy[k].n0 = vs.adj[1].n0; dy[k].n1 = vs.adj[1].n1;
      dy[k].src = plan->adj_work + k * wmax; dy[k].rows = v.nx0; dy[k].src_ld = v.ny1; dy[k].dst_ld = v.nx0;
      if (zg) {
        dy[k].dst = plan->adj_G + k * h0;
      } else {
        dy[k].dst = gout;
        dy[k].accumulate = first ? 0 : 1;
      }
    }
    if (e == cudaSuccess) e = run_pass(plan, vs.adj[0].L, PASS_X_CPLX, dx, nin, s);
    if (e == cudaSuccess) e = run_pass(plan, vs.adj[1].L, PASS_Y, dy, nin, s);
    if (zg && e == cudaSuccess) {
      ZGradArgs za;
      za.g = g; za.u1 = plan->adj_u1;
      za.G0 = plan->adj_G; za.G1 = plan->adj_G + h0; za.G2 = plan->adj_G + 2 * h0;
      za.u0 = u0; za.u0_complex = plan->in_complex ? 1 : 0;
      za.nx0 = v.nx0; za.ny0 = v.ny0; za.nx1 = v.nx1; za.ny1 = v.ny1;
      za.px0 = v.px0; za.py0 = v.py0; za.px1 = v.px1; za.py1 = v.py1;
      za.ox0 = v.ox0; za.oy0 = v.oy0; za.ox1 = v.ox1; za.oy1 = v.oy1;
      const double pi = 3.14159265358979323846;
      const bool pre = !(v.flags & SF_NO_PREFACTOR);
      const double c_re = pre ? -1.0 / v.z : 0.0, c_im = pre ? 2.0 * pi / v.wavelength : 0.0;
      const double q_im = -pi / (v.wavelength * v.z * v.z);
      e = launch_zgrad(za, plan->adj_part, kZGradBlocks, plan->adj_z + vi, c_re, c_im, 0.0, q_im, s);
      g_launches += 2;
      if (e == cudaSuccess && gout) {
        e = launch_axpy(gout, plan->adj_G, h0, first ? 0 : 1, s);
        ++g_launches;
      }
    }
    first = false;
  }
  if (e == cudaSuccess && gout && first) e = cudaMemsetAsync(gout, 0, sizeof(float2) * h0, s);
  if (e == cudaSuccess && gout_host)
    e = cudaMemcpyAsync(grad_holo, gout, sizeof(float2) * h0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad_z)
    e = cudaMemcpyAsync(grad_z, plan->adj_z, sizeof(double) * nv, cudaMemcpyDefault, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

int shifted_fresnel_intensity_loss(sf_plan plan, void* const* fields, const float* const* measured,
                                   void* const* grads, double* loss, void* stream) {
  if (!plan || !fields || !measured || !loss) return SF_ERR_INVALID_ARG;
  const int nv = (int)plan->views.size();
  for (int v = 0; v < nv; ++v) {
    if (!fields[v] || !measured[v]) return SF_ERR_INVALID_ARG;
    for (const void* q : {(const void*)fields[v], (const void*)measured[v], grads ? (const void*)grads[v] : nullptr})
      if (q && classify(q, plan->device) != PTR_DEVICE) return SF_ERR_INVALID_ARG;
  }
  if (classify(loss, plan->device) != PTR_DEVICE) return SF_ERR_INVALID_ARG;
  DeviceGuard guard(plan->device);
  if (!guard.ok) return SF_ERR_CUDA;
  if (!plan->loss_part) {
    void* b = nullptr;
    if (cudaMalloc(&b, sizeof(double) * kZGradBlocks) != cudaSuccess) {
      cudaGetLastError();
      return SF_ERR_OOM;
    }
    plan->staging.push_back(b);
    plan->loss_part = static_cast<double*>(b);
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < nv && e == cudaSuccess; ++v) {
    const sf_view& w = plan->views[v].v;
    e = launch_intensity_loss(static_cast<const float2*>(fields[v]), measured[v],
                              grads ? static_cast<float2*>(grads[v]) : nullptr, (size_t)w.nx1 * w.ny1,
                              plan->loss_part, kZGradBlocks, loss, v > 0 ? 1 : 0, s);
    g_launches += 2;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

int shifted_fresnel_execute_batch(sf_plan plan, const void* const* holos, int n_holos, void* const* view_out,
                                  float* const* intensity, float* const* phase, void* stream) {
  if (!plan || !holos || n_holos < 1) return SF_ERR_INVALID_ARG;
  const int nv = (int)plan->views.size();
  for (int h = 0; h < n_holos; ++h) {
    if (!holos[h]) return SF_ERR_INVALID_ARG;
    for (int v = 0; v < nv; ++v) {
      const size_t i = (size_t)h * nv + v;
      if (!((view_out && view_out[i]) || (intensity && intensity[i]) || (phase && phase[i]))) return SF_ERR_INVALID_ARG;
    }
  }
  DeviceGuard guard(plan->device);
  if (!guard.ok) return SF_ERR_CUDA;
  // device memory of this plan's device only (the batch is one graph launch; nothing is staged)
  for (int h = 0; h < n_holos; ++h) {
    if (classify(holos[h], plan->device) != PTR_DEVICE) return SF_ERR_INVALID_ARG;
    for (int v = 0; v < nv; ++v) {
      const size_t i = (size_t)h * nv + v;
      for (const void* q : {view_out ? (const void*)view_out[i] : nullptr,
                            intensity ? (const void*)intensity[i] : nullptr, phase ? (const void*)phase[i] : nullptr})
        if (q && classify(q, plan->device) != PTR_DEVICE) return SF_ERR_INVALID_ARG;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  int impl = batch_choice(plan, n_holos);
  if (impl < 0) {  // autotune: time both implementations on this call's buffers, keep the faster
    float ms[2] = {-1.f, -1.f};
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t t0 = nullptr, t1 = nullptr;
      int rc = SF_OK;
      if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) rc = SF_ERR_CUDA;
      for (int rep = 0; rep < 2 && rc == SF_OK; ++rep) {  // the first run warms up (graph build, caches)
        if (cudaEventRecord(t0, s) != cudaSuccess) rc = SF_ERR_CUDA;
        if (rc == SF_OK) rc = run_batch(plan, k, holos, n_holos, view_out, intensity, phase, s);
        if (rc == SF_OK && (cudaEventRecord(t1, s) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess))
          rc = SF_ERR_CUDA;
      }
      if (rc == SF_OK) cudaEventElapsedTime(&ms[k], t0, t1);
      if (t0) cudaEventDestroy(t0);
      if (t1) cudaEventDestroy(t1);
      if (rc != SF_OK && rc != SF_ERR_UNSUPPORTED_SIZE) {
        cudaGetLastError();
        return rc;
      }
    }
    impl = (ms[BATCH_PERSISTENT] > 0 && (ms[BATCH_STREAMS] < 0 || ms[BATCH_PERSISTENT] < ms[BATCH_STREAMS]))
               ? BATCH_PERSISTENT : BATCH_STREAMS;
    plan->batch.choice[n_holos] = impl;
    return SF_OK;  // the outputs were written by the timed runs
  }
  return run_batch(plan, impl, holos, n_holos, view_out, intensity, phase, s);
}

int shifted_fresnel_batch_status(sf_plan plan, void* stream) {
  if (!plan) return SF_ERR_INVALID_ARG;
  DeviceGuard guard(plan->device);
  int err = 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
      cudaMemcpy(&err, plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  if (err) {
    cudaMemset(plan->dev_err, 0, sizeof(int));
    return SF_ERR_TIMEOUT;
  }
  return SF_OK;
}

int shifted_fresnel_set_profile_events(sf_plan plan, void* const* events, int n_events) {
  if (!plan) return SF_ERR_INVALID_ARG;
  if (n_events == 0) {
    plan->prof[0] = plan->prof[1] = plan->prof[2] = nullptr;
    return SF_OK;
  }
  if (n_events != 3 || !events || !events[0] || !events[1] || !events[2]) return SF_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i) plan->prof[i] = (cudaEvent_t)events[i];
  return SF_OK;
}

int shifted_fresnel_destroy(sf_plan plan) {
  if (!plan) return SF_ERR_INVALID_ARG;
  DeviceGuard guard(plan->device);
  cudaError_t e = cudaDeviceSynchronize();
  free_plan(plan);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  return SF_OK;
}

}  // extern "C"

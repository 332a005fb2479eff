// sf_tune.cu -- plan-time autotuner for the FP32 row passes.
//
// The cost of a row pass is (rows) x (time per row), and the time per row
// depends only on the FFT length L, the pass kind (real x, complex x, y), the
// kernel and whether the pass is prunable.  Kernels (`impl`): 0 one tile per
// CTA with the default rows per CTA, 1 the persistent kernel with bulk-copy
// prefetch, 2 and 3 one tile per CTA with half and twice the default rows per
// CTA (pass_cta_variant; lengths 1024 to 4096) (n0, n1 <= L / 2: the radix-16 network
// skips the dead half of its first and last stage).  The tuner measures that
// time per row once per device and process for each (L, kind, kernel,
// prunable) a plan asks about: one pass over a synthetic batch of rows (zero
// data; n0 = n1 = L / 2 when prunable, else n0 = L / 2 + 4, n1 = L / 2 - 4;
// rows x L = 2^23), two launches of warm-up, then the median of five launches
// timed with CUDA events.  With SF_AUTOTUNE_CACHE naming a file, measurements
// are also read from and appended to it (one line per measurement: device
// key, L, kind, kernel, prunable, ns per row), so later processes skip the
// timing.
//
// The plan then picks, per axis, the cheaper of the two FFT lengths that can
// hold the linear convolution (the next power of two, and the next length
// with a factor 3 when that one is shorter), and per (L, kind) the cheaper
// kernel.  Every choice computes the same convolution; only rounding differs.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "sf_internal.h"

namespace sf {
namespace {

using Key = std::tuple<std::string, int, int, int, int>;  // device key, L, kind, kernel, prunable

std::mutex g_mu;
std::map<Key, double> g_cost;
bool g_file_read = false;

std::string device_key(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string k = prop.name;
  for (char& c : k)
    if (c == ' ' || c == '\t') c = '_';
  return k + "_sm" + std::to_string(prop.multiProcessorCount);
}

void read_cache_file() {
  if (g_file_read) return;
  g_file_read = true;
  const char* path = std::getenv("SF_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char dev[256];
  int L, kind, impl, prune;
  double ns;
  while (std::fscanf(f, "%255s %d %d %d %d %lf", dev, &L, &kind, &impl, &prune, &ns) == 6)
    if (ns > 0) g_cost[Key(dev, L, kind, impl, prune)] = ns;
  std::fclose(f);
}

void append_cache_file(const Key& k, double ns) {
  const char* path = std::getenv("SF_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d %.6g\n", std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k),
               std::get<4>(k), ns);
  std::fclose(f);
}

// Time per row (ns) of one synthetic pass; < 0 if it could not be measured.
double measure(int L, PassKind kind, int impl, bool prune, int sms, cudaStream_t s) {
  const int variant = impl >= 2 ? impl - 1 : 0;
  const int G = pass_rows_per_cta(L, variant);
  if (G < 1) return -1;
  // not prunable: n0 just above L / 2, keeping rows a multiple of 16 bytes
  // (the persistent kernel's bulk copies need that)
  const int n0 = prune ? L / 2 : L / 2 + 4, n1 = prune ? L / 2 : L / 2 - 4;
  int rows = std::max(256, (1 << 23) / L);
  rows = (rows + G - 1) / G * G;
  const size_t elem = kind == PASS_X_REAL ? sizeof(float) : sizeof(float2);
  const size_t b_src = elem * (size_t)rows * n0, b_dst = sizeof(float2) * (size_t)rows * n1;
  const size_t n_tw = twiddle_entries(L);
  std::vector<float4> tw_host(n_tw);
  build_twiddles(L, tw_host.data());
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_dst = al(b_src), o_cin = o_dst + al(b_dst), o_cout = o_cin + al(sizeof(float2) * n0),
               o_H = o_cout + al(sizeof(float2) * n1), o_tw = o_H + al(sizeof(float2) * L),
               o_err = o_tw + al(sizeof(float4) * std::max<size_t>(n_tw, 1)), total = o_err + 256;
  char* mem = nullptr;
  if (cudaMalloc(&mem, total) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  cudaEvent_t ev[6] = {};
  double result = -1;
  cudaError_t e = cudaMemsetAsync(mem, 0, total, s);
  if (e == cudaSuccess && n_tw)
    e = cudaMemcpyAsync(mem + o_tw, tw_host.data(), sizeof(float4) * n_tw, cudaMemcpyHostToDevice, s);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  if (e == cudaSuccess) {
    PassBatch b;
    std::memset(&b, 0, sizeof(b));
    b.count = 1;
    PassDesc& d = b.d[0];
    d.src = mem;
    d.dst = reinterpret_cast<float2*>(mem + o_dst);
    d.cin = reinterpret_cast<const float2*>(mem + o_cin);
    d.cout = reinterpret_cast<const float2*>(mem + o_cout);
    d.H = reinterpret_cast<const float2*>(mem + o_H);
    d.n0 = n0;
    d.n1 = n1;
    d.rows = rows;
    d.src_ld = n0;
    d.dst_ld = rows;
    const float4* tw = reinterpret_cast<const float4*>(mem + o_tw);
    int* err = reinterpret_cast<int*>(mem + o_err);
    auto launch = [&]() {
      return impl == 1 ? launch_pass_persistent(L, kind, b, tw, err, sms, s)
                       : launch_pass(L, kind, b, rows / G, tw, s, variant);
    };
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch();
    std::vector<float> ms;
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
      e = cudaEventRecord(ev[0], s);
      if (e == cudaSuccess) e = launch();
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      float t = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
      ms.push_back(t);
    }
    int h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_err == 0 && ms.size() == 5) {
      std::sort(ms.begin(), ms.end());
      result = 1e6 * ms[2] / rows;
    }
  }
  if (e != cudaSuccess) cudaGetLastError();
  cudaStreamSynchronize(s);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  cudaFree(mem);
  return result;
}

}  // namespace

int autotune_mode() {
  const char* m = std::getenv("SF_AUTOTUNE");
  return (m && std::strcmp(m, "1") == 0) ? 1 : 0;
}

double row_cost_ns(int device, int L, PassKind kind, int impl, bool prune, int sms, cudaStream_t s) {
  if (impl == 1 && !tma_length_supported(L)) return -1;
  if (impl >= 2 && pass_rows_per_cta(L, impl - 1) < 1) return -1;
  std::lock_guard<std::mutex> lock(g_mu);
  read_cache_file();
  const Key k(device_key(device), L, (int)kind, impl, prune ? 1 : 0);
  auto it = g_cost.find(k);
  if (it != g_cost.end()) return it->second;
  const double ns = measure(L, kind, impl, prune, sms, s);
  if (ns > 0) {
    g_cost[k] = ns;
    append_cache_file(k, ns);
  }
  return ns;
}

}  // namespace sf

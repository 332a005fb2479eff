// sf_plain.cu -- the paper's per-view procedure done literally with cuFFT, as
// a timed comparison for the fused library (never used by it).
//
// Section 2.2, steps 2-10, for each view on a zero-padded Lpy x Lpx grid
// (Lp >= N0 + N1 - 1; 2048 x 2048 for 1024 -> 1024 views, the paper's
// doubled grid):
//   2  zero-pad the hologram into the grid
//   3  multiply by the exponentials of Eq. 3
//   4  2-D FFT (cufftExecC2C)
//   5  generate h of Eq. 4 on the grid
//   6  2-D FFT of h (every call, as the paper does per frame)
//   7  complex multiply of the two spectra
//   8  inverse 2-D FFT
//   9  crop to N1y x N1x and apply C1 of Eq. 2
//   10 intensity |u1|^2 (Eq. 5), when requested
// The 1-D exponential factors are evaluated once per view on the host in
// double precision from Eqs. 2-4 (offsets O = o / p in pixels, index origin
// -floor(N/2)), so the comparison measures the procedure, not phase error.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <complex>
#include <new>
#include <vector>

#include "shifted_fresnel.h"

namespace {

struct PlainView {
  sf_view v;
  int lx, ly;
  float2 *cin_x, *cin_y, *cout_x, *cout_y, *h_x, *h_y;  // device vectors
  cufftHandle fft;
};

int next_pow2(int n) {
  int l = 1;
  while (l < n) l <<= 1;
  return l;
}

using cd = std::complex<double>;

void axis_vectors(const sf_view& v, int axis, int Lp, std::vector<float2>& cin, std::vector<float2>& cout,
                  std::vector<float2>& h) {
  const double lam = v.wavelength, z = v.z, pi = 3.14159265358979323846;
  const int n0 = axis ? v.ny0 : v.nx0, n1 = axis ? v.ny1 : v.nx1;
  const double p0 = axis ? v.py0 : v.px0, p1 = axis ? v.py1 : v.px1;
  const double O0 = (axis ? v.oy0 : v.ox0) / p0, O1 = (axis ? v.oy1 : v.ox1) / p1;
  const double S = p0 * p1 / (lam * z);
  auto e = [](double ph) { return cd(std::cos(ph), std::sin(ph)); };
  cin.resize(n0);
  cout.resize(n1);
  h.assign(Lp, make_float2(0.f, 0.f));
  for (int m0 = 0; m0 < n0; ++m0) {
    const double x0 = (m0 - n0 / 2 + O0) * p0;
    const cd c = e(pi * x0 * x0 / (lam * z)) * e(-2.0 * pi * m0 * S * (-(n1 / 2) + O1)) * e(-pi * S * m0 * (double)m0);
    cin[m0] = make_float2((float)c.real(), (float)c.imag());
  }
  cd pre = 1.0;
  if (axis == 1 && !(v.flags & SF_NO_PREFACTOR)) pre = e(2.0 * pi * std::fmod(z / lam, 1.0)) / cd(0.0, lam * z);
  for (int m1 = 0; m1 < n1; ++m1) {
    const double x1 = (m1 - n1 / 2 + O1) * p1;
    const cd c = pre * e(pi * x1 * x1 / (lam * z)) * e(-2.0 * pi / (lam * z) * (-(n0 / 2) + O0) * p0 * x1) *
                 e(-pi * S * m1 * (double)m1);
    cout[m1] = make_float2((float)c.real(), (float)c.imag());
  }
  for (int j = 0; j < Lp; ++j) {
    long d;
    if (j < n1) d = j;
    else if (j > Lp - n0) d = (long)j - Lp;
    else continue;
    const cd c = e(pi * S * (double)d * (double)d);
    h[j] = make_float2((float)c.real(), (float)c.imag());
  }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// step 2
__global__ void k_pad(const void* holo, int cplx, int nx0, int ny0, float2* B, int lx, int ly) {
  const size_t n = (size_t)lx * ly;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % lx), y = (int)(i / lx);
    float2 v = make_float2(0.f, 0.f);
    if (x < nx0 && y < ny0) {
      const size_t k = (size_t)y * nx0 + x;
      v = cplx ? static_cast<const float2*>(holo)[k] : make_float2(static_cast<const float*>(holo)[k], 0.f);
    }
    B[i] = v;
  }
}

// step 3
__global__ void k_chirp_in(float2* B, int lx, int nx0, int ny0, const float2* cx, const float2* cy) {
  const size_t n = (size_t)nx0 * ny0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx0), y = (int)(i / nx0);
    float2* p = B + (size_t)y * lx + x;
    *p = cmul(*p, cmul(cx[x], cy[y]));
  }
}

// step 5
__global__ void k_hgen(float2* Hb, int lx, int ly, const float2* hx, const float2* hy) {
  const size_t n = (size_t)lx * ly;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    Hb[i] = cmul(hx[i % lx], hy[i / lx]);
}

// step 7
__global__ void k_mul(float2* B, const float2* Hb, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    B[i] = cmul(B[i], Hb[i]);
}

// steps 9-10
__global__ void k_crop(const float2* B, int lx, int nx1, int ny1, const float2* cx, const float2* cy, float scale,
                       float2* out, float* inten) {
  const size_t n = (size_t)nx1 * ny1;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx1), y = (int)(i / nx1);
    float2 u = cmul(B[(size_t)y * lx + x], cmul(cx[x], cy[y]));
    u = make_float2(u.x * scale, u.y * scale);
    if (out) out[i] = u;
    if (inten) inten[i] = u.x * u.x + u.y * u.y;
  }
}

int blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 8192 ? (b ? b : 1) : 8192);
}

}  // namespace

struct sf_plain_s {
  int device = 0;
  std::vector<PlainView> views;
  float2* B = nullptr;
  float2* Hb = nullptr;
  std::vector<void*> allocs;
};

extern "C" {

int sf_plain_destroy(sf_plain_s* p) {
  if (!p) return SF_ERR_INVALID_ARG;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  for (PlainView& pv : p->views)
    if (pv.fft) cufftDestroy(pv.fft);
  for (void* a : p->allocs) cudaFree(a);
  delete p;
  return SF_OK;
}

int sf_plain_create(sf_plain_s** out, const sf_view* views, int n_views, int device) {
  if (!out || !views || n_views < 1) return SF_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return SF_ERR_CUDA;
  sf_plain_s* p = new (std::nothrow) sf_plain_s();
  if (!p) return SF_ERR_OOM;
  p->device = device;
  size_t max_grid = 0;
  for (int i = 0; i < n_views; ++i) {
    PlainView pv{};
    pv.v = views[i];
    pv.lx = next_pow2(views[i].nx0 + views[i].nx1 - 1);
    pv.ly = next_pow2(views[i].ny0 + views[i].ny1 - 1);
    max_grid = std::max(max_grid, (size_t)pv.lx * pv.ly);
    std::vector<float2> cin[2], cout[2], h[2];
    axis_vectors(pv.v, 0, pv.lx, cin[0], cout[0], h[0]);
    axis_vectors(pv.v, 1, pv.ly, cin[1], cout[1], h[1]);
    float2** dst[6] = {&pv.cin_x, &pv.cin_y, &pv.cout_x, &pv.cout_y, &pv.h_x, &pv.h_y};
    std::vector<float2>* src[6] = {&cin[0], &cin[1], &cout[0], &cout[1], &h[0], &h[1]};
    for (int k = 0; k < 6; ++k) {
      void* d = nullptr;
      if (cudaMalloc(&d, sizeof(float2) * src[k]->size()) != cudaSuccess) {
        sf_plain_destroy(p);
        return SF_ERR_OOM;
      }
      p->allocs.push_back(d);
      cudaMemcpy(d, src[k]->data(), sizeof(float2) * src[k]->size(), cudaMemcpyHostToDevice);
      *dst[k] = static_cast<float2*>(d);
    }
    if (cufftPlan2d(&pv.fft, pv.ly, pv.lx, CUFFT_C2C) != CUFFT_SUCCESS) {
      pv.fft = 0;
      p->views.push_back(pv);
      sf_plain_destroy(p);
      return SF_ERR_CUDA;
    }
    p->views.push_back(pv);
  }
  void *b = nullptr, *hb = nullptr;
  if (cudaMalloc(&b, sizeof(float2) * max_grid) != cudaSuccess ||
      cudaMalloc(&hb, sizeof(float2) * max_grid) != cudaSuccess) {
    if (b) cudaFree(b);
    sf_plain_destroy(p);
    return SF_ERR_OOM;
  }
  p->allocs.push_back(b);
  p->allocs.push_back(hb);
  p->B = static_cast<float2*>(b);
  p->Hb = static_cast<float2*>(hb);
  *out = p;
  return SF_OK;
}

// Views are computed one after another on `stream`, reusing two padded grids.
int sf_plain_execute(sf_plain_s* p, const void* holo, void* const* view_out, float* const* intensity, void* stream) {
  if (!p || !holo) return SF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  for (size_t i = 0; i < p->views.size(); ++i) {
    PlainView& pv = p->views[i];
    const sf_view& v = pv.v;
    const size_t n = (size_t)pv.lx * pv.ly;
    const int cplx = (v.flags & SF_IN_COMPLEX) ? 1 : 0;
    k_pad<<<blocks_for(n), 256, 0, s>>>(holo, cplx, v.nx0, v.ny0, p->B, pv.lx, pv.ly);
    k_chirp_in<<<blocks_for((size_t)v.nx0 * v.ny0), 256, 0, s>>>(p->B, pv.lx, v.nx0, v.ny0, pv.cin_x, pv.cin_y);
    if (cufftSetStream(pv.fft, s) != CUFFT_SUCCESS) return SF_ERR_CUDA;
    if (cufftExecC2C(pv.fft, (cufftComplex*)p->B, (cufftComplex*)p->B, CUFFT_FORWARD) != CUFFT_SUCCESS)
      return SF_ERR_CUDA;
    k_hgen<<<blocks_for(n), 256, 0, s>>>(p->Hb, pv.lx, pv.ly, pv.h_x, pv.h_y);
    if (cufftExecC2C(pv.fft, (cufftComplex*)p->Hb, (cufftComplex*)p->Hb, CUFFT_FORWARD) != CUFFT_SUCCESS)
      return SF_ERR_CUDA;
    k_mul<<<blocks_for(n), 256, 0, s>>>(p->B, p->Hb, n);
    if (cufftExecC2C(pv.fft, (cufftComplex*)p->B, (cufftComplex*)p->B, CUFFT_INVERSE) != CUFFT_SUCCESS)
      return SF_ERR_CUDA;
    k_crop<<<blocks_for((size_t)v.nx1 * v.ny1), 256, 0, s>>>(
        p->B, pv.lx, v.nx1, v.ny1, pv.cout_x, pv.cout_y, 1.0f / (float)n,
        view_out ? static_cast<float2*>(view_out[i]) : nullptr, intensity ? intensity[i] : nullptr);
    if (cudaGetLastError() != cudaSuccess) return SF_ERR_CUDA;
  }
  return SF_OK;
}

}  // extern "C"

// sf_adjoint.cu -- element-wise and reduction kernels of the adjoint path.
//
// The adjoint itself (A^H of Eqs. 1-4 per view) runs on the row-pass kernel
// with the adjoint chirps and spectra built at plan time.  This file holds
// what the z-derivative needs.  With beta = 1/(lambda z), differentiating the
// Fresnel sum of Section 2.1 gives
//
//   du1/dz = (dC/dz / C) u1 - (i pi beta / z) [ (x1^2 + y1^2) u1
//            - 2 x1 A(x0 u0) - 2 y1 A(y0 u0) + A((x0^2 + y0^2) u0) ],
//
// so for a loss with view gradient g (dL/dz = Re sum conj(g) du1/dz)
//
//   dL/dz = Re[ c <g, u1> + q ( <g, (x1^2 + y1^2) u1> - 2 <A^H(x1 g), x0 u0>
//                               - 2 <A^H(y1 g), y0 u0> + <A^H g, (x0^2 + y0^2) u0> ) ]
//
// with c = dC/dz / C = i k - 1/z (0 without the prefactor), q = -i pi beta / z
// and <a, b> = sum conj(a) b.  The inner products are accumulated in double
// precision in a fixed order (deterministic).
#include "sf_internal.h"

namespace sf {
namespace {

__device__ __forceinline__ double coord(int m, int n, double p, double o) { return o + (double)(m - n / 2) * p; }

// xg = x1(m1) g, yg = y1(n1) g over the view grid.
__global__ void k_weight_xy(const float2* __restrict__ g, float2* __restrict__ xg, float2* __restrict__ yg,
                            int nx1, int ny1, double px1, double py1, double ox1, double oy1) {
  const unsigned n = (unsigned)nx1 * (unsigned)ny1;  // < 2^31
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int n1 = (int)(i / (unsigned)nx1), m1 = (int)(i - (unsigned)n1 * (unsigned)nx1);
    const float x1 = (float)coord(m1, nx1, px1, ox1), y1 = (float)coord(n1, ny1, py1, oy1);
    const float2 v = g[i];
    xg[i] = make_float2(x1 * v.x, x1 * v.y);
    yg[i] = make_float2(y1 * v.x, y1 * v.y);
  }
}

// acc += conj(a) * b * w
__device__ __forceinline__ void cacc(double2& acc, float2 a, double2 b, double w) {
  acc.x += w * ((double)a.x * b.x + (double)a.y * b.y);
  acc.y += w * ((double)a.x * b.y - (double)a.y * b.x);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-block partial sums of the five inner products, partials[block * 5 + k].
__global__ void __launch_bounds__(256) k_zgrad_partial(const ZGradArgs a, double2* __restrict__ partials) {
  double2 s[5];
  for (int k = 0; k < 5; ++k) s[k] = make_double2(0.0, 0.0);
  // grids are at most 8192 x 8192 (< 2^31 elements): 32-bit index arithmetic
  const unsigned stride = gridDim.x * blockDim.x;
  const unsigned n1 = (unsigned)a.nx1 * (unsigned)a.ny1;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += stride) {
    const int n = (int)(i / (unsigned)a.nx1), m = (int)(i - (unsigned)n * (unsigned)a.nx1);
    const double x1 = coord(m, a.nx1, a.px1, a.ox1), y1 = coord(n, a.ny1, a.py1, a.oy1);
    const float2 u = a.u1[i];
    const double2 ud = make_double2(u.x, u.y);
    cacc(s[0], a.g[i], ud, 1.0);
    cacc(s[1], a.g[i], ud, x1 * x1 + y1 * y1);
  }
  const unsigned n0 = (unsigned)a.nx0 * (unsigned)a.ny0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += stride) {
    const int n = (int)(i / (unsigned)a.nx0), m = (int)(i - (unsigned)n * (unsigned)a.nx0);
    const double x0 = coord(m, a.nx0, a.px0, a.ox0), y0 = coord(n, a.ny0, a.py0, a.oy0);
    double2 u;
    if (a.u0_complex) {
      const float2 f = static_cast<const float2*>(a.u0)[i];
      u = make_double2(f.x, f.y);
    } else {
      u = make_double2(static_cast<const float*>(a.u0)[i], 0.0);
    }
    cacc(s[2], a.G1[i], u, x0);
    cacc(s[3], a.G2[i], u, y0);
    cacc(s[4], a.G0[i], u, x0 * x0 + y0 * y0);
  }
  __shared__ double red[8][10];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 5; ++k) {
    const double re = warp_sum(s[k].x), im = warp_sum(s[k].y);
    if (lane == 0) {
      red[warp][2 * k] = re;
      red[warp][2 * k + 1] = im;
    }
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    double* out = reinterpret_cast<double*>(partials + (size_t)blockIdx.x * 5);
    out[threadIdx.x] = t;
  }
}

// Sum the partials in block order and form dL/dz: thread j < 10 sums the
// real (even j) or imaginary (odd j) part of inner product j / 2.
__global__ void k_zgrad_final(const double2* __restrict__ partials, int n_partials, double* out, double c_re,
                              double c_im, double q_re, double q_im) {
  __shared__ double t[10];
  const int j = threadIdx.x;
  if (blockIdx.x != 0) return;
  if (j < 10) {
    const double* p = reinterpret_cast<const double*>(partials) + j;
    double acc = 0.0;
    for (int b = 0; b < n_partials; ++b) acc += p[(size_t)b * 10];
    t[j] = acc;
  }
  __syncthreads();
  if (j != 0) return;
  const double tr = t[2] - 2.0 * t[4] - 2.0 * t[6] + t[8];
  const double ti = t[3] - 2.0 * t[5] - 2.0 * t[7] + t[9];
  *out = (c_re * t[0] - c_im * t[1]) + (q_re * tr - q_im * ti);
}

// Intensity loss of one view (Eq. 5): r = |u|^2 - I per pixel, block partials
// of sum r^2 in double precision, and (when g is given) the loss gradient
// g = 4 r u, i.e. 2 dL/d(conj u) (the conjugate-Wirtinger convention of
// PyTorch's complex autograd).
__global__ void __launch_bounds__(256) k_intensity_partial(const float2* __restrict__ u, const float* __restrict__ I,
                                                           float2* __restrict__ g, unsigned n,
                                                           double* __restrict__ partials) {
  double acc = 0.0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 v = u[i];
    const float r = fmaf(v.x, v.x, v.y * v.y) - I[i];
    acc += (double)r * (double)r;
    if (g) g[i] = make_float2(4.f * r * v.x, 4.f * r * v.y);
  }
  __shared__ double red[8];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// out (+)= the partials summed in block order.
__global__ void k_sum_partials(const double* __restrict__ partials, int n_partials, double* out, int accumulate) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int b = 0; b < n_partials; ++b) t += partials[b];
  *out = accumulate ? *out + t : t;
}

__global__ void k_axpy(float2* __restrict__ y, const float2* __restrict__ x, size_t n, int accumulate) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = x[i];
    if (accumulate) {
      const float2 w = y[i];
      y[i] = make_float2(w.x + v.x, w.y + v.y);
    } else {
      y[i] = v;
    }
  }
}

int grid_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_weight_xy(const float2* g, float2* xg, float2* yg, int nx1, int ny1, double px1, double py1,
                             double ox1, double oy1, cudaStream_t s) {
  k_weight_xy<<<grid_for((size_t)nx1 * ny1), 256, 0, s>>>(g, xg, yg, nx1, ny1, px1, py1, ox1, oy1);
  return cudaGetLastError();
}

cudaError_t launch_zgrad(const ZGradArgs& a, double2* partials, int n_partials, double* out, double c_re,
                         double c_im, double q_re, double q_im, cudaStream_t s) {
  k_zgrad_partial<<<n_partials, 256, 0, s>>>(a, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_zgrad_final<<<1, 32, 0, s>>>(partials, n_partials, out, c_re, c_im, q_re, q_im);
  return cudaGetLastError();
}

cudaError_t launch_intensity_loss(const float2* u, const float* I, float2* g, size_t n, double* partials,
                                  int n_partials, double* loss, int accumulate, cudaStream_t s) {
  k_intensity_partial<<<n_partials, 256, 0, s>>>(u, I, g, (unsigned)n, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_partials<<<1, 32, 0, s>>>(partials, n_partials, loss, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_axpy(float2* y, const float2* x, size_t n, int accumulate, cudaStream_t s) {
  k_axpy<<<grid_for(n), 256, 0, s>>>(y, x, n, accumulate);
  return cudaGetLastError();
}

}  // namespace sf

/*
 * FP64 CPU oracle for Shifted-Fresnel diffraction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library under paper_1001_4309_gb300/.
 *
 * What it computes (Section 2.1, Eqs. 1-5, read as the discretised Fresnel
 * integral that Shifted-Fresnel diffraction factors):
 *
 *   u1[n1][m1] = C * sum_{n0,m0} u0[n0][m0] * exp(i pi ((x1-x0)^2 + (y1-y0)^2) / (lambda z))
 *   C          = exp(i k z) / (i lambda z),  k = 2 pi / lambda
 *
 * with centred sample coordinates x = o + (m - floor(N/2)) p (o physical,
 * metres).  Multiplying out Eqs. 2-4 with Eq. 1's convolution gives exactly
 * this sum when the paper's offsets O are counted in pixels of their own
 * plane (o = O p) and its index origin is -N/2; that is the reading used here.
 *
 * The sum is evaluated directly and separably, u1 = C * Ky * u0 * Kx^T, with
 * every kernel entry exp(i pi d^2/(lambda z)) computed from its definition in
 * double precision: no FFT, no chirp decomposition, no blocking.  Cost is
 * O(ny0 nx0 nx1 + ny1 ny0 nx1).
 *
 * Also provided (same definition, by hand):
 *   sfo_adjoint   the conjugate transpose A^H g (the back-propagation operator);
 *   sfo_forward_dz the derivative d u1 / d z of the forward sum.
 *
 * Complex arrays are interleaved (re, im) doubles, row-major [rows][cols].
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  double wavelength, z;     /* metres */
  double px0, py0;          /* hologram pitch */
  double px1, py1;          /* view pitch */
  double ox0, oy0;          /* hologram-plane offset */
  double ox1, oy1;          /* view-plane offset */
  int nx0, ny0, nx1, ny1;   /* sizes */
  int no_prefactor;         /* 1: drop exp(ikz)/(i lambda z) */
} sfo_view;

/* Sample coordinate of index m on a plane of n samples, pitch p, offset o. */
static double coord(int m, int n, double p, double o) {
  return o + (double)(m - n / 2) * p;
}

/* One Fresnel kernel entry exp(i pi (x1 - x0)^2 / (lambda z)). */
static double complex fresnel_kernel(double x1, double x0, double wavelength, double z) {
  double d = x1 - x0;
  return cexp(I * (M_PI * d * d / (wavelength * z)));
}

/* C = exp(i k z) / (i lambda z), or 1 when the prefactor is dropped. */
static double complex prefactor(const sfo_view* v) {
  if (v->no_prefactor) return 1.0;
  double k = 2.0 * M_PI / v->wavelength;
  return cexp(I * (k * v->z)) / (I * v->wavelength * v->z);
}

static int check_view(const sfo_view* v) {
  if (!v) return -1;
  if (!(v->wavelength > 0) || !(v->z != 0) || !isfinite(v->z)) return -1;
  if (!(v->px0 > 0) || !(v->py0 > 0) || !(v->px1 > 0) || !(v->py1 > 0)) return -1;
  if (v->nx0 <= 0 || v->ny0 <= 0 || v->nx1 <= 0 || v->ny1 <= 0) return -1;
  return 0;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int sfo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Forward sum for the view columns m1 in [m1_begin, m1_end) and all rows.
 * u0: [ny0][nx0] complex; u1: [ny1][m1_end - m1_begin] complex.
 */
int sfo_forward(const sfo_view* v, const double* u0, int m1_begin, int m1_end,
                double* u1, int nthreads) {
  if (check_view(v) || !u0 || !u1) return -1;
  if (m1_begin < 0 || m1_end > v->nx1 || m1_begin >= m1_end) return -1;
  set_threads(nthreads);
  const int nx0 = v->nx0, ny0 = v->ny0, ny1 = v->ny1;
  const int nc = m1_end - m1_begin;
  const double complex* in = (const double complex*)u0;
  double complex* out = (double complex*)u1;

  double complex* Kx = malloc(sizeof(double complex) * (size_t)nc * nx0);
  double complex* Ky = malloc(sizeof(double complex) * (size_t)ny1 * ny0);
  double complex* tmp = malloc(sizeof(double complex) * (size_t)ny0 * nc);
  if (!Kx || !Ky || !tmp) { free(Kx); free(Ky); free(tmp); return -2; }

  for (int c = 0; c < nc; ++c) {
    double x1 = coord(m1_begin + c, v->nx1, v->px1, v->ox1);
    for (int m0 = 0; m0 < nx0; ++m0)
      Kx[(size_t)c * nx0 + m0] = fresnel_kernel(x1, coord(m0, nx0, v->px0, v->ox0), v->wavelength, v->z);
  }
  for (int n1 = 0; n1 < ny1; ++n1) {
    double y1 = coord(n1, ny1, v->py1, v->oy1);
    for (int n0 = 0; n0 < ny0; ++n0)
      Ky[(size_t)n1 * ny0 + n0] = fresnel_kernel(y1, coord(n0, ny0, v->py0, v->oy0), v->wavelength, v->z);
  }

  /* tmp[n0][c] = sum_m0 u0[n0][m0] Kx[c][m0] */
#pragma omp parallel for schedule(static)
  for (int n0 = 0; n0 < ny0; ++n0) {
    for (int c = 0; c < nc; ++c) {
      double complex s = 0;
      for (int m0 = 0; m0 < nx0; ++m0) s += in[(size_t)n0 * nx0 + m0] * Kx[(size_t)c * nx0 + m0];
      tmp[(size_t)n0 * nc + c] = s;
    }
  }
  /* u1[n1][c] = C sum_n0 Ky[n1][n0] tmp[n0][c] */
  const double complex C = prefactor(v);
#pragma omp parallel for schedule(static)
  for (int n1 = 0; n1 < ny1; ++n1) {
    for (int c = 0; c < nc; ++c) {
      double complex s = 0;
      for (int n0 = 0; n0 < ny0; ++n0) s += Ky[(size_t)n1 * ny0 + n0] * tmp[(size_t)n0 * nc + c];
      out[(size_t)n1 * nc + c] = C * s;
    }
  }
  free(Kx); free(Ky); free(tmp);
  return 0;
}

/*
 * Adjoint (conjugate transpose) of the forward operator:
 *   a[n0][m0] = conj(C) sum_{n1,m1} conj(Ky[n1][n0] Kx[m1][m0]) g[n1][m1].
 * g: [ny1][nx1] complex; a: [ny0][nx0] complex.
 */
int sfo_adjoint(const sfo_view* v, const double* g, double* a, int nthreads) {
  if (check_view(v) || !g || !a) return -1;
  set_threads(nthreads);
  const int nx0 = v->nx0, ny0 = v->ny0, nx1 = v->nx1, ny1 = v->ny1;
  const double complex* in = (const double complex*)g;
  double complex* out = (double complex*)a;

  double complex* Kx = malloc(sizeof(double complex) * (size_t)nx1 * nx0);
  double complex* Ky = malloc(sizeof(double complex) * (size_t)ny1 * ny0);
  double complex* tmp = malloc(sizeof(double complex) * (size_t)ny1 * nx0);
  if (!Kx || !Ky || !tmp) { free(Kx); free(Ky); free(tmp); return -2; }
  for (int m1 = 0; m1 < nx1; ++m1) {
    double x1 = coord(m1, nx1, v->px1, v->ox1);
    for (int m0 = 0; m0 < nx0; ++m0)
      Kx[(size_t)m1 * nx0 + m0] = fresnel_kernel(x1, coord(m0, nx0, v->px0, v->ox0), v->wavelength, v->z);
  }
  for (int n1 = 0; n1 < ny1; ++n1) {
    double y1 = coord(n1, ny1, v->py1, v->oy1);
    for (int n0 = 0; n0 < ny0; ++n0)
      Ky[(size_t)n1 * ny0 + n0] = fresnel_kernel(y1, coord(n0, ny0, v->py0, v->oy0), v->wavelength, v->z);
  }
  /* tmp[n1][m0] = sum_m1 g[n1][m1] conj(Kx[m1][m0]) */
#pragma omp parallel for schedule(static)
  for (int n1 = 0; n1 < ny1; ++n1) {
    for (int m0 = 0; m0 < nx0; ++m0) {
      double complex s = 0;
      for (int m1 = 0; m1 < nx1; ++m1) s += in[(size_t)n1 * nx1 + m1] * conj(Kx[(size_t)m1 * nx0 + m0]);
      tmp[(size_t)n1 * nx0 + m0] = s;
    }
  }
  const double complex Cc = conj(prefactor(v));
#pragma omp parallel for schedule(static)
  for (int n0 = 0; n0 < ny0; ++n0) {
    for (int m0 = 0; m0 < nx0; ++m0) {
      double complex s = 0;
      for (int n1 = 0; n1 < ny1; ++n1) s += conj(Ky[(size_t)n1 * ny0 + n0]) * tmp[(size_t)n1 * nx0 + m0];
      out[(size_t)n0 * nx0 + m0] = Cc * s;
    }
  }
  free(Kx); free(Ky); free(tmp);
  return 0;
}

/*
 * Derivative of the forward sum with respect to z, from differentiating the
 * definition term by term:
 *   d/dz exp(i pi d^2/(lambda z)) = -i pi d^2/(lambda z^2) exp(i pi d^2/(lambda z))
 *   d/dz C                        = C (i k - 1/z)          (0 with no prefactor)
 * du: [ny1][nx1] complex.
 */
int sfo_forward_dz(const sfo_view* v, const double* u0, double* du, int nthreads) {
  if (check_view(v) || !u0 || !du) return -1;
  set_threads(nthreads);
  const int nx0 = v->nx0, ny0 = v->ny0, nx1 = v->nx1, ny1 = v->ny1;
  const double complex* in = (const double complex*)u0;
  double complex* out = (double complex*)du;
  const double wl = v->wavelength, z = v->z;

  double complex* Kx = malloc(sizeof(double complex) * (size_t)nx1 * nx0);
  double* Dx = malloc(sizeof(double) * (size_t)nx1 * nx0);
  double complex* Ky = malloc(sizeof(double complex) * (size_t)ny1 * ny0);
  double* Dy = malloc(sizeof(double) * (size_t)ny1 * ny0);
  double complex* tA = malloc(sizeof(double complex) * (size_t)ny0 * nx1);
  double complex* tB = malloc(sizeof(double complex) * (size_t)ny0 * nx1);
  if (!Kx || !Dx || !Ky || !Dy || !tA || !tB) {
    free(Kx); free(Dx); free(Ky); free(Dy); free(tA); free(tB); return -2;
  }
  for (int m1 = 0; m1 < nx1; ++m1) {
    double x1 = coord(m1, nx1, v->px1, v->ox1);
    for (int m0 = 0; m0 < nx0; ++m0) {
      double x0 = coord(m0, nx0, v->px0, v->ox0);
      Kx[(size_t)m1 * nx0 + m0] = fresnel_kernel(x1, x0, wl, z);
      Dx[(size_t)m1 * nx0 + m0] = (x1 - x0) * (x1 - x0);
    }
  }
  for (int n1 = 0; n1 < ny1; ++n1) {
    double y1 = coord(n1, ny1, v->py1, v->oy1);
    for (int n0 = 0; n0 < ny0; ++n0) {
      double y0 = coord(n0, ny0, v->py0, v->oy0);
      Ky[(size_t)n1 * ny0 + n0] = fresnel_kernel(y1, y0, wl, z);
      Dy[(size_t)n1 * ny0 + n0] = (y1 - y0) * (y1 - y0);
    }
  }
  /* tA = sum_m0 u0 Kx ; tB = sum_m0 u0 Kx dx^2 */
#pragma omp parallel for schedule(static)
  for (int n0 = 0; n0 < ny0; ++n0) {
    for (int m1 = 0; m1 < nx1; ++m1) {
      double complex a = 0, b = 0;
      for (int m0 = 0; m0 < nx0; ++m0) {
        double complex t = in[(size_t)n0 * nx0 + m0] * Kx[(size_t)m1 * nx0 + m0];
        a += t;
        b += t * Dx[(size_t)m1 * nx0 + m0];
      }
      tA[(size_t)n0 * nx1 + m1] = a;
      tB[(size_t)n0 * nx1 + m1] = b;
    }
  }
  const double complex C = prefactor(v);
  const double complex dC = v->no_prefactor ? 0.0 : C * (I * (2.0 * M_PI / wl) - 1.0 / z);
  const double complex dK = -I * M_PI / (wl * z * z);
#pragma omp parallel for schedule(static)
  for (int n1 = 0; n1 < ny1; ++n1) {
    for (int m1 = 0; m1 < nx1; ++m1) {
      double complex s = 0, d = 0;
      for (int n0 = 0; n0 < ny0; ++n0) {
        double complex ky = Ky[(size_t)n1 * ny0 + n0];
        s += ky * tA[(size_t)n0 * nx1 + m1];
        d += ky * (tB[(size_t)n0 * nx1 + m1] + Dy[(size_t)n1 * ny0 + n0] * tA[(size_t)n0 * nx1 + m1]);
      }
      out[(size_t)n1 * nx1 + m1] = dC * s + C * dK * d;
    }
  }
  free(Kx); free(Dx); free(Ky); free(Dy); free(tA); free(tB);
  return 0;
}

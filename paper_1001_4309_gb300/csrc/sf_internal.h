// sf_internal.h -- types shared by the host library and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "shifted_fresnel.h"
#include "sf_pass.h"

namespace sf {

// Per-axis phase polynomials in units of pi, as 64-bit fixed point (2^63 = pi).
struct AxisCoef {
  uint64_t in2, in1, in0;     // psi_in(m0)  = in2 m0^2 + in1 m0 + in0
  uint64_t out2, out1, out0;  // psi_out(m1) = out2 m1^2 + out1 m1 + out0
  uint64_t h2;                // h[d] = exp(i pi h2 d^2)   (S of Eq. 4)
  double out_scale;           // real scale of the output chirp
  int n0, n1, L;
  float2* cin;                // device, n0
  float2* cout;               // device, n1
  float2* H;                  // device, L (register order)
};

// Persistent batch kernel (sf_batch.cu)
constexpr int kBatchThreads = 256;
struct BatchGroup {
  int first_item;  // index of the group's first item within one hologram's items
  int items;       // items of the group (each `chunk` tiles, the last one possibly fewer)
  int tiles;       // row tiles of the group
  int chunk;       // tiles per item
  int L;           // FFT length
  int phase;       // 0: x pass, 1: y pass
};
struct BatchArgs {
  const PassDesc* descs;     // [n_holos][n_groups]
  const BatchGroup* groups;  // [n_groups] (x groups of views 0..V-1, then y groups)
  const int* item_group;     // [items_per_holo] group of each item within a hologram
  int* done;                 // [n_holos][n_groups] completed items
  int* next;                 // item counter
  int* error;                // set to 1 when a bounded wait expires
  const float4* tw[kNumFftLengths];  // per-stage twiddle tables, indexed by fft_length_slot(L)
  int n_holos, n_groups, n_views, items_per_holo, total_items;
  int poison_group;          // -1; a group index makes its dependency unsatisfiable (tests)
  long long spin_limit;      // sleeps before a wait gives up
};
bool batch_length_supported(int L);
int batch_tile_rows(int L);
int batch_item_tiles(int L);
size_t batch_smem_bytes();
const void* batch_kernel(PassKind kind_x);
// The batch kernel specialised to one power-of-two length (512 .. 4096) with
// every pass prunable (sf_batch_one.cu); nullptr / 0 for other lengths.
const void* batch_kernel_one(PassKind kind_x, int L);
size_t batch_smem_bytes_one(int L);

// Persistent row pass with TMA row prefetch (sf_persist.cu)
struct PersistArgs {
  int total_tiles;
  int tile_off[kMaxPassBatch + 1];  // first tile of each descriptor
  int off_cin, off_cout, off_h, off_rows, off_mbar;  // shared-memory byte offsets
  int row_bytes;                    // stride of the staged rows
  long long spin_limit;             // bounded mbarrier waits
  int* err;                         // device error word
};
bool tma_length_supported(int L);
size_t tma_layout(int L, PassKind kind, int n0max, int n1max, PersistArgs& pa);
int tma_occupancy(int L, PassKind kind, size_t smem);
cudaError_t launch_pass_tma(int L, PassKind kind, const PassBatch& b, const float4* tw, const PersistArgs& pa, int grid,
                            size_t smem, cudaStream_t s);
// Whole persistent launch of one pass batch: layout, occupancy-sized grid
// (falls back to the grid kernel when the staged tile does not fit).
cudaError_t launch_pass_persistent(int L, PassKind kind, const PassBatch& b, const float4* tw, int* err, int sms,
                                   cudaStream_t s);

// Mixed-precision row pass (sf_tc.cu)
bool tc_length_supported(int L);
int tc_rows_per_cta(int L);
size_t tc_table_words();  // DFT fragments and twiddle tables of the tensor-core pass (32-bit words)
cudaError_t launch_tc_tables(uint32_t* out, int prec, cudaStream_t s);
cudaError_t launch_hpos(int L, const float2* Hreg, float2* Hpos, cudaStream_t s);
cudaError_t launch_pass_tc(int L, int prec, PassKind kind, const PassBatch& b, int grid_x, const uint32_t* tables,
                           cudaStream_t s);

// Mixed-precision row pass on tcgen05 (sf_tcgen05.cu): lengths with the four-step
// DFT-GEMM split; passes need n0, n1 <= L / 2.  Precisions FP16TC, BF16TC and
// their hi + lo (x3) forms.
bool t5_length_supported(int L);
bool t5_precision(int prec);
size_t t5_const_bytes(int L, int prec);
void t5_build_consts(int L, int prec, void* host);
cudaError_t launch_hnat(int L, const float2* Hreg, float2* Hn, cudaStream_t s);
cudaError_t launch_pass_t5(int L, int prec, PassKind kind, const PassBatch& b, const void* consts, int* err, int sms,
                           cudaStream_t s);
// Both passes of nx views in one persistent launch: b holds the nx x passes
// then the nx y passes (same view order); sched is 1 + nx device ints that
// the launch zeroes first and uses to schedule tiles and order each view's y
// tiles after its x tiles.
cudaError_t launch_views_t5(int L, int prec, PassKind kind_x, const PassBatch& b, int nx, const void* consts, int* err,
                            int* sched, int sms, cudaStream_t s);

// host helpers shared by the entry points (defined in sf_api.cu)
int validate_view(const sf_view& v);
// smallest supported FFT length >= need (powers of two only unless allow_mixed)
int next_fft_length(int need, bool allow_mixed);
// L = 0: the smallest supported length that holds the axis's linear convolution
void axis_coefficients(const sf_view& v, int axis, AxisCoef& a, int L = 0);
void adjoint_axis_coefficients(const sf_view& v, int axis, AxisCoef& a, int L = 0);

// Autotuner (sf_tune.cu): SF_AUTOTUNE=1 selects measured choices; row_cost_ns
// is the measured time per row (ns) of a pass of length L, kind and kernel
// (0 one tile per CTA, 1 persistent), prunable or not, < 0 when not available.
int autotune_mode();
double row_cost_ns(int device, int L, PassKind kind, int impl, bool prune, int sms, cudaStream_t s);

// Inner products for d(loss)/dz of one view (see shifted_fresnel_adjoint).
struct ZGradArgs {
  const float2* g;    // [ny1][nx1] gradient w.r.t. the view
  const float2* u1;   // [ny1][nx1] view field
  const float2* G0;   // [ny0][nx0] A^H g
  const float2* G1;   // [ny0][nx0] A^H (x1 g)
  const float2* G2;   // [ny0][nx0] A^H (y1 g)
  const void* u0;     // [ny0][nx0] hologram, float32 or complex64
  int u0_complex;
  int nx0, ny0, nx1, ny1;
  double px0, py0, px1, py1, ox0, oy0, ox1, oy1;
};
cudaError_t launch_weight_xy(const float2* g, float2* xg, float2* yg, int nx1, int ny1, double px1, double py1,
                             double ox1, double oy1, cudaStream_t s);
cudaError_t launch_zgrad(const ZGradArgs& a, double2* partials, int n_partials, double* out, double c_re,
                         double c_im, double q_re, double q_im, cudaStream_t s);
cudaError_t launch_axpy(float2* y, const float2* x, size_t n, int accumulate, cudaStream_t s);
// loss (+)= sum over pixels of (|u|^2 - I)^2, g = 4 (|u|^2 - I) u (g may be null); two launches
cudaError_t launch_intensity_loss(const float2* u, const float* I, float2* g, size_t n, double* partials,
                                  int n_partials, double* loss, int accumulate, cudaStream_t s);
constexpr int kZGradBlocks = 304;
void count_launches(uint64_t n);

// launchers (one translation unit per FFT length family)
// variant: the CTA size (0 default, 1 half the rows per CTA, 2 twice; pass_rows_per_cta(L, variant) = 0
// where a variant does not exist)
cudaError_t launch_pass(int L, PassKind kind, const PassBatch& b, int grid_x, const float4* tw, cudaStream_t s,
                        int variant = 0);
cudaError_t launch_hspec(int L, const AxisCoef* axes_dev, int n_axes, const float4* tw, cudaStream_t s);
cudaError_t launch_chirps(const AxisCoef* axes_dev, int n_axes, int max_n, cudaStream_t s);
size_t twiddle_entries(int L);
void build_twiddles(int L, float4* host_table);
int pass_rows_per_cta(int L, int variant = 0);
bool fft_length_supported(int L);
int fft_length_slot(int L);  // index in kFftLengths, -1 if unsupported

}  // namespace sf

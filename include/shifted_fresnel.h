/*
 * shifted_fresnel.h -- C ABI of the GB300 (sm_103a) Shifted-Fresnel library.
 *
 * Shifted-Fresnel diffraction (Shimobaba et al., Section 2.1, Eqs. 1-5)
 * reconstructs a view u1 of a hologram u0 at distance z with its own output
 * pitch and lateral offset:
 *
 *   u1[n1][m1] = C sum_{n0,m0} u0[n0][m0] exp(i pi ((x1-x0)^2 + (y1-y0)^2) / (lambda z)),
 *   C = exp(i k z) / (i lambda z),   k = 2 pi / lambda,
 *   x0 = ox0 + (m0 - floor(nx0/2)) px0,   x1 = ox1 + (m1 - floor(nx1/2)) px1
 *   (and the same along y).
 *
 * The library evaluates it as Eq. 1 does: per axis, the input chirp of
 * Eq. 3, a zero-padded FFT convolution with the chirp kernel h of Eq. 4, and
 * the output chirp and constant of Eq. 2; the view intensity is Eq. 5.  The
 * paper's offsets O are in pixels and its index origin is -N/2; here offsets
 * are physical lengths (O = o / p) and the origin is floor(N/2).
 *
 * Conventions shared by every entry point:
 *   - Return value: SF_OK (0) on success, a negative SF_ERR_* code on failure.
 *     No exception or C++ object crosses this interface.
 *   - Arrays are row-major [rows][cols], x (m) fastest.  "complex64" is an
 *     interleaved pair of float32 (re, im), 8 bytes per element.
 *   - A plan is bound to the device it was created on.  Calls are ordered on
 *     the given stream (a cudaStream_t passed as void*; NULL = legacy default
 *     stream) and return before the GPU work finishes.
 *   - The caller owns every input and output buffer; the plan owns its
 *     workspaces, chirp vectors and kernel spectra.
 */
#ifndef SHIFTED_FRESNEL_H
#define SHIFTED_FRESNEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SF_OK 0
#define SF_ERR_INVALID_ARG (-1)      /* bad pointer, NaN/Inf, z = 0, lambda/pitch <= 0, size <= 0 ... */
#define SF_ERR_UNSUPPORTED_SIZE (-2) /* nx0 + nx1 - 1 (or ny0 + ny1 - 1) above SF_MAX_CONV_LENGTH */
#define SF_ERR_CUDA (-3)             /* a CUDA runtime call or kernel launch failed */
#define SF_ERR_OOM (-4)              /* device or host allocation failed */
#define SF_ERR_TIMEOUT (-5)          /* a bounded device-side wait gave up */
#define SF_ERR_DEVICE_MISMATCH (-6)  /* plan used while another device is current */

/* ---- view flags (sf_view.flags) ---- */
#define SF_OUT_INTENSITY 1u /* informational: intensity buffers are passed to execute */
#define SF_OUT_PHASE 2u     /* informational: phase buffers are passed to execute */
#define SF_NO_PREFACTOR 4u  /* drop the constant exp(ikz)/(i lambda z) of Eq. 2 (the paper's choice for intensity) */
#define SF_IN_COMPLEX 8u    /* the hologram is complex64 instead of float32 (same for every view of a plan) */

/* ---- precision selector ---- */
#define SF_PREC_FP32 0     /* FP32 FFT stages on CUDA cores; phases exact (64-bit fixed point) */
#define SF_PREC_FP16TC 1   /* DFT stages as FP16 tensor-core products, FP32 accumulation */
#define SF_PREC_BF16TC 2   /* same with BF16 operands */
#define SF_PREC_FP16X3TC 3 /* FP16 operands split into hi + lo parts, three products per stage */
#define SF_PREC_BF16X3TC 4 /* BF16 operands split into hi + lo parts, three products per stage */
/* Tensor-core precisions.  An axis of FFT length 2048, 1024 or 512 whose
 * input and output lengths are at most half of it (the paper's 2N padding,
 * e.g. 1024 -> 1024, 512 -> 512, 256 -> 256) runs the four-step pass on
 * tcgen05 (64 x 32, 32 x 32, 16 x 32: two DFT matrix products each way, operands in
 * shared memory, FP32 accumulators in tensor memory, one CTA per SM; on
 * FP16TC / BF16TC plans of two to eight views whose axes all share one such
 * length, execute runs both passes in one launch); other axes of length 2048
 * or 4096 run radix-16/8 stages on mma.sync (FP16TC and BF16TC only).  Every other axis, the adjoint and the
 * persistent batch kernel run in FP32.  The x3 precisions apply to the
 * tcgen05 axes only and run every other axis in FP32.  Chirps, twiddles,
 * kernel spectrum and accumulation stay FP32 (phases exact) in every
 * precision. */

/* Longest linear convolution per axis: nx0 + nx1 - 1 <= SF_MAX_CONV_LENGTH. */
#define SF_MAX_CONV_LENGTH 8192

/*
 * One view (Section 2.1): wavelength and distance z (metres, z != 0, its
 * sign is the propagation direction), hologram pitch (px0, py0), view pitch
 * (px1, py1), physical plane offsets (ox0, oy0) and (ox1, oy1), hologram
 * size nx0 x ny0 and view size nx1 x ny1.  All views of one plan share the
 * hologram size, hologram pitch and the SF_IN_COMPLEX flag.
 */
typedef struct {
  double wavelength, z;
  double px0, py0, px1, py1;
  double ox0, oy0, ox1, oy1;
  int32_t nx0, ny0, nx1, ny1;
  uint32_t flags;
} sf_view;

typedef struct sf_plan_s* sf_plan;

/*
 * shifted_fresnel_plan -- prepare n_views views of one hologram (Section 2.2,
 * steps 5-6: the chirp kernel h of Eq. 4 and its FFT are built here, once per
 * view and axis, as two 1-D spectra, and reused by every execute call).
 *
 *   out        receives the plan handle (set to NULL on failure).
 *   views      host array of n_views view descriptions (copied; not retained).
 *   n_views    1 .. 4096.
 *   precision  SF_PREC_FP32, SF_PREC_FP16TC, SF_PREC_BF16TC, SF_PREC_FP16X3TC or
 *              SF_PREC_BF16X3TC.
 *   device     CUDA device ordinal the plan is bound to (made current).
 *   stream     stream for the set-up kernels; the call synchronises it
 *              before returning.
 *
 * Allocates device memory (cudaMalloc): per view 8 * ny0 * nx1 bytes of
 * workspace plus O(nx0 + nx1 + ny0 + ny1 + L) bytes of vectors.
 * Errors: SF_ERR_INVALID_ARG, SF_ERR_UNSUPPORTED_SIZE, SF_ERR_OOM, SF_ERR_CUDA.
 */
int shifted_fresnel_plan(sf_plan* out, const sf_view* views, int n_views, int precision,
                         int device, void* stream);

/*
 * shifted_fresnel_plan_update -- give the plan's views new depths, pitches,
 * offsets, wavelength or SF_NO_PREFACTOR (the paper's interactive change of
 * view, Section 3; or a z step of an optimisation) without a new plan: the
 * chirps of Eqs. 2-3 and the kernel spectra of Eq. 4 (steps 5-6) are rebuilt
 * in place on `stream`, asynchronously (no allocation, no synchronisation).
 *
 *   views      host array of n_views descriptions (copied); view i must keep
 *              view i's nx0, ny0, nx1, ny1 and SF_IN_COMPLEX, so every FFT
 *              length and buffer stays as planned.
 *   n_views    the plan's view count.
 *   stream     stream to run on.  Work on `stream` after the call sees the
 *              new views; calls of this plan still in flight on other
 *              streams must be finished (or ordered before it) by the caller.
 *
 * Results equal those of a new plan with the same views.  On SF_ERR_CUDA the
 * plan's views are undefined until an update succeeds.
 * Errors: SF_ERR_INVALID_ARG (NULL plan or views, other view count or sizes),
 * SF_ERR_UNSUPPORTED_SIZE, SF_ERR_CUDA.
 */
int shifted_fresnel_plan_update(sf_plan plan, const sf_view* views, int n_views, void* stream);

/*
 * shifted_fresnel_execute -- reconstruct every view of the plan from one
 * hologram (Section 2.2, steps 2-10, and Eq. 5).
 *
 *   holo       hologram [ny0][nx0], float32 or (SF_IN_COMPLEX) complex64.
 *   view_out   array of n_views pointers to complex64 [ny1][nx1] views, or
 *              NULL; single entries may be NULL.
 *   intensity  array of n_views pointers to float32 [ny1][nx1] |u1|^2 images
 *              (Eq. 5), or NULL; single entries may be NULL.
 *   phase      array of n_views pointers to float32 [ny1][nx1] phase images
 *              atan2(Im u1, Re u1) in (-pi, pi], or NULL.
 *   stream     stream to run on.
 *
 * Each of holo and the output buffers may be device memory or host memory
 * (pinned or pageable).  Host buffers are staged through plan-owned device
 * buffers that the first call with a host buffer allocates.  With host
 * outputs each view's copies to the host start on a plan-owned copy stream
 * as soon as that view is done, overlapping the following views; the views'
 * x passes run in order on a plan-owned stream of the lowest priority and
 * each y pass, after its x pass, on one of the highest, and a host hologram
 * of at least 1 MiB and 256 rows is copied in two halves, the first view's
 * x pass starting on the first half (FP32 plans).  The caller's stream waits
 * for the last copy, so the caller synchronises its stream before reading
 * host outputs.  Every view needs at least one non-NULL output.
 * With device outputs on an FP16TC or BF16TC plan of two to eight views
 * whose axes all run the tcgen05 pass, both passes of every view run as one
 * launch on `stream` (each view's y pass starting once its x pass is done;
 * SF_T5_FUSED=0 keeps one launch per pass; the streams batch, below, runs
 * one such launch per hologram).
 * Otherwise, with device outputs and two or more views, the views are split
 * into two halves of about equal work run on `stream` and on a plan-owned
 * second stream (x pass then y pass each), so one half's y pass overlaps the
 * other's x pass; `stream` waits for both before the call's work is
 * complete.  SF_EXECUTE_SINGLE_STREAM=1 keeps one launch per pass on
 * `stream` (with host outputs: both passes of each view in turn, copies
 * still on the copy stream); so do profiling events set with
 * shifted_fresnel_set_profile_events when every output is device memory.
 * Implementation (FP32 passes): a one-tile-per-CTA kernel (with the plan's
 * rows per CTA), or, where the plan chose it (by default at FFT length 4096;
 * SF_PASS_IMPL or the autotuner, see shifted_fresnel_fft_length) and the
 * rows' address, stride and length are multiples of 16 bytes (FFT length
 * 256 .. 4096), a persistent kernel that prefetches the next rows with bulk
 * copies while transforming the current ones.  Complex outputs in plain
 * device memory with 16-byte aligned rows leave through tensor stores;
 * intensity, phase, managed or host-mapped outputs through plain stores
 * (the same values either way).
 * Errors: SF_ERR_INVALID_ARG, SF_ERR_DEVICE_MISMATCH, SF_ERR_OOM, SF_ERR_CUDA.
 */
int shifted_fresnel_execute(sf_plan plan, const void* holo, void* const* view_out,
                            float* const* intensity, float* const* phase, void* stream);

/*
 * shifted_fresnel_execute_batch -- reconstruct every view of the plan for
 * each of n_holos holograms (the paper's per-frame loop of Section 2.2,
 * steps 1-11, over a stream of frames) with one of two implementations:
 *
 *   persistent  ONE persistent kernel launch for the whole batch, issued as
 *               a CUDA graph (descriptor upload, counter reset, kernel).
 *               CTAs take (hologram, pass, view, row tile) items in order
 *               from a counter; a y-pass item waits for the x-pass tiles of
 *               its hologram and view, an x-pass item for hologram h waits
 *               for the y pass of hologram h - 2 (two intermediate slots per
 *               view).  The waits are bounded; if one expires the launch
 *               ends early and shifted_fresnel_batch_status reports
 *               SF_ERR_TIMEOUT.  FFT lengths up to 6144, FP32 plans only
 *               (tensor-core plans run the streams implementation).  When every pass of
 *               every view has one power-of-two length 512 .. 4096 and
 *               n0, n1 <= L / 2, a kernel specialised to that length (with
 *               the pruned network) runs instead of the general one
 *               (SF_BATCH_GENERAL=1, read when the plan's batch state is
 *               first built, keeps the general kernel).
 *   streams     execute's per-length row-pass kernels, even holograms on one
 *               plan-owned stream and odd ones on another (one intermediate
 *               slot each), joined back into `stream`; consecutive holograms
 *               overlap.  When one hologram's passes are too small to fill
 *               the GPU, chunks of up to 16 / n_views holograms share each
 *               launch (one slot per hologram of a chunk; the first call
 *               allocates the extra slots, at most 512 MiB).  The launches are captured as a CUDA graph on a
 *               plan-owned stream and the graph is replayed while calls pass
 *               the same hologram count and buffers (other calls capture
 *               anew).  Any FFT length.
 *
 * Choice: SF_BATCH_IMPL=persistent|streams forces one; with SF_AUTOTUNE=1 the
 * first call for each n_holos times both on its own buffers (blocking) and
 * later calls use the faster; otherwise the streams (faster on every
 * workload measured, launch-bound 256^2 views included).  Both compute with
 * the same row-tile code as execute, so outputs equal execute's bit for bit.
 *
 *   holos      n_holos device pointers, each a hologram as for execute.
 *   view_out   n_holos * n_views device pointers (index h * n_views + v) to
 *              complex64 [ny1][nx1] views, or NULL; entries may be NULL.
 *   intensity  same layout, float32 |u1|^2 images, or NULL.
 *   phase      same layout, float32 phase images, or NULL.
 *   stream     stream the batch is ordered on.
 * Every (hologram, view) needs at least one non-NULL output.  All buffers
 * must be device memory of the plan's device (SF_ERR_INVALID_ARG otherwise).
 * Views may have different sizes (ragged).  The persistent kernel forced on
 * a plan with an FFT length above 6144, or on a tensor-core plan, returns
 * SF_ERR_UNSUPPORTED_SIZE.
 *
 * The first call allocates per-view second intermediate slots and two
 * streams; the persistent kernel also allocates, per n_holos, descriptor
 * tables (pinned and device) and its graph.  Calls return after launching
 * and may block the host only until the persistent call two back has
 * finished.  Calls on one plan must not overlap with other calls on another
 * stream.  Testing aids read when the persistent graph is built:
 * SF_BATCH_SPIN_LIMIT (sleeps before a wait gives up, default 4194304) and
 * SF_BATCH_POISON_GROUP (an item group whose dependency is made
 * unsatisfiable).
 * Errors: SF_ERR_INVALID_ARG, SF_ERR_UNSUPPORTED_SIZE, SF_ERR_OOM, SF_ERR_CUDA.
 */
int shifted_fresnel_execute_batch(sf_plan plan, const void* const* holos, int n_holos, void* const* view_out,
                                  float* const* intensity, float* const* phase, void* stream);

/*
 * shifted_fresnel_batch_status -- synchronise `stream` and report whether a
 * bounded device-side wait of an earlier launch on this plan expired
 * (SF_ERR_TIMEOUT, after which the flag is cleared) or not (SF_OK).  It
 * covers the persistent batch kernel and the persistent row pass that
 * execute uses for 16-byte aligned rows (whose copy waits are bounded too).
 */
int shifted_fresnel_batch_status(sf_plan plan, void* stream);

/*
 * shifted_fresnel_adjoint -- back-propagate view gradients to the hologram
 * plane, and optionally differentiate with respect to each view's z.
 *
 * The forward map of view v is the linear operator A_v of Eqs. 1-4
 * (Section 2.1).  With g_v the gradient of a real loss with respect to the
 * view field in the convention g = 2 dL/d(conj u1) (PyTorch's), this
 * computes
 *   grad_holo = sum_v A_v^H g_v                   (complex64 [ny0][nx0])
 *   grad_z[v] = Re sum conj(g_v) d(u1_v)/dz        (double, per view)
 * A^H of each axis is itself a Bluestein pass (conjugate chirps, kernel
 * conj(h), lengths swapped); the z-derivative uses two further adjoint
 * transforms, of x1 g and y1 g, and a recomputed view field.  The paper has
 * no adjoint; this is the conjugate transpose of its operator.
 *
 *   holo       the hologram / object field given to execute (float32 or
 *              complex64 per SF_IN_COMPLEX); required when grad_z != NULL,
 *              otherwise ignored (may be NULL).
 *   grad_view  n_views pointers to complex64 [ny1][nx1] gradients; NULL
 *              entries contribute nothing (and get grad_z = 0).
 *   grad_holo  complex64 [ny0][nx0] output (overwritten), or NULL.
 *   grad_z     n_views doubles, or NULL.  At least one of grad_holo and
 *              grad_z must be non-NULL.
 *   stream     stream to run on.
 * Any buffer may be device or host memory (host buffers are staged).  The
 * first call allocates the plan's adjoint scratch (about
 * 8 * (3 nx0 ny1 + 4 nx0 ny0 + 4 nx1 ny1) bytes); calls on one plan must
 * not overlap with each other or with execute on another stream.
 * Errors: SF_ERR_INVALID_ARG, SF_ERR_DEVICE_MISMATCH, SF_ERR_OOM, SF_ERR_CUDA.
 */
int shifted_fresnel_adjoint(sf_plan plan, const void* holo, const void* const* grad_view, void* grad_holo,
                            double* grad_z, void* stream);

/*
 * shifted_fresnel_intensity_loss -- the multi-depth intensity loss of phase
 * retrieval and the view gradients that shifted_fresnel_adjoint takes back
 * to the object: with u_v the complex views (for instance from execute) and
 * I_v measured intensities,
 *
 *   L = sum_v sum_pixels (|u_v|^2 - I_v)^2          (|u_v|^2 as in Eq. 5)
 *   g_v = 4 (|u_v|^2 - I_v) u_v  = 2 dL/d(conj u_v)
 *
 * (the conjugate-Wirtinger gradient PyTorch's complex autograd uses).
 *
 *   fields     n_views device pointers to complex64 [ny1][nx1] views.
 *   measured   n_views device pointers to float32 [ny1][nx1] intensities.
 *   grads      n_views device pointers receiving complex64 [ny1][nx1]
 *              gradients, or NULL for the loss alone.
 *   loss       device pointer to one double: the loss, written on `stream`
 *              (per view, residuals in FP32 and their squares summed in
 *              double precision in a fixed order: deterministic).
 *   stream     stream to run on.
 * Errors: SF_ERR_INVALID_ARG (NULL or host pointers), SF_ERR_OOM (first call
 * allocates a small partial-sum buffer), SF_ERR_CUDA.
 */
int shifted_fresnel_intensity_loss(sf_plan plan, void* const* fields, const float* const* measured,
                                   void* const* grads, double* loss, void* stream);

/* shifted_fresnel_destroy -- synchronise the plan's device and free everything it owns. */
int shifted_fresnel_destroy(sf_plan plan);

/* shifted_fresnel_strerror -- static description of a status code (never NULL). */
const char* shifted_fresnel_strerror(int status);

/*
 * shifted_fresnel_plan_query -- sizes the plan chose for one view.
 *   lx, ly           FFT (convolution) lengths per axis, >= n0 + n1 - 1.
 *   workspace_bytes  bytes of the view's intermediate buffer.
 * Any output pointer may be NULL.  Errors: SF_ERR_INVALID_ARG.
 */
int shifted_fresnel_plan_query(sf_plan plan, int view, int32_t* lx, int32_t* ly,
                               size_t* workspace_bytes);

/*
 * shifted_fresnel_set_profile_events -- attach timing events to a plan.
 *   events     n_events cudaEvent_t handles (as void*) created by the caller
 *              on the plan's device, or NULL with n_events = 0 to detach.
 *   n_events   0 or 3.
 * While attached, every execute call records events[0] on its stream before
 * the first x-pass launch, events[1] between the x and y passes and
 * events[2] after the last y-pass launch, so cudaEventElapsedTime gives the
 * duration of each pass.  The plan does not own the events.
 * Errors: SF_ERR_INVALID_ARG.
 */
int shifted_fresnel_set_profile_events(sf_plan plan, void* const* events, int n_events);

/*
 * shifted_fresnel_execute_static -- reconstruct one view without allocating.
 *
 * The paper has no counterpart to this entry point.  It exists for callers
 * that cannot allocate device memory while they run -- for example a plugin
 * whose host application owns every device allocation, or an acquisition
 * loop whose memory is fixed before the first frame -- and therefore cannot
 * create a plan (shifted_fresnel_plan calls cudaMalloc).
 *
 * It computes the same view as a one-view plan's shifted_fresnel_execute,
 * on the calling thread's current device, using one fixed device array of
 * SF_STATIC_SCRATCH_BYTES that the library declares at file scope (every GPU
 * that loads the library holds it until the process exits).  Nothing here
 * calls cudaMalloc, cudaFree or an allocating library routine.
 *
 *   view       one view (copied); the hologram size and flags are its own.
 *   holo       device pointer, hologram [ny0][nx0] float32 (complex64 with
 *              SF_IN_COMPLEX).
 *   view_out   device pointer to a complex64 [ny1][nx1] view, or NULL.
 *   intensity  device pointer to a float32 [ny1][nx1] |u1|^2 image, or NULL.
 *   phase      device pointer to a float32 [ny1][nx1] phase image, or NULL.
 *   stream     stream to run on.
 * At least one output must be non-NULL.  Limits: nx0 + nx1 - 1 and
 * ny0 + ny1 - 1 at most SF_STATIC_MAX_FFT_LENGTH after rounding up to the
 * FFT length, and nx1 * ny0 at most SF_STATIC_MAX_WORKSPACE_ELEMS; larger
 * views return SF_ERR_UNSUPPORTED_SIZE.  Host buffers cannot be staged
 * without allocating and return SF_ERR_INVALID_ARG.
 *
 * The array is shared by all calls on a device and keeps the last call's
 * contents; each call rewrites every part it reads, so nothing has to be
 * cleared, but calls that overlap on the GPU (other streams, other host
 * threads on the same device) race and corrupt each other's results.  The
 * first call on each device looks up the array's device address, which may
 * load the module: make that first call before any stream capture.  The
 * address is kept per device and CUDA context; after a device reset the next
 * call looks it up again (make that call outside stream capture too).
 * Errors: SF_ERR_INVALID_ARG, SF_ERR_UNSUPPORTED_SIZE, SF_ERR_DEVICE_MISMATCH,
 * SF_ERR_CUDA.
 */
#define SF_STATIC_MAX_FFT_LENGTH 2048
#define SF_STATIC_MAX_WORKSPACE_ELEMS (1u << 20) /* 8 MiB of complex64 intermediate */
#define SF_STATIC_SCRATCH_BYTES ((size_t)(8u << 20) + (size_t)(256u << 10))
int shifted_fresnel_execute_static(const sf_view* view, const void* holo, void* view_out,
                                   float* intensity, float* phase, void* stream);

/*
 * shifted_fresnel_kernel_launches -- number of CUDA kernels this library has
 * launched in this process so far (all plans, all devices).
 */
uint64_t shifted_fresnel_kernel_launches(void);

/*
 * shifted_fresnel_fft_length -- the FFT length a plan uses, without tuning,
 * for an axis whose linear convolution has `need` = n0 + n1 - 1 samples
 * (Section 2.2, step 2: zero padding so the circular convolution equals the
 * linear one; the paper pads 1024 to 2048 = 2N).  Supported lengths are the
 * powers of two 64 .. 8192 and 1536, 2304, 3072, 4608, 6144 (3 x 2^k and
 * 9 x 2^8, whose FFT network starts with a radix-24 stage); allow_mixed = 0
 * restricts the choice to powers of two.  Pure host function, no device
 * needed.  Returns the length, SF_ERR_INVALID_ARG for need < 1, or
 * SF_ERR_UNSUPPORTED_SIZE above SF_MAX_CONV_LENGTH.
 *
 * Plan-time choices (environment, read by shifted_fresnel_plan):
 *   SF_FFT_LENGTHS=pow2   powers of two only.
 *   SF_PASS_IMPL=grid|tma one-tile-per-CTA row-pass kernel everywhere, or the
 *                         persistent one for every eligible pass (default:
 *                         persistent at 4096 only); =half|double the
 *                         one-tile-per-CTA kernel with half or twice its
 *                         default rows per CTA where that variant exists
 *                         (FFT lengths 1024 .. 4096).
 *   SF_AUTOTUNE=1         measure instead: per axis the cheaper of the two
 *                         candidate lengths (next power of two, next length
 *                         with a factor 3), per (length, pass kind) the
 *                         cheapest row-pass kernel and rows per CTA, by the
 *                         time per row of a synthetic pass timed once per
 *                         device and process.
 *   SF_AUTOTUNE_CACHE=path  file the measurements are read from and appended
 *                         to (one "device L kind kernel prunable ns_per_row"
 *                         line each; kernel: 0 one tile per CTA, 1
 *                         persistent, 2 / 3 one tile per CTA with half / twice
 *                         the rows per CTA; prunable: n0, n1 <= L/2, where the
 *                         power-of-two network skips the dead half of its
 *                         first and last stage).
 * All choices compute the same convolution; results differ by rounding only.
 */
int32_t shifted_fresnel_fft_length(int32_t need, int32_t allow_mixed);

#ifdef __cplusplus
}
#endif

#endif /* SHIFTED_FRESNEL_H */

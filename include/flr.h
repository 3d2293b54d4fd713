/*
 * flr.h -- C ABI of the GB300 (sm_103a) Fast Local Regression library, libflr.so.
 *
 * Fast Local Regression (FLR) is the denoiser of arXiv 2410.11625, "Fast Local Neural
 * Regression for Low-Cost, Path Traced Lambertian Global Illumination".  For every pixel
 * k it fits, over the square window T_k of radius r, an affine model from the Q guide
 * channels (plus an implicit column of ones, Eq. matX) to the noisy RGB radiance
 * (Eq. matY) in the least-squares sense (Eqs. argmin, closed_form), with the per-window
 * normal equations obtained exactly by box-filtering the outer products x x^T and x y^T
 * (Sec. 3.2).  The model is regularised as a centred ridge: the Appendix's decomposition
 * X^T X = [[n, u_X], [u_X^T, S]], W = S/n - mu_X^T mu_X, with eps added to the diagonal
 * of W (the Appendix's additive term; its multiplicative term is zero) and the bias left
 * unpenalised.  Optionally the per-pixel models are averaged over a second window of
 * radius rc before being applied to the centre pixel's guide vector (Sec. 3.1,
 * I_k = x_k A_k).  Windows are clipped to the image.
 *
 * Conventions for every entry point:
 *   - Images are planar float32, channel-major then row-major: element (c, y, x) of a
 *     [C][H][W] image is at index (c * H + y) * W + x.  Device pointers must be 16-byte
 *     aligned; images must not overlap the output.
 *   - The caller owns every image.  A handle owns only its workspace (flag list,
 *     coefficient scratch, host-path staging), allocated by flr_create/flr_reserve or
 *     grown on first use.
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream) unless stated otherwise.  One handle must not be
 *     used on two streams at once.
 *   - Every function returns FLR_OK (0) or a negative flr_status; no exception or abort
 *     crosses the ABI.  flr_status_string() names a status.
 */
#ifndef FLR_H
#define FLR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum flr_status {
    FLR_OK = 0,
    FLR_ERR_ARG = -1,         /* a null pointer, a non-positive size, a bad parameter */
    FLR_ERR_ALIGN = -2,       /* a device pointer is not 16-byte aligned */
    FLR_ERR_CUDA = -3,        /* a CUDA runtime call failed (see flr_last_cuda_error) */
    FLR_ERR_UNSUPPORTED = -4, /* q or a radius outside what this build supports */
    FLR_ERR_NOMEM = -5,       /* a workspace allocation failed */
    FLR_ERR_TIMEOUT = -6      /* a bounded device-side wait ran out of time (reported by
                                 flr_get_stats, flr_fast_batch_status, flnr_status) */
} flr_status;

/* Largest guide count and window radii the kernels are built for. */
#define FLR_MAX_Q 8
#define FLR_MAX_RADIUS 16
#define FLR_MAX_COEF_RADIUS 16

/* flr_params.flags bits */
#define FLR_FLAG_TIMING 1u /* record CUDA events around every kernel (flr_get_kernel_times) */

typedef struct flr_params {
    int q;             /* number of guide channels Q, 1..FLR_MAX_Q (bias column implicit) */
    int radius;        /* window radius r, 0..FLR_MAX_RADIUS; window (2r+1)^2, clipped */
    int coef_radius;   /* coefficient-averaging radius rc, 0..FLR_MAX_COEF_RADIUS; 0 = off */
    float eps;         /* ridge term added to the centred covariance, >= 0 */
    float pivot_ratio; /* FP64 re-solve threshold tau: a pixel whose Cholesky pivot d_j
                          satisfies d_j <= tau * M_jj is re-solved in FP64 on the GPU.
                          <= 0 disables the re-solve. */
    unsigned flags;    /* FLR_FLAG_* bits; other bits must be 0 */
} flr_params;

typedef struct flr_stats {
    unsigned long long flagged;   /* pixels of the last call whose pivot fell below tau */
    unsigned long long resolved;  /* of those, pixels re-solved in FP64 (the rest overflowed
                                     the flag list and kept their FP32 solution) */
    unsigned long long nonfinite; /* output values (pixel x channel) of the last call that are
                                     NaN or infinite: non-finite inputs are not sanitised and
                                     propagate through every window that holds them */
} flr_stats;

typedef struct flr_handle flr_handle;

/*
 * Create a handle for the given parameters (validated here).  Allocates the small
 * device counters; image-sized workspace is allocated by flr_reserve or on first use.
 * *out receives the handle.  Errors: FLR_ERR_ARG, FLR_ERR_UNSUPPORTED, FLR_ERR_CUDA.
 */
int flr_create(const flr_params *params, flr_handle **out);

/* Free a handle and its workspace (synchronises the device first).  NULL is a no-op. */
int flr_destroy(flr_handle *h);

/*
 * Allocate the workspace for frames of up to H x W pixels now, so that later calls of
 * that size allocate nothing (needed before capturing a call in a CUDA graph).
 * Synchronous.  Errors: FLR_ERR_ARG, FLR_ERR_NOMEM.
 */
int flr_reserve(flr_handle *h, int H, int W);

/*
 * FLR forward pass on device images (Sec. 3.1-3.2, Appendix; see the file header).
 *   guide      [q][H][W]  guides X the per-pixel models are fitted on
 *   map_guide  [q][H][W]  guides z the models are applied to, or NULL to use `guide`
 *                         (the model/map split of Sec. 3.3)
 *   radiance   [3][H][W]  noisy demodulated radiance Y
 *   out        [3][H][W]  result I; must not overlap any input
 * The result of every pixel whose Cholesky pivot ratio falls below params.pivot_ratio
 * is replaced by an FP64 re-solve of its window on the GPU; flr_get_stats reports how
 * many.  Grows the workspace if the frame is larger than reserved (a synchronous
 * allocation).  Errors: FLR_ERR_ARG, FLR_ERR_ALIGN, FLR_ERR_NOMEM, FLR_ERR_CUDA.
 */
int flr_denoise(flr_handle *h, const float *guide, const float *map_guide,
                const float *radiance, float *out, int H, int W, void *stream);

/*
 * Gradient of L = <grad_out, I> through the FLR pass with the same inputs: the adjoint of
 * every step of flr_denoise (the paper trains through FLR by backpropagation, Sec. 3.2,
 * and builds FLNR on a differentiable FLR, Sec. 3.3).  The window moments and per-pixel
 * solves are recomputed from the inputs, not stored by the forward call.
 *   grad_out        [3][H][W]  dL/dI
 *   grad_guide      [q][H][W]  dL/d guide; with map_guide == NULL it includes the path
 *                              through the applied guide
 *   grad_map_guide  [q][H][W]  dL/d map_guide, or NULL (ignored when map_guide is NULL)
 *   grad_radiance   [3][H][W]  dL/d radiance
 *   grad_eps        device pointer to one double receiving dL/d eps, or NULL
 * All pointers are device pointers; outputs must not overlap inputs.  Pixels flagged by the
 * pivot test get FP64 models, as in flr_denoise; the adjoint solve itself is FP32.  The
 * first call at a frame size allocates the handle's backward workspace: 9 (Q+1) + 2 NCH
 * floats per pixel for Q = FLR_MAX_Q, NCH = Q + 3 + Q(Q+1)/2 + 3Q (223 floats, 892 B).
 * Errors: FLR_ERR_ARG, FLR_ERR_ALIGN, FLR_ERR_NOMEM, FLR_ERR_CUDA.
 */
int flr_backward(flr_handle *h, const float *guide, const float *map_guide, const float *radiance,
                 const float *grad_out, float *grad_guide, float *grad_map_guide, float *grad_radiance,
                 double *grad_eps, int H, int W, void *stream);

/*
 * The same pass on HOST images: copies guide, map_guide (if not NULL) and radiance to
 * handle-owned device staging, runs the FLR kernels, copies the result back to `out`, and
 * waits.  Frames of 540 rows or more are processed in row bands of about 360 rows (at
 * most 8; three at 1080 rows) so that the copies overlap the kernels: band k + 1 is copied in on a handle-owned stream while
 * band k's kernels run on `stream`, and band k's output is copied out on a second handle-
 * owned stream while band k + 1 runs (the copies start after the work already queued on
 * `stream`).  The bands choose their own segment heights and sample the frame reference
 * from the first band, so the result equals flr_denoise's to FP32 rounding (not bit for
 * bit; both meet the same bar against an FP64 solve); smaller frames run exactly
 * flr_denoise.  Page-locked host memory gives asynchronous copies; pageable memory works
 * but is slower.  Errors as flr_denoise.
 */
int flr_denoise_host(flr_handle *h, const float *guide, const float *map_guide,
                     const float *radiance, float *out, int H, int W, void *stream);

/*
 * The same pass on HOST images of a stream of frames (a renderer's frame sequence),
 * without waiting: enqueues the copy of guide, map_guide (if not NULL) and radiance to a
 * handle-owned device staging slot on a handle-owned copy-in stream, flr_denoise's kernels
 * on `stream`, and the copy of the result to `out` on a handle-owned copy-out stream, then
 * returns.  Consecutive calls on one handle alternate between two staging slots, so frame
 * i + 1 is copied in while frame i's kernels run and frame i's result is copied out while
 * frame i + 1's kernels run; the result equals flr_denoise's bit for bit.  The kernels also
 * follow the work already queued on `stream`; the input copies do not wait for it.
 * Ownership: the host buffers stay the caller's, must not be written (inputs) or read
 * (out) until flr_host_wait(h) returns, and should be page-locked (cudaHostAlloc or
 * cudaHostRegister): with pageable memory the copies are correct but do not overlap.  A
 * frame larger than its slot first waits for the frames in flight, then grows the slot
 * ((2 Q + 6) floats per pixel per slot).  Errors as flr_denoise; after an error, call
 * flr_host_wait before queueing further frames.
 */
int flr_denoise_host_async(flr_handle *h, const float *guide, const float *map_guide,
                           const float *radiance, float *out, int H, int W, void *stream);

/*
 * Blocks until every frame queued by flr_denoise_host_async on this handle is in host
 * memory (returns at once when none is queued).  flr_denoise_host calls it first.  A
 * kernel's expired bounded wait is reported by flr_get_stats, as for flr_denoise.
 * Errors: FLR_ERR_ARG, FLR_ERR_CUDA.
 */
int flr_host_wait(flr_handle *h);

/* Most row bands flr_denoise_host cuts a frame into. */
#define FLR_HOST_MAX_BANDS 8

/*
 * The row bands flr_denoise_host uses for a frame of H rows (host arithmetic only, no
 * device call; not a paper operation: it exposes the host path's plan to tests).  Returns
 * K >= 1 and fills K + 1 entries of each array: band k computes the models of rows
 * [c[k], c[k+1]), copies in input rows [in_end[k], in_end[k+1]) (so rows below
 * in_end[k+1] = min(H, c[k+1] + radius) are on the device when it runs) and writes output
 * rows [out_lo[k], out_lo[k+1]) (c[k] - coef_radius inside the frame).  The arrays need
 * FLR_HOST_MAX_BANDS + 1 entries.  Errors: FLR_ERR_ARG.
 */
int flr_host_band_plan(int H, int radius, int coef_radius, int *c, int *in_end, int *out_lo);

/*
 * Statistics of the last flr_denoise on this handle.  Waits for that call's stream.
 * Returns FLR_ERR_TIMEOUT (after filling *out) if a kernel of an earlier call on this
 * handle stopped because one of its bounded device waits (1 s) ran out; the flag is then
 * cleared.  Errors: FLR_ERR_ARG, FLR_ERR_CUDA.
 */
int flr_get_stats(flr_handle *h, flr_stats *out);

/* Per-kernel launch counts and (with FLR_FLAG_TIMING) summed CUDA-event durations. */
typedef struct flr_kernel_times {
    double fwd_ms, fp64_ms, apply_ms;           /* summed durations; 0 without timing */
    unsigned long long fwd_n, fp64_n, apply_n;  /* kernels launched */
} flr_kernel_times;

/*
 * Launch counts and, when the handle was created with FLR_FLAG_TIMING, the summed
 * durations of the forward, FP64 re-solve and apply kernels over the calls since the
 * last reset, each measured by CUDA events recorded on the call's stream directly before
 * and after the kernel.  Waits for the last timed call.  reset != 0 zeroes the sums
 * afterwards.  Not a paper operation: instrumentation for roofline measurement.
 * Errors: FLR_ERR_ARG, FLR_ERR_CUDA.
 */
int flr_get_kernel_times(flr_handle *h, flr_kernel_times *out, int reset);

/*
 * FLR pass without any device allocation, for callers that cannot call cudaMalloc: code
 * running inside a custom device allocator or a memory-pool callback, a host application
 * that forbids allocations after start-up, or a plugin that only receives the buffers its
 * host hands it.  The paper has no counterpart: this is an integration variant of
 * flr_denoise, with the same arguments except that the parameters replace the handle.
 *
 * The workspace (coefficient planes, flag list, flag counter, reference shift) is one
 * file-scope __device__ array sized for FLR_NOALLOC_MAX_PIXELS pixels; every GPU that loads
 * the library holds it until the process exits.  Frames larger than that are rejected with
 * FLR_ERR_UNSUPPORTED.  The first call on a device looks up the array's device address and
 * configures the kernels (no allocation); make that first call before capturing any stream.
 * All calls on a device share the array and leave the last call's contents in it: calls
 * that overlap on the GPU race, so the caller must serialise them.  No statistics are kept
 * (flr_get_stats needs a handle), and a bounded device wait that runs out (a copy that has
 * not completed after 1 s) is not reported: the kernels stop and leave part of out
 * unwritten, but the call has returned before they run and keeps no status to query.
 * Errors: FLR_ERR_ARG, FLR_ERR_ALIGN, FLR_ERR_UNSUPPORTED, FLR_ERR_CUDA.
 */
#define FLR_NOALLOC_MAX_PIXELS (256 * 256)
int flr_denoise_noalloc(const flr_params *params, const float *guide, const float *map_guide,
                        const float *radiance, float *out, int H, int W, void *stream);

/*
 * Fast FLR: the paper's own implementation of the method (Sec. 3.2, "Fast Local
 * Regression"), and its joint denoising and upsampling (Sec. 3.2.1).  The outer products
 * are summed over factor x factor blocks of the input grid (a strided box filter), blurred
 * over the block grid by a separable Gaussian, the centred ridge model of flr_denoise is
 * solved once per block, and the block models are bilinearly interpolated to every output
 * pixel and applied to the map guide there.  Equivalent to weighted least squares with
 * each pixel weighted by the Gaussian weight of its block (Sec. 3.2's WLS equation).
 */
typedef struct flr_fast_params {
    int q;             /* guide channels, 1..FLR_MAX_Q */
    int factor;        /* input pixels per block side: 2, 4 or 8 (the paper: 8) */
    int scale;         /* output pixels per input pixel side, 1..8: 1 = fast FLR; 2, 4 =
                          joint denoising and upsampling (model guide and radiance at the
                          input resolution, map guide and output at scale x it) */
    float sigma;       /* Gaussian standard deviation in blocks (the paper: sigma / 8, i.e.
                          1.25 for Fig. 3's sigma = 10 pixels) */
    int taps;          /* Gaussian half-width in blocks, 0..8 */
    float eps;         /* ridge term, >= 0; with FLR_FAST_APPENDIX the additive term */
    float pivot_ratio; /* FP64 re-solve threshold per block (as flr_params); <= 0: off */
    unsigned flags;    /* 0 or FLR_FAST_APPENDIX */
    float eps_mul;     /* with FLR_FAST_APPENDIX the multiplicative term, in [0, 1]; else 0 */
} flr_fast_params;

/*
 * flr_fast_params.flags: solve each block with the Appendix's regularised normalised
 * system instead of the centred ridge.  With the window's guide means mu (absolute),
 * centred covariance W = S/n - mu^T mu and D = X^T Y / n - mu^T mu_Y:
 *   W^ = S/n + eps_mul diag(mu^T mu) + eps I - (1 - eps_mul) mu^T mu,
 *   sigma^ = sqrt(diag W^), C^ = W^ / (sigma^ sigma^^T), B^ = D / sigma^,
 *   A^ = (C^ + eps I)^-1 B^,  y = ((x - mu) / sigma^) A^ + mu_Y
 * (eps used in both places, as printed).  The kernel solves the equivalent
 * a = (W^ + eps diag(W^))^-1 D in one Cholesky, without the divisions by sigma^.
 */
#define FLR_FAST_APPENDIX 1u

typedef struct flr_fast_handle flr_fast_handle;

/* Create / destroy a fast-FLR handle.  Errors: FLR_ERR_ARG, FLR_ERR_UNSUPPORTED, FLR_ERR_NOMEM. */
int flr_fast_create(const flr_fast_params *params, flr_fast_handle **out);
int flr_fast_destroy(flr_fast_handle *h);

/*
 * Fast FLR on device images.
 *   guide      [q][Hi][Wi]            model guides (input resolution)
 *   radiance   [3][Hi][Wi]            noisy radiance (input resolution)
 *   map_guide  [q][Hi*s][Wi*s]        guides the models are applied to; NULL = guide (s = 1)
 *   out        [3][Hi*s][Wi*s]        result
 * Block (i, j) covers input rows [i F, i F + F) and columns [j F, j F + F) (clipped) and has
 * its centre at output coordinate ((i + 1/2) F s - 1/2, (j + 1/2) F s - 1/2); outputs
 * beyond the outermost centres use the edge models.  The per-block workspace
 * (2 NCH + 3 (q+1) floats per block) is allocated on first use.
 * Errors: FLR_ERR_ARG, FLR_ERR_ALIGN, FLR_ERR_NOMEM, FLR_ERR_CUDA.
 */
int flr_fast_denoise(flr_fast_handle *h, const float *guide, const float *map_guide,
                     const float *radiance, float *out, int Hi, int Wi, void *stream);

/* Blocks of the last call whose pivot fell below the threshold (re-solved in FP64); the
 * fast path does not count non-finite outputs (nonfinite = 0). */
int flr_fast_get_stats(flr_fast_handle *h, flr_stats *out);

/*
 * Gradients of L = <grad_out, fast FLR output> with respect to the handle's parameters, for
 * learning them by backpropagation (Sec. 3.2: the Gaussian's width and the regularisation
 * terms are learned): grad (device, 3 doubles, overwritten) = dL/dsigma (sigma in block
 * units, as flr_fast_params.sigma), dL/deps (the ridge term, or the Appendix's additive
 * term with FLR_FAST_APPENDIX) and dL/deps_mul (the Appendix's multiplicative term; 0
 * without the flag).  Inputs as flr_fast_denoise, grad_out [3][Ho][Wo] device float32.
 * Forward-mode tangents: the blur of the block moments with dw/dsigma gives dS/dsigma; each
 * block's model tangent solves M da = dD - dM a with the block's Cholesky factor
 * (db = dmu_y - da^T mu - a^T dmu); each tangent model is applied like the model and reduced
 * against grad_out in double, in a fixed order (deterministic).  Blocks whose pivot ratio is
 * below pivot_ratio use the FP32 factor here.  Runs on `stream` without waiting.
 * Errors: FLR_ERR_ARG, FLR_ERR_ALIGN (grad_out and images 16-byte, grad 8-byte aligned),
 * FLR_ERR_NOMEM, FLR_ERR_CUDA.
 */
int flr_fast_param_grad(flr_fast_handle *h, const float *guide, const float *map_guide, const float *radiance,
                        const float *grad_out, double *grad, int Hi, int Wi, void *stream);

/* One frame of a batch: device pointers as in flr_denoise / flr_fast_denoise. */
typedef struct flr_frame {
    const float *guide;     /* [q][H][W] (fast path: input resolution) */
    const float *map_guide; /* [q][H*s][W*s], or NULL to use the guide (s = 1) */
    const float *radiance;  /* [3][H][W] */
    float *out;             /* [3][H*s][W*s] */
    int H, W;               /* input size */
} flr_frame;

#define FLR_MAX_BATCH 16
#define FLR_BATCH_TIMEOUT 1 /* device status word value after a barrier wait ran out */

/*
 * The per-pixel FLR pass (flr_denoise, Sec. 3.1-3.2) over n frames of any sizes, in order, on
 * one stream: the serving form of a frame sequence (the paper's real-time setting, Sec. 4).
 * Errors as flr_denoise, for the first frame that fails.
 */
int flr_denoise_batch(flr_handle *h, int n, const flr_frame *frames, void *stream);

/*
 * Batched fast FLR / joint denoising and upsampling (Sec. 3.2, 3.2.1) of n <= FLR_MAX_BATCH
 * frames of mixed sizes in ONE persistent cooperative kernel launch: every stage of every
 * frame is a work item of the same kernel, with a grid barrier between the four stages.
 * The frame table is passed by value in the kernel parameters, so the call can be captured
 * in a CUDA graph once flr_fast_reserve_batch has allocated the workspace for these sizes
 * (after that the call allocates nothing).  Supported for q in {1, 4, 8} and every factor.
 * Each barrier wait is bounded (2 s): if it runs out, the kernel records FLR_BATCH_TIMEOUT
 * and finishes without hanging; flr_fast_batch_status reports it.
 * Errors: FLR_ERR_ARG, FLR_ERR_ALIGN, FLR_ERR_UNSUPPORTED, FLR_ERR_NOMEM, FLR_ERR_CUDA.
 */
int flr_fast_reserve_batch(flr_fast_handle *h, int n, const flr_frame *frames);
int flr_fast_denoise_batch(flr_fast_handle *h, int n, const flr_frame *frames, void *stream);

/* Waits for the last batch and returns FLR_OK, or FLR_ERR_TIMEOUT if a barrier ran out. */
int flr_fast_batch_status(flr_fast_handle *h);

/*
 * Self-test of the bounded device wait: launches `ctas` CTAs on a grid barrier that expects
 * one more CTA than exists, so every wait runs out after timeout_ns; *status receives the
 * device status word (FLR_BATCH_TIMEOUT on success of the test).  No fault is involved.
 * Not a paper operation.  Errors: FLR_ERR_ARG, FLR_ERR_NOMEM, FLR_ERR_CUDA.
 */
int flr_barrier_selftest(int ctas, unsigned long long timeout_ns, int *status);

/*
 * Self-test of the bounded mbarrier wait used by the TMA-staged and tensor-core kernels
 * (every such wait gives up after a time limit and sets a status word instead of hanging):
 * `ctas` CTAs each wait on an mbarrier whose phase never completes (one of two expected
 * arrivals) and on one that does.  *status receives bit 0 if the first wait ran out (the
 * expected result) and bit 1 if the second one did (a failure); so 1 is a pass.  No fault is
 * involved.  Not a paper operation.  Errors: FLR_ERR_ARG, FLR_ERR_NOMEM, FLR_ERR_CUDA.
 */
int flr_mbarrier_selftest(int ctas, unsigned long long timeout_ns, int *status);

/*
 * FLNR (Sec. 3.3, "Fast Local Neural Regression"): a U-Net maps the guides and the noisy
 * radiance, concatenated channel-wise (11 channels: Q = 8 guides, then RGB), to enhanced
 * guide channels that FLR then uses (Fig. 2): 8 (one set, used both to fit and to apply the
 * models), or 16 = 2Q, the two sets of Sec. 3.3 (channels 0-7 the model guides X'_model,
 * 8-15 the map guides X'_map, for FLR's map_guide).  Layers, in order (3x3 convolutions with zero
 * padding 1, stride 1 unless stated; ReLU unless stated):
 *   in0 3x3 11->16, in1 1x1 16->16 | e1a 3x3 16->32, e1b 3x3 32->32 stride 2 |
 *   e2a 3x3 32->64, e2b 3x3 64->64 stride 2 | up2 ++ e1b: d1a 3x3 96->32, d1b 3x3 32->32 |
 *   up2 ++ in1: d0a 3x3 48->16, d0b 3x3 16->16 | o0 3x3 16->16, o1 1x1 16->nout + sigmoid.
 * Each encoder block downsamples with its second convolution (stride 2, Sec. 3.3): output
 * (i, j) reads inputs (2i - 1 .. 2i + 1, 2j - 1 .. 2j + 1).
 * The network reads the radiance channels as log(1 + max(Y, 0)) (fireflies stay bounded).
 * BF16 convolutions on the fifth-generation tensor cores (tcgen05 UMMA, FP32 accumulators in
 * tensor memory) for the forward pass, the input gradients and the weight gradients; FP32
 * master weights.  Parameters are one flat float array: per layer its weights
 * [Cout][Cin][k][k] then its biases [Cout], layers in the order above
 * (flnr_param_count(nout) floats).
 */
typedef struct flnr_net flnr_net;

/* Number of parameters (floats) of the network with nout = 8 or 16 outputs; 0 otherwise. */
size_t flnr_param_count(int nout);

/* Create a network with nout = 8 or 16 outputs whose activation buffers hold up to
 * max_pixels = N*H*W input pixels.  Errors: FLR_ERR_ARG, FLR_ERR_NOMEM. */
int flnr_create(int max_pixels, int nout, flnr_net **out);
int flnr_destroy(flnr_net *net);

/* Copy the master weights from / to host memory (count = flnr_param_count(nout)); synchronous.
 * flnr_set_weights also clears the Adam moments (a new model starts a new optimisation). */
int flnr_set_weights(flnr_net *net, const float *host, size_t count);
int flnr_get_weights(flnr_net *net, float *host, size_t count);

/* The optimiser state, for checkpoints: the master weights, then Adam's first and second
 * moments, each flnr_param_count(nout) floats (count = 3 * flnr_param_count(nout), host
 * memory); synchronous.  flnr_set_state restores all three exactly and refreshes the
 * bfloat16 weight copies, so training resumed from a saved state continues as it would have
 * without the interruption (given the same step count, learning rate and data).  The paper
 * has no counterpart: checkpointing is part of training the network it describes (Sec. 3.3).
 * Errors: FLR_ERR_ARG (count), FLR_ERR_CUDA. */
int flnr_get_state(flnr_net *net, float *host, size_t count);
int flnr_set_state(flnr_net *net, const float *host, size_t count);

/*
 * Forward pass on N images: in [N][11][H][W] planar float32 (device), guide_out
 * [N][nout][H][W] planar float32 (device; NULL keeps the result only inside the network).
 * H and W multiples of 4.  Keeps the activations for flnr_guide_backward.
 * Errors: FLR_ERR_ARG, FLR_ERR_UNSUPPORTED (more than max_pixels), FLR_ERR_CUDA.
 */
int flnr_guide_forward(flnr_net *net, const float *in, float *guide_out, int N, int H, int W, void *stream);

/*
 * One layer of the network by itself, with the network's current weights: the kernels
 * flnr_guide_forward and flnr_guide_backward use for that layer (Sec. 3.3), so that each
 * can be checked on its own.  (flnr_guide_forward runs in0 with in1, and o0 with o1, as
 * one fused pass each; the products and their order are those of the separate layers.)
 * layer = 0..11 in the order above; (N, H, W) is the layer's input size.  Tensors are
 * device NHWC bfloat16 (raw 16-bit patterns) with channel counts padded to multiples of
 * 16: CinP = 16 * ceil(Cin / 16), CoutP likewise; the padding channels of the outputs are
 * written (as zero where the padded weights are zero).  The output size (Ho, Wo) is
 * (H, W), or (H/2, W/2) for the stride-2 layers 3 and 5 (which need H and W even).
 *   FLNR_OP_FORWARD  a = x [N][H][W][CinP]; out = y [N][Ho][Wo][CoutP] = bf16(ReLU(conv(x) + b)),
 *                    or, for layer 11, float32 planar [N][nout][H][W] = sigmoid(conv(x) + b).
 *                    Layers 6 and 8 with b != NULL: a = the half-resolution decoder input
 *                    [N][H/2][W/2][64 or 32] and b = the skip [N][H][W][32 or 16]; the
 *                    result is the convolution of their concatenation (nearest 2x
 *                    upsampling of a, then b), which the kernel never forms: each output
 *                    parity class reads a and the skip's parity planes directly, as the
 *                    network does (H and W even).
 *   FLNR_OP_DGRAD    a = dz [N][Ho][Wo][CoutP] (gradient w.r.t. the layer's pre-activation);
 *                    mask = [N][H][W][CinP] or NULL; out = dx [N][H][W][CinP] =
 *                    bf16((mask > 0) * transposed convolution of dz)
 *   FLNR_OP_WGRAD    a = x [N][H][W][CinP], b = dz [N][Ho][Wo][CoutP]; adds dL/dW and dL/db
 *                    of the layer into the gradient buffer (flnr_get_grads / flnr_zero_grads)
 * For layers 3 and 5 the two gradient ops first spread dz onto the input grid (zeros at odd
 * rows and columns) in the network's scratch, which must hold N*H*W*CoutP values
 * (N*H*W*CoutP <= 48 * max_pixels, else FLR_ERR_UNSUPPORTED).
 * Runs on `stream` without waiting.  Errors: FLR_ERR_ARG, FLR_ERR_UNSUPPORTED, FLR_ERR_CUDA.
 */
/*
 * Waits for the device and reports whether a tensor-core kernel of this network ran out of
 * time waiting for its own MMAs (each wait is bounded at 1 s; the kernel then stops and frees
 * its tensor memory instead of hanging).  Returns FLR_OK or FLR_ERR_TIMEOUT (and clears the
 * flag); FLR_ERR_ARG, FLR_ERR_CUDA.
 */
int flnr_status(flnr_net *net);

#define FLNR_OP_FORWARD 0
#define FLNR_OP_DGRAD 1
#define FLNR_OP_WGRAD 2
int flnr_layer(flnr_net *net, int layer, int op, const void *a, const void *b, const void *mask, void *out,
               int N, int H, int W, void *stream);

/*
 * Backward pass of the last forward (Sec. 3.3's network trained end to end through FLR):
 * grad_out [N][nout][H][W] = dL/d(enhanced guides), planar float32 (device).  ACCUMULATES the
 * parameter gradients (flnr_zero_grads clears them).  grad_in (device, may be NULL)
 * receives dL/d(in), [N][11][H][W] planar float32, overwritten: the guide channels'
 * gradients, and for the radiance channels the gradient through log(1 + max(Y, 0)), i.e.
 * times 1 / (1 + Y) for Y > 0 and 0 for Y <= 0 (evaluated from the stored bfloat16 input).
 * Values carry the bfloat16 storage of the backward pass.  Runs on `stream`.
 * Errors: FLR_ERR_ARG (no forward yet), FLR_ERR_CUDA.
 */
int flnr_guide_backward(flnr_net *net, const float *grad_out, float *grad_in, void *stream);
int flnr_zero_grads(flnr_net *net, void *stream);
int flnr_get_grads(flnr_net *net, float *host, size_t count);

/* One Adam step on the FP32 master weights (step >= 1), then the BF16 copies are refreshed. */
int flnr_adam_step(flnr_net *net, float lr, float beta1, float beta2, float eps, int step, void *stream);

/*
 * Mean absolute error of pred against ref (count floats, device): *loss (device float)
 * receives it and grad (device) its gradient sign(pred - ref) / count.
 */
int flnr_l1_loss(const float *pred, const float *ref, float *grad, float *loss, size_t count, void *stream);

/*
 * SMAPE of pred against ref, the loss Sec. 3.3 trains FLNR on (count floats, device):
 * *loss (device float) receives mean |p - r| / (|p| + |r| + eps) and grad (device) its
 * gradient (sign(p - r) / D - |p - r| sign(p) / D^2) / count, D = |p| + |r| + eps (sign(0) = 0).
 * Errors: FLR_ERR_ARG (eps <= 0), FLR_ERR_CUDA.
 */
int flnr_smape_loss(const float *pred, const float *ref, float *grad, float *loss, size_t count, float eps,
                    void *stream);

/*
 * Measured FP32 FMA throughput of the current device, for the roofline of the per-pixel FLR
 * path, which is bound by the FP32 ALUs (not a paper operation).  Runs `iters` x 16 rounds of
 * 8 independent FMA chains in 4 x 256 threads per SM, four times, and reports the fastest of
 * the last three runs: *ms its duration (CUDA events) and *tflops = flops / time, one FMA
 * counting 2 flops.  Synchronous; allocates and frees one small buffer.
 * Errors: FLR_ERR_ARG, FLR_ERR_NOMEM, FLR_ERR_CUDA.
 */
int flr_fp32_fma_peak(int iters, double *tflops, double *ms);

/* Human-readable name of a status code (static storage). */
const char *flr_status_string(int status);

/* Message of the last CUDA error seen by this library on the calling thread. */
const char *flr_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FLR_H */

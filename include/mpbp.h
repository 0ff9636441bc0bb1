/*
 * mpbp.h -- C ABI of the GB300 multi-peak Bragg ptychography (MPBP) library.
 *
 * The library evaluates, on one GPU, the loss and gradient that the paper's
 * reconstruction repeats every iteration (Kandel et al., arXiv 2312.14907):
 *
 *   objects   O_m(r) = alpha_m rho(r) exp(i phi_m(r)),
 *             phi_m(r) = phase_scale * sum_c G_{m,c} u_c(r)            (Eq. 1, Eq. 3)
 *   model     I_{m,j} = | F diag(P_m) S_j O_m |^2 + b_{m,j}            (Eq. 2)
 *   loss      f = 1/2 sum_{m,j,q} ( sqrt(I_{m,j}(q)) - sqrt(y_{m,j}(q)) )^2  (Eq. 4)
 *   gradient  df/drho, df/du_c, df/dalpha_m of that loss (the minibatch sums of
 *             Eq. 11 when a frame subset is given)
 *
 * in the thin-membrane form of Eq. 2 (R = identity).  F is the unnormalised
 * 2-D DFT with kernel exp(-2 pi i q.k / M) and DC at index [0][0]; S_j takes the
 * M x M patch whose top-left pixel is scan[j], reading 0 outside the grid.
 *
 * Conventions for every entry point:
 *   - Arrays are row-major and C-contiguous.  Complex values are interleaved
 *     float pairs (re, im).  A "frame" is one (peak m, scan position j) pair,
 *     numbered f = m * nscan + j; frame-indexed arrays are [npeaks][nscan][M][M].
 *   - Array arguments marked "dev" are device pointers owned by the caller and
 *     must stay valid until the stream work that uses them has finished.
 *     Arguments marked "host" are read before the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls only enqueue work on it; none synchronises, except
 *     mpbp_sync_status, mpbp_loss_grad_host and mpbp_create/mpbp_destroy.
 *   - Argument errors are detected on the host and returned before anything is
 *     enqueued.  Errors found on the device (a frame index out of range, a
 *     non-finite loss) are latched in the context and reported by
 *     mpbp_sync_status.  No C++ exception crosses this boundary.
 *   - There is no CPU fallback: without a usable GPU, mpbp_create fails with
 *     MPBP_ERR_CUDA.
 */
#ifndef MPBP_H_
#define MPBP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpbp_ctx mpbp_ctx;

typedef enum {
  MPBP_OK = 0,
  MPBP_ERR_INVALID_ARG = 1,  /* a pointer, size or value is not allowed       */
  MPBP_ERR_UNSUPPORTED = 2,  /* valid problem the kernels do not cover (M)   */
  MPBP_ERR_CUDA = 3,         /* a CUDA runtime call failed                   */
  MPBP_ERR_NONFINITE = 4,    /* the loss came out NaN or infinite            */
  MPBP_ERR_TIMEOUT = 5,      /* a bounded wait on the GPU ran out (tile copies,
                                tensor-core MMAs, grid barriers)             */
  MPBP_ERR_BOUNDS = 6,       /* a frame index outside [0, npeaks*nscan)      */
  MPBP_ERR_OOM = 7,          /* device allocation failed                     */
  MPBP_ERR_NO_DATA = 8       /* probe or measured data not set yet           */
} mpbp_status;

/* Geometry of one problem (Sec. 3: the variables U, chi, alpha and the
 * measurements y_{hk,j}).  Copied by mpbp_create; the caller may free it. */
typedef struct {
  int32_t n1, n2;          /* object grid rows, columns (>= 1)                  */
  int32_t ncomp;           /* displacement components C: 1, 2 or 3             */
  int32_t npeaks;          /* Bragg peaks D: 1..16                              */
  int32_t m;               /* frame and probe side M: 8, 16, 32, 64 or 128      */
  int32_t nscan;           /* scan positions J per peak (>= 1)                  */
  const double *G;         /* host [npeaks][ncomp] scattering vectors G_m       */
  const int32_t *scan;     /* host [nscan][2] top-left (row, col) of frame j;
                              any value, pixels outside the grid read as 0     */
  int32_t probe_per_peak;  /* 0: one probe [M][M] for all peaks; 1: [D][M][M]  */
  double phase_scale;      /* phi = phase_scale * G.u; 2*pi gives Eq. 1        */
} mpbp_problem;

/* Lagged-Armijo gradient descent (the update step of Alg. 1 with plain
 * gradient descent in place of Adam).  Weights scale each block's step. */
typedef struct {
  double c_armijo;         /* sufficient-decrease constant, e.g. 1e-4          */
  double grow;             /* step growth after an accepted step, e.g. 1.25    */
  double shrink;           /* step shrink after a rejected step, e.g. 0.5      */
  double t0;               /* first step length                                */
  double w_rho, w_u, w_alpha;
} mpbp_step_params;

/* Device-resident optimizer state; written by mpbp_step_init, advanced by
 * mpbp_step, readable by copying it back. */
typedef struct {
  double f_prev;           /* loss at the last accepted iterate                */
  double gn2_prev;         /* sum_b w_b |g_b|^2 there (alpha_0 excluded)       */
  double t;                /* step length of the pending trial                 */
  double f_last;           /* loss evaluated by the last mpbp_step             */
  int32_t k;               /* mpbp_step calls so far                           */
  int32_t accepted;        /* 1 if the last call accepted its iterate          */
  int32_t n_accept, n_reject;
  double c_armijo, grow, shrink, w_rho, w_u, w_alpha;
} mpbp_step_state;

typedef struct {
  int64_t workspace_bytes; /* device memory owned by the context               */
  int32_t frames_grid;     /* blocks of the fused frame kernel                 */
  int32_t frames_block;    /* threads per block of the fused frame kernel      */
  int32_t frames_smem;     /* dynamic shared memory per block (bytes)          */
  int32_t blocks_per_sm;   /* resident blocks per SM the schedule assumes      */
  int32_t num_sms;
  int32_t launches_loss_grad; /* kernels + memsets enqueued by mpbp_loss_grad  */
  int32_t launches_step;      /* kernels + memsets enqueued by mpbp_step       */
  int32_t precision;          /* MPBP_PRECISION_* of the gradient evaluations */
  int32_t tile_copies;        /* FFT kernels that take their inputs by TMA tile and
                                 bulk copies: bit 0 the gradient kernel, bit 1 the
                                 forward kernel (none when a row of O is not a
                                 multiple of 16 bytes, i.e. odd n2: cp.async)  */
  int32_t fft_schedule;       /* MPBP_FFT_* in use (frame side 128)            */
  int32_t deterministic;      /* 1: the gradient sums are bitwise reproducible
                                 (mpbp_set_deterministic)                     */
} mpbp_info;

/* How the 128-point lines of the frame side M = 128 are split over the four
 * threads that hold one (mpbp_set_fft_schedule). */
enum {
  MPBP_FFT_SHUFFLE = 0,   /* 32-point FFTs in registers and the last two radix-2
                             stages across the threads by warp shuffles      */
  MPBP_FFT_EXCHANGE = 1   /* columns as 32 x 4 and rows as 8 x 16 transforms in
                             three register layouts joined by two shared-memory
                             exchanges per 2-D transform (default)           */
};

/* Arithmetic of the 2-D DFTs (F of Eq. 2 and its adjoint in the gradient). */
enum {
  MPBP_PRECISION_FP32 = 0,      /* FP32 radix-2 FFTs on the CUDA cores (default) */
  MPBP_PRECISION_TC_SPLIT16 = 1 /* dense DFT matrices on the tensor cores (M >= 32) */
};

/* Name of a status code (static string). */
const char *mpbp_status_string(mpbp_status s);

/* Creates a context for `problem` on the current CUDA device: validates the
 * geometry, copies G and the scan table to the device and allocates the
 * workspace (objects, gradient accumulators, a = sqrt(y), partial sums,
 * optimizer buffers).  Synchronous.  On failure *out is NULL. */
mpbp_status mpbp_create(const mpbp_problem *problem, mpbp_ctx **out);

/* Frees the context and its workspace (synchronises the device first). */
void mpbp_destroy(mpbp_ctx *ctx);

/* Message describing the last error this context returned ("" if none). */
const char *mpbp_last_error(const mpbp_ctx *ctx);

/* Workspace and launch configuration of the context. */
mpbp_status mpbp_get_info(const mpbp_ctx *ctx, mpbp_info *info);

/* Sets the probe P_m of Eq. 2: dev [Dp][M][M] complex (Dp = npeaks when
 * probe_per_peak, else 1), copied into the context. */
mpbp_status mpbp_set_probe(mpbp_ctx *ctx, const float *probe, void *stream);

/* Scan positions off the pixel grid.  Eq. 2's shift S_j moves the object
 * laterally by the scan position; for s_j = n_j + d_j (n_j the integer
 * position of mpbp_problem.scan, |d_j| <= 1/2 per axis) the exit wave on the
 * object's pixels r = n_j + k is P(r - s_j) O(r) = P(k - d_j) O(n_j + k), so
 * frame j keeps its integer window and takes the probe shifted by d_j, the
 * band-limited interpolation P_d(k) = (1/M^2) sum_q Phat(q) exp(2 pi i q.(k -
 * d)/M), Phat = F P, q of each axis in [-M/2, M/2).  d: host [J][2] (row,
 * column) offsets, copied; NULL returns to the integer positions.  The
 * shifted probes (J of them, or D*J with probe_per_peak, M*M complex each,
 * owned by the context) are formed on `stream` from the current probe, and
 * again by every later mpbp_set_probe; every evaluation, the forward model
 * and the illumination map use them.  MPBP_ERR_INVALID_ARG if an offset is
 * outside [-1/2, 1/2] (or not finite); MPBP_ERR_OOM if the probes do not
 * fit and MPBP_ERR_CUDA if they cannot be formed, after which the context
 * is back at the integer positions. */
mpbp_status mpbp_set_scan_offsets(mpbp_ctx *ctx, const double *d, void *stream);

/* The same band-limited shift as a standalone call: out[i] = P(k - d_i) for
 * one probe P (dev [M][M] complex, 1 <= M <= 128) and n offsets d (host
 * [n][2], |d| <= 1/2); out: dev [n][M][M] complex.  FP32, on the CUDA cores.
 * Synchronous (returns after the probes are written).  MPBP_ERR_INVALID_ARG
 * for bad sizes or offsets. */
mpbp_status mpbp_shift_probe(const float *probe, int32_t m, const double *d, int32_t n, float *out,
                             void *stream);

/* Sets the measured intensities y of Eq. 4: dev [D][J][M][M] float counts
 * (>= 0), and the optional background b of Eq. 2 (dev, same shape, or NULL).
 * The context derives and keeps a = sqrt(y) (and b) in its own layout; the
 * caller may free y and b once the stream has passed this call. */
mpbp_status mpbp_set_data(mpbp_ctx *ctx, const float *y, const float *bg, void *stream);

/* Eq. 1 / Eq. 3: O_out = dev [D][n1][n2] complex objects of every peak from
 * rho (dev [n1][n2]), u (dev [C][n1][n2]) and alpha (dev [D]). */
mpbp_status mpbp_object_build(mpbp_ctx *ctx, const float *rho, const float *u,
                              const float *alpha, float *O_out, void *stream);

/* Eq. 2: I_out = dev [D][J][M][M] model intensities |F P S O|^2 + b (b from
 * mpbp_set_data when set, else 0).  Needs the probe. */
mpbp_status mpbp_forward(mpbp_ctx *ctx, const float *rho, const float *u,
                         const float *alpha, float *I_out, void *stream);

/* Eq. 4 and its gradient over the frames listed in `frames` (dev int32
 * [nframes], each in [0, D*J); NULL = all D*J frames, nframes ignored).
 * Outputs (all dev, overwritten): loss (1 double), g_rho [n1][n2],
 * g_u [C][n1][n2], g_alpha [D] doubles (NULL to skip).  Needs probe and data.
 * Loss and gradients are sums over frames and pixels (no normalisation). */
mpbp_status mpbp_loss_grad(mpbp_ctx *ctx, const float *rho, const float *u,
                           const float *alpha, const int32_t *frames, int32_t nframes,
                           double *loss, float *g_rho, float *g_u, double *g_alpha,
                           void *stream);

/* Eq. 4 alone, without its gradient, over the frames listed in `frames` (as
 * mpbp_loss_grad; NULL = all D*J frames): loss (dev, 1 double, overwritten).
 * The fused frame kernel stops after the amplitude residual (no adjoint
 * transform, no scatter-add); the per-frame terms are mpbp_loss_grad's (FFT
 * kernels), summed in FP64 in another fixed order.  Always uses the FP32 FFTs, whatever
 * mpbp_set_precision selected.  Needs probe and data.  For callers that need
 * the loss without the gradient (a line search, or an autograd function that
 * recomputes the gradient in its backward pass). */
mpbp_status mpbp_loss(mpbp_ctx *ctx, const float *rho, const float *u, const float *alpha,
                      const int32_t *frames, int32_t nframes, double *loss, void *stream);

/* End-to-end variant of mpbp_loss_grad on HOST buffers: copies y (host
 * [D][J][M][M], or NULL to keep the data already set; when given it also
 * becomes the context's data for later calls), rho, u, alpha to the device,
 * evaluates all frames, returns loss (1 double), g_rho, g_u and g_alpha (host,
 * NULL to skip), and synchronises the stream.  y is copied in chunks that are
 * evaluated while later chunks are still in flight.  Page-locked host memory
 * makes the copies asynchronous and fast; when every requested output is
 * page-locked the device writes the outputs in place (no separate read-back),
 * otherwise they are copied back from the workspace. */
mpbp_status mpbp_loss_grad_host(mpbp_ctx *ctx, const float *y, const float *rho,
                                const float *u, const float *alpha, double *loss,
                                float *g_rho, float *g_u, double *g_alpha, void *stream);

/* mpbp_loss_grad_host with the measured data as 16-bit photon counts: y is
 * host uint16 [D][J][M][M] (natural layout, each count exact; counts above
 * 65535 cannot be given this way), half the bytes of the float call across
 * the host link.  On frame side 64 (FP32 precision, even n2) the frame
 * kernel reads the staged 16-bit counts itself; otherwise they are widened
 * to floats on the device first.  Everything else as
 * mpbp_loss_grad_host; y must not be NULL. */
mpbp_status mpbp_loss_grad_host_counts16(mpbp_ctx *ctx, const uint16_t *y, const float *rho,
                                         const float *u, const float *alpha, double *loss,
                                         float *g_rho, float *g_u, double *g_alpha,
                                         void *stream);

/* Initialises the device-resident optimizer state st (dev) from prm (host). */
mpbp_status mpbp_step_init(mpbp_ctx *ctx, const mpbp_step_params *prm,
                           mpbp_step_state *st, void *stream);

/* One optimizer iteration on rho, u, alpha (dev, updated in place):
 *   1. f, g = loss and gradient at the current iterate (all frames);
 *   2. accept it on the first call, or when f is finite and
 *      f <= f_prev - c_armijo * t * gn2_prev;
 *   3. accepted: keep the iterate and its gradient as the new base point,
 *      t *= grow (not on the first call); rejected: t *= shrink;
 *   4. rho, u, alpha = base - t * w * g_base, alpha_0 held fixed (the
 *      reference peak of Eq. 3 has no scaling variable).
 * All decisions are taken on the device in FP64, so a sequence of calls can be
 * captured in a CUDA graph and replayed without host synchronisation. */
mpbp_status mpbp_step(mpbp_ctx *ctx, float *rho, float *u, float *alpha,
                      mpbp_step_state *st, void *stream);

/* Records one mpbp_step(ctx, rho, u, alpha, st) -- object synthesis, fused
 * frame kernel, gradient assembly with the line-search decision and the
 * update --
 * as a CUDA graph owned by the context (replacing an earlier one), on a
 * stream of the context's own; nothing runs.  The pointers (dev) are baked
 * into the graph, and so are the kernels, the schedule and the probes
 * (scan offsets) in force at capture (later mpbp_set_precision,
 * mpbp_set_schedule or mpbp_set_scan_offsets calls need a new capture; a new
 * probe of the same kind is picked up, since the graph reads the context's
 * probe buffers).
 * Frame-kernel timing (mpbp_frames_timing) must be off.  Synchronous.
 * MPBP_ERR_CUDA if capture or instantiation fails. */
mpbp_status mpbp_step_capture(mpbp_ctx *ctx, float *rho, float *u, float *alpha,
                              mpbp_step_state *st);

/* Launches the captured step on `stream`: the same work as mpbp_step with
 * the captured arguments, with one launch from the host instead of three.
 * MPBP_ERR_INVALID_ARG if no step has been captured. */
mpbp_status mpbp_step_replay(mpbp_ctx *ctx, void *stream);

/* ------------------------------------------------------------------------
 * The paper's own optimizer, Alg. 1 without its projector line (the
 * "concurrent-wrapped" reconstruction): minibatches of frames from a shuffled
 * epoch, the auxiliary variables of Eq. 8 -- rho = mask * e^{chi} (mask: the
 * support constraint), alpha_0 = 1, alpha_m = e^{alpha_t[m]} -- and Adam
 * (Kingma and Ba) with step sizes per block (the paper: 0.01 for u, 0.1 for
 * chi and alpha_t).
 * ------------------------------------------------------------------------ */
typedef struct {
  double lr_u, lr_chi, lr_alpha;   /* Adam step sizes of u, chi, alpha_t     */
  double beta1, beta2, eps;        /* moment decay rates and denominator term */
} mpbp_adam_params;

typedef struct {
  double lr_u, lr_chi, lr_alpha, beta1, beta2, eps;   /* copied from the params */
  double f_last;         /* minibatch loss of the last step, before its update */
  double bc1, bc2;       /* 1 - beta1^t, 1 - beta2^t of the last step           */
  int64_t t;             /* steps taken                                         */
} mpbp_adam_state;

/* Initialises Adam: st (dev) from prm (host), t = 0, and the context's moment
 * buffers (allocated on the first call, 4 * (2 (1 + C) n1 n2) + 16 D bytes)
 * to zero.  Synchronous on the first call. */
mpbp_status mpbp_adam_init(mpbp_ctx *ctx, const mpbp_adam_params *prm, mpbp_adam_state *st,
                           void *stream);

/* One minibatch iteration: the loss of Eq. 4 and its gradient over `frames`
 * (dev int32 [nframes]; NULL = all frames) at rho = mask * e^{chi}, u,
 * alpha = (1, e^{alpha_t[1..]}); the chain rule to chi (rho df/drho) and
 * alpha_t (alpha df/dalpha); Adam on chi [n1][n2], u [C][n1][n2] and
 * alpha_t[1..D-1] (dev, updated in place; alpha_t[0] is never read or
 * moved).  mask (dev [n1][n2], or NULL for none) must stay fixed between
 * steps.  st->f_last receives the minibatch loss.  Needs probe, data and
 * mpbp_adam_init; the frame order is the caller's (e.g. a seeded shuffle per
 * epoch, Alg. 1 line 1). */
mpbp_status mpbp_adam_step(mpbp_ctx *ctx, const int32_t *frames, int32_t nframes, float *chi,
                           float *u, float *alpha_t, const float *mask, mpbp_adam_state *st,
                           void *stream);

/* Copies the Adam moments out of (get) or into (set) the context, for
 * checkpoint and resume: m_chi, v_chi [n1][n2], m_u, v_u [C][n1][n2] floats,
 * m_alpha, v_alpha [D] doubles (dev).  Together with st and the variables they
 * are the whole optimizer state.  Needs mpbp_adam_init. */
mpbp_status mpbp_adam_get_state(mpbp_ctx *ctx, float *m_chi, float *v_chi, float *m_u,
                                float *v_u, double *m_alpha, double *v_alpha, void *stream);
mpbp_status mpbp_adam_set_state(mpbp_ctx *ctx, const float *m_chi, const float *v_chi,
                                const float *m_u, const float *v_u, const double *m_alpha,
                                const double *v_alpha, void *stream);

/* The illumination behind the final threshold of the reconstruction (the
 * remark after Eq. 8: the density is set to zero where the probe did not
 * illuminate the object): out (dev [n1][n2], overwritten) = sum over every
 * frame (peak m, scan j) of |P_m(r - s_j)|^2.  Needs the probe. */
mpbp_status mpbp_illumination(mpbp_ctx *ctx, float *out, void *stream);

/* W^{-1} of Eq. 9: 2-D phase unwrapping of D maps (dev [D][n1][n2], the
 * context's grid, values in [-pi, pi)) into out (dev, same shape; may be the
 * input), inside mask (dev [n1][n2], nonzero = inside, or NULL).  The method
 * is reliability-ordered path following (Herraez et al., Appl. Opt. 41, 7437,
 * 2002): pixel reliability 1 / sqrt(H^2 + V^2 + D1^2 + D2^2) from the wrapped
 * second differences (0 at the border and next to the mask's edge), edges
 * between 4-neighbours weighted by the sum of their pixels' reliabilities and
 * taken in decreasing order (ties: lower edge number, 2 r + {0: right,
 * 1: down}), i.e. integration along the maximum spanning forest.  Each
 * connected region is then shifted by the multiple of 2 pi that gives its
 * lowest-numbered pixel its wrapped value; pixels off the mask keep theirs.
 * The first call allocates the unwrapper's workspace (~52 bytes per pixel
 * and map) and synchronises.  One cooperative launch; its grid barriers are
 * bounded in time (MPBP_ERR_TIMEOUT via mpbp_sync_status if one runs out). */
mpbp_status mpbp_unwrap_phases(mpbp_ctx *ctx, const float *wrapped, const float *mask,
                               float *out, void *stream);

/* Pi_U of Eq. 10 on u (dev [C][n1][n2], in place): Phi_m = phase_scale G_m . u,
 * wrapped, unwrapped as mpbp_unwrap_phases inside mask, and mapped back with
 * the Moore-Penrose pseudo-inverse of G (the H^T (H H^T)^{-1} of Eq. 10 when
 * the G_m span the components of u), as the correction
 * u += (Phi' - Phi) pinv(G)^T / phase_scale; components no G_m reaches and
 * pixels off the mask are left as they are.  Alg. 1 applies it after every
 * Adam step (the paper's C-UW reconstruction). */
mpbp_status mpbp_project_displacement(mpbp_ctx *ctx, float *u, const float *mask, void *stream);

/* The per-peak-phase form of Eq. 3 (the variables of the paper's two-step
 * reconstruction, Sec. 5): objects O_m = alpha_m rho e^{i phi_m} from D
 * independent phase maps phi (dev [D][n1][n2]) instead of the displacement
 * field.  Loss and gradient as mpbp_loss_grad, with g_phi (dev [D][n1][n2]) =
 * df/dphi_m in place of g_u. */
mpbp_status mpbp_loss_grad_phases(mpbp_ctx *ctx, const float *rho, const float *phi,
                                  const float *alpha, const int32_t *frames, int32_t nframes,
                                  double *loss, float *g_rho, float *g_phi, double *g_alpha,
                                  void *stream);

/* Loss and gradient of n independent problems (frame sides may differ) in
 * one persistent launch of the fused frame kernel.  Each argument is a host
 * array of n per-problem pointers with the meaning of mpbp_loss_grad
 * (all frames of each problem). */
mpbp_status mpbp_loss_grad_batched(int32_t n, mpbp_ctx *const *ctxs,
                                   const float *const *rho, const float *const *u,
                                   const float *const *alpha, double *const *loss,
                                   float *const *g_rho, float *const *g_u,
                                   double *const *g_alpha, void *stream);

/* Loss and gradient of all frames, like mpbp_loss_grad, without allocating
 * anything.  The paper has no counterpart: this exists for callers that cannot
 * call cudaMalloc (code that runs under another framework's allocator, or
 * that has already reserved the GPU's memory) and so cannot create a context.
 * The caller passes every input and output as a device pointer: probe
 * [Dp][M][M] complex, measured intensities y [D][J][M][M] (no background),
 * rho, u, alpha, and the outputs loss (1 double), g_rho, g_u, g_alpha [D]
 * doubles (g_alpha may be NULL).  G and the scan table stay on the host in
 * *problem; the scan table is copied to the device on `stream` by
 * cudaMemcpyAsync, so a page-locked scan array must stay valid until the
 * stream has passed the call (a pageable one is read before the call
 * returns).  dev_err (dev, one int32, or NULL) receives this call's device
 * error bits, cleared first: MPBP_DEVERR_NONFINITE when the loss came out NaN
 * or infinite, MPBP_DEVERR_TIMEOUT when a bounded wait of a kernel ran out,
 * MPBP_DEVERR_BOUNDS for a frame index out of range (cannot happen here:
 * every frame is evaluated); with NULL these bits are not reported.  The
 * problem is checked as mpbp_create checks it (MPBP_ERR_INVALID_ARG,
 * MPBP_ERR_UNSUPPORTED).  The workspace lives in one fixed 16 MiB array
 * inside the library's device image, present on every GPU that loads the
 * library until the process exits; a problem needs about 8*(2*D*n1*n2 +
 * nscan) + 4*D*nscan*M*M bytes of it plus a few KiB, and a larger one returns
 * MPBP_ERR_UNSUPPORTED before anything is enqueued.  The first call on a
 * device looks up the array's device address (once per device), so make that
 * first call before capturing the stream into a graph.  All calls share the
 * array: each call clears what must start at zero, and calls whose GPU work
 * overlaps (other streams, other threads) race on it. */
enum {
  MPBP_DEVERR_BOUNDS = 1,     /* a frame index outside [0, npeaks*nscan)      */
  MPBP_DEVERR_NONFINITE = 2,  /* the loss came out NaN or infinite            */
  MPBP_DEVERR_TIMEOUT = 4     /* a bounded wait on the GPU ran out            */
};
mpbp_status mpbp_loss_grad_noalloc(const mpbp_problem *problem, const float *probe,
                                   const float *y, const float *rho, const float *u,
                                   const float *alpha, double *loss, float *g_rho,
                                   float *g_u, double *g_alpha, int32_t *dev_err,
                                   void *stream);

/* Selects the FFT schedule (MPBP_FFT_*) of this context's FP32 loss-and-
 * gradient kernel for frame side 128 (both compute the same transforms of
 * Eq. 2; other frame sides ignore it).  Host-side only; a captured step keeps
 * the schedule of its capture.  MPBP_ERR_INVALID_ARG for an unknown value. */
mpbp_status mpbp_set_fft_schedule(mpbp_ctx *ctx, int32_t schedule);

/* Deterministic gradient (the A7 sums of Eq. 11 in a fixed order).  With on
 * != 0 the frame kernel keeps each column's gradient rows in a window in
 * tensor memory and writes them back into per-block pieces (a run of frames
 * of one scan column strip) with plain stores, and a second
 * kernel sums, for every object pixel, the pieces covering it in a fixed
 * order, in place of red.global.add into one accumulator: loss, g_rho, g_u
 * and g_alpha are then the same bits on every call with the same inputs and
 * schedule (with the atomic sums they agree only to rounding).  Costs a
 * device workspace of about 8 x 128 x (rows spanned by a strip + 128) bytes
 * per piece for frame side 128 (about 1 GB for 87,846 frames of 128 x 128
 * on a 1024^2 object; 8 x 64 x (rows + 64) at side 64),
 * allocated here and kept while the context lives, and the clearing and
 * summing of it on each evaluation.  Needs frame side 64 or 128 on FP32 FFTs
 * (at 128 the exchange schedule) and tile copies (rows of O a multiple of 16
 * bytes): else MPBP_ERR_UNSUPPORTED.  While on, evaluations over a frame list
 * (mpbp_loss_grad with frames, mpbp_adam_step minibatches), the host-buffer
 * calls, mpbp_loss_grad_batched and mpbp_autotune return
 * MPBP_ERR_UNSUPPORTED, and so do mpbp_set_precision / mpbp_set_fft_schedule
 * to another arithmetic or schedule.  mpbp_loss_grad over every frame,
 * mpbp_loss_grad_phases, mpbp_step and its captured replay are
 * deterministic.  Synchronous (builds its plan on the host); a later
 * mpbp_set_schedule rebuilds it.  on == 0 returns to the atomic sums. */
mpbp_status mpbp_set_deterministic(mpbp_ctx *ctx, int32_t on);

/* Overrides the fused frame kernel's schedule: resident blocks per SM used to
 * size its persistent grid (0 = occupancy maximum).  Host-side only. */
mpbp_status mpbp_set_schedule(mpbp_ctx *ctx, int32_t blocks_per_sm);

/* Selects the arithmetic of the DFT passes (Eq. 2: Psi = F psi, and the
 * adjoint F^H chi of the gradient) in this context's gradient evaluations.
 *   MPBP_PRECISION_FP32: FP32 radix-2 FFTs in registers (default).
 *   MPBP_PRECISION_TC_SPLIT16: each 1-D pass is a product with the dense DFT
 *     matrix on the tensor cores (tcgen05.mma): operands split into an FP16
 *     high and low part after a per-frame power-of-two scaling, products
 *     hi*hi + hi*lo + lo*hi accumulated in FP32 (about 2^-21 relative error
 *     per transform, against about 2^-22 log2(M) for the FFTs).  Frame sides
 *     64 (one frame per 64 x 64 tile), 32 (four frames per tile, with the
 *     block-diagonal pair of 32-point DFT matrices, each frame scaled on its
 *     own) and 128 (a radix-2 x 2 step on the CUDA cores splits each
 *     transform into four 64 x 64 ones on the tensor cores):
 *     MPBP_ERR_UNSUPPORTED for other M, and the context keeps its previous
 *     mode.
 * Applies to mpbp_loss_grad, mpbp_loss_grad_host, mpbp_step and to problems
 * that mpbp_loss_grad_batched launches on their own (batch mode 3, or a side
 * the mode does not fuse); mpbp_forward and the fused batched kernels always
 * use the FFTs.  Resets the schedule to the selected kernel's occupancy
 * maximum.  The first switch to TC_SPLIT16 allocates and uploads a 64 KB
 * table and synchronises the device.  A device error word bit from a bounded
 * wait of that kernel is reported by mpbp_sync_status as MPBP_ERR_TIMEOUT. */
mpbp_status mpbp_set_precision(mpbp_ctx *ctx, int32_t mode);

/* Test hook for the timeout paths (on != 0): every bounded wait on the GPU
 * is made to run out without a fault.  The FFT gradient kernels' tile-copy
 * barriers are told to expect 16 bytes more than the copies deliver (each
 * block's wait, 0.2 s, runs out and the block leaves with no copy in flight);
 * the tensor-core kernel issues no MMA and no completion signal (its 0.2 s
 * wait runs out; no MMA is in flight when it frees its tensor memory); block
 * 0 of the phase unwrapper (mpbp_unwrap_phases, mpbp_project_displacement)
 * never arrives at a grid barrier (the others' 0.1 s waits run out).  The
 * next mpbp_sync_status returns MPBP_ERR_TIMEOUT.  Results of calls made
 * while it is on are meaningless.  No effect on contexts whose frame kernels
 * use cp.async copies (odd n2, M <= 16).  Off by default. */
mpbp_status mpbp_set_test_stall(mpbp_ctx *ctx, int32_t on);

/* Turns on (enable != 0) or off the recording of CUDA events around every
 * launch of the fused frame kernel, on the stream it is launched on.  Off by
 * default; must not be on while a stream is being captured into a graph. */
mpbp_status mpbp_frames_timing(mpbp_ctx *ctx, int32_t enable);

/* Waits for the recorded events, then returns the summed duration in
 * milliseconds (*total_ms) and the number of timed launches (*count) since the
 * last read, and clears them.  Host pointers. */
mpbp_status mpbp_frames_timing_read(mpbp_ctx *ctx, double *total_ms, int32_t *count);

/* Schedule of mpbp_loss_grad_batched calls whose first context is ctx:
 * mode 0 = one persistent launch for every frame side (work items of 1, 2 or
 * 4 frames per 256-thread block); mode 1 = one persistent launch per frame
 * side with that side's own block shape; mode 2 = as mode 1 for sides 32 and
 * 64, one launch per problem for side 128; mode 3 = one launch per problem.
 * Problems with M <= 16 always get their own launch.  order 0 = work items
 * grouped by problem, 1 = problems interleaved.  Host-side only. */
mpbp_status mpbp_set_batch_schedule(mpbp_ctx *ctx, int32_t mode, int32_t order);

/* Autotuner for one context: times mpbp_loss_grad at rho, u, alpha (dev)
 * over every candidate schedule and keeps the fastest: the DFT arithmetic
 * (frame sides 32 and 64: FP32 FFTs or split tensor-core DFTs, both within the
 * same error bounds; mpbp_set_precision), the FFT schedule (frame side 128,
 * FP32: mpbp_set_fft_schedule) and the resident frame-kernel blocks per SM
 * from 1 to the occupancy limit (mpbp_set_schedule).  loss, g_rho and g_u
 * (dev) receive the evaluations.  With cache_path != NULL (host string) the
 * choice is first looked up in that JSON-lines file under a key made of the
 * GPU name, M, D, n1 x n2 and the frame count, and appended to it after
 * tuning.  Synchronous.  Needs probe and data. */
mpbp_status mpbp_autotune(mpbp_ctx *ctx, const float *rho, const float *u, const float *alpha,
                          double *loss, float *g_rho, float *g_u, const char *cache_path,
                          void *stream);

/* Autotuner for mpbp_loss_grad_batched calls on these contexts: times every
 * batch mode and item order (mpbp_set_batch_schedule) on the given states and
 * keeps the fastest in ctxs[0]; cache as for mpbp_autotune, keyed by the GPU
 * and every problem's shape.  Synchronous. */
mpbp_status mpbp_autotune_batched(int32_t n, mpbp_ctx *const *ctxs, const float *const *rho,
                                  const float *const *u, const float *const *alpha,
                                  double *const *loss, float *const *g_rho, float *const *g_u,
                                  const char *cache_path, void *stream);

/* Synchronises `stream`, then clears the errors latched on the device since
 * the last call and returns one of them (MPBP_OK if none): MPBP_ERR_BOUNDS,
 * else MPBP_ERR_TIMEOUT (the results of a call whose bounded wait ran out are
 * undefined, a non-finite loss among them), else MPBP_ERR_NONFINITE. */
mpbp_status mpbp_sync_status(mpbp_ctx *ctx, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPBP_H_ */

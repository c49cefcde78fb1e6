/*
 * fpm.h -- C ABI of the GB300 Batch-FPM engine.
 *
 * The engine reconstructs a high-resolution complex object spectrum O (N x N)
 * from a stack of low-resolution intensity images (one m x m image per LED),
 * jointly with the pupil aberrations (Zernike coefficients), the defocus
 * distance z, a per-LED intensity factor gamma_i and a per-LED sub-pixel
 * spectral offset delta_i, by random mini-batch gradient steps with Adam.
 * The method is Batch-FPM (Sun et al., arXiv 2408.13782):
 *   forward model          Section 2.1, Eq. (1)-(3)
 *       I_i = gamma_i |F^-1( O(k - k_mi) P(k) H(k, z) )|^2
 *   loss over a batch      Section 2.2, Eq. (5); Eq. (4) for the intensity form
 *   random batch update    Section 2.3, Eq. (13); equal use per pass, Eq. (14)
 *   initial object         Section 2.3 (bilinear-interpolated centre image)
 *
 * Conventions
 *   - Complex arrays are interleaved float pairs (re, im), row-major.
 *   - O is the centred spectrum of the object transmission o(r):
 *         O = fftshift(fft2(o)) / s^2,  s = N / m,  DC at (N/2, N/2).
 *   - LED i: crop centred at DC + n_i (n_i = rounded nominal offset), pupil
 *     evaluated at q = p - delta_i, p in [-m/2, m/2)^2:
 *         M_i(p) = A(q) exp(i (sum_j c_j Z_j(q/R) + z kappa(q))),
 *         kappa(q) = 2 pi (sqrt(lambda^-2 - |q dk|^2) - 1/lambda),
 *         Z_j = Noll-ordered Zernike polynomials j = 2..15 (Noll 1976),
 *         A = hard circle |q| <= R, or anti-aliased clamp(R + 1/2 - |q|, 0, 1).
 *       psi_i = ifft2(ifftshift(crop_i(O) * M_i))   (1/m^2 normalised)
 *       I_i   = gamma_i |psi_i|^2
 *   - Loss (amplitude form, default):
 *         L = sum_{i in batch} sum_r (sqrt(gamma_i)|psi_i| - sqrt(max(I_meas,0)))^2
 *     Intensity form (Eq. 4): L = sum (gamma_i |psi_i|^2 - I_meas)^2.
 *   - Gradients of real L w.r.t. complex w are dL/dRe w + i dL/dIm w.
 *   - Adam (Kingma & Ba, bias corrected) per real component of every learnable
 *     tensor, every step; delta is clamped to +-FPM_OFFSET_BOUND_PX per axis and
 *     gamma held at or above FPM_GAMMA_FLOOR after each update.
 *
 * Pointers: any buffer argument may be host memory (pageable or pinned) or
 * device memory of the engine's device; the direction of each copy is taken
 * from unified addressing. Buffers are borrowed for the duration of the call
 * only; the engine owns all of its device state.
 *
 * Errors: every int-returning call returns FPM_OK (0) or a negative FPM_ERR_*
 * code, and fpm_last_error() gives a one-line description. No call throws,
 * aborts the process or leaves the handle unusable on an argument error.
 *
 * Threading: a handle is used by one host thread at a time. All device work
 * of a handle is ordered on the CUDA stream given to fpm_create.
 */
#ifndef FPM_GB300_H
#define FPM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPM_OK             0
#define FPM_ERR_ARG       -1  /* null handle/pointer, bad flag or hyper-parameter */
#define FPM_ERR_SHAPE     -2  /* unsupported m, upsample, radius, LED geometry or batch size */
#define FPM_ERR_RANGE     -3  /* batch index outside [0, n_leds) or repeated within a batch */
#define FPM_ERR_OOM       -4  /* device allocation failed */
#define FPM_ERR_NONFINITE -5  /* a loss came out NaN or Inf (state may hold non-finite values) */
#define FPM_ERR_TIMEOUT   -6  /* a bounded device wait gave up */
#define FPM_ERR_CUDA      -7  /* a CUDA runtime call failed (message in fpm_last_error) */
#define FPM_ERR_STATE     -8  /* call out of order, e.g. a step before fpm_load */

#define FPM_EDGE_AA        0  /* anti-aliased pupil edge: A = clamp(R + 1/2 - |q|, 0, 1) */
#define FPM_EDGE_HARD      1  /* hard pupil edge: A = [|q| <= R] */

#define FPM_LOSS_AMPLITUDE 0
#define FPM_LOSS_INTENSITY 1

#define FPM_LEARN_OBJECT   (1u << 0)
#define FPM_LEARN_ZERNIKE  (1u << 1)
#define FPM_LEARN_DEFOCUS  (1u << 2)
#define FPM_LEARN_GAMMA    (1u << 3)
#define FPM_LEARN_OFFSET   (1u << 4)
#define FPM_LEARN_PUPIL    (1u << 5)  /* the free-form pupil field (see fpm_set_pupil) */
#define FPM_LEARN_ALL      0x3Fu

#define FPM_PRECISION_FP32_FFT 0  /* hand-written shared-memory FFTs, FP32 */
/* The m-point 2-D (inverse) DFTs of the forward model (Section 2.1, Eq. 3) and
 * their adjoints computed as dense complex contractions with the DFT matrix on
 * the tensor cores (tcgen05.mma, FP32 accumulation in tensor memory), one CTA
 * per LED image. Operands rounded to BF16 or TF32; the X3 forms split every
 * operand into hi + lo parts and sum hi*hi + hi*lo + lo*hi (three products).
 * Need m in {64, 128, 256} and a crop box of at most 128 px
 * (2 * (floor(R + 1/2 + sqrt 2) + 1) + 1 <= 128, i.e. R <= 61); fpm_set_hparams
 * returns FPM_ERR_SHAPE otherwise. Loss, gradients and the Adam step are the
 * same as in the FFT path; only the transforms' arithmetic differs. */
#define FPM_PRECISION_BF16_GEMM   1
#define FPM_PRECISION_BF16X3_GEMM 2
#define FPM_PRECISION_TF32_GEMM   3
#define FPM_PRECISION_TF32X3_GEMM 4

#define FPM_LOAD_INIT      1  /* fpm_load flag: initialise O from the centre LED and reset parameters and Adam state */

#define FPM_N_ZERNIKE     14  /* Noll j = 2..15 */
#define FPM_OFFSET_BOUND_PX 1.0f
#define FPM_GAMMA_FLOOR     1e-3f  /* learned intensity factors are held >= this (the amplitude loss takes sqrt) */

typedef struct fpm_handle fpm_handle;

/* Imaging geometry (Section 2.1). */
typedef struct fpm_geometry {
  int32_t m;                /* low-res image side: 32, 64, 128, 256 or 512 (512 needs 16-CTA thread-block clusters) */
  int32_t n_leds;           /* number of LED images, >= 1 */
  const float* led_offset;  /* [n_leds][2] (row, col) nominal spectral LED centre in px of the
                               spectrum grid, relative to DC; host memory. The rounded value is
                               the crop position n_i, the remainder the initial delta_i. */
  float lambda_um;          /* wavelength, um */
  float dk_per_um;          /* spectral bin of both grids, 1/um (= 1 / (m * low-res pixel)) */
  int32_t pupil_edge;       /* FPM_EDGE_AA or FPM_EDGE_HARD */
} fpm_geometry;

/* Optimisers of the Adam family (Section 2.2 leaves the choice open). Each takes one
 * step per batch on every real component of every learnable tensor, with the
 * group's learning rate lr and the gradient g of the batch loss:
 *   ADAM     m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
 *            w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)   (Kingma & Ba)
 *   ADAMW    w <- w (1 - lr weight_decay), then the ADAM step (decoupled decay,
 *            Loshchilov & Hutter)
 *   NADAM    the ADAM moments; with mu_t = b1 (1 - 0.96^(0.004 t) / 2) and
 *            P_t = mu_1 ... mu_t: w <- w - lr (mu_(t+1) m / (1 - P_(t+1))
 *            + (1 - mu_t) g / (1 - P_t)) / (sqrt(v / (1 - b2^t)) + eps)   (Dozat)
 *   RMSPROP  v <- b2 v + (1 - b2) g^2, w <- w - lr g / (sqrt(v) + eps)
 *            (Tieleman & Hinton; beta2 is the smoothing constant, beta1 unused) */
#define FPM_OPT_ADAM 0
#define FPM_OPT_ADAMW 1
#define FPM_OPT_NADAM 2
#define FPM_OPT_RMSPROP 3

/* Optimiser and loss settings (Section 2.2: Adam-family optimiser, free loss choice). */
typedef struct fpm_hparams {
  float lr_object, lr_zernike, lr_defocus, lr_gamma, lr_offset;
  float beta1, beta2, eps;
  int32_t loss;             /* FPM_LOSS_AMPLITUDE or FPM_LOSS_INTENSITY */
  uint32_t learn_mask;      /* FPM_LEARN_* bits; cleared groups are held fixed */
  int32_t precision;        /* FPM_PRECISION_*: FP32 FFTs (default) or a tensor-core DFT form */
  int32_t optimizer;        /* FPM_OPT_*; default FPM_OPT_ADAM */
  float weight_decay;       /* FPM_OPT_ADAMW's decay rate (>= 0), applied to every learnable group */
  float lr_pupil;           /* learning rate of the free-form pupil field (FPM_LEARN_PUPIL) */
} fpm_hparams;

/* Create an engine for N = m * upsample, pupil radius R (spectral px).
 * Requires every crop box (half-width floor(R + 1/2 + sqrt(2) * FPM_OFFSET_BOUND_PX) + 1)
 * to lie inside the N x N spectrum and inside the m x m window.
 * cuda_stream: a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream); NULL = default.
 * Default hyper-parameters: lr 0.1 / 0.01 / 0.1 / 0.01 / 0.01 (pupil field 0.01), betas 0.9 / 0.999,
 * eps 1e-8, amplitude loss, learn object only, Adam, no weight decay. On success *out owns device memory
 * until fpm_destroy. */
int fpm_create(const fpm_geometry* g, float pupil_radius_px, int32_t upsample,
               void* cuda_stream, fpm_handle** out);

/* Replace the hyper-parameters. Takes effect at the next step. */
int fpm_set_hparams(fpm_handle* h, const fpm_hparams* hp);
int fpm_get_hparams(const fpm_handle* h, fpm_hparams* hp);

/* Copy the measured stack [n_leds][m][m] (intensities, float) into the engine.
 * With FPM_LOAD_INIT: O <- bilinear upsample (low-res pixel r on high-res pixel s*r,
 * periodic) of sqrt(max(I_centre, 0)) with zero phase, transformed as above;
 * centre = LED with the smallest |nominal offset|; zernike = 0, z = 0, gamma = 1,
 * delta = fractional part of the nominal offsets; Adam moments and step count reset. */
int fpm_load(fpm_handle* h, const float* stack, int32_t flags);

/* One random-batch update (Eq. 13): loss and gradients over the B LEDs in
 * batch_idx (host, [B], distinct, in [0, n_leds)), then Adam on every learnable
 * tensor. The gradient of O is accumulated over the batch in batch order.
 * loss_out (nullable, host): the batch loss before the update; when non-NULL the
 * call waits for the step to finish. */
int fpm_step(fpm_handle* h, const int32_t* batch_idx, int32_t B, double* loss_out);

/* n_steps consecutive updates; schedule is [n_steps][B] (host). Launched as one
 * CUDA graph per (n_steps, B), reused across calls. losses_out (nullable,
 * host or device, [n_steps]) receives each batch loss; when it is host memory
 * the call waits for the run to finish. */
int fpm_run(fpm_handle* h, const int32_t* schedule, int32_t n_steps, int32_t B, double* losses_out);

/* Timing variant of fpm_run for profiling: the same steps, launched directly on the
 * engine's stream (not as a graph), with, before every step, a clear of flush_bytes of the device buffer `flush`
 * (nullable: no clear; a buffer larger than the L2 cache evicts the working set so
 * each step starts cold), and CUDA events on the engine's stream. Outputs (host,
 * [n_steps] each, nullable): elapsed ms of the per-LED kernel, of the update
 * kernel and of the whole step (excluding the clear). With led_ms or update_ms
 * given, events also separate the two kernels (so they run back to back); with
 * both NULL only the step is bracketed and the update kernel starts early by
 * programmatic dependent launch, as inside fpm_run. In the dataflow form (see
 * fpm_set_step_form) a step is one kernel: led_ms gets the step and update_ms
 * zero. Waits for completion. The state advances exactly as with fpm_run. */
int fpm_profile_run(fpm_handle* h, const int32_t* schedule, int32_t n_steps, int32_t B,
                    void* flush, int64_t flush_bytes, float* led_ms, float* update_ms, float* step_ms);

/* Form of the kernels that run a step (the same model and results, up to the
 * order of FP32 rounding in the per-pixel partial sums):
 *   FPM_STEP_AUTO      the per-LED form (the fastest for one job's step);
 *   FPM_STEP_CLUSTER   the per-LED form: one thread-block cluster per LED image
 *                      for the model and its adjoint, the intermediate transforms
 *                      exchanged in distributed shared memory, then an update
 *                      launch (the batch-ordered gather and the optimiser);
 *   FPM_STEP_DATAFLOW  m = 256, FP32 FFT form: one launch per step whose CTAs
 *                      take the step's column transforms, row transforms with the
 *                      residual, adjoint column transforms and update as tasks
 *                      from a shared counter, spread over every SM; a task waits
 *                      (bounded) only for the tasks it reads, which hand their
 *                      results over through L2. Elsewhere the per-LED form.
 * Applies to fpm_step, fpm_run, fpm_profile_run, fpm_forward, fpm_backward and
 * their stored-field forms. fpm_get_step_form gives the form asked for and
 * whether the dataflow form is in use (each pointer nullable). */
#define FPM_STEP_AUTO     0
#define FPM_STEP_CLUSTER  1
#define FPM_STEP_DATAFLOW 2
int fpm_set_step_form(fpm_handle* h, int32_t form);
int fpm_get_step_form(const fpm_handle* h, int32_t* form, int32_t* dataflow);

/* Failure-injection check of the bounded device waits of the dataflow form (the
 * paper has no counterpart; it tests the engine's failure detection). Runs one
 * step over batch idx in which every row task waits for a count of column tasks
 * that is never reached, with every wait bounded by limit_s seconds (in
 * (0, 10]); the waits give up, the kernel records the timeout in its error
 * flag and returns, and the call returns FPM_ERR_TIMEOUT (FPM_ERR_STATE if no
 * wait gave up). The GPU context stays usable; the handle's estimate is
 * undefined afterwards (load or set a new one). Needs the dataflow form. */
int fpm_check_wait_timeout(fpm_handle* h, const int32_t* idx, int32_t B, double limit_s);

/* Sum of the batch losses since the last reset (FP64), optionally resetting it. */
int fpm_epoch_loss(fpm_handle* h, double* out, int32_t reset);

/* Forward model only: I_out[B][m][m] = gamma_i |psi_i|^2 for the LEDs in idx (host). */
int fpm_forward(fpm_handle* h, const int32_t* idx, int32_t B, float* I_out);

/* Gradients without an update. dL_dI (nullable, [B][m][m]): upstream gradient of
 * the predicted intensities; NULL means the built-in loss against the loaded stack.
 * Outputs (each nullable): g_object [N][N][2], g_zernike [14], g_defocus [1],
 * g_gamma [n_leds], g_offset [n_leds][2]; LEDs outside idx get 0. loss_out
 * (nullable): the built-in batch loss (only with dL_dI == NULL). */
int fpm_backward(fpm_handle* h, const int32_t* idx, int32_t B, const float* dL_dI,
                 float* g_object, float* g_zernike, float* g_defocus, float* g_gamma,
                 float* g_offset, double* loss_out);

/* Store-the-fields form of the pair above (the alternative to recomputing the
 * fields in the backward pass; FP32 FFT form only). fpm_forward_fields is
 * fpm_forward that also writes the low-res fields psi_i = IFFT(Phi_i) (Section
 * 2.1, Eq. 3, before |.|^2) to psi_out [B][m][m][2] (device memory, 8-byte
 * aligned; I_out device memory, 16-byte aligned). fpm_backward_fields takes
 * those fields (device) and the upstream dL_dI [B][m][m] (device) for the same
 * idx and the same engine state, and returns the gradients of fpm_backward
 * without recomputing psi (outputs as in fpm_backward). The caller owns the
 * field buffer: B * m * m * 8 bytes between the two calls. */
int fpm_forward_fields(fpm_handle* h, const int32_t* idx, int32_t B, float* I_out, float* psi_out);
int fpm_backward_fields(fpm_handle* h, const int32_t* idx, int32_t B, const float* psi, const float* dL_dI,
                        float* g_object, float* g_zernike, float* g_defocus, float* g_gamma,
                        float* g_offset);

/* Read / write the current estimate; each pointer nullable (skipped).
 * O [N][N][2], zernike [14], defocus [1], gamma [n_leds], offset [n_leds][2] (delta). */
int fpm_get(fpm_handle* h, float* O, float* zernike, float* defocus, float* gamma, float* offset);
int fpm_set(fpm_handle* h, const float* O, const float* zernike, const float* defocus,
            const float* gamma, const float* offset);

/* O <- fftshift(fft2(o)) / s^2 for a real-space transmission o [N][N][2]. */
int fpm_set_object_field(fpm_handle* h, const float* o);

/* Free-form pupil (the pupil-recovery reading of Section 2.2, "pupil function"):
 * a complex field P on the integer nodes n of the crop box (|n_y|, |n_x| <= h,
 * W = 2h + 1 nodes a side, W from fpm_dims) that multiplies the parametric
 * pupil. LED i sees it at q = p - delta_i by bilinear interpolation between the
 * four nodes around q:
 *     M_i(p) = A(q) exp(i (sum_j c_j Z_j(q/R) + z kappa(q))) * P~(q).
 * Without a field (the default) M_i is the parametric pupil. fpm_set_pupil
 * puts P (host or device, [W][W][2], row-major: node (n_y, n_x) at
 * (n_y + h) * W + n_x + h) into the model; P == NULL takes it out (refused
 * while FPM_LEARN_PUPIL is set). Setting FPM_LEARN_PUPIL puts the field in
 * (at its current values; fpm_load with FPM_LOAD_INIT resets it to 1 and its
 * moments to 0) and the optimiser then updates it every step with lr_pupil.
 * fpm_get_pupil copies the field out (P nullable; *in_use nullable: whether it
 * is in the model). fpm_pupil_gradient gives dL/dRe P + i dL/dIm P of the last
 * fpm_backward or fpm_backward_fields ([W][W][2], same layout; FPM_ERR_STATE
 * without a field). The field needs the FP32 FFT form (FPM_ERR_ARG otherwise). */
int fpm_set_pupil(fpm_handle* h, const float* P);
int fpm_get_pupil(fpm_handle* h, float* P, int32_t* in_use);
int fpm_pupil_gradient(fpm_handle* h, float* g);

/* Full optimiser state for checkpoint / resume. Sizes in floats: */
int64_t fpm_state_size(const fpm_handle* h);
/* Layout: O, m_O, v_O ([N][N][2] each), then params, m_params, v_params
 * ([15 + 3 n_leds] each: zernike, z, gamma, delta), then the free-form pupil
 * field, m_P, v_P ([W][W][2] each, node (n_y, n_x) at (n_x + h) * W + n_y + h),
 * then {step count, epoch loss, field in the model (0 or 1)} stored as three
 * float64 in the last six floats. The layout is the same for every
 * optimiser: RMSprop leaves the m arrays at zero, and NAdam's product of momentum
 * coefficients is rebuilt from the step count. */
int fpm_get_state(fpm_handle* h, float* state);
int fpm_set_state(fpm_handle* h, const float* state);

/* Sizes of this handle. */
int fpm_dims(const fpm_handle* h, int32_t* N, int32_t* m, int32_t* n_leds, int32_t* box);

/* Device memory held by the handle (bytes), and a limit on it (bytes; <= 0:
 * none, the default). A call that would grow the handle's buffers past the
 * limit (a larger batch, a longer run, a tensor-core form) returns FPM_ERR_OOM
 * before touching any buffer, and the handle stays usable with what it has;
 * the limit does not shrink what is already held. fpm_memory_used returns
 * FPM_ERR_ARG for a NULL handle. */
int fpm_set_memory_limit(fpm_handle* h, int64_t bytes);
int64_t fpm_memory_used(const fpm_handle* h);

/* Host-side random batch order (Eq. 13-14): the permutation of range(n) for
 * pass `epoch`: SplitMix64 (Steele, Lea & Flood 2014) seeded with
 * seed ^ ((epoch + 1) * 0xA0761D6478BD642F), driving a Durstenfeld shuffle of the
 * identity (for i = n-1 .. 1: j = next() mod (i + 1); swap). No GPU needed. */
int fpm_epoch_permutation(int32_t n, uint64_t seed, int32_t epoch, int32_t* out);

/* ---- Allocation-free gradients -------------------------------------------
 * For callers that cannot allocate device memory: code running while a host
 * framework owns the device memory pool (where a cudaMalloc would bypass it or
 * is not allowed), or real-time acquisition loops in which an allocation may
 * block. The paper has no counterpart: this is an interface convenience, not
 * a step of the method.
 *
 * Computes the same batch loss and gradients as fpm_backward with the built-in
 * loss (same model, same kernels), without a handle and without allocating
 * anything. Every input and output is a device buffer owned by the caller; the
 * intermediates (per-LED gradient boxes, per-LED FP64 partials, LED tables)
 * live in one static device array of FPM_STATIC_SCRATCH_BYTES inside the
 * library, which every GPU that loads the library holds until the process
 * exits. A batch needs about B * (2h+1)^2 * 8 + B * C * 152 bytes of it
 * (h = floor(R + 1/2 + sqrt(2)) + 1; C = 8 for m = 256, m/16 below) plus small
 * tables; larger batches are
 * rejected with FPM_ERR_SHAPE and a message giving both sizes.
 *
 * The array is shared by all calls on a device and keeps the last call's
 * contents (each call clears what must start at zero); calls whose device
 * work overlaps (two streams, two host threads) race on it.
 * The first call on a device looks up the array's device address, sets the
 * kernels' attributes and writes the transform twiddles into the array (once
 * per device, with that device current); make that first call before any
 * stream capture. Every call copies its batch tables from host memory, so a
 * call on a stream that is being captured returns FPM_ERR_STATE.
 *
 * g, pupil_radius_px, upsample: as fpm_create, m up to 256 (the rounded LED offsets give the
 *   crop positions; delta comes from `params`).
 * O_t      device [N][N][2] object spectrum, COLUMN-major: element (row y, col x)
 *          at index x * N + y (the transpose of fpm_get's layout).
 * params   device [15 + 3 n_leds]: zernike[14], defocus, gamma[n_leds], delta[n_leds][2];
 *          every delta of the batch must lie within +-FPM_OFFSET_BOUND_PX (the crop
 *          box is sized for that bound; beyond it the results are unspecified
 *          and err_out gets FPM_DEVERR_OFFSET).
 * stack    device [n_leds][m][m] measured intensities.
 * idx      host [B] distinct LED indices; B in [1, n_leds].
 * loss     FPM_LOSS_AMPLITUDE or FPM_LOSS_INTENSITY.
 * g_object_t  device [N][N][2], column-major like O_t; every element is written.
 * g_params    device [15 + 3 n_leds], same layout as params; LEDs outside idx get 0.
 * loss_out    device [1] FP64 batch loss (NaN/Inf if the data are not finite).
 * err_out     device [1] int32 (nullable): the kernels' error bits of this call,
 *             written after the gradients: 0, or an OR of FPM_DEVERR_INDEX (a
 *             batch index the kernels found out of range), FPM_DEVERR_NONFINITE
 *             (the batch loss is not finite) and FPM_DEVERR_OFFSET (a delta beyond
 *             the bound). Without err_out only a non-finite loss_out shows them.
 * cuda_stream cudaStream_t for all of the call's device work (NULL = default).
 * All device buffers must belong to the current device. Returns after
 * enqueueing; results are ready when the stream reaches them. Errors found on
 * the host are reported by the return code and fpm_last_error(NULL). */
#define FPM_DEVERR_INDEX     1
#define FPM_DEVERR_NONFINITE 2
#define FPM_DEVERR_OFFSET    8
#define FPM_STATIC_SCRATCH_BYTES (4u << 20)
int fpm_gradients_static(const fpm_geometry* g, float pupil_radius_px, int32_t upsample,
                         const float* O_t, const float* params, const float* stack,
                         const int32_t* idx, int32_t B, int32_t loss,
                         float* g_object_t, float* g_params, double* loss_out, int32_t* err_out,
                         void* cuda_stream);

/* ---- Measurement ----------------------------------------------------------
 * FP32 fused multiply-add throughput of the current device (TFLOP/s): the
 * CUDA-core peak that the per-LED kernel's ALU roofline is quoted against.
 * Not a step of the method (the paper has no counterpart). Runs reps + 1
 * launches of a kernel in which every thread (8 CTAs of 256 threads per SM)
 * advances 16 independent fmaf chains `iters` times, and reports the fastest
 * launch timed by CUDA events: 2 * 16 * iters * threads / time. ms_out
 * (nullable): that launch's duration. Allocates and frees a small output
 * buffer; synchronises. Returns FPM_ERR_ARG for iters or reps below 1. */
int fpm_probe_fp32_fma(int32_t iters, int32_t reps, double* tflops_out, double* ms_out);

/* ---- Serving: continuous batching of reconstruction jobs -----------------
 * A request loop for many reconstructions of uneven size. Submitted jobs are
 * queued and admitted in arrival order, each as soon as its device-memory
 * footprint fits the rest of the server's budget and a slot is free (first fit;
 * a job too large for now does not hold back smaller ones) (the paper picks the
 * batch size from the available GPU memory, Section 2.2; here memory decides
 * which jobs are resident). An admitted job keeps its object spectrum, pupil,
 * defocus, LED parameters and Adam state resident on the device. Each epoch
 * is a fresh random batch order (Eq. 13-14, seed = job seed). Resident jobs
 * (FP32 FFT form) with the same number of steps per epoch run their epochs
 * together in rounds, grouped as fpm_server_set_grouping says: each step of a
 * round is one per-LED launch and one update launch covering all of them, and
 * a round is one CUDA graph, captured once per set of jobs. Rounds of different
 * sets run on their own
 * streams, so all resident jobs overlap on the GPU; each job's arithmetic is
 * the same alone or in a round, so its result is too (bit for bit). A job
 * stops when the relative change of its epoch loss drops below rel_tol, or
 * after max_epochs; its result is then copied to host memory and its device
 * memory freed for the next admissions.
 * All server calls are made from one host thread. */
typedef struct fpm_server fpm_server;

typedef struct fpm_job_desc {
  fpm_geometry geometry;     /* led_offset is copied at submit */
  float pupil_radius_px;
  int32_t upsample;
  fpm_hparams hparams;
  int32_t batch;             /* B, in [1, n_leds] */
  int32_t max_epochs;
  double rel_tol;            /* stop when |L_e - L_{e-1}| < rel_tol * L_{e-1} */
  uint64_t seed;             /* batch order seed */
} fpm_job_desc;

#define FPM_JOB_QUEUED 0
#define FPM_JOB_ACTIVE 1
#define FPM_JOB_DONE   2
#define FPM_JOB_FAILED 3

typedef struct fpm_job_status {
  int32_t state;             /* FPM_JOB_* */
  int32_t epochs;            /* completed */
  double loss;               /* last epoch loss */
  double t_submit, t_admit, t_done;  /* seconds on the server clock */
  int64_t led_updates;       /* LED images processed (forward + backward) */
  int64_t footprint;         /* device bytes reserved while resident */
} fpm_job_status;

/* Order in which queued jobs are considered for admission (each still needs a
 * free slot and room in the memory budget; a job that does not fit is passed
 * over for now): FPM_ADMIT_ARRIVAL (default) in arrival order;
 * FPM_ADMIT_SMALLEST smallest expected work first (LED images x m^2 x
 * max_epochs), ties in arrival order - shorter jobs then finish sooner, which
 * lowers the median time to converge under load at the cost of the larger
 * jobs' wait. */
#define FPM_ADMIT_ARRIVAL  0
#define FPM_ADMIT_SMALLEST 1
int fpm_server_set_admission(fpm_server* s, int32_t order);

/* Which resident jobs share a round (all with the same number of steps per
 * epoch, FP32 FFT form):
 * FPM_GROUP_CONFIG  (default) the same low-res size, crop box, LED count and
 *                   batch size;
 * FPM_GROUP_SIZE    the same low-res size; sizes 64, 128 and 256 use
 *                   the mixed per-LED launch, which takes any crop box (up to
 *                   h < 64 at 256), LED count and batch size;
 * FPM_GROUP_MIXED   sizes 64, 128 and 256 together in one mixed launch (their
 *                   LEDs share clusters of 16 CTAs), other sizes as SIZE.
 * A round steps at the pace of its slowest job, so mixing sizes trades the
 * small jobs' time to converge for fewer launches; on a stream of 100 uneven
 * jobs the three policies gave the same throughput and median time to converge
 * within the run-to-run spread, MIXED about 40 % fewer launches. A job's result does not
 * depend on the other jobs of its round; at m = 64 it also equals a direct run
 * bit for bit (the same CTA layout), at m = 128 and 256 within rounding. */
#define FPM_GROUP_CONFIG 0
#define FPM_GROUP_SIZE   1
#define FPM_GROUP_MIXED  2
int fpm_server_set_grouping(fpm_server* s, int32_t grouping);

/* Device bytes a job holds while resident (its admission size). */
int64_t fpm_job_footprint(const fpm_job_desc* d);
int fpm_server_create(int64_t hbm_budget_bytes, int32_t max_active, fpm_server** out);
/* Queue a job; stack is host [n_leds][m][m] intensities, copied. FPM_ERR_OOM if
 * its footprint exceeds the whole budget. */
int fpm_server_submit(fpm_server* s, const fpm_job_desc* d, const float* stack, int64_t* job_id);
/* Make progress without blocking: retire finished epochs, stop converged jobs,
 * admit queued ones, launch the next rounds. Outputs (nullable): jobs
 * resident, jobs waiting. */
int fpm_server_tick(fpm_server* s, int32_t* n_active, int32_t* n_queued);
int fpm_server_status(const fpm_server* s, int64_t job_id, fpm_job_status* st);
/* Result of a finished job (host buffers, each nullable; layouts as fpm_get). */
int fpm_server_result(fpm_server* s, int64_t job_id, float* O, float* zernike, float* defocus,
                      float* gamma, float* offset);
double fpm_server_clock(const fpm_server* s);      /* seconds since fpm_server_create */
/* Counters since creation (each nullable): rounds launched, job epochs they
 * ran, the most jobs in one round, kernel launches of the rounds. */
int fpm_server_stats(const fpm_server* s, int64_t* rounds, int64_t* round_epochs, int64_t* max_jobs_per_round,
                     int64_t* launches);
const char* fpm_server_error(const fpm_server* s);
void fpm_server_destroy(fpm_server* s);

void fpm_destroy(fpm_handle* h);

/* Last error message of the handle (or, when h is NULL, of the last failed
 * fpm_create or fpm_gradients_static on this thread). */
const char* fpm_last_error(const fpm_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* FPM_GB300_H */

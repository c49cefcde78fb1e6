// Launch arguments shared by the host engine and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

struct fpm_handle;

namespace fpmk {

// Per-CTA partial sums written by the LED kernel (FP64).
constexpr int NPART = 19;
// The mixed-size per-LED launch of the serving loop: clusters of 16 CTAs of
// 128 threads shared by LEDs of m = 64, 128 and 256 (4, 8 and 16 CTAs each).
constexpr int LED_MIX_CLUSTER = 16;
constexpr int LED_MIX_THREADS = 128;
enum : int { P_LOSS = 0, P_GAMMA = 1, P_ZERN = 2, P_DEFOCUS = 16, P_DY = 17, P_DX = 18 };

// Scalar parameter vector layout: [zernike 14][defocus 1][gamma n][delta n x (dy, dx)].
constexpr int SP_ZERN = 0, SP_DEFOCUS = 14, SP_GAMMA = 15;
__host__ __device__ inline int sp_offset(int n_leds) { return SP_GAMMA + n_leds; }
__host__ __device__ inline int sp_size(int n_leds) { return SP_GAMMA + 3 * n_leds; }

// MODE_FORWARD_STORE: MODE_FORWARD that also writes the fields psi;
// MODE_UPSTREAM_STORED: MODE_UPSTREAM that reads psi instead of recomputing it.
enum LedMode : int { MODE_LOSS = 0, MODE_FORWARD = 1, MODE_UPSTREAM = 2, MODE_FORWARD_STORE = 3, MODE_UPSTREAM_STORED = 4 };

// Device error flags (bit set, OR-accumulated). DERR_OFFSET: an LED offset
// beyond +-FPM_OFFSET_BOUND_PX (the crop box is sized for the bound).
enum : int { DERR_INDEX = 1, DERR_NONFINITE = 2, DERR_TIMEOUT = 4, DERR_OFFSET = 8 };

constexpr int MAX_BATCH = 1024;

struct LedArgs {
  const float2* Ot;     // [N][N] spectrum, column-major: element (row y, col x) at Ot[x * N + y]
  const float* meas;    // [n_leds][m][m] measured intensities (MODE_LOSS), or amplitudes if meas_is_amp
  const float* dLdI;    // [B][m][m] upstream gradient of the intensities (MODE_UPSTREAM)
  float* I_out;         // [B][m][m] predicted intensities (MODE_FORWARD)
  float2* psi;          // [B][m][m] low-res fields (written in MODE_FORWARD_STORE, read in MODE_UPSTREAM_STORED)
  const float* sp;      // scalar parameters, layout above
  const int4* slot;     // [B] batch slots: (LED, crop row offset n_row, crop col offset n_col, 0)
  float2* gbox;         // [B][W][W] per-LED object-gradient boxes, [slot][col][row]
  double* part;         // [B][cluster][NPART] per-CTA FP64 partials
  const float2* tw;     // [m] exp(-2 pi i t / m)
  int N, n_leds, B, h, W;
  float R, Rinv, inv_lambda, dk2;
  int hard_edge, loss, mode;
  int meas_is_amp;      // meas holds sqrt(max(I, 0)) (amplitude loss in MODE_LOSS)
  int* err;
  // free-form pupil (nullable: none): node field [W][W], column-major like the
  // boxes (node (ny, nx) at (nx + h) * W + ny + h); per-LED gradient boxes
  // [B][W][W] and per-slot bilinear placement (fy, fx, ay, ax) for the update
  const float2* pupil;
  float2* pbox;
  float4* pwt;
};

struct UpdArgs {
  float2* Ot;           // [N][N] column-major
  float2* mO;           // Adam first moment of (Re, Im)
  float2* vO;           // Adam second moment of (Re, Im)
  float* sp;            // scalar parameters
  float* msp;
  float* vsp;
  const float2* gbox;   // from the LED kernel
  const double* part;
  const int4* slot;     // [B] batch slots, as in LedArgs
  const int2* span;     // [N] per column: [row_lo, row_hi) of the update region
  int x_lo, n_cols;     // update-region columns [x_lo, x_lo + n_cols)
  int N, n_leds, B, C, h, W;
  float lr_obj, lr_zern, lr_def, lr_gam, lr_off, b1, b2, eps;
  float offset_bound;
  // per step of the sequence, by optimiser (nullable: (1, 1, 0, 0)):
  //   Adam, AdamW: (1/(1-b1^t), 1/sqrt(1-b2^t), 0, 0)
  //   NAdam: (mu_(t+1)/(1-P_(t+1)), 1/sqrt(1-b2^t), (1-mu_t)/(1-P_t), 0)
  //   RMSprop: (0, 1, 0, 0)
  const float4* coef;
  int opt;                  // FPM_OPT_*
  float wd;                 // AdamW weight decay
  int step_off;             // this step's position in the sequence
  unsigned learn;
  double* loss_slot;        // batch loss of this step
  double* epoch_loss;       // running FP64 sum
  int* err;
  int assemble;             // 1: write gradients (g_obj, g_sc) instead of updating
  float2* g_obj;            // [N][N] column-major, zeroed by the caller
  float* g_sc;              // [15 + 3 n_leds]
  // free-form pupil (pupil_cols = 0: none): the node field, its moments, the
  // per-LED gradient boxes and placements of the LED kernel, its gradient
  // (assembling); learned under FPM_LEARN_PUPIL with rate lr_pupil
  float2* Pff;
  float2* mPff;
  float2* vPff;
  const float2* pbox;
  const float4* pwt;
  float2* g_pupil;
  float lr_pupil;
  int pupil_cols;
};

// ---- dataflow form of the step (step.cu), m = 256 ------------------------
// One launch per step. Its CTAs take tasks from a ticket counter, in the
// order: column transforms of every LED (A), row transforms with the residual
// (B), adjoint column transforms with the box gradients (C), then the update
// (scalar sums and optimiser, AdamW decay outside the update region, one task
// per spectrum column of the update region). A task waits only for the tasks
// it reads from, through per-LED completion counters (bounded waits).
struct StepSync {
  // each counter on its own 128-byte line: waiting CTAs poll one line per LED
  struct alignas(128) Ctr {
    unsigned v;
  };
  Ctr ticket;              // next task
  Ctr exit_count;          // CTAs done; the last one resets every counter
  Ctr c_all;               // adjoint column tasks done (all LEDs)
  Ctr a_done[MAX_BATCH];   // column-transform tasks done, per batch slot
  Ctr b_done[MAX_BATCH];   // row tasks done, per batch slot
};

constexpr int STEP_NPB = 2;   // partials of a row task: loss, gamma term
constexpr int STEP_NPC = 17;  // partials of an adjoint column task: 14 Zernike, defocus, dy, dx

struct StepArgs {
  LedArgs L;            // model, mode and per-LED tables (L.gbox, L.part unused: see below)
  UpdArgs U;            // the update (U.part unused)
  float2* T;            // [B][W][256] column transforms, overwritten in place by the row tasks
  double* partB;        // [B][nB][STEP_NPB]
  double* partC;        // [B][nC][STEP_NPC]
  StepSync* sync;       // counters, all zero between launches
  int nA, nB, nC;       // tasks per LED of each phase
  int do_update;        // run the update tasks (modes with an adjoint)
  long long wait_ns;    // bound of every dependency wait
  int stall;            // failure injection: row tasks wait for a count no task reaches
};

// Shared-memory bytes and CTAs of one launch (W: box width, B: batch).
size_t step_smem_bytes(int W, int B);
cudaError_t step_prepare(int W, int B, int* max_ctas);
int step_tasks(const StepArgs& s);
cudaError_t launch_step(const StepArgs& s, int max_ctas, cudaStream_t st, bool pdl);

// Cluster size C (CTAs cooperating on one LED image) for low-res side m.
int led_cluster_size(int m);
int led_choose_cluster(int m, int W);
size_t led_smem_bytes(int m, int C, int W);
cudaError_t led_prepare(int m, int C, int W);
// pdl: allow programmatic dependent launch after the previous kernel in the stream.
cudaError_t launch_led(int m, int C, const LedArgs& a, cudaStream_t s, bool pdl);
cudaError_t launch_update(const UpdArgs& a, cudaStream_t s, bool pdl);

// Enqueue a copy of the handle's running FP64 loss sum into pinned host
// memory, ordered after all earlier work of the handle on its caller stream.
int engine_snapshot_loss(fpm_handle* h, double* pinned);

// Several jobs in one launch (the serving loop's rounds): cluster q of the
// per-LED launch takes slot map[q].y of job map[q].x, CTA q of the update
// launch is CTA map[q].y of job map[q].x's update.
cudaError_t launch_led_jobs(int m, int C, const LedArgs* jobs, const int2* map, int n_clusters, int W_max,
                            cudaStream_t s, bool pdl, bool ff);  // ff: some job holds a free-form pupil field
// Jobs of several low-res sizes in one launch: map[b] = (job, slot, rank among
// the LED's CTAs, m) for each of n_ctas CTAs (a multiple of LED_MIX_CLUSTER;
// job < 0: idle); smem = the largest led_mixed_smem_bytes of the jobs.
int led_mixed_cluster(int m);  // CTAs per LED in the mixed launch, 0 if m is not offered there
size_t led_mixed_smem_bytes(int m, int W);
bool led_mixed_fits(int m, int W);  // the mixed launch can hold an LED of size m and box W
cudaError_t led_mixed_prepare();
cudaError_t launch_led_mixed(const LedArgs* jobs, const int4* map, int n_ctas, size_t smem, cudaStream_t s, bool pdl,
                             bool ff);
cudaError_t launch_update_jobs(const UpdArgs* jobs, const int2* map, int n_ctas, int B_max, cudaStream_t s,
                               bool pdl, int opt);  // opt: the optimiser of every job, or -1 if they differ
int update_ctas(const UpdArgs& a);  // CTAs of one job's update launch

// A handle as seen by the serving loop.
struct EngineRound {
  int m, C, W, n_leds, fft;     // kernel configuration; fft: FP32 FFT form (groupable)
  int4* slots;                  // device: batch slots of the round's steps
  float4* coef;                 // device: optimiser coefficients per step (see UpdArgs)
  double* losses;               // device: batch loss per step
  double* epoch;                // device: running FP64 loss sum
};
// Reserve device room for n_steps steps of at most B slots and describe the handle.
int engine_round_reserve(fpm_handle* h, int n_steps, int B, EngineRound* out);
// Host side of one round: slot tables for idx[0..count), and the optimiser
// coefficients of the next n_steps steps (advancing the handle's step count).
void engine_round_slots(const fpm_handle* h, const int32_t* idx, int count, int4* dst);
void engine_round_coef(fpm_handle* h, int n_steps, float4* dst);
// Launch arguments of one step of the handle (built-in loss, updating).
LedArgs engine_led_args(fpm_handle* h, const int4* slot_dev, int B);
UpdArgs engine_upd_args(fpm_handle* h, const int4* slot_dev, int B, int step_off, double* loss_slot);

// Message returned by fpm_last_error(NULL) (calls that have no handle).
void set_unbound_error(const char* msg);

// Tensor-core DFT form of the per-LED kernel (gemm_led.cu). Every operand of
// the four contractions is stored in K-step slices (see tc.cuh): the constant
// DFT factors once per handle, the per-LED data operands in a scratch area
// per batch slot. Sizes in bytes.
struct GemmPlan {
  int prec = 0, tf32 = 0, split = 0, e = 2;  // element bytes e: 2 (BF16) or 4 (TF32)
  int m = 0, W = 0, h = 0, Wp = 0;           // box width W padded to Wp (multiple of 16)
  int YT = 0, ntile = 0;                     // image rows per tile (<= 128), tiles
  int X = 0, nchunk = 0;                     // image columns per chunk, chunks
  int ks1 = 0, ks3 = 0, ks4 = 0;             // K-steps of contractions 1 and 2, 3, 4
  size_t S1 = 0, S2 = 0, S3 = 0, S4 = 0;     // one hi copy of each constant block
  size_t c2_base = 0, c3_base = 0, c4_base = 0, const_bytes = 0;
  size_t SP = 0, SA = 0, SB = 0, SU = 0;     // one hi copy of each data operand
  size_t o_phi = 0, o_at = 0, o_bg = 0, o_au = 0, o_spill = 0, slot_bytes = 0;
  int ns = 0, kps = 0;                       // pipeline stages, K-steps per stage
  int ncta = 1;                              // CTAs per LED (a cluster of 2 at m = 256), scratch slots per LED
  size_t stage = 0, aux = 0, smem = 0;       // stage bytes, staging area of per-pixel inputs
};

// 0 if the form is available for this size, else an FPM_ERR_* code with why.
int gemm_plan(int m, int W, int h, int prec, GemmPlan* p, const char** why);
// The constant DFT factors of a plan (host bytes, laid out for the device).
std::vector<unsigned char> gemm_constants(const GemmPlan& p);
cudaError_t gemm_prepare(const GemmPlan& p);
cudaError_t launch_led_gemm(const GemmPlan& p, const LedArgs& a, const unsigned char* consts,
                            unsigned char* scratch, cudaStream_t s, bool pdl);

// Shared-memory carveout and attributes of the update kernel (call once).
cudaError_t update_prepare();

// Field kernels (initialisation, object transforms, layout changes).
cudaError_t launch_amplitude(const float* I, float* amp, size_t n, cudaStream_t st);
cudaError_t launch_upsample_centre(const float* I, int m, int s, float2* out_rowmajor, cudaStream_t st);
cudaError_t launch_fft_rows(float2* data, int N, const float2* twN, int dir, cudaStream_t st);
cudaError_t launch_fft_cols_centre(const float2* rows, float2* Ot, int N, const float2* twN, float scale,
                                   cudaStream_t st);
cudaError_t launch_transpose(const float2* in, float2* out, int N, cudaStream_t st);

}  // namespace fpmk

// Host side of the Batch-FPM engine: the C ABI declared in include/fpm.h.
//
// All device work of a handle runs on an internal non-blocking stream that is
// joined to the caller's stream at entry and exit of every call (event
// record/wait), so work stays ordered with the caller's stream while the
// engine can capture CUDA graphs even when the caller uses the legacy default
// stream. Multi-step runs are captured once per (n_steps, B) as a graph whose
// first nodes copy the batch schedule and the Adam step count from pinned
// staging buffers, followed by two kernels per step (fused per-LED forward
// and adjoint, then the batch-ordered gather with Adam).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fpm.h"
#include "internal.h"
#include "optcoef.h"

using namespace fpmk;

namespace {
thread_local std::string g_create_error;
}

void fpmk::set_unbound_error(const char* msg) { g_create_error = msg; }

struct fpm_handle {
  int N = 0, m = 0, n = 0, s = 0, h = 0, W = 0, C = 0;
  float R = 0.f, lambda = 0.f, dk = 0.f;
  int edge = 0;
  int centre = 0;
  std::vector<float> nominal;
  std::vector<int2> nint_h;
  std::vector<float> sp0;  // initial scalar parameters
  int x_lo = 0, n_cols = 0;
  cudaStream_t user = nullptr, st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  fpm_hparams hp{};
  // device state
  float2 *Ot = nullptr, *mO = nullptr, *vO = nullptr, *tmp = nullptr, *tmp2 = nullptr;
  float2 *tw_m = nullptr, *tw_N = nullptr;
  float *meas = nullptr, *amp = nullptr, *sp = nullptr, *msp = nullptr, *vsp = nullptr, *gsc = nullptr, *fbuf = nullptr;
  int2 *nint = nullptr, *span = nullptr;
  float2* gbox = nullptr;
  double* part = nullptr;
  int capB = 0;
  int4* sched = nullptr;  // batch slots (LED, n_row, n_col, 0) of the current run
  int cap_sched = 0;
  double* losses = nullptr;
  int cap_losses = 0;
  size_t cap_fbuf = 0;
  double* epoch = nullptr;
  float4* coef = nullptr;  // per-step optimiser coefficients of the current run
  int cap_coef = 0;
  int* err = nullptr;
  // pinned staging of handle-free copies
  int* h_err = nullptr;
  long long t_host = 0;
  // NAdam's product of momentum coefficients P_t for t = nadam_t (with beta1 = nadam_b1)
  long long nadam_t = 0;
  double nadam_prod = 1.0;
  float nadam_b1 = -1.f;
  bool loaded = false;
  // One captured graph per (n_steps, B), each with its own pinned staging for
  // the batch slots and Adam coefficients its first nodes copy, and an event
  // marking the end of its last launch: different graphs of a handle can be
  // queued back to back without waiting on the host.
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int4* h_slots = nullptr;
    float4* h_coef = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::map<std::pair<int, int>, Graph> graphs;
  std::string msg;
  // tensor-core DFT form (hp.precision != FPM_PRECISION_FP32_FFT)
  GemmPlan gp;
  unsigned char* gconst = nullptr;  // constant DFT factors of gp
  unsigned char* gscr = nullptr;    // per-slot scratch, capacity cap_gscr slots
  int cap_gscr = 0;
  // dataflow form of the step (m = 256, FP32 FFT form): scratch for capB slots
  int step_form = FPM_STEP_AUTO;
  float2* T = nullptr;         // [capB][W][256]
  double* partB = nullptr;     // [capB][nB][STEP_NPB]
  double* partC = nullptr;     // [capB][nC][STEP_NPC]
  StepSync* sync = nullptr;    // zero between launches
  int step_ctas = 0;           // CTAs that fit at once (for capB)
  long long wait_ns = 200000000LL;  // bound of the kernels' dependency waits
  // free-form pupil: node field on the box grid [W][W] (column-major by box
  // column), its moments, its gradient (fpm_backward), per-LED gradient boxes
  // and placements; pupil_on: the field takes part in the model
  float2 *Pff = nullptr, *mPff = nullptr, *vPff = nullptr, *gPff = nullptr, *pbox = nullptr;
  float4* pwt = nullptr;
  bool pupil_on = false;
  // device memory of the handle (every buffer goes through dalloc / dfree)
  int64_t mem_used = 0, mem_limit = 0;  // limit <= 0: none
  std::map<void*, size_t> mem_sizes;
};

namespace {

int fail(fpm_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->msg = buf;
  else g_create_error = buf;
  return code;
}

// Device memory of a handle: each buffer is allocated and freed through these,
// so the handle knows its footprint and can refuse to grow past its limit
// (fpm_set_memory_limit) before any buffer is touched.
size_t mem_of(const fpm_handle* h, const void* p) {
  const auto it = h->mem_sizes.find(const_cast<void*>(p));
  return it == h->mem_sizes.end() ? 0 : it->second;
}
bool mem_fits(const fpm_handle* h, size_t freed, size_t added) {
  return h->mem_limit <= 0 || (int64_t)(h->mem_used - (int64_t)freed + (int64_t)added) <= h->mem_limit;
}
// Buffers are stream-ordered allocations from the device's memory pool on the
// handle's stream (cudaMallocAsync / cudaFreeAsync), which unlike cudaFree do
// not synchronise the whole device: a serving process that admits and retires
// jobs does not stall the jobs still running. The pool keeps freed memory for
// reuse (release threshold raised once per device in this process).
void keep_pool_memory() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(mu);
  for (int d : done)
    if (d == dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done.push_back(dev);
}

template <class T>
cudaError_t dalloc(fpm_handle* h, T** p, size_t bytes) {
  if (!mem_fits(h, 0, bytes)) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMallocAsync((void**)p, bytes, h->st);
  if (e == cudaSuccess) {
    h->mem_used += (int64_t)bytes;
    h->mem_sizes[(void*)*p] = bytes;
  }
  return e;
}
template <class T>
cudaError_t dfree(fpm_handle* h, T*& p) {
  if (!p) return cudaSuccess;
  const auto it = h->mem_sizes.find((void*)p);
  if (it != h->mem_sizes.end()) {
    h->mem_used -= (int64_t)it->second;
    h->mem_sizes.erase(it);
  }
  const cudaError_t e = cudaFreeAsync((void*)p, h->st);
  p = nullptr;
  return e;
}

#define CK(h, call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail((h), e_ == cudaErrorMemoryAllocation ? FPM_ERR_OOM : FPM_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool is_pageable_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeUnregistered;
}

void destroy_graphs(fpm_handle* h) {
  for (auto& kv : h->graphs) {
    if (kv.second.done) cudaEventSynchronize(kv.second.done);
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.h_slots) cudaFreeHost(kv.second.h_slots);
    if (kv.second.h_coef) cudaFreeHost(kv.second.h_coef);
    if (kv.second.done) cudaEventDestroy(kv.second.done);
  }
  h->graphs.clear();
}

void free_all(fpm_handle* h) {
  destroy_graphs(h);
  for (auto& kv : h->mem_sizes) cudaFreeAsync(kv.first, h->st);  // every device buffer of the handle
  h->mem_sizes.clear();
  h->mem_used = 0;
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->st) cudaStreamDestroy(h->st);
}

// Order the internal stream after the caller's stream.
int enter(fpm_handle* h) {
  CK(h, cudaEventRecord(h->ev_in, h->user));
  CK(h, cudaStreamWaitEvent(h->st, h->ev_in, 0));
  return FPM_OK;
}
// Order the caller's stream after the internal stream.
int leave(fpm_handle* h) {
  CK(h, cudaEventRecord(h->ev_out, h->st));
  CK(h, cudaStreamWaitEvent(h->user, h->ev_out, 0));
  return FPM_OK;
}

// Read and clear the device error flag (synchronises the internal stream).
int check_device_error(fpm_handle* h) {
  CK(h, cudaMemcpyAsync(h->h_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  const int e = *h->h_err;
  if (e) {
    CK(h, cudaMemsetAsync(h->err, 0, sizeof(int), h->st));
    // a launch whose waits gave up may have left its counters non-zero
    if (h->sync) CK(h, cudaMemsetAsync(h->sync, 0, sizeof(StepSync), h->st));
    if (e & DERR_NONFINITE) return fail(h, FPM_ERR_NONFINITE, "a batch loss was not finite");
    if (e & DERR_TIMEOUT) return fail(h, FPM_ERR_TIMEOUT, "a bounded wait in a kernel gave up");
    if (e & DERR_OFFSET) return fail(h, FPM_ERR_RANGE, "an LED offset lies outside +-%.2f px", (double)FPM_OFFSET_BOUND_PX);
    return fail(h, FPM_ERR_RANGE, "a kernel saw an LED index out of range");
  }
  return FPM_OK;
}

std::vector<float2> twiddles(int n) {
  std::vector<float2> t(n);
  for (int i = 0; i < n; ++i) {
    const double a = -2.0 * M_PI * (double)i / (double)n;
    t[i] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  return t;
}

int validate_batches(fpm_handle* h, const int32_t* idx, int n_steps, int B) {
  if (!idx) return fail(h, FPM_ERR_ARG, "null batch index pointer");
  if (B < 1 || B > h->n || B > MAX_BATCH) return fail(h, FPM_ERR_SHAPE, "batch size %d outside [1, %d]", B, h->n);
  std::vector<int> seen(h->n, -1);
  for (int s = 0; s < n_steps; ++s)
    for (int b = 0; b < B; ++b) {
      const int i = idx[(size_t)s * B + b];
      if (i < 0 || i >= h->n) return fail(h, FPM_ERR_RANGE, "LED index %d outside [0, %d)", i, h->n);
      if (seen[i] == s) return fail(h, FPM_ERR_RANGE, "LED index %d repeated in batch %d", i, s);
      seen[i] = s;
    }
  return FPM_OK;
}

int over_limit(fpm_handle* h, size_t freed, size_t added) {
  return fail(h, FPM_ERR_OOM, "the handle's device-memory limit of %lld bytes would be exceeded (%lld in use, "
              "%zu more asked for)", (long long)h->mem_limit, (long long)h->mem_used, added - freed);
}

template <class T>
int grow(fpm_handle* h, T** p, int* cap, int need) {
  if (*cap >= need) return FPM_OK;
  if (!mem_fits(h, mem_of(h, *p), sizeof(T) * (size_t)need)) return over_limit(h, mem_of(h, *p), sizeof(T) * (size_t)need);
  CK(h, dfree(h, *p));
  *cap = 0;
  CK(h, dalloc(h, p, sizeof(T) * (size_t)need));
  *cap = need;
  destroy_graphs(h);  // graphs hold the old address
  return FPM_OK;
}

// The optimiser's per-step coefficients for steps t = t_host + 1 .. t_host +
// n_steps, in FP64, into dst (host); the layout per optimiser is UpdArgs::coef's.
// NAdam's momentum coefficient mu_t = b1 (1 - 0.96^(0.004 t) / 2) and the running
// product P_t = mu_1 ... mu_t (kept on the handle, rebuilt when the step count
// moves back or beta1 changes).
void fill_coef(fpm_handle* h, int n_steps, float4* dst) {
  const double b1 = h->hp.beta1, b2 = h->hp.beta2;
  const int opt = h->hp.optimizer;
  if (opt == FPM_OPT_NADAM) {
    if (h->nadam_t > h->t_host || h->nadam_b1 != h->hp.beta1) {
      h->nadam_t = 0;
      h->nadam_prod = 1.0;
      h->nadam_b1 = h->hp.beta1;
    }
    h->nadam_prod = nadam_advance(b1, h->nadam_t, h->nadam_prod, h->t_host);
    h->nadam_t = h->t_host;
  }
  double prod = h->nadam_prod;  // P at t_host (NAdam)
  for (int s = 0; s < n_steps; ++s) {
    float k[4];
    prod = opt_coefficients(opt, b1, b2, h->t_host + s + 1, prod, k);
    dst[s] = make_float4(k[0], k[1], k[2], k[3]);
  }
}

// Tasks per LED of the dataflow step: column tasks of at most 8 box columns,
// row tasks of 8 image rows.
int step_nA(const fpm_handle* h) { return (h->W + 7) / 8; }
int step_nB() { return 256 / 8; }

// The dataflow step kernel serves the FP32 FFT form at m = 256 when asked for.
bool uses_step(const fpm_handle* h) {
  return h->sync && h->hp.precision == FPM_PRECISION_FP32_FFT && h->step_form == FPM_STEP_DATAFLOW;
}

int ensure_batch(fpm_handle* h, int B) {
  if (h->hp.precision != FPM_PRECISION_FP32_FFT && h->cap_gscr < B) {
    const size_t add = h->gp.slot_bytes * (size_t)h->gp.ncta * (size_t)B;
    if (!mem_fits(h, mem_of(h, h->gscr), add)) return over_limit(h, mem_of(h, h->gscr), add);
    CK(h, dfree(h, h->gscr));
    h->cap_gscr = 0;
    CK(h, dalloc(h, &h->gscr, add));
    h->cap_gscr = B;
    destroy_graphs(h);
  }
  if (h->capB >= B) return FPM_OK;
  const size_t sz_box = sizeof(float2) * (size_t)B * h->W * h->W;
  // (room for the serving loop's mixed-size launch too, whose split of an LED may be finer)
  const size_t sz_part = sizeof(double) * (size_t)B * std::max(h->C, led_mixed_cluster(h->m)) * NPART;
  const size_t sz_T = h->sync ? sizeof(float2) * (size_t)B * h->W * 256 : 0;
  const size_t sz_pB = h->sync ? sizeof(double) * (size_t)B * step_nB() * STEP_NPB : 0;
  const size_t sz_pC = h->sync ? sizeof(double) * (size_t)B * step_nA(h) * STEP_NPC : 0;
  const size_t sz_pbox = sz_box, sz_pwt = sizeof(float4) * (size_t)B;
  const size_t freed = mem_of(h, h->gbox) + mem_of(h, h->part) + mem_of(h, h->T) + mem_of(h, h->partB) +
                       mem_of(h, h->partC) + mem_of(h, h->pbox) + mem_of(h, h->pwt);
  const size_t added = sz_box + sz_part + sz_T + sz_pB + sz_pC + sz_pbox + sz_pwt;
  if (!mem_fits(h, freed, added)) return over_limit(h, freed, added);
  CK(h, dfree(h, h->gbox));
  CK(h, dfree(h, h->part));
  CK(h, dfree(h, h->T));
  CK(h, dfree(h, h->partB));
  CK(h, dfree(h, h->partC));
  CK(h, dfree(h, h->pbox));
  CK(h, dfree(h, h->pwt));
  h->capB = 0;
  CK(h, dalloc(h, &h->gbox, sz_box));
  CK(h, dalloc(h, &h->part, sz_part));
  CK(h, dalloc(h, &h->pbox, sz_pbox));
  CK(h, dalloc(h, &h->pwt, sz_pwt));
  if (h->sync) {  // the dataflow form (m = 256)
    CK(h, dalloc(h, &h->T, sz_T));
    CK(h, dalloc(h, &h->partB, sz_pB));
    CK(h, dalloc(h, &h->partC, sz_pC));
    CK(h, step_prepare(h->W, B, &h->step_ctas));
  }
  h->capB = B;
  destroy_graphs(h);
  return FPM_OK;
}

int ensure_fbuf(fpm_handle* h, size_t floats) {
  if (h->cap_fbuf >= floats) return FPM_OK;
  if (!mem_fits(h, mem_of(h, h->fbuf), sizeof(float) * floats))
    return over_limit(h, mem_of(h, h->fbuf), sizeof(float) * floats);
  CK(h, dfree(h, h->fbuf));
  h->cap_fbuf = 0;
  CK(h, dalloc(h, &h->fbuf, sizeof(float) * floats));
  h->cap_fbuf = floats;
  return FPM_OK;
}

// Batch slots for LED indices idx[0..count): (LED, crop row, crop col, 0).
void fill_slots(const fpm_handle* h, const int32_t* idx, int count, int4* dst) {
  for (int q = 0; q < count; ++q) {
    const int i = idx[q];
    dst[q] = make_int4(i, h->nint_h[i].x, h->nint_h[i].y, 0);
  }
}

LedArgs led_args(fpm_handle* h, const int4* slot_dev, int B, int mode) {
  LedArgs a{};
  a.Ot = h->Ot;
  // the FFT form's amplitude loss reads the amplitudes computed at load
  a.meas_is_amp = mode == MODE_LOSS && h->hp.loss == FPM_LOSS_AMPLITUDE && h->hp.precision == FPM_PRECISION_FP32_FFT;
  a.meas = a.meas_is_amp ? h->amp : h->meas;
  a.sp = h->sp;
  a.slot = slot_dev;
  a.gbox = h->gbox;
  a.part = h->part;
  a.tw = h->tw_m;
  a.N = h->N;
  a.n_leds = h->n;
  a.B = B;
  a.h = h->h;
  a.W = h->W;
  a.R = h->R;
  a.Rinv = 1.f / h->R;
  a.inv_lambda = 1.f / h->lambda;
  a.dk2 = h->dk * h->dk;
  a.hard_edge = h->edge == FPM_EDGE_HARD;
  a.loss = h->hp.loss;
  a.mode = mode;
  a.err = h->err;
  a.pupil = h->pupil_on ? h->Pff : nullptr;
  a.pbox = h->pbox;
  a.pwt = h->pwt;
  return a;
}

// The per-LED kernel of the handle's precision mode.
cudaError_t launch_led_mode(fpm_handle* h, const LedArgs& a, bool pdl) {
  if (h->hp.precision != FPM_PRECISION_FP32_FFT) return launch_led_gemm(h->gp, a, h->gconst, h->gscr, h->st, pdl);
  return launch_led(h->m, h->C, a, h->st, pdl);
}

UpdArgs upd_args(fpm_handle* h, const int4* slot_dev, int B, int step_off, double* loss_slot, int assemble) {
  UpdArgs u{};
  u.Ot = h->Ot;
  u.mO = h->mO;
  u.vO = h->vO;
  u.sp = h->sp;
  u.msp = h->msp;
  u.vsp = h->vsp;
  u.gbox = h->gbox;
  u.part = h->part;
  u.slot = slot_dev;
  u.span = h->span;
  u.x_lo = h->x_lo;
  u.n_cols = h->n_cols;
  u.N = h->N;
  u.n_leds = h->n;
  u.B = B;
  u.C = h->hp.precision != FPM_PRECISION_FP32_FFT ? h->gp.ncta : h->C;  // partials per LED
  u.h = h->h;
  u.W = h->W;
  u.lr_obj = h->hp.lr_object;
  u.lr_zern = h->hp.lr_zernike;
  u.lr_def = h->hp.lr_defocus;
  u.lr_gam = h->hp.lr_gamma;
  u.lr_off = h->hp.lr_offset;
  u.b1 = h->hp.beta1;
  u.b2 = h->hp.beta2;
  u.eps = h->hp.eps;
  u.opt = h->hp.optimizer;
  u.wd = h->hp.weight_decay;
  u.offset_bound = FPM_OFFSET_BOUND_PX;
  u.coef = assemble ? nullptr : h->coef;
  u.step_off = step_off;
  u.learn = h->hp.learn_mask;
  u.loss_slot = loss_slot;
  u.epoch_loss = h->epoch;
  u.err = h->err;
  u.assemble = assemble;
  u.g_obj = h->tmp;
  u.g_sc = h->gsc;
  u.Pff = h->Pff;
  u.mPff = h->mPff;
  u.vPff = h->vPff;
  u.pbox = h->pbox;
  u.pwt = h->pwt;
  u.g_pupil = h->gPff;
  u.lr_pupil = h->hp.lr_pupil;
  u.pupil_cols = h->pupil_on ? h->W : 0;
  return u;
}

StepArgs step_args(fpm_handle* h, const LedArgs& a, const UpdArgs* u) {
  StepArgs s{};
  s.L = a;
  if (u) s.U = *u;
  s.T = h->T;
  s.partB = h->partB;
  s.partC = h->partC;
  s.sync = h->sync;
  s.nA = step_nA(h);
  s.nB = step_nB();
  s.nC = s.nA;
  s.do_update = u != nullptr;
  s.wait_ns = h->wait_ns;
  s.stall = 0;
  return s;
}

// One step (built-in loss, updating) in the handle's form.
cudaError_t launch_train_step(fpm_handle* h, const int4* idx, int B, int step_off, double* loss_slot, bool pdl,
                              bool split_update = false) {
  const LedArgs a = led_args(h, idx, B, MODE_LOSS);
  const UpdArgs u = upd_args(h, idx, B, step_off, loss_slot, 0);
  if (uses_step(h)) return launch_step(step_args(h, a, &u), h->step_ctas, h->st, pdl);
  cudaError_t e = launch_led_mode(h, a, pdl);
  if (e == cudaSuccess && !split_update) e = launch_update(u, h->st, true);
  return e;
}

int reset_state(fpm_handle* h) {
  const size_t NN = (size_t)h->N * h->N;
  CK(h, cudaMemsetAsync(h->mO, 0, sizeof(float2) * NN, h->st));
  CK(h, cudaMemsetAsync(h->vO, 0, sizeof(float2) * NN, h->st));
  const int P = sp_size(h->n);
  CK(h, cudaMemcpyAsync(h->sp, h->sp0.data(), sizeof(float) * P, cudaMemcpyHostToDevice, h->st));
  CK(h, cudaMemsetAsync(h->msp, 0, sizeof(float) * P, h->st));
  CK(h, cudaMemsetAsync(h->vsp, 0, sizeof(float) * P, h->st));
  CK(h, cudaMemsetAsync(h->epoch, 0, sizeof(double), h->st));
  const size_t WW = (size_t)h->W * h->W;
  const std::vector<float2> ones(WW, make_float2(1.f, 0.f));
  CK(h, cudaMemcpyAsync(h->Pff, ones.data(), sizeof(float2) * WW, cudaMemcpyHostToDevice, h->st));
  CK(h, cudaMemsetAsync(h->mPff, 0, sizeof(float2) * WW, h->st));
  CK(h, cudaMemsetAsync(h->vPff, 0, sizeof(float2) * WW, h->st));
  CK(h, cudaStreamSynchronize(h->st));  // (the host vector above)
  h->t_host = 0;
  return FPM_OK;
}

// real-space object (row-major, in tmp) -> centred spectrum in Ot
int object_from_field(fpm_handle* h) {
  CK(h, launch_fft_rows(h->tmp, h->N, h->tw_N, -1, h->st));
  CK(h, launch_fft_cols_centre(h->tmp, h->Ot, h->N, h->tw_N, 1.f / (float)(h->s * h->s), h->st));
  return FPM_OK;
}

int copy_out(fpm_handle* h, void* dst, const void* src, size_t bytes, bool* host_dst) {
  if (!dst) return FPM_OK;
  if (!is_device_ptr(dst)) *host_dst = true;
  CK(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->st));
  return FPM_OK;
}

int build_graph(fpm_handle* h, int n_steps, int B, fpm_handle::Graph* gr) {
  CK(h, cudaMallocHost(&gr->h_slots, sizeof(int4) * (size_t)n_steps * B));
  CK(h, cudaMallocHost(&gr->h_coef, sizeof(float4) * (size_t)n_steps));
  CK(h, cudaEventCreateWithFlags(&gr->done, cudaEventDisableTiming));
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemcpyAsync(h->sched, gr->h_slots, sizeof(int4) * (size_t)n_steps * B,
                                  cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->coef, gr->h_coef, sizeof(float4) * n_steps, cudaMemcpyHostToDevice, h->st);
  // kernels after the first may start early (programmatic dependent launch)
  // and wait in-kernel for their predecessor's results
  for (int s = 0; s < n_steps && e == cudaSuccess; ++s)
    e = launch_train_step(h, h->sched + (size_t)s * B, B, s, h->losses + s, s > 0);
  cudaError_t e2 = cudaStreamEndCapture(h->st, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(h, FPM_ERR_CUDA, "graph capture failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&gr->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, FPM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  return FPM_OK;
}

}  // namespace

namespace {
int forward_impl(fpm_handle* h, const int32_t* idx, int32_t B, float* I_out, float2* psi_out);
int backward_impl(fpm_handle* h, const int32_t* idx, int32_t B, const float* dL_dI, const float2* psi,
                  float* g_object, float* g_zernike, float* g_defocus, float* g_gamma, float* g_offset,
                  double* loss_out);
}  // namespace

int fpmk::engine_round_reserve(fpm_handle* h, int n_steps, int B, EngineRound* out) {
  if (!h || !out || n_steps < 1 || B < 1) return FPM_ERR_ARG;
  if (!h->loaded) return fail(h, FPM_ERR_STATE, "no stack loaded");
  int rc;
  if ((rc = ensure_batch(h, B))) return rc;
  if ((rc = grow(h, &h->sched, &h->cap_sched, n_steps * B))) return rc;
  if ((rc = grow(h, &h->losses, &h->cap_losses, n_steps))) return rc;
  if ((rc = grow(h, &h->coef, &h->cap_coef, n_steps))) return rc;
  out->m = h->m;
  out->C = h->hp.precision != FPM_PRECISION_FP32_FFT ? h->gp.ncta : h->C;
  out->W = h->W;
  out->n_leds = h->n;
  // rounds group jobs of the per-LED cluster form; a job in the dataflow form
  // (m = 256) runs its own epochs, so its arithmetic is the same alone or not
  out->fft = h->hp.precision == FPM_PRECISION_FP32_FFT && !uses_step(h);
  out->slots = h->sched;
  out->coef = h->coef;
  out->losses = h->losses;
  out->epoch = h->epoch;
  return FPM_OK;
}

void fpmk::engine_round_slots(const fpm_handle* h, const int32_t* idx, int count, int4* dst) {
  fill_slots(h, idx, count, dst);
}

void fpmk::engine_round_coef(fpm_handle* h, int n_steps, float4* dst) {
  fill_coef(h, n_steps, dst);
  h->t_host += n_steps;
}

LedArgs fpmk::engine_led_args(fpm_handle* h, const int4* slot_dev, int B) {
  return led_args(h, slot_dev, B, MODE_LOSS);
}

UpdArgs fpmk::engine_upd_args(fpm_handle* h, const int4* slot_dev, int B, int step_off, double* loss_slot) {
  return upd_args(h, slot_dev, B, step_off, loss_slot, 0);
}

int fpmk::engine_snapshot_loss(fpm_handle* h, double* pinned) {
  int rc = enter(h);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(pinned, h->epoch, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  return leave(h);
}

extern "C" {

int fpm_create(const fpm_geometry* g, float R, int32_t upsample, void* cuda_stream, fpm_handle** out) {
  g_create_error.clear();
  if (!g || !out || !g->led_offset) return fail(nullptr, FPM_ERR_ARG, "null argument");
  *out = nullptr;
  if (led_cluster_size(g->m) == 0) return fail(nullptr, FPM_ERR_SHAPE, "m=%d not in {32, 64, 128, 256, 512}", g->m);
  if (upsample < 1 || (long long)g->m * upsample > 8192 || (upsample & (upsample - 1)))
    return fail(nullptr, FPM_ERR_SHAPE, "upsample=%d must be a power of two with m*upsample <= 8192", upsample);
  if (g->n_leds < 1 || g->n_leds > 1024) return fail(nullptr, FPM_ERR_SHAPE, "n_leds=%d outside [1, 1024]", g->n_leds);
  if (!(R > 0.f) || !(g->lambda_um > 0.f) || !(g->dk_per_um > 0.f))
    return fail(nullptr, FPM_ERR_ARG, "radius, wavelength and spectral bin must be positive");
  if (g->pupil_edge != FPM_EDGE_AA && g->pupil_edge != FPM_EDGE_HARD)
    return fail(nullptr, FPM_ERR_ARG, "unknown pupil edge %d", g->pupil_edge);
  fpm_handle* h = new fpm_handle();
  h->m = g->m;
  h->s = upsample;
  h->N = g->m * upsample;
  h->n = g->n_leds;
  h->R = R;
  h->lambda = g->lambda_um;
  h->dk = g->dk_per_um;
  h->edge = g->pupil_edge;
  h->user = (cudaStream_t)cuda_stream;
  h->C = led_cluster_size(h->m);  // refined once a device is available
  h->h = (int)std::floor((double)R + 0.5 + std::sqrt(2.0) * FPM_OFFSET_BOUND_PX) + 1;
  h->W = 2 * h->h + 1;
  auto bad = [&](int code, const char* why) {
    g_create_error = why;
    delete h;
    return code;
  };
  if (2 * h->h >= h->m) return bad(FPM_ERR_SHAPE, "pupil box does not fit the low-res window (2h >= m)");
  if ((double)(R + 2.f) * g->dk_per_um * g->lambda_um >= 1.0)
    return bad(FPM_ERR_SHAPE, "pupil reaches evanescent frequencies (radius * dk * lambda >= 1)");
  h->nominal.assign(g->led_offset, g->led_offset + 2 * (size_t)h->n);
  h->nint_h.resize(h->n);
  h->sp0.assign(sp_size(h->n), 0.f);
  double best = 1e300;
  int lo_x = h->N, hi_x = -1;
  std::vector<int2> span(h->N, make_int2(h->N, 0));
  for (int i = 0; i < h->n; ++i) {
    const double r = h->nominal[2 * i], c = h->nominal[2 * i + 1];
    if (!std::isfinite(r) || !std::isfinite(c)) return bad(FPM_ERR_ARG, "non-finite LED offset");
    const int ri = (int)std::nearbyint(r), ci = (int)std::nearbyint(c);
    h->nint_h[i] = make_int2(ri, ci);
    h->sp0[sp_offset(h->n) + 2 * i] = (float)(r - ri);
    h->sp0[sp_offset(h->n) + 2 * i + 1] = (float)(c - ci);
    const int r0 = h->N / 2 + ri - h->h, c0 = h->N / 2 + ci - h->h;
    if (r0 < 0 || c0 < 0 || r0 + h->W > h->N || c0 + h->W > h->N)
      return bad(FPM_ERR_SHAPE, "an LED crop box leaves the high-res spectrum");
    for (int x = c0; x < c0 + h->W; ++x) {
      span[x].x = std::min(span[x].x, r0);
      span[x].y = std::max(span[x].y, r0 + h->W);
    }
    lo_x = std::min(lo_x, c0);
    hi_x = std::max(hi_x, c0 + h->W);
    const double d = std::hypot(r, c);
    if (d < best) {
      best = d;
      h->centre = i;
    }
  }
  for (int i = 0; i < h->n; ++i) h->sp0[SP_GAMMA + i] = 1.f;
  h->x_lo = lo_x;
  h->n_cols = hi_x - lo_x;
  h->hp.lr_object = 0.1f;
  h->hp.lr_zernike = 0.01f;
  h->hp.lr_defocus = 0.1f;
  h->hp.lr_gamma = 0.01f;
  h->hp.lr_offset = 0.01f;
  h->hp.lr_pupil = 0.01f;
  h->hp.beta1 = 0.9f;
  h->hp.beta2 = 0.999f;
  h->hp.eps = 1e-8f;
  h->hp.loss = FPM_LOSS_AMPLITUDE;
  h->hp.learn_mask = FPM_LEARN_OBJECT;
  h->hp.precision = FPM_PRECISION_FP32_FFT;
  h->hp.optimizer = FPM_OPT_ADAM;
  h->hp.weight_decay = 0.f;

  auto ck = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    g_create_error = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
  };
  const size_t NN = (size_t)h->N * h->N;
  const int P = sp_size(h->n);
  keep_pool_memory();
  bool ok = ck(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking), "stream") &&
            ck(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming), "event") &&
            ck(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming), "event") &&
            ck(dalloc(h, &h->Ot, sizeof(float2) * NN), "alloc O") &&
            ck(dalloc(h, &h->mO, sizeof(float2) * NN), "alloc m") &&
            ck(dalloc(h, &h->vO, sizeof(float2) * NN), "alloc v") &&
            ck(dalloc(h, &h->tmp, sizeof(float2) * NN), "alloc tmp") &&
            ck(dalloc(h, &h->tmp2, sizeof(float2) * NN), "alloc tmp2") &&
            ck(dalloc(h, &h->tw_m, sizeof(float2) * h->m), "alloc tw") &&
            ck(dalloc(h, &h->tw_N, sizeof(float2) * h->N), "alloc tw") &&
            ck(dalloc(h, &h->meas, sizeof(float) * (size_t)h->n * h->m * h->m), "alloc stack") &&
            ck(dalloc(h, &h->amp, sizeof(float) * (size_t)h->n * h->m * h->m), "alloc stack") &&
            ck(dalloc(h, &h->sp, sizeof(float) * P), "alloc params") &&
            ck(dalloc(h, &h->msp, sizeof(float) * P), "alloc params") &&
            ck(dalloc(h, &h->vsp, sizeof(float) * P), "alloc params") &&
            ck(dalloc(h, &h->gsc, sizeof(float) * P), "alloc params") &&
            ck(dalloc(h, &h->nint, sizeof(int2) * h->n), "alloc leds") &&
            ck(dalloc(h, &h->span, sizeof(int2) * h->N), "alloc span") &&
            ck(dalloc(h, &h->epoch, sizeof(double)), "alloc") &&
            ck(dalloc(h, &h->err, sizeof(int)), "alloc") &&
            ck(dalloc(h, &h->Pff, sizeof(float2) * (size_t)h->W * h->W), "alloc pupil") &&
            ck(dalloc(h, &h->mPff, sizeof(float2) * (size_t)h->W * h->W), "alloc pupil") &&
            ck(dalloc(h, &h->vPff, sizeof(float2) * (size_t)h->W * h->W), "alloc pupil") &&
            ck(dalloc(h, &h->gPff, sizeof(float2) * (size_t)h->W * h->W), "alloc pupil") &&
            (h->m != 256 || ck(dalloc(h, &h->sync, sizeof(StepSync)), "alloc")) &&
            ck(cudaMallocHost(&h->h_err, sizeof(int)), "pinned") &&
            ck((h->C = led_choose_cluster(h->m, h->W)) > 0 ? cudaSuccess : cudaErrorNotSupported,
               "this device cannot run the per-LED kernel for this size") &&
            ck(led_prepare(h->m, h->C, h->W), "kernel attributes") &&
            ck(update_prepare(), "kernel attributes") &&
            // the stream-ordered allocations are complete before the copies below
            ck(cudaStreamSynchronize(h->st), "sync");
  if (ok) {
    const auto twm = twiddles(h->m), twN = twiddles(h->N);
    ok = ck(cudaMemcpy(h->tw_m, twm.data(), sizeof(float2) * h->m, cudaMemcpyHostToDevice), "copy") &&
         ck(cudaMemcpy(h->tw_N, twN.data(), sizeof(float2) * h->N, cudaMemcpyHostToDevice), "copy") &&
         ck(cudaMemcpy(h->nint, h->nint_h.data(), sizeof(int2) * h->n, cudaMemcpyHostToDevice), "copy") &&
         ck(cudaMemcpy(h->span, span.data(), sizeof(int2) * h->N, cudaMemcpyHostToDevice), "copy") &&
         ck(cudaMemset(h->Ot, 0, sizeof(float2) * NN), "memset") &&
         ck(cudaMemset(h->err, 0, sizeof(int)), "memset") &&
         (!h->sync || ck(cudaMemset(h->sync, 0, sizeof(StepSync)), "memset"));
  }
  if (ok) ok = reset_state(h) == FPM_OK && ck(cudaStreamSynchronize(h->st), "sync");
  if (!ok) {
    if (g_create_error.empty()) g_create_error = h->msg;
    free_all(h);
    delete h;
    return FPM_ERR_CUDA;
  }
  *out = h;
  return FPM_OK;
}

void fpm_destroy(fpm_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  free_all(h);
  delete h;
}

const char* fpm_last_error(const fpm_handle* h) { return h ? h->msg.c_str() : g_create_error.c_str(); }

int fpm_set_hparams(fpm_handle* h, const fpm_hparams* hp) {
  if (!h || !hp) return fail(h, FPM_ERR_ARG, "null argument");
  if (hp->loss != FPM_LOSS_AMPLITUDE && hp->loss != FPM_LOSS_INTENSITY) return fail(h, FPM_ERR_ARG, "unknown loss");
  if (hp->learn_mask & ~FPM_LEARN_ALL) return fail(h, FPM_ERR_ARG, "unknown learn bits");
  const bool want_pupil = h->pupil_on || (hp->learn_mask & FPM_LEARN_PUPIL);
  if (want_pupil && hp->precision != FPM_PRECISION_FP32_FFT)
    return fail(h, FPM_ERR_ARG, "the free-form pupil needs the FP32 FFT form");
  if (!std::isfinite(hp->lr_pupil)) return fail(h, FPM_ERR_ARG, "non-finite learning rate");
  if (hp->precision < FPM_PRECISION_FP32_FFT || hp->precision > FPM_PRECISION_TF32X3_GEMM)
    return fail(h, FPM_ERR_ARG, "unknown precision mode");
  if (!(hp->beta1 >= 0.f && hp->beta1 < 1.f && hp->beta2 >= 0.f && hp->beta2 < 1.f && hp->eps > 0.f))
    return fail(h, FPM_ERR_ARG, "betas must lie in [0, 1) and eps be positive");
  if (hp->optimizer < FPM_OPT_ADAM || hp->optimizer > FPM_OPT_RMSPROP) return fail(h, FPM_ERR_ARG, "unknown optimiser");
  if (!(std::isfinite(hp->weight_decay) && hp->weight_decay >= 0.f))
    return fail(h, FPM_ERR_ARG, "weight decay must be finite and non-negative");
  const bool lr_ok = std::isfinite(hp->lr_object) && std::isfinite(hp->lr_zernike) &&
                     std::isfinite(hp->lr_defocus) && std::isfinite(hp->lr_gamma) && std::isfinite(hp->lr_offset);
  if (!lr_ok) return fail(h, FPM_ERR_ARG, "non-finite learning rate");
  const bool graph_relevant = hp->loss != h->hp.loss || std::memcmp(hp, &h->hp, sizeof *hp) != 0;
  if (hp->precision != h->hp.precision) {
    // a new DFT form: plan it, build its constant factors, drop the old buffers
    GemmPlan gp;
    if (hp->precision != FPM_PRECISION_FP32_FFT) {
      const char* why = "";
      const int rc = gemm_plan(h->m, h->W, h->h, hp->precision, &gp, &why);
      if (rc) return fail(h, rc, "%s", why);
    }
    CK(h, cudaStreamSynchronize(h->st));  // kernels in flight may still read the old buffers
    destroy_graphs(h);
    CK(h, dfree(h, h->gconst));
    CK(h, dfree(h, h->gscr));
    h->cap_gscr = 0;
    h->gp = gp;
    h->hp.precision = FPM_PRECISION_FP32_FFT;  // until the new form is ready
    if (hp->precision != FPM_PRECISION_FP32_FFT) {
      const std::vector<unsigned char> cst = gemm_constants(gp);
      CK(h, gemm_prepare(gp));
      if (!mem_fits(h, 0, cst.size())) return over_limit(h, 0, cst.size());
      CK(h, dalloc(h, &h->gconst, cst.size()));
      CK(h, cudaMemcpyAsync(h->gconst, cst.data(), cst.size(), cudaMemcpyHostToDevice, h->st));
      CK(h, cudaStreamSynchronize(h->st));
    }
  }
  h->hp = *hp;
  if ((hp->learn_mask & FPM_LEARN_PUPIL) && !h->pupil_on) {
    h->pupil_on = true;  // a learned field enters the model (it starts at 1 after fpm_load's reset)
    destroy_graphs(h);
  }
  if (graph_relevant) destroy_graphs(h);  // the captured kernels hold the hyper-parameters by value
  return FPM_OK;
}

int fpm_get_hparams(const fpm_handle* h, fpm_hparams* hp) {
  if (!h || !hp) return FPM_ERR_ARG;
  *hp = h->hp;
  return FPM_OK;
}

int fpm_dims(const fpm_handle* h, int32_t* N, int32_t* m, int32_t* n_leds, int32_t* box) {
  if (!h) return FPM_ERR_ARG;
  if (N) *N = h->N;
  if (m) *m = h->m;
  if (n_leds) *n_leds = h->n;
  if (box) *box = h->W;
  return FPM_OK;
}

int fpm_set_memory_limit(fpm_handle* h, int64_t bytes) {
  if (!h) return FPM_ERR_ARG;
  h->mem_limit = bytes > 0 ? bytes : 0;
  return FPM_OK;
}

int64_t fpm_memory_used(const fpm_handle* h) { return h ? h->mem_used : FPM_ERR_ARG; }

int fpm_load(fpm_handle* h, const float* stack, int32_t flags) {
  if (!h || !stack) return fail(h, FPM_ERR_ARG, "null argument");
  if (flags & ~FPM_LOAD_INIT) return fail(h, FPM_ERR_ARG, "unknown load flags");
  int rc = enter(h);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(h->meas, stack, sizeof(float) * (size_t)h->n * h->m * h->m, cudaMemcpyDefault, h->st));
  CK(h, launch_amplitude(h->meas, h->amp, (size_t)h->n * h->m * h->m, h->st));
  if (flags & FPM_LOAD_INIT) {
    CK(h, launch_upsample_centre(h->meas + (size_t)h->centre * h->m * h->m, h->m, h->s, h->tmp, h->st));
    if ((rc = object_from_field(h))) return rc;
    if ((rc = reset_state(h))) return rc;
  }
  h->loaded = true;
  return leave(h);
}

int fpm_run(fpm_handle* h, const int32_t* schedule, int32_t n_steps, int32_t B, double* losses_out) {
  if (!h) return FPM_ERR_ARG;
  if (!h->loaded) return fail(h, FPM_ERR_STATE, "no stack loaded");
  if (n_steps < 1) return fail(h, FPM_ERR_SHAPE, "n_steps must be >= 1");
  int rc = validate_batches(h, schedule, n_steps, B);
  if (rc) return rc;
  if ((rc = ensure_batch(h, B))) return rc;
  if ((rc = grow(h, &h->sched, &h->cap_sched, n_steps * B))) return rc;
  if ((rc = grow(h, &h->losses, &h->cap_losses, n_steps))) return rc;
  if ((rc = grow(h, &h->coef, &h->cap_coef, n_steps))) return rc;
  auto key = std::make_pair(n_steps, B);
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    it = h->graphs.emplace(key, fpm_handle::Graph{}).first;
    if ((rc = build_graph(h, n_steps, B, &it->second))) {
      fpm_handle::Graph g = it->second;
      h->graphs.erase(it);
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.h_slots) cudaFreeHost(g.h_slots);
      if (g.h_coef) cudaFreeHost(g.h_coef);
      if (g.done) cudaEventDestroy(g.done);
      return rc;
    }
  } else {
    // the previous launch of this graph may still be reading its staging
    CK(h, cudaEventSynchronize(it->second.done));
  }
  fill_slots(h, schedule, n_steps * B, it->second.h_slots);
  fill_coef(h, n_steps, it->second.h_coef);
  if ((rc = enter(h))) return rc;
  CK(h, cudaGraphLaunch(it->second.exec, h->st));
  CK(h, cudaEventRecord(it->second.done, h->st));
  h->t_host += n_steps;
  if (losses_out) {
    bool host = false;
    if ((rc = copy_out(h, losses_out, h->losses, sizeof(double) * n_steps, &host))) return rc;
    if (host) {
      if ((rc = check_device_error(h))) return rc;
    }
  }
  return leave(h);
}

int fpm_profile_run(fpm_handle* h, const int32_t* schedule, int32_t n_steps, int32_t B, void* flush,
                    int64_t flush_bytes, float* led_ms, float* update_ms, float* step_ms) {
  if (!h) return FPM_ERR_ARG;
  if (!h->loaded) return fail(h, FPM_ERR_STATE, "no stack loaded");
  if (n_steps < 1) return fail(h, FPM_ERR_SHAPE, "n_steps must be >= 1");
  if (flush && flush_bytes <= 0) return fail(h, FPM_ERR_ARG, "flush buffer without a size");
  if (flush && !is_device_ptr(flush)) return fail(h, FPM_ERR_ARG, "flush buffer must be device memory");
  int rc = validate_batches(h, schedule, n_steps, B);
  if (rc) return rc;
  if ((rc = ensure_batch(h, B))) return rc;
  if ((rc = grow(h, &h->sched, &h->cap_sched, n_steps * B))) return rc;
  if ((rc = grow(h, &h->losses, &h->cap_losses, n_steps))) return rc;
  if ((rc = enter(h))) return rc;
  if ((rc = grow(h, &h->coef, &h->cap_coef, n_steps))) return rc;
  std::vector<int4> slots((size_t)n_steps * B);
  fill_slots(h, schedule, n_steps * B, slots.data());
  CK(h, cudaMemcpyAsync(h->sched, slots.data(), sizeof(int4) * slots.size(), cudaMemcpyHostToDevice, h->st));
  std::vector<float4> coef(n_steps);
  fill_coef(h, n_steps, coef.data());
  CK(h, cudaMemcpyAsync(h->coef, coef.data(), sizeof(float4) * n_steps, cudaMemcpyHostToDevice, h->st));
  std::vector<cudaEvent_t> ev((size_t)3 * n_steps, nullptr);
  auto destroy = [&]() {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  };
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      destroy();
      return fail(h, FPM_ERR_CUDA, "event creation failed");
    }
  const bool per_kernel = led_ms || update_ms;
  // Direct launches (events recorded inside captured graphs cannot be timed);
  // with a flush before every step the host stays ahead of the device, so
  // each timed window holds only device work.
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < n_steps && e == cudaSuccess; ++s) {
    const int4* idx = h->sched + (size_t)s * B;
    if (flush) e = cudaMemsetAsync(flush, s & 0xff, (size_t)flush_bytes, h->st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3 * s], h->st);
    if (uses_step(h)) {  // one kernel per step: no split
      if (e == cudaSuccess) e = launch_train_step(h, idx, B, s, h->losses + s, false);
      if (e == cudaSuccess) e = cudaEventRecord(ev[3 * s + 1], h->st);
    } else {
      if (e == cudaSuccess) e = launch_train_step(h, idx, B, s, h->losses + s, false, per_kernel);
      if (e == cudaSuccess && per_kernel) e = cudaEventRecord(ev[3 * s + 1], h->st);
      if (e == cudaSuccess && per_kernel) e = launch_update(upd_args(h, idx, B, s, h->losses + s, 0), h->st, false);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[3 * s + 2], h->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    destroy();
    return fail(h, FPM_ERR_CUDA, "profiled run failed: %s", cudaGetErrorString(e));
  }
  h->t_host += n_steps;
  for (int s = 0; s < n_steps && e == cudaSuccess; ++s) {
    float a = 0.f, b = 0.f;
    if (per_kernel) {
      e = cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[3 * s + 1], ev[3 * s + 2]);
    } else {
      e = cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 2]);
    }
    if (led_ms) led_ms[s] = a;
    if (update_ms) update_ms[s] = b;
    if (step_ms) step_ms[s] = a + b;
  }
  destroy();
  if (e != cudaSuccess) return fail(h, FPM_ERR_CUDA, "event timing failed: %s", cudaGetErrorString(e));
  if ((rc = check_device_error(h))) return rc;
  return leave(h);
}

int fpm_step(fpm_handle* h, const int32_t* batch_idx, int32_t B, double* loss_out) {
  return fpm_run(h, batch_idx, 1, B, loss_out);
}

int fpm_set_step_form(fpm_handle* h, int32_t form) {
  if (!h) return FPM_ERR_ARG;
  if (form != FPM_STEP_AUTO && form != FPM_STEP_CLUSTER && form != FPM_STEP_DATAFLOW)
    return fail(h, FPM_ERR_ARG, "unknown step form %d", form);
  if (form != h->step_form) {
    CK(h, cudaStreamSynchronize(h->st));
    destroy_graphs(h);  // captured launches of the other form
    h->step_form = form;
  }
  return FPM_OK;
}

int fpm_get_step_form(const fpm_handle* h, int32_t* form, int32_t* dataflow) {
  if (!h) return FPM_ERR_ARG;
  if (form) *form = h->step_form;
  if (dataflow) *dataflow = uses_step(h) ? 1 : 0;
  return FPM_OK;
}

int fpm_check_wait_timeout(fpm_handle* h, const int32_t* idx, int32_t B, double limit_s) {
  if (!h) return FPM_ERR_ARG;
  if (!uses_step(h))
    return fail(h, FPM_ERR_STATE, "the dataflow step form is not in use (m = 256, FP32 FFT form, FPM_STEP_DATAFLOW)");
  if (!h->loaded) return fail(h, FPM_ERR_STATE, "no stack loaded");
  if (!(limit_s > 0.0 && limit_s <= 10.0)) return fail(h, FPM_ERR_ARG, "limit must lie in (0, 10] s");
  int rc = validate_batches(h, idx, 1, B);
  if (rc) return rc;
  if ((rc = ensure_batch(h, B))) return rc;
  if ((rc = grow(h, &h->sched, &h->cap_sched, B))) return rc;
  if ((rc = grow(h, &h->losses, &h->cap_losses, 1))) return rc;
  if ((rc = grow(h, &h->coef, &h->cap_coef, 1))) return rc;
  if ((rc = enter(h))) return rc;
  std::vector<int4> slots(B);
  fill_slots(h, idx, B, slots.data());
  CK(h, cudaMemcpyAsync(h->sched, slots.data(), sizeof(int4) * B, cudaMemcpyHostToDevice, h->st));
  std::vector<float4> coef(1);
  fill_coef(h, 1, coef.data());
  CK(h, cudaMemcpyAsync(h->coef, coef.data(), sizeof(float4), cudaMemcpyHostToDevice, h->st));
  const LedArgs a = led_args(h, h->sched, B, MODE_LOSS);
  const UpdArgs u = upd_args(h, h->sched, B, 0, h->losses, 0);
  StepArgs s = step_args(h, a, &u);
  s.stall = 1;
  s.wait_ns = (long long)(limit_s * 1e9);
  CK(h, launch_step(s, h->step_ctas, h->st, false));
  h->t_host += 1;
  rc = check_device_error(h);  // synchronises; resets the counters on an error
  if (rc == FPM_OK) return fail(h, FPM_ERR_STATE, "the injected wait did not give up");
  const int rc2 = leave(h);
  return rc2 ? rc2 : rc;
}

int fpm_epoch_loss(fpm_handle* h, double* out, int32_t reset) {
  if (!h) return FPM_ERR_ARG;
  int rc = enter(h);
  if (rc) return rc;
  if (out) {
    bool host = false;
    if ((rc = copy_out(h, out, h->epoch, sizeof(double), &host))) return rc;
  }
  if (reset) CK(h, cudaMemsetAsync(h->epoch, 0, sizeof(double), h->st));
  if ((rc = check_device_error(h))) return rc;
  return leave(h);
}

int fpm_forward(fpm_handle* h, const int32_t* idx, int32_t B, float* I_out) {
  return forward_impl(h, idx, B, I_out, nullptr);
}

int fpm_forward_fields(fpm_handle* h, const int32_t* idx, int32_t B, float* I_out, float* psi_out) {
  if (!h || !I_out || !psi_out) return fail(h, FPM_ERR_ARG, "null argument");
  if (!is_device_ptr(I_out) || !is_device_ptr(psi_out)) return fail(h, FPM_ERR_ARG, "I_out and psi_out must be device memory");
  return forward_impl(h, idx, B, I_out, reinterpret_cast<float2*>(psi_out));
}

int fpm_backward_fields(fpm_handle* h, const int32_t* idx, int32_t B, const float* psi, const float* dL_dI,
                        float* g_object, float* g_zernike, float* g_defocus, float* g_gamma, float* g_offset) {
  if (!h || !psi || !dL_dI) return fail(h, FPM_ERR_ARG, "null argument");
  if (!is_device_ptr(psi) || !is_device_ptr(dL_dI)) return fail(h, FPM_ERR_ARG, "psi and dL_dI must be device memory");
  return backward_impl(h, idx, B, dL_dI, reinterpret_cast<const float2*>(psi), g_object, g_zernike, g_defocus,
                       g_gamma, g_offset, nullptr);
}

int fpm_backward(fpm_handle* h, const int32_t* idx, int32_t B, const float* dL_dI, float* g_object,
                 float* g_zernike, float* g_defocus, float* g_gamma, float* g_offset, double* loss_out) {
  return backward_impl(h, idx, B, dL_dI, nullptr, g_object, g_zernike, g_defocus, g_gamma, g_offset, loss_out);
}

}  // extern "C"

namespace {

int forward_impl(fpm_handle* h, const int32_t* idx, int32_t B, float* I_out, float2* psi_out) {
  if (!h || !I_out) return fail(h, FPM_ERR_ARG, "null argument");
  if (psi_out && h->hp.precision != FPM_PRECISION_FP32_FFT)
    return fail(h, FPM_ERR_ARG, "stored fields need the FP32 FFT form");
  int rc = validate_batches(h, idx, 1, B);
  if (rc) return rc;
  if ((rc = ensure_batch(h, B))) return rc;
  if ((rc = grow(h, &h->sched, &h->cap_sched, B))) return rc;
  const size_t img = (size_t)B * h->m * h->m;
  const bool dev_out = is_device_ptr(I_out);
  if (dev_out && ((uintptr_t)I_out & 15)) return fail(h, FPM_ERR_ARG, "device I_out must be 16-byte aligned");
  if (!dev_out && (rc = ensure_fbuf(h, img))) return rc;
  if ((rc = enter(h))) return rc;
  std::vector<int4> slots(B);
  fill_slots(h, idx, B, slots.data());
  CK(h, cudaMemcpyAsync(h->sched, slots.data(), sizeof(int4) * B, cudaMemcpyHostToDevice, h->st));
  LedArgs a = led_args(h, h->sched, B, psi_out ? MODE_FORWARD_STORE : MODE_FORWARD);
  a.I_out = dev_out ? I_out : h->fbuf;
  a.psi = psi_out;
  if (uses_step(h)) CK(h, launch_step(step_args(h, a, nullptr), h->step_ctas, h->st, false));
  else CK(h, launch_led_mode(h, a, false));
  if (!dev_out) {
    CK(h, cudaMemcpyAsync(I_out, h->fbuf, sizeof(float) * img, cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
  }
  return leave(h);
}

int backward_impl(fpm_handle* h, const int32_t* idx, int32_t B, const float* dL_dI, const float2* psi,
                  float* g_object, float* g_zernike, float* g_defocus, float* g_gamma, float* g_offset,
                  double* loss_out) {
  if (!h) return FPM_ERR_ARG;
  if (psi && h->hp.precision != FPM_PRECISION_FP32_FFT)
    return fail(h, FPM_ERR_ARG, "stored fields need the FP32 FFT form");
  if (!dL_dI && !h->loaded) return fail(h, FPM_ERR_STATE, "no stack loaded");
  int rc = validate_batches(h, idx, 1, B);
  if (rc) return rc;
  if ((rc = ensure_batch(h, B))) return rc;
  if ((rc = grow(h, &h->sched, &h->cap_sched, B))) return rc;
  if ((rc = grow(h, &h->losses, &h->cap_losses, 1))) return rc;
  const size_t img = (size_t)B * h->m * h->m;
  const bool dev_in = dL_dI && is_device_ptr(dL_dI);
  if (dev_in && ((uintptr_t)dL_dI & 15)) return fail(h, FPM_ERR_ARG, "device dL_dI must be 16-byte aligned");
  if (dL_dI && !dev_in && (rc = ensure_fbuf(h, img))) return rc;
  if ((rc = enter(h))) return rc;
  std::vector<int4> slots(B);
  fill_slots(h, idx, B, slots.data());
  CK(h, cudaMemcpyAsync(h->sched, slots.data(), sizeof(int4) * B, cudaMemcpyHostToDevice, h->st));
  LedArgs a = led_args(h, h->sched, B, psi ? MODE_UPSTREAM_STORED : dL_dI ? MODE_UPSTREAM : MODE_LOSS);
  a.psi = const_cast<float2*>(psi);
  if (dL_dI) {
    if (!dev_in) CK(h, cudaMemcpyAsync(h->fbuf, dL_dI, sizeof(float) * img, cudaMemcpyHostToDevice, h->st));
    a.dLdI = dev_in ? dL_dI : h->fbuf;
  }
  const size_t NN = (size_t)h->N * h->N;
  const UpdArgs u = upd_args(h, h->sched, B, 0, h->losses, 1);
  if (uses_step(h)) {
    CK(h, cudaMemsetAsync(h->tmp, 0, sizeof(float2) * NN, h->st));
    CK(h, launch_step(step_args(h, a, &u), h->step_ctas, h->st, false));
  } else {
    CK(h, launch_led_mode(h, a, false));
    CK(h, cudaMemsetAsync(h->tmp, 0, sizeof(float2) * NN, h->st));
    CK(h, launch_update(u, h->st, false));
  }
  bool host = false;
  if (g_object) {
    CK(h, launch_transpose(h->tmp, h->tmp2, h->N, h->st));
    if ((rc = copy_out(h, g_object, h->tmp2, sizeof(float2) * NN, &host))) return rc;
  }
  const int off = sp_offset(h->n);
  if ((rc = copy_out(h, g_zernike, h->gsc + SP_ZERN, sizeof(float) * 14, &host))) return rc;
  if ((rc = copy_out(h, g_defocus, h->gsc + SP_DEFOCUS, sizeof(float), &host))) return rc;
  if ((rc = copy_out(h, g_gamma, h->gsc + SP_GAMMA, sizeof(float) * h->n, &host))) return rc;
  if ((rc = copy_out(h, g_offset, h->gsc + off, sizeof(float) * 2 * h->n, &host))) return rc;
  if (loss_out) {
    if (dL_dI) *loss_out = 0.0;
    else if ((rc = copy_out(h, loss_out, h->losses, sizeof(double), &host))) return rc;
  }
  if (host) CK(h, cudaStreamSynchronize(h->st));
  return leave(h);
}

}  // namespace

extern "C" {

int fpm_get(fpm_handle* h, float* O, float* zernike, float* defocus, float* gamma, float* offset) {
  if (!h) return FPM_ERR_ARG;
  int rc = enter(h);
  if (rc) return rc;
  bool host = false;
  if (O) {
    CK(h, launch_transpose(h->Ot, h->tmp2, h->N, h->st));
    if ((rc = copy_out(h, O, h->tmp2, sizeof(float2) * (size_t)h->N * h->N, &host))) return rc;
  }
  if ((rc = copy_out(h, zernike, h->sp + SP_ZERN, sizeof(float) * 14, &host))) return rc;
  if ((rc = copy_out(h, defocus, h->sp + SP_DEFOCUS, sizeof(float), &host))) return rc;
  if ((rc = copy_out(h, gamma, h->sp + SP_GAMMA, sizeof(float) * h->n, &host))) return rc;
  if ((rc = copy_out(h, offset, h->sp + sp_offset(h->n), sizeof(float) * 2 * h->n, &host))) return rc;
  if (host) CK(h, cudaStreamSynchronize(h->st));
  return leave(h);
}

int fpm_set(fpm_handle* h, const float* O, const float* zernike, const float* defocus, const float* gamma,
            const float* offset) {
  if (!h) return FPM_ERR_ARG;
  if (offset) {
    const bool host = !is_device_ptr(offset);
    if (host)
      for (int i = 0; i < 2 * h->n; ++i)
        if (!(std::fabs(offset[i]) <= FPM_OFFSET_BOUND_PX))
          return fail(h, FPM_ERR_RANGE, "offset %d outside +-%.2f px", i, (double)FPM_OFFSET_BOUND_PX);
  }
  int rc = enter(h);
  if (rc) return rc;
  if (O) {
    CK(h, cudaMemcpyAsync(h->tmp2, O, sizeof(float2) * (size_t)h->N * h->N, cudaMemcpyDefault, h->st));
    CK(h, launch_transpose(h->tmp2, h->Ot, h->N, h->st));
  }
  if (zernike) CK(h, cudaMemcpyAsync(h->sp + SP_ZERN, zernike, sizeof(float) * 14, cudaMemcpyDefault, h->st));
  if (defocus) CK(h, cudaMemcpyAsync(h->sp + SP_DEFOCUS, defocus, sizeof(float), cudaMemcpyDefault, h->st));
  if (gamma) CK(h, cudaMemcpyAsync(h->sp + SP_GAMMA, gamma, sizeof(float) * h->n, cudaMemcpyDefault, h->st));
  if (offset)
    CK(h, cudaMemcpyAsync(h->sp + sp_offset(h->n), offset, sizeof(float) * 2 * h->n, cudaMemcpyDefault, h->st));
  const bool any_host = (O && is_pageable_host(O)) || (zernike && is_pageable_host(zernike)) ||
                        (defocus && is_pageable_host(defocus)) || (gamma && is_pageable_host(gamma)) ||
                        (offset && is_pageable_host(offset));
  if (any_host) CK(h, cudaStreamSynchronize(h->st));
  return leave(h);
}

int fpm_set_object_field(fpm_handle* h, const float* o) {
  if (!h || !o) return fail(h, FPM_ERR_ARG, "null argument");
  int rc = enter(h);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(h->tmp, o, sizeof(float2) * (size_t)h->N * h->N, cudaMemcpyDefault, h->st));
  if ((rc = object_from_field(h))) return rc;
  if (is_pageable_host(o)) CK(h, cudaStreamSynchronize(h->st));
  return leave(h);
}

int fpm_set_pupil(fpm_handle* h, const float* P) {
  if (!h) return FPM_ERR_ARG;
  const int W = h->W;
  const size_t WW = (size_t)W * W;
  if (!P) {  // back to the parametric pupil
    if (h->hp.learn_mask & FPM_LEARN_PUPIL)
      return fail(h, FPM_ERR_STATE, "the free-form pupil is learned (clear FPM_LEARN_PUPIL first)");
    if (h->pupil_on) {
      CK(h, cudaStreamSynchronize(h->st));
      destroy_graphs(h);
    }
    h->pupil_on = false;
    return FPM_OK;
  }
  if (h->hp.precision != FPM_PRECISION_FP32_FFT)
    return fail(h, FPM_ERR_ARG, "the free-form pupil needs the FP32 FFT form");
  std::vector<float2> hostP(WW), col(WW);
  int rc = enter(h);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(hostP.data(), P, sizeof(float2) * WW, cudaMemcpyDefault, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  for (int ny = 0; ny < W; ++ny)  // row-major [ny][nx] -> column-major by node column
    for (int nx = 0; nx < W; ++nx) col[(size_t)nx * W + ny] = hostP[(size_t)ny * W + nx];
  CK(h, cudaMemcpyAsync(h->Pff, col.data(), sizeof(float2) * WW, cudaMemcpyHostToDevice, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  if (!h->pupil_on) destroy_graphs(h);
  h->pupil_on = true;
  return leave(h);
}

namespace {
// Copy a node field ([W][W], column-major by node column) into P (row-major [ny][nx]).
int pupil_field_out(fpm_handle* h, const float2* src, float* P) {
  const int W = h->W;
  const size_t WW = (size_t)W * W;
  std::vector<float2> col(WW), row(WW);
  int rc = enter(h);
  if (rc) return rc;
  CK(h, cudaMemcpyAsync(col.data(), src, sizeof(float2) * WW, cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  for (int ny = 0; ny < W; ++ny)
    for (int nx = 0; nx < W; ++nx) row[(size_t)ny * W + nx] = col[(size_t)nx * W + ny];
  CK(h, cudaMemcpyAsync(P, row.data(), sizeof(float2) * WW, cudaMemcpyDefault, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  return leave(h);
}
}  // namespace

int fpm_get_pupil(fpm_handle* h, float* P, int32_t* in_use) {
  if (!h) return FPM_ERR_ARG;
  if (in_use) *in_use = h->pupil_on ? 1 : 0;
  if (!P) return FPM_OK;
  return pupil_field_out(h, h->Pff, P);
}

int fpm_pupil_gradient(fpm_handle* h, float* g) {
  if (!h || !g) return fail(h, FPM_ERR_ARG, "null argument");
  if (!h->pupil_on) return fail(h, FPM_ERR_STATE, "no free-form pupil in the model");
  return pupil_field_out(h, h->gPff, g);
}

int64_t fpm_state_size(const fpm_handle* h) {
  if (!h) return FPM_ERR_ARG;
  return (int64_t)6 * h->N * h->N + 3LL * sp_size(h->n) + 6LL * h->W * h->W + 6;
}

int fpm_get_state(fpm_handle* h, float* state) {
  if (!h || !state) return fail(h, FPM_ERR_ARG, "null argument");
  int rc = enter(h);
  if (rc) return rc;
  const size_t NN = (size_t)h->N * h->N;
  const int P = sp_size(h->n);
  bool host = false;
  float2* src[3] = {h->Ot, h->mO, h->vO};
  for (int q = 0; q < 3; ++q) {
    CK(h, launch_transpose(src[q], h->tmp2, h->N, h->st));
    if ((rc = copy_out(h, state + 2 * NN * q, h->tmp2, sizeof(float2) * NN, &host))) return rc;
    CK(h, cudaStreamSynchronize(h->st));  // tmp2 is reused by the next transpose
  }
  float* sps[3] = {h->sp, h->msp, h->vsp};
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_out(h, state + 6 * NN + (size_t)P * q, sps[q], sizeof(float) * P, &host))) return rc;
  const size_t WW = (size_t)h->W * h->W;
  float* pst = state + 6 * NN + 3 * (size_t)P;
  float2* pps[3] = {h->Pff, h->mPff, h->vPff};
  for (int q = 0; q < 3; ++q)
    if ((rc = copy_out(h, pst + 2 * WW * q, pps[q], sizeof(float2) * WW, &host))) return rc;
  double tail[3];
  CK(h, cudaMemcpyAsync(&tail[1], h->epoch, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  tail[0] = (double)h->t_host;
  tail[2] = h->pupil_on ? 1.0 : 0.0;
  CK(h, cudaMemcpyAsync(pst + 6 * WW, tail, sizeof tail, cudaMemcpyDefault, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  return leave(h);
}

int fpm_set_state(fpm_handle* h, const float* state) {
  if (!h || !state) return fail(h, FPM_ERR_ARG, "null argument");
  int rc = enter(h);
  if (rc) return rc;
  const size_t NN = (size_t)h->N * h->N;
  const int P = sp_size(h->n);
  float2* dst[3] = {h->Ot, h->mO, h->vO};
  for (int q = 0; q < 3; ++q) {
    CK(h, cudaMemcpyAsync(h->tmp2, state + 2 * NN * q, sizeof(float2) * NN, cudaMemcpyDefault, h->st));
    CK(h, launch_transpose(h->tmp2, dst[q], h->N, h->st));
    CK(h, cudaStreamSynchronize(h->st));
  }
  float* sps[3] = {h->sp, h->msp, h->vsp};
  for (int q = 0; q < 3; ++q)
    CK(h, cudaMemcpyAsync(sps[q], state + 6 * NN + (size_t)P * q, sizeof(float) * P, cudaMemcpyDefault, h->st));
  const size_t WW = (size_t)h->W * h->W;
  const float* pst = state + 6 * NN + 3 * (size_t)P;
  float2* pps[3] = {h->Pff, h->mPff, h->vPff};
  for (int q = 0; q < 3; ++q)
    CK(h, cudaMemcpyAsync(pps[q], pst + 2 * WW * q, sizeof(float2) * WW, cudaMemcpyDefault, h->st));
  double tail[3];
  CK(h, cudaMemcpyAsync(tail, pst + 6 * WW, sizeof tail, cudaMemcpyDefault, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  if (!(tail[0] >= 0.0) || !std::isfinite(tail[1]) || !(tail[2] == 0.0 || tail[2] == 1.0))
    return fail(h, FPM_ERR_ARG, "corrupt state tail");
  if (tail[2] == 1.0 && h->hp.precision != FPM_PRECISION_FP32_FFT)
    return fail(h, FPM_ERR_ARG, "the state holds a free-form pupil, which needs the FP32 FFT form");
  if (h->pupil_on != (tail[2] == 1.0)) destroy_graphs(h);
  h->pupil_on = tail[2] == 1.0;
  h->t_host = (long long)tail[0];
  CK(h, cudaMemcpyAsync(h->epoch, &tail[1], sizeof(double), cudaMemcpyHostToDevice, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  h->loaded = true;
  return leave(h);
}

int fpm_epoch_permutation(int32_t n, uint64_t seed, int32_t epoch, int32_t* out) {
  if (n < 1 || !out || epoch < 0) return FPM_ERR_ARG;
  uint64_t s = seed ^ ((uint64_t)(epoch + 1) * 0xA0761D6478BD642FULL);
  auto next = [&s]() {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  for (int i = 0; i < n; ++i) out[i] = i;
  for (int i = n - 1; i > 0; --i) {
    const int j = (int)(next() % (uint64_t)(i + 1));
    const int t = out[i];
    out[i] = out[j];
    out[j] = t;
  }
  return FPM_OK;
}

}  // extern "C"

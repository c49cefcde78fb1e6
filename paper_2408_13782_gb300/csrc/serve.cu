// Continuous-batching reconstruction server (fpm_server_* in include/fpm.h).
//
// Requests (one reconstruction job each: geometry, stack, hyper-parameters,
// batch size, stopping rule) are queued on submit and admitted in arrival
// order, each one as soon as it fits the device-memory budget and a slot is
// free (first fit). An
// admitted job owns an engine handle - its object spectrum, pupil, defocus,
// LED parameters and Adam state stay resident until it finishes - and a
// private stream, so the epochs of all admitted jobs run concurrently on the
// GPU. Each epoch (a fresh random permutation chopped into batches, Eq. 13-14)
// is two graph launches at most (the full batches, then the short one);
// after it, the running FP64 loss is copied to pinned memory and an event is
// recorded. fpm_server_tick() never blocks: it retires epochs whose events
// have fired, applies the stopping rule (relative change of the epoch loss
// below rel_tol, or max_epochs), copies finished results to host memory and
// frees their device memory, then admits queued jobs.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/fpm.h"
#include "internal.h"

using namespace fpmk;

namespace {

struct Job {
  int64_t id = 0;
  fpm_job_desc desc{};
  std::vector<float> offsets;
  std::vector<float> stack;  // host copy until admitted
  int64_t footprint = 0;
  int state = FPM_JOB_QUEUED;
  fpm_handle* h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  double* pinned = nullptr;  // running FP64 loss sum after the epoch in flight
  bool in_flight = false;
  int epochs = 0;
  double acc_prev = 0.0, loss = 0.0, loss_prev = -1.0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  int64_t led_updates = 0;
  std::vector<float> O, zern, defocus, gamma, offset;  // results
  std::string error;
};

}  // namespace

struct fpm_server {
  int64_t budget = 0, used = 0;
  int max_active = 0;
  std::deque<Job*> queue;
  std::vector<Job*> active;
  std::map<int64_t, std::unique_ptr<Job>> jobs;
  int64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  std::string msg;
};

namespace {

double now(const fpm_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

int srv_fail(fpm_server* s, int code, const std::string& m) {
  if (s) s->msg = m;
  return code;
}

void release(fpm_server* s, Job* j) {
  if (j->h) fpm_destroy(j->h);
  j->h = nullptr;
  if (j->ev) cudaEventDestroy(j->ev);
  j->ev = nullptr;
  if (j->stream) cudaStreamDestroy(j->stream);
  j->stream = nullptr;
  if (j->pinned) cudaFreeHost(j->pinned);
  j->pinned = nullptr;
  s->used -= j->footprint;
}

void fail_job(fpm_server* s, Job* j, const std::string& why) {
  j->error = why;
  j->state = FPM_JOB_FAILED;
  j->t_done = now(s);
  release(s, j);
}

// Queue one epoch of job j: the full batches as one graph, the short batch as another.
int launch_epoch(Job* j) {
  const int n = j->desc.geometry.n_leds, B = j->desc.batch;
  std::vector<int32_t> perm(n);
  fpm_epoch_permutation(n, j->desc.seed, j->epochs, perm.data());
  const int nfull = n / B, rem = n - nfull * B;
  int rc = FPM_OK;
  if (nfull > 0) rc = fpm_run(j->h, perm.data(), nfull, B, nullptr);
  if (rc == FPM_OK && rem > 0) rc = fpm_run(j->h, perm.data() + (size_t)nfull * B, 1, rem, nullptr);
  if (rc == FPM_OK) rc = engine_snapshot_loss(j->h, j->pinned);
  if (rc == FPM_OK && cudaEventRecord(j->ev, j->stream) != cudaSuccess) rc = FPM_ERR_CUDA;
  if (rc == FPM_OK) j->in_flight = true;
  return rc;
}

int admit(fpm_server* s, Job* j) {
  const fpm_job_desc& d = j->desc;
  if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&j->pinned, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return FPM_ERR_CUDA;
  }
  fpm_geometry g = d.geometry;
  g.led_offset = j->offsets.data();
  int rc = fpm_create(&g, d.pupil_radius_px, d.upsample, j->stream, &j->h);
  if (rc) {
    j->error = fpm_last_error(nullptr);
    return rc;
  }
  if ((rc = fpm_set_hparams(j->h, &d.hparams)) || (rc = fpm_load(j->h, j->stack.data(), FPM_LOAD_INIT))) {
    j->error = fpm_last_error(j->h);
    return rc;
  }
  std::vector<float>().swap(j->stack);  // the stack now lives on the device
  j->state = FPM_JOB_ACTIVE;
  j->t_admit = now(s);
  return launch_epoch(j);
}

// After an epoch: stop, or queue the next one.
int retire_epoch(fpm_server* s, Job* j) {
  j->in_flight = false;
  const double acc = *j->pinned;
  const double L = acc - j->acc_prev;
  j->acc_prev = acc;
  j->loss_prev = j->epochs > 0 ? j->loss : -1.0;
  j->loss = L;
  j->epochs += 1;
  j->led_updates += j->desc.geometry.n_leds;
  if (!std::isfinite(L)) {
    fail_job(s, j, "non-finite epoch loss");
    return FPM_OK;
  }
  const bool converged = j->loss_prev > 0.0 && std::fabs(L - j->loss_prev) < j->desc.rel_tol * j->loss_prev;
  if (converged || j->epochs >= j->desc.max_epochs) {
    const int64_t N = (int64_t)j->desc.geometry.m * j->desc.upsample;
    const int n = j->desc.geometry.n_leds;
    j->O.resize((size_t)N * N * 2);
    j->zern.resize(14);
    j->defocus.resize(1);
    j->gamma.resize(n);
    j->offset.resize((size_t)2 * n);
    const int rc = fpm_get(j->h, j->O.data(), j->zern.data(), j->defocus.data(), j->gamma.data(), j->offset.data());
    if (rc) {
      fail_job(s, j, fpm_last_error(j->h));
      return FPM_OK;
    }
    j->state = FPM_JOB_DONE;
    j->t_done = now(s);
    release(s, j);
    return FPM_OK;
  }
  return launch_epoch(j);
}

}  // namespace

extern "C" {

int64_t fpm_job_footprint(const fpm_job_desc* d) {
  if (!d || d->geometry.m < 1 || d->upsample < 1 || d->geometry.n_leds < 1 || d->batch < 1) return FPM_ERR_ARG;
  const int64_t m = d->geometry.m, N = m * d->upsample, n = d->geometry.n_leds, B = d->batch;
  const int64_t h = (int64_t)std::floor((double)d->pupil_radius_px + 0.5 + std::sqrt(2.0) * FPM_OFFSET_BOUND_PX) + 1;
  const int64_t W = 2 * h + 1, C = m >= 256 ? 16 : (m == 128 ? 8 : (m == 64 ? 4 : 2));  // upper bound
  const int64_t steps = n / B + 1;
  int64_t bytes = 5 * N * N * 8          // O, Adam m and v, two transform buffers
                  + 2 * n * m * m * 4    // measured stack and its amplitudes
                  + (m + N) * 8          // twiddles
                  + 4 * (15 + 3 * n) * 4 // parameters, moments, gradient
                  + n * 8 + N * 8        // LED table, update spans
                  + B * W * W * 8        // per-LED gradient boxes
                  + B * C * NPART * 8    // FP64 partials
                  + steps * B * 16 + steps * (8 + 8);  // batch slots, losses, coefficients
  return bytes + (1 << 20);              // allocator granularity and small buffers
}

int fpm_server_create(int64_t budget, int32_t max_active, fpm_server** out) {
  if (!out || budget <= 0 || max_active < 1) return FPM_ERR_ARG;
  fpm_server* s = new fpm_server();
  s->budget = budget;
  s->max_active = max_active;
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return FPM_OK;
}

void fpm_server_destroy(fpm_server* s) {
  if (!s) return;
  for (Job* j : s->active)
    if (j->stream) cudaStreamSynchronize(j->stream);
  for (auto& kv : s->jobs)
    if (kv.second->state == FPM_JOB_ACTIVE) release(s, kv.second.get());
  delete s;
}

const char* fpm_server_error(const fpm_server* s) { return s ? s->msg.c_str() : ""; }

double fpm_server_clock(const fpm_server* s) { return s ? now(s) : 0.0; }

int fpm_server_submit(fpm_server* s, const fpm_job_desc* d, const float* stack, int64_t* job_id) {
  if (!s || !d || !stack || !job_id || !d->geometry.led_offset) return srv_fail(s, FPM_ERR_ARG, "null argument");
  if (d->batch < 1 || d->batch > d->geometry.n_leds) return srv_fail(s, FPM_ERR_SHAPE, "batch outside [1, n_leds]");
  if (d->max_epochs < 1 || !(d->rel_tol >= 0.0)) return srv_fail(s, FPM_ERR_ARG, "bad stopping rule");
  const int64_t fp = fpm_job_footprint(d);
  if (fp <= 0) return srv_fail(s, FPM_ERR_ARG, "bad job description");
  if (fp > s->budget) return srv_fail(s, FPM_ERR_OOM, "job footprint exceeds the server's memory budget");
  auto j = std::make_unique<Job>();
  j->id = s->next_id++;
  j->desc = *d;
  const int n = d->geometry.n_leds, m = d->geometry.m;
  j->offsets.assign(d->geometry.led_offset, d->geometry.led_offset + 2 * (size_t)n);
  j->desc.geometry.led_offset = nullptr;
  j->stack.assign(stack, stack + (size_t)n * m * m);
  j->footprint = fp;
  j->t_submit = now(s);
  *job_id = j->id;
  s->queue.push_back(j.get());
  s->jobs.emplace(j->id, std::move(j));
  return FPM_OK;
}

int fpm_server_tick(fpm_server* s, int32_t* n_active, int32_t* n_queued) {
  if (!s) return FPM_ERR_ARG;
  // retire finished epochs (frees memory of finished jobs)
  std::vector<Job*> still;
  for (Job* j : s->active) {
    if (j->in_flight) {
      const cudaError_t q = cudaEventQuery(j->ev);
      if (q == cudaErrorNotReady) {
        still.push_back(j);
        continue;
      }
      if (q != cudaSuccess) {
        cudaGetLastError();
        fail_job(s, j, cudaGetErrorString(q));
        continue;
      }
      const int rc = retire_epoch(s, j);
      if (rc) fail_job(s, j, fpm_last_error(j->h));
    }
    if (j->state == FPM_JOB_ACTIVE) still.push_back(j);
  }
  s->active.swap(still);
  // admit queued jobs in arrival order, each one that fits the remaining
  // memory (first fit: a job too large for now does not hold back smaller
  // ones behind it), while slots allow
  for (auto it = s->queue.begin(); it != s->queue.end() && (int)s->active.size() < s->max_active;) {
    Job* j = *it;
    if (s->used + j->footprint > s->budget) {
      ++it;
      continue;
    }
    it = s->queue.erase(it);
    s->used += j->footprint;
    const int rc = admit(s, j);
    if (rc) {
      fail_job(s, j, j->error.empty() ? "admission failed" : j->error);
      continue;
    }
    s->active.push_back(j);
  }
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  return FPM_OK;
}

int fpm_server_status(const fpm_server* s, int64_t id, fpm_job_status* st) {
  if (!s || !st) return FPM_ERR_ARG;
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return FPM_ERR_RANGE;
  const Job* j = it->second.get();
  st->state = j->state;
  st->epochs = j->epochs;
  st->loss = j->loss;
  st->t_submit = j->t_submit;
  st->t_admit = j->t_admit;
  st->t_done = j->t_done;
  st->led_updates = j->led_updates;
  st->footprint = j->footprint;
  return FPM_OK;
}

int fpm_server_result(fpm_server* s, int64_t id, float* O, float* zernike, float* defocus, float* gamma,
                      float* offset) {
  if (!s) return FPM_ERR_ARG;
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return srv_fail(s, FPM_ERR_RANGE, "unknown job");
  Job* j = it->second.get();
  if (j->state != FPM_JOB_DONE) return srv_fail(s, FPM_ERR_STATE, j->error.empty() ? "job not finished" : j->error);
  if (O) std::memcpy(O, j->O.data(), j->O.size() * sizeof(float));
  if (zernike) std::memcpy(zernike, j->zern.data(), 14 * sizeof(float));
  if (defocus) *defocus = j->defocus[0];
  if (gamma) std::memcpy(gamma, j->gamma.data(), j->gamma.size() * sizeof(float));
  if (offset) std::memcpy(offset, j->offset.data(), j->offset.size() * sizeof(float));
  return FPM_OK;
}

}  // extern "C"

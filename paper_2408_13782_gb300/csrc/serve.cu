// Continuous-batching reconstruction server (fpm_server_* in include/fpm.h).
//
// Requests (one reconstruction job each: geometry, stack, hyper-parameters,
// batch size, stopping rule) are queued on submit and admitted in arrival
// order, each one as soon as it fits the device-memory budget and a slot is
// free (first fit). An admitted job owns an engine handle: its object
// spectrum, pupil, defocus, LED parameters and Adam state stay resident until
// it finishes.
//
// Work is issued in rounds of one epoch (a fresh random permutation chopped
// into batches, Eq. 13-14) per job. FP32 FFT-form jobs with the same number
// of steps per epoch share a round (grouped by the server's policy: the same
// kernel configuration, the same low-res size, or sizes 64, 128 and 256
// together): step s of the round is one per-LED launch and one update launch
// covering step s of every job in it, the jobs' arguments read from device
// tables. Jobs of size 64, 128 and 256 grouped by size or mixed use the
// mixed-size launch (clusters of 16 CTAs shared by their LEDs, 4, 8 or 16 CTAs
// each), whatever their crop box, LED count and batch size; other jobs use the
// same-configuration launch. A round is captured once as a CUDA graph (kept while
// its jobs are resident) and relaunched every epoch with the new schedules
// and Adam coefficients copied from pinned staging inside the graph. Rounds
// of different groups run on their own streams, so all admitted jobs overlap
// on the GPU. Other jobs (tensor-core forms) run their epochs through fpm_run.
// After a round, each job's running FP64 loss is in pinned memory.
// fpm_server_tick() never blocks: it retires rounds whose events have fired,
// applies the stopping rule (relative change of the epoch loss below
// rel_tol, or max_epochs), copies finished results to host memory and frees
// their device memory, admits queued jobs, then launches the next rounds.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <algorithm>
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
  int4* h_slots = nullptr;   // pinned: the slot table of the epoch a round is about to run
  float4* h_coef = nullptr;  // pinned: that epoch's optimiser coefficients per step
  bool in_flight = false;
  int epochs = 0;
  double acc_prev = 0.0, loss = 0.0, loss_prev = -1.0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  int64_t led_updates = 0;
  std::vector<float> O, zern, defocus, gamma, offset;  // results
  std::string error;
  EngineRound er{};  // device buffers of the handle used by rounds
  bool fresh = true;  // admitted, its load not yet ordered before a round
};

// One round: an epoch of each of its jobs (same epoch shape) in lock-step.
struct Round {
  std::vector<Job*> jobs;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t exec = nullptr;
  int steps = 0;
  bool mixed = false;            // the mixed-size per-LED launch
  unsigned char* d_tables = nullptr;  // LedArgs / UpdArgs tables and maps of all steps
  bool in_flight = false;
};

}  // namespace

struct fpm_server {
  int64_t budget = 0, used = 0;
  int max_active = 0;
  int admission = FPM_ADMIT_ARRIVAL;
  int grouping = FPM_GROUP_CONFIG;
  std::deque<Job*> queue;
  std::vector<Job*> active;
  std::map<int64_t, std::unique_ptr<Job>> jobs;
  std::map<std::string, std::unique_ptr<Round>> rounds;  // by composition
  // Pinned host buffers, reused across jobs (size classes of powers of two):
  // freeing pinned memory can wait for the whole device, so blocks go back to
  // the pool instead and are freed only with the server.
  std::multimap<size_t, void*> pin_free;
  std::map<void*, size_t> pin_size;
  int64_t n_rounds = 0, n_round_epochs = 0, max_round_jobs = 0, n_launches = 0;
  int64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  std::string msg;
};

namespace {

// Expected work of a job: LED images x pixels x epochs at most (the stopping rule may end it sooner).
double job_work(const Job* j) {
  const double m = j->desc.geometry.m;
  return (double)j->desc.geometry.n_leds * m * m * (double)j->desc.max_epochs;
}

double now(const fpm_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

int srv_fail(fpm_server* s, int code, const std::string& m) {
  if (s) s->msg = m;
  return code;
}

// A retired round's tables go back to the stream-ordered pool (a plain
// cudaFree would wait for every other round in flight).
void destroy_round(Round* r) {
  if (r->stream) cudaStreamSynchronize(r->stream);
  if (r->exec) cudaGraphExecDestroy(r->exec);
  if (r->d_tables) cudaFreeAsync(r->d_tables, r->stream);
  if (r->ev) cudaEventDestroy(r->ev);
  if (r->stream) cudaStreamDestroy(r->stream);
}

void* pin_get(fpm_server* s, size_t bytes) {
  size_t cls = 64;
  while (cls < bytes) cls <<= 1;
  auto it = s->pin_free.find(cls);
  if (it != s->pin_free.end()) {
    void* p = it->second;
    s->pin_free.erase(it);
    return p;
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, cls) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  s->pin_size[p] = cls;
  return p;
}

void pin_put(fpm_server* s, void* p) {
  if (p) s->pin_free.emplace(s->pin_size[p], p);
}

void forget_rounds_of(fpm_server* s, const Job* j) {
  for (auto it = s->rounds.begin(); it != s->rounds.end();) {
    const auto& js = it->second->jobs;
    if (std::find(js.begin(), js.end(), j) != js.end()) {
      destroy_round(it->second.get());
      it = s->rounds.erase(it);
    } else {
      ++it;
    }
  }
}

void release(fpm_server* s, Job* j) {
  forget_rounds_of(s, j);
  if (j->h) fpm_destroy(j->h);
  j->h = nullptr;
  if (j->ev) cudaEventDestroy(j->ev);
  j->ev = nullptr;
  if (j->stream) cudaStreamDestroy(j->stream);
  j->stream = nullptr;
  pin_put(s, j->pinned);
  pin_put(s, j->h_slots);
  pin_put(s, j->h_coef);
  j->pinned = nullptr;
  j->h_slots = nullptr;
  j->h_coef = nullptr;
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
  const int steps_per_epoch = (d.geometry.n_leds + d.batch - 1) / d.batch;
  if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return FPM_ERR_CUDA;
  }
  j->pinned = static_cast<double*>(pin_get(s, sizeof(double)));
  j->h_slots = static_cast<int4*>(pin_get(s, sizeof(int4) * d.geometry.n_leds));
  j->h_coef = static_cast<float4*>(pin_get(s, sizeof(float4) * steps_per_epoch));
  if (!j->pinned || !j->h_slots || !j->h_coef) return FPM_ERR_OOM;
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
  const int n = d.geometry.n_leds, B = d.batch;
  const int steps = n / B + (n % B ? 1 : 0);
  if ((rc = engine_round_reserve(j->h, steps, B, &j->er))) {
    j->error = fpm_last_error(j->h);
    return rc;
  }
  if (cudaEventRecord(j->ev, j->stream) != cudaSuccess) return FPM_ERR_CUDA;  // the load, for the first round
  j->state = FPM_JOB_ACTIVE;
  j->t_admit = now(s);
  return FPM_OK;
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
  return FPM_OK;  // the next epoch is launched by the tick
}

// ---------------------------------------------------------------- rounds

bool groupable(const Job* j) { return j->er.fft != 0; }

int epoch_steps(const Job* j) { return (j->er.n_leds + j->desc.batch - 1) / j->desc.batch; }

// Jobs the mixed-size launch takes (sizes 64, 128, 256 whose box fits it). Its
// split of an LED (led_mixed_cluster) may differ from the handle's own at
// m = 256; the handle's partials have room for both.
bool mixable(const Job* j) { return groupable(j) && led_mixed_cluster(j->er.m) > 0 && led_mixed_fits(j->er.m, j->er.W); }

// The round a job joins under the server's grouping (a key starting "mix"
// marks the mixed-size launch).
std::string group_key(const fpm_server* s, const Job* j) {
  char b[96];
  if (s->grouping == FPM_GROUP_MIXED && mixable(j))
    std::snprintf(b, sizeof b, "mix S%d", epoch_steps(j));
  else if (s->grouping == FPM_GROUP_SIZE && mixable(j))
    std::snprintf(b, sizeof b, "mix S%d m%d", epoch_steps(j), j->er.m);
  else
    std::snprintf(b, sizeof b, "m%d C%d W%d n%d B%d", j->er.m, j->er.C, j->er.W, j->er.n_leds, j->desc.batch);
  return b;
}

// Build the round of jobs js (same group: the same number of steps per
// epoch): tables, staging, and its graph.
int build_round(Round* r, const std::vector<Job*>& js, bool mixed) {
  r->jobs = js;
  const Job* j0 = js[0];
  const int m = j0->er.m, C = j0->er.C;
  r->mixed = mixed;
  r->steps = epoch_steps(j0);
  const int J = (int)js.size(), S = r->steps;
  if (r->mixed && led_mixed_prepare() != cudaSuccess) return FPM_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
    return FPM_ERR_CUDA;
  // per step: J LedArgs, J UpdArgs, the per-LED map and the update-CTA map.
  // Same-configuration rounds map each cluster to (job, slot); the mixed
  // launch maps each CTA to (job, slot, rank among the LED's CTAs, m), the
  // LEDs ordered by CTAs per LED, largest first, so that none straddles a
  // cluster (every split divides 16), and the last cluster filled with idle CTAs.
  std::vector<LedArgs> led((size_t)S * J);
  std::vector<UpdArgs> upd((size_t)S * J);
  std::vector<std::vector<int4>> lmap(S);
  std::vector<std::vector<int2>> umap(S);
  std::vector<int> bmax(S, 0);
  size_t smem = 0;
  bool ff = false;  // some job models a free-form pupil field: the instantiation that has it
  for (int st = 0; st < S; ++st) {
    for (int q = 0; q < J; ++q) {
      Job* j = js[q];
      const int B = j->desc.batch, nfull = j->er.n_leds / B;
      const int Bs = st < nfull ? B : j->er.n_leds - nfull * B;
      const int4* sl = j->er.slots + (size_t)st * B;
      LedArgs& la = led[(size_t)st * J + q];
      la = engine_led_args(j->h, sl, Bs);
      UpdArgs& ua = upd[(size_t)st * J + q];
      ua = engine_upd_args(j->h, sl, Bs, st, j->er.losses + st);
      if (r->mixed) ua.C = led_mixed_cluster(j->er.m);  // partials per LED in the mixed launch
      ff = ff || la.pupil != nullptr;
      bmax[st] = std::max(bmax[st], Bs);
      if (r->mixed) smem = std::max(smem, led_mixed_smem_bytes(j->er.m, j->er.W));
      if (!r->mixed)
        for (int k = 0; k < Bs; ++k) lmap[st].push_back(make_int4(q, k, 0, 0));
      const int nc = update_ctas(upd[(size_t)st * J + q]);
      for (int b = 0; b < nc; ++b) umap[st].push_back(make_int2(q, b));
    }
    if (r->mixed) {
      for (int c = LED_MIX_CLUSTER; c >= 1; c /= 2)
        for (int q = 0; q < J; ++q) {
          Job* j = js[q];
          if (led_mixed_cluster(j->er.m) != c) continue;
          const int B = j->desc.batch, nfull = j->er.n_leds / B;
          const int Bs = st < nfull ? B : j->er.n_leds - nfull * B;
          for (int k = 0; k < Bs; ++k)
            for (int t = 0; t < c; ++t) lmap[st].push_back(make_int4(q, k, t, j->er.m));
        }
      while (lmap[st].size() % LED_MIX_CLUSTER) lmap[st].push_back(make_int4(-1, 0, 0, 0));
    }
  }
  size_t lm = 0, um = 0;
  for (int st = 0; st < S; ++st) {
    lm += lmap[st].size();
    um += umap[st].size();
  }
  // four tables, each starting on a 256-byte boundary
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_upd = up(sizeof(LedArgs) * led.size()), o_lmap = o_upd + up(sizeof(UpdArgs) * upd.size());
  const size_t o_umap = o_lmap + up(sizeof(int4) * lm), bytes = o_umap + sizeof(int2) * um;
  if (cudaMallocAsync(reinterpret_cast<void**>(&r->d_tables), bytes, r->stream) != cudaSuccess) return FPM_ERR_OOM;
  LedArgs* d_led = reinterpret_cast<LedArgs*>(r->d_tables);
  UpdArgs* d_upd = reinterpret_cast<UpdArgs*>(r->d_tables + o_upd);
  int4* d_lmap = reinterpret_cast<int4*>(r->d_tables + o_lmap);
  int2* d_umap = reinterpret_cast<int2*>(r->d_tables + o_umap);
  std::vector<int4> lmaps;
  std::vector<int2> umaps;
  lmaps.reserve(lm);
  umaps.reserve(um);
  std::vector<size_t> loff(S), uoff(S);
  for (int st = 0; st < S; ++st) {
    loff[st] = lmaps.size();
    lmaps.insert(lmaps.end(), lmap[st].begin(), lmap[st].end());
    uoff[st] = umaps.size();
    umaps.insert(umaps.end(), umap[st].begin(), umap[st].end());
  }
  // the same-configuration launch reads (job, slot) pairs
  std::vector<int2> lpairs;
  if (!r->mixed)
    for (const int4& e : lmaps) lpairs.push_back(make_int2(e.x, e.y));
  // (pageable sources: each copy returns once its source has been staged)
  const auto up_copy = [&](void* dst, const void* src, size_t n) {
    return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, r->stream);
  };
  if (up_copy(d_led, led.data(), sizeof(LedArgs) * led.size()) != cudaSuccess ||
      up_copy(d_upd, upd.data(), sizeof(UpdArgs) * upd.size()) != cudaSuccess ||
      (r->mixed ? up_copy(d_lmap, lmaps.data(), sizeof(int4) * lm)
                : up_copy(d_lmap, lpairs.data(), sizeof(int2) * lm)) != cudaSuccess ||
      up_copy(d_umap, umaps.data(), sizeof(int2) * um) != cudaSuccess)
    return FPM_ERR_CUDA;
  // the graph: schedules and coefficients in, S steps of two launches, losses out
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(r->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FPM_ERR_CUDA;
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < J && e == cudaSuccess; ++q) {
    e = cudaMemcpyAsync(js[q]->er.slots, js[q]->h_slots, sizeof(int4) * js[q]->er.n_leds, cudaMemcpyHostToDevice,
                        r->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(js[q]->er.coef, js[q]->h_coef, sizeof(float4) * S, cudaMemcpyHostToDevice, r->stream);
  }
  const int2* d_lpairs = reinterpret_cast<const int2*>(d_lmap);
  int opt = upd[0].opt;  // one optimiser for the whole round, or -1
  for (const UpdArgs& ua : upd)
    if (ua.opt != opt) opt = -1;
  for (int st = 0; st < S && e == cudaSuccess; ++st) {
    if (r->mixed)
      e = launch_led_mixed(d_led + (size_t)st * J, d_lmap + loff[st], (int)lmap[st].size(), smem, r->stream, st > 0,
                           ff);
    else
      e = launch_led_jobs(m, C, d_led + (size_t)st * J, d_lpairs + loff[st], (int)lmap[st].size(), j0->er.W,
                          r->stream, st > 0, ff);
    if (e == cudaSuccess)
      e = launch_update_jobs(d_upd + (size_t)st * J, d_umap + uoff[st], (int)umap[st].size(), bmax[st], r->stream,
                             true, opt);
  }
  for (int q = 0; q < J && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(js[q]->pinned, js[q]->er.epoch, sizeof(double), cudaMemcpyDeviceToHost, r->stream);
  const cudaError_t e2 = cudaStreamEndCapture(r->stream, &g);
  if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&r->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  return (e == cudaSuccess && e2 == cudaSuccess) ? FPM_OK : FPM_ERR_CUDA;
}

// Launch one epoch of every job of a group as one round.
int launch_round(fpm_server* s, const std::vector<Job*>& js) {
  std::string key = group_key(s, js[0]);
  for (const Job* j : js) {
    char b[32];
    std::snprintf(b, sizeof b, " %p", (const void*)j);
    key += b;
  }
  auto it = s->rounds.find(key);
  Round* r;
  if (it == s->rounds.end()) {
    if (s->rounds.size() >= 32)  // bound the cache: drop the rounds not in flight
      for (auto jt = s->rounds.begin(); jt != s->rounds.end();) {
        if (!jt->second->in_flight) {
          destroy_round(jt->second.get());
          jt = s->rounds.erase(jt);
        } else {
          ++jt;
        }
      }
    auto nr = std::make_unique<Round>();
    const int rc = build_round(nr.get(), js, key.compare(0, 3, "mix") == 0);
    if (rc) {
      cudaGetLastError();
      destroy_round(nr.get());
      return rc;
    }
    r = nr.get();
    s->rounds.emplace(key, std::move(nr));
  } else {
    r = it->second.get();
  }
  for (size_t q = 0; q < js.size(); ++q) {
    Job* j = js[q];
    std::vector<int32_t> perm(j->er.n_leds);
    fpm_epoch_permutation(j->er.n_leds, j->desc.seed, j->epochs, perm.data());
    engine_round_slots(j->h, perm.data(), j->er.n_leds, j->h_slots);
    engine_round_coef(j->h, r->steps, j->h_coef);
    if (j->fresh) {  // order the job's load before its first round
      if (cudaStreamWaitEvent(r->stream, j->ev, 0) != cudaSuccess) return FPM_ERR_CUDA;
      j->fresh = false;
    }
  }
  if (cudaGraphLaunch(r->exec, r->stream) != cudaSuccess || cudaEventRecord(r->ev, r->stream) != cudaSuccess)
    return FPM_ERR_CUDA;
  r->in_flight = true;
  for (Job* j : js) j->in_flight = true;
  s->n_rounds += 1;
  s->n_round_epochs += (int64_t)js.size();
  s->max_round_jobs = std::max<int64_t>(s->max_round_jobs, (int64_t)js.size());
  s->n_launches += 2 * (int64_t)r->steps;
  return FPM_OK;
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
                  + steps * B * 16 + steps * (8 + 16);  // batch slots, losses, coefficients
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
  for (auto& kv : s->rounds) destroy_round(kv.second.get());  // waits for rounds in flight
  s->rounds.clear();
  for (Job* j : s->active)
    if (j->stream) cudaStreamSynchronize(j->stream);
  for (auto& kv : s->jobs)
    if (kv.second->state == FPM_JOB_ACTIVE) release(s, kv.second.get());
  for (auto& kv : s->pin_size) cudaFreeHost(kv.first);
  delete s;
}

const char* fpm_server_error(const fpm_server* s) { return s ? s->msg.c_str() : ""; }

int fpm_server_set_admission(fpm_server* s, int32_t order) {
  if (!s) return FPM_ERR_ARG;
  if (order != FPM_ADMIT_ARRIVAL && order != FPM_ADMIT_SMALLEST) return srv_fail(s, FPM_ERR_ARG, "unknown admission order");
  s->admission = order;
  return FPM_OK;
}

int fpm_server_set_grouping(fpm_server* s, int32_t grouping) {
  if (!s) return FPM_ERR_ARG;
  if (grouping < FPM_GROUP_CONFIG || grouping > FPM_GROUP_MIXED) return srv_fail(s, FPM_ERR_ARG, "unknown grouping");
  if (!s->rounds.empty() || !s->active.empty()) return srv_fail(s, FPM_ERR_STATE, "grouping set with jobs resident");
  s->grouping = grouping;
  return FPM_OK;
}

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
  // 1. retire the epochs that have finished: rounds whose events fired and
  //    jobs running their own epochs (retiring may free a job and its rounds,
  //    so the jobs are collected first)
  std::vector<std::pair<Job*, cudaError_t>> fin;
  for (auto& kv : s->rounds) {
    Round* r = kv.second.get();
    if (!r->in_flight) continue;
    const cudaError_t q = cudaEventQuery(r->ev);
    if (q == cudaErrorNotReady) continue;
    r->in_flight = false;
    for (Job* j : r->jobs) fin.emplace_back(j, q);
  }
  for (Job* j : s->active) {
    if (!j->in_flight || groupable(j)) continue;
    const cudaError_t q = cudaEventQuery(j->ev);
    if (q == cudaErrorNotReady) continue;
    fin.emplace_back(j, q);
  }
  for (auto& f : fin) {
    Job* j = f.first;
    if (j->state != FPM_JOB_ACTIVE) continue;
    if (f.second != cudaSuccess) {
      cudaGetLastError();
      j->in_flight = false;
      fail_job(s, j, cudaGetErrorString(f.second));
      continue;
    }
    const int rc = retire_epoch(s, j);
    if (rc) fail_job(s, j, fpm_last_error(j->h));
  }
  std::vector<Job*> still;
  for (Job* j : s->active)
    if (j->state == FPM_JOB_ACTIVE) still.push_back(j);
  s->active.swap(still);
  // 2. admit queued jobs in arrival order (or smallest expected work first),
  //    each one that fits the remaining memory (first fit: a job too large for
  //    now does not hold back smaller ones behind it), while slots allow
  if (s->admission == FPM_ADMIT_SMALLEST)
    std::stable_sort(s->queue.begin(), s->queue.end(), [](const Job* a, const Job* b) { return job_work(a) < job_work(b); });
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
  // 3. the next epoch of every resident job not in flight: one round per group
  std::map<std::string, std::vector<Job*>> groups;
  for (Job* j : s->active) {
    if (j->in_flight) continue;
    if (groupable(j)) {
      groups[group_key(s, j)].push_back(j);
    } else if (launch_epoch(j)) {
      fail_job(s, j, fpm_last_error(j->h));
    }
  }
  for (auto& kv : groups)
    if (launch_round(s, kv.second))
      for (Job* j : kv.second)
        if (j->state == FPM_JOB_ACTIVE) {
          j->in_flight = false;
          fail_job(s, j, "round launch failed");
        }
  still.clear();
  for (Job* j : s->active)
    if (j->state == FPM_JOB_ACTIVE) still.push_back(j);
  s->active.swap(still);
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  return FPM_OK;
}

int fpm_server_stats(const fpm_server* s, int64_t* rounds, int64_t* round_epochs, int64_t* max_jobs_per_round,
                     int64_t* launches) {
  if (!s) return FPM_ERR_ARG;
  if (rounds) *rounds = s->n_rounds;
  if (round_epochs) *round_epochs = s->n_round_epochs;
  if (max_jobs_per_round) *max_jobs_per_round = s->max_round_jobs;
  if (launches) *launches = s->n_launches;
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

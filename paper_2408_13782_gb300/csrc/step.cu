// Dataflow form of the Batch-FPM mini-batch step for 256 x 256 low-res images:
// the forward model of Section 2.1 Eq. (3), the loss of Section 2.2 Eq. (5)
// (Eq. (4) for the intensity form), its adjoint, and the random-batch update
// of Section 2.3 Eq. (13) with an Adam-family optimiser, in one launch.
//
// The spectrum of LED i is non-zero only on a W x W box (W = 2h + 1) around
// its crop centre, so the 256 x 256 inverse transform and its adjoint split
// into four sets of 256-point transforms:
//   A  T(c, y)  = sum_ky Phi(c, ky) e^{+2 pi i ky y / 256}   per box column c
//   B  psi(x,y) = sum_kx T(kx, y) e^{+2 pi i kx x / 256}     per image row y,
//      the residual field g(x, y) of the loss, then
//      U(c, y)  = sum_x g(x, y) e^{-2 pi i kx x / 256}       kept on the box
//   C  gPhi(c, ky) = sum_y U(c, y) e^{-2 pi i ky y / 256}     kept on the box,
//      then the object-gradient box conj(M) gPhi and the pupil-parameter terms
// followed by the update (D): the batch-ordered sum of the gradient boxes and
// the optimiser on every element of the update region and on every scalar.
//
// Instead of one thread-block cluster per LED image, every phase of every LED
// is cut into tasks of 8 transforms (a CTA of 128 threads, 16 per transform)
// and the CTAs of the launch (as many as fit on the GPU at once) take tasks in
// the order A, B, C, D from an atomic ticket counter. A task waits only for the
// tasks it reads: a row task of LED k for the column tasks of LED k, an adjoint
// column task of LED k for the row tasks of LED k, an update task for all
// adjoint column tasks. So the phases of different LEDs overlap and every SM
// works in every phase. T and U (B x W x 256 complex) pass between the phases
// through global memory (they stay in L2). Tasks are handed only to running
// CTAs, in increasing order, and each waits only for lower tickets, so the
// launch makes progress whatever the number of co-resident CTAs. Every wait is
// bounded: when it gives up it sets DERR_TIMEOUT (FPM_ERR_TIMEOUT on the host)
// and the task's outputs are not computed.
//
// The 256-point transforms are two radix-16 passes by 16 threads (thread j
// holds the points j + 16 n). With h < 64 the box lies in the points with
// n in {0..3, 12..15} only, so the first pass of an inverse transform whose
// inputs are the box (A, the first of B) and the last pass of a forward
// transform kept on the box (the second of B, C) are pruned. Between the two
// radix-16 passes of B the field stays in registers: the residual is formed on
// the inverse transform's outputs, which are already the forward transform's
// first-pass inputs.
//
// Every sum has a fixed order (per-task FP32 partials in fixed slots, FP64
// sums over the slots in slot order, the gradient boxes in batch order), so
// results are bitwise reproducible regardless of which CTA runs which task.
#include "../../include/fpm.h"
#include "device.cuh"
#include "internal.h"
#include "optim.cuh"
#include "pixel.cuh"

namespace fpmk {

namespace {

constexpr int SK_M = 256;                 // low-res side
constexpr int SK_G = 16;                  // threads per 256-point transform
constexpr int SK_NT = 128;                // threads per CTA
constexpr int SK_NG = SK_NT / SK_G;       // transforms per task (8)
constexpr int SK_NW = SK_NT / 32;         // warps
constexpr int SK_FS = SK_M + SK_M / 16;   // padded transform buffer (pidx16)
constexpr int SK_TS = SK_NG + 1;          // staging stride (float2) of one box column's 8 rows: odd, conflict-free
constexpr int SK_AS = SK_M + 16;          // image-row stride (floats): the two half-warps hit disjoint banks
constexpr int SK_NSC = 17;                // scalar update tasks: loss, 14 Zernike, defocus; per-LED parameters
constexpr int SK_NDECAY = 64;             // AdamW decay tasks (spectrum outside the update region)

// Dynamic shared memory: constant tables, then a region used either by the
// transform tasks or by the update tasks.
struct SkLayout {
  size_t tw2, zmt, poly, red, fsum, dred, misc, uni;  // byte offsets
  size_t buf, ts, as;                                 // inside the union: transform tasks
  size_t corner, lst, gl, inb;                        // inside the union: update tasks
  size_t total;
  __host__ __device__ SkLayout(int W, int B) {
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = (o + bytes + 15) & ~(size_t)15; return at; };
    tw2 = take(sizeof(float2) * 15 * 16);
    zmt = take(sizeof(float) * 14 * 15);
    poly = take(sizeof(float) * 40);
    red = take(sizeof(float) * SK_NW * 32);
    fsum = take(sizeof(float) * 32);
    dred = take(sizeof(double) * SK_NW);
    misc = take(sizeof(int) * 8);
    uni = o;
    size_t u = 0;
    auto utake = [&](size_t bytes) { const size_t at = uni + u; u = (u + bytes + 15) & ~(size_t)15; return at; };
    buf = utake(sizeof(float2) * SK_NG * SK_FS);
    ts = utake(sizeof(float2) * (size_t)W * SK_TS);
    as = utake(sizeof(float) * SK_NG * SK_AS);
    const size_t fft_bytes = u;
    u = 0;
    corner = utake(sizeof(int2) * (size_t)B);
    lst = utake(sizeof(int) * (size_t)B);
    gl = utake(sizeof(double) * 3 * (size_t)B);
    inb = utake(1024);
    const size_t upd_bytes = u;
    total = uni + (fft_bytes > upd_bytes ? fft_bytes : upd_bytes);
  }
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Thread 0: wait until *ctr >= target, at most s.wait_ns. On giving up (or when
// another wait already gave up) it records DERR_TIMEOUT and returns false.
// Polls with relaxed loads; the fence after the last one orders the task's
// reads after the producers' writes (which every consumer reads through L2).
__device__ bool wait_count(const StepArgs& s, const unsigned* ctr, unsigned target) {
  if (ld_relaxed(ctr) < target) {
    const unsigned long long t0 = globaltimer();
    unsigned ns = 20;
    while (ld_relaxed(ctr) < target) {
      if (ld_volatile(s.L.err) & DERR_TIMEOUT) return false;
      if ((long long)(globaltimer() - t0) > s.wait_ns) {
        atomicOr(s.L.err, DERR_TIMEOUT);
        return false;
      }
      __nanosleep(ns);
      ns = ns < 160 ? 2 * ns : ns;
    }
  }
  __threadfence();
  return true;
}

// All threads: wait for the tasks this one reads; thread 0 waits on the
// counter and shares the outcome through misc[4].
__device__ __forceinline__ bool cta_wait(const StepArgs& s, const unsigned* ctr, unsigned target, int* misc) {
  if (threadIdx.x == 0) misc[4] = wait_count(s, ctr, target) ? 1 : 0;
  __syncthreads();
  return misc[4] != 0;
}

// All threads: make the task's global writes visible, then count it done.
__device__ __forceinline__ void cta_signal(const StepArgs& s, unsigned* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
  }
}

// Between the two radix-16 passes of a 256-point transform by the 16 threads
// of a group: thread j's first-pass outputs (k1 = 0..15 of its column j) go
// to 16 j + k1; it takes the second-pass inputs j + 16 r with their twiddles
// W256^(r j) (DIR < 0) or their conjugates.
template <int DIR>
__device__ __forceinline__ void r16_exchange(float2 (&v)[16], float2* __restrict__ buf,
                                             const float2* __restrict__ tw2, int j) {
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[pidx16(16 * j + r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = buf[pidx16(j + 16 * r)];
#pragma unroll
  for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw_dir<DIR>(tw2[(r - 1) * 16 + j]));
}

// Points n of a thread that can lie in the box: all 16, or n in {0..3, 12..15}.
template <bool PRUNE>
__device__ __forceinline__ constexpr bool maybe_box(int n) {
  return !PRUNE || n < 4 || n >= 12;
}

struct Sk {  // shared-memory pointers of the CTA
  float2* tw2;
  float* zmt;
  float* poly;
  float* red;
  float* fsum;
  double* dred;
  int* misc;
  float2* buf;
  float2* ts;
  float* as;
  int2* corner;
  int* lst;
  double* gl;
  unsigned char* inb;
};

// Columns [c_lo, c_hi) of a column task (at most SK_NG).
__device__ __forceinline__ void task_columns(int W, int ntask, int t, int& c_lo, int& c_hi) {
  c_lo = t * W / ntask;
  c_hi = (t + 1) * W / ntask;
}

// Per-LED pupil quantities of batch slot k.
struct LedView {
  int led, row0;
  size_t col0;  // spectrum column of box column 0 (column-major O: index col * N + row)
  float gam, dly, dlx, zdef;
};

__device__ __forceinline__ bool led_view(const LedArgs& a, int k, LedView& v) {
  const int4 slot = a.slot[k];
  if (slot.x < 0 || slot.x >= a.n_leds) return false;
  v.led = slot.x;
  v.row0 = a.N / 2 + slot.y;
  v.col0 = (size_t)(a.N / 2 + slot.z - a.h);
  v.gam = a.sp[SP_GAMMA + v.led];
  v.dly = a.sp[sp_offset(a.n_leds) + 2 * v.led];
  v.dlx = a.sp[sp_offset(a.n_leds) + 2 * v.led + 1];
  v.zdef = a.sp[SP_DEFOCUS];
  return true;
}

// A pixel of the support can have A > 0 only inside this radius (squared);
// slightly generous, the exact amplitude decides.
__device__ __forceinline__ float support_r2(const PupilConst& P) {
  const float r = (P.hard_edge ? P.R : P.R + 0.5f) + 1e-3f;
  return r * r;
}

// ---------------------------------------------------------------- A ------
template <bool PRUNE>
__device__ void task_A(const StepArgs& s, const Sk& sm, int k, int ta) {
  const LedArgs& a = s.L;
  const int tid = threadIdx.x, grp = tid >> 4, j = tid & 15;
  const int W = a.W, h = a.h, N = a.N;
  int c_lo, c_hi;
  task_columns(W, s.nA, ta, c_lo, c_hi);
  const int c = c_lo + grp;
  const bool act = c < c_hi;
  LedView lv;
  if (!led_view(a, k, lv)) {  // the same for every thread: uniform
    if (tid == 0) atomicOr(a.err, DERR_INDEX);
    cta_signal(s, &s.sync->a_done[k].v);
    return;
  }
  if (tid == 0 && ta == 0 && !(fabsf(lv.dly) <= FPM_OFFSET_BOUND_PX && fabsf(lv.dlx) <= FPM_OFFSET_BOUND_PX))
    atomicOr(a.err, DERR_OFFSET);  // the box holds the support only within the bound
  const PupilConst P{a.R, a.Rinv, a.inv_lambda, a.dk2, a.hard_edge};
  const FreeForm ff = free_form(a.pupil, W, lv.dly, lv.dlx);
  if (a.pupil && a.pwt && tid == 0 && ta == 0) a.pwt[k] = make_float4(ff.fy, ff.fx, (float)ff.ay, (float)ff.ax);
  const float2* Oc = a.Ot + (lv.col0 + (act ? c : 0)) * N + lv.row0;  // index by ky
  const float qx = (float)(c - h) - lv.dlx, qx2 = qx * qx;
  const float rs2 = support_r2(P);
  float2 v[16];
  // O on the support first (every load in flight), then the pupil
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    v[n] = make_float2(0.f, 0.f);
    if (!maybe_box<PRUNE>(n)) continue;
    const int b = box256(j, n, h);
    const float qy = (float)(b - h) - lv.dly;
    if (act && b >= 0 && fmaf(qy, qy, qx2) <= rs2) v[n] = Oc[b - h];
  }
  ColPoly cp;
  col_poly(qx * P.Rinv, sm.poly, cp);
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    if (!maybe_box<PRUNE>(n)) continue;
    const int b = box256(j, n, h);
    const float qy = (float)(b - h) - lv.dly, r2 = fmaf(qy, qy, qx2);
    if (act && b >= 0 && r2 <= rs2) {
      float rad;
      const float A = pupil_amp_r2(r2, P, rad);
      v[n] = A > 0.f ? cmul(v[n], pupil_col(qy, r2, A, P, cp, lv.zdef)) : make_float2(0.f, 0.f);
      if (ff.P && A > 0.f) v[n] = cmul(v[n], ff_value(ff, b, c));
    }
  }
  float2* buf = sm.buf + grp * SK_FS;
  dft16p<+1, PRUNE, false>(v);
  r16_exchange<+1>(v, buf, sm.tw2, j);
  dft16p<+1, false, false>(v);
  if (act) {
    float2* Tc = s.T + ((size_t)k * W + c) * SK_M;
#pragma unroll
    for (int r = 0; r < 16; ++r) Tc[j + 16 * r] = v[r];
  }
  cta_signal(s, &s.sync->a_done[k].v);
}

// ---------------------------------------------------------------- B ------
template <bool PRUNE>
__device__ void task_B(const StepArgs& s, const Sk& sm, int k, int tb) {
  const LedArgs& a = s.L;
  const int tid = threadIdx.x, grp = tid >> 4, j = tid & 15;
  const int W = a.W, h = a.h;
  const int y0 = tb * SK_NG, y = y0 + grp;
  LedView lv;
  const bool ok = led_view(a, k, lv);
  const bool stored = a.mode == MODE_UPSTREAM_STORED;  // psi from memory: no inverse transforms
  const bool fwd = a.mode == MODE_FORWARD || a.mode == MODE_FORWARD_STORE;
  // the task's image rows (amplitudes, intensities or dL/dI), in flight during the wait
  const float* rows = a.mode == MODE_LOSS ? a.meas + ((size_t)(ok ? lv.led : 0) * SK_M + y0) * SK_M
                    : (a.mode == MODE_UPSTREAM || stored) ? a.dLdI + ((size_t)k * SK_M + y0) * SK_M : nullptr;
  if (ok && rows) {
    for (int q = tid; q < SK_NG * SK_M / 4; q += SK_NT) {
      const int r = q >> 6, x4 = q & 63;
      cp_async16(sm.as + r * SK_AS + 4 * x4, rows + (size_t)r * SK_M + 4 * x4);
    }
  }
  cp_async_commit();
  bool go = ok;
  if (!stored) {
    const bool w = cta_wait(s, &s.sync->a_done[k].v, (unsigned)s.nA + (s.stall ? 1u : 0u), sm.misc);
    go = go && w;
  }
  if (!ok && tid == 0) atomicOr(a.err, DERR_INDEX);
  cp_async_wait_all();
  float2* Tk = s.T + (size_t)k * W * SK_M;
  if (go && !stored) {  // rows y0..y0+7 of every box column of T
    for (int q = tid; q < W * 4; q += SK_NT) {
      const int c = q >> 2, p = q & 3;
      const float4 u = __ldcg(reinterpret_cast<const float4*>(Tk + (size_t)c * SK_M + y0) + p);
      sm.ts[c * SK_TS + 2 * p] = make_float2(u.x, u.y);
      sm.ts[c * SK_TS + 2 * p + 1] = make_float2(u.z, u.w);
    }
  }
  __syncthreads();
  float acc_loss = 0.f, acc_g = 0.f;
  if (go) {
    float2 v[16];
    float2* buf = sm.buf + grp * SK_FS;
    const float inv_m2 = 1.f / (float)(SK_M * SK_M);
    if (stored) {
      const float2* pr = a.psi + ((size_t)k * SK_M + y) * SK_M;
#pragma unroll
      for (int n = 0; n < 16; ++n) v[n] = pr[j + 16 * n];
    } else {
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        v[n] = make_float2(0.f, 0.f);
        if (!maybe_box<PRUNE>(n)) continue;
        const int b = box256(j, n, h);
        if (b >= 0) v[n] = sm.ts[b * SK_TS + grp];
      }
      dft16p<+1, PRUNE, false>(v);
      r16_exchange<+1>(v, buf, sm.tw2, j);
      dft16p<+1, false, false>(v);  // thread j: psi at x = j + 16 n (times m^2)
#pragma unroll
      for (int n = 0; n < 16; ++n) v[n] = cscale(v[n], inv_m2);
    }
    const float gam = lv.gam, sg = sqrtf(gam);
    const float* ar = sm.as + grp * SK_AS;
    if (fwd) {
      float* Io = a.I_out + ((size_t)k * SK_M + y) * SK_M;
#pragma unroll
      for (int n = 0; n < 16; ++n) Io[j + 16 * n] = gam * (v[n].x * v[n].x + v[n].y * v[n].y);
      if (a.mode == MODE_FORWARD_STORE) {
        float2* po = a.psi + ((size_t)k * SK_M + y) * SK_M;
#pragma unroll
        for (int n = 0; n < 16; ++n) po[j + 16 * n] = v[n];
      }
    } else {
      if (a.mode == MODE_LOSS && a.loss == FPM_LOSS_AMPLITUDE && a.meas_is_amp) {
#pragma unroll
        for (int n = 0; n < 16; ++n) v[n] = residual_amp_pixel(v[n], ar[j + 16 * n], sg, acc_loss, acc_g);
      } else if (a.mode == MODE_LOSS) {
#pragma unroll
        for (int n = 0; n < 16; ++n)
          v[n] = residual_pixel(v[n], ar[j + 16 * n], MODE_LOSS, a.loss, gam, sg, acc_loss, acc_g);
      } else {
#pragma unroll
        for (int n = 0; n < 16; ++n)
          v[n] = residual_pixel(v[n], ar[j + 16 * n], MODE_UPSTREAM, 0, gam, sg, acc_loss, acc_g);
      }
      // forward transform over x: thread j already holds the first-pass inputs
      dft16p<-1, false, false>(v);
      r16_exchange<-1>(v, buf, sm.tw2, j);
      dft16p<-1, false, PRUNE>(v);  // U at kx = j + 16 n, kept on the box
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        if (!maybe_box<PRUNE>(n)) continue;
        const int b = box256(j, n, h);
        if (b >= 0) sm.ts[b * SK_TS + grp] = v[n];
      }
    }
  }
  __syncthreads();
  if (go && !fwd) {  // U back over T's rows y0..y0+7 (only this task reads or writes them)
    for (int q = tid; q < W * 4; q += SK_NT) {
      const int c = q >> 2, p = q & 3;
      const float2 u0 = sm.ts[c * SK_TS + 2 * p], u1 = sm.ts[c * SK_TS + 2 * p + 1];
      reinterpret_cast<float4*>(Tk + (size_t)c * SK_M + y0)[p] = make_float4(u0.x, u0.y, u1.x, u1.y);
    }
  }
  if (!fwd) {  // per-task partials: loss and the gamma term
    acc_loss = warp_sum_f(acc_loss);
    acc_g = warp_sum_f(acc_g);
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) {
      sm.red[warp * 2] = acc_loss;
      sm.red[warp * 2 + 1] = acc_g;
    }
    __syncthreads();
    if (tid < 2) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < SK_NW; ++w) t += sm.red[w * 2 + tid];
      const bool amp_gamma = a.mode == MODE_LOSS && a.loss == FPM_LOSS_AMPLITUDE;
      double* out = s.partB + ((size_t)k * s.nB + tb) * STEP_NPB;
      out[tid] = !ok ? 0.0 : (tid == 1 && amp_gamma) ? (double)(t / sqrtf(lv.gam)) : (double)t;
    }
  }
  cta_signal(s, &s.sync->b_done[k].v);
}

// ---------------------------------------------------------------- C ------
template <bool PRUNE>
__device__ void task_C(const StepArgs& s, const Sk& sm, int k, int tc) {
  const LedArgs& a = s.L;
  const int tid = threadIdx.x, grp = tid >> 4, j = tid & 15;
  const int W = a.W, h = a.h, N = a.N;
  int c_lo, c_hi;
  task_columns(W, s.nC, tc, c_lo, c_hi);
  const int c = c_lo + grp;
  const bool act = c < c_hi;
  LedView lv;
  const bool ok = led_view(a, k, lv);
  const PupilConst P{a.R, a.Rinv, a.inv_lambda, a.dk2, a.hard_edge};
  const float qx = (float)(c - h) - (ok ? lv.dlx : 0.f), qx2 = qx * qx;
  const float rs2 = support_r2(P);
  // O on this thread's kept rows, loaded before the wait
  float2 o[16];
  const float2* Oc = a.Ot + ((ok ? lv.col0 : 0) + (act ? c : 0)) * N + (ok ? lv.row0 : 0);
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    o[n] = make_float2(0.f, 0.f);
    if (!maybe_box<PRUNE>(n)) continue;
    const int b = box256(j, n, h);
    const float qy = (float)(b - h) - (ok ? lv.dly : 0.f);
    if (ok && act && b >= 0 && fmaf(qy, qy, qx2) <= rs2) o[n] = Oc[b - h];
  }
  const bool w = cta_wait(s, &s.sync->b_done[k].v, (unsigned)s.nB, sm.misc);
  const bool go = ok && w;
  if (!ok && tid == 0) atomicOr(a.err, DERR_INDEX);
  float acc[18];
#pragma unroll
  for (int q = 0; q < 18; ++q) acc[q] = 0.f;
  if (go) {
    float2 v[16];
    const float2* Uc = s.T + ((size_t)k * W + (act ? c : 0)) * SK_M;
#pragma unroll
    for (int n = 0; n < 16; ++n) v[n] = act ? __ldcg(Uc + j + 16 * n) : make_float2(0.f, 0.f);
    float2* buf = sm.buf + grp * SK_FS;
    dft16p<-1, false, false>(v);
    r16_exchange<-1>(v, buf, sm.tw2, j);
    dft16p<-1, false, PRUNE>(v);  // gPhi at ky = j + 16 n (times m^2), kept on the box
    if (act) {
      const float inv_m2 = 1.f / (float)(SK_M * SK_M);
      ColPoly cp;
      col_poly(qx * P.Rinv, sm.poly, cp);
      BoxAcc bacc;
      box_acc_zero(bacc);
      float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      float2* gb = a.gbox + ((size_t)k * W + c) * W;
      float2* pb = a.pupil ? a.pbox + ((size_t)k * W + c) * W : nullptr;
      const FreeForm ff = free_form(a.pupil, W, lv.dly, lv.dlx);
#pragma unroll
      for (int n = 0; n < 16; ++n) {
        if (!maybe_box<PRUNE>(n)) continue;
        const int b = box256(j, n, h);
        if (b < 0) continue;
        const float qy = (float)(b - h) - lv.dly, r2 = fmaf(qy, qy, qx2);
        float rad;
        const float A = pupil_amp_r2(r2, P, rad);
        float2 out = make_float2(0.f, 0.f), Gp = out;
        if (A > 0.f)
          out = box_pixel_col(qy, qx, r2, A, rad, cscale(v[n], inv_m2), o[n], P, cp, lv.zdef, S, bacc, ff, b, c, &Gp);
        gb[b] = out;
        if (pb) pb[b] = Gp;
      }
      col_fold(cp, S, bacc);
#pragma unroll
      for (int q = 0; q < 15; ++q) acc[q] = bacc.m[q];
      acc[15] = bacc.def;
      acc[16] = bacc.dy;
      acc[17] = bacc.dx;
    }
  }
  // per-task partials: the 15 monomial moments (as 14 Zernike terms), defocus, dy, dx
  {
    const int warp = tid >> 5, lane = tid & 31;
    float v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = q < 18 ? acc[q] : 0.f;
    // recursive halving: after the step of distance o lane keeps the half of
    // its vector chosen by bit o and adds the partner's copy; lane q ends with
    // the warp total of value q
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < o; ++i) {
        const float keep = up ? v[i + o] : v[i];
        const float send = up ? v[i] : v[i + o];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    if (lane < 18) sm.red[warp * 32 + lane] = v[0];
    __syncthreads();
    if (tid < 18) {
      float t = 0.f;
#pragma unroll
      for (int w2 = 0; w2 < SK_NW; ++w2) t += sm.red[w2 * 32 + tid];
      sm.fsum[tid] = t;
    }
    __syncthreads();
    double* out = s.partC + ((size_t)k * s.nC + tc) * STEP_NPC;
    if (tid < 14) {  // dL/dc_j = sum_m (Z_j)_m * (sum_p t(p) mo_m(p))
      float z = 0.f;
#pragma unroll
      for (int m = 0; m < 15; ++m) z = fmaf(sm.zmt[tid * 15 + m], sm.fsum[m], z);
      out[tid] = z;
    } else if (tid < 17) {
      out[tid] = sm.fsum[tid + 1];  // defocus, dy, dx
    }
  }
  cta_signal(s, &s.sync->c_all.v);
}

// ---------------------------------------------------------------- D ------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Scalar task q < 16: one quantity shared by all LEDs (0 the loss, 1..14 the
// Zernike coefficients, 15 the defocus), the FP64 sum of its per-task partials.
__device__ void task_shared_scalar(const StepArgs& s, const Sk& sm, int q, float4 bc) {
  const UpdArgs& u = s.U;
  const int i = q == 0 ? -1 : q <= 14 ? SP_ZERN + q - 1 : SP_DEFOCUS;  // parameter index
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float w = 0.f, m = 0.f, v = 0.f;
  if (tid == 0 && i >= 0 && !u.assemble) {  // written only by earlier steps
    w = __ldcg(u.sp + i);
    m = __ldcg(u.msp + i);
    v = __ldcg(u.vsp + i);
  }
  const int B = u.B;
  if (!cta_wait(s, &s.sync->c_all.v, (unsigned)(B * s.nC), sm.misc)) return;
  const double* p = q == 0 ? s.partB : s.partC + (q - 1);
  const int n = q == 0 ? B * s.nB : B * s.nC;
  const int stride = q == 0 ? STEP_NPB : STEP_NPC;
  double acc = 0.0;
  for (int e = tid; e < n; e += SK_NT) acc += __ldcg(p + (size_t)e * stride);
  acc = warp_sum_d(acc);
  if (lane == 0) sm.dred[warp] = acc;
  __syncthreads();
  if (tid != 0) return;
  const double tot = (sm.dred[0] + sm.dred[1]) + (sm.dred[2] + sm.dred[3]);
  if (q == 0) {
    *u.loss_slot = tot;
    if (!u.assemble) *u.epoch_loss += tot;
    if (!isfinite(tot)) atomicOr(u.err, DERR_NONFINITE);
    return;
  }
  if (u.assemble) {
    u.g_sc[i] = (float)tot;
    return;
  }
  if (learned(u, i)) scalar_adam(u, i, w, m, v, tot, bc);
}

// FP64 sum of n <= 32 values at stride `stride` by a fixed pairwise tree.
__device__ __forceinline__ double tree_sum32(const double* p, int n, int stride) {
  double t[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) t[c] = c < n ? __ldcg(p + (size_t)c * stride) : 0.0;
#pragma unroll
  for (int w = 1; w < 32; w <<= 1)
#pragma unroll
    for (int c = 0; c + w < 32; c += 2 * w) t[c] += t[c + w];
  double r = t[0];
  for (int c = 32; c < n; ++c) r += __ldcg(p + (size_t)c * stride);
  return r;
}

// Scalar task 16: the per-LED intensity factors and offsets of every LED. The
// LEDs outside the batch have zero gradient and take their steps before the
// wait; after it only the batch's 3 B parameters remain.
__device__ void task_led_scalars(const StepArgs& s, const Sk& sm, float4 bc) {
  const UpdArgs& u = s.U;
  const int n = u.n_leds, tid = threadIdx.x, B = u.B;
  double* gl = sm.gl;
  unsigned char* in_batch = sm.inb;
  const bool small = n <= 1024;
  if (small) {
    for (int l = tid; l < n; l += SK_NT) in_batch[l] = 0;
    __syncthreads();
    for (int kk = tid; kk < B; kk += SK_NT) {
      const int led = u.slot[kk].x;
      if ((unsigned)led < (unsigned)n) in_batch[led] = 1;
    }
    __syncthreads();
  }
  auto idx_led = [&](int jj) { return jj < n ? jj : (jj - n) >> 1; };
  auto batch_param = [&](int q) {  // -1 for a slot whose LED index is out of range
    const int led = u.slot[q / 3].x, r = q % 3;
    if ((unsigned)led >= (unsigned)n) return -1;
    return r == 0 ? SP_GAMMA + led : sp_offset(n) + 2 * led + (r - 1);
  };
  if (!u.assemble)
    for (int jj = tid; jj < 3 * n; jj += SK_NT) {
      const int i = SP_GAMMA + jj;
      if (!small || in_batch[idx_led(jj)] || !learned(u, i)) continue;
      scalar_adam(u, i, __ldcg(u.sp + i), __ldcg(u.msp + i), __ldcg(u.vsp + i), 0.0, bc);
    }
  if (!cta_wait(s, &s.sync->c_all.v, (unsigned)(B * s.nC), sm.misc)) return;
  for (int q = tid; q < 3 * B; q += SK_NT) {
    const int kk = q / 3, r = q - 3 * kk;
    gl[q] = r == 0 ? tree_sum32(s.partB + (size_t)kk * s.nB * STEP_NPB + 1, s.nB, STEP_NPB)
                   : tree_sum32(s.partC + (size_t)kk * s.nC * STEP_NPC + 14 + r, s.nC, STEP_NPC);
  }
  __syncthreads();
  if (u.assemble) {
    for (int jj = tid; jj < 3 * n; jj += SK_NT) u.g_sc[SP_GAMMA + jj] = 0.f;
    __syncthreads();
    for (int q = tid; q < 3 * B; q += SK_NT) {
      const int i = batch_param(q);
      if (i >= 0) u.g_sc[i] = (float)gl[q];
    }
    return;
  }
  if (small) {
    for (int q = tid; q < 3 * B; q += SK_NT) {
      const int i = batch_param(q);
      if (i < 0 || !learned(u, i)) continue;
      scalar_adam(u, i, __ldcg(u.sp + i), __ldcg(u.msp + i), __ldcg(u.vsp + i), gl[q], bc);
    }
    return;
  }
  for (int jj = tid; jj < 3 * n; jj += SK_NT) {
    const int i = SP_GAMMA + jj, led = idx_led(jj);
    if (!learned(u, i)) continue;
    double g = 0.0;
    for (int kk = 0; kk < B; ++kk)
      if (u.slot[kk].x == led) g = gl[3 * kk + (jj < n ? 0 : 1 + ((jj - n) & 1))];
    scalar_adam(u, i, __ldcg(u.sp + i), __ldcg(u.msp + i), __ldcg(u.vsp + i), g, bc);
  }
}

// AdamW's decoupled decay on the spectrum outside the update region (no crop
// reads it, so it needs no wait): columns q, q + SK_NDECAY, ...
__device__ void task_decay(const UpdArgs& u, int q) {
  const float f = 1.f - u.lr_obj * u.wd;
  for (int x = q; x < u.N; x += SK_NDECAY) {
    const int2 sp = u.span[x];
    float2* col = u.Ot + (size_t)x * u.N;
    for (int y = threadIdx.x; y < u.N; y += SK_NT)
      if (y < sp.x || y >= sp.y) {
        float2 w = col[y];
        w.x *= f;
        w.y *= f;
        col[y] = w;
      }
  }
}

// One spectrum column x of the update region: every element gathers the
// gradient boxes that cover it in batch order and takes one optimiser step
// (or, assembling, writes the gradient). A thread takes the rows
// span.x + tid + 128 i; the first PRE of them are loaded before the wait and
// their box loads are all in flight together.
template <int NE>
__device__ __forceinline__ void column_rows(const UpdArgs& u, const Sk& sm, int x, int n_l, int y_first, int y_end,
                                           float2 (&w)[NE], float2 (&m)[NE], float2 (&v)[NE], bool loaded, float4 bc) {
  const int W = u.W;
  float2 g[NE];
#pragma unroll
  for (int i = 0; i < NE; ++i) g[i] = make_float2(0.f, 0.f);
  for (int q = 0; q < n_l; q += 8) {
    float2 t[NE][8];
#pragma unroll
    for (int i = 0; i < NE; ++i)
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        t[i][e] = make_float2(0.f, 0.f);
        const int y = y_first + SK_NT * i;
        if (q + e < n_l && y < y_end) {
          const int kk = sm.lst[q + e];
          const int ry = y - sm.corner[kk].y, cx = x - sm.corner[kk].x;
          if ((unsigned)ry < (unsigned)W) t[i][e] = __ldcg(u.gbox + ((size_t)kk * W + cx) * W + ry);
        }
      }
#pragma unroll
    for (int i = 0; i < NE; ++i)
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (q + e < n_l) g[i] = cadd(g[i], t[i][e]);
  }
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    const int y = y_first + SK_NT * i;
    if (y >= y_end) continue;
    const size_t o = (size_t)x * u.N + y;
    if (u.assemble) {
      u.g_obj[o] = g[i];
      continue;
    }
    float2 ww = w[i], mm = m[i], vv = v[i];
    if (!loaded) {
      ww = __ldcg(u.Ot + o);
      mm = __ldcg(u.mO + o);
      vv = __ldcg(u.vO + o);
    }
    opt1(u, ww.x, mm.x, vv.x, g[i].x, u.lr_obj, bc);
    opt1(u, ww.y, mm.y, vv.y, g[i].y, u.lr_obj, bc);
    u.Ot[o] = ww;
    u.mO[o] = mm;
    u.vO[o] = vv;
  }
}

__device__ void task_column(const StepArgs& s, const Sk& sm, int xc, float4 bc) {
  const UpdArgs& u = s.U;
  const int tid = threadIdx.x, B = u.B, W = u.W, N = u.N;
  const int x = u.x_lo + xc;
  const int2 span = u.span[x];
  for (int kk = tid; kk < B; kk += SK_NT) {
    const int4 sl = u.slot[kk];
    sm.corner[kk] = make_int2(N / 2 + sl.z - u.h, N / 2 + sl.y - u.h);
  }
  constexpr int PRE = 3;  // elements per thread loaded before the wait
  float2 w[PRE], m[PRE], v[PRE];
  const int y_first = span.x + tid;
#pragma unroll
  for (int i = 0; i < PRE; ++i) {
    const int y = y_first + SK_NT * i;
    w[i] = m[i] = v[i] = make_float2(0.f, 0.f);
    if (!u.assemble && y < span.y) {
      const size_t o = (size_t)x * N + y;
      w[i] = __ldcg(u.Ot + o);
      m[i] = __ldcg(u.mO + o);
      v[i] = __ldcg(u.vO + o);
    }
  }
  __syncthreads();
  if (tid == 0) {  // batch slots whose box covers this column, in batch order
    int c = 0;
    for (int kk = 0; kk < B; ++kk)
      if ((unsigned)(x - sm.corner[kk].x) < (unsigned)W) sm.lst[c++] = kk;
    sm.misc[5] = c;
  }
  if (!cta_wait(s, &s.sync->c_all.v, (unsigned)(B * s.nC), sm.misc)) return;
  const int n_l = sm.misc[5];
  column_rows<PRE>(u, sm, x, n_l, y_first, span.y, w, m, v, true, bc);
  // taller columns (high-res sides above 384 rows of update region)
  for (int y = y_first + SK_NT * PRE; y < span.y; y += SK_NT) {
    float2 w1[1], m1[1], v1[1];
    column_rows<1>(u, sm, x, n_l, y, span.y, w1, m1, v1, false, bc);
  }
}

// One node column of the free-form pupil: the gather of the pupil-gradient
// boxes and the optimiser (see pupil_node).
__device__ void task_pupil_column(const StepArgs& s, const Sk& sm, int cn, float4 bc) {
  const UpdArgs& u = s.U;
  const int W = u.W;
  constexpr int PRE = 2;  // W <= 255 nodes: two per thread
  float2 w[PRE], m[PRE], v[PRE];
#pragma unroll
  for (int i = 0; i < PRE; ++i) {
    const int rn = threadIdx.x + SK_NT * i;
    w[i] = m[i] = v[i] = make_float2(0.f, 0.f);
    if (!u.assemble && rn < W) {
      const size_t o = (size_t)cn * W + rn;
      w[i] = __ldcg(u.Pff + o);
      m[i] = __ldcg(u.mPff + o);
      v[i] = __ldcg(u.vPff + o);
    }
  }
  if (!cta_wait(s, &s.sync->c_all.v, (unsigned)(u.B * s.nC), sm.misc)) return;
#pragma unroll
  for (int i = 0; i < PRE; ++i) {
    const int rn = threadIdx.x + SK_NT * i;
    if (rn < W) pupil_node(u, cn, rn, w[i], m[i], v[i], bc);
  }
}

// ------------------------------------------------------------ kernel -----
template <bool PRUNE>
__global__ void __launch_bounds__(SK_NT, 4) step_kernel(const StepArgs s) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LedArgs& a = s.L;
  const SkLayout lay(a.W, a.B);
  Sk sm;
  sm.tw2 = reinterpret_cast<float2*>(smem + lay.tw2);
  sm.zmt = reinterpret_cast<float*>(smem + lay.zmt);
  sm.poly = reinterpret_cast<float*>(smem + lay.poly);
  sm.red = reinterpret_cast<float*>(smem + lay.red);
  sm.fsum = reinterpret_cast<float*>(smem + lay.fsum);
  sm.dred = reinterpret_cast<double*>(smem + lay.dred);
  sm.misc = reinterpret_cast<int*>(smem + lay.misc);
  sm.buf = reinterpret_cast<float2*>(smem + lay.buf);
  sm.ts = reinterpret_cast<float2*>(smem + lay.ts);
  sm.as = reinterpret_cast<float*>(smem + lay.as);
  sm.corner = reinterpret_cast<int2*>(smem + lay.corner);
  sm.lst = reinterpret_cast<int*>(smem + lay.lst);
  sm.gl = reinterpret_cast<double*>(smem + lay.gl);
  sm.inb = smem + lay.inb;
  const int tid = threadIdx.x;

  // constant tables (not written by any step)
  for (int t = tid; t < 15 * 16; t += SK_NT) sm.tw2[t] = a.tw[(t / 16 + 1) * (t % 16)];
  for (int t = tid; t < 14 * 15; t += SK_NT) sm.zmt[t] = zern_mono_table()[t];
  // the previous step (programmatic dependent launch) must be complete before
  // the counters, O or the scalar parameters are touched
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  if (tid < 14) sm.fsum[tid] = a.sp[SP_ZERN + tid];  // the aberration coefficients
  __syncthreads();
  if (tid < 35) sm.poly[tid] = theta_poly_entry_tab(sm.fsum, sm.zmt, tid);  // phase as monomials of q/R

  const int B = a.B;
  const int TA = a.mode == MODE_UPSTREAM_STORED ? 0 : B * s.nA;
  const int TB = B * s.nB;
  const int TC = s.do_update ? B * s.nC : 0;
  const UpdArgs& u = s.U;
  const bool decay = s.do_update && u.opt == FPM_OPT_ADAMW && u.wd > 0.f && !u.assemble && (u.learn & 1u);
  const int TDEC = decay ? SK_NDECAY : 0;
  const int TS = s.do_update ? SK_NSC : 0;
  const int TCOL = s.do_update && (u.assemble || (u.learn & 1u)) ? u.n_cols : 0;
  const int TPUP = s.do_update ? u.pupil_cols : 0;
  const int total = TA + TB + TC + TDEC + TS + TCOL + TPUP;
  const float4 bc = s.do_update && u.coef ? u.coef[u.step_off] : make_float4(1.f, 1.f, 0.f, 0.f);

  if (tid == 0) sm.misc[0] = (int)atomicAdd(&s.sync->ticket.v, 1u);
  __syncthreads();
  int t = sm.misc[0];
  for (int it = 0; t < total; ++it) {
    int r = t;
    if (r < TA) {
      task_A<PRUNE>(s, sm, r / s.nA, r % s.nA);
    } else if ((r -= TA) < TB) {
      task_B<PRUNE>(s, sm, r / s.nB, r % s.nB);
    } else if ((r -= TB) < TC) {
      task_C<PRUNE>(s, sm, r / s.nC, r % s.nC);
    } else if ((r -= TC) < TDEC) {
      task_decay(u, r);
    } else if ((r -= TDEC) < TS) {
      if (r < 16) task_shared_scalar(s, sm, r, bc);
      else task_led_scalars(s, sm, bc);
    } else if ((r -= TS) < TCOL) {
      task_column(s, sm, r, bc);
    } else {
      task_pupil_column(s, sm, r - TCOL, bc);
    }
    // the next ticket, taken once this task is done (a ticket taken earlier
    // would hold a task back behind this one)
    const int slot = 1 + ((it + 1) & 1);
    if (tid == 0) sm.misc[slot] = (int)atomicAdd(&s.sync->ticket.v, 1u);
    __syncthreads();
    t = sm.misc[slot];
  }

  // the last CTA to finish resets the counters for the next launch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    sm.misc[3] = atomicAdd(&s.sync->exit_count.v, 1u) == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (sm.misc[3]) {
    __threadfence();
    for (int kk = tid; kk < B; kk += SK_NT) {
      s.sync->a_done[kk].v = 0u;
      s.sync->b_done[kk].v = 0u;
    }
    if (tid == 0) {
      s.sync->ticket.v = 0u;
      s.sync->c_all.v = 0u;
      s.sync->exit_count.v = 0u;
    }
  }
}

}  // namespace

size_t step_smem_bytes(int W, int B) { return SkLayout(W, B).total; }

int step_tasks(const StepArgs& s) {
  const int B = s.L.B;
  int t = (s.L.mode == MODE_UPSTREAM_STORED ? 0 : B * s.nA) + B * s.nB;
  if (s.do_update) {
    const UpdArgs& u = s.U;
    const bool decay = u.opt == FPM_OPT_ADAMW && u.wd > 0.f && !u.assemble && (u.learn & 1u);
    t += B * s.nC + (decay ? SK_NDECAY : 0) + SK_NSC + (u.assemble || (u.learn & 1u) ? u.n_cols : 0) +
         u.pupil_cols;
  }
  return t;
}

// Attributes of both instantiations, and the CTAs that fit on the device at
// once for a launch of box width W and batch B.
cudaError_t step_prepare(int W, int B, int* max_ctas) {
  int dev = 0, optin = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const size_t bytes = step_smem_bytes(W, B);
  if (bytes > (size_t)optin) return cudaErrorInvalidValue;
  const void* fns[2] = {(const void*)step_kernel<true>, (const void*)step_kernel<false>};
  for (const void* f : fns) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<true>, SK_NT, bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (max_ctas) *max_ctas = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_step(const StepArgs& s, int max_ctas, cudaStream_t st, bool pdl) {
  if (s.L.h >= 128 || s.L.W != 2 * s.L.h + 1) return cudaErrorInvalidValue;
  const int total = step_tasks(s);
  const int grid = total < max_ctas ? total : max_ctas;
  if (grid < 1) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(SK_NT, 1, 1);
  cfg.dynamicSmemBytes = step_smem_bytes(s.L.W, s.L.B);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  if (s.L.h < 64) return cudaLaunchKernelEx(&cfg, step_kernel<true>, s);
  return cudaLaunchKernelEx(&cfg, step_kernel<false>, s);
}

}  // namespace fpmk

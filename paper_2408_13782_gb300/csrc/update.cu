// Random-batch update (Section 2.3, Eq. 13) with an optimiser of the Adam
// family (Adam, AdamW, NAdam, RMSprop; the rules are in fpm.h). The per-step
// coefficients (bias corrections, NAdam's momentum schedule) are computed on
// the host in FP64 and passed in per step (no FP64 math here apart from the
// fixed-order reduction of the FP64 partials).
//
// Object: every element of the update region (the union of all LEDs' crop
// boxes; outside it the gradient has always been zero and Adam is an exact
// no-op) gathers the per-LED gradient boxes in batch order - a fixed-order
// sum, so results are bitwise reproducible - and takes one Adam step on its
// real and imaginary parts. One CTA per spectrum column of the region.
// Scalars: 17 CTAs reduce the per-CTA FP64 partials in a fixed order, one per
// quantity shared by all LEDs and one for the per-LED parameters, and update
// all of them (every element, every step).
#include <cmath>

#include "../../include/fpm.h"
#include "device.cuh"
#include "internal.h"
#include "optim.cuh"

namespace fpmk {

// Threads per CTA: enough that a column of the update region is one element
// per thread (up to 320 rows; 273 on a 15 x 15 grid of pitch 12 at m = 256),
// so every element's box loads and Adam step are in flight at once.
constexpr int UPD_NT = 320;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The scalar parameters are updated by NSC CTAs in parallel: CTA q < 16 owns
// one quantity shared by all LEDs (q = 0 the loss, 1..14 the Zernike
// coefficients, 15 the defocus) and sums it over all B x C per-CTA partials
// with a fixed tree; CTA 16 owns the per-LED intensity factors and offsets,
// each the sum of its slot's C partials in rank order. Every parameter takes
// an Adam step every step (zero gradient for LEDs outside the batch).
constexpr int NSC = 17;

// CTA q < 16: one shared quantity.
__device__ void shared_scalar(const UpdArgs& a, int q, float4 k) {
  __shared__ double wsum[UPD_NT / 32];
  const int P = q == 0 ? P_LOSS : q <= 14 ? P_ZERN + q - 1 : P_DEFOCUS;
  const int i = q == 0 ? -1 : q <= 14 ? SP_ZERN + q - 1 : SP_DEFOCUS;  // parameter index
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float w = 0.f, m = 0.f, v = 0.f;
  if (tid == 0 && i >= 0 && !a.assemble) {  // written only by earlier update kernels
    w = __ldcg(a.sp + i);
    m = __ldcg(a.msp + i);
    v = __ldcg(a.vsp + i);
  }
  asm volatile("griddepcontrol.wait;\n" ::: "memory");  // partials of the LED kernel
  const int nparts = a.B * a.C;
  double s = 0.0;
  for (int e = tid; e < nparts; e += blockDim.x) s += a.part[(size_t)e * NPART + P];
  s = warp_sum_d(s);
  if (lane == 0) wsum[warp] = s;
  __syncthreads();
  if (tid != 0) return;
  // the warps' sums by a fixed pairwise tree (short FP64 dependency chains)
  double ws[UPD_NT / 32];
#pragma unroll
  for (int k = 0; k < UPD_NT / 32; ++k) ws[k] = wsum[k];
#pragma unroll
  for (int w = 1; w < UPD_NT / 32; w <<= 1)
#pragma unroll
    for (int k = 0; k + w < UPD_NT / 32; k += 2 * w) ws[k] += ws[k + w];
  const double tot = ws[0];
  if (q == 0) {
    *a.loss_slot = tot;
    if (!a.assemble) *a.epoch_loss += tot;
    if (!isfinite(tot)) atomicOr(a.err, DERR_NONFINITE);
    return;
  }
  if (a.assemble) {
    a.g_sc[i] = (float)tot;
    return;
  }
  if (learned(a, i)) scalar_adam(a, i, w, m, v, tot, k);
}

// CTA 16: the per-LED intensity factors and offsets of every LED. The LEDs
// outside the batch have zero gradient and are not read by this step's LED
// kernel, so their Adam steps run before the wait; after it only the batch's
// 3 B parameters remain.
__device__ void led_scalars(const UpdArgs& a, float4 k) {
  extern __shared__ double gl[];  // [3 B]: per batch slot gamma, dy, dx
  __shared__ unsigned char in_batch[1024];
  const int n = a.n_leds, tid = threadIdx.x;
  const bool small = n <= 1024;  // else every LED waits (no membership table)
  if (small) {
    for (int l = tid; l < n; l += blockDim.x) in_batch[l] = 0;
    __syncthreads();
    for (int kk = tid; kk < a.B; kk += blockDim.x) in_batch[a.slot[kk].x] = 1;
    __syncthreads();
  }
  auto idx_led = [&](int j) { return j < n ? j : (j - n) >> 1; };  // parameter j of the 3n -> its LED
  auto batch_param = [&](int q) {  // parameter r = q % 3 (gamma, dy, dx) of batch slot q / 3
    const int led = a.slot[q / 3].x, r = q % 3;
    return r == 0 ? SP_GAMMA + led : sp_offset(n) + 2 * led + (r - 1);
  };
  // the batch's own parameter state, for the Adam steps after the wait (one per thread)
  float bw = 0.f, bm = 0.f, bv = 0.f;
  const int bi = tid < 3 * a.B ? batch_param(tid) : -1;  // (the slot table is not read again after the wait)
  if (!a.assemble && tid < 3 * a.B) {
    const int i = bi;
    bw = __ldcg(a.sp + i);
    bm = __ldcg(a.msp + i);
    bv = __ldcg(a.vsp + i);
  }
  if (!a.assemble)
    for (int j = tid; j < 3 * n; j += blockDim.x) {
      const int i = SP_GAMMA + j;
      if (!small || in_batch[idx_led(j)] || !learned(a, i)) continue;
      scalar_adam(a, i, __ldcg(a.sp + i), __ldcg(a.msp + i), __ldcg(a.vsp + i), 0.0, k);
    }
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  // one thread per (slot, quantity) sums the slot's C partials with a fixed
  // pairwise tree over the ranks: all loads in flight, four levels of FP64
  // adds on two warps (FP64 is slow on this part: no long dependent chains
  // and no shuffle tree over all the CTA's warps)
  const int C = a.C;
  for (int q = tid; q < 3 * a.B; q += blockDim.x) {
    const int kk = q / 3, r = q - 3 * kk;
    const double* p = a.part + (size_t)kk * C * NPART + (r == 0 ? P_GAMMA : r == 1 ? P_DY : P_DX);
    double t[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) t[c] = c < C ? p[(size_t)c * NPART] : 0.0;
#pragma unroll
    for (int w = 1; w < 16; w <<= 1)
#pragma unroll
      for (int c = 0; c + w < 16; c += 2 * w) t[c] += t[c + w];
    for (int c = 16; c < C; ++c) t[0] += p[(size_t)c * NPART];
    gl[q] = t[0];
  }
  __syncthreads();
  if (a.assemble) {  // gradients of every LED: zero outside the batch
    for (int j = tid; j < 3 * n; j += blockDim.x) a.g_sc[SP_GAMMA + j] = 0.f;
    __syncthreads();
    for (int q = tid; q < 3 * a.B; q += blockDim.x) {
      const int led = a.slot[q / 3].x, r = q % 3;
      a.g_sc[r == 0 ? SP_GAMMA + led : sp_offset(n) + 2 * led + (r - 1)] = (float)gl[q];
    }
    return;
  }
  if (small) {
    for (int q = tid; q < 3 * a.B; q += blockDim.x) {
      const int i = q == tid ? bi : batch_param(q);
      if (!learned(a, i)) continue;
      if (q == tid) scalar_adam(a, i, bw, bm, bv, gl[q], k);
      else scalar_adam(a, i, a.sp[i], a.msp[i], a.vsp[i], gl[q], k);
    }
    return;
  }
  // many LEDs: every parameter here, the batch's from the sums
  for (int j = tid; j < 3 * n; j += blockDim.x) {
    const int i = SP_GAMMA + j, led = idx_led(j);
    if (!learned(a, i)) continue;
    double g = 0.0;
    for (int kk = 0; kk < a.B; ++kk)
      if (a.slot[kk].x == led) g = gl[3 * kk + (j < n ? 0 : 1 + ((j - n) & 1))];
    scalar_adam(a, i, a.sp[i], a.msp[i], a.vsp[i], g, k);
  }
}

// AdamW's decoupled decay reaches every element of the object spectrum, also
// those outside the update region, whose gradient is always zero (there every
// other rule of the family is an exact no-op). NDECAY extra CTAs take the
// columns q, q + NDECAY, ... and scale the rows outside the region. No
// per-LED kernel reads those elements (every crop box lies inside the
// region), so this runs before the grid-dependency wait.
constexpr int NDECAY = 64;

__device__ void decay_outside(const UpdArgs& a, int q) {
  const float f = 1.f - a.lr_obj * a.wd;
  for (int x = q; x < a.N; x += NDECAY) {
    const int2 sp = a.span[x];  // rows [sp.x, sp.y) of the region (empty: (N, 0))
    float2* col = a.Ot + (size_t)x * a.N;
    for (int y = threadIdx.x; y < a.N; y += blockDim.x)
      if (y < sp.x || y >= sp.y) {
        float2 w = col[y];
        w.x *= f;
        w.y *= f;
        col[y] = w;
      }
  }
}

// AdamW's decay CTAs of a launch (0 or NDECAY).
__host__ __device__ inline int update_decay_ctas(const UpdArgs& a) {
  const bool decay = a.opt == FPM_OPT_ADAMW && a.wd > 0.f && !a.assemble && (a.learn & 1u);
  return decay ? NDECAY : 0;
}

// CTA bid of the update of the job described by a. OPT: the optimiser fixed at
// compile time for the object elements (a.opt), or -1 to branch on a.opt.
template <int OPT>
__device__ __forceinline__ void update_body(const UpdArgs& a, const int bid) {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  // the launch's dynamic shared memory (3 B doubles) holds, in the column
  // CTAs, the first column and row of each slot's box and the list of slots
  // that cover the column: batch-sized, so the CTA stays small
  extern __shared__ double dyn_smem[];
  int2* corner = reinterpret_cast<int2*>(dyn_smem);  // [B]
  int* lst = reinterpret_cast<int*>(corner + a.B);     // [B]
  __shared__ int nl;
  // Everything read before the wait is untouched by the LED kernel this
  // kernel depends on: step coefficients, LED tables, and O, m, v (the LED
  // kernel only reads O, and lets this kernel start only after the previous
  // update has completed). The gradient boxes and partials come after it.
  const float4 bc = a.coef ? a.coef[a.step_off] : make_float4(1.f, 1.f, 0.f, 0.f);
  if (bid < NSC) {  // the scalar parameters (the longest dependency chain)
    if (bid < 16) shared_scalar(a, bid, bc);
    else led_scalars(a, bc);
    return;
  }
  if (bid >= NSC + a.n_cols + update_decay_ctas(a)) {  // free-form pupil: one CTA per node column
    const int cn = bid - NSC - a.n_cols - update_decay_ctas(a);
    float2 w0 = make_float2(0.f, 0.f), m0 = w0, v0 = w0;
    const int rn = threadIdx.x;  // W <= 255 < UPD_NT: one node per thread
    if (!a.assemble && rn < a.W) {
      const size_t o = (size_t)cn * a.W + rn;
      w0 = __ldcg(a.Pff + o);
      m0 = __ldcg(a.mPff + o);
      v0 = __ldcg(a.vPff + o);
    }
    asm volatile("griddepcontrol.wait;\n" ::: "memory");  // pupil-gradient boxes of the LED kernel
    if (rn < a.W) pupil_node(a, cn, rn, w0, m0, v0, bc);
    return;
  }
  if (bid >= NSC + a.n_cols) {  // AdamW only (see update_ctas)
    decay_outside(a, bid - NSC - a.n_cols);
    return;
  }
  if (!a.assemble && !(a.learn & 1u)) return;
  const int x = a.x_lo + bid - NSC;
  const int W = a.W;
  const int2 span = a.span[x];
  for (int kk = threadIdx.x; kk < a.B; kk += blockDim.x) {
    const int4 sl = a.slot[kk];
    corner[kk] = make_int2(a.N / 2 + sl.z - a.h, a.N / 2 + sl.y - a.h);
  }
  // this thread's first two elements of the column (taller columns at
  // m = 512 need the second), loaded before the wait
  const int y0 = span.x + (int)threadIdx.x, y1 = y0 + (int)blockDim.x;
  float2 w0 = make_float2(0.f, 0.f), m0 = w0, v0 = w0, w1 = w0, m1 = w0, v1 = w0;
  if (!a.assemble && y0 < span.y) {
    const size_t o = (size_t)x * a.N + y0;
    w0 = __ldcg(a.Ot + o);  // L2 (not L1): written by the previous update kernel
    m0 = __ldcg(a.mO + o);
    v0 = __ldcg(a.vO + o);
  }
  if (!a.assemble && y1 < span.y) {
    const size_t o = (size_t)x * a.N + y1;
    w1 = __ldcg(a.Ot + o);
    m1 = __ldcg(a.mO + o);
    v1 = __ldcg(a.vO + o);
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // batch slots whose box covers this column, in batch order
    int c = 0;
    for (int kk = 0; kk < a.B; ++kk)
      if ((unsigned)(x - corner[kk].x) < (unsigned)W) lst[c++] = kk;
    nl = c;
  }
  asm volatile("griddepcontrol.wait;\n" ::: "memory");  // gradient boxes of the LED kernel
  __syncthreads();
  const int n_l = nl;
  for (int y = y0; y < span.y; y += blockDim.x) {
    const size_t o = (size_t)x * a.N + y;
    float2 w, m, v;
    if (!a.assemble) {
      if (y == y0) {
        w = w0; m = m0; v = v0;
      } else if (y == y1) {
        w = w1; m = m1; v = v1;
      } else {
        w = a.Ot[o]; m = a.mO[o]; v = a.vO[o];
      }
    }
    // sum of the covering boxes in batch order (adding zeros where a box
    // does not reach this row), sixteen loads in flight at a time
    float2 g = make_float2(0.f, 0.f);
    int q = 0;
    for (; q + 16 <= n_l; q += 16) {
      float2 t[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int kk = lst[q + u];
        const int ry = y - corner[kk].y, cx = x - corner[kk].x;
        t[u] = (unsigned)ry < (unsigned)W ? a.gbox[((size_t)kk * W + cx) * W + ry] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) g = cadd(g, t[u]);
    }
    if (q < n_l) {  // the rest (fewer than 16), also all in flight before the sum
      float2 t[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        t[u] = make_float2(0.f, 0.f);
        if (q + u < n_l) {
          const int kk = lst[q + u];
          const int ry = y - corner[kk].y, cx = x - corner[kk].x;
          if ((unsigned)ry < (unsigned)W) t[u] = a.gbox[((size_t)kk * W + cx) * W + ry];
        }
      }
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (q + u < n_l) g = cadd(g, t[u]);
    }
    if (a.assemble) {
      a.g_obj[o] = g;
      continue;
    }
    opt1<OPT>(a, w.x, m.x, v.x, g.x, a.lr_obj, bc);
    opt1<OPT>(a, w.y, m.y, v.y, g.y, a.lr_obj, bc);
    a.Ot[o] = w;
    a.mO[o] = m;
    a.vO[o] = v;
  }
}

// One job; one instantiation per optimiser, so the element loop carries only its rule.
template <int OPT>
__global__ void __launch_bounds__(UPD_NT) update_kernel(const UpdArgs a) { update_body<OPT>(a, (int)blockIdx.x); }

// Several jobs in one launch (the serving loop): CTA q is CTA map[q].y of the
// update of job map[q].x, whose arguments are copied to shared memory. OPT:
// the optimiser every job of the launch uses (Adam), or -1 to branch per job.
template <int OPT>
__global__ void __launch_bounds__(UPD_NT) update_kernel_jobs(const UpdArgs* __restrict__ jobs,
                                                             const int2* __restrict__ map) {
  __shared__ UpdArgs sa;
  const int2 q = map[blockIdx.x];
  if (threadIdx.x == 0) sa = jobs[q.x];
  __syncthreads();
  update_body<OPT>(sa, q.y);
}

int update_ctas(const UpdArgs& a) { return a.n_cols + NSC + update_decay_ctas(a) + a.pupil_cols; }

cudaError_t update_prepare() {
  const void* fns[4] = {(const void*)update_kernel<FPM_OPT_ADAM>, (const void*)update_kernel<FPM_OPT_ADAMW>,
                        (const void*)update_kernel<FPM_OPT_NADAM>, (const void*)update_kernel<FPM_OPT_RMSPROP>};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = cudaFuncSetAttribute(update_kernel_jobs<-1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(update_kernel_jobs<FPM_OPT_ADAM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}

cudaError_t launch_update_jobs(const UpdArgs* jobs, const int2* map, int n_ctas, int B_max, cudaStream_t s,
                               bool pdl, int opt) {
  if (n_ctas < 1) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_ctas, 1, 1);
  cfg.blockDim = dim3(UPD_NT, 1, 1);
  cfg.dynamicSmemBytes = sizeof(double) * 3 * (size_t)B_max;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return opt == FPM_OPT_ADAM ? cudaLaunchKernelEx(&cfg, update_kernel_jobs<FPM_OPT_ADAM>, jobs, map)
                             : cudaLaunchKernelEx(&cfg, update_kernel_jobs<-1>, jobs, map);
}

cudaError_t launch_update(const UpdArgs& a, cudaStream_t s, bool pdl) {
  const size_t smem = sizeof(double) * 3 * (size_t)a.B;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)update_ctas(a), 1, 1);
  cfg.blockDim = dim3(UPD_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  switch (a.opt) {
    case FPM_OPT_ADAMW: return cudaLaunchKernelEx(&cfg, update_kernel<FPM_OPT_ADAMW>, a);
    case FPM_OPT_NADAM: return cudaLaunchKernelEx(&cfg, update_kernel<FPM_OPT_NADAM>, a);
    case FPM_OPT_RMSPROP: return cudaLaunchKernelEx(&cfg, update_kernel<FPM_OPT_RMSPROP>, a);
    default: return cudaLaunchKernelEx(&cfg, update_kernel<FPM_OPT_ADAM>, a);
  }
}

}  // namespace fpmk

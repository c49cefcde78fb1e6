// Random-batch update (Section 2.3, Eq. 13) with Adam (Kingma & Ba 2015).
//
// Object: every element of the update region (the union of all LEDs' crop
// boxes; outside it the gradient has always been zero and Adam is an exact
// no-op) gathers the per-LED gradient boxes in batch order - a fixed-order
// sum, so results are bitwise reproducible - and takes one Adam step on its
// real and imaginary parts. One CTA per spectrum column of the region.
// Scalars: the last CTA reduces the per-CTA FP64 partials in a fixed order,
// forms the gradients of the Zernike coefficients, defocus, intensity factors
// and LED offsets, and updates all of them (every element, every step).
#include <cmath>

#include "device.cuh"
#include "internal.h"

namespace fpmk {

constexpr int UPD_NT = 256;

__device__ __forceinline__ void adam1(float& w, float& m, float& v, float g, float lr_bc1, float inv_sqrt_bc2,
                                      float b1, float b2, float eps) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  w -= lr_bc1 * m / fmaf(sqrtf(v), inv_sqrt_bc2, eps);
}

__device__ void scalar_update(const UpdArgs& a, double bc1, double bc2) {
  extern __shared__ double gsh[];  // [sp_size(n_leds)] gradients, then NPART totals
  const int n = a.n_leds, P = sp_size(n);
  double* tot = gsh + P;
  const int tid = threadIdx.x;
  for (int i = tid; i < P; i += blockDim.x) gsh[i] = 0.0;
  __syncthreads();
  // quantities shared by all LEDs: loss, Zernike, defocus (fixed summation order)
  if (tid < NPART && tid != P_GAMMA && tid != P_DY && tid != P_DX) {
    double s = 0.0;
    for (int kk = 0; kk < a.B; ++kk)
      for (int r = 0; r < a.C; ++r) s += a.part[((size_t)kk * a.C + r) * NPART + tid];
    tot[tid] = s;
  }
  // per-LED quantities
  for (int kk = tid; kk < a.B; kk += blockDim.x) {
    const int led = a.idx[kk];
    double g = 0.0, dy = 0.0, dx = 0.0;
    for (int r = 0; r < a.C; ++r) {
      const double* p = a.part + ((size_t)kk * a.C + r) * NPART;
      g += p[P_GAMMA];
      dy += p[P_DY];
      dx += p[P_DX];
    }
    gsh[SP_GAMMA + led] = g;
    gsh[sp_offset(n) + 2 * led] = dy;
    gsh[sp_offset(n) + 2 * led + 1] = dx;
  }
  __syncthreads();
  if (tid < 14) gsh[SP_ZERN + tid] = tot[P_ZERN + tid];
  if (tid == 14) gsh[SP_DEFOCUS] = tot[P_DEFOCUS];
  __syncthreads();
  if (tid == 0) {
    const double L = tot[P_LOSS];
    *a.loss_slot = L;
    if (!a.assemble) *a.epoch_loss += L;
    if (!isfinite(L)) atomicOr(a.err, DERR_NONFINITE);
  }
  if (a.assemble) {
    for (int i = tid; i < P; i += blockDim.x) a.g_sc[i] = (float)gsh[i];
    return;
  }
  const float inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
  for (int i = tid; i < P; i += blockDim.x) {
    float lr;
    unsigned bit;
    if (i < SP_DEFOCUS) { lr = a.lr_zern; bit = 1u << 1; }
    else if (i == SP_DEFOCUS) { lr = a.lr_def; bit = 1u << 2; }
    else if (i < sp_offset(n)) { lr = a.lr_gam; bit = 1u << 3; }
    else { lr = a.lr_off; bit = 1u << 4; }
    if (!(a.learn & bit)) continue;
    float w = a.sp[i], m = a.msp[i], v = a.vsp[i];
    adam1(w, m, v, (float)gsh[i], (float)(lr / bc1), inv_sqrt_bc2, a.b1, a.b2, a.eps);
    if (i >= sp_offset(n)) w = fminf(fmaxf(w, -a.offset_bound), a.offset_bound);
    a.sp[i] = w;
    a.msp[i] = m;
    a.vsp[i] = v;
  }
}

__global__ void __launch_bounds__(UPD_NT) update_kernel(const UpdArgs a) {
  const long long t = *a.t_base + a.step_off + 1;
  const double bc1 = 1.0 - pow((double)a.b1, (double)t);
  const double bc2 = 1.0 - pow((double)a.b2, (double)t);
  if (blockIdx.x == (unsigned)a.n_cols) {
    scalar_update(a, bc1, bc2);
    return;
  }
  if (!a.assemble && !(a.learn & 1u)) return;
  __shared__ int2 corner[MAX_BATCH];  // (first column, first row) of each slot's box
  for (int kk = threadIdx.x; kk < a.B; kk += blockDim.x) {
    const int2 n = a.n_int[a.idx[kk]];
    corner[kk] = make_int2(a.N / 2 + n.y - a.h, a.N / 2 + n.x - a.h);
  }
  __syncthreads();
  const int x = a.x_lo + blockIdx.x;
  const int2 span = a.span[x];
  const float lr_bc1 = (float)(a.lr_obj / bc1);
  const float inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
  const int W = a.W;
  for (int y = span.x + threadIdx.x; y < span.y; y += blockDim.x) {
    float2 g = make_float2(0.f, 0.f);
    for (int kk = 0; kk < a.B; ++kk) {
      const int cx = x - corner[kk].x, ry = y - corner[kk].y;
      if ((unsigned)cx < (unsigned)W && (unsigned)ry < (unsigned)W)
        g = cadd(g, a.gbox[((size_t)kk * W + cx) * W + ry]);
    }
    const size_t o = (size_t)x * a.N + y;
    if (a.assemble) {
      a.g_obj[o] = g;
      continue;
    }
    float2 w = a.Ot[o], m = a.mO[o], v = a.vO[o];
    adam1(w.x, m.x, v.x, g.x, lr_bc1, inv_sqrt_bc2, a.b1, a.b2, a.eps);
    adam1(w.y, m.y, v.y, g.y, lr_bc1, inv_sqrt_bc2, a.b1, a.b2, a.eps);
    a.Ot[o] = w;
    a.mO[o] = m;
    a.vO[o] = v;
  }
}

cudaError_t launch_update(const UpdArgs& a, cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)sp_size(a.n_leds) + NPART);
  update_kernel<<<a.n_cols + 1, UPD_NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fpmk

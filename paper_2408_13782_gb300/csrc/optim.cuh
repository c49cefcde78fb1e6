// Per-element rules of the Adam-family optimisers (the definitions are in
// fpm.h) shared by the update kernel and the dataflow step kernel. The per-step
// coefficients k (bias corrections, NAdam's momentum terms) come from the host
// in FP64 (see UpdArgs::coef).
#pragma once

#include "../../include/fpm.h"
#include "internal.h"

namespace fpmk {

__device__ __forceinline__ void adam1(float& w, float& m, float& v, float g, float lr_bc1, float inv_sqrt_bc2,
                                      float b1, float b2, float eps) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  w -= lr_bc1 * m / fmaf(sqrtf(v), inv_sqrt_bc2, eps);
}

// One step of the handle's optimiser on one real component with learning rate
// lr and this step's coefficients k (see UpdArgs::coef). OPT >= 0 fixes the
// rule at compile time (it must equal a.opt); OPT < 0 branches on a.opt, the
// same for every thread of a launch.
template <int OPT = -1>
__device__ __forceinline__ void opt1(const UpdArgs& a, float& w, float& m, float& v, float g, float lr, float4 k) {
  switch (OPT >= 0 ? OPT : a.opt) {
    case FPM_OPT_ADAMW:
      w *= 1.f - lr * a.wd;
      adam1(w, m, v, g, lr * k.x, k.y, a.b1, a.b2, a.eps);
      break;
    case FPM_OPT_NADAM:
      m = fmaf(a.b1, m, (1.f - a.b1) * g);
      v = fmaf(a.b2, v, (1.f - a.b2) * g * g);
      w -= lr * fmaf(k.x, m, k.z * g) / fmaf(sqrtf(v), k.y, a.eps);
      break;
    case FPM_OPT_RMSPROP:
      v = fmaf(a.b2, v, (1.f - a.b2) * g * g);
      w -= lr * g / (sqrtf(v) + a.eps);
      break;
    default:
      adam1(w, m, v, g, lr * k.x, k.y, a.b1, a.b2, a.eps);
  }
}

__device__ __forceinline__ bool learned(const UpdArgs& a, int i) {
  const unsigned bit = i < SP_DEFOCUS ? 1u << 1 : i == SP_DEFOCUS ? 1u << 2 : i < sp_offset(a.n_leds) ? 1u << 3 : 1u << 4;
  return (a.learn & bit) != 0;
}
__device__ __forceinline__ float lr_of(const UpdArgs& a, int i) {
  return i < SP_DEFOCUS ? a.lr_zern : i == SP_DEFOCUS ? a.lr_def : i < sp_offset(a.n_leds) ? a.lr_gam : a.lr_off;
}

// The optimiser step of scalar i with FP64 gradient g; offsets are clamped to
// the box bound and intensity factors held at or above FPM_GAMMA_FLOOR.
__device__ __forceinline__ void scalar_adam(const UpdArgs& a, int i, float w, float m, float v, double g, float4 k) {
  opt1(a, w, m, v, (float)g, lr_of(a, i), k);
  if (i >= sp_offset(a.n_leds)) w = fminf(fmaxf(w, -a.offset_bound), a.offset_bound);
  else if (i >= SP_GAMMA) w = fmaxf(w, FPM_GAMMA_FLOOR);
  a.sp[i] = w;
  a.msp[i] = m;
  a.vsp[i] = v;
}

// Free-form pupil node (rn, cn) of the update: its gradient is the sum over
// the batch slots (in batch order) and the four bilinear corners of the slot's
// pupil-gradient box at the pixel that sits (ay + dy, ax + dx) below it, with
// weights (1 - fy or fy)(1 - fx or fx); then the optimiser (learned) or the
// gradient (assembling). w, m, v: the node's state, read before the gradient.
__device__ __forceinline__ void pupil_node(const UpdArgs& a, int cn, int rn, float2 w, float2 m, float2 v,
                                           float4 bc) {
  const int W = a.W;
  float2 g = make_float2(0.f, 0.f);
  for (int k = 0; k < a.B; ++k) {
    const float4 pw = __ldcg(a.pwt + k);  // (fy, fx, ay, ax) of the slot, from the LED kernel
    const int ay = (int)pw.z, ax = (int)pw.w;
    const float2* box = a.pbox + (size_t)k * W * W;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int dy = q >> 1, dx = q & 1;
      const int r = rn - ay - dy, c = cn - ax - dx;
      if ((unsigned)r < (unsigned)W && (unsigned)c < (unsigned)W) {
        const float wt = (dy ? pw.x : 1.f - pw.x) * (dx ? pw.y : 1.f - pw.y);
        const float2 G = __ldcg(box + (size_t)c * W + r);
        g.x = fmaf(wt, G.x, g.x);
        g.y = fmaf(wt, G.y, g.y);
      }
    }
  }
  const size_t o = (size_t)cn * W + rn;
  if (a.assemble) {
    a.g_pupil[o] = g;
    return;
  }
  if (!(a.learn & (1u << 5))) return;
  opt1(a, w.x, m.x, v.x, g.x, a.lr_pupil, bc);
  opt1(a, w.y, m.y, v.y, g.y, a.lr_pupil, bc);
  a.Pff[o] = w;
  a.mPff[o] = m;
  a.vPff[o] = v;
}

}  // namespace fpmk

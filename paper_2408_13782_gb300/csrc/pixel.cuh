// Per-pixel pieces of the per-LED step shared by the FFT and the GEMM kernels:
// the loss residual (Section 2.2, Eq. 4-5) and the box gradients of the object
// and of the pupil parameters (adjoint of Section 2.1, Eq. 3).
#pragma once

#include "device.cuh"
#include "internal.h"

namespace fpmk {

// Residual at one pixel for a predicted field psi (already 1/m^2 scaled).
// v is the measured intensity (loss modes) or the upstream dL/dI. Returns
// the field gradient dL/dpsi and accumulates the loss and dL/dgamma terms.
__device__ __forceinline__ float2 residual_pixel(float2 psi, float v, int mode, int loss, float gam, float sg,
                                                 float& acc_loss, float& acc_g) {
  const float mag2 = psi.x * psi.x + psi.y * psi.y;
  if (mode == MODE_LOSS) {
    if (loss == 0) {
      const float rinv = mag2 > 0.f ? rsqrtf(mag2) : 0.f;
      const float mag = mag2 * rinv;
      const float res = sg * mag - sqrtf(fmaxf(v, 0.f));
      acc_loss = fmaf(res, res, acc_loss);
      acc_g = fmaf(res, mag, acc_g);
      return cscale(psi, 2.f * res * sg * rinv);  // 0 where psi = 0
    }
    const float res = gam * mag2 - v;
    acc_loss = fmaf(res, res, acc_loss);
    acc_g = fmaf(2.f * res, mag2, acc_g);
    return cscale(psi, 4.f * gam * res);
  }
  acc_g = fmaf(v, mag2, acc_g);
  return cscale(psi, 2.f * gam * v);
}

// Amplitude-loss residual with the measured amplitude amp = sqrt(max(I, 0))
// given (the same arithmetic as residual_pixel's amplitude branch).
__device__ __forceinline__ float2 residual_amp_pixel(float2 psi, float amp, float sg, float& acc_loss, float& acc_g) {
  const float mag2 = psi.x * psi.x + psi.y * psi.y;
  const float rinv = mag2 > 0.f ? rsqrtf(mag2) : 0.f;
  const float mag = mag2 * rinv;
  const float res = sg * mag - amp;
  acc_loss = fmaf(res, res, acc_loss);
  acc_g = fmaf(res, mag, acc_g);
  return cscale(psi, 2.f * res * sg * rinv);  // 0 where psi = 0
}

struct BoxAcc {
  float m[15];  // monomial moments sum t(p) x^a y^b
  float def, dy, dx;
};

__device__ __forceinline__ void box_acc_zero(BoxAcc& b) {
#pragma unroll
  for (int q = 0; q < 15; ++q) b.m[q] = 0.f;
  b.def = b.dy = b.dx = 0.f;
}

// ---- column form (fixed qx, pixels along y; ColPoly in device.cuh) --------
// Pupil amplitude from r2 = |q|^2; rad = |q| is also returned (anti-aliased
// edge only: the hard edge needs no square root).
__device__ __forceinline__ float pupil_amp_r2(float r2, const PupilConst& P, float& rad) {
  if (P.hard_edge) {
    rad = 0.f;
    return r2 <= P.R * P.R ? 1.f : 0.f;
  }
  rad = sqrtf(r2);
  return fminf(fmaxf(P.R + 0.5f - rad, 0.f), 1.f);
}

// Pupil value M = A exp(i chi) of a pixel of the column (A > 0 given).
__device__ __forceinline__ float2 pupil_col(float qy, float r2, float A, const PupilConst& P, const ColPoly& cp,
                                            float zdef) {
  const float th = col_theta(cp, qy * P.Rinv);
  float root;
  const float kap = defocus_kappa(r2, P, &root);
  float sn, cs;
  sincos_phase(fmaf(zdef, kap, th), &sn, &cs);
  return make_float2(A * cs, A * sn);
}

// ---- free-form pupil factor ------------------------------------------------
// The node field P (box grid, column-major by box column, W x W) evaluated at
// q = p - delta by bilinear interpolation. For one LED q - floor(q) is the
// same at every pixel: f = -delta - floor(-delta), and the lower-left node of
// box pixel (row r, column c) is (r + ay, c + ax) with a = floor(-delta).
struct FreeForm {
  const float2* P;  // nullptr: no free-form factor
  int W, ay, ax;
  float fy, fx;
};

__device__ __forceinline__ FreeForm free_form(const float2* P, int W, float dly, float dlx) {
  FreeForm f;
  f.P = P;
  f.W = W;
  const float by = floorf(-dly), bx = floorf(-dlx);
  f.ay = (int)by;
  f.ax = (int)bx;
  f.fy = -dly - by;
  f.fx = -dlx - bx;
  return f;
}

// P~ at box pixel (r, c) of a support pixel, and (with d) its derivatives
// along qy and qx. The node indices are clamped to the field (a support pixel
// never needs the clamp).
__device__ __forceinline__ float2 ff_value(const FreeForm& f, int r, int c, float2* dqy = nullptr,
                                           float2* dqx = nullptr) {
  const int rn = min(max(r + f.ay, 0), f.W - 2), cn = min(max(c + f.ax, 0), f.W - 2);
  const float2* p = f.P + (size_t)cn * f.W + rn;
  const float2 p00 = __ldg(p), p10 = __ldg(p + 1), p01 = __ldg(p + f.W), p11 = __ldg(p + f.W + 1);
  const float gy = 1.f - f.fy, gx = 1.f - f.fx;
  const float2 a0 = make_float2(fmaf(gx, p00.x, f.fx * p01.x), fmaf(gx, p00.y, f.fx * p01.y));  // row rn
  const float2 a1 = make_float2(fmaf(gx, p10.x, f.fx * p11.x), fmaf(gx, p10.y, f.fx * p11.y));  // row rn + 1
  if (dqy) *dqy = csub(a1, a0);
  if (dqx) {
    const float2 b0 = csub(p01, p00), b1 = csub(p11, p10);
    *dqx = make_float2(fmaf(gy, b0.x, f.fy * b1.x), fmaf(gy, b0.y, f.fy * b1.y));
  }
  return make_float2(fmaf(gy, a0.x, f.fy * a1.x), fmaf(gy, a0.y, f.fy * a1.y));
}

// One pixel of an LED's support box at q = (qy, qx) = p - delta (A > 0, r2 =
// |q|^2, rad = |q| for the anti-aliased edge) with the spectrum gradient gphi
// and the object value o there: returns the object gradient conj(M) gphi and
// accumulates the pupil-parameter gradient terms. The aberration phase comes
// from the column's polynomials (ColPoly); the monomial moments sum t x^a y^b
// are kept as the column sums S[b] = sum t y^b and folded into acc.m by
// col_fold once per column.
//
// With a free-form factor (ff.P != nullptr; r, c: the pixel's box row and
// column) the pupil is M = A e^{i chi} P~(q): the object gradient and the
// chi and A terms use it, *G receives dL/dP~ = conj(A e^{i chi}) conj(O) gPhi
// (the pixel's entry of the pupil-gradient box), and the offsets gain
// -Re(conj(G) dP~/dq).
__device__ __forceinline__ float2 box_pixel_col(float qy, float qx, float r2, float A, float rad, float2 gphi, float2 o,
                                                const PupilConst& P, const ColPoly& cp, float zdef, float (&S)[5],
                                                BoxAcc& acc, const FreeForm& ff = FreeForm{nullptr, 0, 0, 0, 0.f, 0.f},
                                                int r = 0, int c = 0, float2* G = nullptr) {
  const float y = qy * P.Rinv;
  const float th = col_theta(cp, y);
  float dthx, dthy;
  col_grad(cp, y, dthx, dthy);
  float root;
  const float kap = defocus_kappa(r2, P, &root);
  float sn, cs;
  sincos_phase(fmaf(zdef, kap, th), &sn, &cs);
  float2 e = make_float2(cs, sn);
  float2 Mv = cscale(e, A);
  const float2 gM = cmulc(o, gphi);     // conj(O) gPhi
  float2 dPy = make_float2(0.f, 0.f), dPx = dPy;
  if (ff.P) {
    const float2 M0 = Mv;
    const float2 Pt = ff_value(ff, r, c, &dPy, &dPx);
    Mv = cmul(M0, Pt);
    e = cmul(e, Pt);
    *G = cmulc(M0, gM);
  }
  const float tt = -cmulc(gM, Mv).y;    // dL/dchi = Re(conj(gM) i M)
  const float ee = cmulc(gM, e).x;      // dL/dA   = Re(conj(gM) e^{i chi} P~)
  const float y2 = y * y;
  S[0] += tt;
  S[1] = fmaf(tt, y, S[1]);
  S[2] = fmaf(tt, y2, S[2]);
  S[3] = fmaf(tt, y2 * y, S[3]);
  S[4] = fmaf(tt, y2 * y2, S[4]);
  acc.def = fmaf(tt, kap, acc.def);
  const float dk = fdiv_fast(-6.283185307179586f * P.dk2, root);  // d kappa / d q = dk * q
  const float dchiy = fmaf(dthy, P.Rinv, zdef * dk * qy);
  const float dchix = fmaf(dthx, P.Rinv, zdef * dk * qx);
  float dAy = 0.f, dAx = 0.f;
  if (!P.hard_edge && rad > P.R - 0.5f && rad < P.R + 0.5f) {
    dAy = -qy / rad;
    dAx = -qx / rad;
  }
  acc.dy -= fmaf(tt, dchiy, ee * dAy);
  acc.dx -= fmaf(tt, dchix, ee * dAx);
  if (ff.P) {                           // P~ moves with q = p - delta
    acc.dy -= cmulc(*G, dPy).x;
    acc.dx -= cmulc(*G, dPx).x;
  }
  return cmulc(Mv, gphi);               // conj(M) gPhi
}

// acc.m[x^a y^b] += x^a S[b] for the column's x.
__device__ __forceinline__ void col_fold(const ColPoly& cp, const float (&S)[5], BoxAcc& acc) {
  const float x = cp.x, x2 = x * x;
  const float xp[5] = {1.f, x, x2, x2 * x, x2 * x2};
#pragma unroll
  for (int b = 0; b <= 4; ++b)
#pragma unroll
    for (int a = 0; a + b <= 4; ++a) acc.m[mono_idx(a, b)] = fmaf(xp[a], S[b], acc.m[mono_idx(a, b)]);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-thread accumulators: loss, gamma, 15 monomial moments, defocus, dy, dx.
constexpr int NACC = 20;
enum : int { A_LOSS = 0, A_GAMMA = 1, A_MONO = 2, A_DEF = 17, A_DY = 18, A_DX = 19 };

// Reduce the block's accumulators and write its partials (NPART values, stored
// as FP64 for the update kernel's FP64 sums over all CTAs of the batch). The
// block's own sums (a few thousand pixels) stay in FP32: FP64 arithmetic is
// slow on this part. The monomial moments become Zernike gradients through
// the table zmt (row j-2 = Z_j). red: [nwarps][NACC], fsum: [16] floats of
// shared memory. Called by every thread.
__device__ __forceinline__ void write_partials(float acc_loss, float acc_g, const BoxAcc& b, bool amp_loss_gamma,
                                               float sg, float* red, float* fsum, const float* zmt, double* out) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  float vals[NACC];
  vals[A_LOSS] = acc_loss;
  vals[A_GAMMA] = acc_g;
#pragma unroll
  for (int q = 0; q < 15; ++q) vals[A_MONO + q] = b.m[q];
  vals[A_DEF] = b.def;
  vals[A_DY] = b.dy;
  vals[A_DX] = b.dx;
  // Warp sums of all NACC values at once by recursive halving: at the step of
  // distance o every lane keeps the half of its vector selected by bit o of
  // its lane index and adds the partner's copy of that half; after five steps
  // lane q holds the warp's total of value q (31 shuffles instead of 5 NACC).
  float v[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = q < NACC ? vals[q] : 0.f;
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
  if (lane < NACC) red[warp * NACC + lane] = v[0];
  __syncthreads();
  float tot = 0.f;
  if (tid < NACC)
    for (int w = 0; w < nw; ++w) tot += red[w * NACC + tid];
  if (tid >= A_MONO && tid < A_MONO + 15) fsum[tid - A_MONO] = tot;
  __syncthreads();
  if (tid == A_LOSS) out[P_LOSS] = tot;
  if (tid == A_GAMMA) out[P_GAMMA] = amp_loss_gamma ? (double)(tot / sg) : (double)tot;
  if (tid == A_DEF) out[P_DEFOCUS] = tot;
  if (tid == A_DY) out[P_DY] = tot;
  if (tid == A_DX) out[P_DX] = tot;
  if (tid < 14) {  // dL/dc_j = sum_m (Z_j)_m * (sum_p t(p) mo_m(p))
    float z = 0.f;
#pragma unroll
    for (int m = 0; m < 15; ++m) z = fmaf(zmt[tid * 15 + m], fsum[m], z);
    out[P_ZERN + tid] = z;
  }
}

}  // namespace fpmk

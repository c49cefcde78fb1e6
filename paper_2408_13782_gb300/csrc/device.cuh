// Device helpers for the Batch-FPM engine (sm_103a): complex arithmetic, the
// pupil model of Section 2.1 Eq. (3), and a shared-memory Stockham FFT run by
// a group of M/8 threads, each holding 8 points per pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define FPM_HD __host__ __device__ __forceinline__
#else
#define FPM_HD inline
#endif

namespace fpmk {

FPM_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
FPM_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
FPM_HD float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
FPM_HD float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
FPM_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Zernike polynomials j = 2..15 in Noll's ordering and normalisation, written
// out in Cartesian form on the unit disk (x = rho cos t, y = rho sin t), with
// their partial derivatives. Index 0 of the arrays is j = 2.
// ---------------------------------------------------------------------------
struct Zern {
  float v[14], dx[14], dy[14];
};

FPM_HD void zernike_eval(float x, float y, Zern& z) {
  const float s3 = 1.7320508075688772f, s5 = 2.2360679774997896f, s6 = 2.449489742783178f;
  const float s8 = 2.8284271247461903f, s10 = 3.1622776601683795f;
  const float x2 = x * x, y2 = y * y, r2 = x2 + y2, xy = x * y;
  // j=2,3: tilt
  z.v[0] = 2.f * x;            z.dx[0] = 2.f;               z.dy[0] = 0.f;
  z.v[1] = 2.f * y;            z.dx[1] = 0.f;               z.dy[1] = 2.f;
  // j=4: defocus
  z.v[2] = s3 * (2.f * r2 - 1.f); z.dx[2] = 4.f * s3 * x;  z.dy[2] = 4.f * s3 * y;
  // j=5,6: astigmatism
  z.v[3] = 2.f * s6 * xy;      z.dx[3] = 2.f * s6 * y;      z.dy[3] = 2.f * s6 * x;
  z.v[4] = s6 * (x2 - y2);     z.dx[4] = 2.f * s6 * x;      z.dy[4] = -2.f * s6 * y;
  // j=7,8: coma
  z.v[5] = s8 * (3.f * r2 - 2.f) * y;  z.dx[5] = s8 * 6.f * xy;  z.dy[5] = s8 * (3.f * x2 + 9.f * y2 - 2.f);
  z.v[6] = s8 * (3.f * r2 - 2.f) * x;  z.dx[6] = s8 * (9.f * x2 + 3.f * y2 - 2.f);  z.dy[6] = s8 * 6.f * xy;
  // j=9,10: trefoil
  z.v[7] = s8 * (3.f * x2 * y - y2 * y);  z.dx[7] = s8 * 6.f * xy;  z.dy[7] = s8 * 3.f * (x2 - y2);
  z.v[8] = s8 * (x2 * x - 3.f * x * y2);  z.dx[8] = s8 * 3.f * (x2 - y2);  z.dy[8] = -s8 * 6.f * xy;
  // j=11: spherical
  z.v[9] = s5 * (6.f * r2 * r2 - 6.f * r2 + 1.f);
  z.dx[9] = s5 * 12.f * x * (2.f * r2 - 1.f);
  z.dy[9] = s5 * 12.f * y * (2.f * r2 - 1.f);
  // j=12,13: secondary astigmatism, (4 r^2 - 3) * {x^2 - y^2, 2xy}
  const float a = 4.f * r2 - 3.f, u = x2 - y2, w = 2.f * xy;
  z.v[10] = s10 * a * u;  z.dx[10] = s10 * (8.f * x * u + 2.f * a * x);  z.dy[10] = s10 * (8.f * y * u - 2.f * a * y);
  z.v[11] = s10 * a * w;  z.dx[11] = s10 * (8.f * x * w + 2.f * a * y);  z.dy[11] = s10 * (8.f * y * w + 2.f * a * x);
  // j=14,15: tetrafoil, Re/Im (x + i y)^4
  z.v[12] = s10 * (x2 * x2 - 6.f * x2 * y2 + y2 * y2);
  z.dx[12] = s10 * (4.f * x2 * x - 12.f * x * y2);
  z.dy[12] = s10 * (4.f * y2 * y - 12.f * x2 * y);
  z.v[13] = s10 * (4.f * x2 * xy - 4.f * xy * y2);
  z.dx[13] = s10 * (12.f * x2 * y - 4.f * y2 * y);
  z.dy[13] = s10 * (4.f * x2 * x - 12.f * x * y2);
}

// The same polynomials as combinations of the 15 monomials x^a y^b with
// a + b <= 4, ordered by degree d = a + b and then by b: monomial index
// d(d+1)/2 + b, i.e. 1, x, y, x2, xy, y2, x3, x2y, xy2, y3, x4, x3y, x2y2,
// xy3, y4. Row j-2 holds the coefficients of Z_j.
#define FPM_S3 1.7320508075688772f
#define FPM_S5 2.2360679774997896f
#define FPM_S6 2.449489742783178f
#define FPM_S8 2.8284271247461903f
#define FPM_S10 3.1622776601683795f
#define FPM_ZERN_MONO_TABLE                                                                          \
  {                                                                                                  \
    /* Z2  */ {0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},                                         \
    /* Z3  */ {0, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},                                         \
    /* Z4  */ {-FPM_S3, 0, 0, 2 * FPM_S3, 0, 2 * FPM_S3, 0, 0, 0, 0, 0, 0, 0, 0, 0},                 \
    /* Z5  */ {0, 0, 0, 0, 2 * FPM_S6, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},                                \
    /* Z6  */ {0, 0, 0, FPM_S6, 0, -FPM_S6, 0, 0, 0, 0, 0, 0, 0, 0, 0},                             \
    /* Z7  */ {0, 0, -2 * FPM_S8, 0, 0, 0, 0, 3 * FPM_S8, 0, 3 * FPM_S8, 0, 0, 0, 0, 0},             \
    /* Z8  */ {0, -2 * FPM_S8, 0, 0, 0, 0, 3 * FPM_S8, 0, 3 * FPM_S8, 0, 0, 0, 0, 0, 0},             \
    /* Z9  */ {0, 0, 0, 0, 0, 0, 0, 3 * FPM_S8, 0, -FPM_S8, 0, 0, 0, 0, 0},                          \
    /* Z10 */ {0, 0, 0, 0, 0, 0, FPM_S8, 0, -3 * FPM_S8, 0, 0, 0, 0, 0, 0},                          \
    /* Z11 */ {FPM_S5, 0, 0, -6 * FPM_S5, 0, -6 * FPM_S5, 0, 0, 0, 0, 6 * FPM_S5, 0, 12 * FPM_S5, 0, 6 * FPM_S5}, \
    /* Z12 */ {0, 0, 0, -3 * FPM_S10, 0, 3 * FPM_S10, 0, 0, 0, 0, 4 * FPM_S10, 0, 0, 0, -4 * FPM_S10},  \
    /* Z13 */ {0, 0, 0, 0, -6 * FPM_S10, 0, 0, 0, 0, 0, 0, 8 * FPM_S10, 0, 8 * FPM_S10, 0},         \
    /* Z14 */ {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, FPM_S10, 0, -6 * FPM_S10, 0, FPM_S10},                  \
    /* Z15 */ {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 4 * FPM_S10, 0, -4 * FPM_S10, 0},                    \
  }
#if defined(__CUDACC__)
// global (not __constant__) memory: kernels read it with divergent indices,
// which the constant cache would serialise
static __device__ const float kZernMonoDev[14][15] = FPM_ZERN_MONO_TABLE;
#endif
static const float kZernMonoHost[14][15] = FPM_ZERN_MONO_TABLE;

// Coefficient of monomial m in Z_{j+2}.
FPM_HD float zern_mono(int j, int m) {
#if defined(__CUDA_ARCH__)
  return kZernMonoDev[j][m];
#else
  return kZernMonoHost[j][m];
#endif
}

FPM_HD void monomials(float x, float y, float (&mo)[15]) {
  const float x2 = x * x, y2 = y * y, xy = x * y;
  mo[0] = 1.f; mo[1] = x; mo[2] = y;
  mo[3] = x2; mo[4] = xy; mo[5] = y2;
  mo[6] = x2 * x; mo[7] = x2 * y; mo[8] = x * y2; mo[9] = y2 * y;
  mo[10] = x2 * x2; mo[11] = x2 * xy; mo[12] = x2 * y2; mo[13] = xy * y2; mo[14] = y2 * y2;
}

// Entry e of the 35 polynomial coefficients (K[15], Dx[10], Dy[10] below)
// computed on its own, so 35 threads can fill them in parallel:
// K[m] = sum_j c_j (Z_j)_m; Dx for monomial x^a y^b (a + b <= 3) is
// (a+1) K[x^(a+1) y^b], Dy is (b+1) K[x^a y^(b+1)].
// zm: the 14 x 15 table (row j-2 = Z_j), e.g. staged in shared memory.
FPM_HD float theta_poly_entry_tab(const float* c, const float* zm, int e) {
  int m = e, f = 1;
  if (e >= 15) {
    const int mm = e < 25 ? e - 15 : e - 25;
    const int d = mm == 0 ? 0 : (mm < 3 ? 1 : (mm < 6 ? 2 : 3));
    const int b = mm - d * (d + 1) / 2, a = d - b;
    if (e < 25) { m = (d + 1) * (d + 2) / 2 + b; f = a + 1; }
    else { m = (d + 1) * (d + 2) / 2 + b + 1; f = b + 1; }
  }
  float s = 0.f;
  for (int j = 0; j < 14; ++j) s = fmaf(c[j], zm[j * 15 + m], s);
  return (float)f * s;
}

#if defined(__CUDACC__)
__device__ __forceinline__ const float* zern_mono_table() { return &kZernMonoDev[0][0]; }
#endif

FPM_HD float theta_poly_entry(const float* c, int e) {
  int m = e, f = 1;
  if (e >= 15) {
    const int mm = e < 25 ? e - 15 : e - 25;
    const int d = mm == 0 ? 0 : (mm < 3 ? 1 : (mm < 6 ? 2 : 3));
    const int b = mm - d * (d + 1) / 2, a = d - b;
    if (e < 25) { m = (d + 1) * (d + 2) / 2 + b; f = a + 1; }
    else { m = (d + 1) * (d + 2) / 2 + b + 1; f = b + 1; }
  }
  float s = 0.f;
  for (int j = 0; j < 14; ++j) s = fmaf(c[j], zern_mono(j, m), s);
  return (float)f * s;
}

// For aberration coefficients c[14] (Noll 2..15): theta = sum_m K[m] mo[m],
// d theta/dx = sum_{m<10} Dx[m] mo[m], d theta/dy = sum_{m<10} Dy[m] mo[m].
FPM_HD void theta_poly(const float* c, float (&K)[15], float (&Dx)[10], float (&Dy)[10]) {
  for (int m = 0; m < 15; ++m) {
    float s = 0.f;
    for (int j = 0; j < 14; ++j) s = fmaf(c[j], zern_mono(j, m), s);
    K[m] = s;
  }
  for (int m = 0; m < 10; ++m) Dx[m] = Dy[m] = 0.f;
  for (int d = 1; d <= 4; ++d)
    for (int b = 0; b <= d; ++b) {
      const int a = d - b, m = d * (d + 1) / 2 + b;
      if (a > 0) Dx[(d - 1) * d / 2 + b] += (float)a * K[m];        // x^(a-1) y^b
      if (b > 0) Dy[(d - 1) * d / 2 + (b - 1)] += (float)b * K[m];  // x^a y^(b-1)
    }
}

// ---- column form of the aberration phase (fixed qx, pixels along y) -----
// Monomial x^a y^b of the aberration polynomials sits at (a+b)(a+b+1)/2 + b.
FPM_HD constexpr int mono_idx(int a, int b) { return (a + b) * (a + b + 1) / 2 + b; }

// On one box column x = qx / R is fixed, so theta(x, y) = sum_b th[b] y^b and
// its x / y derivatives are cubic polynomials in y with coefficients that
// depend on x only: a pixel then costs three Horner steps in y instead of
// evaluating 15 monomials and 35 products.
struct ColPoly {
  float x;
  float th[5], gx[4], gy[4];
};

// poly: K[15], Dx[10], Dy[10] (theta and its gradient as monomials of q / R).
FPM_HD void col_poly(float x, const float* poly, ColPoly& cp) {
  cp.x = x;
#pragma unroll
  for (int b = 0; b <= 4; ++b) {
    float s = poly[mono_idx(4 - b, b)];
#pragma unroll
    for (int a = 3 - b; a >= 0; --a) s = fmaf(s, x, poly[mono_idx(a, b)]);
    cp.th[b] = s;
  }
#pragma unroll
  for (int b = 0; b <= 3; ++b) {
    float sx = poly[15 + mono_idx(3 - b, b)], sy = poly[25 + mono_idx(3 - b, b)];
#pragma unroll
    for (int a = 2 - b; a >= 0; --a) {
      sx = fmaf(sx, x, poly[15 + mono_idx(a, b)]);
      sy = fmaf(sy, x, poly[25 + mono_idx(a, b)]);
    }
    cp.gx[b] = sx;
    cp.gy[b] = sy;
  }
}

FPM_HD float col_theta(const ColPoly& cp, float y) {
  return fmaf(fmaf(fmaf(fmaf(cp.th[4], y, cp.th[3]), y, cp.th[2]), y, cp.th[1]), y, cp.th[0]);
}

// d theta / dx and d theta / dy on the column (in units of q / R).
FPM_HD void col_grad(const ColPoly& cp, float y, float& gx, float& gy) {
  gx = fmaf(fmaf(fmaf(cp.gx[3], y, cp.gx[2]), y, cp.gx[1]), y, cp.gx[0]);
  gy = fmaf(fmaf(fmaf(cp.gy[3], y, cp.gy[2]), y, cp.gy[1]), y, cp.gy[0]);
}

// Per-launch pupil constants.
struct PupilConst {
  float R, Rinv, inv_lambda, dk2;
  int hard_edge;
};

// Pupil value at q = p - delta (spectral px): M = A exp(i chi),
// chi = sum_j c_j Z_j(q/R) + z kappa(q),
// kappa = 2 pi (sqrt(lambda^-2 - |q|^2 dk^2) - 1/lambda), evaluated in the
// cancellation-free form -2 pi k^2 / (sqrt(lambda^-2 - k^2) + 1/lambda).
FPM_HD float pupil_amp(float qy, float qx, const PupilConst& P) {
  const float r2 = qx * qx + qy * qy;
  if (P.hard_edge) return r2 <= P.R * P.R ? 1.f : 0.f;
  const float r = sqrtf(r2);
  return fminf(fmaxf(P.R + 0.5f - r, 0.f), 1.f);
}

// a / b by the hardware reciprocal on the device (at most 2 ulp for the
// divisors used here, which are of order 1 / lambda); plain division on the host.
FPM_HD float fdiv_fast(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}

// sin and cos of a pupil phase (at most tens of radians). On the device the
// argument is first reduced to [-pi, pi] by the Cody-Waite two-constant scheme
// (2 pi = C1 + C2 with C1 the float nearest 2 pi and C2 the remainder), so the
// hardware sine and cosine can be used: their absolute error is documented as
// 2^-21.41 on that interval. The host calls sincosf.
FPM_HD void sincos_phase(float x, float* s, float* c) {
#ifdef __CUDA_ARCH__
  const float n = rintf(x * 0.15915494309189535f);  // x / (2 pi), rounded
  float r = fmaf(-n, 6.28318548202514648f, x);
  r = fmaf(-n, -1.7484556000744883e-07f, r);
  __sincosf(r, s, c);
#else
  sincosf(x, s, c);
#endif
}

FPM_HD float defocus_kappa(float r2, const PupilConst& P, float* root_out) {
  const float k2 = r2 * P.dk2;
  const float root = sqrtf(P.inv_lambda * P.inv_lambda - k2);
  *root_out = root;
  return fdiv_fast(-6.283185307179586f * k2, root + P.inv_lambda);
}

FPM_HD float2 pupil_value(float qy, float qx, const PupilConst& P,
                                              const float* __restrict__ zc, float z) {
  const float A = pupil_amp(qy, qx, P);
  if (A == 0.f) return make_float2(0.f, 0.f);
  Zern Z;
  zernike_eval(qx * P.Rinv, qy * P.Rinv, Z);
  float th = 0.f;
#pragma unroll
  for (int j = 0; j < 14; ++j) th = fmaf(zc[j], Z.v[j], th);
  float root;
  const float kap = defocus_kappa(qx * qx + qy * qy, P, &root);
  float sn, cs;
  sincos_phase(fmaf(z, kap, th), &sn, &cs);
  return make_float2(A * cs, A * sn);
}

// ---------------------------------------------------------------------------
// FFT: Stockham autosort over a (padded) shared-memory buffer of M points,
// run by a group of G = M/8 consecutive threads of one warp (so M <= 256).
// Each pass reads 8 (radix 8), 2x4 (radix-4 tail) or 4x2 (radix-2 tail)
// points per thread into registers, applies twiddles W_{R Ns}^{r k} (k =
// butterfly mod Ns), a radix-R DFT, and writes them to (b - k) R + k + r Ns.
// All threads of the warp call it together; the warp synchronises between the
// read and write halves of each pass. Twiddle table tw[t] = exp(-2 pi i t/M).
// DIR = -1: forward (exp(-)), +1: inverse (exp(+)); both unnormalised. The
// load/store halves are host-callable so the index arithmetic can be emulated
// on a CPU.
// ---------------------------------------------------------------------------
template <int DIR>
FPM_HD float2 tw_dir(float2 w) { return DIR < 0 ? w : make_float2(w.x, -w.y); }

// multiply by DIR * i = exp(DIR * i pi / 2)
template <int DIR>
FPM_HD float2 mul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int DIR>
FPM_HD void dft2(float2& a0, float2& a1) {
  const float2 t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <int DIR>
FPM_HD void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  const float2 t2 = cadd(a1, a3), t3 = mul_i<DIR>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int DIR>
FPM_HD void dft8(float2 (&v)[8]) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  const float h = 0.70710678118654752f;
  const float d = (float)DIR;
  // o_k * W8^k with W8 = exp(DIR * i pi / 4)
  const float2 w1 = make_float2((o1.x - d * o1.y) * h, (o1.y + d * o1.x) * h);
  const float2 w2 = mul_i<DIR>(o2);
  const float2 w3 = make_float2((-o3.x - d * o3.y) * h, (-o3.y + d * o3.x) * h);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1); v[5] = csub(e1, w1);
  v[2] = cadd(e2, w2); v[6] = csub(e2, w2);
  v[3] = cadd(e3, w3); v[7] = csub(e3, w3);
}

template <int M>
struct FftShape {
  static_assert(M >= 16 && M <= 256 && (M & (M - 1)) == 0, "group FFT size");
  static constexpr int G = M / 8;                 // threads per transform
  static constexpr int LOG = (M == 16) ? 4 : (M == 32) ? 5 : (M == 64) ? 6 : (M == 128) ? 7 : 8;
  static constexpr int N8 = LOG / 3;              // radix-8 passes
  static constexpr int TAIL = LOG % 3;            // 0: none, 1: radix 2, 2: radix 4
};

// Buffers are padded with one point after every 8 (index i stored at
// i + i/8): with the Stockham read/write strides below every pass is free of
// shared-memory bank conflicts (to within one doubled bank in the contiguous
// reads).
FPM_HD int pidx(int i) { return i + (i >> 3); }
// 256-point transforms use two radix-16 passes (16 threads x 16 points); for
// their access pattern one pad point every 16 makes every pass conflict-free.
FPM_HD int pidx16(int i) { return i + (i >> 4); }
template <int M>
FPM_HD int bidx(int i) { return M >= 256 ? pidx16(i) : pidx(i); }
template <int M>
struct FftBuf {
  static constexpr int SIZE = M >= 256 ? M + M / 16 : M + M / 8;   // padded length of one buffer
  static constexpr int G = M == 256 ? 16 : (M == 512 ? 32 : M / 8);  // threads per transform
};

// Per-thread twiddles: thread j of a group only ever needs W_{R Ns}^{r k}
// with k = (butterfly index) mod Ns fixed by j, so they are loaded once.
template <int M>
struct FftTw {
  using S = FftShape<M>;
  static constexpr int N8T = (S::N8 > 1 ? (S::N8 - 1) * 7 : 0);
  static constexpr int TT = S::TAIL == 2 ? 6 : (S::TAIL == 1 ? 4 : 0);
  float2 w[(N8T + TT) > 0 ? (N8T + TT) : 1];
};

// Fill the twiddles of thread j from the table tw[t] = exp(-2 pi i t / M).
template <int M>
FPM_HD void fft_twiddles(const float2* tw, int j, FftTw<M>& T) {
  using S = FftShape<M>;
  constexpr int G = M / 8;
  int q = 0, Ns = 8;
  for (int pass = 1; pass < S::N8; ++pass, Ns *= 8) {
    const int k = j & (Ns - 1), step = M / (8 * Ns);
    for (int r = 1; r < 8; ++r) T.w[q++] = tw[r * k * step];
  }
  if (S::TAIL == 2) {
    for (int b = 0; b < 2; ++b) {
      const int jj = j + b * G, k = jj & (Ns - 1), step = M / (4 * Ns);
      for (int r = 1; r < 4; ++r) T.w[q++] = tw[r * k * step];
    }
  } else if (S::TAIL == 1) {
    for (int b = 0; b < 4; ++b) {
      const int jj = j + b * G, k = jj & (Ns - 1), step = M / (2 * Ns);
      T.w[q++] = tw[k * step];
    }
  }
}

// One radix-8 pass, read half: 8 points of butterfly j, twiddled, transformed.
// tw points at this pass's 7 twiddles (unused when Ns == 1).
template <int M, int DIR>
FPM_HD void r8_load(const float2* buf, const float2* tw, int j, int Ns, float2 (&v)[8]) {
  constexpr int G = M / 8;
  for (int r = 0; r < 8; ++r) v[r] = buf[pidx(j + r * G)];
  if (Ns > 1)
    for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], tw_dir<DIR>(tw[r - 1]));
  dft8<DIR>(v);
}
template <int M>
FPM_HD void r8_store(float2* buf, int j, int Ns, const float2 (&v)[8]) {
  const int k = j & (Ns - 1);
  const int base = (j - k) * 8 + k;
  for (int r = 0; r < 8; ++r) buf[pidx(base + r * Ns)] = v[r];
}
// radix-4 tail: butterflies j and j + G; tw points at 2 x 3 twiddles
template <int M, int DIR>
FPM_HD void r4_load(const float2* buf, const float2* tw, int j, int Ns, float2 (&v)[8]) {
  constexpr int G = M / 8;
  for (int b = 0; b < 2; ++b) {
    const int jj = j + b * G;
    float2* w = v + 4 * b;
    for (int r = 0; r < 4; ++r) w[r] = buf[pidx(jj + r * (M / 4))];
    for (int r = 1; r < 4; ++r) w[r] = cmul(w[r], tw_dir<DIR>(tw[3 * b + r - 1]));
    dft4<DIR>(w[0], w[1], w[2], w[3]);
  }
}
template <int M>
FPM_HD void r4_store(float2* buf, int j, int Ns, const float2 (&v)[8]) {
  constexpr int G = M / 8;
  for (int b = 0; b < 2; ++b) {
    const int jj = j + b * G;
    const int k = jj & (Ns - 1);
    const int base = (jj - k) * 4 + k;
    for (int r = 0; r < 4; ++r) buf[pidx(base + r * Ns)] = v[4 * b + r];
  }
}
// radix-2 tail: butterflies j + b G, b = 0..3; tw points at 4 twiddles
template <int M, int DIR>
FPM_HD void r2_load(const float2* buf, const float2* tw, int j, int Ns, float2 (&v)[8]) {
  constexpr int G = M / 8;
  for (int b = 0; b < 4; ++b) {
    const int jj = j + b * G;
    v[2 * b] = buf[pidx(jj)];
    v[2 * b + 1] = cmul(buf[pidx(jj + M / 2)], tw_dir<DIR>(tw[b]));
    dft2<DIR>(v[2 * b], v[2 * b + 1]);
  }
}
template <int M>
FPM_HD void r2_store(float2* buf, int j, int Ns, const float2 (&v)[8]) {
  constexpr int G = M / 8;
  for (int b = 0; b < 4; ++b) {
    const int jj = j + b * G;
    const int k = jj & (Ns - 1);
    const int base = (jj - k) * 2 + k;
    buf[pidx(base)] = v[2 * b];
    buf[pidx(base + Ns)] = v[2 * b + 1];
  }
}

// ---- radix 16 (M = 256: two passes, 16 threads per transform) ----
// 16-point DFT in registers: n = n1 + 4 n2, k = k2 + 4 k1; DFT4 over n2,
// twiddles W16^(n1 k2), DFT4 over n1.
template <int DIR>
FPM_HD void dft16(float2 (&v)[16]) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  const float d = (float)DIR;
  float2 y[4][4];
  for (int n1 = 0; n1 < 4; ++n1) {
    float2 a0 = v[n1], a1 = v[n1 + 4], a2 = v[n1 + 8], a3 = v[n1 + 12];
    dft4<DIR>(a0, a1, a2, a3);
    y[n1][0] = a0; y[n1][1] = a1; y[n1][2] = a2; y[n1][3] = a3;
  }
  const float2 w1 = make_float2(c1, d * s1), w2 = make_float2(h, d * h), w3 = make_float2(s1, d * c1);
  const float2 w6 = make_float2(-h, d * h), w9 = make_float2(-c1, -d * s1);
  y[1][1] = cmul(y[1][1], w1); y[1][2] = cmul(y[1][2], w2); y[1][3] = cmul(y[1][3], w3);
  y[2][1] = cmul(y[2][1], w2); y[2][2] = mul_i<DIR>(y[2][2]); y[2][3] = cmul(y[2][3], w6);
  y[3][1] = cmul(y[3][1], w3); y[3][2] = cmul(y[3][2], w6); y[3][3] = cmul(y[3][3], w9);
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 a0 = y[0][k2], a1 = y[1][k2], a2 = y[2][k2], a3 = y[3][k2];
    dft4<DIR>(a0, a1, a2, a3);
    v[k2] = a0; v[k2 + 4] = a1; v[k2 + 8] = a2; v[k2 + 12] = a3;
  }
}

// Pruned forms of dft16 for transforms restricted to a box |t| <= h < 64 of a
// 256-point transform (index t taken mod 256). A thread's first-pass points
// are t = j + 16 n (n = 0..15); those with n = 4..11 lie in [64, 192) and are
// outside the box, so:
//  - ZIN:  inputs n = 4..11 are zero (first DFT4 stage has two inputs);
//  - ZOUT: only outputs k = 0..3 and 12..15 are wanted (last DFT4 stage
//          computes two of its four outputs; the others are left zero).
// Both give the same values as dft16 on the outputs they produce.
template <int DIR, bool ZIN, bool ZOUT>
FPM_HD void dft16p(float2 (&v)[16]) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  const float d = (float)DIR;
  float2 y[4][4];
  for (int n1 = 0; n1 < 4; ++n1) {
    if (ZIN) {
      const float2 a0 = v[n1], a3 = v[n1 + 12], ia3 = mul_i<DIR>(a3);
      y[n1][0] = cadd(a0, a3);
      y[n1][1] = csub(a0, ia3);
      y[n1][2] = csub(a0, a3);
      y[n1][3] = cadd(a0, ia3);
    } else {
      float2 a0 = v[n1], a1 = v[n1 + 4], a2 = v[n1 + 8], a3 = v[n1 + 12];
      dft4<DIR>(a0, a1, a2, a3);
      y[n1][0] = a0; y[n1][1] = a1; y[n1][2] = a2; y[n1][3] = a3;
    }
  }
  const float2 w1 = make_float2(c1, d * s1), w2 = make_float2(h, d * h), w3 = make_float2(s1, d * c1);
  const float2 w6 = make_float2(-h, d * h), w9 = make_float2(-c1, -d * s1);
  y[1][1] = cmul(y[1][1], w1); y[1][2] = cmul(y[1][2], w2); y[1][3] = cmul(y[1][3], w3);
  y[2][1] = cmul(y[2][1], w2); y[2][2] = mul_i<DIR>(y[2][2]); y[2][3] = cmul(y[2][3], w6);
  y[3][1] = cmul(y[3][1], w3); y[3][2] = cmul(y[3][2], w6); y[3][3] = cmul(y[3][3], w9);
  for (int k2 = 0; k2 < 4; ++k2) {
    if (ZOUT) {
      // outputs k2 (k1 = 0) and k2 + 12 (k1 = 3) of the DFT4 over n1
      const float2 a0 = y[0][k2], a1 = y[1][k2], a2 = y[2][k2], a3 = y[3][k2];
      const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_i<DIR>(csub(a1, a3));
      v[k2] = cadd(t0, t2);
      v[k2 + 12] = csub(t1, t3);
      v[k2 + 4] = make_float2(0.f, 0.f);
      v[k2 + 8] = make_float2(0.f, 0.f);
    } else {
      float2 a0 = y[0][k2], a1 = y[1][k2], a2 = y[2][k2], a3 = y[3][k2];
      dft4<DIR>(a0, a1, a2, a3);
      v[k2] = a0; v[k2 + 4] = a1; v[k2 + 8] = a2; v[k2 + 12] = a3;
    }
  }
}

// First-pass point t = j + 16 n of a 256-point transform whose non-zero
// inputs (or wanted outputs) are a box |t| <= h (t mod 256) of W = 2h + 1
// entries: the box index t + h or t - 256 + h, or -1 outside the box.
FPM_HD int box256(int j, int n, int h) {
  const int t = j + 16 * n;
  return t <= h ? t + h : (t >= 256 - h ? t - 256 + h : -1);
}

// Second-pass twiddles of thread j (256 points): tw2[(r-1) * 16 + j] = W256^(r j).
FPM_HD void fft256_twiddles(const float2* tw, float2* tw2, int j) {
  for (int r = 1; r < 16; ++r) tw2[(r - 1) * 16 + j] = tw[r * j];
}

template <int DIR>
FPM_HD void r16_load(const float2* buf, const float2* tw2, int j, int pass, float2 (&v)[16]) {
  for (int r = 0; r < 16; ++r) v[r] = buf[pidx16(j + 16 * r)];
  if (pass == 1)
    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw_dir<DIR>(tw2[(r - 1) * 16 + j]));
  dft16<DIR>(v);
}
FPM_HD void r16_store(float2* buf, int j, int pass, const float2 (&v)[16]) {
  if (pass == 0)
    for (int r = 0; r < 16; ++r) buf[pidx16(16 * j + r)] = v[r];
  else
    for (int r = 0; r < 16; ++r) buf[pidx16(j + 16 * r)] = v[r];
}

#if defined(__CUDACC__)
// 256-point transform by 16 threads (half a warp); tw2 in shared memory.
template <int DIR>
__device__ __forceinline__ void fft256_group(float2* __restrict__ buf, const float2* __restrict__ tw2, int j) {
  float2 v[16];
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    r16_load<DIR>(buf, tw2, j, pass, v);
    __syncwarp();
    r16_store(buf, j, pass, v);
    __syncwarp();
  }
}
// The same transform with the first pass's inputs (elements j + 16 r) given
// in registers: buf serves only as the exchange between the two passes and
// holds the result as fft256_group leaves it. Spares a zero-filled buffer
// when most inputs are known to be zero.
template <int DIR>
__device__ __forceinline__ void fft256_group_in(float2 (&v)[16], float2* __restrict__ buf,
                                                const float2* __restrict__ tw2, int j) {
  dft16<DIR>(v);
  __syncwarp();
  r16_store(buf, j, 0, v);
  __syncwarp();
  r16_load<DIR>(buf, tw2, j, 1, v);
  __syncwarp();
  r16_store(buf, j, 1, v);
  __syncwarp();
}
// Pruned 256-point transforms for a box |t| <= h < 64 (t mod 256): ZIN, the
// first pass's inputs are zero outside the box (points j + 16 n, n = 4..11);
// ZOUT, only the outputs in the box are wanted (j + 16 r, r = 0..3, 12..15),
// and only those are stored. The inputs of the first pass are in registers
// (points j + 16 r, as fft256_group_in takes them) or in buf.
template <int DIR, bool ZIN, bool ZOUT>
__device__ __forceinline__ void fft256_inreg_p(float2 (&v)[16], float2* __restrict__ buf,
                                               const float2* __restrict__ tw2, int j) {
  dft16p<DIR, ZIN, false>(v);
  __syncwarp();
  r16_store(buf, j, 0, v);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = buf[pidx16(j + 16 * r)];
#pragma unroll
  for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw_dir<DIR>(tw2[(r - 1) * 16 + j]));
  dft16p<DIR, false, ZOUT>(v);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r)
    if (!ZOUT || r < 4 || r >= 12) buf[pidx16(j + 16 * r)] = v[r];
  __syncwarp();
}
template <int DIR, bool ZOUT>
__device__ __forceinline__ void fft256_group_p(float2* __restrict__ buf, const float2* __restrict__ tw2, int j) {
  float2 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = buf[pidx16(j + 16 * r)];
  fft256_inreg_p<DIR, false, ZOUT>(v, buf, tw2, j);
}
#endif

// Box column (or row) stored at transform index t when a box of half-width h
// is centred on index 0 (indices t <= h and t >= n - h), else -1.
FPM_HD int box_index(int t, int n, int h) { return t <= h ? t + h : (t >= n - h ? t - n + h : -1); }

// ---- 512 points: radix 16, radix 16, radix 2 (32 threads x 16 points) ----
// Second-pass twiddles depend on k = j mod 16 only: tw2[(r-1) * 16 + k] =
// W256^(r k) = tw[2 r k] of the 512-point table.
FPM_HD void fft512_twiddles(const float2* tw, float2* tw2, int k) {
  for (int r = 1; r < 16; ++r) tw2[(r - 1) * 16 + k] = tw[2 * r * k];
}

template <int DIR>
FPM_HD void r16x512_load(const float2* buf, const float2* tw2, int j, int pass, float2 (&v)[16]) {
  for (int r = 0; r < 16; ++r) v[r] = buf[pidx16(j + 32 * r)];
  if (pass == 1)
    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw_dir<DIR>(tw2[(r - 1) * 16 + (j & 15)]));
  dft16<DIR>(v);
}
FPM_HD void r16x512_store(float2* buf, int j, int pass, const float2 (&v)[16]) {
  const int Ns = pass == 0 ? 1 : 16;
  const int k = j & (Ns - 1);
  const int base = (j - k) * 16 + k;
  for (int r = 0; r < 16; ++r) buf[pidx16(base + r * Ns)] = v[r];
}
// final radix-2 pass (Ns = 256): butterflies jj = j + 32 b, twiddle W512^jj
template <int DIR>
FPM_HD void r2x512_load(const float2* buf, const float2* tw, int j, float2 (&v)[16]) {
  for (int b = 0; b < 8; ++b) {
    const int jj = j + 32 * b;
    v[2 * b] = buf[pidx16(jj)];
    v[2 * b + 1] = cmul(buf[pidx16(jj + 256)], tw_dir<DIR>(tw[jj]));
    dft2<DIR>(v[2 * b], v[2 * b + 1]);
  }
}
FPM_HD void r2x512_store(float2* buf, int j, const float2 (&v)[16]) {
  for (int b = 0; b < 8; ++b) {
    const int jj = j + 32 * b;
    buf[pidx16(jj)] = v[2 * b];
    buf[pidx16(jj + 256)] = v[2 * b + 1];
  }
}

#if defined(__CUDACC__)
// 512-point transform by one warp; tw: 512-point table, tw2: second-pass twiddles.
template <int DIR>
__device__ __forceinline__ void fft512_group(float2* __restrict__ buf, const float2* __restrict__ tw,
                                             const float2* __restrict__ tw2, int j) {
  float2 v[16];
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    r16x512_load<DIR>(buf, tw2, j, pass, v);
    __syncwarp();
    r16x512_store(buf, j, pass, v);
    __syncwarp();
  }
  r2x512_load<DIR>(buf, tw, j, v);
  __syncwarp();
  r2x512_store(buf, j, v);
  __syncwarp();
}
#endif

template <int DIR>
inline void fft512_emulate(float2* buf, const float2* tw) {
  float2 tw2[15 * 16];
  for (int k = 0; k < 16; ++k) fft512_twiddles(tw, tw2, k);
  float2 V[32][16];
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < 32; ++j) r16x512_load<DIR>(buf, tw2, j, pass, V[j]);
    for (int j = 0; j < 32; ++j) r16x512_store(buf, j, pass, V[j]);
  }
  for (int j = 0; j < 32; ++j) r2x512_load<DIR>(buf, tw, j, V[j]);
  for (int j = 0; j < 32; ++j) r2x512_store(buf, j, V[j]);
}

template <int DIR>
inline void fft256_emulate(float2* buf, const float2* tw) {
  float2 tw2[15 * 16];
  for (int j = 0; j < 16; ++j) fft256_twiddles(tw, tw2, j);
  float2 V[16][16];
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < 16; ++j) r16_load<DIR>(buf, tw2, j, pass, V[j]);
    for (int j = 0; j < 16; ++j) r16_store(buf, j, pass, V[j]);
  }
}

#if defined(__CUDACC__)
// In-place transform of the padded buffer buf by the G threads of a group.
template <int M, int DIR>
__device__ __forceinline__ void fft_group(float2* __restrict__ buf, const FftTw<M>& T, int j) {
  using S = FftShape<M>;
  int Ns = 1;
#pragma unroll
  for (int pass = 0; pass < S::N8; ++pass) {
    float2 v[8];
    r8_load<M, DIR>(buf, pass > 0 ? T.w + (pass - 1) * 7 : T.w, j, Ns, v);
    __syncwarp();
    r8_store<M>(buf, j, Ns, v);
    __syncwarp();
    Ns *= 8;
  }
  if (S::TAIL == 2) {
    float2 v[8];
    r4_load<M, DIR>(buf, T.w + FftTw<M>::N8T, j, Ns, v);
    __syncwarp();
    r4_store<M>(buf, j, Ns, v);
    __syncwarp();
  } else if (S::TAIL == 1) {
    float2 v[8];
    r2_load<M, DIR>(buf, T.w + FftTw<M>::N8T, j, Ns, v);
    __syncwarp();
    r2_store<M>(buf, j, Ns, v);
    __syncwarp();
  }
}
#endif

// Host emulation of fft_group (all threads' read halves, then all write
// halves, pass by pass) for checking the index arithmetic on a CPU.
template <int M, int DIR>
inline void fft_group_emulate(float2* buf, const float2* tw) {
  using S = FftShape<M>;
  constexpr int G = M / 8;
  float2 V[G][8];
  FftTw<M> T[G];
  for (int j = 0; j < G; ++j) fft_twiddles<M>(tw, j, T[j]);
  int Ns = 1;
  for (int pass = 0; pass < S::N8; ++pass) {
    for (int j = 0; j < G; ++j) r8_load<M, DIR>(buf, pass > 0 ? T[j].w + (pass - 1) * 7 : T[j].w, j, Ns, V[j]);
    for (int j = 0; j < G; ++j) r8_store<M>(buf, j, Ns, V[j]);
    Ns *= 8;
  }
  if (S::TAIL == 2) {
    for (int j = 0; j < G; ++j) r4_load<M, DIR>(buf, T[j].w + FftTw<M>::N8T, j, Ns, V[j]);
    for (int j = 0; j < G; ++j) r4_store<M>(buf, j, Ns, V[j]);
  } else if (S::TAIL == 1) {
    for (int j = 0; j < G; ++j) r2_load<M, DIR>(buf, T[j].w + FftTw<M>::N8T, j, Ns, V[j]);
    for (int j = 0; j < G; ++j) r2_store<M>(buf, j, Ns, V[j]);
  }
}

}  // namespace fpmk

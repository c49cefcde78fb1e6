// CPU emulation of the engine's device helpers (FFT passes, Zernike
// polynomials, pupil). Built and run by tests/test_device_helpers_cpu.py,
// which compares the printed values against numpy and the FP64 oracle.
#include <cmath>
#include <cstdio>
#include <vector>

#include "device.cuh"
#include "optcoef.h"

using namespace fpmk;

template <int M>
static void run_fft() {
  std::vector<float2> tw(M), buf(M + M / 8);
  for (int t = 0; t < M; ++t) {
    const double a = -2.0 * M_PI * t / M;
    tw[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  for (int dir = -1; dir <= 1; dir += 2) {
    for (int t = 0; t < M; ++t)
      buf[pidx(t)] = make_float2((float)std::sin(0.37 * t + 0.1 * M), (float)std::cos(0.91 * t) - 0.25f);
    if (dir < 0) fft_group_emulate<M, -1>(buf.data(), tw.data());
    else fft_group_emulate<M, +1>(buf.data(), tw.data());
    std::printf("fft %d %d", M, dir);
    for (int t = 0; t < M; ++t) std::printf(" %.9g %.9g", buf[pidx(t)].x, buf[pidx(t)].y);
    std::printf("\n");
  }
}

template <int M>
static void run_fft_big() {
  std::vector<float2> tw(M), buf(M + M / 16);
  for (int t = 0; t < M; ++t) {
    const double a = -2.0 * M_PI * t / M;
    tw[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  for (int dir = -1; dir <= 1; dir += 2) {
    for (int t = 0; t < M; ++t)
      buf[pidx16(t)] = make_float2((float)std::sin(0.37 * t + 0.1 * M), (float)std::cos(0.91 * t) - 0.25f);
    if (M == 256) {
      if (dir < 0) fft256_emulate<-1>(buf.data(), tw.data());
      else fft256_emulate<+1>(buf.data(), tw.data());
    } else {
      if (dir < 0) fft512_emulate<-1>(buf.data(), tw.data());
      else fft512_emulate<+1>(buf.data(), tw.data());
    }
    std::printf("fft %d %d", M, dir);
    for (int t = 0; t < M; ++t) std::printf(" %.9g %.9g", buf[pidx16(t)].x, buf[pidx16(t)].y);
    std::printf("\n");
  }
}

// The 256-point transform as the dataflow step kernel runs it: 16 threads, thread j
// holding the first-pass points j + 16 n, dft16p (pruned on a box of half-width
// h < 64 when ZIN / ZOUT), the exchange between the two passes through a padded
// buffer, then dft16p again; outputs at j + 16 k.
template <int DIR, bool ZIN, bool ZOUT>
static void fft256_box_emulate(const float2* in, float2* out, const float2* tw) {
  float2 tw2[15 * 16];
  for (int j = 0; j < 16; ++j) fft256_twiddles(tw, tw2, j);
  float2 V[16][16], buf[256 + 16];
  for (int j = 0; j < 16; ++j) {
    for (int n = 0; n < 16; ++n) V[j][n] = in[j + 16 * n];
    dft16p<DIR, ZIN, false>(V[j]);
  }
  for (int j = 0; j < 16; ++j)
    for (int r = 0; r < 16; ++r) buf[pidx16(16 * j + r)] = V[j][r];
  for (int j = 0; j < 16; ++j) {
    for (int r = 0; r < 16; ++r) V[j][r] = buf[pidx16(j + 16 * r)];
    for (int r = 1; r < 16; ++r) V[j][r] = cmul(V[j][r], tw_dir<DIR>(tw2[(r - 1) * 16 + j]));
    dft16p<DIR, false, ZOUT>(V[j]);
  }
  for (int j = 0; j < 16; ++j)
    for (int k = 0; k < 16; ++k) out[j + 16 * k] = V[j][k];
}

static void run_box256() {
  std::vector<float2> tw(256), in(256), out(256);
  for (int t = 0; t < 256; ++t) {
    const double a = -2.0 * M_PI * t / 256;
    tw[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  for (int h : {53, 63, 72}) {
    // the box index of every first-pass point, and whether it is in the box
    int covered = 0;
    for (int j = 0; j < 16; ++j)
      for (int n = 0; n < 16; ++n) {
        const int b = box256(j, n, h);
        if (b >= 0) ++covered;
        const int t = j + 16 * n, ky = t <= 128 ? t : t - 256;
        const int want = (ky >= -h && ky <= h) ? ky + h : -1;
        if (b != want) std::printf("boxmap_bad %d %d %d %d\n", h, j, n, b);
        if (h < 64 && n >= 4 && n < 12 && b >= 0) std::printf("boxmap_bad %d %d %d %d\n", h, j, n, b);
      }
    std::printf("boxmap %d %d\n", h, covered);
  }
  // inverse transform of box-supported inputs (h = 53, pruned first pass) and
  // forward transform of a full input kept on the box (pruned last pass)
  const int h = 53;
  for (int t = 0; t < 256; ++t) {
    const int ky = t <= 128 ? t : t - 256;
    const bool inb = ky >= -h && ky <= h;
    in[t] = inb ? make_float2((float)std::sin(0.41 * t + 0.3), (float)std::cos(0.77 * t) - 0.2f) : make_float2(0.f, 0.f);
  }
  fft256_box_emulate<+1, true, false>(in.data(), out.data(), tw.data());
  std::printf("box256inv");
  for (int t = 0; t < 256; ++t) std::printf(" %.9g %.9g", out[t].x, out[t].y);
  std::printf("\n");
  for (int t = 0; t < 256; ++t) in[t] = make_float2((float)std::cos(0.23 * t + 1.1), (float)std::sin(0.59 * t) + 0.1f);
  fft256_box_emulate<-1, false, true>(in.data(), out.data(), tw.data());
  std::printf("box256fwd");
  for (int t = 0; t < 256; ++t) std::printf(" %.9g %.9g", out[t].x, out[t].y);
  std::printf("\n");
}

int main() {
  run_box256();
  run_fft_big<256>();
  run_fft_big<512>();
  run_fft<16>();
  run_fft<32>();
  run_fft<64>();
  run_fft<128>();
  for (int i = 0; i < 40; ++i) {
    const float x = (float)std::sin(1.3 * i) * 1.05f, y = (float)std::cos(0.7 * i + 0.2) * 0.9f;
    Zern z;
    zernike_eval(x, y, z);
    std::printf("zern %.9g %.9g", x, y);
    for (int j = 0; j < 14; ++j) std::printf(" %.9g %.9g %.9g", z.v[j], z.dx[j], z.dy[j]);
    std::printf("\n");
  }
  // aberration phase and its gradient through the monomial basis
  {
    float c[14];
    for (int j = 0; j < 14; ++j) c[j] = 0.3f * (float)std::cos(1.7 * j + 0.4);
    float K[15], Dx[10], Dy[10];
    theta_poly(c, K, Dx, Dy);
    float dmax = 0.f;  // the per-entry form used by the kernels must agree
    for (int e = 0; e < 35; ++e) {
      const float ref = e < 15 ? K[e] : (e < 25 ? Dx[e - 15] : Dy[e - 25]);
      dmax = std::fmax(dmax, std::fabs(theta_poly_entry(c, e) - ref));
    }
    std::printf("polyentry %.9g\n", dmax);
    // column form: theta and its gradient as polynomials in y on a column of fixed x
    float poly[35];
    for (int e = 0; e < 35; ++e) poly[e] = e < 15 ? K[e] : (e < 25 ? Dx[e - 15] : Dy[e - 25]);
    for (int i = 0; i < 30; ++i) {
      const float x = (float)std::cos(1.9 * i + 0.3) * 1.05f, y = (float)std::sin(0.83 * i) * 1.05f;
      ColPoly cp;
      col_poly(x, poly, cp);
      float gx, gy;
      col_grad(cp, y, gx, gy);
      std::printf("colform %.9g %.9g %.9g %.9g %.9g\n", x, y, col_theta(cp, y), gx, gy);
    }
    for (int i = 0; i < 30; ++i) {
      const float x = (float)std::sin(2.3 * i) * 1.05f, y = (float)std::cos(0.37 * i + 1.0) * 1.05f;
      float mo[15];
      monomials(x, y, mo);
      float th = 0.f, gx = 0.f, gy = 0.f;
      for (int m = 0; m < 15; ++m) th += K[m] * mo[m];
      for (int m = 0; m < 10; ++m) { gx += Dx[m] * mo[m]; gy += Dy[m] * mo[m]; }
      std::printf("theta %.9g %.9g %.9g %.9g %.9g", x, y, th, gx, gy);
      for (int j = 0; j < 14; ++j) {  // Z_j through the monomial rows
        float z = 0.f;
        for (int m = 0; m < 15; ++m) z += zern_mono(j, m) * mo[m];
        std::printf(" %.9g", z);
      }
      std::printf("\n");
    }
  }
  // the optimisers' per-step coefficients (b1 = 0.9, b2 = 0.999), steps 1..12
  for (int opt = 0; opt < 4; ++opt) {
    double prod = 1.0;
    for (int t = 1; t <= 12; ++t) {
      float k[4];
      prod = opt_coefficients(opt, 0.9, 0.999, t, prod, k);
      std::printf("coef %d %d %.9g %.9g %.9g %.9g %.17g\n", opt, t, k[0], k[1], k[2], k[3], prod);
    }
  }
  std::printf("nadam_advance %.17g\n", nadam_advance(0.9, 3, nadam_advance(0.9, 0, 1.0, 3), 12));
  // pupil value on a few q for fixed coefficients
  float zc[14];
  for (int j = 0; j < 14; ++j) zc[j] = 0.3f * (float)std::sin(2.1 * j + 0.3);
  const float R = 10.f, lambda = 0.532f, dk = 1.f / (32 * 0.6f), zz = 2.5f;
  for (int edge = 0; edge < 2; ++edge) {
    PupilConst P{R, 1.f / R, 1.f / lambda, dk * dk, edge};
    for (int i = 0; i < 60; ++i) {
      const float qy = (float)(std::sin(0.9 * i) * 11.0), qx = (float)(std::cos(1.7 * i) * 11.0);
      const float2 Mv = pupil_value(qy, qx, P, zc, zz);
      std::printf("pupil %d %.9g %.9g %.9g %.9g\n", edge, qy, qx, Mv.x, Mv.y);
    }
  }
  return 0;
}

// Fused per-LED forward model and adjoint of Batch-FPM (Section 2.1 Eq. 3,
// loss of Section 2.2 Eq. 5 / Eq. 4), one thread-block cluster per LED image.
//
// The spectrum of LED i is non-zero only on a (2h+1)^2 box around its crop
// centre, so the m x m inverse 2-D transform is split as
//   A  T(kx, y)   = sum_ky Phi(kx, ky) e^{+2 pi i ky y / m}   box columns only
//   B  psi(x, y)  = sum_kx T(kx, y)    e^{+2 pi i kx x / m}   every row y
//      residual gradient g(x, y), then
//      U(kx, y)   = sum_x g(x, y)      e^{-2 pi i kx x / m}   box columns kept
//   C  gPhi(kx,ky)= sum_y U(kx, y)     e^{-2 pi i ky y / m}   box rows kept
// CTA r of the cluster owns a slice of box columns (phases A and C) and a
// slice of image rows (phase B). T / U live in the owners' shared memory and
// are gathered / scattered through distributed shared memory in phase B.
#include <cooperative_groups.h>

#include "device.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace fpmk {

template <int M> struct LedCfg;
template <> struct LedCfg<32> { static constexpr int C = 2, NT = 64; };
template <> struct LedCfg<64> { static constexpr int C = 4, NT = 128; };
template <> struct LedCfg<128> { static constexpr int C = 8, NT = 256; };
template <> struct LedCfg<256> { static constexpr int C = 8, NT = 256; };

template <int M>
struct LedLayout {
  static constexpr int C = LedCfg<M>::C, NT = LedCfg<M>::NT;
  static constexpr int G = M / 8;                  // threads per transform
  static constexpr int NG = NT / G;                // transform groups per CTA
  static constexpr int ROWS = M / C;               // image rows per CTA
  static constexpr int TS = M + 1;                 // T row stride (odd: conflict-free gathers)
  static constexpr int FS = M + (G < 16 ? G : 0);  // per-group FFT buffer stride
  static size_t bytes(int W) {
    const int chunk = (W + C - 1) / C;
    return sizeof(float2) * ((size_t)chunk * TS + (size_t)NG * FS + M) + 16 * sizeof(float) +
           sizeof(double) * (NT / 32) * NPART;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int M>
__global__ void __launch_bounds__(LedCfg<M>::NT) led_kernel(const LedArgs a) {
  using L = LedLayout<M>;
  constexpr int C = L::C, NT = L::NT, G = L::G, NG = L::NG, ROWS = L::ROWS, TS = L::TS, FS = L::FS;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int k = blockIdx.x / C;
  const int W = a.W, h = a.h, N = a.N;
  const int chunk = (W + C - 1) / C;
  const int c0 = rank * chunk, c1 = min(W, c0 + chunk);

  extern __shared__ __align__(16) unsigned char smem[];
  float2* T = reinterpret_cast<float2*>(smem);
  float2* fb = T + (size_t)chunk * TS;
  float2* tws = fb + NG * FS;
  float* zc = reinterpret_cast<float*>(tws + M);
  double* red = reinterpret_cast<double*>(zc + 16);

  const int tid = threadIdx.x;
  const int led = a.idx[k];
  if (led < 0 || led >= a.n_leds) {  // same value for every CTA of the cluster: uniform exit
    if (tid == 0 && rank == 0) atomicOr(a.err, DERR_INDEX);
    return;
  }
  for (int t = tid; t < M; t += NT) tws[t] = a.tw[t];
  if (tid < 14) zc[tid] = a.sp[SP_ZERN + tid];
  const float zdef = a.sp[SP_DEFOCUS];
  const float gam = a.sp[SP_GAMMA + led];
  const float dly = a.sp[sp_offset(a.n_leds) + 2 * led];
  const float dlx = a.sp[sp_offset(a.n_leds) + 2 * led + 1];
  const int2 nn = a.n_int[led];
  const PupilConst P{a.R, a.Rinv, a.inv_lambda, a.dk2, a.hard_edge};
  __syncthreads();

  const int grp = tid / G, j = tid % G;
  float2* buf = fb + grp * FS;
  // column-major spectrum: box column c holds spectrum column N/2 + n.y - h + c,
  // and row ky of it sits at offset N/2 + n.x + ky
  const size_t col0 = (size_t)(N / 2 + nn.y - h);
  const int row0 = N / 2 + nn.x;

  // ---------------- phase A: column inverse transforms over ky -------------
  for (int cb = c0; cb < c1; cb += NG) {
    const int c = cb + grp;
    const bool act = c < c1;
    const float2* Ocol = a.Ot + (col0 + (act ? c : c0)) * N + row0;
    const float qx = (float)(c - h) - dlx;
    for (int t = j; t < M; t += G) {
      const int ky = t < M / 2 ? t : t - M;
      float2 v = make_float2(0.f, 0.f);
      if (act && ky >= -h && ky <= h) {
        const float2 Mv = pupil_value((float)ky - dly, qx, P, zc, zdef);
        if (Mv.x != 0.f || Mv.y != 0.f) v = cmul(Ocol[ky], Mv);
      }
      buf[t] = v;
    }
    __syncwarp();
    fft_group<M, +1>(buf, tws, j);
    if (act)
      for (int t = j; t < M; t += G) T[(c - c0) * TS + t] = buf[t];
    __syncwarp();
  }
  cluster.sync();

  // ---------------- phase B: rows: psi, residual, adjoint row transform ----
  const float inv_m2 = 1.f / (float)(M * M);
  const float sg = sqrtf(gam);
  float acc_loss = 0.f, acc_g = 0.f;
  for (int rb = 0; rb < ROWS; rb += NG) {
    const int rr = rb + grp;
    const bool act = rr < ROWS;
    const int y = rank * ROWS + (act ? rr : 0);
    for (int t = j; t < M; t += G) {
      const int kx = t < M / 2 ? t : t - M;
      float2 v = make_float2(0.f, 0.f);
      if (act && kx >= -h && kx <= h) {
        const int c = kx + h, own = c / chunk, lc = c - own * chunk;
        const float2* Tr = cluster.map_shared_rank(T, own);
        v = Tr[lc * TS + y];
      }
      buf[t] = v;
    }
    __syncwarp();
    fft_group<M, +1>(buf, tws, j);
    for (int t = j; t < M; t += G) {
      const float2 psi = cscale(buf[t], inv_m2);
      const float mag2 = psi.x * psi.x + psi.y * psi.y;
      float2 gp = make_float2(0.f, 0.f);
      if (act) {
        const size_t pix = (size_t)y * M + t;
        if (a.mode == MODE_FORWARD) {
          a.I_out[(size_t)k * M * M + pix] = gam * mag2;
        } else if (a.mode == MODE_LOSS) {
          const float meas = a.meas[(size_t)led * M * M + pix];
          if (a.loss == 0) {
            const float mag = sqrtf(mag2);
            const float res = sg * mag - sqrtf(fmaxf(meas, 0.f));
            acc_loss = fmaf(res, res, acc_loss);
            acc_g = fmaf(res, mag, acc_g);
            if (mag > 0.f) gp = cscale(psi, 2.f * res * sg / mag);
          } else {
            const float res = gam * mag2 - meas;
            acc_loss = fmaf(res, res, acc_loss);
            acc_g = fmaf(2.f * res, mag2, acc_g);
            gp = cscale(psi, 4.f * gam * res);
          }
        } else {
          const float d = a.dLdI[(size_t)k * M * M + pix];
          acc_g = fmaf(d, mag2, acc_g);
          gp = cscale(psi, 2.f * gam * d);
        }
      }
      buf[t] = gp;
    }
    __syncwarp();
    if (a.mode != MODE_FORWARD) {
      fft_group<M, -1>(buf, tws, j);
      if (act)
        for (int c = j; c < W; c += G) {
          const int kx = c - h, own = c / chunk, lc = c - own * chunk;
          float2* Tr = cluster.map_shared_rank(T, own);
          Tr[lc * TS + y] = buf[kx & (M - 1)];
        }
      __syncwarp();
    }
  }
  cluster.sync();
  if (a.mode == MODE_FORWARD) return;

  // ---------------- phase C: column transforms over y, box gradients -------
  float acc_z[14];
#pragma unroll
  for (int q = 0; q < 14; ++q) acc_z[q] = 0.f;
  float acc_def = 0.f, acc_dy = 0.f, acc_dx = 0.f;
  float2* gb = a.gbox + (size_t)k * W * W;
  for (int cb = c0; cb < c1; cb += NG) {
    const int c = cb + grp;
    const bool act = c < c1;
    for (int t = j; t < M; t += G) buf[t] = act ? T[(c - c0) * TS + t] : make_float2(0.f, 0.f);
    __syncwarp();
    fft_group<M, -1>(buf, tws, j);
    if (act) {
      const float2* Ocol = a.Ot + (col0 + c) * N + row0;
      const float qx = (float)(c - h) - dlx;
      for (int r = j; r < W; r += G) {
        const int ky = r - h;
        const float qy = (float)ky - dly;
        float2 out = make_float2(0.f, 0.f);
        const float A = pupil_amp(qy, qx, P);
        if (A > 0.f) {
          const float2 gphi = cscale(buf[ky & (M - 1)], inv_m2);
          Zern Z;
          zernike_eval(qx * P.Rinv, qy * P.Rinv, Z);
          float th = 0.f, dthx = 0.f, dthy = 0.f;
#pragma unroll
          for (int q = 0; q < 14; ++q) {
            th = fmaf(zc[q], Z.v[q], th);
            dthx = fmaf(zc[q], Z.dx[q], dthx);
            dthy = fmaf(zc[q], Z.dy[q], dthy);
          }
          const float r2 = qx * qx + qy * qy;
          float root;
          const float kap = defocus_kappa(r2, P, &root);
          float sn, cs;
          sincosf(fmaf(zdef, kap, th), &sn, &cs);
          const float2 e = make_float2(cs, sn);
          const float2 Mv = cscale(e, A);
          out = cmulc(Mv, gphi);                 // conj(M) gPhi
          const float2 gM = cmulc(Ocol[ky], gphi);  // conj(O) gPhi
          const float tt = -cmulc(gM, Mv).y;     // dL/dchi = Re(conj(gM) i M)
          const float ee = cmulc(gM, e).x;       // dL/dA   = Re(conj(gM) e^{i chi})
#pragma unroll
          for (int q = 0; q < 14; ++q) acc_z[q] = fmaf(tt, Z.v[q], acc_z[q]);
          acc_def = fmaf(tt, kap, acc_def);
          const float dk = -6.283185307179586f * P.dk2 / root;  // d kappa / d q = dk * q
          const float dchiy = fmaf(dthy, P.Rinv, zdef * dk * qy);
          const float dchix = fmaf(dthx, P.Rinv, zdef * dk * qx);
          float dAy = 0.f, dAx = 0.f;
          if (!P.hard_edge) {
            const float rad = sqrtf(r2);
            if (rad > P.R - 0.5f && rad < P.R + 0.5f) {
              dAy = -qy / rad;
              dAx = -qx / rad;
            }
          }
          acc_dy -= fmaf(tt, dchiy, ee * dAy);
          acc_dx -= fmaf(tt, dchix, ee * dAx);
        }
        gb[(size_t)c * W + r] = out;
      }
    }
    __syncwarp();
  }

  // ---------------- reduction of the scalar partials -----------------------
  const int warp = tid >> 5, lane = tid & 31;
  float vals[NPART];
  vals[P_LOSS] = acc_loss;
  vals[P_GAMMA] = acc_g;
#pragma unroll
  for (int q = 0; q < 14; ++q) vals[P_ZERN + q] = acc_z[q];
  vals[P_DEFOCUS] = acc_def;
  vals[P_DY] = acc_dy;
  vals[P_DX] = acc_dx;
#pragma unroll
  for (int q = 0; q < NPART; ++q) {
    const double s = warp_sum((double)vals[q]);
    if (lane == 0) red[warp * NPART + q] = s;
  }
  __syncthreads();
  if (tid < NPART) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w * NPART + tid];
    if (tid == P_GAMMA && a.mode == MODE_LOSS && a.loss == 0) s /= (double)sg;
    a.part[((size_t)k * C + rank) * NPART + tid] = s;
  }
}

int led_cluster_size(int m) {
  switch (m) {
    case 32: return LedCfg<32>::C;
    case 64: return LedCfg<64>::C;
    case 128: return LedCfg<128>::C;
    case 256: return LedCfg<256>::C;
  }
  return 0;
}

size_t led_smem_bytes(int m, int W) {
  switch (m) {
    case 32: return LedLayout<32>::bytes(W);
    case 64: return LedLayout<64>::bytes(W);
    case 128: return LedLayout<128>::bytes(W);
    case 256: return LedLayout<256>::bytes(W);
  }
  return 0;
}

// The dynamic shared-memory limit is a per-function attribute shared by all
// handles, so it is raised once to the device's opt-in maximum; each launch
// then asks for what its box width needs.
template <int M>
static cudaError_t prepare_t(int W) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (LedLayout<M>::bytes(W) > (size_t)optin) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(led_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

cudaError_t led_prepare(int m, int W) {
  switch (m) {
    case 32: return prepare_t<32>(W);
    case 64: return prepare_t<64>(W);
    case 128: return prepare_t<128>(W);
    case 256: return prepare_t<256>(W);
  }
  return cudaErrorInvalidValue;
}

template <int M>
static cudaError_t launch_t(const LedArgs& a, cudaStream_t s) {
  using L = LedLayout<M>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.B * L::C), 1, 1);
  cfg.blockDim = dim3(L::NT, 1, 1);
  cfg.dynamicSmemBytes = L::bytes(a.W);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L::C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, led_kernel<M>, a);
}

cudaError_t launch_led(int m, const LedArgs& a, cudaStream_t s) {
  switch (m) {
    case 32: return launch_t<32>(a, s);
    case 64: return launch_t<64>(a, s);
    case 128: return launch_t<128>(a, s);
    case 256: return launch_t<256>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fpmk

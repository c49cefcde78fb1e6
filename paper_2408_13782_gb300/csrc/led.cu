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
// The CTA's slice of O (support pixels only) and its rows of the measured
// image are copied into shared memory with cp.async at the start, so each
// kernel exposes global-memory latency about once. (Bulk copies on mbarriers
// gave the same kernel time and a step window longer by 0.6-1 us beside the
// update kernel's prologue, so the per-thread form stays.)
#include <cooperative_groups.h>

#include "../../include/fpm.h"
#include "device.cuh"
#include "internal.h"
#include "pixel.cuh"

namespace cg = cooperative_groups;

namespace fpmk {

// Threads per CTA for each low-res size; the cluster size C (CTAs per LED
// image) is a second template parameter (led_choose_cluster picks it).
template <int M> struct LedCfg;
template <> struct LedCfg<32> { static constexpr int NT = 64; };
template <> struct LedCfg<64> { static constexpr int NT = 128; };
template <> struct LedCfg<128> { static constexpr int NT = 256; };
template <> struct LedCfg<256> { static constexpr int NT = 256; };
template <> struct LedCfg<512> { static constexpr int NT = 256; };
// At m = 256 the 16-CTA cluster uses 128-thread CTAs (the threads per LED of
// the 8-CTA form): small CTAs pack two or three to an SM, so a whole 16-LED
// batch of clusters is co-resident and no cluster has to share its SMs.
template <int M, int C>
constexpr int led_threads() { return (M == 256 && C == 16) ? 128 : LedCfg<M>::NT; }


template <int M, int C, int NT_ = led_threads<M, C>()>
struct LedLayout {
  static constexpr int NT = NT_;
  static constexpr int G = FftBuf<M>::G;           // threads per transform
  static constexpr int NG = NT / G;                // transform groups per CTA
  static constexpr int ROWS = M / C;               // image rows per CTA
  static constexpr int TS = M + 1;                 // T row stride (odd: conflict-free gathers)
  static constexpr int FS = FftBuf<M>::SIZE;       // padded per-group buffer (stride = 8 mod 16 when G = 8)
  static constexpr int NW = NT / 32;
  static constexpr int NPOLY = 40;                 // K[15], Dx[10], Dy[10], pad
  static constexpr int NTW2 = M >= 256 ? 15 * 16 : 0;  // second-pass twiddles (M = 256, 512)
  // Phase A pushes its results into the row owners' staging rows (posted
  // remote stores) instead of phase B pulling them; m = 512 lacks the room.
  static constexpr bool PUSH = M <= 256;
  // staging rows are stored by box column, RS row slots per column (even, for
  // 16-byte stores of row pairs)
  static constexpr int RS = ROWS + 2;
  static size_t bytes(int W) {
    const int chunk = (W + C - 1) / C;
    return sizeof(float) * (size_t)ROWS * M +
           sizeof(float2) * ((size_t)chunk * TS + (size_t)NG * FS + M + NTW2 + (size_t)chunk * W +
                             (PUSH ? (size_t)RS * W + 1 : 0)) +   // + 1: 16-byte alignment of the staging rows
           sizeof(float) * (NPOLY + 14 * 15 + 2 + (size_t)NW * NACC) + sizeof(double) * 16;
  }
};


__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Programmatic dependent launch: let the next kernel in the stream be
// scheduled early / wait here until the previous kernel's writes are visible.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// In-place transform of one padded buffer by its thread group.
template <int M, int DIR>
__device__ __forceinline__ void transform(float2* buf, const FftTw<(M >= 256) ? 128 : M>& TW, const float2* tws,
                                          const float2* tw2, int j) {
  if constexpr (M == 256) fft256_group<DIR>(buf, tw2, j);
  else if constexpr (M == 512) fft512_group<DIR>(buf, tws, tw2, j);
  else fft_group<M, DIR>(buf, TW, j);
}

// The per-LED step for batch slot k of the job described by a (run by every
// thread of the slot's cluster).
// FF: the free-form pupil field is in the model (a separate instantiation, so
// the parametric kernels carry none of its registers). NT_: threads per CTA.
// SUB: the LED's C CTAs are CTAs base .. base + C - 1 of a larger cluster
// (sub_rank = this CTA's rank among them), which calls its two cluster
// barriers together with the other LEDs of the cluster. PR (m = 256 with a
// box half-width h < 64): the transforms skip the first-pass arithmetic on
// inputs known to be zero outside the box and the last-pass outputs outside it.
template <int M, int C, bool FF, int NT_ = led_threads<M, C>(), bool SUB = false, bool PR = false>
__device__ __forceinline__ void led_body(const LedArgs& a, const int k, const int sub_rank = 0) {
  static_assert(!PR || M == 256, "pruned transforms are the 256-point ones");
  using L = LedLayout<M, C, NT_>;
  constexpr int NT = L::NT, G = L::G, NG = L::NG, ROWS = L::ROWS, TS = L::TS, FS = L::FS;
  constexpr int NW = L::NW;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int rank = SUB ? sub_rank : crank;
  const int base = crank - rank;  // the LED's first CTA in the cluster
  const int W = a.W, h = a.h, N = a.N;
  const int chunk = (W + C - 1) / C;
  const int c0 = rank * chunk, c1 = min(W, c0 + chunk);
  const int y0 = rank * ROWS;

  // layout: image rows first (16-byte aligned for cp.async), then the float2 arrays
  extern __shared__ __align__(16) unsigned char smem[];
  float* ms = reinterpret_cast<float*>(smem);             // [ROWS][M] measured image / dL/dI rows
  float2* T = reinterpret_cast<float2*>(ms + ROWS * M);   // [chunk][TS] T, then U, by box column
  float2* fb = T + (size_t)chunk * TS;                    // [NG][FS] transform buffers
  float2* tws = fb + NG * FS;                             // [M] twiddle table
  float2* tw2 = tws + M;                                  // [15][16] second-pass twiddles (M = 256)
  float2* Ob = tw2 + L::NTW2;                             // [chunk][W] O on this CTA's box columns
  // [W][RS] this CTA's rows of T by box column (push form), 16-byte aligned
  float2* Rw = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(Ob + (size_t)chunk * W) + 15) & ~(uintptr_t)15);
  float* poly = L::PUSH ? reinterpret_cast<float*>(Rw + (size_t)L::RS * W)      // K[15] Dx[10] Dy[10]
                        : reinterpret_cast<float*>(Ob + (size_t)chunk * W);
  float* zmt = poly + L::NPOLY;                           // [14 * 15] Zernike -> monomial table
  float* red = zmt + 14 * 15 + 2;                         // [NW][NACC]
  double* dsum = reinterpret_cast<double*>(red + NW * NACC);  // [16] (8-byte aligned: float counts are even)

  const int tid = threadIdx.x;
  const int4 slot = a.slot[k];  // (LED, crop row, crop col): one load gives every address
  const int led = slot.x;
  if (led < 0 || led >= a.n_leds) {  // the same for every CTA of the LED: uniform exit
    if (tid == 0 && rank == 0) atomicOr(a.err, DERR_INDEX);
    if constexpr (SUB) {  // the cluster's other LEDs still pass both barriers
      cluster.sync();
      cluster.sync();
    }
    return;
  }
  // constant tables by cp.async (group 0): no stall before the O copies below
  for (int t = tid; t < M; t += NT) cp_async8(tws + t, a.tw + t);
  for (int t = tid; t < 14 * 15; t += NT) cp_async4(zmt + t, zern_mono_table() + t);
  cp_async_commit();
  pdl_wait();  // O and the scalar parameters come from the previous update
  // Only now may the next kernel (this step's update) start: it reads O, m
  // and v before its own wait, which is safe once the previous update, the
  // one this kernel just waited for, has completed.
  pdl_launch_dependents();
  // column-major spectrum: box column c is spectrum column N/2 + n_col - h + c,
  // and row ky of it sits at offset N/2 + n_row + ky
  const size_t col0 = (size_t)(N / 2 + slot.z - h);
  const int row0 = N / 2 + slot.y;
  {
    // O on a disk that contains the support for every admissible delta
    // (|delta| <= sqrt(2) * bound), so the copy does not wait for delta
    const float rs = (a.hard_edge ? a.R : a.R + 0.5f) + 1.41422f * FPM_OFFSET_BOUND_PX + 1e-3f;
    const int ncol = c1 > c0 ? c1 - c0 : 0;
    for (int q = tid; q < ncol * W; q += NT) {
      const int cl = q / W, r = q - cl * W;
      const float px = (float)(c0 + cl - h), py = (float)(r - h);
      if (px * px + py * py <= rs * rs)
        cp_async8(Ob + q, a.Ot + (col0 + c0 + cl) * N + (row0 - h + r));
    }
  }
  cp_async_commit();  // group 1: O (needed by phase A)
  // group 2: this CTA's image rows (needed by phase B), arriving during phase A
  const bool fwd_only = a.mode == MODE_FORWARD || a.mode == MODE_FORWARD_STORE;
  const bool stored = a.mode == MODE_UPSTREAM_STORED;  // psi comes from memory: no inverse transforms
  const float* rows_src = a.mode == MODE_LOSS ? a.meas + ((size_t)led * M + y0) * M
                        : (a.mode == MODE_UPSTREAM || stored) ? a.dLdI + ((size_t)k * M + y0) * M : nullptr;
  if (rows_src)
    for (int q = tid; q < ROWS * M / 4; q += NT) cp_async16(ms + 4 * q, rows_src + 4 * q);
  cp_async_commit();
  float zc = 0.f;
  if (tid < 14) zc = a.sp[SP_ZERN + tid];
  const float zdef = a.sp[SP_DEFOCUS];
  const float gam = a.sp[SP_GAMMA + led];
  const float dly = a.sp[sp_offset(a.n_leds) + 2 * led];
  const float dlx = a.sp[sp_offset(a.n_leds) + 2 * led + 1];
  // the box and the staged O disk hold the support only for offsets within the bound
  if (tid == 0 && rank == 0 && !(fabsf(dly) <= FPM_OFFSET_BOUND_PX && fabsf(dlx) <= FPM_OFFSET_BOUND_PX))
    atomicOr(a.err, DERR_OFFSET);
  const PupilConst P{a.R, a.Rinv, a.inv_lambda, a.dk2, a.hard_edge};
  const FreeForm ff = FF ? free_form(a.pupil, W, dly, dlx) : FreeForm{nullptr, 0, 0, 0, 0.f, 0.f};  // (ff.P == nullptr: none)
  if (FF && a.pupil && a.pwt && tid == 0 && rank == 0) a.pwt[k] = make_float4(ff.fy, ff.fx, (float)ff.ay, (float)ff.ax);
  const int grp = tid / G, j = tid % G;
  float2* buf = fb + grp * FS;
  if (tid < 14) red[tid] = zc;   // the aberration coefficients, via the (still unused) reduction area
  cp_async_wait<2>();  // group 0: the constant tables
  __syncthreads();
  if (tid < 35) poly[tid] = theta_poly_entry_tab(red, zmt, tid);  // aberration phase as monomials of q/R
  FftTw<(M >= 256) ? 128 : M> TW;  // radix-8 path: per-thread twiddles in registers
  __syncthreads();                // twiddle table
  if constexpr (M == 256) {
    if (tid < 16) fft256_twiddles(tws, tw2, tid);
  } else if constexpr (M == 512) {
    if (tid < 16) fft512_twiddles(tws, tw2, tid);
  } else {
    fft_twiddles<M>(tws, j, TW);
  }
  // the O slice (a wait that gives up flags the launch; the kernel runs on, so
  // the CTA stays resident while the copies could still land)
  cp_async_wait<1>();  // all but the most recent group: the O slice
  __syncthreads();     // O slice in shared memory

  // ---------------- phase A: column inverse transforms over ky -------------
  for (int cb = c0; cb < (stored ? c0 : c1); cb += NG) {
    const int c = cb + grp;
    const bool act = c < c1;
    const float2* Oc = Ob + (size_t)(act ? c - c0 : 0) * W + h;   // index by ky
    const float qx = (float)(c - h) - dlx, qx2 = qx * qx;
    ColPoly cp;  // the aberration phase along this column
    col_poly(qx * P.Rinv, poly, cp);
    if constexpr (M != 256)  // (m = 256 reads only the box back below)
      for (int t = h + 1 + j; t < M - h; t += G) buf[bidx<M>(t)] = make_float2(0.f, 0.f);  // outside the box
    for (int r = j; r < W; r += G) {
      const int ky = r - h;
      const float qy = (float)ky - dly, r2 = fmaf(qy, qy, qx2);
      float rad;
      const float A = act ? pupil_amp_r2(r2, P, rad) : 0.f;
      float2 v = make_float2(0.f, 0.f);
      if (A > 0.f) {
        v = cmul(Oc[ky], pupil_col(qy, r2, A, P, cp, zdef));
        if (FF && ff.P) v = cmul(v, ff_value(ff, r, c));
      }
      buf[bidx<M>(ky & (M - 1))] = v;
    }
    __syncwarp();
    if constexpr (M == 256) {
      // first-pass inputs: the box values just written, zeros elsewhere
      float2 v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r)
        v[r] = box_index(j + 16 * r, M, h) >= 0 ? buf[bidx<M>(j + 16 * r)] : make_float2(0.f, 0.f);
      if constexpr (PR) fft256_inreg_p<+1, true, false>(v, buf, tw2, j);
      else fft256_group_in<+1>(v, buf, tw2, j);
    } else {
      transform<M, +1>(buf, TW, tws, tw2, j);
    }
    if (act) {
      if constexpr (L::PUSH) {
        // rows t, t + 1 of T belong to CTA t / ROWS: one 16-byte remote store per pair
        for (int t = 2 * j; t < M; t += 2 * G) {
          const float2 u0 = buf[bidx<M>(t)], u1 = buf[bidx<M>(t + 1)];
          float4* dst = reinterpret_cast<float4*>(cluster.map_shared_rank(Rw, base + t / ROWS) + (size_t)c * L::RS + t % ROWS);
          *dst = make_float4(u0.x, u0.y, u1.x, u1.y);
        }
      } else {
        for (int t = j; t < M; t += G) T[(c - c0) * TS + t] = buf[bidx<M>(t)];
      }
    }
    __syncwarp();
  }
  cp_async_wait<0>();  // image rows
  cluster.sync();      // (also a block-wide barrier for the rows)

  // ---------------- phase B: rows: psi, residual, adjoint row transform ----
  const float inv_m2 = 1.f / (float)(M * M);
  const float sg = sqrtf(gam);
  float acc_loss = 0.f, acc_g = 0.f;
  for (int rb = 0; rb < ROWS; rb += NG) {
    const int rr = rb + grp;
    const bool act = rr < ROWS;
    const int yl = act ? rr : 0, y = y0 + yl;
    if (stored) {
      for (int t = j; t < M; t += G)
        buf[bidx<M>(t)] = act ? a.psi[((size_t)k * M + y) * M + t] : make_float2(0.f, 0.f);
    } else if constexpr (M == 256 && L::PUSH) {
      // first-pass inputs straight from the staging rows (zeros outside the box)
      float2 v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int c = box_index(j + 16 * r, M, h);
        v[r] = (act && c >= 0) ? Rw[(size_t)c * L::RS + yl] : make_float2(0.f, 0.f);
      }
      if constexpr (PR) fft256_inreg_p<+1, true, false>(v, buf, tw2, j);
      else fft256_group_in<+1>(v, buf, tw2, j);
    } else {
      for (int t = h + 1 + j; t < M - h; t += G) buf[bidx<M>(t)] = make_float2(0.f, 0.f);  // outside the box
      if constexpr (L::PUSH) {
        for (int c = j; c < W; c += G)
          buf[bidx<M>((c - h) & (M - 1))] = act ? Rw[(size_t)c * L::RS + yl] : make_float2(0.f, 0.f);
      } else
      // remote loads from the owning CTAs, eight in flight before any is stored
      for (int cb = j; cb < W; cb += 8 * G) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = cb + u * G;
          v[u] = make_float2(0.f, 0.f);
          if (act && c < W) {
            const int own = c / chunk, lc = c - own * chunk;
            v[u] = cluster.map_shared_rank(T, base + own)[lc * TS + y];
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = cb + u * G;
          if (c < W) buf[bidx<M>((c - h) & (M - 1))] = v[u];
        }
      }
      __syncwarp();
      transform<M, +1>(buf, TW, tws, tw2, j);
    }
    // residual per pixel; the loop for each loss form is branch-free so that
    // the pixels of a thread interleave
    const float sc = stored ? 1.f : inv_m2;
    if (!act) {
      for (int t = j; t < M; t += G) buf[bidx<M>(t)] = make_float2(0.f, 0.f);
    } else if (fwd_only) {
      for (int t = j; t < M; t += G) {
        const float2 psi = cscale(buf[bidx<M>(t)], sc);
        a.I_out[((size_t)k * M + y) * M + t] = gam * (psi.x * psi.x + psi.y * psi.y);
        if (a.mode == MODE_FORWARD_STORE) a.psi[((size_t)k * M + y) * M + t] = psi;
        buf[bidx<M>(t)] = make_float2(0.f, 0.f);
      }
    } else if (a.mode == MODE_LOSS && a.loss == 0 && a.meas_is_amp) {
      // all of this thread's pixels loaded first: the stores into buf cannot
      // then hold back the loads (the compiler cannot tell buf and ms apart)
      constexpr int NU = M / G;
      float2 pv[NU];
      float av[NU];
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        pv[u] = buf[bidx<M>(j + G * u)];
        av[u] = ms[yl * M + j + G * u];
      }
#pragma unroll
      for (int u = 0; u < NU; ++u) pv[u] = residual_amp_pixel(cscale(pv[u], sc), av[u], sg, acc_loss, acc_g);
#pragma unroll
      for (int u = 0; u < NU; ++u) buf[bidx<M>(j + G * u)] = pv[u];
    } else if (a.mode == MODE_LOSS && a.loss == 0) {
#pragma unroll 4
      for (int t = j; t < M; t += G)
        buf[bidx<M>(t)] = residual_pixel(cscale(buf[bidx<M>(t)], sc), ms[yl * M + t], MODE_LOSS, 0, gam, sg,
                                         acc_loss, acc_g);
    } else if (a.mode == MODE_LOSS) {
#pragma unroll 4
      for (int t = j; t < M; t += G)
        buf[bidx<M>(t)] = residual_pixel(cscale(buf[bidx<M>(t)], sc), ms[yl * M + t], MODE_LOSS, 1, gam, sg,
                                         acc_loss, acc_g);
    } else {
#pragma unroll 4
      for (int t = j; t < M; t += G)
        buf[bidx<M>(t)] = residual_pixel(cscale(buf[bidx<M>(t)], sc), ms[yl * M + t], MODE_UPSTREAM, 0, gam, sg,
                                         acc_loss, acc_g);
    }
    __syncwarp();
    if (!fwd_only) {
      if constexpr (PR) fft256_group_p<-1, true>(buf, tw2, j);  // only the box columns are kept
      else transform<M, -1>(buf, TW, tws, tw2, j);
      if (act)
        for (int c = j; c < W; c += G) {
          const int kx = c - h, own = c / chunk, lc = c - own * chunk;
          float2* Tr = cluster.map_shared_rank(T, base + own);
          Tr[lc * TS + y] = buf[bidx<M>(kx & (M - 1))];
        }
      __syncwarp();
    }
  }
  cluster.sync();
  if (fwd_only) return;

  // ---------------- phase C: column transforms over y, box gradients -------
  BoxAcc bacc;
  box_acc_zero(bacc);
  float2* gb = a.gbox + (size_t)k * W * W;
  float2* pb = (FF && a.pupil) ? a.pbox + (size_t)k * W * W : nullptr;
  for (int cb = c0; cb < c1; cb += NG) {
    const int c = cb + grp;
    const bool act = c < c1;
    if constexpr (M == 256) {  // first-pass inputs straight from T
      float2 v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = act ? T[(c - c0) * TS + j + 16 * r] : make_float2(0.f, 0.f);
      if constexpr (PR) fft256_inreg_p<-1, false, true>(v, buf, tw2, j);  // only the box rows are kept
      else fft256_group_in<-1>(v, buf, tw2, j);
    } else {
      for (int t = j; t < M; t += G) buf[bidx<M>(t)] = act ? T[(c - c0) * TS + t] : make_float2(0.f, 0.f);
      __syncwarp();
      transform<M, -1>(buf, TW, tws, tw2, j);
    }
    if (act) {
      const float2* Oc = Ob + (size_t)(c - c0) * W + h;
      const float qx = (float)(c - h) - dlx, qx2 = qx * qx;
      ColPoly cp;  // the aberration phase along this column
      col_poly(qx * P.Rinv, poly, cp);
      float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // sum t(p) y^b over this thread's pixels of the column
      for (int r = j; r < W; r += G) {
        const int ky = r - h;
        const float qy = (float)ky - dly, r2 = fmaf(qy, qy, qx2);
        float rad;
        const float A = pupil_amp_r2(r2, P, rad);
        float2 out = make_float2(0.f, 0.f), Gp = out;
        if (A > 0.f)
          out = box_pixel_col(qy, qx, r2, A, rad, cscale(buf[bidx<M>(ky & (M - 1))], inv_m2), Oc[ky], P, cp, zdef, S,
                              bacc, ff, r, c, &Gp);
        gb[(size_t)c * W + r] = out;
        if (FF && pb) pb[(size_t)c * W + r] = Gp;
      }
      col_fold(cp, S, bacc);
    }
    __syncwarp();
  }

  // ---------------- reduction of the scalar partials -----------------------
  write_partials(acc_loss, acc_g, bacc, a.mode == MODE_LOSS && a.loss == 0, sg, red, reinterpret_cast<float*>(dsum), zmt,
                 a.part + ((size_t)k * C + rank) * NPART);
}

// One job: cluster k takes batch slot k.
template <int M, int C, bool FF, bool PR = false>
__global__ void __launch_bounds__(led_threads<M, C>(), M == 512 ? 1 : 2) led_kernel(const LedArgs a) {
  led_body<M, C, FF, led_threads<M, C>(), false, PR>(a, (int)(blockIdx.x / C));
}

// Several jobs in one launch (the serving loop): cluster q takes slot
// map[q].y of job map[q].x, whose arguments are copied to shared memory.
template <int M, int C, bool FF, bool PR = false>
__global__ void __launch_bounds__(led_threads<M, C>(), M == 512 ? 1 : 2)
    led_kernel_jobs(const LedArgs* __restrict__ jobs, const int2* __restrict__ map) {
  __shared__ LedArgs sa;
  const int2 q = map[blockIdx.x / C];
  if (threadIdx.x == 0) sa = jobs[q.x];
  __syncthreads();
  led_body<M, C, FF, led_threads<M, C>(), false, PR>(sa, q.y);
}

// Jobs of different low-res sizes in one launch (the serving loop's mixed
// rounds): clusters of LED_MIX_CLUSTER CTAs of LED_MIX_THREADS threads, in
// which an LED of size m takes C(m) = m / 16 consecutive CTAs (m = 64, 128,
// 256: 4, 8, 16), so a cluster holds 4, 2 or 1 LEDs, of one job or several.
// map[b] = (job, batch slot, rank among the LED's CTAs, m) for CTA b; job < 0
// marks an idle CTA, which passes the cluster's two barriers and exits.
template <bool FF>
__global__ void __launch_bounds__(LED_MIX_THREADS, 2)
    led_kernel_mixed(const LedArgs* __restrict__ jobs, const int4* __restrict__ map) {
  __shared__ LedArgs sa;
  const int4 q = map[blockIdx.x];
  if (q.x >= 0 && threadIdx.x == 0) sa = jobs[q.x];
  __syncthreads();
  switch (q.x < 0 ? 0 : q.w) {
    case 64: led_body<64, 4, FF, LED_MIX_THREADS, true>(sa, q.y, q.z); break;
    case 128: led_body<128, 8, FF, LED_MIX_THREADS, true>(sa, q.y, q.z); break;
    case 256: led_body<256, 16, FF, LED_MIX_THREADS, true, true>(sa, q.y, q.z); break;  // h < 64 (led_mixed_fits)
    default: {
      cg::cluster_group cluster = cg::this_cluster();
      cluster.sync();
      cluster.sync();
    }
  }
}

// Cluster sizes built for each low-res size (CTAs cooperating on one LED).
int led_cluster_size(int m) {
  switch (m) {
    case 32: return 2;
    case 64: return 4;
    case 128: return 8;
    case 256: return 8;
    case 512: return 16;
  }
  return 0;
}

template <int M, int C>
static const void* kernel_ptr(int W) {  // the parametric kernel a launch with box W uses
  if constexpr (M == 256)
    if ((W - 1) / 2 < 64) return (const void*)led_kernel<M, C, false, true>;
  return (const void*)led_kernel<M, C, false>;
}

template <int M, int C>
static cudaError_t prepare_t(int W);

template <int M, int C>
static int max_active_clusters(int W) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(led_threads<M, C>(), 1, 1);
  cfg.dynamicSmemBytes = LedLayout<M, C>::bytes(W);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel_ptr<M, C>(W), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// m = 256: a 16-CTA cluster of 128-thread CTAs (a non-portable size) when the
// device can hold 16 of them at once (a whole 16-LED batch in one wave), else 8.
// m = 512 needs 16 (shared memory per CTA); 0 if the device cannot run it.
int led_choose_cluster(int m, int W) {
  if (m == 512) {
    if (prepare_t<512, 16>(W) != cudaSuccess || max_active_clusters<512, 16>(W) < 1) {
      cudaGetLastError();
      return 0;
    }
    return 16;
  }
  if (m != 256) return led_cluster_size(m);
  if (prepare_t<256, 16>(W) != cudaSuccess || max_active_clusters<256, 16>(W) < 16) {
    cudaGetLastError();
    return 8;  // a 16-LED batch of 16-CTA clusters would need a second wave
  }
  return 16;
}

size_t led_smem_bytes(int m, int C, int W) {
  if (m == 32) return LedLayout<32, 2>::bytes(W);
  if (m == 64) return LedLayout<64, 4>::bytes(W);
  if (m == 128) return LedLayout<128, 8>::bytes(W);
  if (m == 256) return C == 16 ? LedLayout<256, 16>::bytes(W) : LedLayout<256, 8>::bytes(W);
  if (m == 512) return LedLayout<512, 16>::bytes(W);
  return 0;
}

// The dynamic shared-memory limit is a per-function attribute shared by all
// handles, so it is raised once to the device's opt-in maximum; each launch
// then asks for what its box width needs.
template <int M, int C>
static cudaError_t prepare_t(int W) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (LedLayout<M, C>::bytes(W) > (size_t)optin) return cudaErrorInvalidValue;
  // both entry points (one job, several jobs; the latter also holds a copy
  // of its job's arguments in static shared memory), with and without the
  // free-form field
  // and, at m = 256, in the pruned forms for boxes with h < 64
  const void* fns[8] = {(const void*)led_kernel<M, C, false>, (const void*)led_kernel_jobs<M, C, false>,
                        (const void*)led_kernel<M, C, true>, (const void*)led_kernel_jobs<M, C, true>,
                        (const void*)led_kernel<M, C, false, M == 256>, (const void*)led_kernel_jobs<M, C, false, M == 256>,
                        (const void*)led_kernel<M, C, true, M == 256>, (const void*)led_kernel_jobs<M, C, true, M == 256>};
  for (int f = 0; f < (M == 256 ? 8 : 4); ++f) {
    if (C > 8) {
      e = cudaFuncSetAttribute(fns[f], cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    // the largest shared-memory carveout, so the SM configuration does not flip between kernels
    e = cudaFuncSetAttribute(fns[f], cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fns[f]);
    if (e != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes;  // room left beside the static shared memory
    e = cudaFuncSetAttribute(fns[f], cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t led_prepare(int m, int C, int W) {
  if (m == 32) return prepare_t<32, 2>(W);
  if (m == 64) return prepare_t<64, 4>(W);
  if (m == 128) return prepare_t<128, 8>(W);
  if (m == 256) return C == 16 ? prepare_t<256, 16>(W) : prepare_t<256, 8>(W);
  if (m == 512 && C == 16) return prepare_t<512, 16>(W);
  return cudaErrorInvalidValue;
}

template <int M, int C>
static cudaError_t launch_t(const LedArgs& a, cudaStream_t s, bool pdl) {
  using L = LedLayout<M, C>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.B * C), 1, 1);
  cfg.blockDim = dim3(L::NT, 1, 1);
  cfg.dynamicSmemBytes = L::bytes(a.W);
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  if (M == 256 && a.h < 64)
    return a.pupil ? cudaLaunchKernelEx(&cfg, led_kernel<M, C, true, M == 256>, a)
                   : cudaLaunchKernelEx(&cfg, led_kernel<M, C, false, M == 256>, a);
  return a.pupil ? cudaLaunchKernelEx(&cfg, led_kernel<M, C, true>, a) : cudaLaunchKernelEx(&cfg, led_kernel<M, C, false>, a);
}

template <int M, int C>
static cudaError_t launch_jobs_t(const LedArgs* jobs, const int2* map, int n_clusters, int W_max, cudaStream_t s,
                                 bool pdl, bool ff) {
  using L = LedLayout<M, C>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_clusters * C), 1, 1);
  cfg.blockDim = dim3(L::NT, 1, 1);
  cfg.dynamicSmemBytes = L::bytes(W_max);
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  if (M == 256 && (W_max - 1) / 2 < 64)  // the jobs of a same-configuration round share their box
    return ff ? cudaLaunchKernelEx(&cfg, led_kernel_jobs<M, C, true, M == 256>, jobs, map)
              : cudaLaunchKernelEx(&cfg, led_kernel_jobs<M, C, false, M == 256>, jobs, map);
  return ff ? cudaLaunchKernelEx(&cfg, led_kernel_jobs<M, C, true>, jobs, map)
            : cudaLaunchKernelEx(&cfg, led_kernel_jobs<M, C, false>, jobs, map);
}

cudaError_t launch_led_jobs(int m, int C, const LedArgs* jobs, const int2* map, int n_clusters, int W_max,
                            cudaStream_t s, bool pdl, bool ff) {
  if (n_clusters < 1) return cudaErrorInvalidValue;
  if (m == 32) return launch_jobs_t<32, 2>(jobs, map, n_clusters, W_max, s, pdl, ff);
  if (m == 64) return launch_jobs_t<64, 4>(jobs, map, n_clusters, W_max, s, pdl, ff);
  if (m == 128) return launch_jobs_t<128, 8>(jobs, map, n_clusters, W_max, s, pdl, ff);
  if (m == 256)
    return C == 16 ? launch_jobs_t<256, 16>(jobs, map, n_clusters, W_max, s, pdl, ff)
                   : launch_jobs_t<256, 8>(jobs, map, n_clusters, W_max, s, pdl, ff);
  if (m == 512 && C == 16) return launch_jobs_t<512, 16>(jobs, map, n_clusters, W_max, s, pdl, ff);
  return cudaErrorInvalidValue;
}

int led_mixed_cluster(int m) { return (m == 64 || m == 128 || m == 256) ? m / 16 : 0; }

size_t led_mixed_smem_bytes(int m, int W) {
  if (m == 64) return LedLayout<64, 4, LED_MIX_THREADS>::bytes(W);
  if (m == 128) return LedLayout<128, 8, LED_MIX_THREADS>::bytes(W);
  if (m == 256) return LedLayout<256, 16, LED_MIX_THREADS>::bytes(W);
  return 0;
}

bool led_mixed_fits(int m, int W) {
  static int room = -1;  // opt-in shared memory beside the kernel's static shared memory
  if (room < 0) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, (const void*)led_kernel_mixed<true>) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    room = optin - (int)fa.sharedSizeBytes;
  }
  const size_t b = led_mixed_smem_bytes(m, W);
  return b > 0 && b <= (size_t)room && (m != 256 || (W - 1) / 2 < 64);  // m = 256: the pruned body only
}

cudaError_t led_mixed_prepare() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const void* fns[2] = {(const void*)led_kernel_mixed<false>, (const void*)led_kernel_mixed<true>};
  for (int f = 0; f < 2 && e == cudaSuccess; ++f) {
    e = cudaFuncSetAttribute(fns[f], cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fns[f], cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fns[f]);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fns[f], cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  }
  return e;
}

cudaError_t launch_led_mixed(const LedArgs* jobs, const int4* map, int n_ctas, size_t smem, cudaStream_t s, bool pdl,
                             bool ff) {
  if (n_ctas < 1 || n_ctas % LED_MIX_CLUSTER) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_ctas, 1, 1);
  cfg.blockDim = dim3(LED_MIX_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = LED_MIX_CLUSTER;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  return ff ? cudaLaunchKernelEx(&cfg, led_kernel_mixed<true>, jobs, map)
            : cudaLaunchKernelEx(&cfg, led_kernel_mixed<false>, jobs, map);
}

cudaError_t launch_led(int m, int C, const LedArgs& a, cudaStream_t s, bool pdl) {
  if (m == 32) return launch_t<32, 2>(a, s, pdl);
  if (m == 64) return launch_t<64, 4>(a, s, pdl);
  if (m == 128) return launch_t<128, 8>(a, s, pdl);
  if (m == 256) return C == 16 ? launch_t<256, 16>(a, s, pdl) : launch_t<256, 8>(a, s, pdl);
  if (m == 512 && C == 16) return launch_t<512, 16>(a, s, pdl);
  return cudaErrorInvalidValue;
}

}  // namespace fpmk

// Per-LED forward model and adjoint of Batch-FPM (Section 2.1 Eq. 3, loss of
// Section 2.2 Eq. 5 / Eq. 4) with the m-point DFTs written as dense complex
// contractions on the tensor cores: one CTA per LED image, tcgen05.mma with
// FP32 accumulators in tensor memory, operands in shared memory brought in by
// bulk copies (TMA engine) through a ring of stages.
//
// With E(y, k) = exp(+2 pi i y k / m), box index c <-> frequency k_c = c - h,
// and the spectrum Phi(r, c) = O(row r, col c) M(r, c) on the (padded) box:
//   1  T(y, c)   = sum_r E(y, k_r) Phi(r, c)          rows y of a tile
//   2  psi(y, x) = sum_c T(y, c) E(x, k_c) / m^2      per chunk of columns x
//      residual g(y, x) = dL/dpsi, then
//   3  U(y, c)   = sum_x g(y, x) conj E(x, k_c)       accumulated over chunks
//   4  gPhi(r,c) = sum_y U(y, c) conj E(y, k_r) / m^2 summed over tiles
// A complex contraction is one real contraction of twice the depth: the data
// operand holds [Re | Im] along K and the constant DFT factor is expanded to
// [[Re, -Im], [Im, Re]] (two output blocks, real and imaginary part). Steps 1
// and 3 put the constant in A (outputs in two TMEM column blocks, lanes = the
// data's rows), steps 2 and 4 put it in B; so every intermediate that leaves
// tensor memory is one row per thread, written out without a transpose.
// Data operands go through a per-slot scratch area in global memory (L2).
// At m = 256 (two row tiles) an LED takes a cluster of two CTAs: each builds
// half of the box spectrum Phi, then runs steps 1-4 for one row tile; the two
// tiles' partial sums of step 4 are exchanged through global memory and each
// CTA finishes the box gradients of half of the box rows.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "../../include/fpm.h"
#include "device.cuh"
#include "internal.h"
#include "pixel.cuh"
#include "tc.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace fpmk {
namespace {

constexpr int GT = 256;                        // threads per CTA
constexpr uint64_t WAIT_NS = 200000000ull;     // bounded waits: 200 ms
constexpr int MAX_STAGES = 12;
constexpr uint32_t A_SLICE = 128 * 32;         // one K-step of a 128-row operand

__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Byte offset of element (r, k) of an R-row operand with e-byte elements.
__host__ __device__ inline size_t opnd_off(int R, int e, int r, int k) {
  const int KE = 32 / e, T = 16 / e;
  return (size_t)(k / KE) * (size_t)(R * 32) + (size_t)(r >> 3) * 256 + (size_t)((k % KE) / T) * 128 +
         (size_t)(r & 7) * 16 + (size_t)(k % T) * e;
}

// Store 8 consecutive K-elements k0..k0+7 (k0 a multiple of 8) of row r,
// rounded to the operand format; with SPLIT also the remainders (lo copy).
template <bool TF32, bool SPLIT>
__device__ __forceinline__ void put8(unsigned char* hi, unsigned char* lo, int R, int r, int k0, const float* v) {
  if constexpr (TF32) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const size_t off = opnd_off(R, 4, r, k0 + 4 * q);
      float4 hv, lv;
      hv.x = tc::to_tf32(v[4 * q + 0]);
      hv.y = tc::to_tf32(v[4 * q + 1]);
      hv.z = tc::to_tf32(v[4 * q + 2]);
      hv.w = tc::to_tf32(v[4 * q + 3]);
      *reinterpret_cast<float4*>(hi + off) = hv;
      if constexpr (SPLIT) {
        lv.x = tc::to_tf32(v[4 * q + 0] - hv.x);
        lv.y = tc::to_tf32(v[4 * q + 1] - hv.y);
        lv.z = tc::to_tf32(v[4 * q + 2] - hv.z);
        lv.w = tc::to_tf32(v[4 * q + 3] - hv.w);
        *reinterpret_cast<float4*>(lo + off) = lv;
      }
    }
  } else {
    const size_t off = opnd_off(R, 2, r, k0);
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]), h1 = __float2bfloat16_rn(v[2 * q + 1]);
      hw[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      if constexpr (SPLIT) {
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
        lw[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
      }
    }
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    if constexpr (SPLIT) *reinterpret_cast<uint4*>(lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

struct GemmArgs {
  LedArgs a;
  const unsigned char* cst;  // constant DFT factors
  unsigned char* scr;        // per-slot scratch
  int m, Wp, YT, ntile, X, nchunk, ks1, ks3, ks4, ns, kps;
  int ncta;                  // CTAs per LED: 2 (a cluster, one row tile each) or 1
  size_t aux;
  uint32_t S1, S2, S3, S4, SP, SA, SB, SU, stage;
  size_t c2_base, c3_base, c4_base, slot_bytes, o_phi, o_at, o_bg, o_au, o_spill;
};

// One contraction D (+)= A * B^T over ks K-steps; A: nA constant or data
// operands of 128 rows (one TMEM block each), B: data or constant of
// b_slice / 32 rows. hi copies at the given bases, lo copies lo bytes further.
struct Call {
  const unsigned char* A[2];
  uint32_t a_lo;
  int nA;
  const unsigned char* B;
  uint32_t b_lo, b_slice;
  int ks;
  uint32_t dcol[2];
  uint32_t id;
  int accum;
};

// Producer (one thread): bulk-copies groups of up to kps K-steps of A and B
// (one copy per operand and group: a group's slices are contiguous) into the
// stage ring, reusing a stage once the MMAs that read it have completed.
// q counts groups through the ring (the same count as the issuer's).
template <bool SPLIT>
__device__ bool gemm_produce(const Call& c, unsigned char* stages, uint32_t stage_bytes, int ns, int kps,
                             uint64_t* full, uint64_t* empty, uint32_t& q) {
  constexpr int F = SPLIT ? 2 : 1;
  const int ngrp = (c.ks + kps - 1) / kps;
  const uint32_t q0 = q;
  int issued = 0;
  bool ok = true;
  for (int gi = 0; gi < ngrp; ++gi) {
    const uint32_t Q = q0 + gi, s = Q % ns, u = Q / ns;
    if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, WAIT_NS)) {
      ok = false;
      break;
    }
    const int k0 = gi * kps, nk = min(kps, c.ks - k0);
    const uint32_t abytes = (uint32_t)nk * A_SLICE, bbytes = (uint32_t)nk * c.b_slice;
    unsigned char* st = stages + (size_t)s * stage_bytes;
    tc::mbar_expect_tx(&full[s], (uint32_t)(c.nA * F) * abytes + F * bbytes);
    for (int j = 0; j < c.nA; ++j) {
      tc::bulk_g2s(st + (size_t)(j * F) * kps * A_SLICE, c.A[j] + (size_t)k0 * A_SLICE, abytes, &full[s]);
      if (SPLIT)
        tc::bulk_g2s(st + (size_t)(j * F + 1) * kps * A_SLICE, c.A[j] + c.a_lo + (size_t)k0 * A_SLICE, abytes,
                     &full[s]);
    }
    unsigned char* sb = st + (size_t)(c.nA * F) * kps * A_SLICE;
    tc::bulk_g2s(sb, c.B + (size_t)k0 * c.b_slice, bbytes, &full[s]);
    if (SPLIT) tc::bulk_g2s(sb + (size_t)kps * c.b_slice, c.B + c.b_lo + (size_t)k0 * c.b_slice, bbytes, &full[s]);
    issued = gi + 1;
  }
  if (!ok)  // let the copies in flight land before anything is torn down
    for (int gi = issued > ns ? issued - ns : 0; gi < issued; ++gi) {
      const uint32_t Q = q0 + gi;
      tc::mbar_wait(&full[Q % ns], (Q / ns) & 1, WAIT_NS);
    }
  q = q0 + (uint32_t)ngrp;
  return ok;
}

// MMA issuer (one thread): waits for each stage, issues its MMAs (three per
// output block and K-step in the split forms), releases the stage; commits
// `done` at the end, also after a failed wait.
template <bool TF32, bool SPLIT>
__device__ bool gemm_issue(const Call& c, unsigned char* stages, uint32_t stage_bytes, int ns, int kps,
                           uint64_t* full, uint64_t* empty, uint64_t* done, uint32_t tbase, uint32_t& q) {
  constexpr int F = SPLIT ? 2 : 1;
  const int ngrp = (c.ks + kps - 1) / kps;
  const uint32_t q0 = q;
  bool ok = true;
  for (int gi = 0; gi < ngrp; ++gi) {
    const uint32_t Q = q0 + gi, s = Q % ns, u = Q / ns;
    if (!tc::mbar_wait(&full[s], u & 1, WAIT_NS)) {
      ok = false;
      break;
    }
    tc::fence_after_sync();
    const int k0 = gi * kps, nk = min(kps, c.ks - k0);
    const uint32_t sa = tc::smem_u32(stages + (size_t)s * stage_bytes);
    const uint32_t sbb = sa + (uint32_t)(c.nA * F * kps) * A_SLICE;
    for (int kk = 0; kk < nk; ++kk) {
      const uint64_t bh = tc::sdesc(sbb + kk * c.b_slice, 128, 256);
      const uint64_t bl = SPLIT ? tc::sdesc(sbb + (kps + kk) * c.b_slice, 128, 256) : 0;
      for (int j = 0; j < c.nA; ++j) {
        const uint64_t ah = tc::sdesc(sa + (uint32_t)(j * F * kps + kk) * A_SLICE, 128, 256);
        const uint32_t d = tbase + c.dcol[j];
        tc::mma<TF32>(d, ah, bh, c.id, (c.accum || k0 + kk > 0) ? 1u : 0u);
        if constexpr (SPLIT) {
          const uint64_t al = tc::sdesc(sa + (uint32_t)((j * F + 1) * kps + kk) * A_SLICE, 128, 256);
          tc::mma<TF32>(d, ah, bl, c.id, 1u);
          tc::mma<TF32>(d, al, bh, c.id, 1u);
        }
      }
    }
    tc::mma_commit(&empty[s]);
  }
  q = q0 + (uint32_t)ngrp;
  tc::mma_commit(done);
  return ok;
}

template <bool TF32, bool SPLIT>
__global__ void __launch_bounds__(GT, 1) gemm_led_kernel(const GemmArgs g) {
  constexpr uint32_t FMT = TF32 ? 2u : 1u;
  const LedArgs& a = g.a;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* stages = smem;
  // staging of per-pixel inputs: the O box [W][W] (column c contiguous in r),
  // or one tile-chunk of the image / dL/dI rows [YT][X + 4]
  float2* ob = reinterpret_cast<float2*>(smem + (size_t)g.ns * g.stage);
  float* ms = reinterpret_cast<float*>(ob);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)g.ns * g.stage + g.aux);
  uint64_t* empty = full + g.ns;
  uint64_t* done = empty + g.ns;
  volatile uint32_t* misc = reinterpret_cast<volatile uint32_t*>(done + 1);  // [0] TMEM base, [1] abort
  float* poly = const_cast<float*>(reinterpret_cast<volatile float*>(misc + 4));  // K[15] Dx[10] Dy[10]
  float* zmt = poly + 40;                                                        // [14 * 15] (+2 pad)
  float* red = zmt + 14 * 15 + 2;                                                // [8][NACC]
  double* dsum = reinterpret_cast<double*>(red + (GT / 32) * NACC);             // [16]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = quarter * 32 + lane;  // the TMEM lane (accumulator row) this thread reads
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
  const bool pair = g.ncta == 2;   // (uniform over the launch)
  const int rank = pair ? (int)cooperative_groups::this_cluster().block_rank() : 0;
  const int k = blockIdx.x / g.ncta;
  const int4 slot = a.slot[k];
  const int led = slot.x;
  if (led < 0 || led >= a.n_leds) {  // the same for both CTAs of a pair: no barrier is left waiting
    if (tid == 0 && rank == 0) atomicOr(a.err, DERR_INDEX);
    return;
  }
  const int m = g.m, N = a.N, h = a.h, W = a.W, Wp = g.Wp, YT = g.YT, X = g.X;
  for (int t = tid; t < 14 * 15; t += GT) zmt[t] = zern_mono_table()[t];
  if (warp == 0) {
    tc::tmem_alloc(const_cast<uint32_t*>(&misc[0]), 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < g.ns; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_fence_init();
    misc[1] = 0;
  }
  grid_dep_wait();    // O and the scalar parameters come from the previous update
  grid_dep_launch();  // (see the FFT form: the update reads O, m, v only after its own wait)
  float zc = 0.f;
  if (tid < 14) zc = a.sp[SP_ZERN + tid];
  const float zdef = a.sp[SP_DEFOCUS];
  const float gam = a.sp[SP_GAMMA + led];
  const float dly = a.sp[sp_offset(a.n_leds) + 2 * led];
  const float dlx = a.sp[sp_offset(a.n_leds) + 2 * led + 1];
  const PupilConst P{a.R, a.Rinv, a.inv_lambda, a.dk2, a.hard_edge};
  if (tid < 14) red[tid] = zc;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = misc[0];
  if (tid < 35) poly[tid] = theta_poly_entry_tab(red, zmt, tid);
  __syncthreads();

  unsigned char* scr = g.scr + ((size_t)k * g.ncta + rank) * g.slot_bytes;   // this CTA's operands
  unsigned char* phi = g.scr + (size_t)k * g.ncta * g.slot_bytes + g.o_phi;  // shared by a pair
  unsigned char* at = scr + g.o_at;
  unsigned char* bg = scr + g.o_bg;
  unsigned char* au = scr + g.o_au;
  float* spill = reinterpret_cast<float*>(scr + g.o_spill) + (size_t)row * 2 * Wp;
  const size_t col0 = (size_t)(N / 2 + slot.z - h);  // O column of box column 0 (column-major O)
  const int rowb = N / 2 + slot.y - h;               // O row of box row 0
  const float inv_m2 = 1.f / (float)(m * m);
  const float sg = sqrtf(gam);

  // O on a disk that contains the support for every admissible delta
  // (|delta| <= sqrt(2) * bound) -> ob[c][r], one cp.async group
  const float rs = (a.hard_edge ? a.R : a.R + 0.5f) + 1.41422f * FPM_OFFSET_BOUND_PX + 1e-3f;
  auto fetch_box = [&]() {
    for (int qq = tid; qq < W * W; qq += GT) {
      const int c = qq / W, r = qq - c * W;
      const float px = (float)(c - h), py = (float)(r - h);
      if (px * px + py * py <= rs * rs) tc::cp_async8(ob + qq, a.Ot + (col0 + c) * N + rowb + r);
    }
    tc::cp_async_commit();
  };
  // image (or dL/dI) rows of tile t, columns of chunk ch -> ms[row][X + 4]
  const int MS = X + 4;
  auto fetch_rows = [&](int t, int ch) {
    const float* src = a.mode == MODE_LOSS ? a.meas + (size_t)led * m * m
                     : a.mode == MODE_UPSTREAM ? a.dLdI + (size_t)k * m * m : nullptr;
    if (src)
      for (int qq = tid; qq < YT * (X / 4); qq += GT) {
        const int yl = qq / (X / 4), x4 = qq - yl * (X / 4);
        tc::cp_async16(ms + yl * MS + 4 * x4, src + (size_t)(t * YT + yl) * m + ch * X + 4 * x4);
      }
    tc::cp_async_commit();
  };
  fetch_box();
  tc::cp_async_wait_all();
  __syncthreads();

  // ---- Phi = O x M on the box, as the B operand of step 1 (rows c, K = [Re r | Im r]);
  // a pair builds half of the box columns each
  const int pc = pair ? Wp / 2 : Wp;
  for (int it = tid; it < pc * (Wp / 8); it += GT) {
    const int c = rank * pc + it % pc, r0 = (it / pc) * 8;
    const float qx = (float)(c - h) - dlx, qx2 = qx * qx;
    ColPoly cp;  // the aberration phase along column c
    col_poly(qx * P.Rinv, poly, cp);
    float re[8], im[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int r = r0 + e;
      float2 v = make_float2(0.f, 0.f);
      if (c < W && r < W) {
        const float qy = (float)(r - h) - dly, r2 = fmaf(qy, qy, qx2);
        float rad;
        const float A = pupil_amp_r2(r2, P, rad);
        if (A > 0.f) v = cmul(ob[c * W + r], pupil_col(qy, r2, A, P, cp, zdef));
      }
      re[e] = v.x;
      im[e] = v.y;
    }
    put8<TF32, SPLIT>(phi, phi + g.SP, Wp, c, r0, re);
    put8<TF32, SPLIT>(phi, phi + g.SP, Wp, c, Wp + r0, im);
  }

  if (pair) {  // the other half of Phi, written by the partner, before any bulk copy reads it
    tc::fence_proxy_async_global();
    cooperative_groups::this_cluster().sync();
  }

  uint32_t q = 0, ngemm = 0;  // ring position (threads 0 and 32), contractions so far
  // Run one contraction: every thread publishes its operand writes and its
  // finished TMEM reads; thread 32 streams the operands, thread 0 issues the
  // MMAs; all wait for the result.
  auto run = [&](const Call& c) -> bool {
    tc::fence_proxy_async_global();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {  // MMA issuer
      tc::fence_after_sync();
      if (!gemm_issue<TF32, SPLIT>(c, stages, g.stage, g.ns, g.kps, full, empty, done, tbase, q)) {
        misc[1] = 1;
        atomicOr(a.err, DERR_TIMEOUT);
      }
    } else if (tid == 32) {  // producer
      if (!gemm_produce<SPLIT>(c, stages, g.stage, g.ns, g.kps, full, empty, q)) {
        misc[1] = 1;
        atomicOr(a.err, DERR_TIMEOUT);
      }
    }
    if (!tc::mbar_wait(done, ngemm & 1, WAIT_NS)) {
      misc[1] = 1;
      atomicOr(a.err, DERR_TIMEOUT);
    }
    ++ngemm;
    tc::fence_after_sync();
    __syncthreads();
    return misc[1] == 0;
  };

  float acc_loss = 0.f, acc_g = 0.f;
  BoxAcc bacc;
  box_acc_zero(bacc);
  bool ok = true;
  const int t_lo = pair ? rank : 0, t_hi = pair ? rank + 1 : g.ntile;  // this CTA's row tiles
  for (int t = t_lo; t < t_hi && ok; ++t) {
    // ---- step 1: T = E Phi for the rows y of this tile (TMEM cols [0, Wp) Re, [128, 128 + Wp) Im)
    {
      Call c{};
      c.A[0] = g.cst + (size_t)(t * 2 + 0) * (SPLIT ? 2 : 1) * g.S1;
      c.A[1] = g.cst + (size_t)(t * 2 + 1) * (SPLIT ? 2 : 1) * g.S1;
      c.a_lo = g.S1;
      c.nA = 2;
      c.B = phi;
      c.b_lo = g.SP;
      c.b_slice = (uint32_t)Wp * 32;
      c.ks = g.ks1;
      c.dcol[0] = 0;
      c.dcol[1] = 128;
      c.id = tc::idesc(FMT, 128, Wp);
      c.accum = 0;
      if (!(ok = run(c))) break;
    }
    // T rows (one per thread) -> A operand of step 2 (K = [Re c | Im c])
    for (int c0 = half * (Wp / 2); c0 < (half + 1) * (Wp / 2); c0 += 8) {
      float re[8], im[8];
      tc::tmem_ld8(tbase + lane_off + (uint32_t)c0, re);
      tc::tmem_ld8(tbase + lane_off + 128u + (uint32_t)c0, im);
      put8<TF32, SPLIT>(at, at + g.SA, 128, row, c0, re);
      put8<TF32, SPLIT>(at, at + g.SA, 128, row, Wp + c0, im);
    }
    const int y = t * YT + row;
    const bool yvalid = row < YT;
    for (int ch = 0; ch < g.nchunk && ok; ++ch) {
      // ---- step 2: psi m^2 = T E^T for this chunk of columns (TMEM cols [256, 256 + X) Re, then Im)
      {
        Call c{};
        c.A[0] = at;
        c.a_lo = g.SA;
        c.nA = 1;
        c.B = g.cst + g.c2_base + (size_t)ch * (SPLIT ? 2 : 1) * g.S2;
        c.b_lo = g.S2;
        c.b_slice = (uint32_t)(2 * X) * 32;
        c.ks = g.ks1;
        c.dcol[0] = 256;
        c.id = tc::idesc(FMT, 128, 2 * X);
        c.accum = 0;
        if (a.mode != MODE_FORWARD) fetch_rows(t, ch);  // lands while step 2 runs
        ok = run(c);
        tc::cp_async_wait_all();
        __syncthreads();
        if (!ok) break;
      }
      // residual (Eq. 4-5) per pixel; g rows -> B operand of step 3 (K = [Re x | Im x])
      for (int x0 = half * (X / 2); x0 < (half + 1) * (X / 2); x0 += 8) {
        float re[8], im[8];
        tc::tmem_ld8(tbase + lane_off + 256u + (uint32_t)x0, re);
        tc::tmem_ld8(tbase + lane_off + 256u + (uint32_t)(X + x0), im);
        if (!yvalid) continue;
        const int xa = ch * X + x0;
        if (a.mode == MODE_FORWARD) {
          float Iv[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float pr = re[e] * inv_m2, pi = im[e] * inv_m2;
            Iv[e] = gam * (pr * pr + pi * pi);
          }
          float4* dst = reinterpret_cast<float4*>(a.I_out + ((size_t)k * m + y) * m + xa);
          dst[0] = make_float4(Iv[0], Iv[1], Iv[2], Iv[3]);
          dst[1] = make_float4(Iv[4], Iv[5], Iv[6], Iv[7]);
          continue;
        }
        const float4 v0 = *reinterpret_cast<const float4*>(ms + row * MS + x0);
        const float4 v1 = *reinterpret_cast<const float4*>(ms + row * MS + x0 + 4);
        const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        float gr[8], gi[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float2 gp = residual_pixel(make_float2(re[e] * inv_m2, im[e] * inv_m2), vv[e], a.mode, a.loss, gam,
                                           sg, acc_loss, acc_g);
          gr[e] = gp.x;
          gi[e] = gp.y;
        }
        put8<TF32, SPLIT>(bg, bg + g.SB, YT, row, x0, gr);
        put8<TF32, SPLIT>(bg, bg + g.SB, YT, row, X + x0, gi);
      }
      if (a.mode == MODE_FORWARD) continue;
      // ---- step 3: U^T += conj(E)^T g^T over this chunk (TMEM cols [0, YT) Re, [128, 128 + YT) Im)
      {
        Call c{};
        c.A[0] = g.cst + g.c3_base + (size_t)(ch * 2 + 0) * (SPLIT ? 2 : 1) * g.S3;
        c.A[1] = g.cst + g.c3_base + (size_t)(ch * 2 + 1) * (SPLIT ? 2 : 1) * g.S3;
        c.a_lo = g.S3;
        c.nA = 2;
        c.B = bg;
        c.b_lo = g.SB;
        c.b_slice = (uint32_t)YT * 32;
        c.ks = g.ks3;
        c.dcol[0] = 0;
        c.dcol[1] = 128;
        c.id = tc::idesc(FMT, 128, YT);
        c.accum = ch > 0;
        if (!(ok = run(c))) break;
      }
    }
    if (!ok || a.mode == MODE_FORWARD) continue;
    // U^T rows (box columns c, one per thread) -> A operand of step 4 (K = [Re y | Im y])
    for (int y0 = half * (YT / 2); y0 < (half + 1) * (YT / 2); y0 += 8) {
      float re[8], im[8];
      tc::tmem_ld8(tbase + lane_off + (uint32_t)y0, re);
      tc::tmem_ld8(tbase + lane_off + 128u + (uint32_t)y0, im);
      put8<TF32, SPLIT>(au, au + g.SU, 128, row, y0, re);
      put8<TF32, SPLIT>(au, au + g.SU, 128, row, YT + y0, im);
    }
    // ---- step 4: gPhi^T m^2 = U^T conj(E) over the rows of this tile (TMEM cols [256, 256 + Wp) Re, then Im)
    {
      Call c{};
      c.A[0] = au;
      c.a_lo = g.SU;
      c.nA = 1;
      c.B = g.cst + g.c4_base + (size_t)t * (SPLIT ? 2 : 1) * g.S4;
      c.b_lo = g.S4;
      c.b_slice = (uint32_t)(2 * Wp) * 32;
      c.ks = g.ks4;
      c.dcol[0] = 256;
      c.id = tc::idesc(FMT, 128, 2 * Wp);
      c.accum = 0;
      if (t == t_hi - 1) fetch_box();  // lands while step 4 runs
      ok = run(c);
      tc::cp_async_wait_all();
      __syncthreads();
      if (!ok) break;
    }
    if (pair) {  // the partner's half of the box rows, this tile's part, to this CTA's scratch row
      for (int r0 = (1 - rank) * (Wp / 2) + half * 8; r0 < (2 - rank) * (Wp / 2); r0 += 16) {
        float re[8], im[8];
        tc::tmem_ld8(tbase + lane_off + 256u + (uint32_t)r0, re);
        tc::tmem_ld8(tbase + lane_off + 256u + (uint32_t)(Wp + r0), im);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          spill[r0 + e] = re[e];
          spill[Wp + r0 + e] = im[e];
        }
      }
      continue;  // this CTA's own half is finished after the exchange below
    }
    // box column c = row: sum over tiles (in this thread's scratch row), then
    // the object and pupil-parameter gradients per box pixel
    const bool last = t == g.ntile - 1;
    const int c = row;
    for (int r0 = half * (Wp / 2); r0 < (half + 1) * (Wp / 2); r0 += 8) {
      float re[8], im[8];
      tc::tmem_ld8(tbase + lane_off + 256u + (uint32_t)r0, re);
      tc::tmem_ld8(tbase + lane_off + 256u + (uint32_t)(Wp + r0), im);
      if (g.ntile > 1) {
        if (t > 0)
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            re[e] += spill[r0 + e];
            im[e] += spill[Wp + r0 + e];
          }
        if (!last) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            spill[r0 + e] = re[e];
            spill[Wp + r0 + e] = im[e];
          }
          continue;
        }
      }
      if (c >= W) continue;
      const float2* Oc = ob + c * W;
      const float qx = (float)(c - h) - dlx, qx2 = qx * qx;
      ColPoly cp;  // the aberration phase along column c
      col_poly(qx * P.Rinv, poly, cp);
      float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // sum t(p) y^b over these pixels of the column
      float2* gb = a.gbox + ((size_t)k * W + c) * W;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int r = r0 + e;
        if (r >= W) continue;
        const float qy = (float)(r - h) - dly, r2 = fmaf(qy, qy, qx2);
        float2 out = make_float2(0.f, 0.f);
        float rad;
        const float A = pupil_amp_r2(r2, P, rad);
        if (A > 0.f)
          out = box_pixel_col(qy, qx, r2, A, rad, make_float2(re[e] * inv_m2, im[e] * inv_m2), Oc[r], P, cp, zdef,
                              S, bacc);
        gb[r] = out;
      }
      col_fold(cp, S, bacc);
    }
  }

  if (pair && a.mode != MODE_FORWARD) {
    // both CTAs reach this barrier whatever happened above (a wait that gave up
    // only skips work), then each adds the partner's part of its half of the
    // box rows and finishes their box gradients
    __threadfence();
    cooperative_groups::this_cluster().sync();
    const float* other = reinterpret_cast<const float*>(g.scr + ((size_t)k * 2 + (1 - rank)) * g.slot_bytes +
                                                        g.o_spill) + (size_t)row * 2 * Wp;
    const int c = row;
    const bool mine = ok && c < W;  // (the tensor-memory loads below are warp-wide: every lane runs them)
    const float2* Oc = ob + (mine ? c : 0) * W;
    const float qx = (float)(c - h) - dlx, qx2 = qx * qx;
    ColPoly cp;  // the aberration phase along column c
    col_poly(qx * P.Rinv, poly, cp);
    float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float2* gb = a.gbox + ((size_t)k * W + (mine ? c : 0)) * W;
    for (int r0 = rank * (Wp / 2) + half * 8; r0 < (rank + 1) * (Wp / 2); r0 += 16) {
      float re[8], im[8];
      tc::tmem_ld8(tbase + lane_off + 256u + (uint32_t)r0, re);
      tc::tmem_ld8(tbase + lane_off + 256u + (uint32_t)(Wp + r0), im);
      if (!mine) continue;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        re[e] += __ldcg(other + r0 + e);
        im[e] += __ldcg(other + Wp + r0 + e);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int r = r0 + e;
        if (r >= W) continue;
        const float qy = (float)(r - h) - dly, r2 = fmaf(qy, qy, qx2);
        float2 out = make_float2(0.f, 0.f);
        float rad;
        const float A = pupil_amp_r2(r2, P, rad);
        if (A > 0.f)
          out = box_pixel_col(qy, qx, r2, A, rad, make_float2(re[e] * inv_m2, im[e] * inv_m2), Oc[r], P, cp, zdef,
                              S, bacc);
        gb[r] = out;
      }
    }
    if (mine) col_fold(cp, S, bacc);
  }
  if (ok && a.mode != MODE_FORWARD)
    write_partials(acc_loss, acc_g, bacc, a.mode == MODE_LOSS && a.loss == 0, sg, red, reinterpret_cast<float*>(dsum), zmt,
                   a.part + ((size_t)k * g.ncta + rank) * NPART);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, 512);
  }
}

// ---------------------------------------------------------------- host side

float round_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}
float round_tf32(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= 0xFFFFE000u;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

// Write value v (FP64) at (r, k) of an R-row operand block: hi copy at hi, lo copy at lo.
void put_const(const GemmPlan& p, unsigned char* hi, unsigned char* lo, int R, int r, int k, double v) {
  const size_t off = opnd_off(R, p.e, r, k);
  const float hv = p.tf32 ? round_tf32((float)v) : round_bf16((float)v);
  const float lv = p.tf32 ? round_tf32((float)(v - (double)hv)) : round_bf16((float)(v - (double)hv));
  auto st = [&](unsigned char* dst, float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if (p.tf32) std::memcpy(dst + off, &u, 4);
    else {
      const uint16_t b = (uint16_t)(u >> 16);
      std::memcpy(dst + off, &b, 2);
    }
  };
  st(hi, hv);
  if (p.split) st(lo, lv);
}

template <bool TF32, bool SPLIT>
const void* kernel_of() {
  return (const void*)gemm_led_kernel<TF32, SPLIT>;
}
const void* kernel_for(const GemmPlan& p) {
  if (p.tf32) return p.split ? kernel_of<true, true>() : kernel_of<true, false>();
  return p.split ? kernel_of<false, true>() : kernel_of<false, false>();
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

int gemm_plan(int m, int W, int h, int prec, GemmPlan* p, const char** why) {
  *p = GemmPlan{};
  if (prec < FPM_PRECISION_BF16_GEMM || prec > FPM_PRECISION_TF32X3_GEMM) {
    *why = "unknown precision mode";
    return FPM_ERR_ARG;
  }
  if (m != 64 && m != 128 && m != 256) {
    *why = "the tensor-core DFT form needs m in {64, 128, 256}";
    return FPM_ERR_SHAPE;
  }
  const int Wp = (W + 15) / 16 * 16;
  if (Wp > 128) {
    *why = "the tensor-core DFT form needs a crop box of at most 128 px (pupil radius <= 61 px)";
    return FPM_ERR_SHAPE;
  }
  p->prec = prec;
  p->tf32 = prec == FPM_PRECISION_TF32_GEMM || prec == FPM_PRECISION_TF32X3_GEMM;
  p->split = prec == FPM_PRECISION_BF16X3_GEMM || prec == FPM_PRECISION_TF32X3_GEMM;
  p->e = p->tf32 ? 4 : 2;
  p->m = m;
  p->W = W;
  p->h = h;
  p->Wp = Wp;
  p->YT = m < 128 ? m : 128;
  p->ntile = m / p->YT;
  p->X = m < 128 ? m : 128;
  p->nchunk = m / p->X;
  p->ncta = p->ntile == 2 ? 2 : 1;  // one row tile per CTA of a pair
  const int KE = 32 / p->e;  // K elements per K-step
  p->ks1 = 2 * Wp / KE;
  p->ks3 = 2 * p->X / KE;
  p->ks4 = 2 * p->YT / KE;
  const size_t F = p->split ? 2 : 1;
  p->S1 = (size_t)p->ks1 * A_SLICE;
  p->S2 = (size_t)p->ks1 * (2 * p->X) * 32;
  p->S3 = (size_t)p->ks3 * A_SLICE;
  p->S4 = (size_t)p->ks4 * (2 * Wp) * 32;
  p->c2_base = (size_t)p->ntile * 2 * F * p->S1;
  p->c3_base = p->c2_base + (size_t)p->nchunk * F * p->S2;
  p->c4_base = p->c3_base + (size_t)p->nchunk * 2 * F * p->S3;
  p->const_bytes = p->c4_base + (size_t)p->ntile * F * p->S4;
  p->SP = (size_t)p->ks1 * Wp * 32;
  p->SA = (size_t)p->ks1 * A_SLICE;
  p->SB = (size_t)p->ks3 * p->YT * 32;
  p->SU = (size_t)p->ks4 * A_SLICE;
  p->o_phi = 0;
  p->o_at = round_up(p->o_phi + F * p->SP, 256);
  p->o_bg = round_up(p->o_at + F * p->SA, 256);
  p->o_au = round_up(p->o_bg + F * p->SB, 256);
  p->o_spill = round_up(p->o_au + F * p->SU, 256);
  p->slot_bytes = round_up(p->o_spill + (p->ntile > 1 ? (size_t)128 * 2 * Wp * sizeof(float) : 0), 1024);
  // bytes of one K-step of each contraction; the stage holds the largest
  const size_t st1 = F * (2 * A_SLICE + (size_t)Wp * 32), st2 = F * (A_SLICE + (size_t)2 * p->X * 32);
  const size_t st3 = F * (2 * A_SLICE + (size_t)p->YT * 32), st4 = F * (A_SLICE + (size_t)2 * Wp * 32);
  p->kps = p->split ? 1 : 2;  // K-steps per stage (one bulk copy per operand and stage)
  p->stage = round_up((size_t)p->kps * std::max(std::max(st1, st2), std::max(st3, st4)), 1024);
  p->aux = round_up(std::max((size_t)W * W * sizeof(float2), (size_t)p->YT * (p->X + 4) * sizeof(float)), 1024);
  const size_t misc = (2 * MAX_STAGES + 1) * 8 + 16 + sizeof(float) * (40 + 14 * 15 + 2 + (GT / 32) * NACC) +
                      sizeof(double) * 16;
  const size_t budget = 227 * 1024 - round_up(misc, 1024) - p->aux;
  p->ns = (int)std::min<size_t>(MAX_STAGES, budget / p->stage);
  if (p->ns < 2) {
    *why = "tensor-core DFT stages do not fit in shared memory";
    return FPM_ERR_SHAPE;
  }
  p->smem = (size_t)p->ns * p->stage + p->aux + misc;
  return FPM_OK;
}

std::vector<unsigned char> gemm_constants(const GemmPlan& p) {
  std::vector<unsigned char> buf(p.const_bytes, 0);
  const int m = p.m, Wp = p.Wp, W = p.W, h = p.h, YT = p.YT, X = p.X;
  const size_t F = p.split ? 2 : 1;
  // E(y, k) = exp(+2 pi i y k / m), angle reduced exactly in integers
  auto E = [&](int y, int kk, double* re, double* im) {
    long long t = ((long long)y * kk) % m;
    if (t < 0) t += m;
    const double ang = 2.0 * M_PI * (double)t / (double)m;
    *re = std::cos(ang);
    *im = std::sin(ang);
  };
  double er, ei;
  // step 1, A (rows y of tile t; K = [Re r | Im r]); block j = 0 real output, 1 imaginary
  for (int t = 0; t < p.ntile; ++t)
    for (int j = 0; j < 2; ++j) {
      unsigned char* hi = buf.data() + (size_t)(t * 2 + j) * F * p.S1;
      for (int yl = 0; yl < YT; ++yl)
        for (int kq = 0; kq < 2 * Wp; ++kq) {
          const int r = kq % Wp, part = kq / Wp;
          if (r >= W) continue;
          E(t * YT + yl, r - h, &er, &ei);
          const double v = j == 0 ? (part == 0 ? er : -ei) : (part == 0 ? ei : er);
          put_const(p, hi, hi + p.S1, 128, yl, kq, v);
        }
    }
  // step 2, B (rows: X real-output columns x, then X imaginary; K = [Re c | Im c])
  for (int ch = 0; ch < p.nchunk; ++ch) {
    unsigned char* hi = buf.data() + p.c2_base + (size_t)ch * F * p.S2;
    for (int n = 0; n < 2 * X; ++n)
      for (int kq = 0; kq < 2 * Wp; ++kq) {
        const int c = kq % Wp, part = kq / Wp, out = n / X;
        if (c >= W) continue;
        E(ch * X + n % X, c - h, &er, &ei);
        const double v = out == 0 ? (part == 0 ? er : -ei) : (part == 0 ? ei : er);
        put_const(p, hi, hi + p.S2, 2 * X, n, kq, v);
      }
  }
  // step 3, A (rows box column c; K = [Re x | Im x] of the chunk); conj(E)
  for (int ch = 0; ch < p.nchunk; ++ch)
    for (int j = 0; j < 2; ++j) {
      unsigned char* hi = buf.data() + p.c3_base + (size_t)(ch * 2 + j) * F * p.S3;
      for (int c = 0; c < W; ++c)
        for (int kq = 0; kq < 2 * X; ++kq) {
          const int part = kq / X;
          E(ch * X + kq % X, c - h, &er, &ei);
          const double v = j == 0 ? (part == 0 ? er : ei) : (part == 0 ? -ei : er);
          put_const(p, hi, hi + p.S3, 128, c, kq, v);
        }
    }
  // step 4, B (rows: Wp real-output box rows r, then Wp imaginary; K = [Re y | Im y] of tile t); conj(E)
  for (int t = 0; t < p.ntile; ++t) {
    unsigned char* hi = buf.data() + p.c4_base + (size_t)t * F * p.S4;
    for (int n = 0; n < 2 * Wp; ++n) {
      const int r = n % Wp, out = n / Wp;
      if (r >= W) continue;
      for (int kq = 0; kq < 2 * YT; ++kq) {
        const int part = kq / YT;
        E(t * YT + kq % YT, r - h, &er, &ei);
        const double v = out == 0 ? (part == 0 ? er : ei) : (part == 0 ? -ei : er);
        put_const(p, hi, hi + p.S4, 2 * Wp, n, kq, v);
      }
    }
  }
  return buf;
}

cudaError_t gemm_prepare(const GemmPlan& p) {
  const void* f = kernel_for(p);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

cudaError_t launch_led_gemm(const GemmPlan& p, const LedArgs& a, const unsigned char* consts,
                            unsigned char* scratch, cudaStream_t s, bool pdl) {
  GemmArgs g{};
  g.a = a;
  g.cst = consts;
  g.scr = scratch;
  g.m = p.m;
  g.Wp = p.Wp;
  g.YT = p.YT;
  g.ntile = p.ntile;
  g.X = p.X;
  g.nchunk = p.nchunk;
  g.ks1 = p.ks1;
  g.ks3 = p.ks3;
  g.ks4 = p.ks4;
  g.ns = p.ns;
  g.kps = p.kps;
  g.aux = p.aux;
  g.S1 = (uint32_t)p.S1;
  g.S2 = (uint32_t)p.S2;
  g.S3 = (uint32_t)p.S3;
  g.S4 = (uint32_t)p.S4;
  g.SP = (uint32_t)p.SP;
  g.SA = (uint32_t)p.SA;
  g.SB = (uint32_t)p.SB;
  g.SU = (uint32_t)p.SU;
  g.stage = (uint32_t)p.stage;
  g.c2_base = p.c2_base;
  g.c3_base = p.c3_base;
  g.c4_base = p.c4_base;
  g.slot_bytes = p.slot_bytes;
  g.o_phi = p.o_phi;
  g.o_at = p.o_at;
  g.o_bg = p.o_bg;
  g.o_au = p.o_au;
  g.o_spill = p.o_spill;
  g.ncta = p.ncta;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.B * p.ncta), 1, 1);
  cfg.blockDim = dim3(GT, 1, 1);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (p.ncta > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = (unsigned)p.ncta;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  if (p.tf32) {
    if (p.split) return cudaLaunchKernelEx(&cfg, gemm_led_kernel<true, true>, g);
    return cudaLaunchKernelEx(&cfg, gemm_led_kernel<true, false>, g);
  }
  if (p.split) return cudaLaunchKernelEx(&cfg, gemm_led_kernel<false, true>, g);
  return cudaLaunchKernelEx(&cfg, gemm_led_kernel<false, false>, g);
}

}  // namespace fpmk

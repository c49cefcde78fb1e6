// Measurement of the GPU's FP32 fused multiply-add throughput (the CUDA-core
// peak that the ALU roofline of the per-LED kernel is quoted against). Not a
// step of the method.
//
// Every thread runs NACC independent chains of fmaf for `iters` rounds (so
// each scheduler always has independent FMAs to issue), over a grid of
// `ctas_per_sm` CTAs of 256 threads per SM; the chains' results are written
// out so no FMA can be dropped. FLOPs = 2 * NACC * iters * threads.
#include <cuda_runtime.h>

#include "../../include/fpm.h"

namespace {

constexpr int NACC = 16;
constexpr int PROBE_NT = 256;

__global__ void __launch_bounds__(PROBE_NT) fma_probe_kernel(float* out, int iters, float a, float b) {
  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < NACC; ++i) acc[i] = fmaf(acc[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NACC; ++i) s += acc[i];
  out[(size_t)blockIdx.x * PROBE_NT + threadIdx.x] = s;
}

}  // namespace

extern "C" int fpm_probe_fp32_fma(int32_t iters, int32_t reps, double* tflops_out, double* ms_out) {
  if (iters < 1 || reps < 1 || !tflops_out) return FPM_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FPM_ERR_CUDA;
  const int ctas = sms * 8;  // 2048 threads per SM
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FPM_OK;
  float best = 0.f;
  if (cudaMalloc(&out, sizeof(float) * (size_t)ctas * PROBE_NT) != cudaSuccess) return FPM_ERR_OOM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = FPM_ERR_CUDA;
  }
  for (int r = 0; r <= reps && rc == FPM_OK; ++r) {  // round 0 warms up
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = FPM_ERR_CUDA;
    fma_probe_kernel<<<ctas, PROBE_NT, 0, st>>>(out, iters, 0.999999f, 1e-7f);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess)
      rc = FPM_ERR_CUDA;
    float ms = 0.f;
    if (rc == FPM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = FPM_ERR_CUDA;
    if (rc == FPM_OK && r > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (rc == FPM_OK) {
    const double flops = 2.0 * NACC * (double)iters * ctas * PROBE_NT;
    *tflops_out = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}

// Whole-field kernels, run once per job or per state transfer:
//  - the initial object of Section 2.3: sqrt of the centre-LED image,
//    bilinearly upsampled with low-res pixel r on high-res pixel s*r
//    (periodic boundary), zero phase;
//  - the centred object spectrum O = fftshift(fft2(o)) / s^2 (Eq. 1-2),
//    written in the engine's column-major layout;
//  - a tiled transpose between row-major (the ABI's layout) and column-major.
// The N-point transforms are radix-2 Stockham in shared memory, one CTA per
// row or column, with a twiddle table rounded from double precision.
#include "device.cuh"
#include "internal.h"

#include <algorithm>

namespace fpmk {

__global__ void upsample_centre_kernel(const float* __restrict__ I, int m, int s, float2* __restrict__ out) {
  const int N = m * s;
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y;
  if (X >= N || Y >= N) return;
  const int y0 = Y / s, x0 = X / s;
  const float wy = (float)(Y - y0 * s) / (float)s, wx = (float)(X - x0 * s) / (float)s;
  const int y1 = (y0 + 1) % m, x1 = (x0 + 1) % m;
  const float a00 = sqrtf(fmaxf(I[y0 * m + x0], 0.f)), a01 = sqrtf(fmaxf(I[y0 * m + x1], 0.f));
  const float a10 = sqrtf(fmaxf(I[y1 * m + x0], 0.f)), a11 = sqrtf(fmaxf(I[y1 * m + x1], 0.f));
  const float top = a00 * (1.f - wx) + a01 * wx;
  const float bot = a10 * (1.f - wx) + a11 * wx;
  out[(size_t)Y * N + X] = make_float2(top * (1.f - wy) + bot * wy, 0.f);
}

// In-block radix-2 Stockham FFT of n points between two shared buffers;
// returns the buffer holding the result. DIR = -1 forward, +1 inverse.
template <int DIR>
__device__ float2* block_fft(float2* a, float2* b, int n, const float2* __restrict__ tw) {
  for (int Ns = 1; Ns < n; Ns <<= 1) {
    for (int jj = threadIdx.x; jj < n / 2; jj += blockDim.x) {
      const int k = jj & (Ns - 1);
      const float2 u = a[jj];
      const float2 v = cmul(a[jj + n / 2], tw_dir<DIR>(tw[k * (n / (2 * Ns))]));
      const int base = (jj - k) * 2 + k;
      b[base] = cadd(u, v);
      b[base + Ns] = csub(u, v);
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  return a;
}

template <int DIR>
__global__ void fft_rows_kernel(float2* data, int N, const float2* __restrict__ tw) {
  extern __shared__ float2 sh[];
  float2* a = sh;
  float2* b = sh + N;
  float2* row = data + (size_t)blockIdx.x * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) a[i] = row[i];
  __syncthreads();
  float2* r = block_fft<DIR>(a, b, N, tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) row[i] = r[i];
}

// Column kx of the row-transformed array -> forward transform over rows ->
// centred spectrum column (kx + N/2) mod N, rows shifted by N/2, scaled.
__global__ void fft_cols_centre_kernel(const float2* __restrict__ rows, float2* __restrict__ Ot, int N,
                                       const float2* __restrict__ tw, float scale) {
  extern __shared__ float2 sh[];
  float2* a = sh;
  float2* b = sh + N;
  const int kx = blockIdx.x;
  for (int i = threadIdx.x; i < N; i += blockDim.x) a[i] = rows[(size_t)i * N + kx];
  __syncthreads();
  float2* r = block_fft<-1>(a, b, N, tw);
  float2* col = Ot + (size_t)((kx + N / 2) & (N - 1)) * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) col[(i + N / 2) & (N - 1)] = cscale(r[i], scale);
}

__global__ void transpose_kernel(const float2* __restrict__ in, float2* __restrict__ out, int N) {
  __shared__ float2 tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int y = by + i, x = bx + threadIdx.x;
    if (y < N && x < N) tile[i][threadIdx.x] = in[(size_t)y * N + x];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int x = bx + i, y = by + threadIdx.x;
    if (y < N && x < N) out[(size_t)x * N + y] = tile[threadIdx.x][i];
  }
}

// Measured amplitude sqrt(max(I, 0)) of the whole stack (the amplitude loss,
// Section 2.2, compares |psi| with it), computed once per load.
__global__ void amplitude_kernel(const float* I, float* amp, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    amp[i] = sqrtf(fmaxf(I[i], 0.f));
}

cudaError_t launch_amplitude(const float* I, float* amp, size_t n, cudaStream_t st) {
  const size_t blocks = std::min<size_t>((n + 255) / 256, 152 * 16);
  amplitude_kernel<<<(unsigned)blocks, 256, 0, st>>>(I, amp, n);
  return cudaGetLastError();
}

cudaError_t launch_upsample_centre(const float* I, int m, int s, float2* out, cudaStream_t st) {
  const int N = m * s;
  dim3 grid((N + 255) / 256, N);
  upsample_centre_kernel<<<grid, 256, 0, st>>>(I, m, s, out);
  return cudaGetLastError();
}

static cudaError_t fft_smem_attr(const void* fn, int N) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * N * sizeof(float2)));
}

cudaError_t launch_fft_rows(float2* data, int N, const float2* twN, int dir, cudaStream_t st) {
  const size_t smem = 2 * (size_t)N * sizeof(float2);
  cudaError_t e;
  if (dir < 0) {
    if ((e = fft_smem_attr((const void*)fft_rows_kernel<-1>, N)) != cudaSuccess) return e;
    fft_rows_kernel<-1><<<N, 256, smem, st>>>(data, N, twN);
  } else {
    if ((e = fft_smem_attr((const void*)fft_rows_kernel<1>, N)) != cudaSuccess) return e;
    fft_rows_kernel<1><<<N, 256, smem, st>>>(data, N, twN);
  }
  return cudaGetLastError();
}

cudaError_t launch_fft_cols_centre(const float2* rows, float2* Ot, int N, const float2* twN, float scale,
                                   cudaStream_t st) {
  const size_t smem = 2 * (size_t)N * sizeof(float2);
  cudaError_t e = fft_smem_attr((const void*)fft_cols_centre_kernel, N);
  if (e != cudaSuccess) return e;
  fft_cols_centre_kernel<<<N, 256, smem, st>>>(rows, Ot, N, twN, scale);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const float2* in, float2* out, int N, cudaStream_t st) {
  dim3 grid((N + 31) / 32, (N + 31) / 32);
  transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, out, N);
  return cudaGetLastError();
}

}  // namespace fpmk

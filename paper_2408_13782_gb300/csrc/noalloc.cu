// Allocation-free gradient call (fpm_gradients_static in include/fpm.h).
//
// Who needs it: callers that must not call cudaMalloc - for example code that
// runs while a host framework owns the device memory pool (an allocation
// would bypass or fragment it, or is forbidden outright), or a real-time
// acquisition loop in which an allocation can block for an unbounded time.
// They pass their own device buffers for every input and output; the
// intermediates of the per-LED kernel (per-LED gradient boxes, per-LED FP64
// partials, batch slots, column spans, twiddles, error flag) live in one fixed array,
// g_static_scratch, declared below. Every GPU that loads this library holds
// that array until the process exits.
//
// The array is shared by all calls on a device and keeps the last call's
// contents; each call clears what must start at zero (the error flag) and
// overwrites the rest. Calls whose device work overlaps - on two streams, or
// from two host threads - race on it.
//
// The address of the array is obtained on the host with cudaGetSymbolAddress
// once per device (in host code the symbol itself is only a host-side
// stand-in, not a device address), on the first call made with that device
// current. That first call also sets the kernels' shared-memory attributes,
// reads the device's shared-memory limit and writes the transform twiddles
// into the array, so it should be made before any stream capture. Every call
// copies its batch tables from host memory, so a call on a stream that is
// being captured is refused.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fpm.h"
#include "internal.h"

using namespace fpmk;

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[FPM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
bool g_ready[kMaxDevices] = {};
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_smem_optin[kMaxDevices] = {};
int fail_static(int code, const std::string& msg) {
  set_unbound_error(msg.c_str());  // reported by fpm_last_error(NULL)
  return code;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Cluster size used by this call for low-res side m: the portable sizes.
int static_cluster(int m) { return m == 256 ? 8 : led_cluster_size(m); }

// The twiddle tables tw_m[t] = exp(-2 pi i t / m) for m = 32, 64, 128, 256,
// written once per device at the start of the array: offset of table m.
constexpr int kTwSizes[4] = {32, 64, 128, 256};
size_t tw_offset(int m) {
  size_t o = 0;
  for (int q = 0; q < 4 && kTwSizes[q] != m; ++q) o += sizeof(float2) * kTwSizes[q];
  return o;
}
constexpr size_t kTwBytes = sizeof(float2) * (32 + 64 + 128 + 256);

// Once per device: the array's device address, the kernels' attributes, the
// device's opt-in shared memory per block, and the twiddle tables.
int setup_device(int dev, unsigned char** out, int* smem_optin) {
  std::lock_guard<std::mutex> lk(g_setup_mutex);
  if (dev < 0 || dev >= kMaxDevices) return fail_static(FPM_ERR_CUDA, "device ordinal out of range");
  if (!g_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
      return fail_static(FPM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess)
      return fail_static(FPM_ERR_CUDA, std::string("device attribute: ") + cudaGetErrorString(e));
    // the attributes do not depend on the box width (each launch asks for the
    // shared memory its box needs; a call whose box does not fit is rejected)
    for (int m : {32, 64, 128, 256}) {
      e = led_prepare(m, static_cluster(m), 1);
      if (e != cudaSuccess)
        return fail_static(FPM_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    }
    e = update_prepare();
    if (e != cudaSuccess)
      return fail_static(FPM_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    std::vector<float2> tw(kTwBytes / sizeof(float2));
    size_t k = 0;
    for (int m : kTwSizes)
      for (int i = 0; i < m; ++i, ++k) {
        const double a = -2.0 * M_PI * (double)i / (double)m;
        tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
      }
    e = cudaMemcpy(p, tw.data(), kTwBytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail_static(FPM_ERR_CUDA, std::string("twiddles: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = (unsigned char*)p;
    g_smem_optin[dev] = optin;
    g_ready[dev] = true;
  }
  *out = g_scratch_ptr[dev];
  *smem_optin = g_smem_optin[dev];
  return FPM_OK;
}

// Device (or managed) memory of device dev.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" int fpm_gradients_static(const fpm_geometry* g, float R, int32_t upsample, const float* O_t,
                                    const float* params, const float* stack, const int32_t* idx, int32_t B,
                                    int32_t loss, float* g_object_t, float* g_params, double* loss_out,
                                    int32_t* err_out, void* cuda_stream) {
  // ---- arguments (host-side checks only; nothing is allocated) ----
  if (!g || !g->led_offset || !O_t || !params || !stack || !idx || !g_object_t || !g_params || !loss_out)
    return fail_static(FPM_ERR_ARG, "null argument");
  const int m = g->m, n = g->n_leds;
  if (led_cluster_size(m) == 0 || m == 512)
    return fail_static(FPM_ERR_SHAPE, "m not in {32, 64, 128, 256}");
  if (upsample < 1 || (long long)m * upsample > 8192 || (upsample & (upsample - 1)))
    return fail_static(FPM_ERR_SHAPE, "upsample must be a power of two with m * upsample <= 8192");
  if (n < 1 || n > 1024) return fail_static(FPM_ERR_SHAPE, "n_leds outside [1, 1024]");
  if (!(R > 0.f) || !(g->lambda_um > 0.f) || !(g->dk_per_um > 0.f))
    return fail_static(FPM_ERR_ARG, "radius, wavelength and spectral bin must be positive");
  if (g->pupil_edge != FPM_EDGE_AA && g->pupil_edge != FPM_EDGE_HARD)
    return fail_static(FPM_ERR_ARG, "unknown pupil edge");
  if (loss != FPM_LOSS_AMPLITUDE && loss != FPM_LOSS_INTENSITY) return fail_static(FPM_ERR_ARG, "unknown loss");
  if (B < 1 || B > n || B > MAX_BATCH) return fail_static(FPM_ERR_SHAPE, "batch size outside [1, n_leds]");
  const int N = m * upsample;
  const int h = (int)std::floor((double)R + 0.5 + std::sqrt(2.0) * FPM_OFFSET_BOUND_PX) + 1;
  const int W = 2 * h + 1;
  if (2 * h >= m) return fail_static(FPM_ERR_SHAPE, "pupil box does not fit the low-res window (2h >= m)");
  if ((double)(R + 2.f) * g->dk_per_um * g->lambda_um >= 1.0)
    return fail_static(FPM_ERR_SHAPE, "pupil reaches evanescent frequencies");
  std::vector<int> seen(n, 0);
  for (int b = 0; b < B; ++b) {
    if (idx[b] < 0 || idx[b] >= n) return fail_static(FPM_ERR_RANGE, "LED index outside [0, n_leds)");
    if (seen[idx[b]]++) return fail_static(FPM_ERR_RANGE, "LED index repeated in the batch");
  }
  // LED tables and the update region (host, small)
  std::vector<int2> nint(n);
  std::vector<int2> span(N, make_int2(N, 0));
  int lo_x = N, hi_x = -1;
  for (int i = 0; i < n; ++i) {
    const double r = g->led_offset[2 * i], c = g->led_offset[2 * i + 1];
    if (!std::isfinite(r) || !std::isfinite(c)) return fail_static(FPM_ERR_ARG, "non-finite LED offset");
    const int ri = (int)std::nearbyint(r), ci = (int)std::nearbyint(c);
    nint[i] = make_int2(ri, ci);
    const int r0 = N / 2 + ri - h, c0 = N / 2 + ci - h;
    if (r0 < 0 || c0 < 0 || r0 + W > N || c0 + W > N)
      return fail_static(FPM_ERR_SHAPE, "an LED crop box leaves the high-res spectrum");
    for (int x = c0; x < c0 + W; ++x) {
      span[x].x = std::min(span[x].x, r0);
      span[x].y = std::max(span[x].y, r0 + W);
    }
    lo_x = std::min(lo_x, c0);
    hi_x = std::max(hi_x, c0 + W);
  }
  // ---- layout of the static array; reject what does not fit ----
  const size_t o_span = align256(kTwBytes);
  const size_t o_slot = align256(o_span + sizeof(int2) * N);
  const size_t o_flags = align256(o_slot + sizeof(int4) * B);  // int err, then a double sink
  const size_t o_part = align256(o_flags + 16);
  const size_t o_box = align256(o_part + sizeof(double) * (size_t)B * static_cluster(m) * NPART);
  const size_t need = o_box + sizeof(float2) * (size_t)B * W * W;
  if (need > FPM_STATIC_SCRATCH_BYTES)
    return fail_static(FPM_ERR_SHAPE, "this batch needs " + std::to_string(need) +
                                          " bytes of scratch; the static array holds " +
                                          std::to_string((size_t)FPM_STATIC_SCRATCH_BYTES) +
                                          " (reduce the batch size or the pupil radius)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_static(FPM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess)
    return fail_static(FPM_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone)
    return fail_static(FPM_ERR_STATE, "the stream is being captured; this call copies host tables on every call "
                                      "and cannot be recorded");
  for (const void* p : {(const void*)O_t, (const void*)params, (const void*)stack, (const void*)g_object_t,
                        (const void*)g_params, (const void*)loss_out})
    if (!on_device(p, dev)) return fail_static(FPM_ERR_ARG, "inputs and outputs must be memory of the current device");
  if (err_out && !on_device(err_out, dev))
    return fail_static(FPM_ERR_ARG, "err_out must be memory of the current device");
  unsigned char* base = nullptr;
  int optin = 0;
  int rc = setup_device(dev, &base, &optin);
  if (rc) return rc;
  const int C = static_cluster(m);
  if (led_smem_bytes(m, C, W) > (size_t)optin)
    return fail_static(FPM_ERR_SHAPE, "pupil box too wide for this device's shared memory");

  float2* d_tw = (float2*)(base + tw_offset(m));
  int2* d_span = (int2*)(base + o_span);
  int4* d_slot = (int4*)(base + o_slot);
  int* d_err = (int*)(base + o_flags);
  double* d_sink = (double*)(base + o_flags + 8);
  double* d_part = (double*)(base + o_part);
  float2* d_box = (float2*)(base + o_box);
#define CKS(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail_static(FPM_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)
  std::vector<int4> slots(B);
  for (int b = 0; b < B; ++b) slots[b] = make_int4(idx[b], nint[idx[b]].x, nint[idx[b]].y, 0);
  CKS(cudaMemcpyAsync(d_span, span.data(), sizeof(int2) * N, cudaMemcpyHostToDevice, st));
  CKS(cudaMemcpyAsync(d_slot, slots.data(), sizeof(int4) * B, cudaMemcpyHostToDevice, st));
  CKS(cudaMemsetAsync(d_err, 0, 16, st));
  CKS(cudaMemsetAsync(g_object_t, 0, sizeof(float2) * (size_t)N * N, st));

  LedArgs a{};
  a.Ot = (const float2*)O_t;
  a.meas = stack;
  a.sp = params;
  a.slot = d_slot;
  a.gbox = d_box;
  a.part = d_part;
  a.tw = d_tw;
  a.N = N;
  a.n_leds = n;
  a.B = B;
  a.h = h;
  a.W = W;
  a.R = R;
  a.Rinv = 1.f / R;
  a.inv_lambda = 1.f / g->lambda_um;
  a.dk2 = g->dk_per_um * g->dk_per_um;
  a.hard_edge = g->pupil_edge == FPM_EDGE_HARD;
  a.loss = loss;
  a.mode = MODE_LOSS;
  a.err = d_err;
  CKS(launch_led(m, C, a, st, false));

  UpdArgs u{};
  u.gbox = d_box;
  u.part = d_part;
  u.slot = d_slot;
  u.span = d_span;
  u.x_lo = lo_x;
  u.n_cols = hi_x - lo_x;
  u.N = N;
  u.n_leds = n;
  u.B = B;
  u.C = C;
  u.h = h;
  u.W = W;
  u.b1 = 0.9f;
  u.b2 = 0.999f;
  u.eps = 1e-8f;
  u.offset_bound = FPM_OFFSET_BOUND_PX;
  u.coef = nullptr;
  u.loss_slot = loss_out;
  u.epoch_loss = d_sink;
  u.err = d_err;
  u.assemble = 1;
  u.g_obj = (float2*)g_object_t;
  u.g_sc = g_params;
  CKS(launch_update(u, st, false));
  if (err_out) CKS(cudaMemcpyAsync(err_out, d_err, sizeof(int), cudaMemcpyDeviceToDevice, st));
#undef CKS
  return FPM_OK;
}

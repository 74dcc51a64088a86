// pond_checks.cu -- measurement and self-check entry points (not steps of the
// method): the FMA throughput of this GPU, the denominator of the step
// kernels' roofline, and device-side checks of the step kernels' own
// arithmetic helpers against CUDA's correctly rounded operations.
#include <cuda_runtime.h>

#include <algorithm>

#include "pond.h"
#include "pond_checks.h"
#include "pond_kernels.cuh"

namespace {

// CH independent multiply-add chains per thread, 16 rounds per loop trip:
// enough independent work per warp to cover the pipe latency, nothing else in
// the loop.  The sum of the chains is stored only if it equals a value it
// cannot take (x stays near b/(1-a)), so the chains stay live.
template <typename R, int CH>
__global__ void __launch_bounds__(256) fma_peak_kernel(R *sink, long long trips, R a, R b) {
  R x[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) x[i] = R(threadIdx.x + i) * R(1e-3);
  for (long long t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < CH; ++i) x[i] = fma(x[i], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int i = 0; i < CH; ++i) s += x[i];
  if (sink != nullptr && s == R(-1.25)) sink[blockIdx.x] = s;
}

// one timed launch of `trips` loop trips on stream st; false on a CUDA error
template <typename R, int CH>
bool time_fma(cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int grid, long long trips, float *ms) {
  if (cudaEventRecord(e0, st) != cudaSuccess) return false;
  fma_peak_kernel<R, CH><<<grid, 256, 0, st>>>(nullptr, trips, R(0.9999999), R(1e-7));
  return cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
}

// The grid holds as many 256-thread CTAs as are resident on every SM.  The
// loop is lengthened until one launch lasts min_seconds / 5; the best of five
// launches of that length is kept.
template <typename R, int CH>
pond_status fma_peak(double min_seconds, double *tflops, double *ms_out) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<R, CH>, 256, 0) !=
          cudaSuccess) {
    (void)cudaGetLastError();
    return POND_E_CUDA;
  }
  const int grid = sms * std::max(per_sm, 1);
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  const double target_ms = 1e3 * min_seconds / 5.0;
  long long trips = 64;
  float ms = 0.f;
  double best_rate = 0.0, best_ms = 0.0;
  ok = ok && time_fma<R, CH>(st, e0, e1, grid, trips, &ms);  // first launch: warm-up
  for (int k = 0; ok && k < 24 && ms < target_ms; ++k) {
    trips = (long long)(trips * std::min(8.0, 1.25 * target_ms / std::max((double)ms, 1e-3))) + 1;
    ok = time_fma<R, CH>(st, e0, e1, grid, trips, &ms);
  }
  for (int k = 0; ok && k < 5; ++k) {
    ok = time_fma<R, CH>(st, e0, e1, grid, trips, &ms);
    const double rate = 2.0 * CH * 16.0 * (double)trips * 256.0 * grid / (ms * 1e-3) / 1e12;
    if (ok && rate > best_rate) { best_rate = rate; best_ms = ms; }
  }
  if (!ok) (void)cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (!ok) return POND_E_CUDA;
  if (tflops) *tflops = best_rate;
  if (ms_out) *ms_out = best_ms;
  return POND_OK;
}

__global__ void check_reciprocal_kernel(const double *y, double *r, double *r_ref, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = pond::rcp_nr1(y[i]);
  r_ref[i] = __drcp_rn(y[i]);
}

__global__ void check_vanleer_kernel(const double *x, const double *y, double *l, double *l_ref,
                                     long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = x[i], b = y[i];
  l[i] = pond::limit(a, b, pond::LIM_VANLEER);
  const double p = a * b;
  l_ref[i] = p > 0.0 ? p / (a + b) : 0.0;
}

bool launch_ok(long long n) { return n >= 0 && n <= (1LL << 31); }

}  // namespace

extern "C" pond_status pond_measure_fma_peak(int32_t precision, double min_seconds, double *tflops,
                                             double *ms) {
  if (!(min_seconds > 0.0) || min_seconds > 60.0) return POND_E_INVAL;
  if (precision == POND_FP64) return fma_peak<double, 8>(min_seconds, tflops, ms);
  if (precision == POND_FP32_MIXED) return fma_peak<float, 16>(min_seconds, tflops, ms);
  return POND_E_INVAL;
}

extern "C" pond_status pond_check_reciprocal(const double *y, double *r, double *r_ref, int64_t n,
                                             void *stream) {
  if (!launch_ok(n) || (n > 0 && (!y || !r || !r_ref))) return POND_E_INVAL;
  if (n == 0) return POND_OK;
  check_reciprocal_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(y, r, r_ref, n);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return POND_E_CUDA;
  }
  return POND_OK;
}

extern "C" pond_status pond_check_vanleer(const double *x, const double *y, double *l, double *l_ref,
                                          int64_t n, void *stream) {
  if (!launch_ok(n) || (n > 0 && (!x || !y || !l || !l_ref))) return POND_E_INVAL;
  if (n == 0) return POND_OK;
  check_vanleer_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, l, l_ref, n);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return POND_E_CUDA;
  }
  return POND_OK;
}

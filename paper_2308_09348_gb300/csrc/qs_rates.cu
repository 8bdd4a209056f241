// qs_rates.cu -- unit-rate probe of the pipes the kernels are bound by
// (qs_unit_rates): FP32 FMA, MUFU lg2 / ex2 / rcp (the PTX .approx forms the
// FP32 path issues) and FP64 FMA, as operations per SM per clock.
#include "qscatter.h"
#include "qs_host.hpp"

#include <cuda_runtime.h>

namespace qs {
namespace {

// Eight independent chains per thread, 16 steps unrolled.
__global__ void k_rate_fma(float* out, int iters) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-6f + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], 0.999999f, 1e-7f);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed f32x2 FMA (the instruction the FP32 phase integration issues):
// eight independent float2 chains per thread, 16 steps unrolled; each
// instruction is two lane-operations.
__global__ void k_rate_fma2(float* out, int iters) {
  float2 a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = make_float2(threadIdx.x * 1e-6f + k, k + 0.5f);
  const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], m, c);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// OP: 0 lg2, 1 ex2, 2 rcp; each followed by one FADD to stay in range.
template <int OP>
__global__ void k_rate_mufu(float* out, int iters) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.5f + threadIdx.x * 1e-6f + k * 0.01f;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float y;
        if (OP == 0) asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
        else if (OP == 1) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
        else asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
        a[k] = y + 1.25f;
      }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_rate_dfma(double* out, int iters) {
  double a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = threadIdx.x * 1e-6 + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = fma(a[k], 0.999999, 1e-7);
  out[blockIdx.x * blockDim.x + threadIdx.x] = a[0] + a[1] + a[2] + a[3];
}

}  // namespace
}  // namespace qs

// rates[0..4]: FP32 FMA, lg2, ex2, rcp, FP64 FMA per SM per clock at the
// device's maximum SM clock; rates[5]: the SM count; rates[6]: that clock in
// MHz; rates[7]: packed f32x2 FMA lane-operations (two per instruction) per
// SM per clock.  The kernels run on `stream` and are waited for; d_scratch: device
// memory of at least qs_unit_rates_scratch_bytes() bytes.
extern "C" size_t qs_unit_rates_scratch_bytes(void) {
  int sms = 0;
  if (qs::detail::device_sms(&sms) != QS_OK) return 0;
  return (size_t)sms * 8 * 256 * sizeof(double);
}

extern "C" int32_t qs_unit_rates(double* rates, void* d_scratch, size_t scratch_bytes,
                                 void* stream) {
  using namespace qs;
  int dev = 0, sms = 0, khz = 0;
  if (!rates || !d_scratch) return QS_ERR_INVALID_ARG;
  if (cudaGetDevice(&dev) != cudaSuccess || detail::device_sms(&sms) != QS_OK ||
      cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
    return detail::cuda_fail();
  const int blocks = sms * 8, threads = 256;
  if (scratch_bytes < (size_t)blocks * threads * sizeof(double)) return QS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* fo = static_cast<float*>(d_scratch);
  double* dd = static_cast<double*>(d_scratch);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return detail::cuda_fail();
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return detail::cuda_fail();
  }
  const double clk = (double)khz * 1e3;
  int32_t status = QS_OK;
  auto timed = [&](auto launch, int iters, double per_iter, double* dst) {
    launch(4);                                     // warm-up
    cudaEventRecord(a, st);
    launch(iters);
    cudaEventRecord(b, st);
    float ms = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess) {
      status = QS_ERR_CUDA;
      return;
    }
    const double ops = (double)blocks * threads * iters * per_iter;
    *dst = ops / (ms * 1e-3) / sms / clk;
  };
  timed([&](int it) { k_rate_fma<<<blocks, threads, 0, st>>>(fo, it); }, 4000, 128.0, &rates[0]);
  timed([&](int it) { k_rate_mufu<0><<<blocks, threads, 0, st>>>(fo, it); }, 1000, 128.0, &rates[1]);
  timed([&](int it) { k_rate_mufu<1><<<blocks, threads, 0, st>>>(fo, it); }, 1000, 128.0, &rates[2]);
  timed([&](int it) { k_rate_mufu<2><<<blocks, threads, 0, st>>>(fo, it); }, 1000, 128.0, &rates[3]);
  timed([&](int it) { k_rate_dfma<<<blocks, threads, 0, st>>>(dd, it); }, 100, 64.0, &rates[4]);
  timed([&](int it) { k_rate_fma2<<<blocks, threads, 0, st>>>(fo, it); }, 2000, 256.0, &rates[7]);
  rates[5] = sms;
  rates[6] = (double)khz / 1e3;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (status != QS_OK) (void)cudaGetLastError();
  return status;
}

// qs_pw.cu -- plane-wave reconstruction (qs_pw_reconstruct).
//
// K9 k_pw_reconstruct  out[s][b] = sum_k hist[s][k] pw[k][b]: the 3D spectrum
//                      of each of n_shots beams from its a_eff histogram and a
//                      table of plane-wave spectra at the a-bin centres.
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348, Sec. 3.2, Eq. 5.
#include "qscatter.h"
#include "qs_host.hpp"

#include <cuda_runtime.h>

namespace qs {

// One CTA: kPwShots shots x blockDim.x bins.  Each thread walks k in
// ascending order (the same order for every launch shape), reading its
// pw[k][b] once for all the CTA's shots; the histogram values are
// broadcast loads.
constexpr int kPwShots = 8;

__global__ void __launch_bounds__(256) k_pw_reconstruct(int n_shots, int n_a, int n_bins,
                                                        const double* __restrict__ hist,
                                                        const double* __restrict__ pw,
                                                        double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int s0 = blockIdx.y * kPwShots;
  if (b >= n_bins) return;
  double acc[kPwShots];
#pragma unroll
  for (int j = 0; j < kPwShots; ++j) acc[j] = 0.0;
  for (int k = 0; k < n_a; ++k) {
    const double v = __ldg(pw + (size_t)k * n_bins + b);
#pragma unroll
    for (int j = 0; j < kPwShots; ++j)
      if (s0 + j < n_shots) acc[j] = fma(__ldg(hist + (size_t)(s0 + j) * n_a + k), v, acc[j]);
  }
#pragma unroll
  for (int j = 0; j < kPwShots; ++j)
    if (s0 + j < n_shots) out[(size_t)(s0 + j) * n_bins + b] = acc[j];
}

}  // namespace qs

using namespace qs;

extern "C" int32_t qs_pw_reconstruct(int32_t n_shots, int32_t n_a, int32_t n_bins,
                                     const double* d_hist, const double* d_pw, double* d_out,
                                     void* stream) {
  if (n_shots < 0 || n_a < 0 || n_bins < 0) return QS_ERR_INVALID_ARG;
  if (n_shots == 0 || n_bins == 0) return QS_OK;
  if (!d_out || (n_a > 0 && (!d_hist || !d_pw))) return QS_ERR_INVALID_ARG;
  const int gy = (n_shots + kPwShots - 1) / kPwShots;
  if (gy > 65535) return QS_ERR_INVALID_ARG;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  dim3 grid((n_bins + 255) / 256, gy);
  k_pw_reconstruct<<<grid, 256, 0, cs>>>(n_shots, n_a, n_bins, d_hist, d_pw, d_out);
  return cudaGetLastError() == cudaSuccess ? QS_OK : detail::cuda_fail();
}

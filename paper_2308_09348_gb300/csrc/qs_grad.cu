// qs_grad.cu -- adjoint of the beam phase-space integration (qs_scatter_grad).
//
// K3 k_grad         per sample: recompute the forward with two tangents
//                   (d/d a_eff, d/d gamma0) carried through the discretised
//                   phase integration, form the sample's share of dL/d(outputs)
//                   from the upstream gradient, chain-rule it to the 8
//                   parameters, reduce per CTA in a fixed order (the device
//                   pieces are in qs_grad.cuh).
// K4 k_grad_final   one CTA: per-CTA partials summed in CTA order.
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348 -- Eqs. 2, 3, 6, 8 and
// the reconstruction use of Sec. 6.
#include "qscatter.h"
#include "qs_device.cuh"
#include "qs_grad.cuh"
#include "qs_host.hpp"

#include <cmath>
#include <type_traits>

namespace qs {

// Largest smoothed spectrum whose upstream gradient is staged in shared
// memory (FP32 path); larger ones are read from global memory.
constexpr int kGradStageBins = 8192;

// Shared memory of k_grad: the phase table (the quantum model or the
// per-cell focus), FP32 cycle-resolved chi's node-pair Hermite tables, the
// reduction scratch and (FP32) the staged upstream spectrum gradient.
template <typename T, bool QFP, int VAR>
__host__ __device__ constexpr bool grad_has_table() { return QFP || (VAR & kVarCell) != 0; }
template <typename T, int VAR>
__host__ __device__ constexpr size_t grad_cyc_bytes() {
  return (sizeof(T) == 4 && (VAR & kVarCycle) != 0) ? (size_t)2 * kCycN * sizeof(float4) : 0;
}

template <typename T, bool QFP, int VAR>
__global__ void __launch_bounds__(VAR == 0 ? 512 : 256)
    k_grad(const Params p, const qs_moments* __restrict__ mom, const double* __restrict__ dLdm,
           const double* __restrict__ dLdS) {
  using TT = typename Tab<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  TT* tab = reinterpret_cast<TT*>(smem);
  const size_t tab_bytes =
      grad_has_table<T, QFP, VAR>() ? (((size_t)p.n_phase * sizeof(TT) + 15) & ~(size_t)15) : 0;
  float4* cA = reinterpret_cast<float4*>(smem + tab_bytes);
  const size_t cyc_bytes = grad_cyc_bytes<T, VAR>();
  double* red = reinterpret_cast<double*>(smem + tab_bytes + cyc_bytes);
  T* sdS = reinterpret_cast<T*>(smem + tab_bytes + cyc_bytes +
                                (size_t)(blockDim.x >> 5) * kNumGrad * sizeof(double));
  if (grad_has_table<T, QFP, VAR>())
    for (int j = threadIdx.x; j < p.n_phase; j += blockDim.x) table_entry(p, j, tab);
  if constexpr (grad_cyc_bytes<T, VAR>() > 0) {
    // node-pair tables {G_n, dG_n, G_n+1, dG_n+1}, then {H_n, dH_n, H_n+1, dH_n+1}
    for (int j = threadIdx.x; j < kCycN - 1; j += blockDim.x) {
      const float4 a = p.cyc_a[j], b = p.cyc_a[j + 1];
      cA[j] = make_float4(a.x, a.y, b.x, b.y);
      cA[kCycN + j] = make_float4(a.z, a.w, b.z, b.w);
    }
  }
  // FP32 path: the upstream gradient of the smoothed spectrum staged in
  // shared memory as floats when it is small
  const bool smooth = dLdS != nullptr && p.smooth_sigma > 0.0;
  if (smooth && sizeof(T) == 4 && p.n_bins <= kGradStageBins)
    for (int k = threadIdx.x; k < p.n_bins; k += blockDim.x) sdS[k] = (T)dLdS[k];

  // effective upstream coefficients
  const Seeds<T> sd = make_seeds<T>(mom, dLdm);
  const T w0 = (T)sqrt(1.0 / p.inv_w0sq);
  __syncthreads();

  GAcc<T> acc;
  acc.init();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  if (!smooth)
    grad_range<T, QFP, T, VAR>(p, tab, sd, static_cast<const T*>(nullptr), w0, acc, 0, p.n, tid,
                               nthr, cA);
  else if (sizeof(T) == 4 && p.n_bins <= kGradStageBins)
    grad_range<T, QFP, T, VAR>(p, tab, sd, sdS, w0, acc, 0, p.n, tid, nthr, cA);
  else
    grad_range<T, QFP, double, VAR>(p, tab, sd, dLdS, w0, acc, 0, p.n, tid, nthr, cA);

  // fixed-order block reduction into this CTA's slot
  grad_block_reduce(acc, red, p.partials + (size_t)blockIdx.x * kNumMom);
}

__global__ void k_grad_final(const Params p, int grid, double* grad8) {
  if (threadIdx.x < kNumGrad) {
    double s = 0.0, c = 0.0;
    for (int b = 0; b < grid; ++b) {
      const double x = p.partials[(size_t)b * kNumMom + threadIdx.x];
      const double t = s + x;
      c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    grad8[threadIdx.x] = s + c;
  }
}

}  // namespace qs

using namespace qs;
using namespace qs::detail;

namespace {

template <typename T, bool QFP, int VAR>
int32_t launch_grad(const Params& p, int block, int sms, int grid_req, int gmax,
                    const qs_moments* mom, const double* dLdm, const double* dLdS,
                    cudaStream_t st, int* grid_out) {
  using TT = typename Tab<T>::type;
  const size_t tab =
      grad_has_table<T, QFP, VAR>() ? align_up((size_t)p.n_phase * sizeof(TT), 16) : 0;
  const bool stage = sizeof(T) == 4 && dLdS != nullptr && p.smooth_sigma > 0.0 &&
                     p.n_bins <= kGradStageBins;
  const size_t smem = tab + grad_cyc_bytes<T, VAR>() +
                      (size_t)(block / 32) * kNumGrad * sizeof(double) +
                      (stage ? (size_t)p.n_bins * sizeof(float) : 0);
  auto kern = k_grad<T, QFP, VAR>;
  static CtxMark smem_mark;
  if (int32_t e = allow_smem(kern, smem_mark, kSmemLimit)) return e;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess)
    return cuda_fail();
  const int grid = pick_grid(occ, sms, block, grid_req, p.n, gmax);
  kern<<<grid, block, smem, st>>>(p, mom, dLdm, dLdS);
  *grid_out = grid;
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

}  // namespace

extern "C" int32_t qs_scatter_grad(const qs_laser* laser, const qs_beam* beam,
                                   const qs_samples* samples, const qs_bins* bins,
                                   const qs_exec* exec, const qs_moments* d_moments,
                                   const double* d_dL_dmoments, const double* d_dL_dsmooth,
                                   double* d_grad8, void* d_workspace, size_t ws_bytes,
                                   void* stream) {
  int32_t st;
  if ((st = validate_laser(laser)) || (st = validate_beam(beam)) ||
      (st = validate_samples(samples)) || (st = validate_bins(bins)))
    return st;
  int prec, wbits, block, grid, sms;
  if ((st = exec_opts(exec, &prec, &wbits, &block, &grid))) return st;
  if (!d_moments || !d_dL_dmoments || !d_grad8) return QS_ERR_INVALID_ARG;
  if (d_dL_dsmooth && !(bins->smooth_sigma_bins > 0)) return QS_ERR_INVALID_ARG;
  if ((st = device_sms(&sms))) return st;
  Plan pl;
  make_plan(pl, bins, block, grid, sms);
  if (!d_workspace || ((uintptr_t)d_workspace % 256) || ws_bytes < pl.ws_bytes)
    return QS_ERR_WORKSPACE;
  Params p;
  fill_params(p, laser, beam, samples, bins, wbits);
  p.partials = reinterpret_cast<double*>(static_cast<unsigned char*>(d_workspace) + pl.off_part);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const bool qfp = laser->model == QS_MODEL_QFP;
  const int var = laser->variant;
  if ((var & QS_VARIANT_CYCLE_CHI) && (st = cycle_tables(p, cs))) return st;
  // FP32 QFP variant 0, block left open: one 512-thread CTA per SM (118
  // registers).  CTAs that share an SM are served oldest first and finish far
  // apart, so a single CTA keeps all its warps resident to the end of the
  // launch.  The model variants carry more tangents: 256-thread CTAs.
  int kblock = block;
  if (!(exec && exec->block) && prec == QS_F32 && qfp && var == 0) kblock = 512;
  if (var != 0 && kblock > 256) kblock = 256;
  int g = 1;
  auto run = [&](auto tq, auto tqfp, auto tvar) {
    using T = decltype(tq);
    constexpr bool Q = decltype(tqfp)::value;
    constexpr int VAR = decltype(tvar)::value;
    return launch_grad<T, Q, VAR>(p, kblock, sms, grid, pl.gmax, d_moments, d_dL_dmoments,
                                  d_dL_dsmooth, cs, &g);
  };
  using std::integral_constant;
  using F = std::false_type;
  using Tr = std::true_type;
  auto by_var = [&](auto tq) {
    if (!qfp) {
      if (var & QS_VARIANT_CELL_FOCUS) return run(tq, F{}, integral_constant<int, 1>{});
      return run(tq, F{}, integral_constant<int, 0>{});
    }
    switch (var) {
      case 1: return run(tq, Tr{}, integral_constant<int, 1>{});
      case 2: return run(tq, Tr{}, integral_constant<int, 2>{});
      case 3: return run(tq, Tr{}, integral_constant<int, 3>{});
      default: return run(tq, Tr{}, integral_constant<int, 0>{});
    }
  };
  st = prec == QS_F64 ? by_var(0.0) : by_var(0.0f);
  if (st) return st;
  k_grad_final<<<1, 32, 0, cs>>>(p, g, d_grad8);
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

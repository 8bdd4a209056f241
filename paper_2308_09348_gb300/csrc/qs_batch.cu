// qs_batch.cu -- many shots in one persistent launch (qs_scatter_batch).
//
// B0 k_bsetup   one thread per shot: validate the device-side descriptors,
//               derive the shot's launch constants, point them at its slice
//               of the samples and of the accumulators, count its tiles.
// B1 k_btable   one thread per (shot, phase cell): the shot's envelope table.
// B2 k_bscan    one CTA: exclusive prefix sum of the tile counts.
// B3 k_batch    persistent grid; each CTA pulls tiles from a device counter,
//               stages the tile's shot constants and table in shared memory,
//               evaluates the samples exactly as k_scatter does, writes the
//               tile's moment partials to the tile's own slot and merges its
//               shared-memory spectrum into the shot's accumulators (the
//               shot's divergence map and a_eff histogram take global
//               integer atomics directly).  Launched twice over the same
//               schedule: the paper's model, then the model variants.
// B4 k_bfinal   one warp per shot: partials summed in tile order, histograms
//               converted, moments written.
// G3 k_bgrad    (qs_scatter_grad_batch) the adjoint over the same (shot,
//               tile) schedule: each tile's samples recomputed with tangents,
//               the tile's 8 gradient partials to its own slot.
// G4 k_bgfinal  one warp per shot: gradient slots summed in tile order.
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348 (Sec. 3.2: parallel
// plane-wave runs; Sec. 6: high-repetition-rate data).
#include "qscatter.h"
#include "qs_device.cuh"
#include "qs_derive.cuh"
#include "qs_grad.cuh"
#include "qs_host.hpp"

#include <type_traits>

namespace qs {

struct BatchArgs {
  int32_t n_shots, max_phase, tile, wbits;
  const qs_laser* lasers;
  const qs_beam* beams;
  const int64_t* offsets;
  qs_samples samples;
  qs_bins bins;
  const double* ranges;
  Params* shot;                 // [n_shots]
  int64_t* tiles;               // [n_shots + 1] counts, then exclusive offsets
  void* tables;                 // [n_shots * max_phase] float4 (FP32) or double (FP64)
  unsigned long long* acc;      // [n_shots * (n_bins + 2)]
  unsigned long long* acc_smooth;  // [n_shots * n_bins] (smoothed spectrum) or null
  unsigned long long* acc_map;     // [n_shots * (n_tx n_ty + 1)] (divergence maps) or null
  unsigned long long* acc_aeff;    // [n_shots * (n_aeff + 1)] (a_eff histograms) or null
  double* partials;             // [tiles * kNumMom]
  unsigned long long* counter;  // [0] work counter of the variant-0 kernels,
                                // [1] that of the model-variant kernels,
                                // [2] nonzero if any shot uses a model variant
  int64_t max_tiles;            // tile slots in the workspace
  const double* cyc_gl;         // cycle-resolved chi tables of this context
  const float4* cyc_a;          // (null: shots with that variant are invalid)
  const float4* cyc_m;
  int32_t precision, pad;
};

__global__ void k_bsetup(const BatchArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n_shots) return;
  Params& p = a.shot[s];
  const qs_laser L = a.lasers[s];
  const qs_beam B = a.beams[s];
  qs_bins b = a.bins;
  if (a.ranges) {
    b.lo = a.ranges[2 * s];
    b.hi = a.ranges[2 * s + 1];
  }
  // shared samples (parameter sweep) when no offsets are given
  const int64_t o0 = a.offsets ? a.offsets[s] : 0;
  const int64_t o1 = a.offsets ? a.offsets[s + 1] : a.samples.n;
  // a model variant runs in its own kernels; cycle-resolved chi needs this
  // context's tables
  const bool cells = L.model == QS_MODEL_QFP || (L.variant & QS_VARIANT_CELL_FOCUS);
  bool ok = check_laser(L) == QS_OK &&
            (!(L.variant & QS_VARIANT_CYCLE_CHI) || (a.cyc_a && a.cyc_m && a.cyc_gl)) &&
            check_beam(B) == QS_OK && check_bins(b) == QS_OK &&
            o0 >= 0 && o1 >= o0 && o1 <= a.samples.n &&
            (!cells || L.n_phase <= a.max_phase);
  if (!ok) {
    memset(&p, 0, sizeof(Params));
    p.n = -1;                    // invalid shot
    a.tiles[s] = 0;
    return;
  }
  derive_params(p, L, B, &b, a.wbits);
  const size_t esz = a.samples.dtype == QS_F32 ? 4 : 8;
  p.n = o1 - o0;
  for (int k = 0; k < 8; ++k)
    p.xi[k] = a.samples.xi[k] ? static_cast<const unsigned char*>(a.samples.xi[k]) + o0 * esz
                              : nullptr;
  p.w = a.samples.w ? static_cast<const unsigned char*>(a.samples.w) + o0 * esz : nullptr;
  p.dtype = a.samples.dtype;
  p.weighted = a.samples.w != nullptr;
  p.acc_spec = a.bins.n_bins > 0 ? a.acc + (size_t)s * (a.bins.n_bins + 2) : nullptr;
  p.acc_smooth = a.acc_smooth ? a.acc_smooth + (size_t)s * a.bins.n_bins : nullptr;
  p.acc_map = a.acc_map ? a.acc_map + (size_t)s * ((size_t)a.bins.n_tx * a.bins.n_ty + 1)
                        : nullptr;
  p.acc_aeff = a.acc_aeff ? a.acc_aeff + (size_t)s * (a.bins.n_aeff + 1) : nullptr;
  p.cyc_gl = a.cyc_gl;
  p.cyc_a = a.cyc_a;
  p.cyc_m = a.cyc_m;
  a.tiles[s] = (p.n + a.tile - 1) / a.tile;
  if (L.variant != 0 && a.tiles[s] > 0) a.counter[2] = 1ull;
}

__global__ void k_btable(const BatchArgs a) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = (int)(idx / a.max_phase), j = (int)(idx % a.max_phase);
  if (s >= a.n_shots) return;
  const Params& p = a.shot[s];
  if (p.n < 0 || !(p.model == QS_MODEL_QFP || p.focus) || j >= p.n_phase) return;
  if (a.precision == QS_F32)
    table_entry(p, j, static_cast<float4*>(a.tables) + (size_t)s * a.max_phase);
  else
    table_entry(p, j, static_cast<double*>(a.tables) + (size_t)s * a.max_phase);
}

// Exclusive prefix sum of tiles[0..n) in place, total in tiles[n].  The
// per-shot checks of k_bsetup see one shot's range only; here the offsets
// are checked as a whole: if they decrease anywhere (shot ranges could then
// overlap), or the tiles would exceed the workspace's slots, every shot is
// made invalid and the total set to 0, so no shot does any work.
__global__ void __launch_bounds__(1024) k_bscan(const BatchArgs a) {
  __shared__ int64_t part[1024];
  __shared__ int s_bad;
  const int n = a.n_shots;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(n, b0 + per);
  int64_t s = 0;
  int bad = 0;
  for (int i = b0; i < b1; ++i) {
    s += a.tiles[i];
    if (a.offsets && a.offsets[i + 1] < a.offsets[i]) bad = 1;
  }
  part[threadIdx.x] = s;
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int64_t v = part[t];
      part[t] = run;
      run += v;
    }
    s_bad = bad || run > a.max_tiles;
    a.tiles[n] = s_bad ? 0 : run;
  }
  __syncthreads();
  if (s_bad) {
    for (int i = b0; i < b1; ++i) {
      a.shot[i].n = -1;
      a.tiles[i] = 0;
    }
    return;
  }
  int64_t run = part[threadIdx.x];
  for (int i = b0; i < b1; ++i) {
    const int64_t v = a.tiles[i];
    a.tiles[i] = run;
    run += v;
  }
}

// The tiles of one kind of shot: VARK = false the shots of the paper's model
// (variant 0), VARK = true those with a model variant (the per-cell focus,
// cycle-resolved chi: longer per-sample code, its own kernel so that the
// variant-0 kernel keeps its register budget).  Each kernel pulls tiles from
// its own counter and passes over the other kind's.
template <bool VARK>
__device__ __forceinline__ bool tile_of_kind(const Params& p) {
  return ((p.focus != 0) || (p.cycle != 0)) == VARK;
}

template <typename T, typename H, bool VARK>
__global__ void __launch_bounds__(VARK ? 256 : 512, sizeof(T) == 4 ? 2 : 1)
    k_batch(const BatchArgs a) {
  using TT = typename Tab<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  Params& p = *reinterpret_cast<Params*>(smem);
  const size_t par_bytes = (sizeof(Params) + 15) & ~(size_t)15;
  TT* tab = reinterpret_cast<TT*>(smem + par_bytes);
  const size_t tab_bytes = ((size_t)a.max_phase * sizeof(TT) + 15) & ~(size_t)15;
  double* red = reinterpret_cast<double*>(smem + par_bytes + tab_bytes);
  H* hs = reinterpret_cast<H*>(smem + par_bytes + tab_bytes +
                               (size_t)(blockDim.x >> 5) * kNumMom * sizeof(double));
  // work-item broadcast slots live in the dynamic allocation, after the
  // histogram, so the kernel has no static shared memory
  const size_t hist_bytes =
      ((size_t)(a.bins.n_bins > 0 ? a.bins.n_bins + 2 : 0) * sizeof(H) + 15) & ~(size_t)15;
  int64_t& s_tile = *reinterpret_cast<int64_t*>(reinterpret_cast<unsigned char*>(hs) + hist_bytes);
  int& s_shot = *reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(hs) + hist_bytes + 8);
  // the tile's smoothed-spectrum accumulators (when smoothing), after the
  // broadcast slots
  const int64_t nsm = a.acc_smooth ? (int64_t)a.bins.n_bins : 0;
  unsigned long long* hsm = nsm ? reinterpret_cast<unsigned long long*>(
                                      reinterpret_cast<unsigned char*>(hs) + hist_bytes + 16)
                                : nullptr;
  // FP32 cycle-resolved chi: the per-interval monomial tables of G and H
  // after the smoothed-spectrum accumulators
  float4* cA = VARK ? reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(hs) + hist_bytes +
                                                16 + ((nsm * 8 + 15) & ~(int64_t)15))
                    : nullptr;
  const int64_t total = a.tiles[a.n_shots];
  const int64_t nspec = a.bins.n_bins > 0 ? (int64_t)a.bins.n_bins + 2 : 0;
  // per-shot divergence map and a_eff histogram: global accumulators
  const int64_t nmap = a.acc_map ? (int64_t)a.bins.n_tx * a.bins.n_ty + 1 : 0;
  const int64_t naeff = a.acc_aeff ? (int64_t)a.bins.n_aeff + 1 : 0;
  const int lane = threadIdx.x & 31;
  int cur = -1;
  if (VARK && a.counter[2] == 0ull) return;        // no shot uses a variant

  for (;;) {
    if (threadIdx.x == 0) {
      int64_t t;
      int s;
      do {
        t = (int64_t)atomicAdd(a.counter + (VARK ? 1 : 0), 1ull);
        s = -1;
        if (t < total) {
          // last shot whose first tile is <= t (shots with no tiles are skipped)
          int lo = 0, hi = a.n_shots - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.tiles[mid] <= t) lo = mid;
            else hi = mid - 1;
          }
          s = lo;
        }
      } while (t < total && !tile_of_kind<VARK>(a.shot[s]));
      s_tile = t;
      s_shot = s;
    }
    __syncthreads();
    const int64_t t = s_tile;
    const int s = s_shot;
    if (t >= total) break;
    if (s != cur) {
      // stage the shot's constants and envelope table
      const int nw = (int)(sizeof(Params) / 4);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&a.shot[s]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&p);
      for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      if (p.model == QS_MODEL_QFP || p.focus) {
        const TT* tg = static_cast<const TT*>(a.tables) + (size_t)s * a.max_phase;
        for (int j = threadIdx.x; j < p.n_phase; j += blockDim.x) tab[j] = tg[j];
      }
      if (VARK && sizeof(T) == 4 && p.cycle) {
        // per-interval monomial coefficients of G and H (the forward lookup)
        for (int j = threadIdx.x; j < kCycN - 1; j += blockDim.x) {
          cA[j] = p.cyc_m[j];
          cA[kCycN + j] = p.cyc_m[kCycN + j];
        }
      }
      cur = s;
    }
    for (int64_t b = threadIdx.x; b < nspec; b += blockDim.x) hs[b] = 0;
    for (int64_t b = threadIdx.x; b < nsm; b += blockDim.x) hsm[b] = 0;
    __syncthreads();

    typename AccT<T>::type acc;
    acc_init(acc);
    const int64_t first = (t - a.tiles[s]) * a.tile;
    const int64_t last = min(p.n, first + a.tile);
    // loops advance warp by warp (bounds uniform across the lanes), so that
    // the smoothed deposits run warp-cooperatively after each step
    auto run = [&](auto tvar) {
      constexpr int VAR = decltype(tvar)::value;
      bool pairs = false;
      if constexpr (sizeof(T) == 4) {
        if (p.model == QS_MODEL_QFP) {
          pairs = true;
          // FP32 QFP: each thread carries samples 2k and 2k+1 (first is even)
          for (int64_t kb = first / 2 + threadIdx.x - lane; 2 * kb < last; kb += blockDim.x) {
            const int64_t k = kb + lane;
            const int64_t i0 = 2 * k, i1 = (2 * k + 1 < last) ? 2 * k + 1 : 2 * k;
            DepF d0, d1;
            bool ok0 = false, ok1 = false;
            if (i0 < last) {
              SampleF s0, s1;
              eval_pair_f32_qfp<VAR>(p, reinterpret_cast<const float4*>(tab), i0, i1, s0, s1, cA);
              ok0 = accumulate<T, H, true>(p, s0, i0, acc, hs, nullptr, nullptr, nspec, nmap, naeff);
              if (i1 != i0)
                ok1 = accumulate<T, H, true>(p, s1, i1, acc, hs, nullptr, nullptr, nspec, nmap, naeff);
              dep_set(d0, s0);
              dep_set(d1, s1);
            }
            if (hsm) {
              deposit_warp(p, ok0, d0, i0, hsm);
              deposit_warp(p, ok1, d1, i1, hsm);
            }
          }
        }
      }
      if (!pairs) {
        for (int64_t ib = first + threadIdx.x - lane; ib < last; ib += blockDim.x) {
          const int64_t i = ib + lane;
          typename DepT<T>::type d;
          bool ok = false;
          if (i < last) {
            const auto sm = p.model == QS_MODEL_QFP ? eval_one<T, true, VAR>(p, tab, i, cA)
                                                    : eval_one<T, false, VAR & kVarCell>(p, tab, i, cA);
            ok = accumulate<T, H, true>(p, sm, i, acc, hs, nullptr, nullptr, nspec, nmap, naeff);
            dep_set(d, sm);
          }
          if (hsm) deposit_warp(p, ok, d, i, hsm);
        }
      }
    };
    if constexpr (!VARK) {
      run(std::integral_constant<int, 0>{});
    } else {
      switch ((p.focus ? kVarCell : 0) | (p.cycle ? kVarCycle : 0)) {
        case kVarCell: run(std::integral_constant<int, kVarCell>{}); break;
        case kVarCycle: run(std::integral_constant<int, kVarCycle>{}); break;
        default: run(std::integral_constant<int, kVarCell | kVarCycle>{}); break;
      }
    }
    block_reduce_write(acc, red, a.partials + (size_t)t * kNumMom);
    __syncthreads();
    for (int64_t b = threadIdx.x; b < nspec; b += blockDim.x)
      if (hs[b]) atomicAdd(&p.acc_spec[b], (unsigned long long)hs[b]);
    for (int64_t b = threadIdx.x; b < nsm; b += blockDim.x)
      if (hsm[b]) atomicAdd(&p.acc_smooth[b], hsm[b]);
    __syncthreads();
  }
}

// One warp per shot: moments from its tiles' partials in tile order.
__global__ void k_bfinal(const BatchArgs a, double* spectra, double* smooth, double* divmaps,
                         double* aeff_hists, qs_moments* moments) {
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= a.n_shots) return;
  const Params& p = a.shot[s];
  const int nb = a.bins.n_bins;
  const bool sm = a.acc_smooth != nullptr;
  const int64_t nm = a.acc_map ? (int64_t)a.bins.n_tx * a.bins.n_ty : 0;
  const int na = a.acc_aeff ? a.bins.n_aeff : 0;
  qs_moments m;
  memset(&m, 0, sizeof(m));
  if (p.n < 0) {
    for (int b = lane; b < nb; b += 32) spectra[(size_t)s * nb + b] = 0.0;
    if (sm)
      for (int b = lane; b < nb; b += 32) smooth[(size_t)s * nb + b] = 0.0;
    for (int64_t b = lane; b < nm; b += 32) divmaps[(size_t)s * nm + b] = 0.0;
    for (int b = lane; b < na; b += 32) aeff_hists[(size_t)s * na + b] = 0.0;
    if (lane == 0) {
      m.nonfinite = -1.0;
      moments[s] = m;
    }
    return;
  }
  const double scale = p.weighted ? 1.0 / p.wscale : 1.0;
  const int64_t t0 = a.tiles[s], t1 = (s + 1 < a.n_shots) ? a.tiles[s + 1] : a.tiles[a.n_shots];
  double tot = 0.0, mean_l0 = 0.0, m2_l0 = 0.0;
  if (lane == 0) {
    // (W, mean, M2) merged over the shot's tiles in tile order
    double W = 0.0, mm = 0.0, M2 = 0.0;
    for (int64_t t = t0; t < t1; ++t) {
      const double* q = a.partials + (size_t)t * kNumMom;
      welford_merge(W, mm, M2, q[0], q[1], q[2]);
    }
    tot = W;
    mean_l0 = mm;
    m2_l0 = M2;
  } else if (lane >= 3 && lane < kNumMom) {
    // Neumaier-compensated sums over the shot's tiles in tile order
    double sm = 0.0, c = 0.0;
    for (int64_t t = t0; t < t1; ++t) {
      const double x = a.partials[(size_t)t * kNumMom + lane];
      const double u = sm + x;
      c += fabs(sm) >= fabs(x) ? (sm - u) + x : (x - u) + sm;
      sm = u;
    }
    tot = sm + c;
  }
  double v[kNumMom];
#pragma unroll
  for (int k = 0; k < kNumMom; ++k) v[k] = __shfl_sync(0xffffffffu, tot, k);
  v[1] = __shfl_sync(0xffffffffu, mean_l0, 0);
  v[2] = __shfl_sync(0xffffffffu, m2_l0, 0);
  const unsigned long long* acc = p.acc_spec;
  for (int b = lane; b < nb; b += 32) spectra[(size_t)s * nb + b] = (double)acc[b] * scale;
  if (sm)
    for (int b = lane; b < nb; b += 32)
      smooth[(size_t)s * nb + b] = (double)p.acc_smooth[b] / p.wscale;
  for (int64_t b = lane; b < nm; b += 32) divmaps[(size_t)s * nm + b] = (double)p.acc_map[b] * scale;
  for (int b = lane; b < na; b += 32) aeff_hists[(size_t)s * na + b] = (double)p.acc_aeff[b] * scale;
  if (lane == 0) {
    const double W = v[0];
    m.W = W;
    if (W > 0.0) {
      const double var = v[2] / W + v[3] / W;
      m.mean = v[1];
      m.spread = sqrt(var > 0.0 ? var : 0.0);
      m.rel_spread = m.spread / m.mean;
      m.div_x = sqrt(v[4] / W);
      m.div_y = sqrt(v[5] / W);
      m.div = sqrt((v[4] + v[5]) / W);
      m.mean_aeff = v[6] / W;
      m.mean_gamma0 = v[7] / W;
    }
    m.under = nb > 0 ? (double)acc[nb] * scale : 0.0;
    m.over = nb > 0 ? (double)acc[nb + 1] * scale : 0.0;
    m.map_out = nm ? (double)p.acc_map[nm] * scale : 0.0;
    m.nonfinite = v[8];
    moments[s] = m;
  }
}

// Largest smoothed spectrum whose upstream gradient the FP32 batched adjoint
// stages in shared memory (larger ones are read from global memory).
constexpr int kBGradStageBins = 8192;

// G3: the adjoint of every shot over the (shot, tile) schedule of k_batch.
// Per tile: the shot's launch constants, envelope table and (FP32, when it
// fits) its upstream smoothed-spectrum gradient staged in shared memory, the
// upstream coefficients of its moments in registers; the tile's samples
// recomputed with tangents exactly as k_grad does; the tile's 8 partials
// reduced in a fixed order into its own slot.
//   moms: the forward moments (n_shots); dLdm: n_shots x 13; dLdS: n_shots x
//   n_bins or null.
template <typename T, bool VARK>
__global__ void __launch_bounds__(VARK ? 256 : 512)
    k_bgrad(const BatchArgs a, const qs_moments* __restrict__ moms,
            const double* __restrict__ dLdm, const double* __restrict__ dLdS) {
  using TT = typename Tab<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  Params& p = *reinterpret_cast<Params*>(smem);
  const size_t par_bytes = (sizeof(Params) + 15) & ~(size_t)15;
  TT* tab = reinterpret_cast<TT*>(smem + par_bytes);
  const size_t tab_bytes = ((size_t)a.max_phase * sizeof(TT) + 15) & ~(size_t)15;
  double* red = reinterpret_cast<double*>(smem + par_bytes + tab_bytes);
  unsigned char* after_red = smem + par_bytes + tab_bytes +
                             (((size_t)(blockDim.x >> 5) * kNumGrad * sizeof(double) + 15) &
                              ~(size_t)15);
  int64_t& s_tile = *reinterpret_cast<int64_t*>(after_red);
  int& s_shot = *reinterpret_cast<int*>(after_red + 8);
  const int nb = a.bins.n_bins;
  const bool smooth = dLdS != nullptr && a.bins.smooth_sigma_bins > 0.0;
  const bool stage = smooth && sizeof(T) == 4 && nb <= kBGradStageBins;
  T* sdS = reinterpret_cast<T*>(after_red + 16);
  // FP32 cycle-resolved chi: the node-pair Hermite tables after the stage
  float4* cA = reinterpret_cast<float4*>(
      after_red + 16 + (((stage ? (size_t)nb * sizeof(T) : 0) + 15) & ~(size_t)15));
  const int64_t total = a.tiles[a.n_shots];
  int cur = -1;
  Seeds<T> sd{};
  T w0 = (T)1;
  if (VARK && a.counter[2] == 0ull) return;        // no shot uses a variant

  for (;;) {
    if (threadIdx.x == 0) {
      int64_t t;
      int sh;
      do {
        t = (int64_t)atomicAdd(a.counter + (VARK ? 1 : 0), 1ull);
        sh = -1;
        if (t < total) {
          int lo = 0, hi = a.n_shots - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.tiles[mid] <= t) lo = mid;
            else hi = mid - 1;
          }
          sh = lo;
        }
      } while (t < total && !tile_of_kind<VARK>(a.shot[sh]));
      s_tile = t;
      s_shot = sh;
    }
    __syncthreads();
    const int64_t t = s_tile;
    const int s = s_shot;
    if (t >= total) break;
    if (s != cur) {
      const int nw = (int)(sizeof(Params) / 4);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&a.shot[s]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&p);
      for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      if (p.model == QS_MODEL_QFP || p.focus) {
        const TT* tg = static_cast<const TT*>(a.tables) + (size_t)s * a.max_phase;
        for (int j = threadIdx.x; j < p.n_phase; j += blockDim.x) tab[j] = tg[j];
      }
      if (VARK && sizeof(T) == 4 && p.cycle) {
        for (int j = threadIdx.x; j < kCycN - 1; j += blockDim.x) {
          const float4 u = p.cyc_a[j], v = p.cyc_a[j + 1];
          cA[j] = make_float4(u.x, u.y, v.x, v.y);
          cA[kCycN + j] = make_float4(u.z, u.w, v.z, v.w);
        }
      }
      if (stage)
        for (int k = threadIdx.x; k < nb; k += blockDim.x) sdS[k] = (T)dLdS[(size_t)s * nb + k];
      sd = make_seeds<T>(moms + s, dLdm + (size_t)s * 13);
      w0 = (T)sqrt(1.0 / p.inv_w0sq);
      cur = s;
      __syncthreads();
    }
    GAcc<T> acc;
    acc.init();
    const int64_t first = (t - a.tiles[s]) * a.tile;
    const int64_t last = min(p.n, first + a.tile);
    const int64_t tid = threadIdx.x, nthr = blockDim.x;
    const double* gS = smooth ? dLdS + (size_t)s * nb : nullptr;
    auto run = [&](auto tqfp, auto tvar) {
      constexpr bool Q = decltype(tqfp)::value;
      constexpr int VAR = decltype(tvar)::value;
      if (!smooth)
        grad_range<T, Q, T, VAR>(p, tab, sd, static_cast<const T*>(nullptr), w0, acc, first, last,
                                 tid, nthr, cA);
      else if (stage)
        grad_range<T, Q, T, VAR>(p, tab, sd, sdS, w0, acc, first, last, tid, nthr, cA);
      else
        grad_range<T, Q, double, VAR>(p, tab, sd, gS, w0, acc, first, last, tid, nthr, cA);
    };
    using std::integral_constant;
    using Tr = std::true_type;
    using Fa = std::false_type;
    if constexpr (!VARK) {
      if (p.model == QS_MODEL_QFP) run(Tr{}, integral_constant<int, 0>{});
      else run(Fa{}, integral_constant<int, 0>{});
    } else {
      const int var = (p.focus ? kVarCell : 0) | (p.cycle ? kVarCycle : 0);
      if (p.model != QS_MODEL_QFP) run(Fa{}, integral_constant<int, kVarCell>{});
      else if (var == kVarCell) run(Tr{}, integral_constant<int, kVarCell>{});
      else if (var == kVarCycle) run(Tr{}, integral_constant<int, kVarCycle>{});
      else run(Tr{}, integral_constant<int, kVarCell | kVarCycle>{});
    }
    grad_block_reduce(acc, red, a.partials + (size_t)t * kNumMom);
    __syncthreads();
  }
}

// G4: one warp per shot, lane k < 8 sums gradient component k over the
// shot's tiles in tile order (compensated); invalid shots get zeros.
__global__ void k_bgfinal(const BatchArgs a, double* grad) {
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= a.n_shots || lane >= kNumGrad) return;
  const Params& p = a.shot[s];
  double sm = 0.0, c = 0.0;
  if (p.n >= 0) {
    const int64_t t0 = a.tiles[s], t1 = (s + 1 < a.n_shots) ? a.tiles[s + 1] : a.tiles[a.n_shots];
    for (int64_t t = t0; t < t1; ++t) {
      const double x = a.partials[(size_t)t * kNumMom + lane];
      const double u = sm + x;
      c += fabs(sm) >= fabs(x) ? (sm - u) + x : (x - u) + sm;
      sm = u;
    }
  }
  grad[(size_t)s * kNumGrad + lane] = sm + c;
}

}  // namespace qs

using namespace qs;
using namespace qs::detail;

namespace {

struct BatchPlan {
  size_t off_counter = 0, off_params = 0, off_tiles = 0, off_tables = 0, off_acc = 0,
         off_smooth = 0, off_map = 0, off_aeff = 0, off_part = 0, bytes = 0;
  int64_t max_tiles = 0;
};

bool batch_plan(BatchPlan& bp, int32_t n_shots, int64_t n_total, const qs_bins* bins,
                int32_t max_phase, int precision, int tile, bool shared) {
  if (n_shots < 1 || n_total < 0 || max_phase < 1 || max_phase > kMaxPhase) return false;
  // tile slots: disjoint shots need at most n_total/tile + n_shots; a sweep
  // (every shot covers all samples) needs n_shots * ceil(n_total/tile)
  bp.max_tiles = shared ? (int64_t)n_shots * ((n_total + tile - 1) / tile) + 1
                        : n_total / tile + n_shots + 1;
  size_t off = 0;
  bp.off_counter = off; off = align_up(off + 3 * 8, 256);
  bp.off_params = off; off = align_up(off + (size_t)n_shots * sizeof(Params), 256);
  bp.off_tiles = off; off = align_up(off + (size_t)(n_shots + 1) * 8, 256);
  bp.off_tables = off;
  off = align_up(off + (size_t)n_shots * max_phase * (precision == QS_F64 ? 8 : 16), 256);
  bp.off_acc = off;
  off = align_up(off + (size_t)n_shots * (bins->n_bins > 0 ? bins->n_bins + 2 : 0) * 8, 256);
  bp.off_smooth = off;
  off = align_up(off + (size_t)n_shots * (bins->smooth_sigma_bins > 0 ? bins->n_bins : 0) * 8, 256);
  bp.off_map = off;
  off = align_up(off + (size_t)n_shots *
                           (bins->n_tx > 0 ? (size_t)bins->n_tx * bins->n_ty + 1 : 0) * 8, 256);
  bp.off_aeff = off;
  off = align_up(off + (size_t)n_shots * (bins->n_aeff > 0 ? bins->n_aeff + 1 : 0) * 8, 256);
  bp.off_part = off; off = align_up(off + (size_t)bp.max_tiles * kNumMom * 8, 256);
  bp.bytes = off;
  return true;
}

int32_t batch_checks(int32_t n_shots, const qs_samples* samples, const qs_bins* bins,
                     int32_t max_phase, const qs_exec* exec, int* prec, int* wbits, int* block,
                     int* grid, int* tile) {
  int32_t st;
  if (n_shots < 1 || max_phase < 1 || max_phase > kMaxPhase) return QS_ERR_INVALID_ARG;
  if ((st = validate_samples(samples)) || (st = validate_bins(bins))) return st;
  if ((st = exec_opts(exec, prec, wbits, block, grid))) return st;
  if ((st = exec_tile(exec, tile))) return st;
  return QS_OK;
}

template <typename T, typename H>
int32_t launch_batch_kind(const BatchArgs& a, int block, int grid_req, int sms, cudaStream_t st,
                          bool vark) {
  using TT = typename Tab<T>::type;
  const size_t smem = align_up(sizeof(Params), 16) + align_up((size_t)a.max_phase * sizeof(TT), 16) +
                      (size_t)(block / 32) * kNumMom * sizeof(double) +
                      align_up((size_t)(a.bins.n_bins > 0 ? a.bins.n_bins + 2 : 0) * sizeof(H), 16) +
                      16 + (a.acc_smooth ? align_up((size_t)a.bins.n_bins * 8, 16) : 0) +
                      (vark && sizeof(T) == 4 ? (size_t)2 * kCycN * sizeof(float4) : 0);
  if (smem > (size_t)kSmemLimit) return QS_ERR_UNSUPPORTED;
  auto kern = vark ? k_batch<T, H, true> : k_batch<T, H, false>;
  static CtxMark smem_mark[2];
  if (int32_t e = allow_smem(kern, smem_mark[vark ? 1 : 0], kSmemLimit)) return e;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess)
    return cuda_fail();
  const int grid = grid_req > 0 ? grid_req : sms * (occ > 0 ? occ : 1);
  kern<<<grid, block, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

// The variant-0 kernel, then the model-variant kernel (which returns at once
// when no shot uses a variant).
template <typename T, typename H>
int32_t launch_batch(const BatchArgs& a, int block, int grid_req, int sms, cudaStream_t st) {
  if (int32_t e = launch_batch_kind<T, H>(a, block, grid_req, sms, st, false)) return e;
  return launch_batch_kind<T, H>(a, block, grid_req, sms, st, true);
}

}  // namespace

extern "C" size_t qs_batch_workspace_bytes(int32_t n_shots, int64_t n_total, const qs_bins* bins,
                                           int32_t max_phase, const qs_exec* exec,
                                           int32_t shared_samples) {
  int prec, wbits, block, grid, tile;
  if (!bins || validate_bins(bins) != QS_OK) return 0;
  if (exec_opts(exec, &prec, &wbits, &block, &grid) || exec_tile(exec, &tile)) return 0;
  BatchPlan bp;
  if (!batch_plan(bp, n_shots, n_total, bins, max_phase, prec, tile, shared_samples != 0))
    return 0;
  return bp.bytes;
}

namespace {

// Device descriptors, workspace layout and the set-up kernels shared by the
// batched forward and adjoint: validates on the host, fills `a`, zeroes the
// work counter (and, for the forward, the accumulators) and launches
// k_bsetup, k_btable and k_bscan on `cs`.
int32_t batch_prepare(BatchArgs& a, int32_t n_shots, const qs_laser* d_lasers,
                      const qs_beam* d_beams, const int64_t* d_offsets,
                      const qs_samples* samples, const qs_bins* bins, const double* d_ranges,
                      int32_t max_phase, int prec, int wbits, int tile, void* d_workspace,
                      size_t ws_bytes, bool zero_acc, cudaStream_t cs) {
  if (!d_lasers || !d_beams) return QS_ERR_INVALID_ARG;
  BatchPlan bp;
  if (!batch_plan(bp, n_shots, samples->n, bins, max_phase, prec, tile, d_offsets == nullptr))
    return QS_ERR_INVALID_ARG;
  if (!d_workspace || ((uintptr_t)d_workspace % 256) || ws_bytes < bp.bytes)
    return QS_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(d_workspace);
  memset(&a, 0, sizeof(a));
  a.n_shots = n_shots;
  a.max_phase = max_phase;
  a.tile = tile;
  a.wbits = wbits;
  a.lasers = d_lasers;
  a.beams = d_beams;
  a.offsets = d_offsets;
  a.samples = *samples;
  a.bins = *bins;
  a.ranges = d_ranges;
  a.shot = reinterpret_cast<Params*>(ws + bp.off_params);
  a.tiles = reinterpret_cast<int64_t*>(ws + bp.off_tiles);
  a.tables = ws + bp.off_tables;
  a.acc = reinterpret_cast<unsigned long long*>(ws + bp.off_acc);
  a.acc_smooth = bins->smooth_sigma_bins > 0
                     ? reinterpret_cast<unsigned long long*>(ws + bp.off_smooth)
                     : nullptr;
  a.acc_map = bins->n_tx > 0 ? reinterpret_cast<unsigned long long*>(ws + bp.off_map) : nullptr;
  a.acc_aeff = bins->n_aeff > 0 ? reinterpret_cast<unsigned long long*>(ws + bp.off_aeff) : nullptr;
  a.partials = reinterpret_cast<double*>(ws + bp.off_part);
  a.counter = reinterpret_cast<unsigned long long*>(ws + bp.off_counter);
  a.max_tiles = bp.max_tiles;
  a.precision = prec;
  // this context's cycle-resolved chi tables, built here on first use unless
  // the stream is being captured (then shots with that variant are invalid)
  {
    Params tp;
    const int32_t e = cycle_tables(tp, cs);
    if (e == QS_OK) {
      a.cyc_gl = tp.cyc_gl;
      a.cyc_a = tp.cyc_a;
      a.cyc_m = tp.cyc_m;
    } else if (e != QS_ERR_UNSUPPORTED) {
      return e;
    }
  }
  if (cudaMemsetAsync(ws + bp.off_counter, 0, 3 * 8, cs) != cudaSuccess) return cuda_fail();
  if (zero_acc && bp.off_part > bp.off_acc &&
      cudaMemsetAsync(ws + bp.off_acc, 0, bp.off_part - bp.off_acc, cs) != cudaSuccess)
    return cuda_fail();
  k_bsetup<<<(n_shots + 127) / 128, 128, 0, cs>>>(a);
  const int64_t cells = (int64_t)n_shots * max_phase;
  k_btable<<<(unsigned)((cells + 255) / 256), 256, 0, cs>>>(a);
  k_bscan<<<1, 1024, 0, cs>>>(a);
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

template <typename T>
int32_t launch_bgrad_kind(const BatchArgs& a, int block, int grid_req, int sms,
                          const qs_moments* mom, const double* dLdm, const double* dLdS,
                          cudaStream_t st, bool vark) {
  using TT = typename Tab<T>::type;
  const bool stage = dLdS && a.bins.smooth_sigma_bins > 0 && sizeof(T) == 4 &&
                     a.bins.n_bins <= kBGradStageBins;
  if (vark && block > 256) block = 256;
  const size_t smem = align_up(sizeof(Params), 16) + align_up((size_t)a.max_phase * sizeof(TT), 16) +
                      align_up((size_t)(block / 32) * kNumGrad * sizeof(double), 16) + 16 +
                      align_up(stage ? (size_t)a.bins.n_bins * sizeof(T) : 0, 16) +
                      (vark && sizeof(T) == 4 ? (size_t)2 * kCycN * sizeof(float4) : 0);
  if (smem > (size_t)kSmemLimit) return QS_ERR_UNSUPPORTED;
  auto kern = vark ? k_bgrad<T, true> : k_bgrad<T, false>;
  static CtxMark smem_mark[2];
  if (int32_t e = allow_smem(kern, smem_mark[vark ? 1 : 0], kSmemLimit)) return e;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess)
    return cuda_fail();
  const int grid = grid_req > 0 ? grid_req : sms * (occ > 0 ? occ : 1);
  kern<<<grid, block, smem, st>>>(a, mom, dLdm, dLdS);
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

template <typename T>
int32_t launch_bgrad(const BatchArgs& a, int block, int grid_req, int sms, const qs_moments* mom,
                     const double* dLdm, const double* dLdS, cudaStream_t st) {
  if (int32_t e = launch_bgrad_kind<T>(a, block, grid_req, sms, mom, dLdm, dLdS, st, false))
    return e;
  return launch_bgrad_kind<T>(a, block, grid_req, sms, mom, dLdm, dLdS, st, true);
}

}  // namespace

extern "C" int32_t qs_scatter_batch(int32_t n_shots, const qs_laser* d_lasers,
                                    const qs_beam* d_beams, const int64_t* d_offsets,
                                    const qs_samples* samples, const qs_bins* bins,
                                    const double* d_ranges, int32_t max_phase,
                                    const qs_exec* exec, double* d_spectra,
                                    double* d_spec_smooth, double* d_divmaps,
                                    double* d_aeff_hists, qs_moments* d_moments,
                                    void* d_workspace, size_t ws_bytes, void* stream) {
  int prec, wbits, block, grid, tile, sms;
  int32_t st = batch_checks(n_shots, samples, bins, max_phase, exec, &prec, &wbits, &block, &grid,
                            &tile);
  if (st) return st;
  if (!d_moments) return QS_ERR_INVALID_ARG;
  if (bins->n_bins > 0 && !d_spectra) return QS_ERR_INVALID_ARG;
  if (bins->smooth_sigma_bins > 0 && !d_spec_smooth) return QS_ERR_INVALID_ARG;
  if ((bins->n_tx > 0 && !d_divmaps) || (bins->n_aeff > 0 && !d_aeff_hists))
    return QS_ERR_INVALID_ARG;
  if (block > 256) block = 256;
  if ((st = device_sms(&sms))) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const bool check = exec_check_finite(exec);
  if (check && (st = sync_allowed(cs))) return st;
  BatchArgs a;
  if ((st = batch_prepare(a, n_shots, d_lasers, d_beams, d_offsets, samples, bins, d_ranges,
                          max_phase, prec, wbits, tile, d_workspace, ws_bytes, true, cs)))
    return st;
  if (prec == QS_F64)
    st = samples->w ? launch_batch<double, unsigned long long>(a, block, grid, sms, cs)
                    : launch_batch<double, unsigned int>(a, block, grid, sms, cs);
  else
    st = samples->w ? launch_batch<float, unsigned long long>(a, block, grid, sms, cs)
                    : launch_batch<float, unsigned int>(a, block, grid, sms, cs);
  if (st) return st;
  const int64_t thr = (int64_t)n_shots * 32;
  k_bfinal<<<(unsigned)((thr + 255) / 256), 256, 0, cs>>>(a, d_spectra, d_spec_smooth, d_divmaps,
                                                          d_aeff_hists, d_moments);
  if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
  return check ? nonfinite_status(&d_moments[0].nonfinite, n_shots, sizeof(qs_moments), cs)
               : QS_OK;
}

extern "C" int32_t qs_scatter_grad_batch(int32_t n_shots, const qs_laser* d_lasers,
                                         const qs_beam* d_beams, const int64_t* d_offsets,
                                         const qs_samples* samples, const qs_bins* bins,
                                         const double* d_ranges, int32_t max_phase,
                                         const qs_exec* exec, const qs_moments* d_moments,
                                         const double* d_dL_dmoments,
                                         const double* d_dL_dsmooth, double* d_grad,
                                         void* d_workspace, size_t ws_bytes, void* stream) {
  int prec, wbits, block, grid, tile, sms;
  int32_t st = batch_checks(n_shots, samples, bins, max_phase, exec, &prec, &wbits, &block, &grid,
                            &tile);
  if (st) return st;
  if (!d_moments || !d_dL_dmoments || !d_grad) return QS_ERR_INVALID_ARG;
  if (d_dL_dsmooth && !(bins->smooth_sigma_bins > 0)) return QS_ERR_INVALID_ARG;
  if ((st = device_sms(&sms))) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  // FP32 with the block left open: 512-thread CTAs (one per SM at the
  // adjoint's register count), as for the single-shot adjoint
  const int kblock = (!(exec && exec->block) && prec == QS_F32) ? 512 : block;
  // tile left open: the largest power of two up to 8192 samples that still
  // gives every resident CTA (one per SM) at least sixteen tiles: fewer shot
  // and table stagings and tile reductions per sample than the forward's
  // default 2048, and a last round of tiles short against the launch (256
  // shots of 2^16 samples: 4096-sample tiles, 0.800 of the FMA-pipe bound
  // against 0.785 with 8192)
  if (!(exec && exec->tile))
    while (tile < 8192 && samples->n / (2 * (int64_t)tile) >= 16 * (int64_t)sms) tile *= 2;
  BatchArgs a;
  if ((st = batch_prepare(a, n_shots, d_lasers, d_beams, d_offsets, samples, bins, d_ranges,
                          max_phase, prec, wbits, tile, d_workspace, ws_bytes, false, cs)))
    return st;
  st = prec == QS_F64
           ? launch_bgrad<double>(a, kblock, grid, sms, d_moments, d_dL_dmoments, d_dL_dsmooth, cs)
           : launch_bgrad<float>(a, kblock, grid, sms, d_moments, d_dL_dmoments, d_dL_dsmooth, cs);
  if (st) return st;
  const int64_t thr = (int64_t)n_shots * 32;
  k_bgfinal<<<(unsigned)((thr + 255) / 256), 256, 0, cs>>>(a, d_grad);
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

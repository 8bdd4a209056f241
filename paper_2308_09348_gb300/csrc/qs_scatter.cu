// qs_scatter.cu -- kernels and C ABI of libqscatter (single-shot path).
//
// K1 k_scatter   fused per-sample evaluation + integer histograms (shared
//                memory, merged into global with integer atomics) + FP64
//                moment partials per CTA, reduced in fixed lane/warp order.
// K2 k_finalize  one CTA: per-CTA partials summed in CTA order (compensated),
//                integer histograms converted to doubles, moments written.
// K0 k_eval      per-sample records (qs_eval_samples).
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348 (Secs. 2-5).
#include "qscatter.h"
#include "qs_device.cuh"
#include "qs_host.hpp"
#include "qs_derive.cuh"

#include <cuda.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

namespace qs {

// ---------------------------------------------------------------------------
// host: derived constants (shared with the gradient translation unit)
// ---------------------------------------------------------------------------
namespace detail {

int32_t validate_laser(const qs_laser* L) { return L ? check_laser(*L) : QS_ERR_INVALID_ARG; }
int32_t validate_beam(const qs_beam* B) { return B ? check_beam(*B) : QS_ERR_INVALID_ARG; }
int32_t validate_bins(const qs_bins* b) { return b ? check_bins(*b) : QS_ERR_INVALID_ARG; }

int32_t validate_samples(const qs_samples* s) {
  if (!s) return QS_ERR_INVALID_ARG;
  if (s->n < 0) return QS_ERR_INVALID_ARG;
  if (s->dtype != QS_F32 && s->dtype != QS_F64) return QS_ERR_INVALID_ARG;
  if (s->n == 0) return QS_OK;
  const uintptr_t esz = s->dtype == QS_F32 ? 4 : 8;
  for (int k = 0; k < 4; ++k)
    if (!s->xi[k]) return QS_ERR_INVALID_ARG;
  for (int k = 0; k < 8; ++k)
    if (s->xi[k] && ((uintptr_t)s->xi[k] % esz)) return QS_ERR_INVALID_ARG;
  if (s->w && ((uintptr_t)s->w % esz)) return QS_ERR_INVALID_ARG;
  return QS_OK;
}

int32_t exec_tile(const qs_exec* e, int* tile) {
  *tile = (e && e->tile) ? e->tile : 2048;
  if (*tile < 64 || *tile > (1 << 20) || (*tile % 64)) return QS_ERR_INVALID_ARG;
  return QS_OK;
}

int32_t exec_opts(const qs_exec* e, int* precision, int* wbits, int* block, int* grid) {
  *precision = e ? e->precision : QS_F32;
  *wbits = (e && e->weight_frac_bits) ? e->weight_frac_bits : 32;
  *block = (e && e->block) ? e->block : 256;
  *grid = e ? e->grid : 0;
  if (*precision != QS_F32 && *precision != QS_F64) return QS_ERR_INVALID_ARG;
  if (*wbits < 0 || *wbits > 52) return QS_ERR_INVALID_ARG;
  if (*block < 32 || *block > 512 || (*block % 32)) return QS_ERR_INVALID_ARG;
  if (*grid < 0) return QS_ERR_INVALID_ARG;
  if (e && (e->flags & ~QS_EXEC_CHECK_FINITE)) return QS_ERR_INVALID_ARG;
  return QS_OK;
}

bool exec_check_finite(const qs_exec* e) { return e && (e->flags & QS_EXEC_CHECK_FINITE); }

int32_t sync_allowed(cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return cuda_fail();
  return cap == cudaStreamCaptureStatusNone ? QS_OK : QS_ERR_UNSUPPORTED;
}

int32_t nonfinite_status(const double* d_nonfinite, int64_t count, size_t stride,
                         cudaStream_t st) {
  std::vector<double> h((size_t)(count > 0 ? count : 0));
  if (count > 0 && cudaMemcpy2DAsync(h.data(), sizeof(double), d_nonfinite, stride,
                                     sizeof(double), (size_t)count, cudaMemcpyDeviceToHost,
                                     st) != cudaSuccess)
    return cuda_fail();
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_fail();
  for (double v : h)
    if (v > 0.0) return QS_ERR_NONFINITE;
  return QS_OK;
}

void fill_params(Params& p, const qs_laser* L, const qs_beam* B, const qs_samples* S,
                 const qs_bins* b, int wbits) {
  derive_params(p, *L, *B, b, wbits);
  p.n = S->n;
  for (int i = 0; i < 8; ++i) p.xi[i] = S->xi[i];
  p.w = S->w;
  p.dtype = S->dtype;
  p.weighted = S->w != nullptr;
}

struct DevInfo {
  int sms = 0;
  bool init = false;
};
static std::mutex g_mu;
static DevInfo g_dev[64];

int32_t device_sms(int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return QS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev[dev].init) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return QS_ERR_CUDA;
    g_dev[dev].sms = v;
    g_dev[dev].init = true;
  }
  *sms = g_dev[dev].sms;
  return QS_OK;
}

// Driver entry points for the context key, resolved once through the
// runtime (no link-time dependency on the driver library).
namespace {
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);
std::once_flag g_ctx_once;
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
}  // namespace

int32_t current_context(int* dev, unsigned long long* key) {
  std::call_once(g_ctx_once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f);
    (void)cudaGetLastError();
  });
  if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= 64) return cuda_fail();
  if (!g_ctx_get_current || !g_ctx_get_id) return QS_ERR_CUDA;
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return QS_ERR_CUDA;
  if (!ctx) {
    // no context on this thread yet: cudaSetDevice makes the device's
    // primary context current
    if (cudaSetDevice(*dev) != cudaSuccess) return cuda_fail();
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return QS_ERR_CUDA;
  }
  unsigned long long id = 0;
  if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return QS_ERR_CUDA;
  *key = id + 1;
  return QS_OK;
}

// Workspace plan: u64 histogram accumulators (+ under/over/outside slots),
// then FP64 moment partials for the largest grid that can be resident.
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void make_plan(Plan& pl, const qs_bins* b, int block, int grid_req, int sms) {
  pl.nspec = b->n_bins > 0 ? (int64_t)b->n_bins + 2 : 0;
  pl.nmap = (b->n_tx > 0) ? (int64_t)b->n_tx * b->n_ty + 1 : 0;
  pl.naeff = b->n_aeff > 0 ? (int64_t)b->n_aeff + 1 : 0;
  pl.nsmooth = b->smooth_sigma_bins > 0 ? (int64_t)b->n_bins : 0;
  int64_t gmax = (int64_t)sms * (2048 / block < 32 ? 2048 / block : 32);
  if (grid_req > gmax) gmax = grid_req;
  pl.gmax = (int)gmax;
  size_t off = 0;
  pl.off_spec = off; off = align_up(off + (size_t)pl.nspec * 8, 256);
  pl.off_map = off;  off = align_up(off + (size_t)pl.nmap * 8, 256);
  pl.off_aeff = off; off = align_up(off + (size_t)pl.naeff * 8, 256);
  pl.off_smooth = off; off = align_up(off + (size_t)pl.nsmooth * 8, 256);
  pl.off_part = off; off = align_up(off + (size_t)gmax * kNumMom * 8, 256);
  pl.ws_bytes = off;
}

// Shared memory of k_scatter: phase table (QFP), reduction scratch, and the
// histograms when they are kept in shared memory.  The QFP model spends
// ~1000 cycles per sample, so its histograms go straight to global integer
// atomics (negligible traffic) and the freed shared memory buys occupancy;
// the LL model is memory-bound and keeps them in shared memory if they fit.
// cells: phase-table entries (QFP or the per-cell focus, 0 otherwise);
// variant: the model variant bits (histograms always global for a variant;
// FP32 cycle-resolved chi adds its Hermite tables).
Smem smem_plan(const Plan& pl, int precision, int cells, int variant, bool weighted, int block) {
  Smem sm;
  const bool cell_focus = variant != 0;
  // table entries: double G (FP64 path) or float4 {G, G, G^2, G^2} or
  // {G, G, s_j, s_j} (FP32 path); then the cycle tables (replicated)
  const size_t tab = align_up((size_t)cells * (precision == QS_F64 ? 8 : 16), 16) +
                     ((variant & QS_VARIANT_CYCLE_CHI) && precision == QS_F32
                          ? (size_t)2 * kCycN * kCycRep * sizeof(float4)
                          : 0);
  const size_t red = (size_t)(block / 32) * kNumMom * sizeof(double);
  const size_t hist = align_up((size_t)(pl.nspec + pl.nmap + pl.naeff) * (weighted ? 8 : 4), 16);
  sm.hist = !cell_focus && cells < 32 && tab + red + hist <= (size_t)kSmemLimit &&
            (pl.nspec + pl.nmap + pl.naeff) > 0;
  sm.bytes = tab + red + (sm.hist ? hist : 0);
  // smoothed-spectrum accumulators (u64) stay in shared memory when small
  sm.smooth = pl.nsmooth > 0 && pl.nsmooth * 8 <= 32 * 1024 && sm.bytes + pl.nsmooth * 8 <= (size_t)kSmemLimit;
  if (sm.smooth) sm.bytes += align_up((size_t)pl.nsmooth * 8, 16);
  return sm;
}

// Persistent grid: as many CTAs as fit on the device at once, never more
// than there are tiles of samples.
int pick_grid(int occ_per_sm, int sms, int block, int grid_req, int64_t n, int gmax) {
  int64_t g = grid_req > 0 ? grid_req : (int64_t)sms * (occ_per_sm > 0 ? occ_per_sm : 1);
  int64_t tiles = (n + block - 1) / block;
  if (tiles < 1) tiles = 1;
  if (g > tiles) g = tiles;
  if (g > gmax) g = gmax;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace detail

using namespace detail;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// K1: fused evaluation + histograms + moment partials.  T: per-sample
// arithmetic type; H: shared-memory histogram counter (u32 counts or u64
// fixed-point weights); QFP: model; SHIST: histograms in shared memory.
// VAR: model variant bits (kVarCell, kVarCycle).
// Register budget per thread: FP32 QFP and per-cell focus 72 (one
// 896-thread CTA per SM for the pipe-bound loop: at 64 registers and 1024
// threads the packed constants are re-materialised on the FMA pipe every
// cell, 4 % slower), FP32 cycle-resolved chi 80 (one 768-thread CTA per SM;
// it spills at 72), FP32 classical 80 (one 768-thread CTA per SM), FP64 128.
constexpr int scatter_regs(bool f64, bool qfp, int var) {
  return f64 ? 128 : ((var & kVarCycle) ? 80 : ((qfp || var != 0) ? 72 : 80));
}
template <typename T, bool QFP, int VAR>
constexpr int kScatterRegs = scatter_regs(sizeof(T) == 8, QFP, VAR);

// Block size of k_scatter when the caller leaves it open.  The FP32 paths
// that integrate phase cells are bound by the FMA and MUFU pipes.  CTAs that
// share an SM are served oldest first, so with four 256-thread CTAs per SM
// the first one finishes at ~40 % of the launch and the SM ends it with a
// quarter of its warps (22.9 of 32 warps resident on average).  One CTA per
// SM that fills the register file keeps every warp resident to the end:
// 896 threads at 72 registers, 768 at 80 (cycle-resolved chi).  The FP32
// classical path (HBM-bound) also runs one 768-thread CTA per SM: the same
// 24 warps as three 256-thread CTAs, but one shared-memory histogram set per
// SM to clear and merge instead of three, and no CTA finishing early
// (0.285 -> 0.251 ms on 2^26 samples).  The FP64 path keeps 256 threads.
int scatter_block(const qs_exec* e, int block, int prec, bool qfp, int variant) {
  if ((e && e->block) || prec != QS_F32) return block;
  if (!(qfp || (variant & QS_VARIANT_CELL_FOCUS))) return 768;
  const int regs = scatter_regs(false, qfp, variant);
  // warps are granted registers in groups of four
  const int b = ((65536 / (regs * 32)) & ~3) * 32;
  return b > 1024 ? 1024 : b;
}

// Shared memory of the phase table and, FP32 cycle-resolved chi, the cycle
// tables behind it (REP: replicated kCycRep times, as k_scatter reads them).
template <typename T, bool QFP, int VAR, bool REP = false>
__device__ __forceinline__ size_t table_bytes(const Params& p) {
  using TT = typename Tab<T>::type;
  constexpr bool cells = QFP || (VAR & kVarCell);
  constexpr bool cyc = sizeof(T) == 4 && (VAR & kVarCycle);
  return (cells ? (((size_t)p.n_phase * sizeof(TT) + 15) & ~(size_t)15) : 0) +
         (cyc ? (size_t)2 * kCycN * (REP ? kCycRep : 1) * sizeof(float4) : 0);
}
template <typename T, bool QFP, int VAR, bool REP = false>
__device__ __forceinline__ void load_tables(const Params& p, unsigned char* smem,
                                            const float4** cA) {
  using TT = typename Tab<T>::type;
  TT* tab = reinterpret_cast<TT*>(smem);
  if (QFP || (VAR & kVarCell))
    for (int j = threadIdx.x; j < p.n_phase; j += blockDim.x) table_entry(p, j, tab);
  if constexpr (sizeof(T) == 4 && (VAR & kVarCycle)) {
    float4* A = reinterpret_cast<float4*>(smem + (((size_t)p.n_phase * sizeof(TT) + 15) &
                                                  ~(size_t)15));
    // per-interval monomial coefficients of G, then of H
    constexpr int R = REP ? kCycRep : 1;
    for (int jc = threadIdx.x; jc < (kCycN - 1) * R; jc += blockDim.x) {
      const int j = jc / R, c = jc - j * R;
      A[j * R + c] = p.cyc_m[j];
      A[(kCycN + j) * R + c] = p.cyc_m[kCycN + j];
    }
    *cA = A + (REP ? (threadIdx.x % kCycRep) : 0);
  }
}

template <typename T, typename H, bool QFP, bool SHIST, int VAR>
__global__ void __maxnreg__((kScatterRegs<T, QFP, VAR>)) k_scatter(const Params p) {
  using TT = typename Tab<T>::type;
  constexpr bool LOC = (VAR & kVarCell) != 0;
  extern __shared__ __align__(16) unsigned char smem[];
  // FP32 cycle-resolved chi: replicated tables (kVarCycRep)
  constexpr bool REP = sizeof(T) == 4 && (VAR & kVarCycle) != 0;
  constexpr int VR = REP ? (VAR | kVarCycRep) : VAR;
  const size_t tab_bytes = table_bytes<T, QFP, VAR, REP>(p);
  TT* tab = reinterpret_cast<TT*>(smem);
  const float4* cA = nullptr;
  double* red = reinterpret_cast<double*>(smem + tab_bytes);
  H* sh = reinterpret_cast<H*>(smem + tab_bytes + (size_t)(blockDim.x >> 5) * kNumMom * sizeof(double));
  const int64_t nspec = p.n_bins > 0 ? (int64_t)p.n_bins + 2 : 0;
  const int64_t nmap = p.n_tx > 0 ? (int64_t)p.n_tx * p.n_ty + 1 : 0;
  const int64_t naeff = p.n_aeff > 0 ? (int64_t)p.n_aeff + 1 : 0;
  H* hs = sh;
  H* hm = sh + nspec;
  H* ha = sh + nspec + nmap;
  const size_t hist_bytes =
      SHIST ? (((size_t)(nspec + nmap + naeff) * sizeof(H) + 15) & ~(size_t)15) : 0;
  const int64_t nsm = p.smooth_sigma > 0.0 ? (int64_t)p.n_bins : 0;
  unsigned long long* ssm = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(sh) + hist_bytes);
  unsigned long long* hsm = nsm ? (p.smooth_in_smem ? ssm : p.acc_smooth) : nullptr;

  load_tables<T, QFP, VAR, REP>(p, smem, &cA);
  if (SHIST)
    for (int64_t b = threadIdx.x; b < nspec + nmap + naeff; b += blockDim.x) sh[b] = 0;
  if (nsm && p.smooth_in_smem)
    for (int64_t b = threadIdx.x; b < nsm; b += blockDim.x) ssm[b] = 0;
  __syncthreads();

  typename AccT<T>::type acc;
  acc_init(acc);

  // The loops advance warp by warp (bounds uniform across the lanes), so
  // that the smoothed deposits can run warp-cooperatively after each step.
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if constexpr (QFP && sizeof(T) == 4) {
    // FP32 QFP: each thread carries samples 2k and 2k+1 (packed f32x2)
    for (int64_t kb = t0 - lane; 2 * kb < p.n; kb += stride) {
      const int64_t k = kb + lane;
      const int64_t i0 = 2 * k, i1 = (2 * k + 1 < p.n) ? 2 * k + 1 : 2 * k;
      DepF d0, d1;
      bool ok0 = false, ok1 = false;
      if (i0 < p.n) {
        SampleF s0, s1;
        eval_pair_f32_qfp<VR>(p, reinterpret_cast<const float4*>(tab), i0, i1, s0, s1, cA);
        ok0 = accumulate<T, H, SHIST>(p, s0, i0, acc, hs, hm, ha, nspec, nmap, naeff);
        if (i1 != i0)
          ok1 = accumulate<T, H, SHIST>(p, s1, i1, acc, hs, hm, ha, nspec, nmap, naeff);
        dep_set(d0, s0);
        dep_set(d1, s1);
      }
      if (hsm) {
        deposit_warp(p, ok0, d0, i0, hsm);
        deposit_warp(p, ok1, d1, i1, hsm);
      }
    }
  } else {
    int64_t i = t0;
    if constexpr (!QFP && !LOC && sizeof(T) == 4) {
      // FP32 classical path (memory-bound): four consecutive samples per
      // thread through 16-byte loads of every stream, when all streams are
      // FP32 and 16-byte aligned and there is no smoothed spectrum; the
      // remaining samples below.
      bool vec = p.dtype == QS_F32 && hsm == nullptr;
      for (int c = 0; c < 6; ++c) vec = vec && p.xi[c] && ((uintptr_t)p.xi[c] & 15) == 0;
      if (p.weighted) vec = vec && ((uintptr_t)p.w & 15) == 0;
      if (vec) {
        const int64_t n4 = p.n >> 2;
        // two packed pairs per iteration; the moment contributions go to
        // packed partial sums, folded into the compensated sums every
        // kLLFold iterations (accumulate4_ll, ll_fold); unit weights and the
        // case with every histogram present are specialised
        const int ns = (int)nspec, nm = (int)nmap, na = (int)naeff;
        auto run = [&](auto weighted, auto all_hist) {
          constexpr bool W = decltype(weighted)::value;
          constexpr bool ALL = decltype(all_hist)::value;
          LLSums ts;
          ll_sums_zero(ts);
          int it = 0;
          for (int64_t k = t0; k < n4; k += stride) {
            float4 v[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) v[c] = __ldg(static_cast<const float4*>(p.xi[c]) + k);
            const float4 wv = W ? __ldg(static_cast<const float4*>(p.w) + k)
                                : make_float4(1.f, 1.f, 1.f, 1.f);
#define QS_LO2(c) make_float2(v[c].x, v[c].y)
#define QS_HI2(c) make_float2(v[c].z, v[c].w)
            const LL2 P0 = eval_ll_pair(p, QS_LO2(0), QS_LO2(1), QS_LO2(2), QS_LO2(3), QS_LO2(4),
                                        QS_LO2(5));
            const LL2 P1 = eval_ll_pair(p, QS_HI2(0), QS_HI2(1), QS_HI2(2), QS_HI2(3), QS_HI2(4),
                                        QS_HI2(5));
#undef QS_LO2
#undef QS_HI2
            accumulate4_ll<H, SHIST, W, ALL>(p, P0, P1, wv, ts, acc, hs, hm, ha, ns, nm, na);
            if (++it == kLLFold) {
              ll_fold(ts, acc);
              it = 0;
            }
          }
          ll_fold(ts, acc);
        };
        const bool all = nspec && nmap && naeff;
        if (p.weighted) {
          if (all) run(std::true_type{}, std::true_type{});
          else run(std::true_type{}, std::false_type{});
        } else {
          if (all) run(std::false_type{}, std::true_type{});
          else run(std::false_type{}, std::false_type{});
        }
        i = 4 * n4 + t0;
      }
    }
    for (int64_t ib = i - lane; ib < p.n; ib += stride) {
      const int64_t ii = ib + lane;
      typename DepT<T>::type d;
      bool ok = false;
      if (ii < p.n) {
        const auto s = eval_one<T, QFP, VR>(p, tab, ii, cA);
        ok = accumulate<T, H, SHIST>(p, s, ii, acc, hs, hm, ha, nspec, nmap, naeff);
        dep_set(d, s);
      }
      if (hsm) deposit_warp(p, ok, d, ii, hsm);
    }
  }
  block_reduce_write(acc, red, p.partials + (size_t)blockIdx.x * kNumMom);
  if (nsm && p.smooth_in_smem) {
    __syncthreads();
    for (int64_t b = threadIdx.x; b < nsm; b += blockDim.x)
      if (ssm[b]) atomicAdd(&p.acc_smooth[b], ssm[b]);
  }
  if (SHIST) {
    __syncthreads();
    for (int64_t b = threadIdx.x; b < nspec; b += blockDim.x)
      if (hs[b]) atomicAdd(&p.acc_spec[b], (unsigned long long)hs[b]);
    for (int64_t b = threadIdx.x; b < nmap; b += blockDim.x)
      if (hm[b]) atomicAdd(&p.acc_map[b], (unsigned long long)hm[b]);
    for (int64_t b = threadIdx.x; b < naeff; b += blockDim.x)
      if (ha[b]) atomicAdd(&p.acc_aeff[b], (unsigned long long)ha[b]);
  }
}

__global__ void __launch_bounds__(1024) k_finalize(const Params p, int grid, double* spectrum,
                                                   double* divmap, double* aeff_hist,
                                                   double* smooth, qs_moments* mom) {
  // Moment slots [0, grid) reduced in a fixed order: thread t merges the
  // contiguous slots [t*per, (t+1)*per) in order, then threads are merged by
  // a warp shuffle tree and warps in order.  (W, mean, M2) use the
  // parallel-variance merge; the other entries are compensated sums.
  __shared__ double tot[kNumMom];
  __shared__ double wred[32 * kNumMom];
  const double scale = p.weighted ? 1.0 / p.wscale : 1.0;
  {
    const int per = (grid + (int)blockDim.x - 1) / (int)blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(grid, b0 + per);
    double v[kNumMom] = {};
    double comp[kNumMom] = {};
    for (int b = b0; b < b1; ++b) {
      const double* q = p.partials + (size_t)b * kNumMom;
      welford_merge(v[0], v[1], v[2], q[0], q[1], q[2]);
      for (int k = 3; k < kNumMom; ++k) {
        const double x = q[k], t = v[k] + x;
        comp[k] += fabs(v[k]) >= fabs(x) ? (v[k] - t) + x : (x - t) + v[k];
        v[k] = t;
      }
    }
    for (int k = 3; k < kNumMom; ++k) v[k] += comp[k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
      double u[kNumMom];
      for (int k = 0; k < kNumMom; ++k) u[k] = __shfl_down_sync(0xffffffffu, v[k], o);
      welford_merge(v[0], v[1], v[2], u[0], u[1], u[2]);
      for (int k = 3; k < kNumMom; ++k) v[k] += u[k];
    }
    if (lane == 0)
      for (int k = 0; k < kNumMom; ++k) wred[warp * kNumMom + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
      double W = 0.0, m = 0.0, M2 = 0.0, sm[kNumMom] = {};
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        welford_merge(W, m, M2, wred[w * kNumMom], wred[w * kNumMom + 1], wred[w * kNumMom + 2]);
        for (int k = 3; k < kNumMom; ++k) sm[k] += wred[w * kNumMom + k];
      }
      tot[0] = W;
      tot[1] = m;
      tot[2] = M2;
      for (int k = 3; k < kNumMom; ++k) tot[k] = sm[k];
    }
  }
  for (int b = threadIdx.x; b < p.n_bins; b += blockDim.x)
    spectrum[b] = (double)p.acc_spec[b] * scale;
  const int64_t nmap = p.n_tx > 0 ? (int64_t)p.n_tx * p.n_ty : 0;
  for (int64_t b = threadIdx.x; b < nmap; b += blockDim.x) divmap[b] = (double)p.acc_map[b] * scale;
  for (int b = threadIdx.x; b < p.n_aeff; b += blockDim.x)
    aeff_hist[b] = (double)p.acc_aeff[b] * scale;
  if (p.smooth_sigma > 0.0)
    for (int b = threadIdx.x; b < p.n_bins; b += blockDim.x)
      smooth[b] = (double)p.acc_smooth[b] / p.wscale;
  __syncthreads();
  if (threadIdx.x == 0) {
    qs_moments m;
    const double W = tot[0];
    m.W = W;
    m.mean = m.spread = m.rel_spread = m.div_x = m.div_y = m.div = m.mean_aeff = 0.0;
    m.mean_gamma0 = 0.0;
    if (W > 0.0) {
      const double var = tot[2] / W + tot[3] / W;
      m.mean = tot[1];
      m.spread = sqrt(var > 0.0 ? var : 0.0);
      m.rel_spread = m.spread / m.mean;
      m.div_x = sqrt(tot[4] / W);
      m.div_y = sqrt(tot[5] / W);
      m.div = sqrt((tot[4] + tot[5]) / W);
      m.mean_aeff = tot[6] / W;
      m.mean_gamma0 = tot[7] / W;
    }
    m.under = p.n_bins > 0 ? (double)p.acc_spec[p.n_bins] * scale : 0.0;
    m.over = p.n_bins > 0 ? (double)p.acc_spec[p.n_bins + 1] * scale : 0.0;
    m.map_out = nmap ? (double)p.acc_map[nmap] * scale : 0.0;
    m.nonfinite = tot[8];
    *mom = m;
  }
}

__device__ __forceinline__ void write_record(const Params& p, const qs_sample_out& o,
                                             const Sample& s, int64_t i) {
  if (o.gamma0) o.gamma0[i] = s.gamma0;
  if (o.aeff) o.aeff[i] = s.aeff;
  if (o.mu) o.mu[i] = s.mu;
  if (o.V) o.V[i] = s.V;
  if (o.theta_e) o.theta_e[i] = s.theta_e;
  if (o.theta_x) o.theta_x[i] = s.tx;
  if (o.theta_y) o.theta_y[i] = s.ty;
  if (o.gamma_out) o.gamma_out[i] = s.gout;
  if (o.bin) o.bin[i] = p.n_bins > 0 ? energy_bin(p, s.gout) : -1;
  int ix = -1, iy = -1;
  if (p.n_tx > 0) map_cell(p, s.tx, s.ty, &ix, &iy);
  if (o.ix) o.ix[i] = ix;
  if (o.iy) o.iy[i] = iy;
  if (o.abin) o.abin[i] = p.n_aeff > 0 ? aeff_bin(p, s.aeff) : -1;
}

// FP32-path record: bins from the same FP32-path helpers as k_scatter.
__device__ __forceinline__ void write_record(const Params& p, const qs_sample_out& o,
                                             const SampleF& s, int64_t i) {
  if (o.gamma0) o.gamma0[i] = (double)s.g0;
  if (o.aeff) o.aeff[i] = (double)s.aeff;
  if (o.mu) o.mu[i] = (double)s.mu_hi + (double)s.mu_lo;
  if (o.V) o.V[i] = (double)s.V;
  if (o.theta_e) o.theta_e[i] = (double)s.theta_e;
  if (o.theta_x) o.theta_x[i] = (double)s.tx;
  if (o.theta_y) o.theta_y[i] = (double)s.ty;
  if (o.gamma_out) o.gamma_out[i] = (double)s.go_hi + (double)s.go_lo;
  if (o.bin) o.bin[i] = p.n_bins > 0 ? energy_bin_f32(p, s.go_hi, s.go_lo) : -1;
  int ix = -1, iy = -1;
  if (p.n_tx > 0) {
    const int c = map_cell_f32(p, s.tx, s.ty);
    if (c >= 0) {
      ix = c % p.n_tx;
      iy = c / p.n_tx;
    }
  }
  if (o.ix) o.ix[i] = ix;
  if (o.iy) o.iy[i] = iy;
  if (o.abin) o.abin[i] = p.n_aeff > 0 ? aeff_bin_f32(p, s.aeff) : -1;
}

// K0: per-sample records; the same per-sample code path as k_scatter.
template <typename T, bool QFP, int VAR>
__global__ void __launch_bounds__(256) k_eval(const Params p, qs_sample_out o) {
  using TT = typename Tab<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  TT* tab = reinterpret_cast<TT*>(smem);
  const float4* cA = nullptr;
  load_tables<T, QFP, VAR>(p, smem, &cA);
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (QFP && sizeof(T) == 4) {
    for (int64_t k = t0; 2 * k < p.n; k += stride) {
      const int64_t i0 = 2 * k, i1 = (2 * k + 1 < p.n) ? 2 * k + 1 : 2 * k;
      SampleF s0, s1;
      eval_pair_f32_qfp<VAR>(p, reinterpret_cast<const float4*>(tab), i0, i1, s0, s1, cA);
      write_record(p, o, s0, i0);
      if (i1 != i0) write_record(p, o, s1, i1);
    }
  } else {
    for (int64_t i = t0; i < p.n; i += stride)
      write_record(p, o, eval_one<T, QFP, VAR>(p, tab, i, cA), i);
  }
}

namespace {

// Cycle-resolved chi: the Gauss-Legendre rule and the FP32 Hermite tables,
// built once per device by k_cycle_setup (FP64) and kept for the process.
__device__ double g_cyc_gl[2 * kCycGL];
__device__ float4 g_cyc_a[kCycN];
__device__ float4 g_cyc_m[2 * kCycN];

// One CTA of kCycGL/2 threads: thread i finds the i-th root z of P_n (n =
// kCycGL) by Newton's method from cos(pi (i + 3/4)/(n + 1/2)) and its
// mirror; psi = (pi/4)(1 -+ z) on the quarter period, weight 2/((1 - z^2)
// P_n'(z)^2) times pi/4 times the 2/pi of the cycle mean.  Then the table
// nodes u_n = n du, chi_n = chi_s (2^u_n - 1): {G, dG/du du, H, dH/du du}
// (dchi/du = ln2 (chi + chi_s)); S comes from G's interpolant.  From the
// same FP64 node values, per interval n the cubic Hermite interpolants of G
// and H as monomial coefficients in t = u/du - n (c0 = v0, c1 = d0,
// c2 = 3 (v1 - v0) - 2 d0 - d1, c3 = 2 (v0 - v1) + d0 + d1), for the lookup
// by Horner's rule: entry n for G, kCycN + n for H.
__global__ void __launch_bounds__(kCycGL / 2) k_cycle_setup() {
  __shared__ double gl[2 * kCycGL];
  __shared__ double nv[4][kCycN];                    // G, dG du, H, dH du per node
  const int n = kCycGL, i = threadIdx.x;
  double z = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = 0.0;
    for (int k = 1; k <= n; ++k) {
      const double p2 = p1;
      p1 = p0;
      p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
    }
    dp = n * (z * p0 - p1) / (z * z - 1.0);
    const double dz = p0 / dp;
    z -= dz;
    if (fabs(dz) < 1e-16) break;
  }
  const double q = 0.25 * 3.14159265358979323846, w = 1.0 / ((1.0 - z * z) * dp * dp);
  gl[i] = cos(q * (1.0 - z));
  gl[n - 1 - i] = cos(q * (1.0 + z));
  gl[n + i] = w;
  gl[2 * n - 1 - i] = w;
  __syncthreads();
  for (int k = i; k < 2 * n; k += blockDim.x) g_cyc_gl[k] = gl[k];
  for (int m = i; m < kCycN; m += blockDim.x) {
    const double u = m * kCycDu, chi = kCycChiS * (exp2(u) - 1.0);
    const double dchi = 0.69314718055994530942 * (chi + kCycChiS) * kCycDu;
    double G, S, H, dG, dH;
    cycle_factors_d(gl, chi, G, S, H, &dG, nullptr, &dH);
    g_cyc_a[m] = make_float4((float)G, (float)(dG * dchi), (float)H, (float)(dH * dchi));
    nv[0][m] = G;
    nv[1][m] = dG * dchi;
    nv[2][m] = H;
    nv[3][m] = dH * dchi;
  }
  __syncthreads();
  for (int m = i; m < kCycN; m += blockDim.x) {
    if (m == kCycN - 1) {                            // past the last interval: never read
      g_cyc_m[m] = g_cyc_m[kCycN + m] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    for (int f = 0; f < 2; ++f) {
      const double v0 = nv[2 * f][m], d0 = nv[2 * f + 1][m];
      const double v1 = nv[2 * f][m + 1], d1 = nv[2 * f + 1][m + 1];
      g_cyc_m[f * kCycN + m] = make_float4((float)v0, (float)d0,
                                           (float)(3.0 * (v1 - v0) - 2.0 * d0 - d1),
                                           (float)(2.0 * (v0 - v1) + d0 + d1));
    }
  }
}

std::mutex g_cyc_mu;
CtxMark g_cyc_ready;

// Points p at the cycle tables, building them on first use in the device's
// current context (one launch on `st`, then a wait for it; not allowed while
// `st` is being captured into a graph).  A device reset discards the tables
// with the context, so the first use in the next context builds them again.
int32_t cycle_tables_impl(Params& p, cudaStream_t st) {
  int dev = 0;
  unsigned long long key = 0;
  if (int32_t e = current_context(&dev, &key)) return e;
  std::lock_guard<std::mutex> lk(g_cyc_mu);
  if (!g_cyc_ready.done(dev, key)) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return cuda_fail();
    if (cap != cudaStreamCaptureStatusNone) return QS_ERR_UNSUPPORTED;
    k_cycle_setup<<<1, kCycGL / 2, 0, st>>>();
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      return cuda_fail();
    g_cyc_ready.set(dev, key);
  }
  void *gl = nullptr, *a = nullptr, *mc = nullptr;
  if (cudaGetSymbolAddress(&gl, g_cyc_gl) != cudaSuccess ||
      cudaGetSymbolAddress(&a, g_cyc_a) != cudaSuccess ||
      cudaGetSymbolAddress(&mc, g_cyc_m) != cudaSuccess)
    return cuda_fail();
  p.cyc_gl = static_cast<const double*>(gl);
  p.cyc_a = static_cast<const float4*>(a);
  p.cyc_m = static_cast<const float4*>(mc);
  return QS_OK;
}

// k_eval with its dynamic shared memory (phase table) allowed up to the
// largest table.
template <typename T, bool QFP, int VAR>
int32_t launch_eval(int grid, size_t tb, cudaStream_t st, const Params& p,
                    const qs_sample_out& o) {
  auto kern = k_eval<T, QFP, VAR>;
  static CtxMark smem_mark;
  if (int32_t e = allow_smem(kern, smem_mark, kMaxPhase * (int)sizeof(float4) +
                                 2 * kCycN * (int)sizeof(float4))) return e;
  kern<<<grid, 256, tb, st>>>(p, o);
  return QS_OK;
}

template <typename T, typename H, bool QFP, bool SHIST, int VAR = 0>
int32_t launch_scatter_t(const Params& p, int block, size_t smem, int sms, int grid_req, int gmax,
                         cudaStream_t st, int* grid_out, const qs_exec* ex) {
  auto kern = k_scatter<T, H, QFP, SHIST, VAR>;
  static CtxMark smem_mark;
  if (int32_t e = allow_smem(kern, smem_mark, kSmemLimit)) return e;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess)
    return cuda_fail();
  const int grid = pick_grid(occ, sms, block, grid_req, p.n, gmax);
  if (ex && ex->ev_start &&
      cudaEventRecord(static_cast<cudaEvent_t>(ex->ev_start), st) != cudaSuccess)
    return QS_ERR_CUDA;
  kern<<<grid, block, smem, st>>>(p);
  *grid_out = grid;
  if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
  if (ex && ex->ev_stop &&
      cudaEventRecord(static_cast<cudaEvent_t>(ex->ev_stop), st) != cudaSuccess)
    return QS_ERR_CUDA;
  return QS_OK;
}

template <typename T>
int32_t launch_scatter_prec(const Params& p, bool qfp, const Smem& sm, int block, int sms,
                            int grid_req, int gmax, cudaStream_t st, int* g, const qs_exec* ex) {
  typedef unsigned int U32;
  typedef unsigned long long U64;
  const size_t b = sm.bytes;
  // model variants: global histograms (smem_plan)
  if (p.cycle && p.focus)
    return launch_scatter_t<T, U32, true, false, 3>(p, block, b, sms, grid_req, gmax, st, g, ex);
  if (p.cycle)
    return launch_scatter_t<T, U32, true, false, 2>(p, block, b, sms, grid_req, gmax, st, g, ex);
  if (p.focus) {
    if (qfp) return launch_scatter_t<T, U32, true, false, 1>(p, block, b, sms, grid_req, gmax, st, g, ex);
    return launch_scatter_t<T, U32, false, false, 1>(p, block, b, sms, grid_req, gmax, st, g, ex);
  }
  if (qfp) {
    if (!sm.hist) return launch_scatter_t<T, U32, true, false>(p, block, b, sms, grid_req, gmax, st, g, ex);
    return p.weighted ? launch_scatter_t<T, U64, true, true>(p, block, b, sms, grid_req, gmax, st, g, ex)
                      : launch_scatter_t<T, U32, true, true>(p, block, b, sms, grid_req, gmax, st, g, ex);
  }
  if (!sm.hist) return launch_scatter_t<T, U32, false, false>(p, block, b, sms, grid_req, gmax, st, g, ex);
  return p.weighted ? launch_scatter_t<T, U64, false, true>(p, block, b, sms, grid_req, gmax, st, g, ex)
                    : launch_scatter_t<T, U32, false, true>(p, block, b, sms, grid_req, gmax, st, g, ex);
}

}  // namespace

namespace detail {
int32_t cycle_tables(Params& p, cudaStream_t st) { return cycle_tables_impl(p, st); }
}  // namespace detail
}  // namespace qs

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace qs;

extern "C" int32_t qs_version(void) { return QS_VERSION; }

extern "C" const char* qs_status_string(int32_t s) {
  switch (s) {
    case QS_OK: return "ok";
    case QS_ERR_INVALID_ARG: return "invalid argument";
    case QS_ERR_CUDA: return "CUDA error";
    case QS_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case QS_ERR_UNSUPPORTED: return "unsupported";
    case QS_ERR_TIMEOUT: return "device-side wait timed out";
    case QS_ERR_NONFINITE: return "samples excluded as non-finite (outputs written)";
    default: return "unknown status";
  }
}

extern "C" size_t qs_workspace_bytes(const qs_bins* bins, const qs_exec* exec, int64_t n) {
  int prec, wbits, block, grid, sms;
  if (validate_bins(bins) != QS_OK || n < 0) return 0;
  if (exec_opts(exec, &prec, &wbits, &block, &grid) != QS_OK) return 0;
  if (device_sms(&sms) != QS_OK) return 0;
  Plan pl;
  make_plan(pl, bins, block, grid, sms);
  return pl.ws_bytes;
}

extern "C" int32_t qs_scatter(const qs_laser* laser, const qs_beam* beam,
                              const qs_samples* samples, const qs_bins* bins,
                              const qs_exec* exec, double* d_spectrum, double* d_divmap,
                              double* d_aeff_hist, double* d_spec_smooth, qs_moments* d_moments,
                              void* d_workspace, size_t ws_bytes, void* stream) {
  int32_t st;
  if ((st = validate_laser(laser)) || (st = validate_beam(beam)) ||
      (st = validate_samples(samples)) || (st = validate_bins(bins)))
    return st;
  int prec, wbits, block, grid, sms;
  if ((st = exec_opts(exec, &prec, &wbits, &block, &grid))) return st;
  if (!d_moments) return QS_ERR_INVALID_ARG;
  if (bins->n_bins > 0 && !d_spectrum) return QS_ERR_INVALID_ARG;
  if (bins->n_tx > 0 && !d_divmap) return QS_ERR_INVALID_ARG;
  if (bins->n_aeff > 0 && !d_aeff_hist) return QS_ERR_INVALID_ARG;
  if (bins->smooth_sigma_bins > 0 && !d_spec_smooth) return QS_ERR_INVALID_ARG;
  if ((st = device_sms(&sms))) return st;
  Plan pl;
  make_plan(pl, bins, block, grid, sms);
  if (!d_workspace || ((uintptr_t)d_workspace % 256) || ws_bytes < pl.ws_bytes)
    return QS_ERR_WORKSPACE;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const bool check = exec_check_finite(exec);
  if (check && (st = sync_allowed(cs))) return st;
  const bool qfp = laser->model == QS_MODEL_QFP;
  const bool cells = qfp || (laser->variant & QS_VARIANT_CELL_FOCUS) != 0;
  const int kblock = scatter_block(exec, block, prec, qfp, laser->variant);
  const Smem sm = smem_plan(pl, prec, cells ? laser->n_phase : 0, laser->variant,
                            samples->w != nullptr, kblock);

  Params p;
  fill_params(p, laser, beam, samples, bins, wbits);
  unsigned char* ws = static_cast<unsigned char*>(d_workspace);
  p.acc_spec = reinterpret_cast<unsigned long long*>(ws + pl.off_spec);
  p.acc_map = reinterpret_cast<unsigned long long*>(ws + pl.off_map);
  p.acc_aeff = reinterpret_cast<unsigned long long*>(ws + pl.off_aeff);
  p.acc_smooth = reinterpret_cast<unsigned long long*>(ws + pl.off_smooth);
  p.partials = reinterpret_cast<double*>(ws + pl.off_part);
  p.hist_in_smem = sm.hist ? 1 : 0;
  p.smooth_in_smem = sm.smooth ? 1 : 0;
  if ((laser->variant & QS_VARIANT_CYCLE_CHI) && (st = detail::cycle_tables(p, cs))) return st;

  if (cudaMemsetAsync(ws, 0, pl.off_part, cs) != cudaSuccess) return cuda_fail();
  int g = 1;
  if (prec == QS_F64)
    st = launch_scatter_prec<double>(p, qfp, sm, kblock, sms, grid, pl.gmax, cs, &g, exec);
  else
    st = launch_scatter_prec<float>(p, qfp, sm, kblock, sms, grid, pl.gmax, cs, &g, exec);
  if (st) return st;
  k_finalize<<<1, 1024, 0, cs>>>(p, g, d_spectrum, d_divmap, d_aeff_hist, d_spec_smooth,
                                 d_moments);
  if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
  return check ? nonfinite_status(&d_moments->nonfinite, 1, sizeof(qs_moments), cs) : QS_OK;
}

extern "C" int32_t qs_eval_samples(const qs_laser* laser, const qs_beam* beam,
                                   const qs_samples* samples, const qs_bins* bins,
                                   const qs_exec* exec, const qs_sample_out* out, void* stream) {
  int32_t st;
  if ((st = validate_laser(laser)) || (st = validate_beam(beam)) ||
      (st = validate_samples(samples)))
    return st;
  if (bins && (st = validate_bins(bins))) return st;
  if (!out) return QS_ERR_INVALID_ARG;
  int prec, wbits, block, grid, sms;
  if ((st = exec_opts(exec, &prec, &wbits, &block, &grid))) return st;
  if ((st = device_sms(&sms))) return st;
  if (samples->n == 0) return QS_OK;
  Params p;
  fill_params(p, laser, beam, samples, bins, wbits);
  int64_t tiles = (samples->n + 255) / 256;
  int g = (int)(tiles < (int64_t)sms * 8 ? tiles : (int64_t)sms * 8);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const bool qfp = laser->model == QS_MODEL_QFP;
  const int var = laser->variant;
  if ((var & QS_VARIANT_CYCLE_CHI) && (st = detail::cycle_tables(p, cs))) return st;
  const size_t tb = ((qfp || (var & QS_VARIANT_CELL_FOCUS))
                         ? (size_t)p.n_phase * (prec == QS_F64 ? sizeof(double) : sizeof(float4))
                         : 0) +
                    ((var & QS_VARIANT_CYCLE_CHI) && prec == QS_F32
                         ? (size_t)2 * kCycN * sizeof(float4)
                         : 0);
  int32_t est;
  if (prec == QS_F64) {
    switch (var) {
      case 1: est = qfp ? launch_eval<double, true, 1>(g, tb, cs, p, *out)
                        : launch_eval<double, false, 1>(g, tb, cs, p, *out); break;
      case 2: est = launch_eval<double, true, 2>(g, tb, cs, p, *out); break;
      case 3: est = launch_eval<double, true, 3>(g, tb, cs, p, *out); break;
      default: est = qfp ? launch_eval<double, true, 0>(g, tb, cs, p, *out)
                         : launch_eval<double, false, 0>(g, tb, cs, p, *out);
    }
  } else {
    switch (var) {
      case 1: est = qfp ? launch_eval<float, true, 1>(g, tb, cs, p, *out)
                        : launch_eval<float, false, 1>(g, tb, cs, p, *out); break;
      case 2: est = launch_eval<float, true, 2>(g, tb, cs, p, *out); break;
      case 3: est = launch_eval<float, true, 3>(g, tb, cs, p, *out); break;
      default: est = qfp ? launch_eval<float, true, 0>(g, tb, cs, p, *out)
                         : launch_eval<float, false, 0>(g, tb, cs, p, *out);
    }
  }
  if (est) return est;
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// qs_scatter_noalloc: the scratch space lives in a file-scope device array
// instead of a caller workspace (for callers that cannot allocate).
// ---------------------------------------------------------------------------
namespace qs {
namespace {

// Shared by every call on a device; held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QS_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};
CtxMark g_noalloc_mark;

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a stand-in for the symbol, never a device
// address, so it is looked up with the device current: once per device, and
// again when the device's context has changed (after a cudaDeviceReset the
// module, and the array with it, is loaded afresh in the new context).
int32_t noalloc_scratch(void** out) {
  int dev = 0;
  unsigned long long key = 0;
  if (int32_t e = current_context(&dev, &key)) return e;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_mark.done(dev, key)) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return cuda_fail();
    g_noalloc_ptr[dev] = p;
    g_noalloc_mark.set(dev, key);
  }
  *out = g_noalloc_ptr[dev];
  return QS_OK;
}

}  // namespace
}  // namespace qs

extern "C" int32_t qs_scatter_noalloc(const qs_laser* laser, const qs_beam* beam,
                                      const qs_samples* samples, const qs_bins* bins,
                                      const qs_exec* exec, double* d_spectrum, double* d_divmap,
                                      double* d_aeff_hist, double* d_spec_smooth,
                                      qs_moments* d_moments, void* stream) {
  // the size check comes first, so an oversized request fails before any
  // device set-up; qs_scatter then validates everything else
  if (validate_bins(bins) != QS_OK || !samples) return QS_ERR_INVALID_ARG;
  const size_t need = qs_workspace_bytes(bins, exec, samples->n);
  if (need == 0) return QS_ERR_INVALID_ARG;
  if (need > QS_NOALLOC_SCRATCH_BYTES) return QS_ERR_WORKSPACE;
  void* scratch = nullptr;
  int32_t st = noalloc_scratch(&scratch);
  if (st != QS_OK) return st;
  // qs_scatter zeroes the accumulators on the stream before its kernels run
  return qs_scatter(laser, beam, samples, bins, exec, d_spectrum, d_divmap, d_aeff_hist,
                    d_spec_smooth, d_moments, scratch, QS_NOALLOC_SCRATCH_BYTES, stream);
}

// ---------------------------------------------------------------------------
// qs_scatter_host: host-resident samples, chunked and double-buffered so
// that host-to-device copies overlap the evaluation kernel.
// ---------------------------------------------------------------------------
namespace qs {
namespace {

struct HostPipe {
  unsigned long long key = 0;      // context the stream and events belong to
  cudaStream_t copy = nullptr;
  cudaEvent_t start = nullptr, copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
};
std::mutex g_pipe_mu;
HostPipe g_pipe[64];

// The device's copy stream and events, created in the current context (a
// device reset destroys them with their context; the next call creates new
// ones).
int32_t host_pipe(HostPipe** out) {
  int dev = 0;
  unsigned long long key = 0;
  if (int32_t e = current_context(&dev, &key)) return e;
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe& hp = g_pipe[dev];
  if (hp.key != key) {
    if (cudaStreamCreateWithFlags(&hp.copy, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail();
    cudaEvent_t* evs[5] = {&hp.start, &hp.copied[0], &hp.copied[1], &hp.consumed[0], &hp.consumed[1]};
    for (cudaEvent_t* e : evs)
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return cuda_fail();
    hp.key = key;
  }
  *out = &hp;
  return QS_OK;
}

struct HostPlan {
  Plan pl;               // accumulators; partial slots for n_chunks * gmax CTAs
  int64_t chunk = 0, n_chunks = 0;
  int64_t wave = 0;      // automatic schedule: first chunk, growth x3 up to chunk
  int n_streams = 0;     // present sample streams (+ weights)
  size_t esz = 4, off_out = 0, off_stage = 0, stage_bytes = 0, bytes = 0;
  size_t out_spec = 0, out_map = 0, out_aeff = 0, out_smooth = 0, out_mom = 0;
};

// Automatic chunking (chunk = 0): whole waves of the FP32 cell-integrating
// launch (two samples per thread, one scatter_block-sized CTA per SM), so that no
// chunk ends on a partly idle pass over the grid; the first chunk is one
// wave and each next one three times the last, up to 2^23 samples, so the
// copy of chunk c+1 (~4x faster per sample than its evaluation) hides
// behind chunk c from the start.
int64_t next_chunk(const HostPlan& hp, int64_t last) {
  if (!hp.wave) return hp.chunk;
  if (last == 0) return hp.wave;
  return last * 3 < hp.chunk ? last * 3 : hp.chunk;
}

bool host_plan(HostPlan& hp, const qs_bins* b, int block, int grid, int sms,
               const qs_samples* s, int64_t chunk) {
  if (chunk > 0) {
    hp.chunk = chunk;
    hp.wave = 0;
  } else {
    hp.wave = (int64_t)2 * scatter_block(nullptr, 0, QS_F32, true, 0) * sms;
    const int64_t cap = ((int64_t)1 << 23) / hp.wave;
    hp.chunk = (cap > 0 ? cap : 1) * hp.wave;
  }
  if (hp.chunk % 1024) return false;
  hp.n_chunks = 0;
  for (int64_t left = s->n, len = 0; left > 0; left -= len, ++hp.n_chunks)
    len = next_chunk(hp, len);
  make_plan(hp.pl, b, block, grid, sms);
  // partial slots for every chunk's CTAs (the plan's region holds one chunk)
  const size_t part_bytes = (size_t)(hp.n_chunks > 0 ? hp.n_chunks : 1) * hp.pl.gmax * kNumMom * 8;
  size_t off = hp.pl.off_part + align_up(part_bytes, 256);
  hp.off_out = off;
  hp.out_spec = off; off = align_up(off + (size_t)(b->n_bins > 0 ? b->n_bins : 0) * 8, 256);
  hp.out_map = off;  off = align_up(off + (size_t)(b->n_tx > 0 ? (int64_t)b->n_tx * b->n_ty : 0) * 8, 256);
  hp.out_aeff = off; off = align_up(off + (size_t)(b->n_aeff > 0 ? b->n_aeff : 0) * 8, 256);
  hp.out_smooth = off; off = align_up(off + (size_t)(b->smooth_sigma_bins > 0 ? b->n_bins : 0) * 8, 256);
  hp.out_mom = off;  off = align_up(off + sizeof(qs_moments), 256);
  hp.esz = s->dtype == QS_F32 ? 4 : 8;
  hp.n_streams = 0;
  for (int k = 0; k < 8; ++k) hp.n_streams += s->xi[k] ? 1 : 0;
  hp.n_streams += s->w ? 1 : 0;
  hp.stage_bytes = align_up((size_t)hp.chunk * hp.esz, 256);
  hp.off_stage = off;
  off += 2 * (size_t)hp.n_streams * hp.stage_bytes;
  hp.bytes = off;
  return true;
}

}  // namespace
}  // namespace qs

extern "C" size_t qs_host_workspace_bytes(const qs_bins* bins, const qs_exec* exec,
                                          const qs_samples* h_samples, int64_t chunk) {
  int prec, wbits, block, grid, sms;
  if (validate_bins(bins) != QS_OK || validate_samples(h_samples) != QS_OK) return 0;
  if (exec_opts(exec, &prec, &wbits, &block, &grid) != QS_OK) return 0;
  if (device_sms(&sms) != QS_OK) return 0;
  HostPlan hp;
  if (!host_plan(hp, bins, block, grid, sms, h_samples, chunk)) return 0;
  return hp.bytes;
}

extern "C" int32_t qs_scatter_host(const qs_laser* laser, const qs_beam* beam,
                                   const qs_samples* h_samples, const qs_bins* bins,
                                   const qs_exec* exec, int64_t chunk, double* h_spectrum,
                                   double* h_divmap, double* h_aeff_hist, double* h_spec_smooth,
                                   qs_moments* h_moments, void* d_workspace, size_t ws_bytes,
                                   void* stream) {
  int32_t st;
  if ((st = validate_laser(laser)) || (st = validate_beam(beam)) ||
      (st = validate_samples(h_samples)) || (st = validate_bins(bins)))
    return st;
  int prec, wbits, block, grid, sms;
  if ((st = exec_opts(exec, &prec, &wbits, &block, &grid))) return st;
  if (!h_moments) return QS_ERR_INVALID_ARG;
  if (bins->n_bins > 0 && !h_spectrum) return QS_ERR_INVALID_ARG;
  if (bins->n_tx > 0 && !h_divmap) return QS_ERR_INVALID_ARG;
  if (bins->n_aeff > 0 && !h_aeff_hist) return QS_ERR_INVALID_ARG;
  if (bins->smooth_sigma_bins > 0 && !h_spec_smooth) return QS_ERR_INVALID_ARG;
  if (chunk < 0) return QS_ERR_INVALID_ARG;
  if ((st = device_sms(&sms))) return st;
  HostPlan hp;
  if (!host_plan(hp, bins, block, grid, sms, h_samples, chunk)) return QS_ERR_INVALID_ARG;
  if (!d_workspace || ((uintptr_t)d_workspace % 256) || ws_bytes < hp.bytes)
    return QS_ERR_WORKSPACE;
  const bool check = exec_check_finite(exec);
  if (check && (st = sync_allowed(static_cast<cudaStream_t>(stream)))) return st;
  HostPipe* pipe = nullptr;
  if ((st = host_pipe(&pipe))) return st;
  const bool qfp = laser->model == QS_MODEL_QFP;
  const bool cells = qfp || (laser->variant & QS_VARIANT_CELL_FOCUS) != 0;
  const int kblock = scatter_block(exec, block, prec, qfp, laser->variant);
  const Smem sm = smem_plan(hp.pl, prec, cells ? laser->n_phase : 0, laser->variant,
                            h_samples->w != nullptr, kblock);
  unsigned char* ws = static_cast<unsigned char*>(d_workspace);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  Params p;
  fill_params(p, laser, beam, h_samples, bins, wbits);
  if ((laser->variant & QS_VARIANT_CYCLE_CHI) && (st = detail::cycle_tables(p, cs))) return st;
  p.acc_spec = reinterpret_cast<unsigned long long*>(ws + hp.pl.off_spec);
  p.acc_map = reinterpret_cast<unsigned long long*>(ws + hp.pl.off_map);
  p.acc_aeff = reinterpret_cast<unsigned long long*>(ws + hp.pl.off_aeff);
  p.acc_smooth = reinterpret_cast<unsigned long long*>(ws + hp.pl.off_smooth);
  p.hist_in_smem = sm.hist ? 1 : 0;
  p.smooth_in_smem = sm.smooth ? 1 : 0;
  double* part0 = reinterpret_cast<double*>(ws + hp.pl.off_part);

  // accumulators and every partial slot start at zero; copies wait for the
  // caller's earlier work on `stream` (it may still use the workspace)
  if (cudaMemsetAsync(ws, 0, hp.off_out, cs) != cudaSuccess) return cuda_fail();
  if (cudaEventRecord(pipe->start, cs) != cudaSuccess) return cuda_fail();
  if (cudaStreamWaitEvent(pipe->copy, pipe->start, 0) != cudaSuccess) return cuda_fail();

  const void* hsrc[9];
  int ns = 0;
  for (int k = 0; k < 8; ++k)
    if (h_samples->xi[k]) hsrc[ns++] = h_samples->xi[k];
  if (h_samples->w) hsrc[ns++] = h_samples->w;
  int64_t i0 = 0, len = 0;
  for (int64_t c = 0; c < hp.n_chunks; ++c, i0 += len) {
    const int b = (int)(c & 1);
    len = next_chunk(hp, len);
    const int64_t cn = (h_samples->n - i0) < len ? (h_samples->n - i0) : len;
    unsigned char* stage = ws + hp.off_stage + (size_t)b * hp.n_streams * hp.stage_bytes;
    if (c >= 2 && cudaStreamWaitEvent(pipe->copy, pipe->consumed[b], 0) != cudaSuccess)
      return cuda_fail();
    for (int k = 0; k < ns; ++k)
      if (cudaMemcpyAsync(stage + (size_t)k * hp.stage_bytes,
                          static_cast<const unsigned char*>(hsrc[k]) + (size_t)i0 * hp.esz,
                          (size_t)cn * hp.esz, cudaMemcpyHostToDevice, pipe->copy) != cudaSuccess)
        return cuda_fail();
    if (cudaEventRecord(pipe->copied[b], pipe->copy) != cudaSuccess) return cuda_fail();
    if (cudaStreamWaitEvent(cs, pipe->copied[b], 0) != cudaSuccess) return cuda_fail();
    // point the launch at the staged chunk
    Params pc = p;
    pc.n = cn;
    int k2 = 0;
    for (int k = 0; k < 8; ++k)
      pc.xi[k] = h_samples->xi[k] ? stage + (size_t)(k2++) * hp.stage_bytes : nullptr;
    pc.w = h_samples->w ? stage + (size_t)(k2++) * hp.stage_bytes : nullptr;
    pc.partials = part0 + (size_t)c * hp.pl.gmax * kNumMom;
    int g = 1;
    const qs_exec* ex = (c == 0) ? exec : nullptr;
    if (prec == QS_F64)
      st = launch_scatter_prec<double>(pc, qfp, sm, kblock, sms, grid, hp.pl.gmax, cs, &g, ex);
    else
      st = launch_scatter_prec<float>(pc, qfp, sm, kblock, sms, grid, hp.pl.gmax, cs, &g, ex);
    if (st) return st;
    if (cudaEventRecord(pipe->consumed[b], cs) != cudaSuccess) return cuda_fail();
  }
  // finalize over every chunk's slots, in chunk then CTA order
  p.partials = part0;
  double* d_spec = reinterpret_cast<double*>(ws + hp.out_spec);
  double* d_map = reinterpret_cast<double*>(ws + hp.out_map);
  double* d_aeff = reinterpret_cast<double*>(ws + hp.out_aeff);
  double* d_smooth = reinterpret_cast<double*>(ws + hp.out_smooth);
  qs_moments* d_mom = reinterpret_cast<qs_moments*>(ws + hp.out_mom);
  const int slots = (int)((hp.n_chunks > 0 ? hp.n_chunks : 1) * hp.pl.gmax);
  k_finalize<<<1, 1024, 0, cs>>>(p, slots, d_spec, d_map, d_aeff, d_smooth, d_mom);
  if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
  // results to the host
  struct Out { void* h; const void* d; size_t n; } outs[5] = {
      {h_spectrum, d_spec, (size_t)(bins->n_bins > 0 ? bins->n_bins : 0) * 8},
      {h_divmap, d_map, (size_t)(bins->n_tx > 0 ? (int64_t)bins->n_tx * bins->n_ty : 0) * 8},
      {h_aeff_hist, d_aeff, (size_t)(bins->n_aeff > 0 ? bins->n_aeff : 0) * 8},
      {h_spec_smooth, d_smooth, (size_t)(bins->smooth_sigma_bins > 0 ? bins->n_bins : 0) * 8},
      {h_moments, d_mom, sizeof(qs_moments)}};
  for (const Out& o : outs)
    if (o.n && cudaMemcpyAsync(o.h, o.d, o.n, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
      return cuda_fail();
  if (check) {
    if (cudaStreamSynchronize(cs) != cudaSuccess) return cuda_fail();
    if (h_moments->nonfinite > 0.0) return QS_ERR_NONFINITE;
  }
  return QS_OK;
}

// qs_photon.cu -- photon spectrum of the beam (qs_photon_spectrum).
//
// K6 k_photon_setup  once per device: Hermite table (FP64-built) of the two
//                    Bessel functions of the synchrotron spectrum.
// K7 k_photon        per sample: the quantum model's phase integration; in
//                    every cell the locally-constant-field quantum-
//                    synchrotron spectrum at the cell's (mu, chi) is added
//                    to the photon-energy bins, warp-cooperatively (each
//                    lane owns bins b = lane + 32 k and takes the warp's 64
//                    emitters of the cell one at a time); per-CTA partials in
//                    fixed order.
// K8 k_photon_final  one CTA: partials summed in CTA order.
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348, Sec. 4 (cumulative
// photon spectrum from the mean energy along the phase and the local field;
// the LCFA spectrum the paper names, in its standard form, is stated with
// qs_photon_spectrum in qscatter.h).
#include "qscatter.h"
#include "qs_device.cuh"
#include "qs_host.hpp"

#include <cmath>
#include <mutex>
#include <type_traits>

namespace qs {

constexpr int kPhMaxBins = 512;               // photon-energy bins (16 per lane)
constexpr int kPhN = 256;                     // table nodes in u = log2 y (du = 0.18: lanes on
                                              // consecutive log-spaced bins share nodes)
constexpr double kPhUmin = -40.0, kPhUmax = 6.0;
constexpr double kPhDu = (kPhUmax - kPhUmin) / (kPhN - 1);
constexpr double kPhYmax = 60.0;              // F ~ e^-y: photons beyond are dropped
constexpr double kAlpha = 7.2973525693e-3;    // fine-structure constant (CODATA 2018)
constexpr double kLog2e = 1.4426950408889634074;

// K_{2/3}(y), Ki_{1/3}(y) = int_y^inf K_{1/3}, and the derivatives -K_{2/3}'
// and K_{1/3} (= -Ki_{1/3}'), from K_nu(y) = int_0^inf exp(-y cosh t)
// cosh(nu t) dt by the trapezoidal rule (step 1/32 until y cosh t > 800):
// the integrands are analytic in a strip and decay doubly exponentially.
__device__ void bessel_d(double y, double& k23, double& ki13, double* mk23p = nullptr,
                         double* k13 = nullptr) {
  const double dt = 1.0 / 32.0;
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
  for (int k = 0;; ++k) {
    const double t = k * dt, ch = cosh(t), e = exp(-y * ch);
    const double wt = k == 0 ? 0.5 : 1.0;
    const double c23 = cosh(2.0 * t / 3.0), c13 = cosh(t / 3.0);
    a += wt * e * c23;
    b += wt * e * c13 / ch;
    c += wt * e * c23 * ch;
    d += wt * e * c13;
    if (y * ch > 800.0 || t > 60.0) break;
  }
  k23 = dt * a;
  ki13 = dt * b;
  if (mk23p) *mk23p = dt * c;
  if (k13) *k13 = dt * d;
}

// Table node values at u_n = umin + n du, y = 2^u, of the two Bessel
// functions with the large-y exponential taken out: T23 = K_{2/3}(y) e^y and
// T13 = -Ki_{1/3}(y) e^y (smooth in u: a power of y at small y, y^-1/2 at
// large y), with their u-derivatives.  The FP32 table holds, per interval
// [u_n, u_n+1], the cubic Hermite interpolant of each as monomial
// coefficients in t = (u - u_n)/du:  p(t) = c0 + t (c1 + t (c2 + t c3)),
//   c0 = v0, c1 = d0, c2 = 3 (v1 - v0) - 2 d0 - d1, c3 = 2 (v0 - v1) + d0 + d1
// (d = dv/du du), computed in FP64: entry n for T23, kPhN + n for T13 (two
// separate arrays, so that the ~16 consecutive intervals a warp's lanes
// read are contiguous: two conflict-free wavefronts per gather).
__device__ float4 g_ph_tab[2 * kPhN];

__device__ void photon_node(int m, double& v23, double& d23, double& v13, double& d13) {
  const double u = kPhUmin + m * kPhDu, y = exp2(u), ey = exp(y);
  double k23, ki13, mk23p, k13;
  bessel_d(y, k23, ki13, &mk23p, &k13);
  const double dydu = y * 0.69314718055994530942 * kPhDu;   // dy/du du
  v23 = k23 * ey;
  d23 = (k23 - mk23p) * ey * dydu;          // d(K e^y)/dy = (K' + K) e^y
  v13 = -ki13 * ey;
  d13 = -(ki13 - k13) * ey * dydu;          // Ki' = -K_{1/3}
}

__device__ __forceinline__ float4 hermite_coeffs(double v0, double d0, double v1, double d1) {
  return make_float4((float)v0, (float)d0, (float)(3.0 * (v1 - v0) - 2.0 * d0 - d1),
                     (float)(2.0 * (v0 - v1) + d0 + d1));
}

__global__ void __launch_bounds__(256) k_photon_setup() {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < kPhN; m += gridDim.x * blockDim.x) {
    if (m == kPhN - 1) {                      // past the last interval: never read
      g_ph_tab[m] = g_ph_tab[kPhN + m] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    double a0, a1, b0, b1, e0, e1, f0, f1;    // T23, d23 at nodes m, m+1; T13, d13
    photon_node(m, a0, a1, b0, b1);
    photon_node(m + 1, e0, e1, f0, f1);
    g_ph_tab[m] = hermite_coeffs(a0, a1, e0, e1);
    g_ph_tab[kPhN + m] = hermite_coeffs(b0, b1, f0, f1);
  }
}

// FP32: F(xi, chi) = (1 - xi + 1/(1 - xi)) K_{2/3}(y) - Ki_{1/3}(y)
//   = e^-y ((1 - xi + 1/(1 - xi)) T23 + T13)
// from the table (cubic in u by Horner's rule) and one ex2; y in (0, ymax].
__device__ __forceinline__ float horner(float t, float4 c) {
  return __fmaf_rn(__fmaf_rn(__fmaf_rn(c.w, t, c.z), t, c.y), t, c.x);
}

// Two photon energies e (two bins of one lane) against one emitter whose
// {1/mu, 1/mu, 2/(3 chi), 2/(3 chi)} is pq: F for both, packed f32x2 except
// the table gathers and the Horner sums.  Bins beyond the emitter's cut
// (y > ymax, or xi >= 1) give finite or NaN values that the caller discards;
// their table index stays in range (the saturated coordinate is in [0, 1]).
__device__ __forceinline__ float2 synch_F2(const float4* __restrict__ T, float2 e, float4 pq) {
  constexpr float kS = (float)(kPhN - 1) - 1e-3f;            // x = s kS in [0, kPhN - 1)
  const float2 xi = mul2(e, make_float2(pq.x, pq.y));
  const float2 om = fma2(xi, f2(-1.f), f2(1.f));                      // 1 - xi
  const float2 r1 = rcpx2(om);
  const float2 y = mul2(mul2(make_float2(pq.z, pq.w), xi), r1);
  const float2 u = lg2x2(y);
  // x = (u - umin)/du clamped to [0, kS]: s = (u - umin)/(du kS) saturated
  // to [0, 1], then x = s kS
  const float sa = (float)(1.0 / (kPhDu * kS)), sb = (float)(-kPhUmin / (kPhDu * kS));
  const float2 sx = make_float2(fma_sat(u.x, sa, sb), fma_sat(u.y, sa, sb));
  // node index for x = s kS: x - 1/2 (rounded once, within 2^-17) rounded
  // to the nearest integer by adding 1.5 2^23 (the sum lies in [2^23, 2^24),
  // where the float spacing is 1), so the index is in [0, kPhN - 2] and
  // t = x - index (one rounding of the exact difference) in [0, 1] up to
  // 2^-17
  const float2 xm = __fadd2_rn(fma2(sx, f2(kS), f2(-0.5f)), f2(12582912.f));
  const int i0 = __float_as_int(xm.x) - 0x4B400000, i1 = __float_as_int(xm.y) - 0x4B400000;
  const float2 t = fma2(sx, f2(kS), fma2(xm, f2(-1.f), f2(12582912.f)));
  const float2 k23 = make_float2(horner(t.x, T[i0]), horner(t.y, T[i1]));   // K_{2/3} e^y
  const float2 nk13 =
      make_float2(horner(t.x, T[kPhN + i0]), horner(t.y, T[kPhN + i1]));     // -Ki_{1/3} e^y
  const float2 emy = ex2x2(mul2(y, f2((float)(-kLog2e))));               // e^-y
  return mul2(emy, fma2(__fadd2_rn(om, r1), k23, nk13));
}

// FP64: the same F from the integrals.
__device__ __forceinline__ double synch_F_d(double xi, double y) {
  double k23, ki13;
  bessel_d(y, k23, ki13);
  return (1.0 - xi + 1.0 / (1.0 - xi)) * k23 - ki13;
}

// Angular moments (Eq. 7): photons leave along the emitting electron's
// direction, in cell j its initial angle plus the transverse oscillation in
// the linearly polarised field (rms A_j/(sqrt2 mu_j) along x, the
// polarisation axis), within the emission cone ~1/mu_j per axis:
//   theta_x^2 = thx0^2 + A_j^2/(2 mu_j^2) + 1/mu_j^2,
//   theta_y^2 = thy0^2 + 1/mu_j^2,
// with A_j/mu_j = chi_j/(cchi mu_j^2) (chi = cchi A mu).  With ANG the
// kernel also sums the rates times these into T_x, T_y per bin.
constexpr int kPhMaxBinsAng = 256;

// Per-lane bin accumulators (NA = 3 sets with ANG: S, T_x, T_y): compensated
// FP32 sums (FP32 path), FP64 sums.
template <typename T, bool ANG, int KB> struct PhAcc;
template <bool ANG, int KB> struct PhAcc<float, ANG, KB> {
  static constexpr int NA = ANG ? 3 : 1, K = KB;
  float s[NA][K], c[NA][K];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int m = 0; m < NA; ++m)
#pragma unroll
      for (int k = 0; k < K; ++k) s[m][k] = c[m][k] = 0.f;
  }
  __device__ __forceinline__ void add(int m, int k, float x) { kahan(s[m][k], c[m][k], x); }
  __device__ __forceinline__ double get(int m, int k) const {
    return (double)s[m][k] - (double)c[m][k];
  }
};
// FP32: the compensated sums in shared memory instead of registers, one
// {sum, compensation} float pair per (warp, set, bin), in the 8-byte slots
// of the CTA's per-warp partial spectra (which are written only after the
// sums are final, by the same lane, at the same address).
template <bool ANG, int KB> struct PhAccSm {
  static constexpr int NA = ANG ? 3 : 1, K = KB;
  float2* slot;    // this warp's part[(warp * NA + m) * nb + b] viewed as float2
  int nb, lane;
  __device__ __forceinline__ void init(double* part_warp, int nb_, int lane_) {
    slot = reinterpret_cast<float2*>(part_warp);
    nb = nb_;
    lane = lane_;
#pragma unroll
    for (int m = 0; m < NA; ++m)
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (32 * k + lane < nb) slot[m * nb + 32 * k + lane] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void add(int m, int k, float x) {
    if (32 * k + lane >= nb) return;       // lanes past the last bin own no slot
    float2 v = slot[m * nb + 32 * k + lane];
    kahan(v.x, v.y, x);
    slot[m * nb + 32 * k + lane] = v;
  }
  __device__ __forceinline__ double get(int m, int k) const {
    const float2 v = slot[m * nb + 32 * k + lane];
    return (double)v.x - (double)v.y;
  }
};
template <bool ANG, int KB> struct PhAcc<double, ANG, KB> {
  static constexpr int NA = ANG ? 3 : 1, K = KB;
  double s[NA][K];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int m = 0; m < NA; ++m)
#pragma unroll
      for (int k = 0; k < K; ++k) s[m][k] = 0.0;
  }
  __device__ __forceinline__ void add(int m, int k, double x) { s[m][k] += x; }
  __device__ __forceinline__ double get(int m, int k) const { return s[m][k]; }
};

// FP32 emitter of one cell: {1/mu, 2/(3 chi), eps cut where y = ymax, c}
// (a zero cut when c = 0: nothing emitted).
__device__ __forceinline__ float4 emitter(float mu, float chi, float c) {
  if (!(c > 0.f)) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float yc = __fmul_rn(__fmul_rn(1.5f, chi), (float)kPhYmax);
  const float cut = __fmul_rn(__fmul_rn(mu, yc), M<float>::rcp(__fadd_rn(1.f, yc)));
  return make_float4(M<float>::rcp(mu), M<float>::rcp(__fmul_rn(1.5f, chi)), cut, c);
}

// FP32 path: the per-thread state of the sample pair (the pair's constants
// and the scheme's state, weights and initial angles) lives in shared
// memory between cells, one float per field and thread (field-major, so
// that a warp's accesses are conflict-free): only the bin sums and the
// evaluation itself then occupy registers in the bin loop.
//   0-5   c1, ca, ig0 (PairConst, two lanes each)   6-11  du, V, gph (PairState)
//   12-13 w0, w1      14-17 tx0, ty0, tx1, ty1      18-27 zq0, xs, ys, tx, ty
//   (PairConst of the per-cell focus)
__host__ __device__ constexpr int ph_state_fields(int var) { return (var & 1) ? 28 : 18; }

// Shared memory: phase table, photon table (FP32), bin energies, per-warp
// partial spectra for the CTA's fixed-order reduction, per-warp emitters and
// the per-thread state (FP32).
template <typename T>
__host__ __device__ __forceinline__ size_t photon_smem(int n_phase, int nb, int block, bool ang,
                                                       int var) {
  const size_t tab = ((size_t)n_phase * (sizeof(T) == 4 ? 16 : 8) + 15) & ~(size_t)15;
  const size_t pt = sizeof(T) == 4 ? (size_t)2 * kPhN * sizeof(float4) : 0;
  const size_t e = ((size_t)nb * sizeof(T) + 15) & ~(size_t)15;
  const size_t stage = sizeof(T) == 4 ? (size_t)(block / 32) * 64 * (ang ? 3 : 2) * sizeof(float4) : 0;
  const size_t state = sizeof(T) == 4 ? (size_t)ph_state_fields(var) * block * sizeof(float) : 0;
  return tab + pt + e + (size_t)(block / 32) * (ang ? 3 : 1) * nb * sizeof(double) + stage + state;
}

// K7.  pref = h alpha a_S/(2 sqrt3 pi); eps_b at the bin centres.  Per-CTA
// partials: NA x nb doubles (S, then T_x, T_y with ANG).
template <typename T, int VAR, bool ANG, int KB>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : ((KB == 8 && !ANG) ? 3 : 2)) k_photon(const Params p, int nb, double lo, double hi,
                                                int log_spaced, double* __restrict__ partials) {
  using TT = typename Tab<T>::type;
  using Acc = std::conditional_t<sizeof(T) == 4, PhAccSm<ANG, KB>, PhAcc<T, ANG, KB>>;
  constexpr int NA = Acc::NA;
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t tb = ((size_t)p.n_phase * sizeof(TT) + 15) & ~(size_t)15;
  TT* tab = reinterpret_cast<TT*>(smem);
  float4* ptab = reinterpret_cast<float4*>(smem + tb);
  T* eps = reinterpret_cast<T*>(smem + tb + (sizeof(T) == 4 ? 2 * kPhN * sizeof(float4) : 0));
  double* part = reinterpret_cast<double*>(
      reinterpret_cast<unsigned char*>(eps) + (((size_t)nb * sizeof(T) + 15) & ~(size_t)15));
  const int nwarp = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per emitter q of the warp: stP[q] = {1/mu, 1/mu, 2/(3chi), 2/(3chi)},
  // stQ[q] = {c, c, cut, cut}, stA[q] = {c thx^2 term x2, c thy^2 term x2}
  // (pairs ready for the packed evaluation)
  constexpr int NST = ANG ? 3 : 2;
  float4* stP = reinterpret_cast<float4*>(part + (size_t)nwarp * NA * nb) + warp * 64 * NST;
  float4* stQ = stP + 64;
  float4* stA = stP + 128;
  float* tst = reinterpret_cast<float*>(reinterpret_cast<float4*>(part + (size_t)nwarp * NA * nb) +
                                        (size_t)nwarp * 64 * NST);
  auto ldf = [&](int f) { return tst[f * blockDim.x + threadIdx.x]; };
  auto stf = [&](int f, float v) { tst[f * blockDim.x + threadIdx.x] = v; };
  auto ld2 = [&](int f) { return make_float2(ldf(f), ldf(f + 1)); };
  auto st2 = [&](int f, float2 v) {
    stf(f, v.x);
    stf(f + 1, v.y);
  };
  for (int j = threadIdx.x; j < p.n_phase; j += blockDim.x) table_entry(p, j, tab);
  if (sizeof(T) == 4)
    for (int j = threadIdx.x; j < 2 * kPhN; j += blockDim.x) ptab[j] = g_ph_tab[j];
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    eps[b] = (T)(log_spaced ? lo * exp2(log2(hi / lo) * (b + 0.5) / nb)
                            : lo + (b + 0.5) * (hi - lo) / nb);
  __syncthreads();

  const double pref = p.h * kAlpha / (2.0 * 1.7320508075688772935 * 3.14159265358979323846 *
                                      p.cchi / 1.4142135623730950488);   // h alpha a_S/(2 sqrt3 pi)
  Acc acc;
  if constexpr (sizeof(T) == 4) acc.init(part + (size_t)warp * NA * nb, nb, lane);
  else acc.init();
  if constexpr (sizeof(T) == 4) {
    const float prf = (float)pref, icchi = (float)(1.0 / p.cchi);
    // work items of one warp: 64 consecutive samples, two per lane (packed),
    // dealt to the grid's warps in turn
    const int64_t items = (p.n + 63) / 64;
    const int64_t W = (int64_t)gridDim.x * nwarp;
    for (int64_t it = (int64_t)blockIdx.x * nwarp + warp; it < items; it += W) {
      {
        const int64_t i0 = 64 * it + 2 * lane, i1 = (i0 + 1 < p.n) ? i0 + 1 : i0;
        float g0f = 1.f, g1f = 1.f, tx0 = 0.f, ty0 = 0.f, tx1 = 0.f, ty1 = 0.f, a0 = 0.f,
              a1 = 0.f;
        float w0 = 0.f, w1 = 0.f;
        Path<float> P0{}, P1{};
        if (i0 < p.n) {
          a0 = focus<float>(p, i0, g0f, tx0, ty0, (VAR & kVarCell) ? &P0 : nullptr);
          a1 = focus<float>(p, i1, g1f, tx1, ty1, (VAR & kVarCell) ? &P1 : nullptr);
          w0 = p.weighted ? load_t<float>(p.w, i0, p.dtype) : 1.f;
          w1 = i1 != i0 ? (p.weighted ? load_t<float>(p.w, i1, p.dtype) : 1.f) : 0.f;
          if (!(w0 >= 0.f) || !isfinite(w0) || !isfinite(a0) || !isfinite(g0f)) w0 = 0.f;
          if (!(w1 >= 0.f) || !isfinite(w1) || !isfinite(a1) || !isfinite(g1f)) w1 = 0.f;
        }
        const PairConst kc =
            pair_const<VAR>(p, make_float2(a0, a1), make_float2(g0f, g1f), P0, P1);
        st2(0, kc.c1);
        st2(2, kc.ca);
        st2(4, kc.ig0);
        st2(6, f2(0.f));
        st2(8, f2(0.f));
        st2(10, f2(0.5f));
        stf(12, w0);
        stf(13, w1);
        if (ANG) {
          stf(14, tx0);
          stf(15, ty0);
          stf(16, tx1);
          stf(17, ty1);
        }
        if (VAR & kVarCell) {
          st2(18, kc.zq0);
          st2(20, kc.xs);
          st2(22, kc.ys);
          st2(24, kc.tx);
          st2(26, kc.ty);
        }
      }
      for (int j = 0; j < p.n_phase; ++j) {
        float2 mu, chi;
        {
          PairConst kc;
          kc.c1 = ld2(0);
          kc.ca = ld2(2);
          kc.ig0 = ld2(4);
          if (VAR & kVarCell) {
            kc.zq0 = ld2(18);
            kc.xs = ld2(20);
            kc.ys = ld2(22);
            kc.tx = ld2(24);
            kc.ty = ld2(26);
          }
          PairState st{ld2(6), ld2(8), ld2(10)};
          pair_cell<VAR>(p, reinterpret_cast<const float4*>(tab)[j], kc, st, nullptr, &mu, &chi);
          st2(6, st.du);
          st2(8, st.V);
          st2(10, st.gph);
        }
        const float w0 = ldf(12), w1 = ldf(13);
        const float c0 = (w0 > 0.f && chi.x > 0.f) ? __fmul_rn(__fmul_rn(prf, w0), M<float>::rcp(__fmul_rn(mu.x, mu.x))) : 0.f;
        const float c1 = (w1 > 0.f && chi.y > 0.f) ? __fmul_rn(__fmul_rn(prf, w1), M<float>::rcp(__fmul_rn(mu.y, mu.y))) : 0.f;
        // the warp's 64 emitters of this cell, staged once
        const float4 e0 = emitter(mu.x, chi.x, c0), e1 = emitter(mu.y, chi.y, c1);
        stP[lane] = make_float4(e0.x, e0.x, e0.y, e0.y);
        stP[32 + lane] = make_float4(e1.x, e1.x, e1.y, e1.y);
        stQ[lane] = make_float4(e0.w, e0.w, e0.z, e0.z);
        stQ[32 + lane] = make_float4(e1.w, e1.w, e1.z, e1.z);
        if constexpr (ANG) {
          // mean square angles (A/mu = chi/(cchi mu^2)), times c
          const float tx0 = ldf(14), ty0 = ldf(15), tx1 = ldf(16), ty1 = ldf(17);
          const float am0 = __fmul_rn(__fmul_rn(chi.x, icchi), __fmul_rn(e0.x, e0.x));
          const float am1 = __fmul_rn(__fmul_rn(chi.y, icchi), __fmul_rn(e1.x, e1.x));
          const float cone0 = __fmul_rn(e0.x, e0.x), cone1 = __fmul_rn(e1.x, e1.x);
          const float ax0 = __fmul_rn(c0, __fmaf_rn(tx0, tx0, __fmaf_rn(0.5f, __fmul_rn(am0, am0), cone0)));
          const float ay0 = __fmul_rn(c0, __fmaf_rn(ty0, ty0, cone0));
          const float ax1 = __fmul_rn(c1, __fmaf_rn(tx1, tx1, __fmaf_rn(0.5f, __fmul_rn(am1, am1), cone1)));
          const float ay1 = __fmul_rn(c1, __fmaf_rn(ty1, ty1, cone1));
          stA[lane] = make_float4(ax0, ax0, ay0, ay0);
          stA[32 + lane] = make_float4(ax1, ax1, ay1, ay1);
        }
        float emax = fmaxf(e0.z, e1.z);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        __syncwarp();
        // lane b takes bins b + 32 k (k < KB) against every emitter: up to
        // four bin pairs at a time (packed, independent evaluations) share
        // each emitter's staged constants; summed plainly over the 64
        // emitters, then compensated in shared memory.  No branch on the
        // cut: bins beyond an emitter's cut are evaluated and dropped by the
        // select (the saturated table coordinate keeps every read in the
        // table), so the unrolled evaluations interleave.  Bin pairs whose
        // lowest energy is above every emitter's cut are skipped.
#pragma unroll
        for (int kc = 0; kc < KB; kc += 8) {
          int np = 0;                                    // active bin pairs (warp-uniform)
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4)
            if (kc + 2 * k4 < KB && 32 * (kc + 2 * k4) < nb && eps[32 * (kc + 2 * k4)] < emax)
              np = k4 + 1;
          if (np == 0) break;
          float2 e[4], ps[4], px[4], py[4];
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            const int b0 = 32 * (kc + 2 * k4) + lane, b1 = b0 + 32;
            e[k4] = make_float2(b0 < nb ? eps[b0] : 3.4e38f, b1 < nb ? eps[b1] : 3.4e38f);
            ps[k4] = px[k4] = py[k4] = f2(0.f);
          }
#pragma unroll 2
          for (int q = 0; q < 64; ++q) {
            const float4 qq = stQ[q], pq = stP[q];
            float4 aq;
            if constexpr (ANG) aq = stA[q];
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
              if (k4 < np) {
                const float2 F = synch_F2(ptab, e[k4], pq);
                const float2 Fm = make_float2(e[k4].x < qq.z ? F.x : 0.f,
                                              e[k4].y < qq.z ? F.y : 0.f);
                ps[k4] = fma2(make_float2(qq.x, qq.y), Fm, ps[k4]);
                if constexpr (ANG) {
                  px[k4] = fma2(make_float2(aq.x, aq.y), Fm, px[k4]);
                  py[k4] = fma2(make_float2(aq.z, aq.w), Fm, py[k4]);
                }
              }
            }
          }
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            if (k4 < np) {
              const int kk = kc + 2 * k4;
              acc.add(0, kk, ps[k4].x);
              acc.add(0, kk + 1, ps[k4].y);
              if constexpr (ANG) {
                acc.add(1, kk, px[k4].x);
                acc.add(1, kk + 1, px[k4].y);
                acc.add(2, kk, py[k4].x);
                acc.add(2, kk + 1, py[k4].y);
              }
            }
          }
        }
        __syncwarp();
      }
    }
  } else {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double icchi = 1.0 / p.cchi;
    for (int64_t ib = t0 - lane; ib < p.n; ib += stride) {
      const int64_t i = ib + lane;
      double g0 = 1.0, tx = 0.0, ty = 0.0, a = 0.0, w = 0.0;
      Path<double> P{};
      if (i < p.n) {
        a = focus<double>(p, i, g0, tx, ty, (VAR & kVarCell) ? &P : nullptr);
        w = p.weighted ? load_elem(p.w, i, p.dtype) : 1.0;
        if (!(w >= 0.0) || !isfinite(w) || !isfinite(a) || !isfinite(g0)) w = 0.0;
      }
      double du = 0.0, V = 0.0, gprev = 1.0;
      for (int j = 0; j < p.n_phase; ++j) {
        double mu, chi;
        qfp_cell<VAR>(p, reinterpret_cast<const double*>(tab)[j], j, a, g0, P, du, V, gprev, &mu,
                      &chi);
        const double c = (w > 0.0 && chi > 0.0) ? pref * w / (mu * mu) : 0.0;
        double cx = 0.0, cy = 0.0;
        if (ANG && c > 0.0) {
          const double am = chi * icchi / (mu * mu), cone = 1.0 / (mu * mu);
          cx = c * (tx * tx + 0.5 * am * am + cone);
          cy = c * (ty * ty + cone);
        }
        unsigned m = __ballot_sync(0xffffffffu, c > 0.0);
        while (m) {
          const int s = __ffs(m) - 1;
          m &= m - 1;
          const double ms = __shfl_sync(0xffffffffu, mu, s), xs = __shfl_sync(0xffffffffu, chi, s);
          const double cs = __shfl_sync(0xffffffffu, c, s);
          const double cxs = __shfl_sync(0xffffffffu, cx, s), cys = __shfl_sync(0xffffffffu, cy, s);
          const double imu = 1.0 / ms, gy = 2.0 / (3.0 * xs), yc = 1.5 * xs * kPhYmax;
          const double ecut = ms * yc / (1.0 + yc);
#pragma unroll
          for (int kk = 0; kk < KB; ++kk) {
            if (32 * kk >= nb || !(eps[32 * kk] < ecut)) break;
            const int b = 32 * kk + lane;
            if (b < nb && eps[b] < ecut) {
              const double xi = eps[b] * imu;
              const double F = synch_F_d(xi, gy * xi / (1.0 - xi));
              acc.add(0, kk, cs * F);
              if constexpr (ANG) {
                acc.add(1, kk, cxs * F);
                acc.add(2, kk, cys * F);
              }
            }
          }
        }
      }
    }
  }

  // fixed-order reduction: lanes own distinct bins; warps in order
#pragma unroll
  for (int m = 0; m < NA; ++m)
#pragma unroll
    for (int kk = 0; kk < KB; ++kk)
      if (32 * kk + lane < nb) part[(warp * NA + m) * nb + 32 * kk + lane] = acc.get(m, kk);
  __syncthreads();
  for (int mb = threadIdx.x; mb < NA * nb; mb += blockDim.x) {
    double sum = 0.0;
    for (int wv = 0; wv < nwarp; ++wv) sum += part[wv * NA * nb + mb];
    partials[(size_t)blockIdx.x * NA * nb + mb] = sum;
  }
}

// K8: CTA partials in CTA order (compensated); entry m of NA goes to the
// spectrum (m = 0) or theta2 (m = 1, 2).
__global__ void k_photon_final(int grid, int nb, int na, const double* __restrict__ partials,
                               double* __restrict__ out, double* __restrict__ theta2) {
  for (int mb = blockIdx.x * blockDim.x + threadIdx.x; mb < na * nb;
       mb += gridDim.x * blockDim.x) {
    double s = 0.0, c = 0.0;
    for (int g = 0; g < grid; ++g) {
      const double x = partials[(size_t)g * na * nb + mb], t = s + x;
      c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    if (mb < nb) out[mb] = s + c;
    else theta2[mb - nb] = s + c;
  }
}

namespace {

std::mutex g_ph_mu;
detail::CtxMark g_ph_ready;

// The photon table, built on first use in the device's current context (one
// launch on `st` and a wait for it; not while `st` is being captured).  A
// device reset discards it with the context; the next first use rebuilds it.
int32_t photon_table(cudaStream_t st) {
  int dev = 0;
  unsigned long long key = 0;
  if (int32_t e = detail::current_context(&dev, &key)) return e;
  std::lock_guard<std::mutex> lk(g_ph_mu);
  if (g_ph_ready.done(dev, key)) return QS_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return detail::cuda_fail();
  if (cap != cudaStreamCaptureStatusNone) return QS_ERR_UNSUPPORTED;
  k_photon_setup<<<(kPhN + 255) / 256, 256, 0, st>>>();
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return detail::cuda_fail();
  g_ph_ready.set(dev, key);
  return QS_OK;
}

int32_t check_pbins(const qs_bins* b) {
  if (!b) return QS_ERR_INVALID_ARG;
  if (b->n_bins < 1 || b->n_bins > kPhMaxBins) return QS_ERR_INVALID_ARG;
  if (!std::isfinite(b->lo) || !std::isfinite(b->hi) || !(b->hi > b->lo) || b->lo < 0.0)
    return QS_ERR_INVALID_ARG;
  if (b->log_spaced && !(b->lo > 0.0)) return QS_ERR_INVALID_ARG;
  return QS_OK;
}

// Largest grid a call may use (the workspace holds one partial spectrum per
// CTA): the requested grid, else four CTAs per SM; never more CTAs than
// samples in passes of two per thread.
int photon_gmax(int sms, int block, int grid_req, int64_t n) {
  const int64_t per = 2 * (int64_t)block;
  int64_t g = grid_req > 0 ? grid_req : (int64_t)sms * 4;
  const int64_t need = (n + per - 1) / per;
  if (g > need) g = need;
  return (int)(g < 1 ? 1 : g);
}

template <typename T, int VAR, bool ANG, int KB>
int32_t launch_photon_kb(const Params& p, const qs_bins* pb, int block, int* grid_io, size_t smem,
                         double* partials, cudaStream_t st, const qs_exec* ex) {
  int grid = *grid_io;
  auto kern = k_photon<T, VAR, ANG, KB>;
  static detail::CtxMark smem_mark;
  if (int32_t e = detail::allow_smem(kern, smem_mark, detail::kSmemLimit)) return e;
  // persistent grid: the CTAs that fit at once (unless a grid was requested)
  if (!(ex && ex->grid > 0)) {
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess ||
        detail::device_sms(&sms) != QS_OK)
      return detail::cuda_fail();
    const int g = sms * (occ > 0 ? occ : 1);
    if (g < grid) grid = g;
  }
  *grid_io = grid;
  // optional events around the kernel (qs_exec ev_start/ev_stop)
  if (ex && ex->ev_start &&
      cudaEventRecord(static_cast<cudaEvent_t>(ex->ev_start), st) != cudaSuccess)
    return QS_ERR_CUDA;
  kern<<<grid, block, smem, st>>>(p, pb->n_bins, pb->lo, pb->hi, pb->log_spaced, partials);
  if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
  if (ex && ex->ev_stop &&
      cudaEventRecord(static_cast<cudaEvent_t>(ex->ev_stop), st) != cudaSuccess)
    return QS_ERR_CUDA;
  return QS_OK;
}

// Bin groups per lane: 8 (up to 256 bins, and always with the angular sums),
// else 16 (up to 512 bins).
template <typename T, int VAR, bool ANG>
int32_t launch_photon(const Params& p, const qs_bins* pb, int block, int* grid_io, size_t smem,
                      double* partials, cudaStream_t st, const qs_exec* ex) {
  if constexpr (ANG) {
    return launch_photon_kb<T, VAR, ANG, 8>(p, pb, block, grid_io, smem, partials, st, ex);
  } else {
    if (pb->n_bins <= 256)
      return launch_photon_kb<T, VAR, ANG, 8>(p, pb, block, grid_io, smem, partials, st, ex);
    return launch_photon_kb<T, VAR, ANG, 16>(p, pb, block, grid_io, smem, partials, st, ex);
  }
}

}  // namespace
}  // namespace qs

using namespace qs;
using namespace qs::detail;

extern "C" size_t qs_photon_workspace_bytes(const qs_bins* pbins, const qs_exec* exec,
                                            int64_t n) {
  int prec, wbits, block, grid, sms;
  if (check_pbins(pbins) != QS_OK || n < 0) return 0;
  if (exec_opts(exec, &prec, &wbits, &block, &grid) != QS_OK) return 0;
  if (block > 256) block = 256;
  if (device_sms(&sms) != QS_OK) return 0;
  const int g = photon_gmax(sms, block, grid, n);
  return align_up((size_t)g * 3 * pbins->n_bins * sizeof(double), 256);
}

extern "C" int32_t qs_photon_spectrum(const qs_laser* laser, const qs_beam* beam,
                                      const qs_samples* samples, const qs_bins* pbins,
                                      const qs_exec* exec, double* d_spectrum,
                                      double* d_theta2, void* d_workspace, size_t ws_bytes,
                                      void* stream) {
  int32_t st;
  if ((st = validate_laser(laser)) || (st = validate_beam(beam)) ||
      (st = validate_samples(samples)) || (st = check_pbins(pbins)))
    return st;
  if (laser->model != QS_MODEL_QFP) return QS_ERR_INVALID_ARG;
  if (laser->variant & ~QS_VARIANT_CELL_FOCUS) return QS_ERR_UNSUPPORTED;
  if (!d_spectrum) return QS_ERR_INVALID_ARG;
  const bool ang = d_theta2 != nullptr;
  if (ang && pbins->n_bins > kPhMaxBinsAng) return QS_ERR_INVALID_ARG;
  int prec, wbits, block, grid, sms;
  if ((st = exec_opts(exec, &prec, &wbits, &block, &grid))) return st;
  if (block > 256) block = 256;
  if ((st = device_sms(&sms))) return st;
  const int gmax = photon_gmax(sms, block, grid, samples->n);
  int g = gmax;
  const size_t need = align_up((size_t)gmax * 3 * pbins->n_bins * sizeof(double), 256);
  if (!d_workspace || ((uintptr_t)d_workspace % 256) || ws_bytes < need) return QS_ERR_WORKSPACE;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (prec == QS_F32 && (st = photon_table(cs))) return st;
  Params p;
  fill_params(p, laser, beam, samples, nullptr, wbits);
  double* part = static_cast<double*>(d_workspace);
  const bool loc = (laser->variant & QS_VARIANT_CELL_FOCUS) != 0;
  const size_t smem =
      prec == QS_F64 ? photon_smem<double>(p.n_phase, pbins->n_bins, block, ang, laser->variant)
                     : photon_smem<float>(p.n_phase, pbins->n_bins, block, ang, laser->variant);
  if (smem > (size_t)kSmemLimit) return QS_ERR_INVALID_ARG;
  if (prec == QS_F64) {
    if (ang)
      st = loc ? launch_photon<double, kVarCell, true>(p, pbins, block, &g, smem, part, cs, exec)
               : launch_photon<double, 0, true>(p, pbins, block, &g, smem, part, cs, exec);
    else
      st = loc ? launch_photon<double, kVarCell, false>(p, pbins, block, &g, smem, part, cs, exec)
               : launch_photon<double, 0, false>(p, pbins, block, &g, smem, part, cs, exec);
  } else {
    if (ang)
      st = loc ? launch_photon<float, kVarCell, true>(p, pbins, block, &g, smem, part, cs, exec)
               : launch_photon<float, 0, true>(p, pbins, block, &g, smem, part, cs, exec);
    else
      st = loc ? launch_photon<float, kVarCell, false>(p, pbins, block, &g, smem, part, cs, exec)
               : launch_photon<float, 0, false>(p, pbins, block, &g, smem, part, cs, exec);
  }
  if (st) return st;
  const int na = ang ? 3 : 1;
  k_photon_final<<<(na * pbins->n_bins + 127) / 128, 128, 0, cs>>>(g, pbins->n_bins, na, part,
                                                                    d_spectrum, d_theta2);
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

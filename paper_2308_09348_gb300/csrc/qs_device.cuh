// qs_device.cuh -- device-side pieces of libqscatter: launch parameters, the
// per-precision math policy and the per-sample evaluation (decode, collision
// geometry, Gaussian focus, energy-loss model, divergence, bin indices).
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qs {

constexpr int kMaxPhase = 4096;
// Moment slot (per CTA or per tile) layout:
//   0 W, 1 mean of mu, 2 M2 = sum w (mu - mean)^2, 3 sum w V, 4 sum w thx^2,
//   5 sum w thy^2, 6 sum w a_eff, 7 sum w gamma0, 8 #excluded
// (W, mean, M2) triples merge with the parallel-variance formula, the rest add.
constexpr int kNumMom = 9;
// Per-thread accumulator: as the slot, but entries 1 and 2 hold sum w d and
// sum w d^2 with d = mu - shift, shift (entry 9) = the thread's first mu.
constexpr int kNumAcc = 10;

// Everything a launch needs, derived on the host from the descriptors and
// passed by value (kernel parameter space: uniform, cached, stream-safe).
struct Params {
  // laser (Eq. 2, Eq. 3, Eq. 6)
  double a0, inv_w0sq, inv_zR, ldx, ldy, c_delay;
  double cRR;          // (2/3) R_c * integral G^2               (Eq. 3)
  double cK;           // (2/3) R_c: K = cK A^2, loss per phase   (Eq. 6)
  double cchi;         // sqrt2 / a_S: chi = cchi mu A at rms field
  double h, win_lo, Phi, PhiT;
  double phic, inv2k;  // phase of the pulse peak on the window axis; 1/(2k)
  double kappa_s;      // kappa sqrt(2/pi)                         (Eq. 8)
  int32_t envelope, model, n_phase, focus;   // focus: 0 crossing, 1 per cell
  // beam
  double gmean, spread, glo, gspan, sx, sy, sz, div, bdx, bdy;
  int32_t flat, cycle;     // cycle: cycle-resolved chi (QS_VARIANT_CYCLE_CHI)
  // samples
  int64_t n;
  const void* xi[8];
  const void* w;
  int32_t dtype, weighted;
  // bins
  int32_t n_bins, log_spaced;
  double lo, inv_w, log_scale;
  int32_t n_tx, n_ty;
  double tmax, tsx, tsy;
  int32_t n_aeff, pad2;
  double a_scale;
  double wscale;       // 2^weight_frac_bits
  double gamma_ref;    // shift of the energy moments
  // workspace: integer accumulators (spectrum n_bins+2, map n_tx*n_ty+1,
  // a_eff n_aeff+1) and per-CTA moment partials
  unsigned long long* acc_spec;
  unsigned long long* acc_map;
  unsigned long long* acc_aeff;
  double* partials;
  int32_t hist_in_smem, smooth_in_smem;
  // kernel-smoothed spectrum (n_bins accumulators when smooth_sigma > 0)
  double smooth_sigma;     // in bins
  double smooth_pref;      // 1 / (sigma sqrt(2 pi))
  double smooth_c;         // log2(e) / (2 sigma^2)
  unsigned long long* acc_smooth;
  // cycle-resolved chi: Gauss-Legendre cos(psi_k) and weights (FP64 path),
  // Hermite tables of (G, S) and H over u = log2(1 + chi/chi_s) (FP32 path)
  const double* cyc_gl;
  const float4* cyc_a;          // per node {G, dG du, H, dH du} (adjoint)
  const float4* cyc_m;          // per interval monomial coefficients of G, then H
  // FP32 path, log-spaced bins: t = lg2(gamma) * log2_scale - log2_offset
  float log2_scale, log2_offset;
  // FP32 copies of the per-sample constants, each the double above rounded
  // once to nearest when the constants are derived: the FP32 path then reads
  // them as they are (no per-sample double-to-float conversion, which runs
  // on the FP64 pipe).  hcK = h * cK rounded once.
  struct F {
    float a0, inv_w0sq, inv_zR, ldx, ldy, c_delay, cRR, h, cK, hcK, cchi, kappa_s;
    float gmean, spread, glo, gspan, sx, sy, sz, div, bdx, bdy;
    float lo, inv_w, tmax, tsx, tsy, a_scale, n_bins, n_tx, n_ty, n_aeff, smooth_c;
    float wscale;                  // 2^weight_frac_bits (exact)
    float smooth_pw;               // smooth_pref * wscale
    float smooth_lo, smooth_hi;    // 0.5 + 6 sigma, 6 sigma - 0.5 (bins)
    float smooth_sigma, smooth_pref;
  } f;
};

// A per-sample constant in the arithmetic type T: the double for the FP64
// path, its FP32 copy for the FP32 path.
template <typename T> __device__ __forceinline__ T pv(double d, float f);
template <> __device__ __forceinline__ float pv<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pv<double>(double d, float) { return d; }
#define QS_PV(T, field) ::qs::pv<T>(p.field, p.f.field)

// ---- math policy --------------------------------------------------------
template <typename T> struct M;

template <> struct M<float> {
  // Single MUFU instructions (PTX *.approx forms), no library expansion.
  static __device__ __forceinline__ float lg2(float x) {
    float y; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
  }
  static __device__ __forceinline__ float ex2(float x) {
    float y; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
  }
  static __device__ __forceinline__ float rcp(float x) {
    float y; asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
  }
  static __device__ __forceinline__ float rsqrt(float x) {
    float y; asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
  }
};

template <> struct M<double> {
  static __device__ __forceinline__ double lg2(double x) { return log2(x); }
  static __device__ __forceinline__ double ex2(double x) { return exp2(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
};

__device__ __forceinline__ double load_elem(const void* p, int64_t i, int dtype) {
  if (p == nullptr) return 0.0;
  if (dtype == 0) return (double)__ldg(static_cast<const float*>(p) + i);
  return __ldg(static_cast<const double*>(p) + i);
}

// Load in the arithmetic type (no FP64 round trip for FP32 streams on the
// FP32 path).
template <typename T>
__device__ __forceinline__ T load_t(const void* p, int64_t i, int dtype) {
  if (p == nullptr) return (T)0;
  if (dtype == 0) return (T)__ldg(static_cast<const float*>(p) + i);
  return (T)__ldg(static_cast<const double*>(p) + i);
}

// A finite non-negative float rounded to the nearest integer (ties to even)
// as an unsigned 64-bit value, saturating at 2^63 - 1 as the PTX conversion
// does.  Integer operations only: a 64-bit float-to-integer conversion is an
// FP64-pipe instruction, and the FP64 pipe issues at a small fraction of the
// FP32 rate on this GPU.
__device__ __forceinline__ unsigned long long f2u64_rn(float x) {
  const unsigned u = __float_as_uint(x);
  const int e = (int)(u >> 23);                        // biased exponent (sign is 0)
  const unsigned long long m = (u & 0x7fffffu) | (e ? 0x800000u : 0u);
  const int sh = (e ? e : 1) - 150;                    // x = m 2^sh
  if (sh >= 0) return sh >= 40 ? 0x7fffffffffffffffull : m << sh;
  if (sh <= -25) return 0ull;                          // x < 1/2
  const int r = -sh;
  const unsigned long long q = m >> r, rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
  return q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
}

// Phase-cell envelope G(phi_j) at the midpoint of cell j, in double.
__device__ __forceinline__ double envelope_at(const Params& p, int j) {
  double phi = p.win_lo + ((double)j + 0.5) * p.h;
  if (p.envelope == 0) {
    double r = phi / p.Phi;
    return exp(-2.0 * 0.69314718055994530942 * r * r);
  }
  double s = sinpi(phi / p.PhiT);
  return s * s;
}

// Per-cell focus: shift s_j = (phi_j - phi_c)/(2k) of cell j's midpoint
// from the pulse-peak crossing along the electron's path.
__device__ __forceinline__ double cell_shift(const Params& p, int j) {
  return (p.win_lo + ((double)j + 0.5) * p.h - p.phic) * p.inv2k;
}

// Shared-memory phase table: FP64 path G_j; FP32 path {G_j, G_j, G_j^2,
// G_j^2} (the square taken in double, then rounded), so one 16-byte load
// gives both operands already paired for the two samples a thread carries.
template <typename T> struct Tab;
template <> struct Tab<float> { using type = float4; };
template <> struct Tab<double> { using type = double; };

__device__ __forceinline__ void table_entry(const Params& p, int j, float4* t) {
  const double G = envelope_at(p, j);
  const float g = (float)G;
  if (p.focus) {                       // per-cell focus: {G, G, s_j, s_j}
    const float sj = (float)cell_shift(p, j);
    t[j] = make_float4(g, g, sj, sj);
  } else {
    const float g2 = (float)(G * G);
    t[j] = make_float4(g, g, g2, g2);
  }
}
__device__ __forceinline__ void table_entry(const Params& p, int j, double* t) {
  t[j] = envelope_at(p, j);
}

struct Sample {
  double gamma0, aeff, mu, V, theta_e, thx0, thy0, tx, ty, gout;
};

// Uncontracted IEEE operations (the _rn intrinsics are never fused), so the
// per-sample arithmetic is the same instruction sequence in every kernel
// that inlines it (fused histograms equal histograms of per-sample records,
// batched shots equal single-shot calls, bit for bit).
__device__ __forceinline__ float op_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float op_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float op_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float op_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double op_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double op_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double op_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double op_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Model variant bits of the kernels' VAR template argument.
constexpr int kVarCell = 1;    // per-cell focus
constexpr int kVarCycle = 2;   // cycle-resolved chi
// Internal: the FP32 cycle-resolved tables are replicated kCycRep times,
// interleaved element by element (entry e of copy c at e kCycRep + c), and
// each lane reads copy lane % kCycRep through its own table pointer: the
// eight lanes of each quarter-warp phase of a 16-byte shared-memory load
// then fall in eight distinct bank quads whatever their chi.
constexpr int kVarCycRep = 4;
constexpr int kCycRep = 8;

// Cycle-resolved chi (QS_VARIANT_CYCLE_CHI).  Over one cycle of a linearly
// polarised field chi(psi) = sqrt2 chi |cos psi|; the rates take the cycle
// means G = <2 cos^2 g(chi(psi))>, S = 2G + chi G', H = <2 sqrt2 |cos|^3
// h(chi(psi))> in place of g, 2g + chi g', h.  FP64 path: a 128-point
// Gauss-Legendre rule over the quarter period; FP32 path: cubic Hermite
// interpolation in u = log2(1 + chi/chi_s) of G and H on kCycN nodes
// tabulated (in FP64) from the same rule, S = 2G + chi G' from the
// derivative of G's interpolant: relative error below 1e-9 (G, H) and
// 3e-7 (S) for chi up to chi_s (2^U - 1) = 327 (chi_s resolves the steep
// start of h below chi = 0.1).
constexpr int kCycGL = 128;
constexpr int kCycN = 512;
constexpr double kCycChiS = 0.02;
constexpr double kCycU = 14.0;
constexpr double kCycDu = kCycU / (kCycN - 1);

// Second-moment factor of the diffusion coefficient (Eq. 6 reading): the
// Gaunt fit g times a rational function, h = g N / D with
//   N = 1 + 4.26 chi + 0.494 chi^2,  D = 1 + 12.32 chi + 17.44 chi^2 + 1.63 chi^3
// (within 0.57 % of the exact quantum-synchrotron second moment for
// 1e-5 <= chi <= 300; h ~ chi^(-7/3) at large chi).
constexpr double kHA1 = 4.26, kHA2 = 0.494;
constexpr double kHB1 = 12.32, kHB2 = 17.44, kHB3 = 1.63;
constexpr double kC55 = 55.0 / (16.0 * 1.7320508075688772935);   // D2 prefactor

// Closed forms of the fits (Eq. 6 reading): g, g', g'' and h, h'.
__device__ __forceinline__ void gaunt_d(double x, double& g, double& g1, double& g2) {
  const double L = log1p(1.7 * x), r = 1.0 / (1.0 + 1.7 * x);
  const double B = 1.0 + 4.8 * (1.0 + x) * L + 2.44 * x * x;
  const double B1 = 4.8 * L + 8.16 * (1.0 + x) * r + 4.88 * x;
  const double B2 = 8.16 * r - 5.712 * r * r + 4.88;
  const double iB = 1.0 / B;
  g = pow(B, -2.0 / 3.0);
  g1 = (-2.0 / 3.0) * g * iB * B1;
  g2 = (10.0 / 9.0) * g * iB * iB * B1 * B1 - (2.0 / 3.0) * g * iB * B2;
}
// h = g N / D from g and g' (FP64).
__device__ __forceinline__ void h2_d(double x, double g, double g1, double& h, double& h1) {
  const double N = 1.0 + x * (kHA1 + kHA2 * x), N1 = kHA1 + 2.0 * kHA2 * x;
  const double D = 1.0 + x * (kHB1 + x * (kHB2 + kHB3 * x));
  const double D1 = kHB1 + x * (2.0 * kHB2 + 3.0 * kHB3 * x);
  const double R = N / D;
  h = g * R;
  h1 = g1 * R + g * (N1 - R * D1) / D;
}

// FP64 path: G, S, H and the chi-derivatives G', S' = 3G' + chi G'', H'
// (the derivatives only where asked).  gl: cos psi_k, then the weights with
// the 2/pi of the cycle mean folded in.
__device__ __forceinline__ void cycle_factors_d(const double* __restrict__ gl, double chi,
                                                double& G, double& S, double& H,
                                                double* dG = nullptr, double* dS = nullptr,
                                                double* dH = nullptr) {
  const double r2 = 1.4142135623730950488;
  double sg = 0.0, sg1 = 0.0, sg2 = 0.0, sh = 0.0, sh1 = 0.0;
  for (int k = 0; k < kCycGL; ++k) {
    const double c = gl[k], w = gl[kCycGL + k];
    const double x = r2 * chi * c, c2 = 2.0 * c * c;
    double g, g1, g2, h, h1;
    gaunt_d(x, g, g1, g2);
    h2_d(x, g, g1, h, h1);
    sg += w * c2 * g;
    sg1 += w * c2 * g1 * r2 * c;
    sg2 += w * c2 * g2 * 2.0 * c * c;
    sh += w * r2 * c * c2 * h;
    sh1 += w * r2 * c * c2 * h1 * r2 * c;
  }
  G = sg;
  S = 2.0 * sg + chi * sg1;
  H = sh;
  if (dG) *dG = sg1;
  if (dS) *dS = 3.0 * sg1 + chi * sg2;
  if (dH) *dH = sh1;
}

// a b + c rounded once and clamped to [0, 1] by the FMA's saturation (a NaN
// gives 0).
__device__ __forceinline__ float fma_sat(float a, float b, float c) {
  float d;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Per-cell focus (QS_VARIANT_CELL_FOCUS): Eq. 2 evaluated in
// every phase cell at the electron's position there.  Between the crossing
// of the pulse peak and the midpoint of cell j the electron (velocity
// c(theta_x, theta_y, -1)) meets the counter-moving phase at twice the laser
// frequency, so it moves s_j = (phi_j - phi_c)/(2k) along -z and theta s_j
// sideways: z_j = z* - s_j, transverse offsets xs + theta_x s_j,
// ys + theta_y s_j.  Path holds z*/z_R, the offsets at the crossing and the
// angles.
template <typename T> struct Path { T zq, xs, ys, thx, thy; };

// a_j = a0 q^-1/2 exp(-rho^2/(W0^2 q)), q = 1 + (z_j/z_R)^2, 1/q = (q^-1/2)^2.
template <typename T>
__device__ __forceinline__ T a_cell(const Params& p, const Path<T>& g, T s) {
  const T zq = op_fma(-s, QS_PV(T, inv_zR), g.zq);
  const T q = op_fma(zq, zq, (T)1);
  const T xj = op_fma(g.thx, s, g.xs), yj = op_fma(g.thy, s, g.ys);
  const T rho2 = op_fma(xj, xj, op_mul(yj, yj));
  const T rs = M<T>::rsqrt(q);
  const T E = op_mul(op_mul(rho2, QS_PV(T, inv_w0sq)), op_mul(rs, rs));
  if constexpr (sizeof(T) == 4)
    return op_mul(op_mul(QS_PV(T, a0), rs), M<T>::ex2(op_mul(-(T)1.4426950408889634074, E)));
  else
    return op_mul(op_mul(QS_PV(T, a0), rs), exp(-E));
}

// Quantum-corrected Fokker-Planck phase integration (Eq. 6; mean/variance
// closure of the Fokker-Planck regime), second order in the cell width h:
// rates at each cell midpoint, midpoint state predicted with the previous
// cell's Gaunt factor, frozen-rate Taylor step for the linear variance ODE.
//   g(chi)  = B^(-2/3), B  = 1 + 4.8 (1+chi) ln(1+1.7 chi) + 2.44 chi^2
//   h2(chi) = g N / D (the rational second-moment fit above)
//   K = (2/3) R_c A^2, D1 = -K mu^2 g, dD1/dgamma = -K mu (2g + chi g'),
//   D2 = (55/(16 sqrt3)) K mu^3 chi h2.
// Returns du = 1/mu_f - 1/gamma0 and V_f.  FP64 path: written as the
// equations read.
// VAR: kVarCell -- the peak amplitude a_j of cell j from the path;
// kVarCycle -- cycle-resolved Gaunt and diffusion factors.
// One cell j of the FP64 scheme (state du, V, gprev); also hands out the
// cell's midpoint energy and chi (for the photon spectrum).
template <int VAR>
__device__ __forceinline__ void qfp_cell(const Params& p, double Gj, int j, double a, double g0,
                                         const Path<double>& path, double& du, double& V,
                                         double& gprev, double* mu_out = nullptr,
                                         double* chi_out = nullptr) {
  // explicit (uncontracted) operations: see op_fma below
  const double LN2 = 0.69314718055994530942;
  const double cK = p.cK, cchi = p.cchi, h = p.h;
  const double c55 = 55.0 / (16.0 * 1.7320508075688772935);
  const double hh2 = 0.5 * p.h * p.h;
  const double aj = (VAR & kVarCell) ? a_cell<double>(p, path, cell_shift(p, j)) : a;
  const double A = __dmul_rn(aj, Gj);
  const double K = __dmul_rn(__dmul_rn(cK, A), A);
  const double hK = __dmul_rn(h, K);
  const double dum = __fma_rn(__dmul_rn(0.5, hK), gprev, du);
  const double mu = g0 / __fma_rn(g0, dum, 1.0);
  const double chi = __dmul_rn(__dmul_rn(cchi, mu), A);
  if (mu_out) *mu_out = mu;
  if (chi_out) *chi_out = chi;
  double g, sf, h2;                       // g, 2g + chi g', h (or their cycle means)
  if constexpr ((VAR & kVarCycle) != 0) {
    cycle_factors_d(p.cyc_gl, chi, g, sf, h2);
  } else {
    // Gaunt factor and chi g'(chi)
    const double x1 = __fma_rn(1.7, chi, 1.0);
    const double L1 = __dmul_rn(LN2, log2(x1));
    const double opc = __dadd_rn(1.0, chi);
    const double B = __fma_rn(__dmul_rn(4.8, opc), L1, __fma_rn(__dmul_rn(2.44, chi), chi, 1.0));
    const double t = exp2(__dmul_rn(-1.0 / 3.0, log2(B)));     // B^(-1/3)
    g = __dmul_rn(t, t);
    const double dB = __fma_rn(4.8, L1, __fma_rn(4.8 * 1.7, opc / x1, __dmul_rn(4.88, chi)));
    const double chig1 =
        __dmul_rn(__dmul_rn(__dmul_rn(-2.0 / 3.0, g), __dmul_rn(__dmul_rn(t, t), t)),
                  __dmul_rn(dB, chi));
    sf = __fma_rn(2.0, g, chig1);
    // second-moment factor
    const double N = __fma_rn(__fma_rn(kHA2, chi, kHA1), chi, 1.0);
    const double D = __fma_rn(__fma_rn(__fma_rn(kHB3, chi, kHB2), chi, kHB1), chi, 1.0);
    h2 = __dmul_rn(g, N / D);
  }
  // updates
  du = __fma_rn(hK, g, du);
  const double lam = __dmul_rn(__dmul_rn(__dmul_rn(-2.0, K), mu), sf);
  const double D2 = __dmul_rn(__dmul_rn(__dmul_rn(c55, K), __dmul_rn(__dmul_rn(mu, mu), mu)),
                              __dmul_rn(chi, h2));
  const double r = __fma_rn(lam, V, D2);
  V = __fma_rn(__dmul_rn(hh2, lam), r, __fma_rn(h, r, V));
  gprev = g;
}

template <int VAR>
__device__ __forceinline__ void qfp_integrate(const Params& p, const double* __restrict__ sG,
                                              double a, double g0, double& du_out,
                                              double& V_out, const Path<double>& path) {
  double du = 0, V = 0, gprev = 1;
  const int N = p.n_phase;
#pragma unroll 2
  for (int j = 0; j < N; ++j) qfp_cell<VAR>(p, sG[j], j, a, g0, path, du, V, gprev);
  du_out = du;
  V_out = V;
}

// FP32 path of the same scheme for TWO samples at once, arranged for the
// GB300 issue slots.  Every FMA-pipe operation is a packed f32x2 instruction
// (fma/mul/add .rn on float2, sm_100+), so one issue slot serves both
// samples; the transcendentals are single MUFU lg2/ex2/rcp instructions per
// sample.  Per sample the constants c1 = h (2/3) R_c a^2 and ca = cchi a are
// folded in; 1/(1+1.7 chi) is ex2(-lg2(1+1.7 chi)) (ex2 issues at twice the
// rate of rcp); the step works with h-scaled rates:
//   hK = c1 G^2, hlam = h lambda = -2 hK mu s, s = 2g + chi g', hr = h r.
// The arithmetic per sample is identical whichever lane of the pair it
// occupies.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lg2x2(float2 x) {
  return make_float2(M<float>::lg2(x.x), M<float>::lg2(x.y));
}
__device__ __forceinline__ float2 ex2x2(float2 x) {
  return make_float2(M<float>::ex2(x.x), M<float>::ex2(x.y));
}
__device__ __forceinline__ float2 rcpx2(float2 x) {
  return make_float2(M<float>::rcp(x.x), M<float>::rcp(x.y));
}
__device__ __forceinline__ float2 rsqrtx2(float2 x) {
  return make_float2(M<float>::rsqrt(x.x), M<float>::rsqrt(x.y));
}

// The cycle lookup for the two samples of a pair: the table coordinate and
// the factor of S in packed f32x2 arithmetic; per sample one 16-byte entry
// of monomial coefficients for G and one for H (the cubic Hermite
// interpolants of interval idx in t = x - idx), G and its t-derivative by
// synthetic division (5 FMAs), H by Horner's rule (3).  The coordinate
// x = u/du is clamped to [0, kS] by saturating s = u/(du kS) to [0, 1]
// (x = s kS; a NaN gives 0).
template <int CR = 1>
__device__ __forceinline__ void cycle_lookup2(const float4* __restrict__ A, float2 chi,
                                              float2& G, float2& S, float2& H) {
  constexpr float kS = (float)(kCycN - 1) - 1e-3f;
  const float2 u = lg2x2(fma2(chi, f2((float)(1.0 / kCycChiS)), f2(1.f)));
  const float sa = (float)(1.0 / (kCycDu * kS));
  const float2 sx = make_float2(fma_sat(u.x, sa, 0.f), fma_sat(u.y, sa, 0.f));
  // node index: x - 1/2 rounded to the nearest integer by adding 1.5 2^23
  // (the sum lies in [2^23, 2^24), where the float spacing is 1), so idx is
  // in [0, kCycN - 2] and t = x - idx in [0, 1] (up to the rounding of x - 1/2)
  const float2 xm = __fadd2_rn(fma2(sx, f2(kS), f2(-0.5f)), f2(12582912.f));
  const int i0 = __float_as_int(xm.x) - 0x4B400000, i1 = __float_as_int(xm.y) - 0x4B400000;
  const float2 t = fma2(sx, f2(kS), fma2(xm, f2(-1.f), f2(12582912.f)));
  // chi G' = (dG/dt) chi / (du ln2 (chi + chi_s))
  const float2 k = mul2(chi, rcpx2(mul2(f2((float)(kCycDu * 0.69314718055994530942)),
                                        __fadd2_rn(chi, f2((float)kCycChiS)))));
  const float4 ga = A[i0 * CR], ha = A[(kCycN + i0) * CR];
  const float4 gb = A[i1 * CR], hb = A[(kCycN + i1) * CR];
  // p = c3 t^3 + c2 t^2 + c1 t + c0 and dp/dt, one pass
  const float pa2 = __fmaf_rn(ga.w, t.x, ga.z), pb2 = __fmaf_rn(gb.w, t.y, gb.z);
  const float pa1 = __fmaf_rn(pa2, t.x, ga.y), pb1 = __fmaf_rn(pb2, t.y, gb.y);
  const float da1 = __fmaf_rn(ga.w, t.x, pa2), db1 = __fmaf_rn(gb.w, t.y, pb2);
  G.x = __fmaf_rn(pa1, t.x, ga.x);
  G.y = __fmaf_rn(pb1, t.y, gb.x);
  const float gta = __fmaf_rn(da1, t.x, pa1), gtb = __fmaf_rn(db1, t.y, pb1);
  H.x = __fmaf_rn(__fmaf_rn(__fmaf_rn(ha.w, t.x, ha.z), t.x, ha.y), t.x, ha.x);
  H.y = __fmaf_rn(__fmaf_rn(__fmaf_rn(hb.w, t.y, hb.z), t.y, hb.y), t.y, hb.x);
  S.x = __fmaf_rn(gta, k.x, __fadd_rn(G.x, G.x));
  S.y = __fmaf_rn(gtb, k.y, __fadd_rn(G.y, G.y));
}

// VAR & kVarCell: per-cell focus; the table then holds {G, G, s_j, s_j} and
// the two samples' paths give the per-cell amplitudes (same operations as
// a_cell).  VAR & kVarCycle: cycle-resolved factors from the Hermite tables
// cA (shared memory).  The pair's constants and state, and one cell of
// the scheme (which also hands out the cell's midpoint energy and chi, for
// the photon spectrum):
struct PairConst {
  float2 c1, ca, ig0, zq0, xs, ys, tx, ty;     // ig0 = 1/gamma0
};
struct PairState {
  float2 du, V, gph;
};
template <int VAR>
__device__ __forceinline__ PairConst pair_const(const Params& p, float2 a, float2 g0,
                                                const Path<float>& P0, const Path<float>& P1) {
  constexpr bool LOC = (VAR & kVarCell) != 0;
  PairConst k;
  k.c1 = LOC ? f2(p.f.hcK) : mul2(mul2(f2(p.f.hcK), a), a);
  k.ca = LOC ? f2(p.f.cchi) : mul2(f2(p.f.cchi), a);
  k.ig0 = make_float2(__frcp_rn(g0.x), __frcp_rn(g0.y));
  k.zq0 = make_float2(P0.zq, P1.zq);
  k.xs = make_float2(P0.xs, P1.xs);
  k.ys = make_float2(P0.ys, P1.ys);
  k.tx = make_float2(P0.thx, P1.thx);
  k.ty = make_float2(P0.thy, P1.thy);
  return k;
}

template <int VAR>
__device__ __forceinline__ void pair_cell(const Params& p, const float4 gg, const PairConst& k,
                                          PairState& st, const float4* __restrict__ cA,
                                          float2* mu_out = nullptr,
                                          float2* chi_out = nullptr) {
  const float2 C48 = f2((float)(4.8 * 0.69314718055994530942));   // 4.8 ln2
  const float2 C55 = f2((float)kC55);
  const float2 ONE = f2(1.f), HALF = f2(0.5f);
  const float2 G = make_float2(gg.x, gg.y);
  float2 hK, cg;
  if constexpr ((VAR & kVarCell) != 0) {
    const float2 S = make_float2(gg.z, gg.w);
    const float2 zq = fma2(S, f2(-p.f.inv_zR), k.zq0);
    const float2 q = fma2(zq, zq, ONE);
    const float2 xj = fma2(k.tx, S, k.xs), yj = fma2(k.ty, S, k.ys);
    const float2 rho2 = fma2(xj, xj, mul2(yj, yj));
    const float2 rs = rsqrtx2(q);
    const float2 E = mul2(mul2(rho2, f2(p.f.inv_w0sq)), mul2(rs, rs));
    const float2 aj = mul2(mul2(f2(p.f.a0), rs), ex2x2(mul2(f2(-1.4426950408889634074f), E)));
    const float2 AG = mul2(aj, G);
    hK = mul2(k.c1, mul2(AG, AG));
    cg = mul2(k.ca, AG);
  } else {
    hK = mul2(k.c1, make_float2(gg.z, gg.w));
    cg = mul2(k.ca, G);
  }
  // 1/mu = 1/gamma0 + du at the cell midpoint (predicted)
  const float2 mu = rcpx2(__fadd2_rn(fma2(hK, st.gph, st.du), k.ig0));
  const float2 chi = mul2(cg, mu);
  if (mu_out) *mu_out = mu;
  if (chi_out) *chi_out = chi;
  // g, -2 (2g + chi g') and (55/(16 sqrt3)) h (or their cycle means)
  float2 g, s2, h2c;
  if constexpr ((VAR & kVarCycle) != 0) {
    float2 s, h2;
    constexpr int CR = (VAR & kVarCycRep) ? kCycRep : 1;
    cycle_lookup2<CR>(cA, chi, g, s, h2);
    s2 = mul2(f2(-2.f), s);
    h2c = mul2(C55, h2);
  } else {
    // Gaunt factor: B = 1 + 4.8 (1+chi) ln(1+1.7 chi) + 2.44 chi^2
    const float2 x1 = fma2(f2(1.7f), chi, ONE);
    const float2 l1 = lg2x2(x1);
    const float2 B = fma2(fma2(C48, chi, C48), l1, fma2(mul2(f2(2.44f), chi), chi, ONE));
    const float2 t = ex2x2(mul2(f2(-1.f / 3.f), lg2x2(B)));           // B^(-1/3)
    g = mul2(t, t);
    // one reciprocal 1/(x1 D) gives both 1/(1+1.7 chi) and 1/D (x1 D < 2^126
    // for chi < 1e9)
    const float2 Nc = fma2(fma2(f2((float)(kC55 * kHA2)), chi, f2((float)(kC55 * kHA1))), chi,
                           C55);
    const float2 D = fma2(fma2(fma2(f2((float)kHB3), chi, f2((float)kHB2)), chi,
                               f2((float)kHB1)), chi, ONE);
    const float2 inv = rcpx2(mul2(x1, D));
    const float2 r1 = mul2(D, inv);                                    // 1/(1+1.7 chi)
    // -2 chi g' = (4/3) g chi B'/B with 1/B = g t and
    // B' = 4.8 ln(1+1.7 chi) + 4.8 + 3.36/(1+1.7 chi) + 4.88 chi
    const float2 dB = fma2(f2((float)(4.0 / 3.0 * 4.8 * 0.69314718055994530942)), l1,
                           fma2(f2((float)(4.0 / 3.0 * 4.88)), chi,
                                fma2(f2((float)(4.0 / 3.0 * 3.36)), r1,
                                     f2((float)(4.0 / 3.0 * 4.8)))));
    s2 = mul2(g, fma2(mul2(mul2(g, t), dB), chi, f2(-4.f)));
    // second-moment factor with the D2 constant, h2c = (55/(16 sqrt3)) g N / D
    h2c = mul2(mul2(g, Nc), mul2(x1, inv));
  }
  // updates
  st.du = fma2(hK, g, st.du);
  const float2 hKmu = mul2(hK, mu);
  const float2 hlam = mul2(hKmu, s2);
  const float2 hD2 = mul2(mul2(hKmu, mul2(mu, chi)), mul2(mu, h2c));
  const float2 hr = fma2(hlam, st.V, hD2);
  st.V = fma2(hr, fma2(HALF, hlam, ONE), st.V);
  st.gph = mul2(HALF, g);
}

template <int VAR>
__device__ __forceinline__ void qfp_integrate_f32x2(const Params& p,
                                                    const float4* __restrict__ tab, float2 a,
                                                    float2 g0, float2& du_out, float2& V_out,
                                                    const Path<float>& P0, const Path<float>& P1,
                                                    const float4* __restrict__ cA = nullptr) {
  const PairConst k = pair_const<VAR>(p, a, g0, P0, P1);
  PairState st{f2(0.f), f2(0.f), f2(0.5f)};
  const int N = p.n_phase;
  // unrolled 4 cells (8 with a variant's longer step): measured best on GB300
#pragma unroll(VAR == 0 ? 4 : 8)
  for (int j = 0; j < N; ++j) pair_cell<VAR>(p, tab[j], k, st, cA);
  du_out = st.du;
  V_out = st.V;
}

// a_eff at the crossing point and the decoded sample (rows a1-a3), from the
// sample's six normal deviates.
// path (optional) receives the crossing geometry for the per-cell focus.
template <typename T>
__device__ __forceinline__ T focus_xi(const Params& p, T xi0, T xi1, T xi2, T xi3, T xi4, T xi5,
                                      T& gamma0, T& thx, T& thy, Path<T>* path = nullptr) {
  // decode (reparameterised); gamma0 in the arithmetic type
  const T x = op_fma(QS_PV(T, sx), xi0, QS_PV(T, bdx));
  const T y = op_fma(QS_PV(T, sy), xi1, QS_PV(T, bdy));
  const T z = op_mul(QS_PV(T, sz), xi2);
  T g0 = p.flat ? op_fma(QS_PV(T, gspan), xi3, QS_PV(T, glo))
                : op_mul(QS_PV(T, gmean), op_fma(QS_PV(T, spread), xi3, (T)1));
  if (g0 < (T)1) g0 = (T)1;
  gamma0 = g0;
  thx = op_mul(QS_PV(T, div), xi4);
  thy = op_mul(QS_PV(T, div), xi5);
  // collision geometry: crossing of the pulse peak (factor 2 of Eq. 1)
  const T cdel = QS_PV(T, c_delay);
  const T ct = op_mul((T)0.5, op_add(z, cdel));
  const T zs = op_mul((T)0.5, op_sub(z, cdel));
  const T xs = op_sub(op_fma(thx, ct, x), QS_PV(T, ldx));
  const T ys = op_sub(op_fma(thy, ct, y), QS_PV(T, ldy));
  const T rho2 = op_fma(xs, xs, op_mul(ys, ys));
  // local Gaussian focus, Eq. 2
  const T zq = op_mul(zs, QS_PV(T, inv_zR));
  if (path) *path = Path<T>{zq, xs, ys, thx, thy};
  const T q = op_fma(zq, zq, (T)1);
  const T E = op_mul(op_mul(rho2, QS_PV(T, inv_w0sq)), M<T>::rcp(q));
  if (sizeof(T) == 4)
    return op_mul(op_mul(QS_PV(T, a0), M<T>::rsqrt(q)),
                  M<T>::ex2(op_mul(-(T)1.4426950408889634074, E)));
  return op_mul(op_mul(QS_PV(T, a0), M<T>::rsqrt(q)), (T)exp(-(double)E));
}

template <typename T>
__device__ __forceinline__ T focus(const Params& p, int64_t i, T& gamma0, T& thx, T& thy,
                                   Path<T>* path = nullptr) {
  return focus_xi<T>(p, load_t<T>(p.xi[0], i, p.dtype), load_t<T>(p.xi[1], i, p.dtype),
                     load_t<T>(p.xi[2], i, p.dtype), load_t<T>(p.xi[3], i, p.dtype),
                     load_t<T>(p.xi[4], i, p.dtype), load_t<T>(p.xi[5], i, p.dtype), gamma0,
                     thx, thy, path);
}

// One beam sample through the model, in the paper's order (rows a1-a6).
// FP64 path: one sample through the model selected at compile time by QFP
// (the table is unused by LL).
// VAR: model variant bits (per-cell focus; LL then sums Eq. 3's exponent
// cell by cell; cycle-resolved chi).
template <bool QFP, int VAR = 0>
__device__ __forceinline__ Sample eval_sample(const Params& p, const double* __restrict__ tab,
                                              int64_t i) {
  constexpr bool LOC = (VAR & kVarCell) != 0;
  Sample s;
  double gamma0, thx, thy, mu, V = 0.0;
  Path<double> path;
  const double a = focus<double>(p, i, gamma0, thx, thy, LOC ? &path : nullptr);
  if (!QFP && !LOC) {
    // Eq. 3, a0 -> a_eff
    mu = gamma0 / __fma_rn(__dmul_rn(__dmul_rn(p.cRR, gamma0), a), a, 1.0);
  } else if (!QFP) {
    // 1/gamma_f = 1/gamma0 + (2/3) R_c h sum_j (a_j G_j)^2
    double acc = 0.0;
    for (int j = 0; j < p.n_phase; ++j) {
      const double A = __dmul_rn(a_cell<double>(p, path, cell_shift(p, j)), tab[j]);
      acc = __fma_rn(A, A, acc);
    }
    mu = gamma0 / __fma_rn(gamma0, __dmul_rn(__dmul_rn(p.h, p.cK), acc), 1.0);
  } else {
    double du;
    qfp_integrate<VAR>(p, tab, a, gamma0, du, V, path);
    mu = gamma0 / __fma_rn(gamma0, du, 1.0);
  }
  double theta_e = 0.0, gout = mu, tx = thx;
  if (QFP) {
    const double sv = V > 0.0 ? sqrt(V) : 0.0;
    theta_e = __dmul_rn(__dmul_rn(p.kappa_s, a), sv) / __dmul_rn(mu, mu);   // Eq. 8
    tx = __fma_rn(theta_e, load_elem(p.xi[6], i, p.dtype), tx);
    gout = __fma_rn(sv, load_elem(p.xi[7], i, p.dtype), mu);
  }
  s.theta_e = theta_e; s.tx = tx; s.gout = gout;
  s.gamma0 = gamma0; s.aeff = a; s.mu = mu; s.V = V;
  s.thx0 = thx; s.thy0 = thy; s.ty = thy;
  return s;
}

// FP32-path per-sample record.  The mean energy and the realised energy are
// kept as unevaluated sums of two floats (hi + lo, ~2^-44 relative); the
// rest is FP32.
struct SampleF {
  float g0, mu_hi, mu_lo, go_hi, go_lo;
  float aeff, V, theta_e, thx0, thy0, tx, ty;
};

template <typename T> struct SampleT;
template <> struct SampleT<double> { using type = Sample; };
template <> struct SampleT<float> { using type = SampleF; };

// mu = g0 / (1 + g0 du) in two-float arithmetic on the FP32 pipes (the
// "1/gamma recombination": 1/gamma_f = 1/gamma0 + du).  g0 du and 1 + g0 du
// are formed exactly as float pairs (FMA product error, two-sum), the
// quotient from an FP32 reciprocal is corrected once with its FMA residual:
// relative error ~2^-44, and mu == g0 exactly when du == 0.
__device__ __forceinline__ void recombine_f2(float g0, float du, float& hi, float& lo) {
  const float p = __fmul_rn(g0, du);
  const float pe = __fmaf_rn(g0, du, -p);                  // g0 du = p + pe exactly
  const float s = __fadd_rn(1.f, p);                       // 1 + p = s + se exactly
  const float bb = __fsub_rn(s, 1.f);
  const float se = __fadd_rn(__fsub_rn(1.f, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float t = __fadd_rn(se, pe);
  const float dh = __fadd_rn(s, t);                        // den = dh + dl
  const float dl = __fsub_rn(t, __fsub_rn(dh, s));
  const float r0 = M<float>::rcp(dh);
  const float q0 = __fmul_rn(g0, r0);
  const float e1 = __fmaf_rn(-q0, dh, g0);                 // residual g0 - q0 den
  const float e2 = __fmaf_rn(-q0, dl, e1);
  const float c = __fmul_rn(e2, r0);
  hi = __fadd_rn(q0, c);
  lo = __fsub_rn(c, __fsub_rn(hi, q0));
}

// Recombination, then Eq. 8 and the realised energy (rows a5-a6, FP32 path).
__device__ __forceinline__ void finish_f32(const Params& p, int64_t i, float g0, float af,
                                           float thx, float thy, float du, float Vf, SampleF& s) {
  float hi, lo;
  recombine_f2(g0, du, hi, lo);
  const float sv = Vf > 0.f ? sqrtf(Vf) : 0.f;
  const float te = __fmul_rn(__fmul_rn(__fmul_rn(p.f.kappa_s, af), sv),
                             M<float>::rcp(__fmul_rn(hi, hi)));   // Eq. 8
  const float x = __fmul_rn(sv, load_t<float>(p.xi[7], i, p.dtype));
  const float xl = __fadd_rn(lo, x);
  const float gh = __fadd_rn(hi, xl);
  s.g0 = g0; s.aeff = af; s.mu_hi = hi; s.mu_lo = lo; s.V = Vf; s.theta_e = te;
  s.thx0 = thx; s.thy0 = thy; s.ty = thy;
  s.tx = __fmaf_rn(te, load_t<float>(p.xi[6], i, p.dtype), thx);
  s.go_hi = gh;
  s.go_lo = __fsub_rn(xl, __fsub_rn(gh, hi));
}

// FP32 QFP path: samples i0 and i1 through the model together (the phase
// integration runs packed).
template <int VAR = 0>
__device__ __forceinline__ void eval_pair_f32_qfp(const Params& p, const float4* __restrict__ tab,
                                                  int64_t i0, int64_t i1, SampleF& s0,
                                                  SampleF& s1, const float4* cA = nullptr) {
  constexpr bool LOC = (VAR & kVarCell) != 0;
  float g0f, g1f, tx0, ty0, tx1, ty1;
  Path<float> P0{}, P1{};
  const float a0 = focus<float>(p, i0, g0f, tx0, ty0, LOC ? &P0 : nullptr);
  const float a1 = focus<float>(p, i1, g1f, tx1, ty1, LOC ? &P1 : nullptr);
  float2 du, V;
  qfp_integrate_f32x2<VAR>(p, tab, make_float2(a0, a1), make_float2(g0f, g1f), du, V, P0, P1,
                           cA);
  finish_f32(p, i0, g0f, a0, tx0, ty0, du.x, V.x, s0);
  finish_f32(p, i1, g1f, a1, tx1, ty1, du.y, V.y, s1);
}

// Classical closed form in FP32: mu = g0 / (1 + g0 du) from one reciprocal
// of the rounded denominator, corrected once with its FMA residual (within
// about two FP32 ulps; mu == g0 exactly when du == 0).  Unlike the phase
// integration, the closed form carries no accumulated error that a
// two-float recombination would have to preserve.
__device__ __forceinline__ float recombine_f1(float g0, float du) {
  const float d = __fmaf_rn(g0, du, 1.f);
  const float r0 = M<float>::rcp(d);
  const float q0 = __fmul_rn(g0, r0);
  return __fmaf_rn(__fmaf_rn(-q0, d, g0), r0, q0);
}

// FP32 classical path (Eq. 3 as 1/gamma_f - 1/gamma0 = c_RR a^2).
__device__ __forceinline__ SampleF eval_ll_f32_xi(const Params& p, float xi0, float xi1,
                                                  float xi2, float xi3, float xi4, float xi5) {
  SampleF s;
  float gamma0, thx, thy;
  const float a = focus_xi<float>(p, xi0, xi1, xi2, xi3, xi4, xi5, gamma0, thx, thy);
  const float du = __fmul_rn(__fmul_rn(p.f.cRR, a), a);
  const float mu = recombine_f1(gamma0, du);
  s.g0 = gamma0; s.aeff = a; s.mu_hi = mu; s.mu_lo = 0.f; s.V = 0.f; s.theta_e = 0.f;
  s.thx0 = thx; s.thy0 = thy; s.tx = thx; s.ty = thy;
  s.go_hi = mu;
  s.go_lo = 0.f;
  return s;
}

// Two classical samples in the lanes of float2 values.
struct LL2 {
  float2 g0, a, mu, thx, thy;
};

// Two classical samples at once in packed f32x2 arithmetic: the same
// operations in the same order as focus_xi<float>, the LL closed form and
// recombine_f1 (a - b as a + (-b), g0 - q0 d as one fma of -q0), so each
// lane rounds exactly as the scalar path does.
__device__ __forceinline__ LL2 eval_ll_pair(const Params& p, float2 xi0, float2 xi1, float2 xi2,
                                            float2 xi3, float2 xi4, float2 xi5) {
  const float2 ONE = f2(1.f);
  LL2 r;
  // decode and collision geometry (focus_xi)
  const float2 x = fma2(f2(p.f.sx), xi0, f2(p.f.bdx));
  const float2 y = fma2(f2(p.f.sy), xi1, f2(p.f.bdy));
  const float2 z = mul2(f2(p.f.sz), xi2);
  float2 g0 = p.flat ? fma2(f2(p.f.gspan), xi3, f2(p.f.glo))
                     : mul2(f2(p.f.gmean), fma2(f2(p.f.spread), xi3, ONE));
  if (g0.x < 1.f) g0.x = 1.f;
  if (g0.y < 1.f) g0.y = 1.f;
  r.g0 = g0;
  r.thx = mul2(f2(p.f.div), xi4);
  r.thy = mul2(f2(p.f.div), xi5);
  const float2 ct = mul2(f2(0.5f), __fadd2_rn(z, f2(p.f.c_delay)));
  const float2 zs = mul2(f2(0.5f), __fadd2_rn(z, f2(-p.f.c_delay)));
  const float2 xs = __fadd2_rn(fma2(r.thx, ct, x), f2(-p.f.ldx));
  const float2 ys = __fadd2_rn(fma2(r.thy, ct, y), f2(-p.f.ldy));
  const float2 rho2 = fma2(xs, xs, mul2(ys, ys));
  const float2 zq = mul2(zs, f2(p.f.inv_zR));
  const float2 q = fma2(zq, zq, ONE);
  const float2 E = mul2(mul2(rho2, f2(p.f.inv_w0sq)), rcpx2(q));
  r.a = mul2(mul2(f2(p.f.a0), rsqrtx2(q)), ex2x2(mul2(f2(-1.4426950408889634074f), E)));
  // Eq. 3 and the recombination (recombine_f1)
  const float2 du = mul2(mul2(f2(p.f.cRR), r.a), r.a);
  const float2 d = fma2(g0, du, ONE);
  const float2 r0 = rcpx2(d);
  const float2 q0 = mul2(g0, r0);
  r.mu = fma2(fma2(make_float2(-q0.x, -q0.y), d, g0), r0, q0);
  return r;
}

// Lane k of a pair as the scalar path's record.
__device__ __forceinline__ SampleF ll_sample(const LL2& P, int k) {
  SampleF s;
  s.g0 = k ? P.g0.y : P.g0.x;
  s.aeff = k ? P.a.y : P.a.x;
  s.mu_hi = s.go_hi = k ? P.mu.y : P.mu.x;
  s.mu_lo = s.go_lo = 0.f;
  s.V = 0.f;
  s.theta_e = 0.f;
  s.thx0 = s.tx = k ? P.thx.y : P.thx.x;
  s.thy0 = s.ty = k ? P.thy.y : P.thy.x;
  return s;
}

__device__ __forceinline__ SampleF eval_ll_f32(const Params& p, int64_t i) {
  return eval_ll_f32_xi(p, load_t<float>(p.xi[0], i, p.dtype), load_t<float>(p.xi[1], i, p.dtype),
                        load_t<float>(p.xi[2], i, p.dtype), load_t<float>(p.xi[3], i, p.dtype),
                        load_t<float>(p.xi[4], i, p.dtype), load_t<float>(p.xi[5], i, p.dtype));
}

// FP32 classical path with the per-cell focus: the exponent of Eq. 3 summed
// cell by cell, 1/gamma_f - 1/gamma0 = h (2/3) R_c sum_j (a_j G_j)^2.
__device__ __forceinline__ SampleF eval_ll_f32_cells(const Params& p,
                                                     const float4* __restrict__ tab, int64_t i) {
  SampleF s;
  float gamma0, thx, thy;
  Path<float> path;
  const float a = focus<float>(p, i, gamma0, thx, thy, &path);
  float acc = 0.f;
  for (int j = 0; j < p.n_phase; ++j) {
    const float4 e = tab[j];
    const float A = __fmul_rn(a_cell<float>(p, path, e.z), e.x);
    acc = __fmaf_rn(A, A, acc);
  }
  float hi, lo;
  recombine_f2(gamma0, __fmul_rn(p.f.hcK, acc), hi, lo);
  s.g0 = gamma0; s.aeff = a; s.mu_hi = hi; s.mu_lo = lo; s.V = 0.f; s.theta_e = 0.f;
  s.thx0 = thx; s.thy0 = thy; s.tx = thx; s.ty = thy;
  s.go_hi = hi;
  s.go_lo = lo;
  return s;
}

// One sample of the path selected by T, QFP and VAR (FP32 QFP samples are
// normally evaluated in pairs; a single one runs as a pair with itself).
template <typename T, bool QFP, int VAR = 0>
__device__ __forceinline__ typename SampleT<T>::type eval_one(
    const Params& p, const typename Tab<T>::type* __restrict__ tab, int64_t i,
    const float4* cA = nullptr) {
  if constexpr (sizeof(T) == 8) {
    return eval_sample<QFP, VAR>(p, reinterpret_cast<const double*>(tab), i);
  } else if constexpr (QFP) {
    SampleF s0, s1;
    eval_pair_f32_qfp<VAR>(p, reinterpret_cast<const float4*>(tab), i, i, s0, s1, cA);
    return s0;
  } else if constexpr ((VAR & kVarCell) != 0) {
    return eval_ll_f32_cells(p, reinterpret_cast<const float4*>(tab), i);
  } else {
    return eval_ll_f32(p, i);
  }
}

// Energy bin: -1 under, n_bins over (half-open bins).
__device__ __forceinline__ int energy_bin(const Params& p, double g) {
  double t;
  if (!p.log_spaced) t = (g - p.lo) * p.inv_w;
  else t = (g > 0.0) ? log(g / p.lo) * p.log_scale : -1.0;
  if (!(t >= 0.0)) return -1;
  if (t >= (double)p.n_bins) return p.n_bins;
  return (int)t;
}

// Divergence-map cell (row-major iy*n_tx + ix) or -1 outside.
__device__ __forceinline__ int map_cell(const Params& p, double tx, double ty, int* ix_o,
                                        int* iy_o) {
  double fx = (tx + p.tmax) * p.tsx, fy = (ty + p.tmax) * p.tsy;
  if (fx >= 0.0 && fx < (double)p.n_tx && fy >= 0.0 && fy < (double)p.n_ty) {
    int ix = (int)fx, iy = (int)fy;
    if (ix_o) *ix_o = ix;
    if (iy_o) *iy_o = iy;
    return iy * p.n_tx + ix;
  }
  if (ix_o) *ix_o = -1;
  if (iy_o) *iy_o = -1;
  return -1;
}

// Bins k with |k + 1/2 - t| <= 6 sigma of the smoothed spectrum, clamped.
__device__ __forceinline__ void smooth_range(const Params& p, double t, int* k0, int* k1) {
  double lo = ceil(t - 0.5 - 6.0 * p.smooth_sigma), hi = floor(t - 0.5 + 6.0 * p.smooth_sigma);
  if (lo < 0.0) lo = 0.0;
  if (hi > (double)(p.n_bins - 1)) hi = (double)(p.n_bins - 1);
  *k0 = (int)lo;
  *k1 = (int)hi;
}

// FP32 path: the same window with the offsets rounded to FP32.
__device__ __forceinline__ void smooth_range_f32(const Params& p, float t, int* k0, int* k1) {
  float lo = ceilf(__fsub_rn(t, p.f.smooth_lo)), hi = floorf(__fadd_rn(t, p.f.smooth_hi));
  if (lo < 0.f) lo = 0.f;
  if (hi > __fsub_rn(p.f.n_bins, 1.f)) hi = __fsub_rn(p.f.n_bins, 1.f);
  *k0 = (int)lo;
  *k1 = (int)hi;
}

__device__ __forceinline__ int aeff_bin(const Params& p, double a) {
  double f = a * p.a_scale;
  if (f >= 0.0 && f < (double)p.n_aeff) return (int)f;
  return p.n_aeff;
}

// FP32-path binning, all in FP32: the energy index from the realised energy
// as a float pair (hi, lo) -- uniform bins t = ((hi - lo_edge) + lo) inv_w,
// log bins t = lg2(hi + lo) log2_scale - log2_offset -- and the map and
// a_eff indices.  Index error: uniform bins, the subtraction is exact when
// hi lies within a factor 2 of lo_edge and otherwise rounds by half an ulp
// of hi - lo_edge, the addition of lo and the product by inv_w (itself
// rounded once) by half an ulp each, so |t - t_exact| <= 2^-23 t + |hi|
// 2^-24 inv_w; log bins, the MUFU logarithm's error (2^-22 absolute in
// lg2) times log2_scale.  A sample moves to a neighbouring bin only when
// its exact t lies within that bound (plus the per-sample error of the
// energy itself) of an integer; decisions otherwise equal the FP64 path's.
__device__ __forceinline__ int energy_bin_f32(const Params& p, float gh, float gl) {
  if (!p.log_spaced) {
    const float tf = __fmul_rn(__fadd_rn(__fsub_rn(gh, p.f.lo), gl), p.f.inv_w);
    if (!(tf >= 0.f)) return -1;
    if (tf >= p.f.n_bins) return p.n_bins;
    return (int)tf;
  }
  const float g = __fadd_rn(gh, gl);
  const float t =
      (g > 0.f) ? __fsub_rn(__fmul_rn(M<float>::lg2(g), p.log2_scale), p.log2_offset) : -1.f;
  if (!(t >= 0.f)) return -1;
  if (t >= p.f.n_bins) return p.n_bins;
  return (int)t;
}

__device__ __forceinline__ int map_cell_f32(const Params& p, float tx, float ty) {
  const float tm = p.f.tmax;
  const float fx = __fmul_rn(__fadd_rn(tx, tm), p.f.tsx);
  const float fy = __fmul_rn(__fadd_rn(ty, tm), p.f.tsy);
  if (fx >= 0.f && fx < p.f.n_tx && fy >= 0.f && fy < p.f.n_ty)
    return (int)fy * p.n_tx + (int)fx;
  return -1;
}

__device__ __forceinline__ int aeff_bin_f32(const Params& p, float a) {
  const float f = __fmul_rn(a, p.f.a_scale);
  if (f >= 0.f && f < p.f.n_aeff) return (int)f;
  return p.n_aeff;
}

// |x| < inf: isfinite's value (false for +-inf and NaN) as one compare.
__device__ __forceinline__ bool finitef(float x) { return fabsf(x) < __int_as_float(0x7f800000); }

// Accumulator slot of a spectrum bin coordinate t (FP32 paths): bins
// [0, n_bins), n_bins below the range, n_bins + 1 above -- the slots
// energy_bin_f32 leads to, from a floor conversion and one unsigned compare
// (t >= n_bins saturates to or past n_bins; t is never NaN here).
__device__ __forceinline__ int spec_slot(const Params& p, float t) {
  const int b = __float2int_rd(t);
  return (unsigned)b < (unsigned)p.n_bins ? b : (b < 0 ? p.n_bins : p.n_bins + 1);
}
// Bin coordinate of a single-float energy (the classical model's
// gamma_out = mu has no low part): energy_bin_f32's arithmetic without it.
__device__ __forceinline__ float energy_coord_f1(const Params& p, float g) {
  if (!p.log_spaced) return __fmul_rn(__fsub_rn(g, p.f.lo), p.f.inv_w);
  return (g > 0.f) ? __fsub_rn(__fmul_rn(M<float>::lg2(g), p.log2_scale), p.log2_offset) : -1.f;
}
// Map slot from the map coordinates fx = (tx + theta_max) tsx, fy (as
// map_cell_f32 forms them; finite): the cell, or nmap - 1 outside the map.
__device__ __forceinline__ int map_slot(const Params& p, float fx, float fy, int nmap) {
  const int ix = __float2int_rd(fx), iy = __float2int_rd(fy);
  return ((unsigned)ix < (unsigned)p.n_tx && (unsigned)iy < (unsigned)p.n_ty)
             ? iy * p.n_tx + ix : nmap - 1;
}
// a_eff slot from f = a_eff a_scale (a_eff >= 0, finite): the bin, or n_aeff.
__device__ __forceinline__ int aeff_slot(const Params& p, float f) {
  const int b = __float2int_rd(f);
  return (unsigned)b < (unsigned)p.n_aeff ? b : p.n_aeff;
}

// Merge of two (weight, mean, central sum of squares) triples (the parallel
// form of the variance recurrence): exact when one side is empty, no
// cancellation between large raw moments.
__device__ __forceinline__ void welford_merge(double& W, double& m, double& M2, double Wb,
                                              double mb, double M2b) {
  if (!(Wb > 0.0)) return;
  if (!(W > 0.0)) {
    W = Wb;
    m = mb;
    M2 = M2b;
    return;
  }
  const double Wn = W + Wb;
  const double d = mb - m;
  const double f = Wb / Wn;
  m = fma(d, f, m);
  M2 = M2 + M2b + d * d * W * f;
  W = Wn;
}

// Per-thread moment accumulators.  FP64 path: plain FP64 sums.  FP32 path:
// compensated (Kahan) FP32 sums, converted to FP64 once per thread; the
// reductions across threads, CTAs and tiles are FP64.  Entries:
//   0 W, 1 sum w d, 2 sum w d^2 (d = mu - shift, shift = the thread's first
//   mu), 3 sum w V, 4 sum w (thx0^2 + theta_e^2), 5 sum w thy0^2,
//   6 sum w a_eff, 7 sum w gamma0; plus the excluded count and the shift.
struct AccD {
  double a[kNumAcc];
};
struct AccF {
  float s[8], c[8];
  float nonfinite, shift;
};
template <typename T> struct AccT;
template <> struct AccT<double> { using type = AccD; };
template <> struct AccT<float> { using type = AccF; };

__device__ __forceinline__ void acc_init(AccD& A) {
#pragma unroll
  for (int k = 0; k < kNumAcc; ++k) A.a[k] = 0.0;
  A.a[9] = __longlong_as_double(0x7ff8000000000000ll);   // no shift yet (NaN)
}
__device__ __forceinline__ void acc_init(AccF& A) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    A.s[k] = 0.f;
    A.c[k] = 0.f;
  }
  A.nonfinite = 0.f;
  A.shift = __int_as_float(0x7fc00000);                  // no shift yet (NaN)
}

// Kahan step in FP32 (explicit _rn operations: never contracted).
__device__ __forceinline__ void kahan(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// Thread's accumulator as a moment slot (W, mean, M2, sums...).
__device__ __forceinline__ void acc_slot(const AccD& A, double (&v)[kNumMom]) {
  v[0] = A.a[0];
  v[1] = 0.0;
  v[2] = 0.0;
  if (A.a[0] > 0.0) {
    const double q = A.a[1] / A.a[0];
    v[1] = A.a[9] + q;
    v[2] = fmax(A.a[2] - A.a[1] * q, 0.0);
  }
#pragma unroll
  for (int k = 3; k < kNumMom; ++k) v[k] = A.a[k];
}
__device__ __forceinline__ void acc_slot(const AccF& A, double (&v)[kNumMom]) {
  double t[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) t[k] = (double)A.s[k] - (double)A.c[k];
  v[0] = t[0];
  v[1] = 0.0;
  v[2] = 0.0;
  if (t[0] > 0.0) {
    const double q = t[1] / t[0];
    v[1] = (double)A.shift + q;
    v[2] = fmax(t[2] - t[1] * q, 0.0);
  }
#pragma unroll
  for (int k = 3; k < 8; ++k) v[k] = t[k];
  v[8] = (double)A.nonfinite;
}

// Error-free sum of two floats: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (h, l) += (bh, bl) for unevaluated float pairs (relative error ~2^-44).
__device__ __forceinline__ void pair_add(float& h, float& l, float bh, float bl) {
  float sm, e;
  two_sum(h, bh, sm, e);
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(sm, e);
  l = __fsub_rn(e, __fsub_rn(h, sm));
}

// Warp tree of the per-thread accumulators, leaving the warp's moment slot
// in lane 0's v.
__device__ __forceinline__ void warp_reduce(const AccD& acc, double (&v)[kNumMom]) {
  acc_slot(acc, v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double u[kNumMom];
#pragma unroll
    for (int k = 0; k < kNumMom; ++k) u[k] = __shfl_down_sync(0xffffffffu, v[k], o);
    welford_merge(v[0], v[1], v[2], u[0], u[1], u[2]);
#pragma unroll
    for (int k = 3; k < kNumMom; ++k) v[k] += u[k];
  }
}
// (h, l) = a b for unevaluated float pairs (relative error ~2^-44): the
// leading product exactly by FMA, the cross terms rounded.
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float& h,
                                         float& l) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float t = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  h = __fadd_rn(p, t);
  l = __fsub_rn(t, __fsub_rn(h, p));
}

// FP32 path's sums on their way through the reduction tree, all as float
// pairs: W = sum w, S1 = sum w (mu - sh), S2 = sum w (mu - sh)^2 about the
// shift sh, the five plain sums, and the excluded-sample count.  The tree
// runs on the FP32 pipes only (the FP64 pipe of this GPU issues 2 lanes per
// SM and clock, so an FP64 tree would be the launch's tail).
struct PairMom {
  float Wh, Wl, S1h, S1l, S2h, S2l, sh;
  float h[5], l[5];
  float nf;
};
constexpr int kPairMomFloats = 18;        // one warp's record in the red buffer
static_assert(kPairMomFloats * 4 <= kNumMom * 8, "a warp record fits its moment slot");

__device__ __forceinline__ PairMom pair_mom(const AccF& A) {
  PairMom m;
  two_sum(A.s[0], -A.c[0], m.Wh, m.Wl);
  two_sum(A.s[1], -A.c[1], m.S1h, m.S1l);
  two_sum(A.s[2], -A.c[2], m.S2h, m.S2l);
#pragma unroll
  for (int k = 0; k < 5; ++k) two_sum(A.s[k + 3], -A.c[k + 3], m.h[k], m.l[k]);
  m.sh = m.Wh > 0.f ? A.shift : 0.f;
  m.nf = A.nonfinite;
  return m;
}

// The sums moved to the shift s0, with d = sh - s0 (an exact pair):
//   S1' = S1 + W d,   S2' = S2 + d (S1 + S1') = S2 + 2 d S1 + W d^2.
// An empty record (W = 0: S1 = S2 = 0 about any shift) only takes s0.
__device__ __forceinline__ void pair_reshift(PairMom& m, float s0) {
  if (m.Wh > 0.f) {
    float dh, dl, th, tl;
    two_sum(m.sh, -s0, dh, dl);
    pair_mul(m.Wh, m.Wl, dh, dl, th, tl);
    float nh = m.S1h, nl = m.S1l;
    pair_add(nh, nl, th, tl);
    float uh = m.S1h, ul = m.S1l;
    pair_add(uh, ul, nh, nl);
    pair_mul(dh, dl, uh, ul, th, tl);
    pair_add(m.S2h, m.S2l, th, tl);
    m.S1h = nh;
    m.S1l = nl;
  }
  m.sh = s0;
}

// Fixed-order warp tree of the 32 lanes' records (every lane takes part):
// each record is first moved to the shift of the lowest lane with weight
// (when no lane has weight every energy sum is zero and nothing moves), and
// lane 0 ends with the sum.
__device__ __forceinline__ void warp_sum(PairMom& m) {
  const unsigned has = __ballot_sync(0xffffffffu, m.Wh > 0.f);
  if (has) pair_reshift(m, __shfl_sync(0xffffffffu, m.sh, __ffs(has) - 1));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float bh = __shfl_down_sync(0xffffffffu, m.Wh, o), bl = __shfl_down_sync(0xffffffffu, m.Wl, o);
    pair_add(m.Wh, m.Wl, bh, bl);
    bh = __shfl_down_sync(0xffffffffu, m.S1h, o);
    bl = __shfl_down_sync(0xffffffffu, m.S1l, o);
    pair_add(m.S1h, m.S1l, bh, bl);
    bh = __shfl_down_sync(0xffffffffu, m.S2h, o);
    bl = __shfl_down_sync(0xffffffffu, m.S2l, o);
    pair_add(m.S2h, m.S2l, bh, bl);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      bh = __shfl_down_sync(0xffffffffu, m.h[k], o);
      bl = __shfl_down_sync(0xffffffffu, m.l[k], o);
      pair_add(m.h[k], m.l[k], bh, bl);
    }
    m.nf = __fadd_rn(m.nf, __shfl_down_sync(0xffffffffu, m.nf, o));
  }
}

// Fixed-order block reduction of the per-thread accumulators into one
// moment slot out[0..kNumMom): warp shuffle tree, then warps in order.
template <typename A>
__device__ __forceinline__ void block_reduce_write(A& acc, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[kNumMom];
  warp_reduce(acc, v);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kNumMom; ++k) red[warp * kNumMom + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    double W = 0.0, m = 0.0, M2 = 0.0, sm[kNumMom] = {};
    for (int w = 0; w < nw; ++w) {
      welford_merge(W, m, M2, red[w * kNumMom], red[w * kNumMom + 1], red[w * kNumMom + 2]);
      for (int k = 3; k < kNumMom; ++k) sm[k] += red[w * kNumMom + k];
    }
    out[0] = W;
    out[1] = m;
    out[2] = M2;
    for (int k = 3; k < kNumMom; ++k) out[k] = sm[k];
  }
}

// FP32 path: warp trees of float pairs, the warps' records through one more
// tree in warp 0, and only the slot's final mean and M2 in FP64 (thread 0).
__device__ __forceinline__ void block_reduce_write(AccF& acc, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* rf = reinterpret_cast<float*>(red);
  PairMom m = pair_mom(acc);
  warp_sum(m);
  if (lane == 0) {
    float* r = rf + warp * kPairMomFloats;
    r[0] = m.Wh; r[1] = m.Wl; r[2] = m.S1h; r[3] = m.S1l; r[4] = m.S2h; r[5] = m.S2l;
    r[6] = m.sh;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      r[7 + 2 * k] = m.h[k];
      r[8 + 2 * k] = m.l[k];
    }
    r[17] = m.nf;
  }
  __syncthreads();
  if (warp == 0) {
    PairMom b{};
    if (lane < (int)(blockDim.x >> 5)) {
      const float* r = rf + lane * kPairMomFloats;
      b.Wh = r[0]; b.Wl = r[1]; b.S1h = r[2]; b.S1l = r[3]; b.S2h = r[4]; b.S2l = r[5];
      b.sh = r[6];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        b.h[k] = r[7 + 2 * k];
        b.l[k] = r[8 + 2 * k];
      }
      b.nf = r[17];
    }
    warp_sum(b);
    if (lane == 0) {
      const double W = (double)b.Wh + (double)b.Wl;
      out[0] = W;
      out[1] = 0.0;
      out[2] = 0.0;
      if (W > 0.0) {
        const double S1 = (double)b.S1h + (double)b.S1l;
        const double S2 = (double)b.S2h + (double)b.S2l;
        const double q = S1 / W;
        out[1] = (double)b.sh + q;
        out[2] = fmax(S2 - S1 * q, 0.0);
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) out[k + 3] = (double)b.h[k] + (double)b.l[k];
      out[8] = (double)b.nf;
    }
  }
}

// One evaluated sample into the moment partials and histograms (rows a7-a8).
// SHIST: the histograms in shared memory (hs, hm, ha); a null hm or ha keeps
// that histogram in the global accumulators (p.acc_map, p.acc_aeff), as the
// batch does with its per-shot maps.
template <typename T, typename H, bool SHIST>
__device__ __forceinline__ bool accumulate(const Params& p, const Sample& s, int64_t i, AccD& A,
                                           H* hs, H* hm, H* ha, int64_t nspec, int64_t nmap,
                                           int64_t naeff) {
  double* acc = A.a;
  const double w = p.weighted ? load_elem(p.w, i, p.dtype) : 1.0;
  // every value that enters a sum or a bin must be finite
  const bool ok = isfinite(s.mu) && isfinite(s.V) && isfinite(s.gout) && isfinite(s.tx) &&
                  isfinite(s.ty) && isfinite(s.aeff) && isfinite(s.gamma0) && isfinite(w) &&
                  w >= 0.0;
  if (!ok) {
    acc[8] += 1.0;
    return false;
  }
  if (isnan(acc[9])) acc[9] = s.mu;                      // the thread's shift
  const double d = s.mu - acc[9];
  acc[0] += w;
  acc[1] = fma(w, d, acc[1]);
  acc[2] = fma(w * d, d, acc[2]);
  acc[3] = fma(w, s.V, acc[3]);
  acc[4] = fma(w, fma(s.thx0, s.thx0, s.theta_e * s.theta_e), acc[4]);
  acc[5] = fma(w, s.thy0 * s.thy0, acc[5]);
  acc[6] = fma(w, s.aeff, acc[6]);
  acc[7] = fma(w, s.gamma0, acc[7]);
  const unsigned long long q =
      p.weighted ? (unsigned long long)__double2ll_rn(w * p.wscale) : 1ull;
  if (nspec) {
    const int b = energy_bin(p, s.gout);
    const int slot = b < 0 ? p.n_bins : (b >= p.n_bins ? p.n_bins + 1 : b);
    if (SHIST) atomicAdd(&hs[slot], (H)q);
    else atomicAdd(&p.acc_spec[slot], q);
  }
  if (nmap) {
    const int c = map_cell(p, s.tx, s.ty, nullptr, nullptr);
    const int64_t slot = c < 0 ? nmap - 1 : c;
    if (SHIST && hm) atomicAdd(&hm[slot], (H)q);
    else atomicAdd(&p.acc_map[slot], q);
  }
  if (naeff) {
    const int slot = aeff_bin(p, s.aeff);
    if (SHIST && ha) atomicAdd(&ha[slot], (H)q);
    else atomicAdd(&p.acc_aeff[slot], q);
  }
  return true;
}

// QFP = false drops the terms that vanish in the classical model (V = 0,
// theta_e = 0, gamma_out = mu): the same sums, with fewer instructions.
// Returns whether the sample entered the sums (false: counted as excluded).
template <typename H, bool SHIST, bool QFP = true>
__device__ __forceinline__ bool accumulate_w(const Params& p, const SampleF& s, float w, AccF& A,
                                             H* hs, H* hm, H* ha, int64_t nspec, int64_t nmap,
                                             int64_t naeff) {
  const float muf = s.mu_hi;
  // every value that enters a sum or a bin must be finite
  const bool ok = finitef(muf) & (!QFP || (finitef(s.V) & finitef(s.go_hi))) &
                  finitef(s.tx) & finitef(s.ty) & finitef(s.aeff) & finitef(s.g0) &
                  finitef(w) & (w >= 0.f);
  if (!ok) {
    A.nonfinite = __fadd_rn(A.nonfinite, 1.f);
    return false;
  }
  if (isnan(A.shift)) A.shift = muf;                     // the thread's shift
  const float d = __fsub_rn(muf, A.shift);
  const float wd = __fmul_rn(w, d);
  kahan(A.s[0], A.c[0], w);
  kahan(A.s[1], A.c[1], wd);
  kahan(A.s[2], A.c[2], __fmul_rn(wd, d));
  if (QFP) {
    kahan(A.s[3], A.c[3], __fmul_rn(w, s.V));
    kahan(A.s[4], A.c[4], __fmul_rn(w, __fmaf_rn(s.thx0, s.thx0, __fmul_rn(s.theta_e, s.theta_e))));
  } else {
    kahan(A.s[4], A.c[4], __fmul_rn(w, __fmul_rn(s.thx0, s.thx0)));
  }
  kahan(A.s[5], A.c[5], __fmul_rn(w, __fmul_rn(s.thy0, s.thy0)));
  kahan(A.s[6], A.c[6], __fmul_rn(w, s.aeff));
  kahan(A.s[7], A.c[7], __fmul_rn(w, s.g0));
  // w 2^bits is exact in FP32, so this equals the FP64 path's rounding
  const unsigned long long q = p.weighted ? f2u64_rn(__fmul_rn(w, p.f.wscale)) : 1ull;
  if (nspec) {
    int slot;
    if (QFP) {
      const int b = energy_bin_f32(p, s.go_hi, s.go_lo);
      slot = b < 0 ? p.n_bins : (b >= p.n_bins ? p.n_bins + 1 : b);
    } else {
      slot = spec_slot(p, energy_coord_f1(p, s.go_hi));
    }
    if (SHIST) atomicAdd(&hs[slot], (H)q);
    else atomicAdd(&p.acc_spec[slot], q);
  }
  if (nmap) {
    const int c = map_cell_f32(p, s.tx, s.ty);
    const int64_t slot = c < 0 ? nmap - 1 : c;
    if (SHIST && hm) atomicAdd(&hm[slot], (H)q);
    else atomicAdd(&p.acc_map[slot], q);
  }
  if (naeff) {
    const int slot = aeff_bin_f32(p, s.aeff);
    if (SHIST && ha) atomicAdd(&ha[slot], (H)q);
    else atomicAdd(&p.acc_aeff[slot], q);
  }
  return true;
}

// Plain partial sums of the FP32 classical vector path, packed (lane x:
// the first sample of each pair, lane y: the second) over a few iterations,
// then folded into the thread's compensated sums (ll_fold).  t0: weights
// (count when unweighted), t1, t2: w d and w d^2 about the thread's shift,
// t4, t5: w thx^2, w thy^2, t6: w a_eff, t7: w gamma0.
struct LLSums {
  float2 t0, t1, t2, t4, t5, t6, t7;
};
__device__ __forceinline__ void ll_sums_zero(LLSums& T) {
  T.t0 = T.t1 = T.t2 = T.t4 = T.t5 = T.t6 = T.t7 = make_float2(0.f, 0.f);
}
__device__ __forceinline__ void ll_fold(LLSums& T, AccF& A) {
  kahan(A.s[0], A.c[0], __fadd_rn(T.t0.x, T.t0.y));
  kahan(A.s[1], A.c[1], __fadd_rn(T.t1.x, T.t1.y));
  kahan(A.s[2], A.c[2], __fadd_rn(T.t2.x, T.t2.y));
  kahan(A.s[4], A.c[4], __fadd_rn(T.t4.x, T.t4.y));
  kahan(A.s[5], A.c[5], __fadd_rn(T.t5.x, T.t5.y));
  kahan(A.s[6], A.c[6], __fadd_rn(T.t6.x, T.t6.y));
  kahan(A.s[7], A.c[7], __fadd_rn(T.t7.x, T.t7.y));
  ll_sums_zero(T);
}
// Iterations (four samples each) between folds: a partial sum then holds
// at most eight terms per lane, far below the compensated sums' error.
constexpr int kLLFold = 4;

// Histogram deposits of one pair: slots from packed coordinates.  ALL: every
// histogram present (known at compile time); else the sizes decide.
template <typename H, bool SHIST, bool W, bool ALL>
__device__ __forceinline__ void ll_deposit(const Params& p, const LL2& P, float2 w, H* hs, H* hm,
                                           H* ha, int nspec, int nmap, int naeff) {
  const unsigned long long q0 = W ? f2u64_rn(__fmul_rn(w.x, p.f.wscale)) : 1ull;
  const unsigned long long q1 = W ? f2u64_rn(__fmul_rn(w.y, p.f.wscale)) : 1ull;
  if (ALL || nspec) {
    int s0, s1;
    if (!p.log_spaced) {
      const float2 t = mul2(__fadd2_rn(P.mu, f2(-p.f.lo)), f2(p.f.inv_w));
      s0 = spec_slot(p, t.x);
      s1 = spec_slot(p, t.y);
    } else {
      s0 = spec_slot(p, energy_coord_f1(p, P.mu.x));
      s1 = spec_slot(p, energy_coord_f1(p, P.mu.y));
    }
    if (SHIST) {
      atomicAdd(&hs[s0], (H)q0);
      atomicAdd(&hs[s1], (H)q1);
    } else {
      atomicAdd(&p.acc_spec[s0], q0);
      atomicAdd(&p.acc_spec[s1], q1);
    }
  }
  if (ALL || nmap) {
    const float2 fx = mul2(__fadd2_rn(P.thx, f2(p.f.tmax)), f2(p.f.tsx));
    const float2 fy = mul2(__fadd2_rn(P.thy, f2(p.f.tmax)), f2(p.f.tsy));
    const int c0 = map_slot(p, fx.x, fy.x, nmap), c1 = map_slot(p, fx.y, fy.y, nmap);
    if (SHIST) {
      atomicAdd(&hm[c0], (H)q0);
      atomicAdd(&hm[c1], (H)q1);
    } else {
      atomicAdd(&p.acc_map[c0], q0);
      atomicAdd(&p.acc_map[c1], q1);
    }
  }
  if (ALL || naeff) {
    const float2 f = mul2(P.a, f2(p.f.a_scale));
    const int a0 = aeff_slot(p, f.x), a1 = aeff_slot(p, f.y);
    if (SHIST) {
      atomicAdd(&ha[a0], (H)q0);
      atomicAdd(&ha[a1], (H)q1);
    } else {
      atomicAdd(&p.acc_aeff[a0], q0);
      atomicAdd(&p.acc_aeff[a1], q1);
    }
  }
}

// Four classical samples (two pairs; FP32, no variance or electron angle
// terms) into the packed partial sums and the histograms.  If any of the
// four is non-finite or has a negative weight, each goes through
// accumulate_w instead (same skip rule).  W: weights present (else 1).
template <typename H, bool SHIST, bool W, bool ALL>
__device__ __forceinline__ void accumulate4_ll(const Params& p, const LL2& P0, const LL2& P1,
                                               const float4 w4, LLSums& T, AccF& A, H* hs,
                                               H* hm, H* ha, int nspec, int nmap, int naeff) {
  const float2 w01 = make_float2(w4.x, w4.y), w23 = make_float2(w4.z, w4.w);
  bool ok = finitef(P0.mu.x) & finitef(P0.mu.y) & finitef(P1.mu.x) & finitef(P1.mu.y) &
            finitef(P0.thx.x) & finitef(P0.thx.y) & finitef(P1.thx.x) & finitef(P1.thx.y) &
            finitef(P0.thy.x) & finitef(P0.thy.y) & finitef(P1.thy.x) & finitef(P1.thy.y) &
            finitef(P0.a.x) & finitef(P0.a.y) & finitef(P1.a.x) & finitef(P1.a.y) &
            finitef(P0.g0.x) & finitef(P0.g0.y) & finitef(P1.g0.x) & finitef(P1.g0.y);
  if (W)
    ok = ok & (w4.x >= 0.f) & (w4.y >= 0.f) & (w4.z >= 0.f) & (w4.w >= 0.f) & finitef(w4.x) &
         finitef(w4.y) & finitef(w4.z) & finitef(w4.w);
  if (!ok) {
    const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      accumulate_w<H, SHIST, false>(p, ll_sample(k < 2 ? P0 : P1, k & 1), W ? w[k] : 1.f, A, hs,
                                    hm, ha, nspec, nmap, naeff);
    return;
  }
  if (isnan(A.shift)) A.shift = P0.mu.x;
  const float2 nsh = f2(-A.shift);
  const float2 d0 = __fadd2_rn(P0.mu, nsh), d1 = __fadd2_rn(P1.mu, nsh);
  if (W) {
    const float2 wd0 = mul2(w01, d0), wd1 = mul2(w23, d1);
    T.t0 = __fadd2_rn(__fadd2_rn(T.t0, w01), w23);
    T.t1 = __fadd2_rn(__fadd2_rn(T.t1, wd0), wd1);
    T.t2 = fma2(wd1, d1, fma2(wd0, d0, T.t2));
    T.t4 = fma2(mul2(w23, P1.thx), P1.thx, fma2(mul2(w01, P0.thx), P0.thx, T.t4));
    T.t5 = fma2(mul2(w23, P1.thy), P1.thy, fma2(mul2(w01, P0.thy), P0.thy, T.t5));
    T.t6 = fma2(w23, P1.a, fma2(w01, P0.a, T.t6));
    T.t7 = fma2(w23, P1.g0, fma2(w01, P0.g0, T.t7));
  } else {
    T.t0 = __fadd2_rn(T.t0, f2(2.f));
    T.t1 = __fadd2_rn(__fadd2_rn(T.t1, d0), d1);
    T.t2 = fma2(d1, d1, fma2(d0, d0, T.t2));
    T.t4 = fma2(P1.thx, P1.thx, fma2(P0.thx, P0.thx, T.t4));
    T.t5 = fma2(P1.thy, P1.thy, fma2(P0.thy, P0.thy, T.t5));
    T.t6 = __fadd2_rn(__fadd2_rn(T.t6, P0.a), P1.a);
    T.t7 = __fadd2_rn(__fadd2_rn(T.t7, P0.g0), P1.g0);
  }
  ll_deposit<H, SHIST, W, ALL>(p, P0, w01, hs, hm, ha, nspec, nmap, naeff);
  ll_deposit<H, SHIST, W, ALL>(p, P1, w23, hs, hm, ha, nspec, nmap, naeff);
}

template <typename T, typename H, bool SHIST>
__device__ __forceinline__ bool accumulate(const Params& p, const SampleF& s, int64_t i, AccF& A,
                                           H* hs, H* hm, H* ha, int64_t nspec, int64_t nmap,
                                           int64_t naeff) {
  const float w = p.weighted ? load_t<float>(p.w, i, p.dtype) : 1.f;
  return accumulate_w<H, SHIST>(p, s, w, A, hs, hm, ha, nspec, nmap, naeff);
}

// Smoothed-spectrum deposits (fixed point, like the weighted histograms):
// S_k += w exp(-(k + 1/2 - t)^2 / (2 s^2)) / (s sqrt(2 pi)) over the bins
// within 6 s of t.  FP64 path in FP64; FP32 path in FP32 (relative error
// ~1e-7 per deposit).  All 32 lanes call these together (valid = the lane's
// sample entered the sums): the warp's samples are taken one at a time and
// the lanes share out that sample's window of bins, so one atomic
// instruction updates up to 32 consecutive accumulators instead of 32 lanes
// piling onto the same few bins.  Integer sums do not depend on the order.
__device__ __forceinline__ void deposit_smooth_warp(const Params& p, bool valid, double gout,
                                                    double w, unsigned long long* dst) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const double t = (gout - p.lo) * p.inv_w;
  int k0 = 0, k1 = -1;
  if (valid && t > -1e9 && t < 1e9) smooth_range(p, t, &k0, &k1);
  const double wq = w * p.smooth_pref * p.wscale;
  unsigned m = __ballot_sync(full, k1 >= k0);
  while (m) {
    const int j = __ffs(m) - 1;
    m &= m - 1;
    const int a0 = __shfl_sync(full, k0, j), a1 = __shfl_sync(full, k1, j);
    const double tj = __shfl_sync(full, t, j), qj = __shfl_sync(full, wq, j);
    for (int k = a0 + lane; k <= a1; k += 32) {
      const double d = (double)k + 0.5 - tj;
      atomicAdd(&dst[k], (unsigned long long)__double2ll_rn(qj * exp2(-d * d * p.smooth_c)));
    }
  }
}
__device__ __forceinline__ void deposit_smooth_warp_f32(const Params& p, bool valid, float gh,
                                                        float gl, float w,
                                                        unsigned long long* dst) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const float tt = __fmul_rn(__fadd_rn(__fsub_rn(gh, p.f.lo), gl), p.f.inv_w);
  int k0 = 0, k1 = -1;
  if (valid && tt > -1e9f && tt < 1e9f) smooth_range_f32(p, tt, &k0, &k1);
  const float tf = __fsub_rn(tt, (float)k0);            // position relative to bin k0
  const float wq = __fmul_rn(w, p.f.smooth_pw);
  const float c = p.f.smooth_c;
  unsigned m = __ballot_sync(full, k1 >= k0);
  while (m) {
    const int j = __ffs(m) - 1;
    m &= m - 1;
    const int a0 = __shfl_sync(full, k0, j), a1 = __shfl_sync(full, k1, j);
    const float fj = __shfl_sync(full, tf, j), qj = __shfl_sync(full, wq, j);
    for (int k = a0 + lane; k <= a1; k += 32) {
      const float d = __fsub_rn((float)(k - a0) + 0.5f, fj);
      const float e = M<float>::ex2(-__fmul_rn(__fmul_rn(d, d), c));
      const float x = __fmul_rn(qj, e);
      atomicAdd(&dst[k], x < 4294967296.f ? (unsigned long long)__float2uint_rn(x) : f2u64_rn(x));
    }
  }
}
// What a deposit needs of a sample: its realised energy.
struct DepD { double g = 0.0; };
struct DepF { float gh = 0.f, gl = 0.f; };
template <typename T> struct DepT;
template <> struct DepT<double> { using type = DepD; };
template <> struct DepT<float> { using type = DepF; };
__device__ __forceinline__ void dep_set(DepD& d, const Sample& s) { d.g = s.gout; }
__device__ __forceinline__ void dep_set(DepF& d, const SampleF& s) { d.gh = s.go_hi; d.gl = s.go_lo; }
__device__ __forceinline__ void deposit_warp(const Params& p, bool valid, const DepD& d,
                                             int64_t i, unsigned long long* dst) {
  const double w = valid && p.weighted ? load_elem(p.w, i, p.dtype) : 1.0;
  deposit_smooth_warp(p, valid, d.g, w, dst);
}
__device__ __forceinline__ void deposit_warp(const Params& p, bool valid, const DepF& d,
                                             int64_t i, unsigned long long* dst) {
  const float w = valid && p.weighted ? load_t<float>(p.w, i, p.dtype) : 1.f;
  deposit_smooth_warp_f32(p, valid, d.gh, d.gl, w, dst);
}

}  // namespace qs

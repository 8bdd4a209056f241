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
constexpr int kNumMom = 9;   // W, sum w d, sum w d^2, sum w V, sum w thx^2,
                             // sum w thy^2, sum w a_eff, sum w gamma0, #excluded

// Everything a launch needs, derived on the host from the descriptors and
// passed by value (kernel parameter space: uniform, cached, stream-safe).
struct Params {
  // laser (Eq. 2, Eq. 3, Eq. 6)
  double a0, inv_w0sq, inv_zR, ldx, ldy, c_delay;
  double cRR;          // (2/3) R_c * integral G^2               (Eq. 3)
  double cK;           // (2/3) R_c: K = cK A^2, loss per phase   (Eq. 6)
  double cchi;         // sqrt2 / a_S: chi = cchi mu A at rms field
  double h, win_lo, Phi, PhiT;
  double kappa_s;      // kappa sqrt(2/pi)                         (Eq. 8)
  int32_t envelope, model, n_phase, pad0;
  // beam
  double gmean, spread, glo, gspan, sx, sy, sz, div, bdx, bdy;
  int32_t flat, pad1;
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
  int32_t hist_in_smem, pad3;
};

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

struct Sample {
  double gamma0, aeff, mu, V, theta_e, thx0, thy0, tx, ty, gout;
};

// Quantum-corrected Fokker-Planck phase integration (Eq. 6; mean/variance
// closure of the Fokker-Planck regime), second order in the cell width h:
// rates at each cell midpoint, midpoint state predicted with the previous
// cell's Gaunt factor, frozen-rate Taylor step for the linear variance ODE.
//   g(chi)  = B^(-2/3), B  = 1 + 4.8 (1+chi) ln(1+1.7 chi) + 2.44 chi^2
//   h2(chi) = B2^(-7/6), B2 = 1 + (1+4.1 chi) ln(1+12.93 chi) + 4.75 chi^2
//   K = (2/3) R_c A^2, D1 = -K mu^2 g, dD1/dgamma = -K mu (2g + chi g'),
//   D2 = (55/(16 sqrt3)) K mu^3 chi h2.
// Returns du = 1/mu_f - 1/gamma0 and V_f.
template <typename T>
__device__ __forceinline__ void qfp_integrate(const Params& p, const T* __restrict__ sG, T a,
                                              T g0, T& du_out, T& V_out) {
  const T LN2 = (T)0.69314718055994530942;
  const T cK = (T)p.cK, cchi = (T)p.cchi, h = (T)p.h;
  const T c55 = (T)(55.0 / (16.0 * 1.7320508075688772935));
  const T hh2 = (T)(0.5 * p.h * p.h);
  T du = 0, V = 0, gprev = 1;
  const int N = p.n_phase;
#pragma unroll 2
  for (int j = 0; j < N; ++j) {
    T A = a * sG[j];
    T K = cK * A * A;
    T hK = h * K;
    T dum = du + (T)0.5 * hK * gprev;
    T mu = g0 * M<T>::rcp((T)1 + g0 * dum);
    T chi = cchi * mu * A;
    // Gaunt factor and chi g'(chi)
    T x1 = (T)1 + (T)1.7 * chi;
    T L1 = LN2 * M<T>::lg2(x1);
    T opc = (T)1 + chi;
    T B = (T)1 + (T)4.8 * opc * L1 + (T)2.44 * chi * chi;
    T t = M<T>::ex2((T)(-1.0 / 3.0) * M<T>::lg2(B));     // B^(-1/3)
    T g = t * t;
    T dB = (T)4.8 * L1 + (T)(4.8 * 1.7) * opc * M<T>::rcp(x1) + (T)4.88 * chi;
    T chig1 = (T)(-2.0 / 3.0) * g * (t * t * t) * dB * chi;
    // second-moment factor
    T L2 = LN2 * M<T>::lg2((T)1 + (T)12.93 * chi);
    T B2 = (T)1 + ((T)1 + (T)4.1 * chi) * L2 + (T)4.75 * chi * chi;
    T h2 = M<T>::ex2((T)(-7.0 / 6.0) * M<T>::lg2(B2));
    // updates
    du = du + hK * g;
    T lam = (T)-2 * K * mu * ((T)2 * g + chig1);
    T D2 = c55 * K * mu * mu * mu * chi * h2;
    T r = lam * V + D2;
    V = V + h * r + hh2 * lam * r;
    gprev = g;
  }
  du_out = du;
  V_out = V;
}

// One beam sample through the model, in the paper's order.
template <typename T>
__device__ __forceinline__ Sample eval_sample(const Params& p, const T* __restrict__ sG,
                                              int64_t i) {
  Sample s;
  // decode (reparameterised)
  T xi0 = (T)load_elem(p.xi[0], i, p.dtype);
  T xi1 = (T)load_elem(p.xi[1], i, p.dtype);
  T xi2 = (T)load_elem(p.xi[2], i, p.dtype);
  double xi3 = load_elem(p.xi[3], i, p.dtype);
  T xi4 = (T)load_elem(p.xi[4], i, p.dtype);
  T xi5 = (T)load_elem(p.xi[5], i, p.dtype);
  T x = (T)p.bdx + (T)p.sx * xi0;
  T y = (T)p.bdy + (T)p.sy * xi1;
  T z = (T)p.sz * xi2;
  double gamma0 = p.flat ? p.glo + p.gspan * xi3 : p.gmean * (1.0 + p.spread * xi3);
  if (gamma0 < 1.0) gamma0 = 1.0;
  T thx = (T)p.div * xi4;
  T thy = (T)p.div * xi5;
  // collision geometry: crossing of the pulse peak (factor 2 of Eq. 1)
  T ct = (T)0.5 * (z + (T)p.c_delay);
  T zs = (T)0.5 * (z - (T)p.c_delay);
  T xs = x + thx * ct - (T)p.ldx;
  T ys = y + thy * ct - (T)p.ldy;
  T rho2 = xs * xs + ys * ys;
  // local Gaussian focus, Eq. 2
  T zq = zs * (T)p.inv_zR;
  T q = (T)1 + zq * zq;
  T rq = M<T>::rcp(q);
  T a;
  if (sizeof(T) == 4)
    a = (T)p.a0 * M<T>::rsqrt(q) *
        M<T>::ex2(-(T)1.4426950408889634074 * rho2 * (T)p.inv_w0sq * rq);
  else
    a = (T)p.a0 * M<T>::rsqrt(q) * (T)exp((double)(-rho2 * (T)p.inv_w0sq * rq));
  double mu, V = 0.0;
  if (p.model == 0) {
    if (sizeof(T) == 4) {
      T du = (T)p.cRR * a * a;          // Eq. 3 as 1/gamma_f - 1/gamma_0
      mu = gamma0 / (1.0 + gamma0 * (double)du);
    } else {
      double ad = (double)a;
      mu = gamma0 / (1.0 + p.cRR * gamma0 * ad * ad);
    }
  } else {
    T du, Vt;
    qfp_integrate<T>(p, sG, a, (T)gamma0, du, Vt);
    mu = gamma0 / (1.0 + gamma0 * (double)du);   // FP64 recombination
    V = (double)Vt;
  }
  double ad = (double)a;
  double theta_e = 0.0, gout = mu;
  double tx = (double)thx, ty = (double)thy;
  if (p.model != 0) {
    double sv = V > 0.0 ? sqrt(V) : 0.0;
    theta_e = p.kappa_s * ad * sv / (mu * mu);       // Eq. 8
    tx += theta_e * load_elem(p.xi[6], i, p.dtype);
    gout = mu + sv * load_elem(p.xi[7], i, p.dtype);
  }
  s.gamma0 = gamma0; s.aeff = ad; s.mu = mu; s.V = V; s.theta_e = theta_e;
  s.thx0 = (double)thx; s.thy0 = (double)thy; s.tx = tx; s.ty = ty; s.gout = gout;
  return s;
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

__device__ __forceinline__ int aeff_bin(const Params& p, double a) {
  double f = a * p.a_scale;
  if (f >= 0.0 && f < (double)p.n_aeff) return (int)f;
  return p.n_aeff;
}

}  // namespace qs

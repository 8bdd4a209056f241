// qs_grad.cu -- adjoint of the beam phase-space integration (qs_scatter_grad).
//
// K3 k_grad         per sample: recompute the forward with two tangents
//                   (d/d a_eff, d/d gamma0) carried through the discretised
//                   phase integration, form the sample's share of dL/d(outputs)
//                   from the upstream gradient, chain-rule it to the 8
//                   parameters, reduce per CTA in a fixed order.
// K4 k_grad_final   one CTA: per-CTA partials summed in CTA order.
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348 -- Eqs. 2, 3, 6, 8 and
// the reconstruction use of Sec. 6.
#include "qscatter.h"
#include "qs_device.cuh"
#include "qs_host.hpp"

#include <cmath>

namespace qs {

constexpr int kNumGrad = QS_NUM_GRAD;

// Tangents of the phase integration.
template <typename T>
struct QfpTan {
  T du, V, du_a, du_g, V_a, V_g;
};

__device__ __forceinline__ void tab_g(const float4* t, int j, float& G, float& G2) {
  const float4 e = t[j];
  G = e.x;
  G2 = e.z;
}
__device__ __forceinline__ void tab_g(const double* t, int j, double& G, double& G2) {
  G = t[j];
  G2 = G * G;
}

// Forward-mode derivative of the discretised phase integration of qs_device
// (same cells, same midpoint prediction, same frozen-rate variance step),
// with respect to a (= a_eff) and g (= gamma0).  g(chi), h2(chi) and their
// derivatives are taken from the closed forms:
//   g  = B^(-2/3),  g'  = -(2/3) B^(-5/3) B',
//   g'' = (10/9) B^(-8/3) B'^2 - (2/3) B^(-5/3) B'',
//   B' = 4.8 ln(1+1.7chi) + 8.16 (1+chi)/(1+1.7chi) + 4.88 chi,
//   B'' = 8.16/(1+1.7chi) - 5.712/(1+1.7chi)^2 + 4.88,
//   h2 = B2^(-7/6), h2' = -(7/6) h2 B2'/B2,
//   B2' = 4.1 ln(1+12.93chi) + 12.93 (1+4.1chi)/(1+12.93chi) + 9.5 chi.
template <typename T>
__device__ __forceinline__ void qfp_tangent(const Params& p,
                                            const typename Tab<T>::type* __restrict__ tab, T a,
                                            T g0, QfpTan<T>& o) {
  const T LN2 = (T)0.69314718055994530942;
  const T C55 = (T)(55.0 / (16.0 * 1.7320508075688772935));
  const T h = (T)p.h, cK = (T)p.cK, cchi = (T)p.cchi;
  const T c1 = h * cK * a * a, c1a = (T)2 * h * cK * a;
  const T ca = cchi * a;
  T du = 0, V = 0, gph = (T)0.5, du_a = 0, du_g = 0, V_a = 0, V_g = 0, gph_a = 0, gph_g = 0;
  const int N = p.n_phase;
  for (int j = 0; j < N; ++j) {
    T G, G2;
    tab_g(tab, j, G, G2);
    const T hK = c1 * G2, hK_a = c1a * G2;
    const T dum = du + hK * gph;
    const T dum_a = du_a + hK_a * gph + hK * gph_a;
    const T dum_g = du_g + hK * gph_g;
    const T r = M<T>::rcp((T)1 + g0 * dum);
    const T mu = g0 * r;
    const T mu_a = -mu * r * (g0 * dum_a);
    const T mu_g = r - mu * r * (dum + g0 * dum_g);
    const T cg = ca * G;
    const T chi = cg * mu;
    const T chi_a = cchi * G * mu + cg * mu_a;
    const T chi_g = cg * mu_g;
    // Gaunt factor and derivatives
    const T x1 = (T)1 + (T)1.7 * chi;
    const T l1 = M<T>::lg2(x1);
    const T L1 = LN2 * l1;
    const T r1 = M<T>::ex2(-l1);
    const T opc = (T)1 + chi;
    const T B = (T)1 + (T)4.8 * opc * L1 + (T)2.44 * chi * chi;
    const T t = M<T>::ex2((T)(-1.0 / 3.0) * M<T>::lg2(B));
    const T g = t * t, iB = t * t * t;
    const T Bp = (T)4.8 * L1 + (T)8.16 * opc * r1 + (T)4.88 * chi;
    const T Bpp = (T)8.16 * r1 - (T)5.712 * r1 * r1 + (T)4.88;
    const T gp = (T)(-2.0 / 3.0) * g * iB * Bp;
    const T gpp = (T)(10.0 / 9.0) * g * iB * iB * Bp * Bp - (T)(2.0 / 3.0) * g * iB * Bpp;
    const T s = (T)2 * g + chi * gp;
    const T s_chi = (T)3 * gp + chi * gpp;
    // second-moment factor and derivative
    const T l2 = M<T>::lg2((T)1 + (T)12.93 * chi);
    const T L2 = LN2 * l2;
    const T r2 = M<T>::ex2(-l2);
    const T B2 = (T)1 + ((T)1 + (T)4.1 * chi) * L2 + (T)4.75 * chi * chi;
    const T lb2 = M<T>::lg2(B2);
    const T h2 = M<T>::ex2((T)(-7.0 / 6.0) * lb2);
    const T iB2 = M<T>::ex2(-lb2);
    const T B2p = (T)4.1 * L2 + (T)12.93 * ((T)1 + (T)4.1 * chi) * r2 + (T)9.5 * chi;
    const T h2p = (T)(-7.0 / 6.0) * h2 * iB2 * B2p;
    // mean
    const T du_n = du + hK * g;
    const T du_a_n = du_a + hK_a * g + hK * gp * chi_a;
    const T du_g_n = du_g + hK * gp * chi_g;
    // variance
    const T hKmu = hK * mu;
    const T hlam = (T)-2 * hKmu * s;
    const T hlam_a = (T)-2 * (hK_a * mu * s + hK * mu_a * s + hKmu * s_chi * chi_a);
    const T hlam_g = (T)-2 * (hK * mu_g * s + hKmu * s_chi * chi_g);
    const T m2 = mu * mu;
    const T hD2 = C55 * hKmu * m2 * chi * h2;
    const T hh = h2 + chi * h2p;
    const T hD2_a = C55 * m2 * ((hK_a * mu + (T)3 * hK * mu_a) * chi * h2 + hKmu * chi_a * hh);
    const T hD2_g = C55 * m2 * ((T)3 * hK * mu_g * chi * h2 + hKmu * chi_g * hh);
    const T hr = hlam * V + hD2;
    const T hr_a = hlam_a * V + hlam * V_a + hD2_a;
    const T hr_g = hlam_g * V + hlam * V_g + hD2_g;
    const T fac = (T)1 + (T)0.5 * hlam;
    const T V_n = V + hr * fac;
    const T V_a_n = V_a + hr_a * fac + (T)0.5 * hr * hlam_a;
    const T V_g_n = V_g + hr_g * fac + (T)0.5 * hr * hlam_g;
    du = du_n; du_a = du_a_n; du_g = du_g_n;
    V = V_n; V_a = V_a_n; V_g = V_g_n;
    gph = (T)0.5 * g;
    gph_a = (T)0.5 * gp * chi_a;
    gph_g = (T)0.5 * gp * chi_g;
  }
  o.du = du; o.V = V; o.du_a = du_a; o.du_g = du_g; o.V_a = V_a; o.V_g = V_g;
}

// Upstream gradient, reduced to the per-sample coefficients it needs.
struct Seeds {
  double invW, mean, spread, dxr, dyr;        // forward moments
  double gM, gSp, gDx, gDy, gA, gG0;          // effective dL/d(mean, spread, div_x, div_y, a, g0)
};

template <typename T, bool QFP>
__global__ void __launch_bounds__(256) k_grad(const Params p, const qs_moments* __restrict__ mom,
                                              const double* __restrict__ dLdm,
                                              const double* __restrict__ dLdS) {
  using TT = typename Tab<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  TT* tab = reinterpret_cast<TT*>(smem);
  const size_t tab_bytes = QFP ? (((size_t)p.n_phase * sizeof(TT) + 15) & ~(size_t)15) : 0;
  double* red = reinterpret_cast<double*>(smem + tab_bytes);
  if (QFP)
    for (int j = threadIdx.x; j < p.n_phase; j += blockDim.x) table_entry(p, j, tab);

  // effective upstream coefficients (rel_spread = spread/mean,
  // div = sqrt(div_x^2 + div_y^2) folded into mean, spread, div_x, div_y)
  Seeds sd;
  {
    const double W = mom->W;
    sd.invW = W > 0.0 ? 1.0 / W : 0.0;
    sd.mean = mom->mean;
    sd.spread = mom->spread;
    const double Dx = mom->div_x, Dy = mom->div_y, D = mom->div;
    const double d1 = dLdm[1], d2 = dLdm[2], d3 = dLdm[3], d4 = dLdm[4], d5 = dLdm[5],
                 d6 = dLdm[6];
    sd.gM = d1 - (sd.mean != 0.0 ? d3 * sd.spread / (sd.mean * sd.mean) : 0.0);
    sd.gSp = d2 + (sd.mean != 0.0 ? d3 / sd.mean : 0.0);
    sd.gDx = d4 + (D > 0.0 ? d6 * Dx / D : 0.0);
    sd.gDy = d5 + (D > 0.0 ? d6 * Dy / D : 0.0);
    sd.dxr = Dx > 0.0 ? 1.0 / Dx : 0.0;
    sd.dyr = Dy > 0.0 ? 1.0 / Dy : 0.0;
    sd.gA = dLdm[7];
    sd.gG0 = dLdm[11];
  }
  __syncthreads();

  double acc[kNumGrad];
#pragma unroll
  for (int k = 0; k < kNumGrad; ++k) acc[k] = 0.0;

  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
    // ---- decode and focus with derivatives (rows a1-a3) ----
    const double xi0 = load_elem(p.xi[0], i, p.dtype), xi1 = load_elem(p.xi[1], i, p.dtype);
    const double xi2 = load_elem(p.xi[2], i, p.dtype), xi3 = load_elem(p.xi[3], i, p.dtype);
    const double xi4 = load_elem(p.xi[4], i, p.dtype), xi5 = load_elem(p.xi[5], i, p.dtype);
    const double w = p.weighted ? load_elem(p.w, i, p.dtype) : 1.0;
    if (!(w >= 0.0) || !isfinite(w)) continue;
    const T x = (T)p.bdx + (T)p.sx * (T)xi0;
    const T y = (T)p.bdy + (T)p.sy * (T)xi1;
    const T z = (T)p.sz * (T)xi2;
    double gamma0 = p.flat ? p.glo + p.gspan * xi3 : p.gmean * (1.0 + p.spread * xi3);
    const bool clamped = gamma0 < 1.0;
    if (clamped) gamma0 = 1.0;
    const T thx = (T)p.div * (T)xi4, thy = (T)p.div * (T)xi5;
    const T ct = (T)0.5 * (z + (T)p.c_delay);
    const T zs = (T)0.5 * (z - (T)p.c_delay);
    const T xs = x + thx * ct - (T)p.ldx;
    const T ys = y + thy * ct - (T)p.ldy;
    const T rho2 = xs * xs + ys * ys;
    const T zq = zs * (T)p.inv_zR;
    const T q = (T)1 + zq * zq;
    const T rq = M<T>::rcp(q);
    const T E = rho2 * (T)p.inv_w0sq * rq;              // a = a0 q^-1/2 exp(-E)
    T a_over_a0;
    if (sizeof(T) == 4)
      a_over_a0 = M<T>::rsqrt(q) * M<T>::ex2(-(T)1.4426950408889634074 * E);
    else
      a_over_a0 = M<T>::rsqrt(q) * (T)exp(-(double)E);
    const T a = (T)p.a0 * a_over_a0;
    // d ln a / d(parameter)
    const T w0 = (T)sqrt(1.0 / p.inv_w0sq);
    const T k2 = (T)2 * (T)p.inv_w0sq * rq;             // 2 / (W0^2 q)
    const T dla_dx = k2 * xs, dla_dy = k2 * ys;
    const T dla_thx = -k2 * xs * ct, dla_thy = -k2 * ys * ct;
    const T cc = (T)0.299792458;
    const T dq_del = -cc * zq * (T)p.inv_zR;             // dq/d delay
    const T drho_del = cc * (xs * thx + ys * thy);       // d rho^2 / d delay
    const T dla_del = (E - (T)0.5) * dq_del * rq - drho_del * (T)p.inv_w0sq * rq;
    const T dq_w0 = (T)-4 * zq * zq / w0;                // dq/dW0 (z_R ~ W0^2)
    const T dla_w0 = (T)-0.5 * dq_w0 * rq + E * ((T)2 / w0 + dq_w0 * rq);

    // ---- model with tangents (rows a4-a5) ----
    double mu, V = 0.0, mu_a, mu_g, V_a = 0.0, V_g = 0.0;
    if (!QFP) {
      const double ad = (double)a;
      mu = gamma0 / (1.0 + p.cRR * gamma0 * ad * ad);
      mu_a = -mu * mu * 2.0 * p.cRR * ad;
      mu_g = mu * mu / (gamma0 * gamma0);
    } else {
      QfpTan<T> o;
      qfp_tangent<T>(p, tab, a, (T)gamma0, o);
      mu = gamma0 / (1.0 + gamma0 * (double)o.du);
      mu_a = -mu * mu * (double)o.du_a;
      mu_g = mu * mu * (1.0 / (gamma0 * gamma0) - (double)o.du_g);
      V = (double)o.V;
      V_a = (double)o.V_a;
      V_g = (double)o.V_g;
    }
    if (!isfinite(mu) || !isfinite(V)) continue;
    // ---- outputs of the sample (row a6) ----
    const double ad = (double)a;
    double theta_e = 0.0, gout = mu, sv = 0.0;
    const double xi7 = QFP ? load_elem(p.xi[7], i, p.dtype) : 0.0;
    if (QFP && V > 0.0) {
      sv = sqrt(V);
      theta_e = p.kappa_s * ad * sv / (mu * mu);
      gout = mu + sv * xi7;
    }
    const double thx0 = (double)thx, thy0 = (double)thy;

    // ---- sample's share of dL/d(outputs) (adjoint of rows a8-a9) ----
    const double wn = w * sd.invW;
    double g_out = 0.0;                                   // dL/d gamma_out
    if (dLdS != nullptr && p.smooth_sigma > 0.0) {
      const double tt = (gout - p.lo) * p.inv_w;
      if (tt > -1e9 && tt < 1e9) {
        int k0, k1;
        smooth_range(p, tt, &k0, &k1);
        const double sg2 = p.smooth_sigma * p.smooth_sigma;
        if (sizeof(T) == 4) {
          // FP32 path: Gaussian weights in FP32 (as in the forward deposit)
          const float tf = (float)(tt - (double)k0);
          const float c = (float)p.smooth_c;
          float ga = 0.f;
          for (int k = k0; k <= k1; ++k) {
            const float d = (float)(k - k0) + 0.5f - tf;
            ga = fmaf((float)dLdS[k] * M<float>::ex2(-(d * d) * c), d, ga);
          }
          g_out = (double)ga;
        } else {
          for (int k = k0; k <= k1; ++k) {
            const double d = (double)k + 0.5 - tt;
            g_out += dLdS[k] * exp2(-d * d * p.smooth_c) * d;
          }
        }
        g_out *= w * p.smooth_pref * p.inv_w / sg2;
      }
    }
    double g_mu = sd.gM * wn + g_out;
    if (sd.spread > 0.0) g_mu += sd.gSp * wn * (mu - sd.mean) / sd.spread;
    double g_V = (sd.spread > 0.0 ? sd.gSp * wn * 0.5 / sd.spread : 0.0);
    if (QFP && V > 0.0) g_V += g_out * xi7 * 0.5 / sv;
    const double g_te = sd.gDx * wn * theta_e * sd.dxr;
    double g_thx = sd.gDx * wn * thx0 * sd.dxr;
    double g_thy = sd.gDy * wn * thy0 * sd.dyr;
    double g_a = sd.gA * wn;
    double g_g0 = sd.gG0 * wn;
    // theta_e = kappa_s a sqrt(V) / mu^2
    if (QFP && V > 0.0) {
      g_a += g_te * p.kappa_s * sv / (mu * mu);
      g_V += g_te * p.kappa_s * ad * 0.5 / (sv * mu * mu);
      g_mu += g_te * (-2.0 * theta_e / mu);
    }
    // (mu, V) = F(a, gamma0)
    g_a += g_mu * mu_a + g_V * V_a;
    g_g0 += g_mu * mu_g + g_V * V_g;

    // ---- chain to the parameters ----
    const double ga = g_a * ad;                           // dL/d ln a
    acc[QS_G_A0] += p.a0 > 0.0 ? g_a * (double)a_over_a0 : 0.0;
    acc[QS_G_W0] += ga * (double)dla_w0;
    acc[QS_G_DX] += ga * (double)dla_dx;
    acc[QS_G_DY] += ga * (double)dla_dy;
    acc[QS_G_DELAY] += ga * (double)dla_del;
    if (!p.flat && !clamped) {
      acc[QS_G_GAMMA] += g_g0 * (1.0 + p.spread * xi3);
      acc[QS_G_SPREAD] += g_g0 * p.gmean * xi3;
    }
    acc[QS_G_DIV] += (g_thx + ga * (double)dla_thx) * xi4 + (g_thy + ga * (double)dla_thy) * xi5;
  }

  // fixed-order block reduction into this CTA's slot
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNumGrad; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp * kNumGrad + k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNumGrad) {
    double s = 0.0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[wv * kNumGrad + threadIdx.x];
    p.partials[(size_t)blockIdx.x * kNumMom + threadIdx.x] = s;
  }
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

template <typename T, bool QFP>
int32_t launch_grad(const Params& p, int block, int sms, int grid_req, int gmax,
                    const qs_moments* mom, const double* dLdm, const double* dLdS,
                    cudaStream_t st, int* grid_out) {
  using TT = typename Tab<T>::type;
  const size_t tab = QFP ? align_up((size_t)p.n_phase * sizeof(TT), 16) : 0;
  const size_t smem = tab + (size_t)(block / 32) * kNumGrad * sizeof(double);
  auto kern = k_grad<T, QFP>;
  static bool attr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QS_ERR_CUDA;
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit) !=
        cudaSuccess)
      return cuda_fail();
    attr[dev] = true;
  }
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
  if (block > 256) block = 256;
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
  int g = 1;
  if (prec == QS_F64)
    st = qfp ? launch_grad<double, true>(p, block, sms, grid, pl.gmax, d_moments, d_dL_dmoments,
                                         d_dL_dsmooth, cs, &g)
             : launch_grad<double, false>(p, block, sms, grid, pl.gmax, d_moments, d_dL_dmoments,
                                          d_dL_dsmooth, cs, &g);
  else
    st = qfp ? launch_grad<float, true>(p, block, sms, grid, pl.gmax, d_moments, d_dL_dmoments,
                                        d_dL_dsmooth, cs, &g)
             : launch_grad<float, false>(p, block, sms, grid, pl.gmax, d_moments, d_dL_dmoments,
                                         d_dL_dsmooth, cs, &g);
  if (st) return st;
  k_grad_final<<<1, 32, 0, cs>>>(p, g, d_grad8);
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

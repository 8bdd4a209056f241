// qs_analytic.cu -- analytic distributions on a grid (qs_analytic_aeff,
// qs_analytic_ll_spectrum): the cross-check fast path of Table 1 and Table 2.
//
// K10 k_analytic  one thread per grid point, FP64: dN/da_eff of an idealised
//                 beam (Table 1), or the classical final-energy density
//                 dN/dgamma = (dN/da)(a(gamma)) / |dgamma/da| (Eq. 6 with
//                 Eq. 3, Table 2).
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348, Table 1, Eq. 3,
// Eq. 6, Table 2.
#include "qscatter.h"
#include "qs_device.cuh"
#include "qs_host.hpp"
#include "qs_derive.cuh"

#include <cmath>

namespace qs {

// I0(x): power series for x <= 30, asymptotic expansion above.
__device__ double bessel_i0_d(double x) {
  x = fabs(x);
  if (x <= 30.0) {
    double t = 1.0, s = 1.0;
    const double q = 0.25 * x * x;
    for (int k = 1; k < 200; ++k) {
      t *= q / ((double)k * k);
      s += t;
      if (t < 1e-17 * s) break;
    }
    return s;
  }
  const double y = 1.0 / (8.0 * x);
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 30; ++k) {
    t *= (2.0 * k - 1.0) * (2.0 * k - 1.0) * y / k;
    s += t;
    if (fabs(t) < 1e-17) break;
  }
  return exp(x) / sqrt(2.0 * 3.14159265358979323846 * x) * s;
}

struct Geo {
  int kind;
  double a0, w0, zR, R, Lb, dperp, dpar, count, cRR, gamma0;
};

// Table 1 with its readings: the short beam's support is a < a_par; the
// collision positions of a beam of length L span L/2 around d_par.
__device__ double aeff_density(const Geo& g, double a) {
  if (!(a > 0.0)) return 0.0;
  if (g.kind == QS_GEOM_SHORT) {
    const double W = g.w0 * sqrt(1.0 + g.dpar * g.dpar / (g.zR * g.zR)), apar = g.a0 * g.w0 / W;
    if (!(a < apar)) return 0.0;
    const double k = W * W / (g.R * g.R);
    return g.count * k / a * pow(a / apar, k) *
           bessel_i0_d(2.0 * (g.dperp / g.R) * (W / g.R) * sqrt(log(apar / a))) *
           exp(-g.dperp * g.dperp / (g.R * g.R));
  }
  if (!(a < g.a0)) return 0.0;
  const double za = g.zR * sqrt(g.a0 * g.a0 / (a * a) - 1.0);
  const double zm = g.dpar - g.Lb / 4.0, zp = g.dpar + g.Lb / 4.0;
  if (g.kind == QS_GEOM_THIN) {
    const int roots = (za >= zm && za <= zp) + (-za >= zm && -za <= zp);
    return roots * (2.0 * g.count * g.zR / g.Lb) * (g.a0 * g.a0 / (a * a)) /
           sqrt(g.a0 * g.a0 - a * a);
  }
  const double lo = zm > -za ? zm : -za, hi = zp < za ? zp : za;
  if (!(hi > lo)) return 0.0;
  const double Fh = hi * (1.0 + hi * hi / (3.0 * g.zR * g.zR));
  const double Fl = lo * (1.0 + lo * lo / (3.0 * g.zR * g.zR));
  return 2.0 * 3.14159265358979323846 * g.count * g.w0 * g.w0 / a * (Fh - Fl);
}

// ll: x is gamma and the output dN/dgamma; otherwise x is a_eff.
__global__ void k_analytic(Geo g, bool ll, int64_t n, const double* __restrict__ x,
                           double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    double r = 0.0;
    if (!ll) {
      r = aeff_density(g, v);
    } else if (v > 0.0 && v < g.gamma0) {
      const double a = sqrt((g.gamma0 - v) / (g.cRR * g.gamma0 * v));
      r = aeff_density(g, a) / (2.0 * a * g.cRR * v * v);
    }
    out[i] = r;
  }
}

namespace {

int32_t analytic(const qs_laser* laser, const qs_geometry* geom, bool ll, double gamma0,
                 int64_t n, const double* d_x, double* d_out, void* stream) {
  int32_t st;
  if ((st = detail::validate_laser(laser))) return st;
  if (!geom || n < 0 || (n > 0 && (!d_x || !d_out))) return QS_ERR_INVALID_ARG;
  if (geom->kind < QS_GEOM_SHORT || geom->kind > QS_GEOM_WIDE) return QS_ERR_INVALID_ARG;
  if (geom->kind == QS_GEOM_SHORT && !(geom->radius_um > 0.0)) return QS_ERR_INVALID_ARG;
  if (geom->kind != QS_GEOM_SHORT && !(geom->length_um > 0.0)) return QS_ERR_INVALID_ARG;
  if (!std::isfinite(geom->d_perp_um) || !std::isfinite(geom->d_par_um) ||
      !(geom->count >= 0.0) || !std::isfinite(geom->count))
    return QS_ERR_INVALID_ARG;
  if (ll && !(gamma0 > 1.0 && std::isfinite(gamma0))) return QS_ERR_INVALID_ARG;
  if (n == 0) return QS_OK;
  Params p;
  derive_params(p, *laser, qs_beam{1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0, 0},
                nullptr, 32);
  Geo g;
  g.kind = geom->kind;
  g.a0 = laser->a0;
  g.w0 = laser->w0_um;
  g.zR = 1.0 / p.inv_zR;
  g.R = geom->radius_um;
  g.Lb = geom->length_um;
  g.dperp = geom->d_perp_um;
  g.dpar = geom->d_par_um;
  g.count = geom->count;
  g.cRR = p.cRR;
  g.gamma0 = gamma0;
  const int64_t blocks = (n + 255) / 256;
  k_analytic<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      g, ll, n, d_x, d_out);
  return cudaGetLastError() == cudaSuccess ? QS_OK : detail::cuda_fail();
}

}  // namespace
}  // namespace qs

extern "C" int32_t qs_analytic_aeff(const qs_laser* laser, const qs_geometry* geom, int64_t n,
                                    const double* d_a, double* d_out, void* stream) {
  return qs::analytic(laser, geom, false, 0.0, n, d_a, d_out, stream);
}

extern "C" int32_t qs_analytic_ll_spectrum(const qs_laser* laser, const qs_geometry* geom,
                                           double gamma0, int64_t n, const double* d_gamma,
                                           double* d_out, void* stream) {
  return qs::analytic(laser, geom, true, gamma0, n, d_gamma, d_out, stream);
}

// qs_derive.cuh -- descriptor validation and derived launch constants,
// usable on the host (single shot) and on the device (batched shots, where
// the descriptors live in device memory).
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348 (Eq. 2, Eq. 3, Eq. 6,
// Eq. 8; the envelope, window and constant readings are stated with each
// quantity below).
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "qscatter.h"
#include "qs_device.cuh"

#define QS_HD __host__ __device__ __forceinline__

namespace qs {

namespace cst {
constexpr double kC = 0.299792458;          // um / fs
constexpr double kRe = 2.8179403262e-9;     // classical electron radius, um (CODATA 2018)
constexpr double kLbarC = 3.8615926796e-7;  // reduced Compton wavelength, um (CODATA 2018)
constexpr double kPi = 3.14159265358979323846;
constexpr double kGaussWindow = 2.5;        // half-window of the Gaussian envelope in Phi
// Mathematical constants as literals (40-digit values rounded to double), so
// host and device derive bit-identical launch constants:
constexpr double kSin2Fwhm = 0.3640566637738767130;    // 1 - (2/pi) asin(2^-1/4)
constexpr double kGaussIntG2 = 1.0644670194312261793;  // sqrt(pi / (4 ln 2))
constexpr double kSqrt2 = 1.4142135623730950488;
constexpr double kSqrt2OverPi = 0.79788456080286535588;
constexpr double kSqrt2Pi = 2.5066282746310005024;
}  // namespace cst

QS_HD bool qs_fin(double x) {
#ifdef __CUDA_ARCH__
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  std::memcpy(&u, &x, sizeof(u));
#endif
  return ((u >> 52) & 0x7ffull) != 0x7ffull;
}
QS_HD bool qs_pos(double v) { return qs_fin(v) && v > 0.0; }
QS_HD bool qs_nonneg(double v) { return qs_fin(v) && v >= 0.0; }

QS_HD int32_t check_laser(const qs_laser& L) {
  if (!qs_pos(L.lambda_um) || !qs_nonneg(L.a0) || !qs_pos(L.w0_um) || !qs_pos(L.tau_fs) ||
      !qs_fin(L.dx_um) || !qs_fin(L.dy_um) || !qs_fin(L.delay_fs) || !qs_nonneg(L.div_prefactor))
    return QS_ERR_INVALID_ARG;
  if (L.envelope != QS_ENV_GAUSS && L.envelope != QS_ENV_SIN2) return QS_ERR_INVALID_ARG;
  if (L.model != QS_MODEL_LL && L.model != QS_MODEL_QFP) return QS_ERR_INVALID_ARG;
  if (L.variant & ~(QS_VARIANT_CELL_FOCUS | QS_VARIANT_CYCLE_CHI)) return QS_ERR_INVALID_ARG;
  if ((L.variant & QS_VARIANT_CYCLE_CHI) && L.model != QS_MODEL_QFP) return QS_ERR_INVALID_ARG;
  if ((L.model == QS_MODEL_QFP || (L.variant & QS_VARIANT_CELL_FOCUS)) &&
      (L.n_phase < 1 || L.n_phase > kMaxPhase))
    return QS_ERR_INVALID_ARG;
  return QS_OK;
}

QS_HD int32_t check_beam(const qs_beam& B) {
  const double v[10] = {B.gamma_mean, B.rel_spread, B.gamma_lo, B.gamma_hi, B.sigma_x_um,
                        B.sigma_y_um, B.sigma_z_um, B.div_rad, B.dx_um, B.dy_um};
  for (int k = 0; k < 10; ++k)
    if (!qs_fin(v[k])) return QS_ERR_INVALID_ARG;
  if (B.sigma_x_um < 0 || B.sigma_y_um < 0 || B.sigma_z_um < 0 || B.div_rad < 0)
    return QS_ERR_INVALID_ARG;
  if (B.flat_energy) {
    if (!(B.gamma_hi >= B.gamma_lo) || B.gamma_lo < 0) return QS_ERR_INVALID_ARG;
  } else if (!(B.gamma_mean > 0) || B.rel_spread < 0) {
    return QS_ERR_INVALID_ARG;
  }
  return QS_OK;
}

QS_HD int32_t check_bins(const qs_bins& b) {
  if (b.n_bins < 0 || b.n_tx < 0 || b.n_ty < 0 || b.n_aeff < 0) return QS_ERR_INVALID_ARG;
  if (b.n_bins > (1 << 22) || b.n_aeff > (1 << 22)) return QS_ERR_INVALID_ARG;
  if ((int64_t)b.n_tx * b.n_ty > (int64_t)1 << 24) return QS_ERR_INVALID_ARG;
  if (b.n_bins > 0) {
    if (!qs_fin(b.lo) || !qs_fin(b.hi) || !(b.hi > b.lo)) return QS_ERR_INVALID_ARG;
    if (b.log_spaced && !(b.lo > 0)) return QS_ERR_INVALID_ARG;
  }
  if ((b.n_tx > 0) != (b.n_ty > 0)) return QS_ERR_INVALID_ARG;
  if (b.n_tx > 0 && !qs_pos(b.theta_max)) return QS_ERR_INVALID_ARG;
  if (b.n_aeff > 0 && !qs_pos(b.aeff_max)) return QS_ERR_INVALID_ARG;
  if (!qs_nonneg(b.smooth_sigma_bins)) return QS_ERR_INVALID_ARG;
  if (b.smooth_sigma_bins > 0 && (b.n_bins <= 0 || b.log_spaced || b.smooth_sigma_bins > 64))
    return QS_ERR_INVALID_ARG;
  return QS_OK;
}

// Launch constants of one laser/beam/bins combination (no sample or
// workspace pointers).
//   k = 2 pi/lambda, omega0 = c k, z_R = pi W0^2/lambda (Eq. 2)
//   R_c = r_e k, a_S = 1/(k lambdabar_c), Phi = omega0 tau (intensity FWHM)
//   Gaussian field envelope on [-2.5 Phi, 2.5 Phi]; sin^2 field envelope on
//   [0, Phi_T], Phi_T = Phi/(1 - (2/pi) asin 2^-1/4)
// Only IEEE +, -, *, / (no contractible a*b+c) and literal constants are used,
// so the host and the device produce the same doubles; the one data-dependent
// logarithm (log-spaced bins) may differ in the last bit.
//   c_RR = (2/3) R_c int G^2 (Eq. 3), K = (2/3) R_c A^2 (Eq. 6),
//   chi = sqrt2 mu A / a_S (rms field of linear polarisation)
QS_HD void derive_params(Params& p, const qs_laser& L, const qs_beam& B, const qs_bins* b,
                         int wbits) {
  using namespace cst;
  memset(&p, 0, sizeof(p));
  const double k = 2.0 * kPi / L.lambda_um;
  const double omega0 = kC * k;
  const double zR = kPi * L.w0_um * L.w0_um / L.lambda_um;
  const double Rc = kRe * k;
  const double aS = 1.0 / (k * kLbarC);
  const double Phi = omega0 * L.tau_fs;
  const double PhiT = Phi / kSin2Fwhm;
  double lo, hi, intG2;
  if (L.envelope == QS_ENV_GAUSS) {
    lo = -kGaussWindow * Phi;
    hi = kGaussWindow * Phi;
    intG2 = Phi * kGaussIntG2;
  } else {
    lo = 0.0;
    hi = PhiT;
    intG2 = 3.0 * PhiT / 8.0;
  }
  p.a0 = L.a0;
  p.inv_w0sq = 1.0 / (L.w0_um * L.w0_um);
  p.inv_zR = 1.0 / zR;
  p.ldx = L.dx_um;
  p.ldy = L.dy_um;
  p.c_delay = kC * L.delay_fs;
  p.cRR = (2.0 / 3.0) * Rc * intG2;
  p.cK = (2.0 / 3.0) * Rc;
  p.cchi = kSqrt2 / aS;
  p.n_phase = (L.model == QS_MODEL_QFP || (L.variant & QS_VARIANT_CELL_FOCUS)) ? L.n_phase : 1;
  p.h = (hi - lo) / (double)p.n_phase;
  p.win_lo = lo;
  p.Phi = Phi;
  p.PhiT = PhiT;
  p.kappa_s = L.div_prefactor * kSqrt2OverPi;
  p.envelope = L.envelope;
  p.model = L.model;
  p.focus = (L.variant & QS_VARIANT_CELL_FOCUS) ? 1 : 0;
  p.cycle = (L.variant & QS_VARIANT_CYCLE_CHI) ? 1 : 0;
  p.phic = L.envelope == QS_ENV_GAUSS ? 0.0 : 0.5 * PhiT;   // pulse peak on the window axis
  p.inv2k = 1.0 / (2.0 * k);

  p.gmean = B.gamma_mean;
  p.spread = B.rel_spread;
  p.glo = B.gamma_lo;
  p.gspan = B.gamma_hi - B.gamma_lo;
  p.sx = B.sigma_x_um;
  p.sy = B.sigma_y_um;
  p.sz = B.sigma_z_um;
  p.div = B.div_rad;
  p.bdx = B.dx_um;
  p.bdy = B.dy_um;
  p.flat = B.flat_energy ? 1 : 0;

  if (b) {
    p.n_bins = b->n_bins;
    p.log_spaced = b->log_spaced;
    p.lo = b->lo;
    if (b->n_bins > 0) {
      p.inv_w = (double)b->n_bins / (b->hi - b->lo);
      if (b->log_spaced) {
        p.log_scale = (double)b->n_bins / log(b->hi / b->lo);
        const double l2 = log2(b->hi / b->lo);
        p.log2_scale = (float)((double)b->n_bins / l2);
        p.log2_offset = (float)(log2(b->lo) * ((double)b->n_bins / l2));
      }
    }
    p.n_tx = b->n_tx;
    p.n_ty = b->n_ty;
    p.tmax = b->theta_max;
    if (b->n_tx > 0) {
      p.tsx = (double)b->n_tx / (2.0 * b->theta_max);
      p.tsy = (double)b->n_ty / (2.0 * b->theta_max);
    }
    p.n_aeff = b->n_aeff;
    if (b->n_aeff > 0) p.a_scale = (double)b->n_aeff / b->aeff_max;
    if (b->smooth_sigma_bins > 0) {
      const double sg = b->smooth_sigma_bins;
      p.smooth_sigma = sg;
      p.smooth_pref = 1.0 / (sg * kSqrt2Pi);
      p.smooth_c = 1.4426950408889634074 / (2.0 * sg * sg);
    }
  }
  p.wscale = ldexp(1.0, wbits);
  p.gamma_ref = B.flat_energy ? 0.5 * (B.gamma_lo + B.gamma_hi) : B.gamma_mean;

  // FP32 copies (each double rounded once to nearest)
  Params::F& f = p.f;
  f.a0 = (float)p.a0; f.inv_w0sq = (float)p.inv_w0sq; f.inv_zR = (float)p.inv_zR;
  f.ldx = (float)p.ldx; f.ldy = (float)p.ldy; f.c_delay = (float)p.c_delay;
  f.cRR = (float)p.cRR; f.h = (float)p.h; f.cK = (float)p.cK; f.hcK = (float)(p.h * p.cK);
  f.cchi = (float)p.cchi; f.kappa_s = (float)p.kappa_s;
  f.gmean = (float)p.gmean; f.spread = (float)p.spread; f.glo = (float)p.glo;
  f.gspan = (float)p.gspan; f.sx = (float)p.sx; f.sy = (float)p.sy; f.sz = (float)p.sz;
  f.div = (float)p.div; f.bdx = (float)p.bdx; f.bdy = (float)p.bdy;
  f.lo = (float)p.lo; f.inv_w = (float)p.inv_w; f.tmax = (float)p.tmax;
  f.tsx = (float)p.tsx; f.tsy = (float)p.tsy; f.a_scale = (float)p.a_scale;
  f.n_bins = (float)p.n_bins; f.n_tx = (float)p.n_tx; f.n_ty = (float)p.n_ty;
  f.n_aeff = (float)p.n_aeff; f.smooth_c = (float)p.smooth_c;
  f.wscale = (float)p.wscale;
  f.smooth_pw = (float)(p.smooth_pref * p.wscale);
  f.smooth_lo = (float)(0.5 + 6.0 * p.smooth_sigma);
  f.smooth_hi = (float)(6.0 * p.smooth_sigma - 0.5);
  f.smooth_sigma = (float)p.smooth_sigma;
  f.smooth_pref = (float)p.smooth_pref;
}

}  // namespace qs

// qs_grad.cuh -- device side of the adjoint of the beam phase-space
// integration, shared by the single-shot (qs_scatter_grad) and batched
// (qs_scatter_grad_batch) kernels: the discretised phase integration with
// two tangents (d/d a_eff, d/d gamma0), or seven for the per-cell focus
// (every cell's amplitude depends on the geometry in its own way), a
// sample's decode and focus with the derivatives of ln a_eff, the sample's
// share of the upstream gradient and the chain rule to the 8 parameters, and
// the fixed-order reductions.
//
// Paper: Amaro & Vranic, "QScatter", arXiv 2308.09348 -- Eqs. 2, 3, 6, 8 and
// the reconstruction use of Sec. 6.
#pragma once

#include "qscatter.h"
#include "qs_device.cuh"

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
//   h2 = g R, R = N/D (the rational second-moment fit),
//   h2' = g' R + g (N' - R D')/D.
// Cycle-resolved factors and their chi-derivatives (QS_VARIANT_CYCLE_CHI):
// g -> G, g' -> G', 2g + chi g' -> S = 2G + chi G', its derivative
// S' = 3G' + chi G'', h -> H, h' -> H'.  FP64: the Gauss-Legendre cycle
// means; FP32: the node-pair Hermite tables (shared memory), differentiated
// through the interpolant in u = log2(1 + chi/chi_s):
//   dG/dchi = G_u u',  d2G/dchi2 = G_uu u'^2 + G_u u'',
//   u' = 1/(ln2 (chi + chi_s)),  u'' = -ln2 u'^2.
__device__ __forceinline__ void cycle_derivs(const Params& p, const float4* __restrict__ A,
                                             double chi, double& g, double& gp, double& s,
                                             double& s_chi, double& h2, double& h2p) {
  (void)A;
  double dG, dS, dH;
  cycle_factors_d(p.cyc_gl, chi, g, s, h2, &dG, &dS, &dH);
  gp = dG;
  s_chi = dS;
  h2p = dH;
}
__device__ __forceinline__ void cycle_derivs(const Params& p, const float4* __restrict__ A,
                                             float chi, float& g, float& gp, float& s,
                                             float& s_chi, float& h2, float& h2p) {
  (void)p;
  const float LN2 = 0.69314718055994530942f;
  const float u = M<float>::lg2(__fmaf_rn(chi, (float)(1.0 / kCycChiS), 1.f));
  const float x = fminf(fmaxf(u * (float)(1.0 / kCycDu), 0.f), (float)(kCycN - 1) - 1e-3f);
  const float xm = (x - 0.5f) + 12582912.f;
  const int idx = __float_as_int(xm) - 0x4B400000;
  const float t = x - (xm - 12582912.f), t2 = t * t;
  const float4 gg = A[idx], hh = A[kCycN + idx];
  const float dGv = gg.z - gg.x, dHv = hh.z - hh.x;
  // value, t-derivative and second t-derivative of the cubic Hermite basis
  const float h01 = t2 * (3.f - 2.f * t), h10 = t - 2.f * t2 + t2 * t, h11 = t2 * t - t2;
  const float d01 = 6.f * (t - t2), d10 = 1.f - 4.f * t + 3.f * t2, d11 = 3.f * t2 - 2.f * t;
  const float e01 = 6.f - 12.f * t, e10 = 6.f * t - 4.f, e11 = 6.f * t - 2.f;
  g = gg.x + h01 * dGv + h10 * gg.y + h11 * gg.w;
  h2 = hh.x + h01 * dHv + h10 * hh.y + h11 * hh.w;
  const float Gt = d01 * dGv + d10 * gg.y + d11 * gg.w;
  const float Gtt = e01 * dGv + e10 * gg.y + e11 * gg.w;
  const float Ht = d01 * dHv + d10 * hh.y + d11 * hh.w;
  const float up = M<float>::rcp(LN2 * (chi + (float)kCycChiS));      // du/dchi
  const float idu = (float)(1.0 / kCycDu);
  gp = Gt * idu * up;
  const float gpp = Gtt * idu * idu * up * up - Gt * idu * LN2 * up * up;
  h2p = Ht * idu * up;
  s = 2.f * g + chi * gp;
  s_chi = 3.f * gp + chi * gpp;
}

// g, g', 2g + chi g', its chi-derivative, h and h' at chi: the closed forms
// of the fits, or (VAR & kVarCycle) their cycle means.
template <typename T, int VAR>
__device__ __forceinline__ void cell_factors(const Params& p, const float4* __restrict__ cA, T chi,
                                             T& g, T& gp, T& s, T& s_chi, T& h2, T& h2p) {
  if constexpr ((VAR & kVarCycle) != 0) {
    cycle_derivs(p, cA, chi, g, gp, s, s_chi, h2, h2p);
  } else {
    const T LN2 = (T)0.69314718055994530942;
    const T x1 = (T)1 + (T)1.7 * chi;
    const T l1 = M<T>::lg2(x1);
    const T L1 = LN2 * l1;
    const T r1 = M<T>::ex2(-l1);
    const T opc = (T)1 + chi;
    const T B = (T)1 + (T)4.8 * opc * L1 + (T)2.44 * chi * chi;
    const T t = M<T>::ex2((T)(-1.0 / 3.0) * M<T>::lg2(B));
    g = t * t;
    const T iB = t * t * t;
    const T Bp = (T)4.8 * L1 + (T)8.16 * opc * r1 + (T)4.88 * chi;
    const T Bpp = (T)8.16 * r1 - (T)5.712 * r1 * r1 + (T)4.88;
    gp = (T)(-2.0 / 3.0) * g * iB * Bp;
    const T gpp = (T)(10.0 / 9.0) * g * iB * iB * Bp * Bp - (T)(2.0 / 3.0) * g * iB * Bpp;
    s = (T)2 * g + chi * gp;
    s_chi = (T)3 * gp + chi * gpp;
    const T Nh = (T)1 + chi * ((T)kHA1 + (T)kHA2 * chi);
    const T Dh = (T)1 + chi * ((T)kHB1 + chi * ((T)kHB2 + (T)kHB3 * chi));
    const T iD = M<T>::rcp(Dh);
    const T R = Nh * iD;
    const T Rp = ((T)kHA1 + (T)(2.0 * kHA2) * chi -
                  R * ((T)kHB1 + chi * ((T)(2.0 * kHB2) + (T)(3.0 * kHB3) * chi))) * iD;
    h2 = g * R;
    h2p = gp * R + g * Rp;
  }
}

template <typename T, int VAR = 0>
__device__ __forceinline__ void qfp_tangent(const Params& p,
                                            const typename Tab<T>::type* __restrict__ tab, T a,
                                            T g0, QfpTan<T>& o,
                                            const float4* __restrict__ cA = nullptr) {
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
    // Gaunt and second-moment factors and their derivatives
    T g, gp, s, s_chi, h2, h2p;
    cell_factors<T, VAR>(p, cA, chi, g, gp, s, s_chi, h2, h2p);
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

// Packed FP32 version of qfp_tangent for two samples at once (f32x2 FMA-pipe
// instructions, per-sample MUFU), the same recursion written with explicit
// fused multiply-adds and the forward step's forms: 1/mu = 1/gamma0 + du at
// the midpoint, so mu_a = -mu^2 du_a and mu_g = mu^2 (1/gamma0^2 - du_g);
// B' = 4.8 ln(1+1.7 chi) + 4.8 + 3.36/(1+1.7 chi) + 4.88 chi; the factor -2
// of the variance rate folded into s and s' and the D2 constant into h.
__device__ __forceinline__ void qfp_tangent_x2(const Params& p, const float4* __restrict__ tab,
                                               float2 a, float2 g0, QfpTan<float>& o0,
                                               QfpTan<float>& o1) {
  const float2 ONE = f2(1.f), HALF = f2(0.5f), THREE = f2(3.f);
  const float2 C48 = f2((float)(4.8 * 0.69314718055994530942));      // 4.8 ln2
  const float C55 = (float)kC55;
  const float hcK = p.f.h * p.f.cK;
  const float2 c1 = mul2(mul2(f2(hcK), a), a), c1a = mul2(f2(2.f * hcK), a);
  const float2 CCHI = f2(p.f.cchi), ca = mul2(CCHI, a);
  const float2 ig0 = make_float2(__frcp_rn(g0.x), __frcp_rn(g0.y));
  const float2 ig02 = mul2(ig0, ig0);
  float2 du = f2(0.f), V = f2(0.f), gph = HALF, du_a = f2(0.f), du_g = f2(0.f), V_a = f2(0.f),
         V_g = f2(0.f), gph_a = f2(0.f), gph_g = f2(0.f);
  const int N = p.n_phase;
  for (int j = 0; j < N; ++j) {
    const float4 e = tab[j];
    const float2 G = make_float2(e.x, e.y), G2 = make_float2(e.z, e.w);
    const float2 hK = mul2(c1, G2), hK_a = mul2(c1a, G2);
    const float2 dum = fma2(hK, gph, du);
    const float2 dum_a = fma2(hK, gph_a, fma2(hK_a, gph, du_a));
    const float2 dum_g = fma2(hK, gph_g, du_g);
    const float2 mu = rcpx2(__fadd2_rn(dum, ig0));
    const float2 m2 = mul2(mu, mu);
    const float2 mu_a = mul2(make_float2(-m2.x, -m2.y), dum_a);
    const float2 mu_g = mul2(m2, fma2(dum_g, f2(-1.f), ig02));
    const float2 cg = mul2(ca, G);
    const float2 chi = mul2(cg, mu);
    const float2 chi_a = fma2(mul2(CCHI, G), mu, mul2(cg, mu_a));
    const float2 chi_g = mul2(cg, mu_g);
    // Gaunt factor and derivatives
    const float2 l1 = lg2x2(fma2(f2(1.7f), chi, ONE));
    const float2 r1 = ex2x2(make_float2(-l1.x, -l1.y));              // 1/(1+1.7 chi)
    const float2 B = fma2(fma2(C48, chi, C48), l1, fma2(mul2(f2(2.44f), chi), chi, ONE));
    const float2 t = ex2x2(mul2(f2(-1.f / 3.f), lg2x2(B)));
    const float2 g = mul2(t, t), iB = mul2(g, t), giB = mul2(g, iB);
    const float2 Bp = fma2(C48, l1, fma2(f2(4.88f), chi, fma2(f2(3.36f), r1, f2(4.8f))));
    const float2 Bpp = fma2(fma2(f2(-5.712f), r1, f2(8.16f)), r1, f2(4.88f));
    const float2 gp = mul2(mul2(f2(-2.f / 3.f), giB), Bp);
    // -2 g'' and -2 (2g + chi g'), -2 (3g' + chi g'')
    const float2 gpp2 =
        mul2(giB, fma2(mul2(mul2(f2(-20.f / 9.f), iB), Bp), Bp, mul2(f2(4.f / 3.f), Bpp)));
    const float2 s2 = fma2(chi, mul2(f2(-2.f), gp), mul2(f2(-4.f), g));
    const float2 s2_chi = fma2(chi, gpp2, mul2(f2(-6.f), gp));
    // second-moment factor (times the D2 constant) and derivative: h = g R, R = N/D
    const float2 Nh = fma2(fma2(f2((float)(kC55 * kHA2)), chi, f2((float)(kC55 * kHA1))), chi,
                           f2(C55));
    const float2 Dh = fma2(fma2(fma2(f2((float)kHB3), chi, f2((float)kHB2)), chi,
                                f2((float)kHB1)), chi, ONE);
    const float2 iD = rcpx2(Dh);
    const float2 R = mul2(Nh, iD);
    const float2 Np = fma2(f2((float)(2.0 * kC55 * kHA2)), chi, f2((float)(kC55 * kHA1)));
    const float2 Dp = fma2(fma2(f2((float)(3.0 * kHB3)), chi, f2((float)(2.0 * kHB2))), chi,
                           f2((float)kHB1));
    const float2 Rp = mul2(fma2(make_float2(-R.x, -R.y), Dp, Np), iD);
    const float2 h2 = mul2(g, R);
    const float2 h2p = fma2(gp, R, mul2(g, Rp));
    // mean
    const float2 hKgp = mul2(hK, gp);
    const float2 du_n = fma2(hK, g, du);
    const float2 du_a_n = fma2(hKgp, chi_a, fma2(hK_a, g, du_a));
    const float2 du_g_n = fma2(hKgp, chi_g, du_g);
    // variance
    const float2 hKmu = mul2(hK, mu), hKmus = mul2(hKmu, s2_chi);
    const float2 hlam = mul2(hKmu, s2);
    const float2 hlam_a = fma2(hKmus, chi_a, mul2(s2, fma2(hK_a, mu, mul2(hK, mu_a))));
    const float2 hlam_g = fma2(hKmus, chi_g, mul2(mul2(hK, mu_g), s2));
    const float2 chih2 = mul2(chi, h2);
    const float2 hD2 = mul2(mul2(m2, hKmu), chih2);
    const float2 hh = fma2(chi, h2p, h2);
    const float2 hK3 = mul2(THREE, hK), hKmuh = mul2(hKmu, hh);
    const float2 hD2_a = mul2(m2, fma2(fma2(hK_a, mu, mul2(hK3, mu_a)), chih2, mul2(hKmuh, chi_a)));
    const float2 hD2_g = mul2(m2, fma2(mul2(hK3, mu_g), chih2, mul2(hKmuh, chi_g)));
    const float2 hr = fma2(hlam, V, hD2);
    const float2 hr_a = fma2(hlam, V_a, fma2(hlam_a, V, hD2_a));
    const float2 hr_g = fma2(hlam, V_g, fma2(hlam_g, V, hD2_g));
    const float2 fac = fma2(HALF, hlam, ONE), hhr = mul2(HALF, hr);
    V = fma2(hr, fac, V);
    V_a = fma2(hhr, hlam_a, fma2(hr_a, fac, V_a));
    V_g = fma2(hhr, hlam_g, fma2(hr_g, fac, V_g));
    du = du_n; du_a = du_a_n; du_g = du_g_n;
    gph = mul2(HALF, g);
    const float2 hgp = mul2(HALF, gp);
    gph_a = mul2(hgp, chi_a);
    gph_g = mul2(hgp, chi_g);
  }
  o0.du = du.x; o0.V = V.x; o0.du_a = du_a.x; o0.du_g = du_g.x; o0.V_a = V_a.x; o0.V_g = V_g.x;
  o1.du = du.y; o1.V = V.y; o1.du_a = du_a.y; o1.du_g = du_g.y; o1.V_a = V_a.y; o1.V_g = V_g.y;
}

// Upstream gradient, reduced to the per-sample coefficients it needs (in
// the path's arithmetic type).
template <typename T>
struct Seeds {
  T invW, mean, spread, dxr, dyr;             // forward moments
  T gM, gSp, gDx, gDy, gA, gG0;               // effective dL/d(mean, spread, div_x, div_y, a, g0)
};

// A sample's decode and focus with the derivatives of ln a (rows a1-a3).
template <typename T>
struct GFront {
  T w, xi3, xi4, xi5, gamma0, a, a_over_a0;
  T dla_w0, dla_dx, dla_dy, dla_thx, dla_thy, dla_del, thx, thy;
  T zq, xs, ys, ct, w0;        // crossing geometry (per-cell focus)
  bool ok, clamped;
};

template <typename T>
__device__ __forceinline__ void grad_front(const Params& p, int64_t i, T w0, GFront<T>& f) {
  const T xi0 = load_t<T>(p.xi[0], i, p.dtype), xi1 = load_t<T>(p.xi[1], i, p.dtype);
  const T xi2 = load_t<T>(p.xi[2], i, p.dtype);
  f.xi3 = load_t<T>(p.xi[3], i, p.dtype);
  f.xi4 = load_t<T>(p.xi[4], i, p.dtype);
  f.xi5 = load_t<T>(p.xi[5], i, p.dtype);
  f.w = p.weighted ? load_t<T>(p.w, i, p.dtype) : (T)1;
  f.ok = f.w >= (T)0 && isfinite(f.w);
  const T x = QS_PV(T, bdx) + QS_PV(T, sx) * xi0;
  const T y = QS_PV(T, bdy) + QS_PV(T, sy) * xi1;
  const T z = QS_PV(T, sz) * xi2;
  T gamma0 = p.flat ? QS_PV(T, glo) + QS_PV(T, gspan) * f.xi3
                    : QS_PV(T, gmean) * ((T)1 + QS_PV(T, spread) * f.xi3);
  f.clamped = gamma0 < (T)1;
  if (f.clamped) gamma0 = (T)1;
  f.gamma0 = gamma0;
  const T thx = QS_PV(T, div) * f.xi4, thy = QS_PV(T, div) * f.xi5;
  f.thx = thx;
  f.thy = thy;
  const T cdel = QS_PV(T, c_delay);
  const T ct = (T)0.5 * (z + cdel);
  const T zs = (T)0.5 * (z - cdel);
  const T xs = x + thx * ct - QS_PV(T, ldx);
  const T ys = y + thy * ct - QS_PV(T, ldy);
  const T rho2 = xs * xs + ys * ys;
  const T izR = QS_PV(T, inv_zR), iw2 = QS_PV(T, inv_w0sq);
  const T zq = zs * izR;
  const T q = (T)1 + zq * zq;
  const T rq = M<T>::rcp(q);
  const T E = rho2 * iw2 * rq;                         // a = a0 q^-1/2 exp(-E)
  if (sizeof(T) == 4)
    f.a_over_a0 = M<T>::rsqrt(q) * M<T>::ex2(-(T)1.4426950408889634074 * E);
  else
    f.a_over_a0 = M<T>::rsqrt(q) * (T)exp(-(double)E);
  f.a = QS_PV(T, a0) * f.a_over_a0;
  // d ln a / d(parameter)
  const T k2 = (T)2 * iw2 * rq;                        // 2 / (W0^2 q)
  f.dla_dx = k2 * xs;
  f.dla_dy = k2 * ys;
  f.dla_thx = -k2 * xs * ct;
  f.dla_thy = -k2 * ys * ct;
  const T cc = (T)0.299792458;
  const T dq_del = -cc * zq * izR;                     // dq/d delay
  const T drho_del = cc * (xs * thx + ys * thy);       // d rho^2 / d delay
  f.dla_del = (E - (T)0.5) * dq_del * rq - drho_del * iw2 * rq;
  const T dq_w0 = (T)-4 * zq * zq / w0;                // dq/dW0 (z_R ~ W0^2)
  f.dla_w0 = (T)-0.5 * dq_w0 * rq + E * ((T)2 / w0 + dq_w0 * rq);
  f.zq = zq;
  f.xs = xs;
  f.ys = ys;
  f.ct = ct;
  f.w0 = w0;
}

// Per-cell focus (QS_VARIANT_CELL_FOCUS): the local amplitude a_j of a cell
// at shift s along the path (Eq. 2 at z* - s, xs + theta_x s, ys + theta_y s)
// and d ln a_j / d(ln a0, W0, dx, dy, delay, div), from
//   ln a_j = ln a0 - (1/2) ln q_j - E_j,  q_j = 1 + zq_j^2,  E_j = rho_j^2/(W0^2 q_j):
//   W0    (E - 1/2) q'/q + 2E/W0 with q' = -4 zq_j^2/W0 (z_R ~ W0^2)
//   dx    2 x_j/(W0^2 q_j),  dy the same with y_j
//   delay (E - 1/2) q'/q - rho'/(W0^2 q) with q' = -c zq_j/z_R,
//         rho' = c (x_j theta_x + y_j theta_y) (the crossing moves by c/2)
//   div   -2 (x_j xi4 + y_j xi5)(ct + s)/(W0^2 q_j)
template <typename T>
__device__ __forceinline__ T cell_amp(const Params& p, const GFront<T>& f, T s, T (&e)[6]) {
  const T izR = QS_PV(T, inv_zR), iw2 = QS_PV(T, inv_w0sq);
  const T zq = f.zq - s * izR;
  const T q = (T)1 + zq * zq, rq = M<T>::rcp(q);
  const T xj = f.xs + f.thx * s, yj = f.ys + f.thy * s;
  const T E = (xj * xj + yj * yj) * iw2 * rq;
  T ex;
  if constexpr (sizeof(T) == 4) ex = M<T>::ex2(-(T)1.4426950408889634074 * E);
  else ex = exp(-E);
  const T aj = QS_PV(T, a0) * M<T>::rsqrt(q) * ex;
  const T k2 = (T)2 * iw2 * rq;
  const T cc = (T)0.299792458;
  e[0] = (T)1;
  e[1] = (E - (T)0.5) * ((T)-4 * zq * zq / f.w0) * rq + (T)2 * E / f.w0;
  e[2] = k2 * xj;
  e[3] = k2 * yj;
  e[4] = (E - (T)0.5) * (-cc * zq * izR) * rq - cc * (xj * f.thx + yj * f.thy) * iw2 * rq;
  e[5] = -k2 * (xj * f.xi4 + yj * f.xi5) * (f.ct + s);
  return aj;
}

// Tangents of the per-cell-focus model with respect to ln a0, W0, dx, dy,
// delay, div (each through every cell's a_j) and gamma0: the recursion of
// qfp_tangent with a per-cell relative perturbation e_k of the field
// (dhK = 2 hK e_k, dchi = chi e_k + cg dmu), or, for the classical model,
// Eq. 3's exponent summed cell by cell.
constexpr int kNT = 7;
template <typename T> struct FocTan {
  T du, V, du_t[kNT], V_t[kNT];
};

template <typename T, bool QFP, int VAR>
__device__ __forceinline__ void focus_tangent(const Params& p,
                                              const typename Tab<T>::type* __restrict__ tab,
                                              const GFront<T>& f, FocTan<T>& o,
                                              const float4* __restrict__ cA) {
  const T C55 = (T)(55.0 / (16.0 * 1.7320508075688772935));
  const T hcK = (T)p.h * (T)p.cK, cchi = (T)p.cchi, g0 = f.gamma0;
  T du = 0, V = 0, gph = (T)0.5;
  T du_t[kNT], V_t[kNT], gph_t[kNT];
#pragma unroll
  for (int k = 0; k < kNT; ++k) du_t[k] = V_t[k] = gph_t[k] = (T)0;
  const int N = p.n_phase;
  for (int j = 0; j < N; ++j) {
    T G, sj;
    if constexpr (sizeof(T) == 4) {
      const float4 e4 = reinterpret_cast<const float4*>(tab)[j];
      G = e4.x;
      sj = e4.z;
    } else {
      G = reinterpret_cast<const double*>(tab)[j];
      sj = cell_shift(p, j);
    }
    T e[6];
    const T A = cell_amp<T>(p, f, sj, e) * G;
    const T hK = hcK * A * A;
    if constexpr (!QFP) {
      du += hK;
#pragma unroll
      for (int k = 0; k < 6; ++k) du_t[k] += (T)2 * hK * e[k];
      continue;
    } else {
      const T dum = du + hK * gph;
      const T r = M<T>::rcp((T)1 + g0 * dum);
      const T mu = g0 * r;
      const T cg = cchi * A;
      const T chi = cg * mu;
      T g, gp, s, s_chi, h2, h2p;
      cell_factors<T, VAR>(p, cA, chi, g, gp, s, s_chi, h2, h2p);
      const T hKmu = hK * mu;
      const T hlam = (T)-2 * hKmu * s;
      const T m2 = mu * mu;
      const T hD2 = C55 * hKmu * m2 * chi * h2;
      const T hh = h2 + chi * h2p;
      const T hr = hlam * V + hD2;
      const T fac = (T)1 + (T)0.5 * hlam;
#pragma unroll
      for (int k = 0; k < kNT; ++k) {
        const T dhK = k < 6 ? (T)2 * hK * e[k < 6 ? k : 0] : (T)0;
        const T dum_k = du_t[k] + dhK * gph + hK * gph_t[k];
        const T mu_k = k < 6 ? -mu * r * g0 * dum_k : r - mu * r * (dum + g0 * dum_k);
        const T chi_k = (k < 6 ? chi * e[k < 6 ? k : 0] : (T)0) + cg * mu_k;
        du_t[k] = du_t[k] + dhK * g + hK * gp * chi_k;
        const T hlam_k = (T)-2 * (dhK * mu * s + hK * mu_k * s + hKmu * s_chi * chi_k);
        const T hD2_k = C55 * m2 * ((dhK * mu + (T)3 * hK * mu_k) * chi * h2 + hKmu * chi_k * hh);
        const T hr_k = hlam_k * V + hlam * V_t[k] + hD2_k;
        V_t[k] = V_t[k] + hr_k * fac + (T)0.5 * hr * hlam_k;
        gph_t[k] = (T)0.5 * gp * chi_k;
      }
      du = du + hK * g;
      V = V + hr * fac;
      gph = (T)0.5 * g;
    }
  }
  o.du = du;
  o.V = V;
#pragma unroll
  for (int k = 0; k < kNT; ++k) {
    o.du_t[k] = du_t[k];
    o.V_t[k] = V_t[k];
  }
}

// Per-thread gradient partials: FP64 sums (FP64 path), compensated FP32
// sums (FP32 path).
template <typename T> struct GAcc;
template <> struct GAcc<double> {
  double s[kNumGrad];
  __device__ __forceinline__ void init() {
    for (int k = 0; k < kNumGrad; ++k) s[k] = 0.0;
  }
  __device__ __forceinline__ void add(int k, double x) { s[k] += x; }
  __device__ __forceinline__ double get(int k) const { return s[k]; }
};
template <> struct GAcc<float> {
  float s[kNumGrad], c[kNumGrad];
  __device__ __forceinline__ void init() {
    for (int k = 0; k < kNumGrad; ++k) s[k] = c[k] = 0.f;
  }
  __device__ __forceinline__ void add(int k, float x) { kahan(s[k], c[k], x); }
  __device__ __forceinline__ double get(int k) const { return (double)s[k] - (double)c[k]; }
};

// dL/d(the sample's outputs) from the upstream gradient (adjoint of rows
// a8-a9 and of the smoothed spectrum), and through Eq. 8 (theta_e = kappa_s
// a sqrt(V) / mu^2, a the crossing a_eff): the sample's share of dL/d mu,
// dL/d V, dL/d a_eff (directly), dL/d gamma0 (directly) and dL/d theta_x0,
// theta_y0.  False if the sample's result is not finite (it then adds
// nothing, as the forward excluded it).
template <typename T>
struct GOut {
  T g_mu, g_V, g_a, g_g0, g_thx, g_thy;
};

template <typename T, bool QFP, typename S>
__device__ __forceinline__ bool sample_upstream(const Params& p, const Seeds<T>& sd,
                                                const S* __restrict__ dLdS, int64_t i,
                                                const GFront<T>& f, T mu, T V, GOut<T>& go) {
  const T a = f.a;
  if (!isfinite(mu) || !isfinite(V)) return false;
  // outputs of the sample (row a6)
  T theta_e = 0, gout = mu, sv = 0;
  const T xi7 = QFP ? load_t<T>(p.xi[7], i, p.dtype) : (T)0;
  if (QFP && V > (T)0) {
    sv = sqrt(V);
    theta_e = QS_PV(T, kappa_s) * a * sv / (mu * mu);
    gout = mu + sv * xi7;
  }
  // sample's share of dL/d(outputs)
  const T wn = f.w * sd.invW;
  T g_out = 0;                                          // dL/d gamma_out
  if (dLdS != nullptr) {
    const T tt = (gout - QS_PV(T, lo)) * QS_PV(T, inv_w);
    if (tt > (T)-1e9 && tt < (T)1e9) {
      int k0, k1;
      T c;
      if constexpr (sizeof(T) == 4) {
        smooth_range_f32(p, tt, &k0, &k1);
        c = p.f.smooth_c;
      } else {
        smooth_range(p, tt, &k0, &k1);
        c = p.smooth_c;
      }
      const T tf = tt - (T)k0;
      for (int k = k0; k <= k1; ++k) {
        const T d = (T)(k - k0) + (T)0.5 - tf;
        T e;
        if constexpr (sizeof(T) == 4) e = M<float>::ex2(-(d * d) * c);
        else e = exp2(-d * d * c);
        g_out += (T)dLdS[k] * e * d;
      }
      const T sg = QS_PV(T, smooth_sigma);
      g_out *= f.w * QS_PV(T, smooth_pref) * QS_PV(T, inv_w) / (sg * sg);
    }
  }
  T g_mu = sd.gM * wn + g_out;
  if (sd.spread > (T)0) g_mu += sd.gSp * wn * (mu - sd.mean) / sd.spread;
  T g_V = (sd.spread > (T)0 ? sd.gSp * wn * (T)0.5 / sd.spread : (T)0);
  if (QFP && V > (T)0) g_V += g_out * xi7 * (T)0.5 / sv;
  const T g_te = sd.gDx * wn * theta_e * sd.dxr;
  go.g_thx = sd.gDx * wn * f.thx * sd.dxr;
  go.g_thy = sd.gDy * wn * f.thy * sd.dyr;
  T g_a = sd.gA * wn;
  go.g_g0 = sd.gG0 * wn;
  // theta_e = kappa_s a sqrt(V) / mu^2
  if (QFP && V > (T)0) {
    const T ks = QS_PV(T, kappa_s);
    g_a += g_te * ks * sv / (mu * mu);
    g_V += g_te * ks * a * (T)0.5 / (sv * mu * mu);
    g_mu += g_te * ((T)-2 * theta_e / mu);
  }
  go.g_mu = g_mu;
  go.g_V = g_V;
  go.g_a = g_a;
  return true;
}

// The model with its tangents, the sample's outputs, its share of dL/d(outputs)
// and the chain rule to the parameters (rows a4-a6), for the model whose
// phase integration sees a_eff in every cell (variant 0, cycle-resolved chi):
// (mu, V) = F(a_eff, gamma0), and a_eff carries the parameters' dependence.
template <typename T, bool QFP, typename S>
__device__ __forceinline__ void grad_back(const Params& p, const Seeds<T>& sd,
                                          const S* __restrict__ dLdS, int64_t i,
                                          const GFront<T>& f, const QfpTan<T>& o, GAcc<T>& acc) {
  const T g0 = f.gamma0, a = f.a;
  T mu, V = 0, mu_a, mu_g, V_a = 0, V_g = 0;
  if (!QFP) {
    mu = g0 / ((T)1 + QS_PV(T, cRR) * g0 * a * a);
    mu_a = -mu * mu * (T)2 * QS_PV(T, cRR) * a;
    mu_g = mu * mu / (g0 * g0);
  } else {
    mu = g0 / ((T)1 + g0 * o.du);
    mu_a = -mu * mu * o.du_a;
    mu_g = mu * mu * ((T)1 / (g0 * g0) - o.du_g);
    V = o.V;
    V_a = o.V_a;
    V_g = o.V_g;
  }
  GOut<T> go;
  if (!sample_upstream<T, QFP, S>(p, sd, dLdS, i, f, mu, V, go)) return;
  // (mu, V) = F(a, gamma0)
  const T g_a = go.g_a + go.g_mu * mu_a + go.g_V * V_a;
  const T g_g0 = go.g_g0 + go.g_mu * mu_g + go.g_V * V_g;
  // chain to the parameters
  const T ga = g_a * a;                                 // dL/d ln a
  acc.add(QS_G_A0, QS_PV(T, a0) > (T)0 ? g_a * f.a_over_a0 : (T)0);
  acc.add(QS_G_W0, ga * f.dla_w0);
  acc.add(QS_G_DX, ga * f.dla_dx);
  acc.add(QS_G_DY, ga * f.dla_dy);
  acc.add(QS_G_DELAY, ga * f.dla_del);
  if (!p.flat && !f.clamped) {
    acc.add(QS_G_GAMMA, g_g0 * ((T)1 + QS_PV(T, spread) * f.xi3));
    acc.add(QS_G_SPREAD, g_g0 * QS_PV(T, gmean) * f.xi3);
  }
  acc.add(QS_G_DIV, (go.g_thx + ga * f.dla_thx) * f.xi4 + (go.g_thy + ga * f.dla_thy) * f.xi5);
}

// The same for the per-cell focus: mu and V depend on the parameters through
// every cell's a_j (the seven tangents of focus_tangent), while a_eff at the
// crossing still enters Eq. 8 and the a_eff moment directly.
template <typename T, bool QFP, typename S>
__device__ __forceinline__ void grad_back_focus(const Params& p, const Seeds<T>& sd,
                                                const S* __restrict__ dLdS, int64_t i,
                                                const GFront<T>& f, const FocTan<T>& o,
                                                GAcc<T>& acc) {
  const T g0 = f.gamma0, a = f.a;
  const T mu = g0 / ((T)1 + g0 * o.du);
  const T m2 = mu * mu;
  const T V = QFP ? o.V : (T)0;
  GOut<T> go;
  if (!sample_upstream<T, QFP, S>(p, sd, dLdS, i, f, mu, V, go)) return;
  // d(mu, V)/d theta_k through the cells (k: ln a0, W0, dx, dy, delay, div)
  T gk[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) gk[k] = go.g_mu * (-m2 * o.du_t[k]) + (QFP ? go.g_V * o.V_t[k] : (T)0);
  const T g_g0 = go.g_g0 + go.g_mu * m2 * ((T)1 / (g0 * g0) - o.du_t[6]) +
                 (QFP ? go.g_V * o.V_t[6] : (T)0);
  const T ga = go.g_a * a;                              // direct dL/d ln a_eff
  const T a0v = QS_PV(T, a0);
  acc.add(QS_G_A0, a0v > (T)0 ? go.g_a * f.a_over_a0 + gk[0] / a0v : (T)0);
  acc.add(QS_G_W0, ga * f.dla_w0 + gk[1]);
  acc.add(QS_G_DX, ga * f.dla_dx + gk[2]);
  acc.add(QS_G_DY, ga * f.dla_dy + gk[3]);
  acc.add(QS_G_DELAY, ga * f.dla_del + gk[4]);
  if (!p.flat && !f.clamped) {
    acc.add(QS_G_GAMMA, g_g0 * ((T)1 + QS_PV(T, spread) * f.xi3));
    acc.add(QS_G_SPREAD, g_g0 * QS_PV(T, gmean) * f.xi3);
  }
  acc.add(QS_G_DIV,
          (go.g_thx + ga * f.dla_thx) * f.xi4 + (go.g_thy + ga * f.dla_thy) * f.xi5 + gk[5]);
}

// Upstream coefficients from the forward moments and dL/d(moments):
// rel_spread = spread/mean and div = sqrt(div_x^2 + div_y^2) folded into
// mean, spread, div_x, div_y.
template <typename T>
__device__ __forceinline__ Seeds<T> make_seeds(const qs_moments* __restrict__ mom,
                                               const double* __restrict__ dLdm) {
  Seeds<T> sd;
  const double W = mom->W, mean = mom->mean, spread = mom->spread;
  const double Dx = mom->div_x, Dy = mom->div_y, D = mom->div;
  const double d1 = dLdm[1], d2 = dLdm[2], d3 = dLdm[3], d4 = dLdm[4], d5 = dLdm[5],
               d6 = dLdm[6];
  sd.invW = (T)(W > 0.0 ? 1.0 / W : 0.0);
  sd.mean = (T)mean;
  sd.spread = (T)spread;
  sd.gM = (T)(d1 - (mean != 0.0 ? d3 * spread / (mean * mean) : 0.0));
  sd.gSp = (T)(d2 + (mean != 0.0 ? d3 / mean : 0.0));
  sd.gDx = (T)(d4 + (D > 0.0 ? d6 * Dx / D : 0.0));
  sd.gDy = (T)(d5 + (D > 0.0 ? d6 * Dy / D : 0.0));
  sd.dxr = (T)(Dx > 0.0 ? 1.0 / Dx : 0.0);
  sd.dyr = (T)(Dy > 0.0 ? 1.0 / Dy : 0.0);
  sd.gA = (T)dLdm[7];
  sd.gG0 = (T)dLdm[11];
  return sd;
}

// Samples [begin, end) of one launch's samples, thread `tid` of `nthr`:
// FP32 QFP takes two samples per thread through the packed tangent
// integration (begin even), the other paths one.
template <typename T, bool QFP, typename S, int VAR = 0>
__device__ __forceinline__ void grad_range(const Params& p,
                                           const typename Tab<T>::type* __restrict__ tab,
                                           const Seeds<T>& sd, const S* dS, T w0, GAcc<T>& acc,
                                           int64_t begin, int64_t end, int64_t tid,
                                           int64_t nthr, const float4* __restrict__ cA = nullptr) {
  if constexpr ((VAR & kVarCell) != 0) {
    // per-cell focus: one sample at a time, seven tangents
    for (int64_t i = begin + tid; i < end; i += nthr) {
      GFront<T> f;
      grad_front<T>(p, i, w0, f);
      if (!f.ok) continue;
      FocTan<T> o;
      focus_tangent<T, QFP, VAR>(p, tab, f, o, cA);
      grad_back_focus<T, QFP, S>(p, sd, dS, i, f, o, acc);
    }
  } else if constexpr ((VAR & kVarCycle) != 0) {
    // cycle-resolved chi: one sample at a time, the two tangents
    for (int64_t i = begin + tid; i < end; i += nthr) {
      GFront<T> f;
      grad_front<T>(p, i, w0, f);
      if (!f.ok) continue;
      QfpTan<T> o{};
      qfp_tangent<T, VAR>(p, tab, f.a, f.gamma0, o, cA);
      grad_back<T, QFP, S>(p, sd, dS, i, f, o, acc);
    }
  } else if constexpr (QFP && sizeof(T) == 4) {
    for (int64_t k = begin / 2 + tid; 2 * k < end; k += nthr) {
      const int64_t i0 = 2 * k, i1 = (2 * k + 1 < end) ? 2 * k + 1 : 2 * k;
      GFront<T> f0, f1;
      grad_front<T>(p, i0, w0, f0);
      grad_front<T>(p, i1, w0, f1);
      QfpTan<T> o0, o1;
      qfp_tangent_x2(p, reinterpret_cast<const float4*>(tab), make_float2(f0.a, f1.a),
                     make_float2(f0.gamma0, f1.gamma0), o0, o1);
      if (f0.ok) grad_back<T, QFP, S>(p, sd, dS, i0, f0, o0, acc);
      if (i1 != i0 && f1.ok) grad_back<T, QFP, S>(p, sd, dS, i1, f1, o1, acc);
    }
  } else {
    for (int64_t i = begin + tid; i < end; i += nthr) {
      GFront<T> f;
      grad_front<T>(p, i, w0, f);
      if (!f.ok) continue;
      QfpTan<T> o{};
      if (QFP) qfp_tangent<T>(p, tab, f.a, f.gamma0, o);
      grad_back<T, QFP, S>(p, sd, dS, i, f, o, acc);
    }
  }
}

// Fixed-order block reduction of the per-thread gradient partials into
// out[0..kNumGrad): warp shuffle trees, then warps in order.  red holds
// (blockDim.x / 32) * kNumGrad doubles; the caller synchronises before red
// is reused.
template <typename T>
__device__ __forceinline__ void grad_block_reduce(const GAcc<T>& acc, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNumGrad; ++k) {
    double v = acc.get(k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp * kNumGrad + k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNumGrad) {
    double s = 0.0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[wv * kNumGrad + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

}  // namespace qs

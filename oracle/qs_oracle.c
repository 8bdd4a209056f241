/*
 * qs_oracle.c -- plain, slow FP64 CPU oracle for the QScatter beam
 * phase-space integration (arXiv 2308.09348).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library: every quantity below is computed here,
 * from the paper's equations and the readings listed with each function.
 *
 * Style: one sample at a time, in the paper's order, double precision, libm,
 * Neumaier-compensated sums.  No blocking, fusion or reordering.
 *
 * Units: lengths in micrometres, times in femtoseconds, energies as the
 * Lorentz factor gamma.  Constants are CODATA 2018.
 *
 * Parity status per function (the pins live in tests/test_oracle_pins.py):
 *   qso_constants        pinned (paper's omega0 at 0.8 um; RK4 of the LL
 *                        equation of motion fixes the c_RR chain)
 *   qso_gaunt            pinned (exact quantum-synchrotron power, Bessel
 *                        quadrature; g(0)=1; chi^-4/3 tail)
 *   qso_h2               pinned (exact second moment, Bessel quadrature)
 *   qso_qfp_rates        pinned (absolute first/second emission moments)
 *   qso_qfp_integrate    pinned (classical limit == Eq. 3; variance
 *                        transport closed form; library ODE solve)
 *   qso_eval / qso_scatter  pinned (Table 1 / Table 2 closed forms,
 *                        zero intensity, weight conservation, symmetries;
 *                        the moment finalize against the weighted sample
 *                        moments of the realised energies and angles of
 *                        2^20 samples; Eq. 8 against the paper's printed
 *                        coefficient and a log-linear fit of its scaling)
 *   qso_cycle_factors    pinned (small-chi limits and large-chi tails in
 *                        closed form; adaptive quadrature; the cycle mean
 *                        of the exact quantum-synchrotron power)
 *   qso_bessel_pair      pinned (scipy's modified Bessel functions and
 *                        their adaptive integral)
 *   qso_photon_spectrum  pinned (energy balance with the electrons' loss
 *                        to the Gaunt fit's accuracy; exact moments of
 *                        the spectrum; classical synchrotron limit)
 *   qso_analytic_*       pinned (Monte Carlo histograms of the oracle's own
 *                        beams for every geometry; I0 against scipy)
 *   qso_pw_reconstruct   pinned (converges to the direct 3D spectrum at
 *                        first order in the a-grid spacing, classical model)
 *   per-cell focus       pinned (adaptive quadrature of Eq. 3's exponent
 *                        along the electron's path; reduces to the crossing
 *                        focus for a straight path in a long focus)
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

/* ---- physical constants (CODATA 2018), lengths in micrometres ---------- */
#define QSO_C_UM_PER_FS   0.299792458          /* speed of light            */
#define QSO_RE_UM         2.8179403262e-9      /* classical electron radius */
#define QSO_LBARC_UM      3.8615926796e-7      /* reduced Compton wavelength*/
#define QSO_PI            3.14159265358979323846

/* Gaussian envelope: the phase window is [-QSO_GWIN*Phi, +QSO_GWIN*Phi]. */
#define QSO_GWIN 2.5

/* ------------------------------------------------------------------------
 * Descriptors (the oracle's own; the CUDA library has separate ones).
 * ------------------------------------------------------------------------ */
typedef struct {
    double lambda_um;      /* laser central wavelength                     */
    double a0;             /* peak normalised vector potential             */
    double w0_um;          /* spot size W0 (Eq. 2)                         */
    double tau_fs;         /* intensity FWHM duration                      */
    double dx_um, dy_um;   /* transverse offset of the laser axis          */
    double delay_fs;       /* time at which the pulse peak passes z = 0    */
    double div_prefactor;  /* kappa multiplying Eq. 8                      */
    int32_t envelope;      /* 0 = Gaussian, 1 = sin^2 (field envelope)     */
    int32_t model;         /* 0 = classical LL (Eq. 3), 1 = quantum FP     */
    int32_t n_phase;       /* phase cells of the integration               */
    int32_t variant;       /* bit 0: Eq. 2 in every cell (else at the
                              crossing); bit 1: cycle-resolved chi       */
} qso_laser;

typedef struct {
    double gamma_mean, rel_spread;   /* Gaussian energy: gamma_mean(1+s*xi3) */
    double gamma_lo, gamma_hi;       /* flat energy: lo + (hi-lo)*xi3        */
    double sigma_x_um, sigma_y_um, sigma_z_um;
    double div_rad;                  /* rms angle per transverse axis        */
    double dx_um, dy_um;             /* beam centroid offset                 */
    int32_t flat_energy, pad;
} qso_beam;

typedef struct {
    int32_t n_bins, log_spaced;  double lo, hi;      /* energy spectrum      */
    int32_t n_tx, n_ty;          double theta_max;   /* divergence map       */
    int32_t n_aeff, pad;         double aeff_max;    /* a_eff histogram      */
} qso_bins;

typedef struct {
    double W;          /* total weight                                      */
    double mean;       /* <gamma_f>                                         */
    double spread;     /* rms energy spread (law of total variance)         */
    double rel_spread; /* spread / mean                                     */
    double div_x, div_y, div;  /* rms final angles                          */
    double mean_aeff;  /* <a_eff>                                           */
    double under, over;/* spectrum weight below lo / at or above hi         */
    double map_out;    /* weight outside the divergence map                 */
    double mean_gamma0;/* <gamma_0>                                         */
} qso_moments;

/* Per-sample record written by qso_eval. */
typedef struct {
    double gamma0, aeff, mu, V, theta_e, theta_x, theta_y, gamma_out;
    int32_t bin, ix, iy, abin;
} qso_sample;

/* ---- Neumaier compensated sum ------------------------------------------- */
typedef struct { double s, c; } qso_sum;
static void qso_add(qso_sum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static double qso_val(const qso_sum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------
 * Derived laser constants.
 *   k = 2 pi / lambda,  omega0 = c k,  z_R = pi W0^2 / lambda   (Eq. 2)
 *   R_c = r_e omega0 / c = r_e k
 *   a_S = m c^2/(hbar omega0) = 1/(k lambdabar_c)              (Eq. 6)
 *   Phi = omega0 tau  (intensity FWHM in laser phase)
 *   c_RR = (2/3) R_c * integral of G(phi)^2 dphi  (Eq. 3, head-on, linear
 *          polarisation, cycle-averaged a^2 = A^2/2; the integral is the
 *          analytic one over the whole envelope)
 * out[0..9] = k, omega0, zR, Rc, aS, Phi, PhiT, window_lo, window_hi, cRR
 * ------------------------------------------------------------------------ */
static double qso_sin2_period(double Phi) {
    /* sin^2 field envelope: intensity sin^4(pi phi/PhiT); its FWHM is
       PhiT*(1 - (2/pi) asin(2^-1/4)).  Return PhiT for a given FWHM Phi. */
    return Phi / (1.0 - (2.0 / QSO_PI) * asin(pow(2.0, -0.25)));
}

void qso_constants(const qso_laser* L, double* out) {
    double k = 2.0 * QSO_PI / L->lambda_um;
    double omega0 = QSO_C_UM_PER_FS * k;
    double zR = QSO_PI * L->w0_um * L->w0_um / L->lambda_um;
    double Rc = QSO_RE_UM * k;
    double aS = 1.0 / (k * QSO_LBARC_UM);
    double Phi = omega0 * L->tau_fs;
    double PhiT = qso_sin2_period(Phi);
    double lo, hi, intG2;
    if (L->envelope == 0) {
        lo = -QSO_GWIN * Phi; hi = QSO_GWIN * Phi;
        /* G = exp(-2 ln2 (phi/Phi)^2); G^2 = exp(-4 ln2 phi^2/Phi^2) */
        intG2 = Phi * sqrt(QSO_PI / (4.0 * log(2.0)));
    } else {
        lo = 0.0; hi = PhiT;
        intG2 = 3.0 * PhiT / 8.0;   /* integral of sin^4 over one period */
    }
    out[0] = k; out[1] = omega0; out[2] = zR; out[3] = Rc; out[4] = aS;
    out[5] = Phi; out[6] = PhiT; out[7] = lo; out[8] = hi;
    out[9] = (2.0 / 3.0) * Rc * intG2;
}

/* Envelope G at phase phi (relative to the pulse-peak crossing for the
   Gaussian, to the pulse start for sin^2). */
static double qso_envelope(const qso_laser* L, const double* c, double phi) {
    if (L->envelope == 0) {
        double r = phi / c[5];
        return exp(-2.0 * log(2.0) * r * r);
    }
    if (phi < 0.0 || phi > c[6]) return 0.0;
    double s = sin(QSO_PI * phi / c[6]);
    return s * s;
}

/* Midpoint phase grid: N nodes on the window, spacing h. */
void qso_phase_grid(const qso_laser* L, double* phi, double* G, double* h_out) {
    double c[10];
    qso_constants(L, c);
    int N = L->n_phase;
    double h = (c[8] - c[7]) / (double)N;
    for (int j = 0; j < N; ++j) {
        double p = c[7] + ((double)j + 0.5) * h;
        if (phi) phi[j] = p;
        if (G) G[j] = qso_envelope(L, c, p);
    }
    if (h_out) *h_out = h;
}

/* ------------------------------------------------------------------------
 * Gaunt factor g(chi) (Eq. 6): ratio of the quantum to the classical mean
 * emitted power.  The paper names it but prints no formula; this is the
 * widely used closed-form fit
 *     g = [1 + 4.8 (1+chi) ln(1+1.7 chi) + 2.44 chi^2]^(-2/3),
 * with g(0) = 1 and g ~ chi^(-4/3) at large chi.  gp = dg/dchi.
 * ------------------------------------------------------------------------ */
void qso_gaunt(double chi, double* g, double* gp) {
    double B = 1.0 + 4.8 * (1.0 + chi) * log(1.0 + 1.7 * chi) + 2.44 * chi * chi;
    double dB = 4.8 * log(1.0 + 1.7 * chi) + 4.8 * (1.0 + chi) * 1.7 / (1.0 + 1.7 * chi)
              + 2.0 * 2.44 * chi;
    double gv = pow(B, -2.0 / 3.0);
    if (g) *g = gv;
    if (gp) *gp = (-2.0 / 3.0) * gv / B * dB;
}

/* ------------------------------------------------------------------------
 * Second-moment factor h(chi): ratio of the quantum to the classical
 * second moment of the emitted photon energy per unit time.  Classical
 * reference: (55/(16 sqrt 3)) gamma chi P_cl (storage-ring quantum
 * excitation with critical energy (3/2) gamma chi m c^2).  Fit, as the
 * Gaunt fit g(chi) above times a rational function (max 0.57% off the
 * exact Bessel-function moment for 1e-5 <= chi <= 300):
 *     h = g(chi) (1 + 4.26 chi + 0.494 chi^2)
 *               / (1 + 12.32 chi + 17.44 chi^2 + 1.63 chi^3),
 * h(0) = 1, h ~ chi^(-7/3) at large chi (g ~ chi^(-4/3) times 1/chi).
 * ------------------------------------------------------------------------ */
#define QSO_H_A1 4.26
#define QSO_H_A2 0.494
#define QSO_H_B1 12.32
#define QSO_H_B2 17.44
#define QSO_H_B3 1.63
double qso_h2(double chi) {
    double g;
    qso_gaunt(chi, &g, NULL);
    double num = 1.0 + chi * (QSO_H_A1 + QSO_H_A2 * chi);
    double den = 1.0 + chi * (QSO_H_B1 + chi * (QSO_H_B2 + QSO_H_B3 * chi));
    return g * num / den;
}

/* ------------------------------------------------------------------------
 * n-point Gauss-Legendre rule on [a, b]: nodes are the roots of P_n, found
 * by Newton's method from cos(pi (i + 3/4)/(n + 1/2)); the weights are
 * 2/((1 - z^2) P_n'(z)^2), scaled to the interval.
 * ------------------------------------------------------------------------ */
static void qso_gauss_legendre(int n, double a, double b, double* x, double* w) {
    double mid = 0.5 * (a + b), half = 0.5 * (b - a);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(QSO_PI * (i + 0.75) / (n + 0.5)), pn = 0.0, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            pn = p0;
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = mid - half * z;
        x[n - 1 - i] = mid + half * z;
        w[i] = w[n - 1 - i] = 2.0 * half / ((1.0 - z * z) * dp * dp);
    }
}

/* ------------------------------------------------------------------------
 * Cycle-resolved chi (variant bit 1).  Over one cycle of a linearly
 * polarised field the instantaneous chi is sqrt2 chi |cos psi| (chi: the
 * value at the rms field).  The classical power follows the field squared
 * (2 cos^2 psi times its cycle mean) and the classical second moment its
 * cube (2 sqrt2 |cos psi|^3), so the Fokker-Planck rates take
 *   G(chi) = < 2 cos^2 psi g(sqrt2 chi |cos psi|) >
 *   S(chi) = 2 G + chi dG/dchi
 *   H(chi) = < 2 sqrt2 |cos psi|^3 h(sqrt2 chi |cos psi|) >
 * in place of g, 2g + chi g' and h.  Cycle means over the quarter period
 * (the integrands are smooth there) with a 128-point Gauss-Legendre rule
 * (relative error below 1e-13 for chi <= 40; the branch point of g where
 * 1 + 1.7 sqrt2 chi cos psi = 0 nears the interval as chi grows).
 * ------------------------------------------------------------------------ */
#define QSO_CYC_N 128
void qso_cycle_factors(double chi, double* G, double* S, double* H) {
    static double x[QSO_CYC_N], w[QSO_CYC_N];
    static int ready = 0;
    if (!ready) {
        qso_gauss_legendre(QSO_CYC_N, 0.0, 0.5 * QSO_PI, x, w);
        ready = 1;
    }
    qso_sum sg = {0.0, 0.0}, sd = {0.0, 0.0}, sh = {0.0, 0.0};
    for (int k = 0; k < QSO_CYC_N; ++k) {
        double cp = cos(x[k]);
        double ci = sqrt(2.0) * chi * cp;
        double g, gp;
        qso_gaunt(ci, &g, &gp);
        qso_add(&sg, w[k] * 2.0 * cp * cp * g);
        qso_add(&sd, w[k] * 2.0 * cp * cp * gp * sqrt(2.0) * cp);
        qso_add(&sh, w[k] * 2.0 * sqrt(2.0) * cp * cp * cp * qso_h2(ci));
    }
    double nrm = 2.0 / QSO_PI;            /* mean over the quarter period */
    *G = nrm * qso_val(&sg);
    *S = 2.0 * (*G) + chi * nrm * qso_val(&sd);
    *H = nrm * qso_val(&sh);
}

/* ------------------------------------------------------------------------
 * Fokker-Planck moment rates per unit laser phase (Eq. 6 and the
 * Fokker-Planck regime the paper names), for an electron of mean energy mu
 * in a cycle-averaged field of envelope amplitude A (linear polarisation:
 * rms field A/sqrt 2, so chi = 2 mu (A/sqrt2)/a_S).  With K = (2/3) R_c A^2:
 *   D1  = d<gamma>/dphi           = -K mu^2 g(chi)
 *   dD1 = dD1/dgamma              = -K mu (2 g + chi g'(chi))
 *   D2  = d<dgamma^2>/dphi (diff) =  (55/(16 sqrt 3)) K mu^3 chi h(chi)
 * aS_scale multiplies a_S (1 = physical; huge = classical limit).
 * out[0..3] = D1, dD1, D2, chi
 * ------------------------------------------------------------------------ */
static void qso_rates_c(const double* c, double mu, double A, double aS_scale, int cycle,
                        double* out) {
    double Rc = c[3], aS = c[4] * aS_scale;
    double chi = 2.0 * mu * (A / sqrt(2.0)) / aS;
    double g, gp, h2, sf;
    if (cycle) {
        qso_cycle_factors(chi, &g, &sf, &h2);
    } else {
        qso_gaunt(chi, &g, &gp);
        h2 = qso_h2(chi);
        sf = 2.0 * g + chi * gp;
    }
    double K = (2.0 / 3.0) * Rc * A * A;
    out[0] = -K * mu * mu * g;
    out[1] = -K * mu * sf;
    out[2] = (55.0 / (16.0 * sqrt(3.0))) * K * mu * mu * mu * chi * h2;
    out[3] = chi;
}

void qso_qfp_rates(const qso_laser* L, double mu, double A, double aS_scale, double* out) {
    double c[10];
    qso_constants(L, c);
    qso_rates_c(c, mu, A, aS_scale, (L->variant & 2) != 0, out);
}

/* ------------------------------------------------------------------------
 * Quantum-corrected phase integration of one electron of initial energy
 * gamma0 seeing a plane-wave pulse of peak amplitude aeff (Eq. 6, Fokker-
 * Planck mean/variance closure), second order in the step h.
 *
 * State: du = 1/mu - 1/gamma0 (so mu = gamma0/(1 + gamma0 du), exactly
 * gamma0 when nothing is radiated) and the variance V.  Cell j has its
 * midpoint at phi_j, where the envelope and the rates are evaluated:
 *   K_j   = (2/3) R_c A_j^2,  A_j = aeff G(phi_j)
 *   du^   = du_j + (h/2) K_j g_{j-1}        (state at the cell midpoint,
 *           g_{-1} = 1: the previous cell's Gaunt factor predicts it)
 *   mu^   = gamma0/(1 + gamma0 du^),  rates D1, dD1, D2 at (mu^, A_j)
 *   du_{j+1} = du_j + h K_j g_j             (= du_j - h D1/mu^2)
 *   lambda = 2 dD1,  r = lambda V_j + D2
 *   V_{j+1}  = V_j + h r + (h^2/2) lambda r (frozen-rate Taylor step)
 * aS_scale multiplies a_S; d2_scale multiplies D2 (0 = no diffusion).
 * ------------------------------------------------------------------------ */
/* a_cell[j] (NULL: aeff in every cell) is the local peak amplitude of the
   focus in cell j (the per-cell focus variant). */
/* mu_cell, chi_cell (optional): the mean energy at each cell midpoint (the
   state the cell's rates use) and the cell's chi. */
static void qso_qfp_run(const qso_laser* L, const double* a_cell, double aeff, double gamma0,
                        double V0, double aS_scale, double d2_scale, double* mu_out,
                        double* V_out, double* mu_cell, double* chi_cell) {
    int N = L->n_phase;
    double c[10];
    qso_constants(L, c);
    double h = (c[8] - c[7]) / (double)N;
    double du = 0.0, V = V0, g_prev = 1.0;
    for (int j = 0; j < N; ++j) {
        double phi = c[7] + ((double)j + 0.5) * h;   /* midpoint of cell j */
        double A = (a_cell ? a_cell[j] : aeff) * qso_envelope(L, c, phi);
        double K = (2.0 / 3.0) * c[3] * A * A;
        double du_mid = du + 0.5 * h * K * g_prev;
        double mu = gamma0 / (1.0 + gamma0 * du_mid);
        double r[4];
        qso_rates_c(c, mu, A, aS_scale, (L->variant & 2) != 0, r);
        if (mu_cell) mu_cell[j] = mu;
        if (chi_cell) chi_cell[j] = r[3];
        double g = -r[0] / (K * mu * mu);          /* Gaunt factor at chi_j */
        if (!(K > 0.0)) g = 1.0;
        double lam = 2.0 * r[1];
        double rv = lam * V + d2_scale * r[2];
        du += h * K * g;
        V += h * rv + 0.5 * h * h * lam * rv;
        g_prev = g;
    }
    *mu_out = gamma0 / (1.0 + gamma0 * du);
    *V_out = V;
}

void qso_qfp_integrate(const qso_laser* L, double aeff, double gamma0, double V0,
                       double aS_scale, double d2_scale, double* mu_out, double* V_out) {
    qso_qfp_run(L, NULL, aeff, gamma0, V0, aS_scale, d2_scale, mu_out, V_out, NULL, NULL);
}

/* ------------------------------------------------------------------------
 * Local Gaussian focus, Eq. 2, at longitudinal position zz and transverse
 * offsets (xx, yy) from the laser axis.
 * ------------------------------------------------------------------------ */
static double qso_focus(const qso_laser* L, double zR, double zz, double xx, double yy) {
    double q = 1.0 + (zz / zR) * (zz / zR);
    return L->a0 / sqrt(q) * exp(-(xx * xx + yy * yy) / (L->w0_um * L->w0_um * q));
}

/* Phase of the pulse peak on the envelope's phase axis. */
static double qso_peak_phase(const qso_laser* L, const double* c) {
    return L->envelope == 0 ? 0.0 : 0.5 * c[6];
}

/* ------------------------------------------------------------------------
 * Per-cell focus (the variant of Eq. 2 without the paper's neglect of the
 * focus change during the crossing).  The electron (velocity
 * c(theta_x, theta_y, -1)) meets the counter-propagating phase at twice the
 * laser frequency, so between the crossing of the pulse peak and the
 * midpoint of cell j (phase phi_j, the peak at phi_c) it travels
 * s_j = (phi_j - phi_c)/(2k) along -z and theta s_j sideways:
 *   z_j = z* - s_j,  x_j = xs + theta_x s_j,  y_j = ys + theta_y s_j,
 *   a_j = Eq. 2 at (z_j, x_j, y_j).
 * ------------------------------------------------------------------------ */
static void qso_focus_cells(const qso_laser* L, double zs, double xs, double ys, double thx,
                            double thy, double* a_cell) {
    double c[10];
    qso_constants(L, c);
    int N = L->n_phase;
    double h = (c[8] - c[7]) / (double)N, phic = qso_peak_phase(L, c);
    for (int j = 0; j < N; ++j) {
        double phi = c[7] + ((double)j + 0.5) * h;
        double sj = (phi - phic) / (2.0 * c[0]);
        a_cell[j] = qso_focus(L, c[2], zs - sj, xs + thx * sj, ys + thy * sj);
    }
}

/* ------------------------------------------------------------------------
 * One beam sample, steps in the paper's order.
 * xi[0..7]: standard variates for x, y, z, gamma0 (uniform [0,1) if the
 * energy is flat), theta_x, theta_y, angular noise, energy noise.
 *
 * Geometry (Eq. 1 factor 2, Table 1 z_pm = Delta_par +- L/4): the laser
 * moves along +z, focus at the origin, its peak passes z = 0 at t = delay.
 * The electron sits at (x, y, z) at t = 0 and moves with velocity
 * c(theta_x, theta_y, -1).  It meets the pulse peak at
 *   c t* = (z + c delay)/2,   z* = (z - c delay)/2,
 * transverse position x + theta_x c t*, y + theta_y c t*.
 * ------------------------------------------------------------------------ */
static void qso_sample_eval_x(const qso_laser* L, const qso_beam* B, const qso_bins* bins,
                              const double* xi, qso_sample* s, double* mu_cell,
                              double* chi_cell) {
    double c[10];
    qso_constants(L, c);
    double zR = c[2], aS = c[4], cRR = c[9];
    (void)aS;

    /* decode (reparameterised sample) */
    double x = B->dx_um + B->sigma_x_um * xi[0];
    double y = B->dy_um + B->sigma_y_um * xi[1];
    double z = B->sigma_z_um * xi[2];
    double gamma0;
    if (B->flat_energy) gamma0 = B->gamma_lo + (B->gamma_hi - B->gamma_lo) * xi[3];
    else                gamma0 = B->gamma_mean * (1.0 + B->rel_spread * xi[3]);
    if (gamma0 < 1.0) gamma0 = 1.0;     /* unphysical tail clamped to rest */
    double thx = B->div_rad * xi[4];
    double thy = B->div_rad * xi[5];

    /* collision geometry */
    double ct = 0.5 * (z + QSO_C_UM_PER_FS * L->delay_fs);
    double zs = 0.5 * (z - QSO_C_UM_PER_FS * L->delay_fs);
    double xs = x + thx * ct - L->dx_um;
    double ys = y + thy * ct - L->dy_um;
    double rho2 = xs * xs + ys * ys;

    /* local Gaussian focus, Eq. 2 */
    double q = 1.0 + (zs / zR) * (zs / zR);
    double aeff = L->a0 / sqrt(q) * exp(-rho2 / (L->w0_um * L->w0_um * q));

    double mu, V;
    if (!(L->variant & 1)) {
        if (L->model == 0) {
            /* classical LL closed form, Eq. 3 with a0 -> a_eff */
            mu = gamma0 / (1.0 + cRR * gamma0 * aeff * aeff);
            V = 0.0;
        } else {
            qso_qfp_run(L, NULL, aeff, gamma0, 0.0, 1.0, 1.0, &mu, &V, mu_cell, chi_cell);
        }
    } else {
        double* a_cell = (double*)malloc(sizeof(double) * (size_t)L->n_phase);
        qso_focus_cells(L, zs, xs, ys, thx, thy, a_cell);
        if (L->model == 0) {
            /* Eq. 3's exponent cell by cell: 1/gamma_f = 1/gamma0 +
               (2/3) R_c h sum_j (a_j G_j)^2 (compensated sum) */
            double h = (c[8] - c[7]) / (double)L->n_phase;
            qso_sum acc = {0.0, 0.0};
            for (int j = 0; j < L->n_phase; ++j) {
                double A = a_cell[j] * qso_envelope(L, c, c[7] + ((double)j + 0.5) * h);
                qso_add(&acc, A * A);
            }
            double du = (2.0 / 3.0) * c[3] * h * qso_val(&acc);
            mu = gamma0 / (1.0 + gamma0 * du);
            V = 0.0;
        } else {
            qso_qfp_run(L, a_cell, aeff, gamma0, 0.0, 1.0, 1.0, &mu, &V, mu_cell, chi_cell);
        }
        free(a_cell);
    }

    /* final divergence, Eq. 8 with prefactor kappa; the broadening acts
       along the polarisation axis x */
    double theta_e = 0.0;
    if (L->model != 0 && V > 0.0)
        theta_e = L->div_prefactor * sqrt(2.0 / QSO_PI) * aeff * sqrt(V) / (mu * mu);
    double tx = thx + theta_e * xi[6];
    double ty = thy;

    /* realised final energy: mean plus Gaussian spread of variance V */
    double gout = mu;
    if (L->model != 0) gout = mu + sqrt(V > 0.0 ? V : 0.0) * xi[7];

    s->gamma0 = gamma0; s->aeff = aeff; s->mu = mu; s->V = V;
    s->theta_e = theta_e; s->theta_x = tx; s->theta_y = ty; s->gamma_out = gout;

    /* bins: half-open [lo + b w, lo + (b+1) w); -1 = under, n = over */
    s->bin = -1; s->ix = -1; s->iy = -1; s->abin = -1;
    if (bins) {
        int n = bins->n_bins;
        if (n > 0) {
            double t;
            if (!bins->log_spaced) {
                double inv_w = (double)n / (bins->hi - bins->lo);
                t = (gout - bins->lo) * inv_w;
            } else {
                double sc = (double)n / log(bins->hi / bins->lo);
                t = (gout > 0.0) ? log(gout / bins->lo) * sc : -1.0;
            }
            if (!(t >= 0.0)) s->bin = -1;
            else if (t >= (double)n) s->bin = n;
            else s->bin = (int32_t)floor(t);
        }
        if (bins->n_tx > 0 && bins->n_ty > 0) {
            double tm = bins->theta_max;
            double sx = (double)bins->n_tx / (2.0 * tm);
            double sy = (double)bins->n_ty / (2.0 * tm);
            double fx = (tx + tm) * sx, fy = (ty + tm) * sy;
            if (fx >= 0.0 && fx < (double)bins->n_tx && fy >= 0.0 && fy < (double)bins->n_ty) {
                s->ix = (int32_t)floor(fx);
                s->iy = (int32_t)floor(fy);
            }
        }
        if (bins->n_aeff > 0) {
            double fa = aeff * ((double)bins->n_aeff / bins->aeff_max);
            if (fa >= 0.0 && fa < (double)bins->n_aeff) s->abin = (int32_t)floor(fa);
            else s->abin = bins->n_aeff;
        }
    }
}

static void qso_sample_eval(const qso_laser* L, const qso_beam* B, const qso_bins* bins,
                            const double* xi, qso_sample* s) {
    qso_sample_eval_x(L, B, bins, xi, s, NULL, NULL);
}

/* Per-sample evaluation of n samples; xi[k] points to n doubles (NULL = 0). */
void qso_eval(const qso_laser* L, const qso_beam* B, const qso_bins* bins,
              int64_t n, const double* const* xi, qso_sample* out) {
    for (int64_t i = 0; i < n; ++i) {
        double v[8];
        for (int k = 0; k < 8; ++k) v[k] = xi[k] ? xi[k][i] : 0.0;
        qso_sample_eval(L, B, bins, v, &out[i]);
    }
}

/* ------------------------------------------------------------------------
 * Whole-beam integration: weighted histograms (Eq. 4 done as a weighted
 * histogram of the per-sample final energies; Eq. 1 as the a_eff
 * histogram) and moments.  Spectrum entries are bin masses (sum of weights),
 * not densities.  Moments follow their definitions directly:
 *   mean   = sum w mu / W
 *   spread = sqrt( sum w (mu - mean)^2 / W + sum w V / W )
 *   div_x  = sqrt( sum w (theta_x0^2 + theta_e^2) / W ), div_y likewise
 *            without theta_e, div = sqrt(div_x^2 + div_y^2)
 * w == NULL means unit weights.  Arrays may be NULL when disabled.
 * ------------------------------------------------------------------------ */
int qso_scatter(const qso_laser* L, const qso_beam* B, const qso_bins* bins,
                int64_t n, const double* const* xi, const double* w,
                double* spectrum, double* divmap, double* aeff_hist, qso_moments* m) {
    int nb = bins->n_bins, ntx = bins->n_tx, nty = bins->n_ty, na = bins->n_aeff;
    /* compensated accumulators for every output */
    int64_t nmap = (ntx > 0 && nty > 0) ? (int64_t)ntx * nty : 0;
    qso_sum* spec = (qso_sum*)calloc((size_t)(nb > 0 ? nb : 0) + 1, sizeof(qso_sum));
    qso_sum* map = (qso_sum*)calloc((size_t)nmap + 1, sizeof(qso_sum));
    qso_sum* ah = (qso_sum*)calloc((size_t)(na > 0 ? na : 0) + 1, sizeof(qso_sum));
    if (!spec || !map || !ah) { free(spec); free(map); free(ah); return 1; }

    qso_sum W = {0, 0}, Smu = {0, 0}, SV = {0, 0}, Sa = {0, 0}, Sg0 = {0, 0};
    qso_sum Stx = {0, 0}, Sty = {0, 0}, under = {0, 0}, over = {0, 0}, mapout = {0, 0};

    /* first pass: per-sample evaluation, histograms, first moments */
    for (int64_t i = 0; i < n; ++i) {
        double v[8];
        for (int k = 0; k < 8; ++k) v[k] = xi[k] ? xi[k][i] : 0.0;
        qso_sample s;
        qso_sample_eval(L, B, bins, v, &s);
        double wi = w ? w[i] : 1.0;
        qso_add(&W, wi);
        qso_add(&Smu, wi * s.mu);
        qso_add(&SV, wi * s.V);
        qso_add(&Sa, wi * s.aeff);
        qso_add(&Sg0, wi * s.gamma0);
        double thx0 = B->div_rad * v[4], thy0 = B->div_rad * v[5];
        qso_add(&Stx, wi * (thx0 * thx0 + s.theta_e * s.theta_e));
        qso_add(&Sty, wi * (thy0 * thy0));
        if (nb > 0) {
            if (s.bin < 0) qso_add(&under, wi);
            else if (s.bin >= nb) qso_add(&over, wi);
            else qso_add(&spec[s.bin], wi);
        }
        if (ntx > 0 && nty > 0) {
            if (s.ix >= 0) qso_add(&map[(int64_t)s.iy * ntx + s.ix], wi);
            else qso_add(&mapout, wi);
        }
        if (na > 0) qso_add(&ah[s.abin], wi);
    }
    double Wv = qso_val(&W);
    double mean = Wv > 0 ? qso_val(&Smu) / Wv : 0.0;

    /* second pass: central second moment of the per-sample means */
    qso_sum S2 = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double v[8];
        for (int k = 0; k < 8; ++k) v[k] = xi[k] ? xi[k][i] : 0.0;
        qso_sample s;
        qso_sample_eval(L, B, bins, v, &s);
        double wi = w ? w[i] : 1.0;
        double d = s.mu - mean;
        qso_add(&S2, wi * d * d);
    }

    if (spectrum) for (int b = 0; b < nb; ++b) spectrum[b] = qso_val(&spec[b]);
    if (divmap) for (int64_t b = 0; b < nmap; ++b) divmap[b] = qso_val(&map[b]);
    if (aeff_hist) for (int b = 0; b < na; ++b) aeff_hist[b] = qso_val(&ah[b]);
    free(spec); free(map); free(ah);

    memset(m, 0, sizeof(*m));
    m->W = Wv;
    m->under = qso_val(&under);
    m->over = qso_val(&over);
    m->map_out = qso_val(&mapout);
    if (Wv > 0) {
        double var = qso_val(&S2) / Wv + qso_val(&SV) / Wv;
        m->mean = mean;
        m->spread = sqrt(var > 0 ? var : 0.0);
        m->rel_spread = m->spread / mean;
        m->div_x = sqrt(qso_val(&Stx) / Wv);
        m->div_y = sqrt(qso_val(&Sty) / Wv);
        m->div = sqrt((qso_val(&Stx) + qso_val(&Sty)) / Wv);
        m->mean_aeff = qso_val(&Sa) / Wv;
        m->mean_gamma0 = qso_val(&Sg0) / Wv;
    }
    return 0;
}

/* ========================================================================
 * Kernel-smoothed spectrum and gradients (test infrastructure).
 *
 * Smoothed spectrum (uniform bins only), the differentiable stand-in for the
 * energy histogram of Eq. 4 used by a fitting loss:
 *   S_k = sum_i w_i (Delta / (sigma sqrt(2 pi))) exp(-(c_k - g_i)^2 / (2 sigma^2))
 * with c_k = lo + (k + 1/2) Delta, sigma = sigma_bins Delta, g_i the realised
 * final energy, and only bins with |c_k - g_i| <= 6 sigma included.
 *
 * Gradients: forward-mode automatic differentiation with dual numbers that
 * carry the derivatives with respect to the 8 parameters
 *   (a0, W0, dx, dy, delay, gamma_mean, rel_spread, div_rad)
 * through every step of the per-sample evaluation above (decode, geometry,
 * Eq. 2, Eq. 3 or the phase integration, Eq. 8) and through the moment and
 * smoothed-spectrum sums.  The loss gradient is the contraction with the
 * caller's dL/d(moments) and dL/dS.  Nothing here is hand-differentiated.
 * ======================================================================== */
#define QSO_ND 8
typedef struct { double v; double d[QSO_ND]; } qd;

static qd qd_c(double v) { qd r; r.v = v; memset(r.d, 0, sizeof(r.d)); return r; }
static qd qd_var(double v, int k) { qd r = qd_c(v); r.d[k] = 1.0; return r; }
static qd qd_add(qd a, qd b) { qd r; r.v = a.v + b.v; for (int k = 0; k < QSO_ND; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
static qd qd_sub(qd a, qd b) { qd r; r.v = a.v - b.v; for (int k = 0; k < QSO_ND; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
static qd qd_mul(qd a, qd b) { qd r; r.v = a.v * b.v; for (int k = 0; k < QSO_ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
static qd qd_div(qd a, qd b) { qd r; r.v = a.v / b.v; for (int k = 0; k < QSO_ND; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v; return r; }
static qd qd_scale(qd a, double s) { qd r; r.v = a.v * s; for (int k = 0; k < QSO_ND; ++k) r.d[k] = a.d[k] * s; return r; }
static qd qd_addc(qd a, double c) { a.v += c; return a; }
static qd qd_fn(qd a, double f, double df) { qd r; r.v = f; for (int k = 0; k < QSO_ND; ++k) r.d[k] = df * a.d[k]; return r; }
static qd qd_sqrt(qd a) { double s = sqrt(a.v); return qd_fn(a, s, s > 0 ? 0.5 / s : 0.0); }
static qd qd_exp(qd a) { double e = exp(a.v); return qd_fn(a, e, e); }
static qd qd_log(qd a) { return qd_fn(a, log(a.v), 1.0 / a.v); }
static qd qd_pow(qd a, double p) { double y = pow(a.v, p); return qd_fn(a, y, p * pow(a.v, p - 1.0)); }

/* Gaunt and second-moment factors as written above, in dual arithmetic. */
static qd qd_gaunt(qd chi) {
    qd B = qd_addc(qd_add(qd_scale(qd_mul(qd_addc(chi, 1.0), qd_log(qd_addc(qd_scale(chi, 1.7), 1.0))), 4.8),
                          qd_scale(qd_mul(chi, chi), 2.44)), 1.0);
    return qd_pow(B, -2.0 / 3.0);
}
static qd qd_h2(qd chi) {
    qd num = qd_addc(qd_mul(chi, qd_addc(qd_scale(chi, QSO_H_A2), QSO_H_A1)), 1.0);
    qd den = qd_addc(qd_mul(chi, qd_addc(qd_mul(chi, qd_addc(qd_scale(chi, QSO_H_B3), QSO_H_B2)),
                                         QSO_H_B1)), 1.0);
    return qd_div(qd_mul(qd_gaunt(chi), num), den);
}

/* d g / d chi of the Gaunt fit, in dual arithmetic (enters the variance
   transport term), obtained by differentiating B^(-2/3) symbolically once:
   g' = -(2/3) B^(-5/3) B',  B' = 4.8 ln(1+1.7chi) + 4.8 (1+chi) 1.7/(1+1.7chi) + 4.88 chi */
static qd qd_gaunt_prime(qd chi) {
    qd x1 = qd_addc(qd_scale(chi, 1.7), 1.0);
    qd B = qd_addc(qd_add(qd_scale(qd_mul(qd_addc(chi, 1.0), qd_log(x1)), 4.8),
                          qd_scale(qd_mul(chi, chi), 2.44)), 1.0);
    qd dB = qd_add(qd_add(qd_scale(qd_log(x1), 4.8),
                          qd_scale(qd_div(qd_addc(chi, 1.0), x1), 4.8 * 1.7)),
                   qd_scale(chi, 4.88));
    return qd_scale(qd_mul(qd_pow(B, -5.0 / 3.0), dB), -2.0 / 3.0);
}

/* Cycle-resolved factors (variant bit 1) in dual arithmetic: the same
   128-point Gauss-Legendre cycle means as qso_cycle_factors, of the dual
   Gaunt factor, its derivative and the second-moment factor. */
static void qd_cycle_factors(qd chi, qd* G, qd* S, qd* H) {
    static double x[QSO_CYC_N], w[QSO_CYC_N];
    static int ready = 0;
    if (!ready) {
        qso_gauss_legendre(QSO_CYC_N, 0.0, 0.5 * QSO_PI, x, w);
        ready = 1;
    }
    qd sg = qd_c(0.0), sd = qd_c(0.0), sh = qd_c(0.0);
    for (int k = 0; k < QSO_CYC_N; ++k) {
        double cp = cos(x[k]);
        qd ci = qd_scale(chi, sqrt(2.0) * cp);
        sg = qd_add(sg, qd_scale(qd_gaunt(ci), w[k] * 2.0 * cp * cp));
        sd = qd_add(sd, qd_scale(qd_gaunt_prime(ci), w[k] * 2.0 * cp * cp * sqrt(2.0) * cp));
        sh = qd_add(sh, qd_scale(qd_h2(ci), w[k] * 2.0 * sqrt(2.0) * cp * cp * cp));
    }
    double nrm = 2.0 / QSO_PI;
    *G = qd_scale(sg, nrm);
    *S = qd_add(qd_scale(*G, 2.0), qd_mul(chi, qd_scale(sd, nrm)));
    *H = qd_scale(sh, nrm);
}

/* Eq. 2 at (zz, xx, yy) in dual arithmetic (per-cell focus). */
static qd qd_focus(qd a0, qd w0, qd zR, qd zz, qd xx, qd yy) {
    qd zq = qd_div(zz, zR);
    qd q = qd_addc(qd_mul(zq, zq), 1.0);
    qd rho2 = qd_add(qd_mul(xx, xx), qd_mul(yy, yy));
    return qd_mul(qd_div(a0, qd_sqrt(q)),
                  qd_exp(qd_scale(qd_div(rho2, qd_mul(qd_mul(w0, w0), q)), -1.0)));
}

typedef struct {
    qd gamma0, aeff, mu, V, theta_e, thx0, thy0, gout;
} qso_dsample;

/* One sample in dual arithmetic (mirrors qso_sample_eval, same order). */
static void qso_sample_dual(const qso_laser* L, const qso_beam* B, const double* xi,
                            qso_dsample* s) {
    double c[10];
    qso_constants(L, c);
    qd a0 = qd_var(L->a0, 0), w0 = qd_var(L->w0_um, 1), ldx = qd_var(L->dx_um, 2),
       ldy = qd_var(L->dy_um, 3), delay = qd_var(L->delay_fs, 4), gm = qd_var(B->gamma_mean, 5),
       sp = qd_var(B->rel_spread, 6), dv = qd_var(B->div_rad, 7);
    qd x = qd_c(B->dx_um + B->sigma_x_um * xi[0]);
    qd y = qd_c(B->dy_um + B->sigma_y_um * xi[1]);
    qd z = qd_c(B->sigma_z_um * xi[2]);
    qd gamma0;
    if (B->flat_energy) gamma0 = qd_c(B->gamma_lo + (B->gamma_hi - B->gamma_lo) * xi[3]);
    else gamma0 = qd_mul(gm, qd_addc(qd_scale(sp, xi[3]), 1.0));
    if (gamma0.v < 1.0) gamma0 = qd_c(1.0);
    qd thx = qd_scale(dv, xi[4]), thy = qd_scale(dv, xi[5]);
    qd cdel = qd_scale(delay, QSO_C_UM_PER_FS);
    qd ct = qd_scale(qd_add(z, cdel), 0.5);
    qd zs = qd_scale(qd_sub(z, cdel), 0.5);
    qd xs = qd_sub(qd_add(x, qd_mul(thx, ct)), ldx);
    qd ys = qd_sub(qd_add(y, qd_mul(thy, ct)), ldy);
    qd rho2 = qd_add(qd_mul(xs, xs), qd_mul(ys, ys));
    qd zR = qd_scale(qd_mul(w0, w0), QSO_PI / L->lambda_um);
    qd zq = qd_div(zs, zR);
    qd q = qd_addc(qd_mul(zq, zq), 1.0);
    qd aeff = qd_mul(qd_div(a0, qd_sqrt(q)),
                     qd_exp(qd_scale(qd_div(rho2, qd_mul(qd_mul(w0, w0), q)), -1.0)));
    qd mu, V = qd_c(0.0);
    int N = L->n_phase;
    double h = (c[8] - c[7]) / (double)N;
    int cellf = (L->variant & 1) != 0, cyc = (L->variant & 2) != 0;
    /* per-cell focus: the local amplitude of cell j along the path (as in
       qso_focus_cells) in dual arithmetic */
    double phic = qso_peak_phase(L, c);
    if (L->model == 0 && !cellf) {
        mu = qd_div(gamma0, qd_addc(qd_scale(qd_mul(gamma0, qd_mul(aeff, aeff)), c[9]), 1.0));
    } else if (L->model == 0) {
        /* Eq. 3's exponent cell by cell (as in qso_sample_eval_x) */
        qd acc = qd_c(0.0);
        for (int j = 0; j < N; ++j) {
            double phi = c[7] + ((double)j + 0.5) * h, sj = (phi - phic) / (2.0 * c[0]);
            qd aj = qd_focus(a0, w0, zR, qd_addc(zs, -sj), qd_add(xs, qd_scale(thx, sj)),
                             qd_add(ys, qd_scale(thy, sj)));
            qd A = qd_scale(aj, qso_envelope(L, c, phi));
            acc = qd_add(acc, qd_mul(A, A));
        }
        qd du = qd_scale(acc, (2.0 / 3.0) * c[3] * h);
        mu = qd_div(gamma0, qd_addc(qd_mul(gamma0, du), 1.0));
    } else {
        qd du = qd_c(0.0), g_prev = qd_c(1.0);
        for (int j = 0; j < N; ++j) {
            double phi = c[7] + ((double)j + 0.5) * h;
            double G = qso_envelope(L, c, phi);
            qd aj = aeff;
            if (cellf) {
                double sj = (phi - phic) / (2.0 * c[0]);
                aj = qd_focus(a0, w0, zR, qd_addc(zs, -sj), qd_add(xs, qd_scale(thx, sj)),
                              qd_add(ys, qd_scale(thy, sj)));
            }
            qd A = qd_scale(aj, G);
            qd K = qd_scale(qd_mul(A, A), (2.0 / 3.0) * c[3]);
            qd du_mid = qd_add(du, qd_scale(qd_mul(K, g_prev), 0.5 * h));
            qd m = qd_div(gamma0, qd_addc(qd_mul(gamma0, du_mid), 1.0));
            qd chi = qd_scale(qd_mul(m, A), sqrt(2.0) / c[4]);
            qd g, sfac, h2;
            if (cyc) {
                qd_cycle_factors(chi, &g, &sfac, &h2);
            } else {
                g = qd_gaunt(chi);
                h2 = qd_h2(chi);
                sfac = qd_add(qd_scale(g, 2.0), qd_mul(chi, qd_gaunt_prime(chi)));
            }
            qd lam = qd_scale(qd_mul(qd_mul(K, m), sfac), -2.0);
            qd D2 = qd_scale(qd_mul(qd_mul(qd_mul(K, qd_mul(m, qd_mul(m, m))), chi), h2),
                             55.0 / (16.0 * sqrt(3.0)));
            qd rv = qd_add(qd_mul(lam, V), D2);
            du = qd_add(du, qd_scale(qd_mul(K, g), h));
            V = qd_add(V, qd_add(qd_scale(rv, h), qd_scale(qd_mul(lam, rv), 0.5 * h * h)));
            g_prev = g;
        }
        mu = qd_div(gamma0, qd_addc(qd_mul(gamma0, du), 1.0));
    }
    qd theta_e = qd_c(0.0), gout = mu;
    if (L->model != 0 && V.v > 0.0) {
        theta_e = qd_scale(qd_div(qd_mul(aeff, qd_sqrt(V)), qd_mul(mu, mu)),
                           L->div_prefactor * sqrt(2.0 / QSO_PI));
        gout = qd_add(mu, qd_scale(qd_sqrt(V), xi[7]));
    }
    s->gamma0 = gamma0; s->aeff = aeff; s->mu = mu; s->V = V; s->theta_e = theta_e;
    s->thx0 = thx; s->thy0 = thy; s->gout = gout;
}

/* Bins k with |c_k - g| <= 6 sigma, clamped to [0, n). */
static void qso_smooth_range(const qso_bins* b, double sigma_bins, double g, int* k0, int* k1) {
    double t = (g - b->lo) * ((double)b->n_bins / (b->hi - b->lo));
    double lo = ceil(t - 0.5 - 6.0 * sigma_bins), hi = floor(t - 0.5 + 6.0 * sigma_bins);
    if (lo < 0) lo = 0;
    if (hi > b->n_bins - 1) hi = b->n_bins - 1;
    *k0 = (int)lo; *k1 = (int)hi;
}

/* Forward smoothed spectrum and moments, plus the gradient of
   L with respect to the 8 parameters given dL/dm (13 entries, qso_moments
   order; NULL = 0) and dL/dS (n_bins; NULL = 0).  Returns 0, or 1 on bad
   arguments / allocation failure. */
int qso_grad(const qso_laser* L, const qso_beam* B, const qso_bins* bins, double sigma_bins,
             int64_t n, const double* const* xi, const double* w, const double* dL_dm,
             const double* dL_dS, double* grad8, double* smooth, qso_moments* m) {
    int nb = bins->n_bins;
    if (nb <= 0 || bins->log_spaced || !(sigma_bins > 0)) return 1;
    qd* S = (qd*)calloc((size_t)nb, sizeof(qd));
    if (!S) return 1;
    for (int k = 0; k < nb; ++k) S[k] = qd_c(0.0);
    double delta = (bins->hi - bins->lo) / (double)nb;
    double sig = sigma_bins * delta;
    double pref = delta / (sig * sqrt(2.0 * QSO_PI));
    qd W = qd_c(0.0), S1 = qd_c(0.0), SV = qd_c(0.0), Stx = qd_c(0.0), Sty = qd_c(0.0),
       Sa = qd_c(0.0), Sg0 = qd_c(0.0);
    qso_dsample* all = (qso_dsample*)malloc((size_t)(n > 0 ? n : 1) * sizeof(qso_dsample));
    if (!all) { free(S); return 1; }
    for (int64_t i = 0; i < n; ++i) {
        double v[8];
        for (int k = 0; k < 8; ++k) v[k] = xi[k] ? xi[k][i] : 0.0;
        qso_dsample* s = &all[i];
        qso_sample_dual(L, B, v, s);
        double wi = w ? w[i] : 1.0;
        W = qd_addc(W, wi);
        S1 = qd_add(S1, qd_scale(s->mu, wi));
        SV = qd_add(SV, qd_scale(s->V, wi));
        Stx = qd_add(Stx, qd_scale(qd_add(qd_mul(s->thx0, s->thx0), qd_mul(s->theta_e, s->theta_e)), wi));
        Sty = qd_add(Sty, qd_scale(qd_mul(s->thy0, s->thy0), wi));
        Sa = qd_add(Sa, qd_scale(s->aeff, wi));
        Sg0 = qd_add(Sg0, qd_scale(s->gamma0, wi));
        int k0, k1;
        qso_smooth_range(bins, sigma_bins, s->gout.v, &k0, &k1);
        for (int k = k0; k <= k1; ++k) {
            double ck = bins->lo + ((double)k + 0.5) * delta;
            qd dlt = qd_addc(qd_scale(s->gout, -1.0), ck);
            qd e = qd_exp(qd_scale(qd_mul(dlt, dlt), -1.0 / (2.0 * sig * sig)));
            S[k] = qd_add(S[k], qd_scale(e, wi * pref));
        }
    }
    qd mean = qd_scale(S1, 1.0 / W.v);
    /* central second moment: value by the two-pass definition, derivative
       of sum w (mu - mean)^2 / W = sum w mu^2 / W - mean^2 taken exactly */
    qd S2c = qd_c(0.0);
    for (int64_t i = 0; i < n; ++i) {
        double wi = w ? w[i] : 1.0;
        qd d = qd_sub(all[i].mu, mean);
        S2c = qd_add(S2c, qd_scale(qd_mul(d, d), wi));
    }
    qd var = qd_add(qd_scale(S2c, 1.0 / W.v), qd_scale(SV, 1.0 / W.v));
    qd spread = qd_sqrt(var);
    qd mom[13];
    for (int k = 0; k < 13; ++k) mom[k] = qd_c(0.0);
    mom[0] = W;
    mom[1] = mean;
    mom[2] = spread;
    mom[3] = qd_div(spread, mean);
    mom[4] = qd_sqrt(qd_scale(Stx, 1.0 / W.v));
    mom[5] = qd_sqrt(qd_scale(Sty, 1.0 / W.v));
    mom[6] = qd_sqrt(qd_scale(qd_add(Stx, Sty), 1.0 / W.v));
    mom[7] = qd_scale(Sa, 1.0 / W.v);
    mom[11] = qd_scale(Sg0, 1.0 / W.v);
    for (int k = 0; k < QSO_ND; ++k) {
        double g = 0.0;
        if (dL_dm) for (int j = 0; j < 13; ++j) g += dL_dm[j] * mom[j].d[k];
        if (dL_dS) for (int b = 0; b < nb; ++b) g += dL_dS[b] * S[b].d[k];
        grad8[k] = g;
    }
    if (smooth) for (int b = 0; b < nb; ++b) smooth[b] = S[b].v;
    if (m) {
        memset(m, 0, sizeof(*m));
        m->W = W.v; m->mean = mean.v; m->spread = spread.v; m->rel_spread = mom[3].v;
        m->div_x = mom[4].v; m->div_y = mom[5].v; m->div = mom[6].v; m->mean_aeff = mom[7].v;
        m->mean_gamma0 = mom[11].v;
    }
    free(all);
    free(S);
    return 0;
}

/* Plain (non-dual) smoothed spectrum, same definition as in qso_grad. */
int qso_smooth_spectrum(const qso_laser* L, const qso_beam* B, const qso_bins* bins,
                        double sigma_bins, int64_t n, const double* const* xi, const double* w,
                        double* S) {
    int nb = bins->n_bins;
    if (nb <= 0 || bins->log_spaced || !(sigma_bins > 0)) return 1;
    qso_sum* acc = (qso_sum*)calloc((size_t)nb, sizeof(qso_sum));
    if (!acc) return 1;
    double delta = (bins->hi - bins->lo) / (double)nb;
    double sig = sigma_bins * delta;
    double pref = delta / (sig * sqrt(2.0 * QSO_PI));
    for (int64_t i = 0; i < n; ++i) {
        double v[8];
        for (int k = 0; k < 8; ++k) v[k] = xi[k] ? xi[k][i] : 0.0;
        qso_sample s;
        qso_sample_eval(L, B, NULL, v, &s);
        double wi = w ? w[i] : 1.0;
        int k0, k1;
        qso_smooth_range(bins, sigma_bins, s.gamma_out, &k0, &k1);
        for (int k = k0; k <= k1; ++k) {
            double d = bins->lo + ((double)k + 0.5) * delta - s.gamma_out;
            qso_add(&acc[k], wi * pref * exp(-d * d / (2.0 * sig * sig)));
        }
    }
    for (int k = 0; k < nb; ++k) S[k] = qso_val(&acc[k]);
    free(acc);
    return 0;
}

/* ------------------------------------------------------------------------
 * Photon spectrum (Sec. 4): for every phase cell the electron's mean energy
 * mu_j and the field give chi_j; the quantum-synchrotron spectrum in the
 * locally-constant-field approximation at (mu_j, chi_j) is integrated over
 * the phase and summed over the beam.  The paper names the LCFA spectrum
 * without printing it; the standard form (Baier-Katkov / Ritus), per unit
 * time and photon energy fraction xi = eps/gamma (eps in m c^2):
 *   d2N/(dt dxi) = (alpha m c^2/(sqrt3 pi hbar gamma)) F(xi, chi),
 *   F = (1 - xi + 1/(1 - xi)) K_{2/3}(y) - Ki_{1/3}(y),
 *   y = 2 xi/(3 chi (1 - xi)),  Ki_{1/3}(y) = int_y^inf K_{1/3}(s) ds.
 * Per unit phase (head-on, the phase advances at 2 omega0, m c^2/(hbar
 * omega0) = a_S) and per unit eps:
 *   d2N/(dphi deps) = (alpha a_S/(2 sqrt3 pi mu^2)) F(eps/mu, chi),  eps < mu.
 * The output is the beam's photon number per unit eps at the bin centres,
 * S(eps_b) = sum_i w_i sum_j h d2N/(dphi deps)(eps_b; mu_ij, chi_ij).
 * ------------------------------------------------------------------------ */
#define QSO_ALPHA 7.2973525693e-3

/* K_{2/3}(y) and Ki_{1/3}(y) from
 *   K_nu(y) = int_0^inf exp(-y cosh t) cosh(nu t) dt,
 *   Ki_{1/3}(y) = int_0^inf exp(-y cosh t) cosh(t/3)/cosh(t) dt
 * (the second by integrating the first over y), trapezoidal rule in t with
 * step 1/32 until y cosh t > 800: the integrands are analytic in a strip
 * and decay doubly exponentially, so the rule converges geometrically. */
void qso_bessel_pair(double y, double* k23, double* ki13) {
    const double dt = 1.0 / 32.0;
    qso_sum a = {0.0, 0.0}, b = {0.0, 0.0};
    for (int k = 0;; ++k) {
        double t = k * dt, ch = cosh(t), e = exp(-y * ch);
        double wt = (k == 0) ? 0.5 : 1.0;
        qso_add(&a, wt * e * cosh(2.0 * t / 3.0));
        qso_add(&b, wt * e * cosh(t / 3.0) / ch);
        if (y * ch > 800.0 || t > 60.0) break;
    }
    *k23 = dt * qso_val(&a);
    *ki13 = dt * qso_val(&b);
}

/* d2N/(dphi deps) at photon energy eps for an electron of mean energy mu
   at chi (0 for eps <= 0, eps >= mu or chi <= 0). */
double qso_photon_rate(double aS, double mu, double chi, double eps) {
    if (!(eps > 0.0) || !(eps < mu) || !(chi > 0.0)) return 0.0;
    double xi = eps / mu;
    double y = 2.0 * xi / (3.0 * chi * (1.0 - xi));
    double k23, ki13;
    qso_bessel_pair(y, &k23, &ki13);
    double F = (1.0 - xi + 1.0 / (1.0 - xi)) * k23 - ki13;
    return QSO_ALPHA * aS / (2.0 * sqrt(3.0) * QSO_PI * mu * mu) * F;
}

/* Photon spectrum of the beam (quantum model; returns 1 for the classical
   model or invalid bins).  pb: n_bins, lo, hi, log_spaced of the photon
   energy axis (eps in m c^2); out: n_bins values at the bin centres. */
/* Photon divergence (Eq. 7): photons leave along the emitting electron's
   direction, which in cell j is its initial angle plus the transverse
   oscillation in the linearly polarised field (rms A_j/(sqrt2 mu_j) along x,
   the polarisation axis), within the emission cone ~1/mu_j per axis (the
   paper's "~1/gamma"); theta2 (optional, 2 x n_bins) receives
     T_x(eps_b) = sum_i w_i sum_j h rate_ij(eps_b) (thx0^2 + A_j^2/(2 mu_j^2) + 1/mu_j^2)
     T_y(eps_b) = sum_i w_i sum_j h rate_ij(eps_b) (thy0^2 + 1/mu_j^2)
   so that T/S is the mean square photon angle per axis at eps_b. */
int qso_photon_spectrum2(const qso_laser* L, const qso_beam* B, const qso_bins* pb, int64_t n,
                         const double* const* xi, const double* w, double* out, double* theta2);

int qso_photon_spectrum(const qso_laser* L, const qso_beam* B, const qso_bins* pb, int64_t n,
                        const double* const* xi, const double* w, double* out) {
    return qso_photon_spectrum2(L, B, pb, n, xi, w, out, NULL);
}

int qso_photon_spectrum2(const qso_laser* L, const qso_beam* B, const qso_bins* pb, int64_t n,
                         const double* const* xi, const double* w, double* out, double* theta2) {
    int nb = pb->n_bins, N = L->n_phase;
    if (L->model == 0 || nb <= 0 || !(pb->hi > pb->lo) || (pb->log_spaced && !(pb->lo > 0.0)))
        return 1;
    double c[10];
    qso_constants(L, c);
    double h = (c[8] - c[7]) / (double)N, aS = c[4];
    double* eps = (double*)malloc(sizeof(double) * (size_t)nb);
    double* mu_cell = (double*)malloc(sizeof(double) * (size_t)N);
    double* chi_cell = (double*)malloc(sizeof(double) * (size_t)N);
    qso_sum* acc = (qso_sum*)calloc((size_t)nb * 3, sizeof(qso_sum));
    if (!eps || !mu_cell || !chi_cell || !acc) return 1;
    for (int b = 0; b < nb; ++b)
        eps[b] = pb->log_spaced ? pb->lo * pow(pb->hi / pb->lo, (b + 0.5) / nb)
                                : pb->lo + (b + 0.5) * (pb->hi - pb->lo) / nb;
    for (int64_t i = 0; i < n; ++i) {
        double v[8];
        for (int k = 0; k < 8; ++k) v[k] = xi[k] ? xi[k][i] : 0.0;
        double wi = w ? w[i] : 1.0;
        if (!(wi >= 0.0) || !isfinite(wi) || wi == 0.0) continue;
        qso_sample s;
        qso_sample_eval_x(L, B, NULL, v, &s, mu_cell, chi_cell);
        if (!isfinite(s.mu)) continue;
        double thx0 = B->div_rad * v[4], thy0 = B->div_rad * v[5];
        for (int j = 0; j < N; ++j) {
            double mu = mu_cell[j], chi = chi_cell[j];
            /* A_j/mu_j from chi_j = sqrt2 mu_j A_j / a_S */
            double am = chi * aS / (sqrt(2.0) * mu * mu);
            double tx2 = thx0 * thx0 + 0.5 * am * am + 1.0 / (mu * mu);
            double ty2 = thy0 * thy0 + 1.0 / (mu * mu);
            for (int b = 0; b < nb; ++b) {
                double r = wi * h * qso_photon_rate(aS, mu, chi, eps[b]);
                qso_add(&acc[b], r);
                qso_add(&acc[nb + b], r * tx2);
                qso_add(&acc[2 * nb + b], r * ty2);
            }
        }
    }
    for (int b = 0; b < nb; ++b) out[b] = qso_val(&acc[b]);
    if (theta2)
        for (int b = 0; b < 2 * nb; ++b) theta2[b] = qso_val(&acc[nb + b]);
    free(eps); free(mu_cell); free(chi_cell); free(acc);
    return 0;
}

/* ------------------------------------------------------------------------
 * Plane-wave reconstruction (Eq. 5): the 3D spectrum of a beam is the sum
 * over a uniform set of effective amplitudes a_k of the plane-wave spectrum
 * at a_k weighted by the beam's a_eff distribution,
 *   out[s][b] = sum_k hist[s][k] pw[k][b]
 * (k ascending, compensated), for n_shots histograms at once.
 * ------------------------------------------------------------------------ */
void qso_pw_reconstruct(int n_shots, int n_a, int n_bins, const double* hist, const double* pw,
                        double* out) {
    for (int sh = 0; sh < n_shots; ++sh)
        for (int b = 0; b < n_bins; ++b) {
            qso_sum acc = {0.0, 0.0};
            for (int k = 0; k < n_a; ++k)
                qso_add(&acc, hist[(size_t)sh * n_a + k] * pw[(size_t)k * n_bins + b]);
            out[(size_t)sh * n_bins + b] = qso_val(&acc);
        }
}

/* ------------------------------------------------------------------------
 * Analytic distributions (Table 1, Table 2 via Eq. 6) for idealised beams,
 * evaluated on a grid.  Geometry: the collision plane sits at d_par from the
 * focal plane (z_R = pi W0^2/lambda, W = W0 sqrt(1 + d_par^2/z_R^2),
 * a_par = a0 W0/W); transverse offset d_perp of the beam centre from the
 * laser axis.
 *   short beam (all electrons in the collision plane, Gaussian transverse
 *     density ~ exp(-rho^2/R^2)): a = a_par exp(-rho'^2/W^2) with rho' the
 *     distance to the axis, whose square has the offset (Rice) distribution,
 *     so dN/da = N (W^2/R^2)(1/a)(a/a_par)^(W^2/R^2)
 *                  I0(2 (d_perp/R)(W/R) sqrt(ln(a_par/a))) exp(-d_perp^2/R^2),
 *     0 < a < a_par (the printed theta(a - a_par) read with its support the
 *     right way round);
 *   thin beam (on the axis, flat-top length L): collision positions uniform
 *     on [z-, z+], z+- = d_par +- L/4 (the crossing is at half the lag),
 *     a = a0/sqrt(1 + z^2/z_R^2), each root z = +-z_a, z_a = z_R
 *     sqrt(a0^2/a^2 - 1), inside [z-, z+] adds (2N z_R/L)(a0^2/a^2)/
 *     sqrt(a0^2 - a^2);
 *   wide beam (uniform density n_b across the laser, flat-top length L):
 *     per collision plane z the area where a_eff > a grows as pi W0^2 q
 *     ln(...), so dN/da = (2 pi n_b W0^2/a) int q(z) dz over [z-, z+]
 *     clipped to |z| < z_a, q = 1 + z^2/z_R^2 (the factor 2: unit length
 *     of beam is half a unit of collision position).
 * Classical spectrum: gamma_f(a) = gamma0/(1 + c_RR gamma0 a^2) (Eq. 3) is
 * monotone, so dN/dgamma = (dN/da)(a(gamma)) / (2 a c_RR gamma^2) with
 * a(gamma) = sqrt((gamma0 - gamma)/(c_RR gamma0 gamma)).
 * geom: 0 short, 1 thin, 2 wide; par: radius R, length L, d_perp, d_par,
 * N (or n_b for the wide beam).
 * ------------------------------------------------------------------------ */

/* I0 by its power series (x <= 30) or its asymptotic expansion. */
double qso_bessel_i0(double x) {
    x = fabs(x);
    if (x <= 30.0) {
        double t = 1.0, s = 1.0, q = 0.25 * x * x;
        for (int k = 1; k < 200; ++k) {
            t *= q / ((double)k * k);
            s += t;
            if (t < 1e-17 * s) break;
        }
        return s;
    }
    double y = 1.0 / (8.0 * x), t = 1.0, s = 1.0;
    for (int k = 1; k < 30; ++k) {
        t *= (2.0 * k - 1.0) * (2.0 * k - 1.0) * y / k;
        s += t;
        if (fabs(t) < 1e-17) break;
    }
    return exp(x) / sqrt(2.0 * QSO_PI * x) * s;
}

static double qso_aeff_density(const qso_laser* L, int geom, const double* par, double a) {
    double c[10];
    qso_constants(L, c);
    double zR = c[2], a0 = L->a0, W0 = L->w0_um;
    double R = par[0], Lb = par[1], dperp = par[2], dpar = par[3], nb = par[4];
    if (!(a > 0.0)) return 0.0;
    if (geom == 0) {
        double W = W0 * sqrt(1.0 + dpar * dpar / (zR * zR)), apar = a0 * W0 / W;
        if (!(a < apar)) return 0.0;
        double k = W * W / (R * R);
        return nb * k / a * pow(a / apar, k) *
               qso_bessel_i0(2.0 * (dperp / R) * (W / R) * sqrt(log(apar / a))) *
               exp(-dperp * dperp / (R * R));
    }
    if (!(a < a0)) return 0.0;
    double za = zR * sqrt(a0 * a0 / (a * a) - 1.0);
    double zm = dpar - Lb / 4.0, zp = dpar + Lb / 4.0;
    if (geom == 1) {
        int roots = (za >= zm && za <= zp) + (-za >= zm && -za <= zp);
        return roots * (2.0 * nb * zR / Lb) * (a0 * a0 / (a * a)) / sqrt(a0 * a0 - a * a);
    }
    double lo = zm > -za ? zm : -za, hi = zp < za ? zp : za;
    if (!(hi > lo)) return 0.0;
    double Fh = hi * (1.0 + hi * hi / (3.0 * zR * zR)), Fl = lo * (1.0 + lo * lo / (3.0 * zR * zR));
    return 2.0 * QSO_PI * nb * W0 * W0 / a * (Fh - Fl);
}

void qso_analytic_aeff(const qso_laser* L, int geom, const double* par, int n, const double* a,
                       double* out) {
    for (int i = 0; i < n; ++i) out[i] = qso_aeff_density(L, geom, par, a[i]);
}

void qso_analytic_ll(const qso_laser* L, int geom, const double* par, double gamma0, int n,
                     const double* g, double* out) {
    double c[10];
    qso_constants(L, c);
    double cRR = c[9];
    for (int i = 0; i < n; ++i) {
        double gm = g[i];
        out[i] = 0.0;
        if (!(gm > 0.0) || !(gm < gamma0)) continue;
        double a = sqrt((gamma0 - gm) / (cRR * gamma0 * gm));
        out[i] = qso_aeff_density(L, geom, par, a) / (2.0 * a * cRR * gm * gm);
    }
}

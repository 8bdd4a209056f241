/*
 * qscatter.h -- C ABI of libqscatter, a GB300 (sm_103a) implementation of
 * the beam phase-space integration of QScatter (Amaro & Vranic,
 * arXiv 2308.09348): for every electron-beam sample, the local
 * Gaussian-focus field it crosses (Sec. 2, Eqs. 1-2), its final energy from
 * the classical Landau-Lifshitz closed form (Eq. 3) or from the
 * quantum-corrected Fokker-Planck mean/variance phase integration (Eq. 6 and
 * the Fokker-Planck regime of Sec. 1), its final divergence (Eq. 8), then the
 * weighted reduction into spectra (Eq. 4 as a histogram, Eq. 1 as the a_eff
 * histogram) and moments (mean energy, energy spread, divergence).
 *
 * Conventions shared by every entry point
 *  - Units: lengths in micrometres, times in femtoseconds, energies as the
 *    Lorentz factor gamma, angles in radians.
 *  - Pointers named d_* are DEVICE pointers (any CUDA allocation on the
 *    current device); descriptor structs (qs_laser, ...) are HOST pointers
 *    read during the call only.
 *  - Ownership: the caller owns every buffer.  The library allocates no
 *    memory and keeps no per-call state; scratch space is the caller's
 *    workspace (size from qs_workspace_bytes, 256-byte aligned).
 *  - Execution: asynchronous on the given CUDA stream (cudaStream_t passed
 *    as void*; NULL = legacy default stream).  Outputs are valid once the
 *    stream reaches the point of the call.  Calls that share a workspace
 *    must be ordered on one stream.
 *  - Errors: arguments are validated on the host before any launch; on a
 *    non-QS_OK return nothing has been launched and no output was written
 *    (QS_ERR_CUDA: a launch failed; outputs are then undefined).
 *  - Determinism: histograms accumulate in integers (exact, order-free);
 *    moments are reduced in a fixed order for a given device and
 *    qs_exec; repeated calls give bit-identical results.
 */
#ifndef QSCATTER_H
#define QSCATTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QS_VERSION 10

/*
 * Status codes.  QS_ERR_NONFINITE is returned only when the caller asks for
 * the check (QS_EXEC_CHECK_FINITE in qs_exec.flags): the outputs are then
 * complete and valid for the samples that entered them, and the status says
 * that moments.nonfinite > 0 samples were left out.  QS_ERR_TIMEOUT is
 * reserved: no kernel of this version waits on another CTA, stream or
 * device, so no entry point returns it.
 */
typedef enum {
    QS_OK = 0,
    QS_ERR_INVALID_ARG = 1,   /* a descriptor or pointer failed validation   */
    QS_ERR_CUDA = 2,          /* a CUDA runtime call or launch failed        */
    QS_ERR_WORKSPACE = 3,     /* workspace missing, too small or misaligned  */
    QS_ERR_UNSUPPORTED = 4,   /* valid request this build does not support   */
    QS_ERR_TIMEOUT = 5,       /* reserved: a bounded device-side wait gave up */
    QS_ERR_NONFINITE = 6      /* samples were excluded as non-finite (checked
                                 on request, outputs written)                */
} qs_status;

typedef enum { QS_ENV_GAUSS = 0, QS_ENV_SIN2 = 1 } qs_envelope;
typedef enum { QS_MODEL_LL = 0, QS_MODEL_QFP = 1 } qs_model;
typedef enum { QS_VARIANT_CELL_FOCUS = 1, QS_VARIANT_CYCLE_CHI = 2 } qs_variant;
typedef enum { QS_F32 = 0, QS_F64 = 1 } qs_dtype;

/*
 * Laser (Sec. 2 Eq. 2; Eq. 3; Sec. 4; Appendix A).  The laser moves along +z
 * with its focus at the origin; its pulse peak passes z = 0 at t = delay_fs.
 *   lambda_um      central wavelength (> 0)
 *   a0             peak normalised vector potential (>= 0)
 *   w0_um          focal spot size W0 of Eq. 2 (> 0); z_R = pi W0^2/lambda
 *   tau_fs         intensity FWHM duration (> 0)
 *   dx_um, dy_um   position of the laser axis (transverse misalignment)
 *   delay_fs       temporal misalignment
 *   div_prefactor  kappa, the multiplicative prefactor of Eq. 8 (>= 0)
 *   envelope       QS_ENV_GAUSS: field envelope exp(-2 ln2 (phi/Phi)^2),
 *                  Phi = omega0 tau, phase window [-2.5 Phi, 2.5 Phi];
 *                  QS_ENV_SIN2: field envelope sin^2(pi phi/Phi_T) on
 *                  [0, Phi_T], Phi_T chosen so the intensity FWHM is Phi
 *   model          QS_MODEL_LL (Eq. 3) or QS_MODEL_QFP (Eq. 6 + FP closure)
 *   n_phase        phase cells of the integration, 1..4096 (ignored by LL
 *                  without QS_VARIANT_CELL_FOCUS)
 *   variant        bit flags, 0 = the paper's model as read here:
 *                  QS_VARIANT_CELL_FOCUS: Eq. 2 evaluated in every phase
 *                  cell at the electron's position there, instead of once
 *                  where it crosses the pulse peak (the paper neglects the
 *                  focus variation during the crossing, Sec. 2).  In cell j at phase
 *                  phi_j (0 at the crossing) the electron has moved by
 *                  s_j = phi_j/(2k) along -z (it meets the counter-moving
 *                  phase at twice the frequency), so z_j = z* - s_j and the
 *                  transverse offsets grow by theta s_j; the local peak is
 *                  a_j = a0 q_j^-1/2 exp(-rho_j^2/(W0^2 q_j)) and the field
 *                  envelope A_j = a_j G(phi_j).  LL then integrates Eq. 3's
 *                  exponent cell by cell: 1/gamma_f = 1/gamma0 +
 *                  (2/3) R_c h sum_j A_j^2.  a_eff (its histogram, its
 *                  moment and Eq. 8) stays the value at the crossing.
 *                  QS_VARIANT_CYCLE_CHI (quantum model): the Gaunt factor
 *                  and the diffusion factor averaged over the laser cycle
 *                  of a linearly polarised field, chi(psi) = sqrt2 chi
 *                  |cos psi| with chi the value at the rms field, instead
 *                  of taken at the rms field: g -> G(chi) =
 *                  <2 cos^2 psi g(chi(psi))>, 2g + chi g' -> 2G + chi G',
 *                  h -> H(chi) = <2 sqrt2 |cos psi|^3 h(chi(psi))> (Eq. 6
 *                  written for the instantaneous field).
 *                  Every entry point takes every variant (the adjoint
 *                  carries its tangents).  QS_VARIANT_CYCLE_CHI reads
 *                  device tables of G and H that the first call using
 *                  them on a device (context) builds: one launch and a
 *                  wait, so make that call before any stream capture
 *                  (what a capturing first call does is stated per entry
 *                  point).
 */
typedef struct qs_laser {
    double lambda_um, a0, w0_um, tau_fs;
    double dx_um, dy_um, delay_fs, div_prefactor;
    int32_t envelope, model, n_phase, variant;
} qs_laser;

/*
 * Electron beam (Sec. 1: broadband beams and divergence; each sample is a
 * weighted volume element of the beam, as in Eq. 1).  A sample with
 * variates xi[0..7] decodes to
 *   x = dx_um + sigma_x_um xi0,  y = dy_um + sigma_y_um xi1,  z = sigma_z_um xi2
 *   gamma0 = gamma_mean (1 + rel_spread xi3)            (flat_energy == 0)
 *          = gamma_lo + (gamma_hi - gamma_lo) xi3        (flat_energy != 0)
 *   gamma0 is clamped to >= 1
 *   theta_x = div_rad xi4, theta_y = div_rad xi5
 * (x, y, z) is the position at t = 0; the velocity is c(theta_x, theta_y, -1).
 */
typedef struct qs_beam {
    double gamma_mean, rel_spread, gamma_lo, gamma_hi;
    double sigma_x_um, sigma_y_um, sigma_z_um, div_rad, dx_um, dy_um;
    int32_t flat_energy, reserved;
} qs_beam;

/*
 * Samples: structure of arrays on the device.  xi[k] holds n elements of
 * dtype (QS_F32 or QS_F64) each; xi[0..3] are required when n > 0, a NULL
 * xi[4..7] reads as zeros.  xi[6] (angular noise) and xi[7] (energy noise)
 * are only read by the QFP model.  w: n per-sample weights (>= 0, finite) of
 * the same dtype, or NULL for unit weights.  Pointers must be aligned to the
 * element size; 16-byte alignment enables vector loads.
 */
typedef struct qs_samples {
    int64_t n;
    const void* xi[8];
    const void* w;
    int32_t dtype, reserved;
} qs_samples;

/*
 * Binning (Eq. 4 as a weighted histogram; Eq. 1 as the a_eff histogram).
 *   Energy spectrum of the realised final energy gamma_out over [lo, hi):
 *   n_bins bins (0 = off); uniform, or log-spaced (log_spaced != 0, lo > 0).
 *   Bins are half-open; below lo goes to 'under', at or above hi to 'over'.
 *   Divergence map over [-theta_max, theta_max)^2 of (theta_x, theta_y),
 *   n_tx x n_ty bins, row-major [iy][ix] (0 = off).
 *   a_eff histogram over [0, aeff_max), n_aeff bins (0 = off).
 *   Kernel-smoothed spectrum (smooth_sigma_bins > 0, uniform energy bins
 *   only): each sample deposits its weight as a Gaussian of standard
 *   deviation smooth_sigma_bins bin widths centred on its realised energy,
 *   sampled at the bin centres and cut at 6 standard deviations:
 *     S_k = sum_i w_i exp(-(k + 1/2 - t_i)^2 / (2 s^2)) / (s sqrt(2 pi)),
 *     t_i = (gamma_out_i - lo) n_bins / (hi - lo),  s = smooth_sigma_bins.
 *   It is the differentiable stand-in for the histogram in fitting losses
 *   (Sec. 6: reconstruction of experimental parameters).
 * Entries are bin masses (sums of weights), not densities.
 */
typedef struct qs_bins {
    int32_t n_bins, log_spaced;
    double lo, hi;
    int32_t n_tx, n_ty;
    double theta_max;
    int32_t n_aeff, reserved;
    double aeff_max;
    double smooth_sigma_bins;
} qs_bins;

/*
 * Moments (observables of Sec. 1 and Sec. 5): written to device memory.
 *   W            total weight
 *   mean         <gamma_f> (weighted mean of the per-sample means)
 *   spread       sqrt(<(mu - mean)^2> + <V>)  (law of total variance)
 *   rel_spread   spread / mean
 *   div_x        sqrt(<theta_x0^2 + theta_e^2>), theta_e the Eq. 8 broadening
 *   div_y        sqrt(<theta_y0^2>),  div = sqrt(div_x^2 + div_y^2)
 *   mean_aeff    <a_eff>,  mean_gamma0  <gamma0>
 *   under, over  spectrum weight below lo / at or above hi
 *   map_out      weight outside the divergence map
 *   nonfinite    NUMBER of samples excluded from every other output because
 *                their weight was negative or not finite, or their result
 *                was not finite
 * With W == 0 every field is 0.
 */
typedef struct qs_moments {
    double W, mean, spread, rel_spread, div_x, div_y, div, mean_aeff;
    double under, over, map_out, mean_gamma0, nonfinite;
} qs_moments;

/*
 * Execution options (NULL = defaults).
 *   precision         QS_F32: per-sample arithmetic in FP32 (the quantum
 *                     model's final energy recombined as a float pair, ~2^-44
 *                     relative; per-thread moment sums compensated in FP32,
 *                     reduction trees in float pairs, each CTA's slot in
 *                     FP64); QS_F64: everything in FP64.
 *   weight_frac_bits  fixed-point fraction bits of the weighted histograms
 *                     (0 = 32).  Each weight is rounded to a multiple of
 *                     2^-bits; every bin must stay below 2^(63-bits).
 *   block, grid       launch shape of the evaluation kernel (0 = chosen by the
 *                     library: for the FP32 paths one CTA per SM, 896
 *                     threads (quantum model, per-cell focus) or 768
 *                     (cycle-resolved chi, classical model); 256 threads
 *                     elsewhere; the grid
 *                     sized to the resident CTAs).  A caller's block is
 *                     32..512, a multiple of 32.
 *   tile              samples per work item of qs_scatter_batch (0 = 2048)
 *                     and of qs_scatter_grad_batch (0 = the largest power of
 *                     two up to 8192 that leaves at least sixteen work items
 *                     per resident CTA); a multiple of 64, at most 1<<20;
 *                     ignored elsewhere.
 *   flags             QS_EXEC_CHECK_FINITE: after the outputs are written
 *                     the call waits for its stream, reads the excluded-sample
 *                     count(s) and returns QS_ERR_NONFINITE if any sample (of
 *                     any shot) was left out as non-finite or negatively
 *                     weighted.  The call is then synchronous; requested while
 *                     the stream is being captured into a graph it returns
 *                     QS_ERR_UNSUPPORTED before any launch.  Honoured by
 *                     qs_scatter, qs_scatter_noalloc, qs_scatter_host and
 *                     qs_scatter_batch; other bits are invalid.
 *   ev_start, ev_stop optional cudaEvent_t handles (as void*): when set, they
 *                     are recorded on the call's stream immediately before and
 *                     after the evaluation kernel, so a caller can time that
 *                     kernel alone.  The caller creates and owns the events.
 */
#define QS_EXEC_CHECK_FINITE 1

typedef struct qs_exec {
    int32_t precision, weight_frac_bits, block, grid;
    int32_t tile, flags;
    void* ev_start;
    void* ev_stop;
} qs_exec;

/*
 * Per-sample records of qs_eval_samples: device arrays of n elements, any
 * may be NULL.  bin: energy bin, -1 under, n_bins over; ix/iy: map cell or
 * -1 outside; abin: a_eff bin or n_aeff above.
 */
typedef struct qs_sample_out {
    double *gamma0, *aeff, *mu, *V, *theta_e, *theta_x, *theta_y, *gamma_out;
    int32_t *bin, *ix, *iy, *abin;
} qs_sample_out;

/* Version of this ABI (QS_VERSION). */
int32_t qs_version(void);

/* Static message for a status code. */
const char* qs_status_string(int32_t status);

/* Workspace bytes that qs_scatter needs for these bins, options and sample
   count on the current device (0 if the arguments are invalid). */
size_t qs_workspace_bytes(const qs_bins* bins, const qs_exec* exec, int64_t n_samples);

/*
 * qs_scatter: integrate the per-particle energy-loss model over the beam's
 * phase space and reduce into spectra and moments (Sec. 2-5; Eqs. 1-4, 6, 8).
 *   d_spectrum   n_bins doubles (required if n_bins > 0)
 *   d_divmap     n_ty*n_tx doubles (required if the map is on)
 *   d_aeff_hist  n_aeff doubles (required if n_aeff > 0)
 *   d_spec_smooth n_bins doubles (required if smooth_sigma_bins > 0)
 *   d_moments    one qs_moments in device memory (required)
 *   d_workspace  ws_bytes >= qs_workspace_bytes(...), 256-byte aligned
 */
int32_t qs_scatter(const qs_laser* laser, const qs_beam* beam, const qs_samples* samples,
                   const qs_bins* bins, const qs_exec* exec, double* d_spectrum,
                   double* d_divmap, double* d_aeff_hist, double* d_spec_smooth,
                   qs_moments* d_moments,
                   void* d_workspace, size_t ws_bytes, void* stream);

/*
 * qs_eval_samples: the per-sample part of qs_scatter (decode, collision
 * geometry, Eq. 2, Eq. 3 or the QFP integration, Eq. 8, bin indices) with
 * every intermediate written out, for inspection and element-wise checks.
 * bins may be NULL (bin fields then read -1).  No workspace.
 */
int32_t qs_eval_samples(const qs_laser* laser, const qs_beam* beam, const qs_samples* samples,
                        const qs_bins* bins, const qs_exec* exec, const qs_sample_out* out,
                        void* stream);

/*
 * qs_scatter_host: qs_scatter for samples in HOST memory.  The samples are
 * streamed to the device in chunks of `chunk` samples through two staging
 * buffers in the workspace: the copy of chunk c+1 runs on an internal copy
 * stream while chunk c is evaluated on `stream`, so the host-to-device
 * transfer hides behind the computation.  Outputs are written to HOST
 * memory when the stream reaches the end of the call (pinned host memory
 * for every host buffer gives asynchronous copies; pageable memory works
 * but serialises the copies).  Results equal qs_scatter's: identical
 * histograms, moments up to the order of the reduction.
 *   h_samples   qs_samples whose xi[] and w point to host memory
 *   chunk       samples per chunk, a positive multiple of 1024; or 0: chunks
 *               of whole waves of the FP32 launch (1792 samples per SM), the
 *               first one wave and each next three times the last, up to
 *               2^23 samples, so that the first copy is short
 *   h_*         host output buffers (same sizes and rules as qs_scatter)
 *   d_workspace qs_host_workspace_bytes(...) bytes of device memory
 * The first call on a device creates one copy stream and five events that
 * are kept until the process exits (no device memory is allocated).
 */
size_t qs_host_workspace_bytes(const qs_bins* bins, const qs_exec* exec, const qs_samples* h_samples,
                               int64_t chunk);

int32_t qs_scatter_host(const qs_laser* laser, const qs_beam* beam, const qs_samples* h_samples,
                        const qs_bins* bins, const qs_exec* exec, int64_t chunk,
                        double* h_spectrum, double* h_divmap, double* h_aeff_hist,
                        double* h_spec_smooth, qs_moments* h_moments, void* d_workspace,
                        size_t ws_bytes, void* stream);

/*
 * Batched shots (the paper's parallel plane-wave runs, Sec. 3.2, and the
 * high-repetition-rate data sets of Sec. 6): n_shots independent
 * integrations, each with its own laser and beam, in one persistent launch.
 * Shot s owns samples [offsets[s], offsets[s+1]) of one concatenated
 * structure of arrays.  Work items are tiles of exec->tile samples of one
 * shot, pulled from a device counter; each tile's moment partials go to a
 * slot of its own and are reduced per shot in tile order, so results do not
 * depend on scheduling (repeated calls are bit-identical).
 *   d_lasers, d_beams n_shots descriptors in DEVICE memory (validated on the
 *                 device; an invalid shot, or one with n_phase > max_phase,
 *                 gets W = 0 and nonfinite = -1 and no work)
 *   d_offsets     n_shots + 1 non-decreasing int64 (device), offsets[0] >= 0,
 *                 offsets[n_shots] <= samples->n, checked on the device: a
 *                 shot whose range leaves [0, samples->n] is invalid, and
 *                 offsets that decrease anywhere make EVERY shot invalid
 *                 (no shot then does any work); or NULL: every shot
 *                 integrates ALL samples (a parameter sweep, e.g. over the
 *                 delay, on one sampled beam)
 *   samples       the concatenated streams (as for qs_scatter)
 *   bins          energy spectrum, with smooth_sigma_bins > 0 the
 *                 kernel-smoothed spectrum, with n_tx > 0 the divergence map
 *                 and with n_aeff > 0 the a_eff histogram of every shot;
 *                 shared bin counts and map extent, energy range per shot
 *                 from d_ranges if not NULL (n_shots pairs {lo, hi}, device)
 *                 else bins->lo/hi
 *   max_phase     upper bound of the n_phase of the shots that use phase
 *                 cells (QS_MODEL_QFP or QS_VARIANT_CELL_FOCUS), 1..4096
 *   d_spectra     n_shots x n_bins doubles (row per shot), or NULL if n_bins == 0
 *   d_spec_smooth n_shots x n_bins doubles (row per shot) when
 *                 smooth_sigma_bins > 0, else ignored (may be NULL)
 *   d_divmaps     n_shots x n_tx x n_ty doubles (map of shot s at offset
 *                 s n_tx n_ty, layout as qs_scatter's) when n_tx > 0, else
 *                 ignored (may be NULL); the weight outside shot s's map in
 *                 its moments' map_out
 *   d_aeff_hists  n_shots x n_aeff doubles (row per shot) when n_aeff > 0,
 *                 else ignored (may be NULL)
 *   d_moments     n_shots qs_moments
 * The workspace size (qs_batch_workspace_bytes) depends on shared_samples:
 * nonzero for the sweep form (d_offsets == NULL), whose tile slots grow with
 * n_shots x n_total / tile.  The maps and a_eff histograms are accumulated in
 * the workspace (8 bytes per bin and shot: 537 MB for 4096 shots of a
 * 128 x 128 map) with global integer atomics; the energy spectrum per tile in
 * shared memory.
 * Shots may mix the models and the variants; shots with a variant run in a
 * second persistent launch over the same (shot, tile) schedule.  The call
 * is a fixed sequence of two memsets and six kernels on the stream and
 * contains no host synchronisation, except that the first call on a device
 * (context) builds the QS_VARIANT_CYCLE_CHI tables (one launch and a wait);
 * a first call made while the stream is being captured skips them, and its
 * QS_VARIANT_CYCLE_CHI shots are invalid (W = 0, nonfinite = -1).
 */
size_t qs_batch_workspace_bytes(int32_t n_shots, int64_t n_total, const qs_bins* bins,
                                int32_t max_phase, const qs_exec* exec, int32_t shared_samples);

int32_t qs_scatter_batch(int32_t n_shots, const qs_laser* d_lasers, const qs_beam* d_beams,
                         const int64_t* d_offsets, const qs_samples* samples,
                         const qs_bins* bins, const double* d_ranges, int32_t max_phase,
                         const qs_exec* exec, double* d_spectra, double* d_spec_smooth,
                         double* d_divmaps, double* d_aeff_hists, qs_moments* d_moments,
                         void* d_workspace, size_t ws_bytes, void* stream);

/*
 * Parameter order of qs_scatter_grad (the reconstruction use of Sec. 6):
 * laser a0, laser w0_um, laser dx_um, laser dy_um, laser delay_fs,
 * beam gamma_mean, beam rel_spread, beam div_rad.
 */
enum { QS_G_A0 = 0, QS_G_W0, QS_G_DX, QS_G_DY, QS_G_DELAY, QS_G_GAMMA, QS_G_SPREAD, QS_G_DIV,
       QS_NUM_GRAD };

/*
 * qs_scatter_grad: gradient of a loss L with respect to the 8 parameters
 * above, given the upstream gradient of L with respect to the outputs of
 * qs_scatter (adjoint of Eqs. 2, 3, 6, 8 and of the moment and smoothed-
 * spectrum reductions).  Every sample's forward evaluation is recomputed
 * with tangents carried through the discretised phase integration -- the
 * exact derivative of the discrete scheme -- and nothing per sample is
 * stored between the forward and this call: two tangents (d/d a_eff,
 * d/d gamma0) for variant 0 and QS_VARIANT_CYCLE_CHI (whose Gaunt and
 * diffusion factors carry their chi-derivatives); seven under
 * QS_VARIANT_CELL_FOCUS, whose per-cell amplitudes depend on the laser's
 * parameters individually (d/d ln a0, W0, dx, dy, delay, divergence,
 * gamma0).  A QS_VARIANT_CYCLE_CHI call made while the stream is being
 * captured, before the tables exist on the device, returns
 * QS_ERR_UNSUPPORTED before any launch.
 *   d_moments     the forward qs_moments of the same call (device)
 *   d_dL_dmoments 13 doubles (device), dL/d(each qs_moments field) in field
 *                 order; W, under, over, map_out and nonfinite do not
 *                 depend on the parameters and are ignored
 *   d_dL_dsmooth  n_bins doubles (device) dL/dS_k of the smoothed spectrum,
 *                 or NULL (then smooth_sigma_bins is not needed)
 *   d_grad8       QS_NUM_GRAD doubles (device), written (not accumulated)
 *   d_workspace   as for qs_scatter (qs_workspace_bytes)
 * Samples at the gamma0 >= 1 clamp contribute no energy-parameter gradient.
 * The reduction is in a fixed order: repeated calls are bit-identical.
 */
int32_t qs_scatter_grad(const qs_laser* laser, const qs_beam* beam, const qs_samples* samples,
                        const qs_bins* bins, const qs_exec* exec, const qs_moments* d_moments,
                        const double* d_dL_dmoments, const double* d_dL_dsmooth,
                        double* d_grad8, void* d_workspace, size_t ws_bytes, void* stream);

/*
 * qs_scatter_grad_batch: qs_scatter_grad for every shot of a batch at once
 * (the reconstruction of Sec. 6 over many shots: a gradient fit of each
 * shot's parameters), over the same persistent (shot, tile) schedule as
 * qs_scatter_batch.  Arguments as for qs_scatter_batch (the same workspace,
 * qs_batch_workspace_bytes, serves both; its forward results are not
 * needed), plus, per shot s, in device memory:
 *   d_moments     n_shots forward qs_moments (from qs_scatter_batch)
 *   d_dL_dmoments n_shots x 13 doubles, dL/d(each qs_moments field) of shot s
 *                 in row s (W, under, over, map_out, nonfinite ignored)
 *   d_dL_dsmooth  n_shots x n_bins doubles, dL/d(smoothed spectrum) of shot
 *                 s in row s, or NULL
 *   d_grad        n_shots x QS_NUM_GRAD doubles, written (not accumulated),
 *                 row s the gradient with respect to shot s's parameters
 * Shot s's gradient equals qs_scatter_grad's for that shot alone, up to the
 * order of the reduction (tiles in order, then summed per shot); repeated
 * calls are bit-identical.  Invalid shots (as flagged by qs_scatter_batch)
 * get zeros.  Shots may mix the models and the variants, as in
 * qs_scatter_batch.
 */
int32_t qs_scatter_grad_batch(int32_t n_shots, const qs_laser* d_lasers, const qs_beam* d_beams,
                              const int64_t* d_offsets, const qs_samples* samples,
                              const qs_bins* bins, const double* d_ranges, int32_t max_phase,
                              const qs_exec* exec, const qs_moments* d_moments,
                              const double* d_dL_dmoments, const double* d_dL_dsmooth,
                              double* d_grad, void* d_workspace, size_t ws_bytes, void* stream);

/*
 * qs_scatter_noalloc: qs_scatter for callers that cannot allocate device
 * memory -- plugins and embedded components running inside a host
 * application that owns every device allocation (a fixed pool, or no
 * allocator handle at all), so neither they nor the library may call
 * cudaMalloc.  The paper has no counterpart; this is a library convenience.
 *
 * Same arguments, validation and results as qs_scatter, minus the
 * workspace: the scratch space (integer histogram accumulators and per-CTA
 * moment partials) is a file-scope device array of QS_NOALLOC_SCRATCH_BYTES
 * bytes that every GPU which loads the library holds until the process exits.
 *   - Limit: a request whose scratch (qs_workspace_bytes of the same bins
 *     and options) exceeds QS_NOALLOC_SCRATCH_BYTES returns QS_ERR_WORKSPACE
 *     before any launch.
 *   - Set-up: the first call on each device looks up the array's device
 *     address (cudaGetSymbolAddress) with that device current; make that
 *     first call before any stream capture.
 *   - Sharing: all calls on a device share the one array; each call clears
 *     the accumulators it uses before its kernels run.  Calls whose kernels
 *     overlap on the GPU (different streams, or different host threads
 *     without ordering) race on the array and corrupt each other's results:
 *     order them on one stream.
 *   - The library calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define QS_NOALLOC_SCRATCH_BYTES ((size_t)1 << 20)

int32_t qs_scatter_noalloc(const qs_laser* laser, const qs_beam* beam,
                           const qs_samples* samples, const qs_bins* bins, const qs_exec* exec,
                           double* d_spectrum, double* d_divmap, double* d_aeff_hist,
                           double* d_spec_smooth, qs_moments* d_moments, void* stream);

/*
 * qs_photon_spectrum: photon spectrum of the beam (Sec. 4: the cumulative
 * spectrum from the mean energy along the phase and the local field).  In
 * every phase cell j of the quantum model (QS_MODEL_QFP; variant 0 or
 * QS_VARIANT_CELL_FOCUS) the electron's mean energy mu_j at the cell midpoint
 * (the state the cell's rates use) and chi_j give the quantum-synchrotron
 * emission of a locally constant field, which the paper names; its standard
 * (Baier-Katkov / Ritus) form per unit phase (head-on: the phase advances at
 * 2 omega0, and m c^2/(hbar omega0) = a_S) and photon energy eps (m c^2):
 *   d2N/(dphi deps) = alpha a_S / (2 sqrt3 pi mu^2) F(eps/mu, chi),  eps < mu,
 *   F(xi, chi) = (1 - xi + 1/(1 - xi)) K_{2/3}(y) - int_y^inf K_{1/3}(s) ds,
 *   y = 2 xi / (3 chi (1 - xi)).
 * Output: the beam's photon number per unit eps at the bin centres,
 *   S(eps_b) = sum_i w_i sum_j h d2N/(dphi deps)(eps_b; mu_ij, chi_ij),
 * into d_spectrum (device, pbins->n_bins doubles).  pbins: n_bins 1..512,
 * 0 <= lo < hi (lo > 0 when log_spaced); its map, a_eff and smoothing
 * fields are ignored.  Photons with y > 60 (relative weight e^-60) are
 * dropped.  FP64: the Bessel functions from their integral representations
 * (slow: for checks); FP32: cubic Hermite tables of K e^y in log y (relative
 * error ~3e-7), built on the device by the first FP32 call on that device
 * (one launch and a wait: make that call before any stream capture; a
 * capturing first call returns QS_ERR_UNSUPPORTED).  Sums are in a fixed
 * order (repeatable bit for bit).  Workspace: qs_photon_workspace_bytes.
 * Photon divergence (Eq. 7): d_theta2 (optional, device, 2 x n_bins doubles,
 * n_bins <= 256 when given) receives the same sums weighted by the photon's
 * mean square angle per axis, photons leaving along the emitting electron:
 *   x (polarisation): thx0^2 + A_j^2/(2 mu_j^2) + 1/mu_j^2,   y: thy0^2 + 1/mu_j^2
 * (initial angle, the rms transverse oscillation in the linearly polarised
 * field, the emission cone ~1/gamma the paper names); sum_b T_x/sum_b S over
 * the bins above a threshold is the mean square photon angle there.
 * Errors: QS_ERR_INVALID_ARG (descriptors, the classical model),
 * QS_ERR_UNSUPPORTED (QS_VARIANT_CYCLE_CHI), QS_ERR_WORKSPACE, QS_ERR_CUDA.
 */
size_t qs_photon_workspace_bytes(const qs_bins* pbins, const qs_exec* exec, int64_t n);

int32_t qs_photon_spectrum(const qs_laser* laser, const qs_beam* beam,
                           const qs_samples* samples, const qs_bins* pbins,
                           const qs_exec* exec, double* d_spectrum, double* d_theta2,
                           void* d_workspace, size_t ws_bytes, void* stream);

/*
 * qs_pw_reconstruct: plane-wave reconstruction, Eq. 5 (Sec. 3.2): the 3D
 * spectrum of a beam is the sum, over a uniform set of effective amplitudes
 * a_k, of the plane-wave spectrum at a_k weighted by the beam's a_eff
 * distribution:
 *   d_out[s][b] = sum_k d_hist[s][k] d_pw[k][b],   k ascending,
 * for n_shots beams at once.  d_hist: n_shots x n_a doubles (e.g. the a_eff
 * histograms of qs_scatter, a_k the bin centres); d_pw: n_a x n_bins doubles
 * (plane-wave spectra per unit weight at the a_k, e.g. from a qs_scatter_batch
 * sweep with a0 = a_k over a beam of zero size at the focus); d_out:
 * n_shots x n_bins doubles.  All device pointers, row-major.  FP64 sums in a
 * fixed order.  n_shots <= 524280.  Errors: QS_ERR_INVALID_ARG, QS_ERR_CUDA.
 */
int32_t qs_pw_reconstruct(int32_t n_shots, int32_t n_a, int32_t n_bins, const double* d_hist,
                          const double* d_pw, double* d_out, void* stream);

/*
 * Analytic fast path (Table 1; Table 2 via Eq. 6): distributions of
 * idealised beams evaluated on a grid, as a cross-check of the Monte Carlo
 * integration.  Geometry (qs_geometry): the collision centre sits d_par_um
 * from the focal plane (W = W0 sqrt(1 + d_par^2/z_R^2), z_R = pi W0^2/lambda,
 * a_par = a0 W0/W) and d_perp_um from the laser axis;
 *   QS_GEOM_SHORT  all electrons in the collision plane, transverse density
 *                  ~ exp(-rho^2/R^2), R = radius_um (R = sqrt2 sigma), count
 *                  = N:  dN/da = N (W^2/R^2)(1/a)(a/a_par)^(W^2/R^2)
 *                  I0(2 (d_perp/R)(W/R) sqrt(ln(a_par/a))) exp(-d_perp^2/R^2)
 *                  for 0 < a < a_par (the table's theta read with its
 *                  support the right way round);
 *   QS_GEOM_THIN   on the axis, flat-top length L = length_um, count = N:
 *                  collision positions uniform on [d_par - L/4, d_par + L/4]
 *                  (the crossing is at half the lag); each of z = +-z_R
 *                  sqrt(a0^2/a^2 - 1) inside adds (2N z_R/L)(a0^2/a^2)/
 *                  sqrt(a0^2 - a^2);
 *   QS_GEOM_WIDE   uniform density n_b = count (per um^3) across the laser,
 *                  flat-top length L: dN/da = (2 pi n_b W0^2/a) times the
 *                  integral of 1 + z^2/z_R^2 over the collision positions
 *                  with a_eff(z) > a.
 * qs_analytic_aeff writes dN/da at the n points d_a; qs_analytic_ll_spectrum
 * the classical final-energy density dN/dgamma = (dN/da)(a(gamma)) /
 * |dgamma/da| with gamma = gamma0/(1 + c_RR gamma0 a^2) (Eq. 3, c_RR from the
 * laser as in qs_scatter) at the n energies d_gamma.  Device arrays; FP64.
 * Errors: QS_ERR_INVALID_ARG, QS_ERR_CUDA.
 */
typedef enum { QS_GEOM_SHORT = 0, QS_GEOM_THIN = 1, QS_GEOM_WIDE = 2 } qs_geometry_kind;

typedef struct qs_geometry {
    int32_t kind, reserved;
    double radius_um, length_um, d_perp_um, d_par_um, count;
} qs_geometry;

int32_t qs_analytic_aeff(const qs_laser* laser, const qs_geometry* geom, int64_t n,
                         const double* d_a, double* d_out, void* stream);

int32_t qs_analytic_ll_spectrum(const qs_laser* laser, const qs_geometry* geom, double gamma0,
                                int64_t n, const double* d_gamma, double* d_out, void* stream);

/*
 * qs_unit_rates: throughput probe of the pipes the kernels are bound by (no
 * counterpart in the paper; it supplies the roofline denominators).
 * rates[0..7] (host): FP32 FMA, MUFU lg2, ex2, rcp (the .approx forms the
 * FP32 path issues), FP64 FMA, each in operations per SM per clock at the
 * device's maximum SM clock (a throttled clock reads as a lower rate), then
 * the SM count and that clock in MHz, then the packed f32x2 FMA
 * (fma.rn.f32x2, the form the FP32 phase integration issues) in
 * lane-operations (two per instruction) per SM per clock.  d_scratch: device memory of
 * qs_unit_rates_scratch_bytes() bytes.  Runs a few milliseconds of
 * dependent-chain kernels on `stream` and waits for them.
 * Errors: QS_ERR_INVALID_ARG, QS_ERR_WORKSPACE, QS_ERR_CUDA.
 */
size_t qs_unit_rates_scratch_bytes(void);

int32_t qs_unit_rates(double* rates, void* d_scratch, size_t scratch_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QSCATTER_H */

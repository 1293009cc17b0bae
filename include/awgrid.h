/*
 * awgrid.h - C ABI of the GB300 (sm_103a) AW-projection gridding / degridding library.
 *
 * The library implements the convolutional resampling operators of the imaging
 * measurement equation (arXiv 2508.17187, Sec. 2):
 *   degridding  D(c_ij):  V_ij = D(c_ij) F[I]                      (Eq. ME-MOD-GRIDDED)
 *   gridding    G(c_ij):  I    = F^dagger sum_ij G(c_ij) w_ij V_ij  (Eq. IMAGE-MOD)
 * with the per-visibility kernel c_ij = CF_ij(nu, w, t) and the optional phase-gradient
 * term of Eq. CIJ (Sec. 6), the CF being one of the Tab. AWP-CFSETUP configurations
 * (PS, PS*W, PS*A, PS*A*W).  G is the exact adjoint of D (the residual image of Eq. ResIm
 * is the chi^2 gradient of Eq. ImChisq only if it is).  The Fourier transform F itself is
 * not part of this library; the caller runs it (cuFFT / torch.fft) between the calls.
 *
 * Conventions shared by every entry point:
 *  - Pointers documented "device" point to memory of the current CUDA device; "host"
 *    pointers to ordinary host memory.  The caller owns every buffer it passes; the
 *    library owns the CF set and the plan it creates until the matching *_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Compute calls are asynchronous and stream-ordered: argument checks run on the host
 *    before any launch and return a status synchronously; a fault in a kernel surfaces as
 *    AWG_ERR_CUDA from a later call or from the caller's own synchronisation.
 *  - Complex values are interleaved (re, im) float32 ("c64") unless stated otherwise.
 *  - Layouts: uvw [R][3] float64 metres; freq [C] float64 Hz; visibilities and weights
 *    [R][C][P] (row-major, pols innermost, P in {1, 2, 4}); grid and image [N][N][P] c64
 *    (row = v, column = u; the uv origin and the image centre are pixel (N/2, N/2)).
 *  - On a non-OK status nothing is launched and awg_last_error() describes the reason.
 *  - Calls are thread-safe for distinct objects; one object must not be used from two
 *    host threads at once.
 */
#ifndef AWGRID_H
#define AWGRID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct awg_cf_set_s* awg_cf_set; /* device-resident CF cache (PreCompute, Sec. 4.1 / 6) */
typedef struct awg_plan_s* awg_plan;     /* sorted, tiled sample index (PreSolvePrep, Sec. 5.2) */

typedef enum {
  AWG_OK = 0,
  AWG_ERR_INVALID_ARG = 1, /* a NULL, out-of-range or inconsistent argument */
  AWG_ERR_UNSUPPORTED = 2, /* a valid request this build does not handle (e.g. support > 64) */
  AWG_ERR_OOM = 3,         /* a device or host allocation failed; nothing leaked */
  AWG_ERR_CUDA = 4,        /* a CUDA runtime error (launch failure or an earlier fault) */
  AWG_ERR_TIMEOUT = 5      /* a bounded device wait gave up (reported by a status word) */
} awg_status;

/* CF storage type. */
enum { AWG_CF_FP32 = 0, AWG_CF_BF16 = 1 };

/* grid_visibilities flags. */
enum {
  AWG_GRID_KAHAN = 1, /* compensated flush: rounding error of every flush add goes to grid_lo */
  AWG_GRID_FP64 = 2   /* grid (and grid_lo unused) is complex128 [N][N][P]; flush adds in FP64 */
};

/* degrid_visibilities flags. */
enum {
  AWG_DEGRID_SUBTRACT = 1 /* residual: vis_out holds V on entry and receives V - D(grid) */
};

/*
 * Parameters of a CF set (Tab. AWP-CFSETUP switches plus the imaging geometry).
 * CF index: cf = (pa_bin * n_subbands + subband) * n_signed + ks, with n_signed = 2 n_wplanes - 1
 * when use_w, else 1; signed w-plane ks = n_wplanes - 1 + k (w >= 0) or n_wplanes - 1 - k (w < 0),
 * planes linear in |w|: w_k = k w_max / (n_wplanes - 1).
 * CF of S taps: c(du, dv) = (1/M^2) sum_{i,j<M} screen(x_i, y_j) exp(-2 pi i (du (i - M/2) + dv (j - M/2)) / M),
 * screen = T(x) T(y) [A(l, m; nu_sb, PA)] exp(-2 pi i w_k (sqrt(1 - l^2 - m^2) - 1)), x_i = (i - M/2) N / M
 * image pixels, l = x cell, T(x) = psi_0(pi W / 2, 2x/N) / psi_0(pi W / 2, 0) (zeroth prolate spheroidal
 * function, W = ps_support), M = the smallest power of two >= max(16, 2S).  Tap t of oversampling
 * offset o sits at du = S/2 - t - o/OS; a table is stored offset-major [OS+1][OS+1][S][S] c64.
 * Support schedule: without W every CF has max_support taps; with W, plane k has
 * S_k = min(max_support, 8 ceil((8 + (max_support - 8) sqrt(k / (n_wplanes - 1))) / 8)), at least ps_support.
 * A-term (synthetic; the paper gives none): Airy power pattern (2 J1(z)/z)^2, z = pi D rho nu / c,
 * rho^2 = (l'/(1+eps))^2 + (m'/(1-eps))^2, (l', m') = (l, m) rotated by the bin's parallactic angle.
 */
typedef struct {
  int grid_n;                       /* N: grid side in pixels, even, 16..65536 */
  double cell_rad;                  /* image pixel size (rad); uv pixel du = 1 / (N cell) */
  int oversampling;                 /* OS >= 1 */
  int ps_support;                   /* W: PS kernel width in pixels (e.g. 7) */
  int use_ps;                       /* 1: PS term on (T as above); 0: T = 1 */
  int use_w;                        /* 1: W-projection planes */
  int n_wplanes;                    /* >= 2 when use_w */
  double w_max_lambda;              /* > 0 when use_w */
  int use_a;                        /* 1: A-term on */
  int n_pa_bins;                    /* >= 1 */
  const double* pa_bin_centers_rad; /* host [n_pa_bins] (read when use_a) */
  int n_subbands;                   /* >= 1 */
  const double* subband_freq_hz;    /* host [n_subbands] (read when use_a) */
  int max_support;                  /* 1..64 taps */
  double dish_diameter_m;           /* A-term aperture (e.g. 25) */
  double ellipticity;               /* A-term distortion (e.g. 0.05) */
  int cf_dtype;                     /* AWG_CF_FP32 or AWG_CF_BF16 */
  int separable;                    /* 1: store each CF as a sum of r <= 6 outer products
                                       fy_k[oy][ty] fx_k[ox][tx] when every CF of the set fits one
                                       to 1e-6 of its peak (PS and W-projection CFs with r = 1,
                                       A-term CFs with r of about 4); 0: always full tables */
  /* Full-polarisation A-terms (the sparse Mueller matrix of CFs, Sec. 2 and Sec. 6): with use_a and
     use_pol, each antenna's Jones matrix is J = [[A_R, d A_R], [d A_L, A_L]] with A_R, A_L the
     Airy voltage patterns of the R and L feeds squinted by +-squint_rad along the rotated l axis
     and d = leakage_re + i leakage_im; Mueller element (p, q), pols ordered RR, RL, LR, LL
     (p = (a, b), q = (c, d)), has the image-plane screen J_ac conj(J_bd) (times PS and W).  An
     element is kept when |d|^n >= mueller_threshold, n the number of leakage factors in it (the
     diagonal always).  Needs separable storage and 4 pols in gridding / degridding. */
  int use_pol;
  double squint_rad;
  double leakage_re, leakage_im;
  double mueller_threshold;
} awg_cf_params;

/*
 * Build the CF set on the host in FP64 (PreCompute, Sec. 4.1 and Sec. 6 CFCache) and upload it,
 * rounded to cf_dtype, to the current device.  Negative-w planes are the conjugate point
 * reflections of the positive ones (screen(-w) = conj(screen(w))).  With params->separable and FP32
 * storage, each table seen as a ((OS+1) S)^2 matrix is fitted as sum_k g_k f_k^T, one term at a
 * time from the residual (alternating least squares), until the residual is within 1e-6 of the
 * table's peak; if every CF fits with at most 6 terms only the factors are kept (2 (OS+1) S values
 * per term instead of ((OS+1) S)^2 per CF; the set's rank r is the largest term count, smaller fits
 * are padded with zero terms), otherwise the full tables are.  A plan on a rank-r set holds r
 * records per sample, so gridding and degridding cost r times the rank-1 work.  Blocking: returns
 * once the tables are resident.  Errors: INVALID_ARG (bad params), UNSUPPORTED (max_support > 64),
 * OOM.
 */
awg_status cf_set_create(const awg_cf_params* params, void* stream, awg_cf_set* out);

/*
 * Same, with caller-supplied tables instead of the built ones (e.g. a support-1 delta kernel).
 * supports: host [n_cf] taps per CF (1..64); table: host c64, all CFs concatenated in CF-index
 * order, each [OS+1][OS+1][S][S].  Only grid_n, oversampling, use_w, n_wplanes, w_max_lambda,
 * n_pa_bins, n_subbands, cf_dtype and separable of params are read.  With separable and FP32
 * storage, only factors are kept when every table is a sum of at most 6 outer products to 1e-6 of
 * its peak (the fit of cf_set_create); otherwise the full tables are.
 */
awg_status cf_set_create_from_table(const awg_cf_params* params, const int32_t* supports,
                                    const float* table, void* stream, awg_cf_set* out);

awg_status cf_set_destroy(awg_cf_set cf);

/* Number of CFs, complex values held (2-D tables or factors) and the separable rank: the number of
 * outer-product terms per CF, or 0 for full tables. */
awg_status cf_set_info(awg_cf_set cf, int32_t* n_cf, int64_t* n_values, int32_t* separable);

/* Outer-product terms that the gridding and degridding kernels combine per tap: RK in [2, 4] when
 * every stored CF of a factored set has at most RK terms (RK the largest) and every support has an
 * exact-support kernel, so that a plan holds one record per sample and each tap's CF value is
 * formed from the RK terms in registers; 0 otherwise (rank 1, full tables, or a set whose plans
 * hold one record per sample and term).  A full-polarisation set with fused kernels runs one 4-pol
 * pass per base CF (A_R A_R, A_R A_L, A_L A_L) with its elements' scalars as a pol-mixing matrix;
 * otherwise one single-pol pass per Mueller element.  terms: host. */
awg_status cf_set_fused_terms(awg_cf_set cf, int32_t* terms);

/*
 * Per-support autotuner of the separable kernels (a project addition; the paper fixes no kernel
 * shapes).  Every support of the W-projection schedule (8, 16, ..., 64) has four compiled kernel
 * configurations: 0 and 1 differ in the tile of first-tap positions per work item, threads per
 * CTA and samples staged per chunk; 2 is the warp-specialised pair (a producer warp stages chunks
 * into a ring of shared-memory stages handed over on mbarriers, consumer warps only multiply and
 * add, a flush warp (gridding) or reduce warp (degridding) finishes each item, and degridding
 * loads each item's grid window with one TMA tile copy); 3 runs both operators on the tensor
 * cores (tcgen05, 3xTF32 products, FP32 accumulation in tensor memory: a gridding window is the
 * product of the item's x-factor rows and its y-factor rows times w V; degridding forms the
 * samples' y-factor rows times TMA-loaded window slices and finishes the x sum per sample;
 * relative RMS error a few 1e-6 against the FP64 result) with tiles of odd side so that a window
 * fills the MMA shape (support 64, whose window is wider than 64 pixels, degrids with the
 * warp-specialised kernel on those tiles).  For each configuration this builds a plan of the
 * given geometry (uvw_m, freq_hz, pa_bin, chan_subband: device arrays as for plan_create, typically the data to be imaged or a
 * slice of it), grids and degrids unit visibilities with n_pol pols once, then times every
 * support's gridding and degridding launch three times (CUDA events on `stream`), and keeps the
 * fastest configuration per support in the CF set.  Plans created before the call are invalid
 * afterwards (their calls return INVALID_ARG); create plans after tuning.  Blocking.  Allocates
 * scratch of about (R C n_pol) 20 B plus one grid and two plans, and frees it before returning.
 * choice_out: host int32 [65] or NULL, the chosen configuration (0, 1, 2 or 3) per support, -1
 * where none was timed; ms_out: host float [4][65] or NULL, grid + degrid milliseconds of each
 * configuration per support (0 where not timed).  Fused multi-term sets (cf_set_fused_terms > 0)
 * have configurations 0 and 1 of the fused kernels (the tiles and staging of the cp.async
 * configurations), which are timed the same way; full-table and full-polarisation sets have
 * nothing to tune (choices -1).  Errors: INVALID_ARG, OOM, CUDA.
 */
awg_status cf_set_autotune(awg_cf_set cf, const double* uvw_m, int64_t n_rows, const double* freq_hz, int32_t n_chan,
                           const int32_t* pa_bin, const int32_t* chan_subband, int32_t n_pol, void* stream,
                           int32_t* choice_out, float* ms_out);

/* Select configuration `config` (0, 1, 2 or 3) of the separable kernels for one support of the
 * W-projection schedule by hand (what cf_set_autotune does by timing); plans created before the
 * call are invalid afterwards.  Fused multi-term sets take 0 or 1, full-polarisation sets 0.
 * Errors: INVALID_ARG (no configurations for that support), UNSUPPORTED (a configuration the
 * set's kernels do not have). */
awg_status cf_set_choose(awg_cf_set cf, int32_t support, int32_t config);

/* Mueller elements of a full-polarisation CF set (use_pol): *n_elem (0 otherwise) and, when not
 * NULL, host int32 [16] arrays of each element's output pol p and input pol q (0..3 = RR, RL, LR,
 * LL).  CF index = element * (n_pa_bins n_subbands n_signed) + the per-sample CF index.  Gridding
 * with such a set adds conj(CF_pq) w_p V_p into grid pol q (the diagonal elements add the weights
 * to sumwt[q]); degridding sets vis pol p to the sum over its elements of CF_pq applied to grid
 * pol q.  Both need n_pol = 4. */
awg_status cf_set_mueller(awg_cf_set cf, int32_t* n_elem, int32_t* elem_p, int32_t* elem_q);

/* The parameters a CF set was made with (pointers NULL in *out); when not NULL,
 * pa_bin_centers_rad host [n_pa_bins] and subband_freq_hz host [n_subbands] receive the A-term
 * bins (left untouched without use_a). */
awg_status cf_set_get_params(awg_cf_set cf, awg_cf_params* out, double* pa_bin_centers_rad, double* subband_freq_hz);

/*
 * Persistent CF cache (the CFCache of Sec. 6, which the paper keeps in memory and on disk): save a
 * CF set to a file and load it back without rebuilding it.  The file holds the parameters, the
 * storage mode, the support and autotuned kernel choice of every support, and the stored CF data
 * (FP32 factors, or the FP32 / BF16 tables) exactly, so that a loaded set computes bit-identical
 * results; it is read on hosts of the same byte order and awg_cf_params layout.  cf_set_save
 * copies the device data first (blocking) and writes nothing when that fails; cf_set_load checks
 * the magic, version, parameter layout, the parameters (as cf_set_create does), the storage mode
 * against the parameters and the end marker.  Errors: INVALID_ARG (NULL, unreadable / unwritable
 * path, a file that is not a CF cache, truncated or inconsistent), OOM, CUDA.
 */
awg_status cf_set_save(awg_cf_set cf, const char* path);
awg_status cf_set_load(const char* path, void* stream, awg_cf_set* out);

/* Host copy of the support of every CF: supports_out host [n_cf]. */
awg_status cf_set_get_supports(awg_cf_set cf, int32_t* supports_out);

/* Host copy of one CF table as c64 [OS+1][OS+1][S][S] (BF16 tables are widened; a separable CF
 * is expanded as the sum of its FP32 products fy_k fx_k). Blocking. */
awg_status cf_set_copy_table(awg_cf_set cf, int32_t cf_index, float* table_out);

/* Host copy of the stored factors of one term of a separable CF: CF_ci = scale * sum over the terms
 * k of fy_k[oy][ty] fx_k[ox][tx].  fx_out, fy_out: host c64 [OS+1][S] (term `term` < the set's
 * rank; zero rows for the padding terms of CFs fitted with fewer); scale_out: host float [2] or
 * NULL, the element scalar s_pq (re, im) of a Mueller element stored as a base CF, else (1, 0).
 * The FP32 values are the ones the kernels read.  Blocking.  Errors: INVALID_ARG (NULL, full-table
 * set, index or term out of range), CUDA. */
awg_status cf_set_copy_factors(awg_cf_set cf, int32_t cf_index, int32_t term, float* fx_out, float* fy_out,
                               float* scale_out);

/*
 * Create a plan: per-visibility index and the tiled ordering of all R*C samples
 * (PreSolvePrep re-ordering, Sec. 5.2 and Sec. 6.1).  For every (row r, channel c), in FP64 with
 * no fused multiply-add: u_l = u_m (nu_c / c_light); x = u_l (N cell) + N/2 (same for v, y);
 * w-plane k = floor(|w_l| (n_w - 1) / w_max + 1/2) (k > n_w - 1 drops the sample); cf as above;
 * hx = x - S/2, first tap p0x = floor(hx) + 1, offset ox = floor((p0x - hx) OS + 1/2) in [0, OS].
 * A sample is kept iff -1 <= hx < N - S and -1 <= hy < N - S; others are dropped and counted.
 * uvw_m: device [R][3] f64; freq_hz: device [C] f64; pa_bin: device int32 [R] (needed when
 * n_pa_bins > 1, else may be NULL); chan_subband: device int32 [C] (needed when n_subbands > 1);
 * phase_shift: host f64 [2] (dl, dm) of the image centre from the phase centre, or NULL for none:
 * G multiplies w V by exp(+2 pi i (u dl + v dm + w dn)), dn = sqrt(1 - dl^2 - dm^2) - 1, D by its
 * conjugate (the phase term of Eq. CIJ); the plan forms every sample's phasor once per build and
 * the kernels read it.  The plan allocates device memory (about 44 bytes per sample and CF term,
 * 8 more per sample with a phase term) and keeps pointers to no caller buffer.  It also owns two
 * CUDA streams and three events: the per-support launches of one gridding or degridding call
 * alternate between those streams, ordered by the events after the work queued on the call's
 * `stream` and before the work queued on it afterwards (so calls stay stream-ordered and
 * graph-capturable), and a support's launch starts on the SMs that the previous one has finished
 * with.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 */
awg_status plan_create(awg_cf_set cf, const double* uvw_m, int64_t n_rows, const double* freq_hz,
                       int32_t n_chan, const int32_t* pa_bin, const int32_t* chan_subband,
                       const double* phase_shift, void* stream, awg_plan* out);

/*
 * Per-row phase centres: mosaic pointings and antenna pointing offsets (the phase-gradient term
 * of Eq. CIJ with s(P) and (Delta s_i + Delta s_j) / 2 per row; Tab. AWPSETUP-MOSAICKING).
 * row_dlm: device f64 [R][2], (dl, dm) of the image centre relative to row r's phase centre,
 * dl^2 + dm^2 < 1 (not checked); from here on G multiplies w V of every sample of row r by
 * exp(+2 pi i (u dl_r + v dm_r + w dn_r)), dn_r = sqrt(1 - dl_r^2 - dm_r^2) - 1, and D by its
 * conjugate, replacing the plan-wide shift of plan_create.  uvw_m [R][3] and freq_hz [C] (device)
 * are the plan's current geometry, copied together with row_dlm into plan-owned memory (allocated
 * on the first call; later plan_update calls refresh the geometry copy).  row_dlm = NULL returns
 * to the plan-wide shift (or none) and frees the per-row copy (synchronising `stream`).
 * Asynchronous otherwise.  Errors: INVALID_ARG, CUDA.
 */
awg_status plan_set_row_phase(awg_plan plan, const double* row_dlm, const double* uvw_m, const double* freq_hz,
                              void* stream);

/*
 * Recompute the plan for new uvw / frequency / bin data of the same R and C (no allocation;
 * stream-ordered; capturable in a CUDA graph).
 */
awg_status plan_update(awg_plan plan, const double* uvw_m, const double* freq_hz, const int32_t* pa_bin,
                       const int32_t* chan_subband, void* stream);

awg_status plan_destroy(awg_plan plan);

/*
 * Plan statistics (synchronises the plan's last stream): kept and dropped samples and
 * sum over kept samples of S^2 (complex multiply-accumulates per pol for one G or D pass).
 */
awg_status plan_stats(awg_plan plan, int64_t* n_kept, int64_t* n_dropped, int64_t* sum_taps);

/*
 * Host copy of the plan's per-sample index (the CF_ij(nu, w, t) selection of Eq. CIJ and the pixel
 * and offset rules of plan_create), in sample order s = row * n_chan + chan, for inspection and
 * tests: kept[s] = number of records of sample s in the plan (1 when kept, 0 when dropped), and for
 * kept samples cf_out[s] (the CF index), p0x[s], p0y[s] (first tap pixel) and ox[s], oy[s]
 * (oversampling offsets in [0, OS]); -1 for dropped ones.  All outputs: host int32 [n_rows * n_chan].
 * Synchronises the plan's last stream and copies the records back (blocking).
 * Errors: INVALID_ARG, OOM, CUDA.
 */
awg_status plan_copy_index(awg_plan plan, int32_t* kept, int32_t* cf_out, int32_t* p0x, int32_t* p0y, int32_t* ox,
                           int32_t* oy);

/*
 * Completion check of the plan's gridding and degridding launches (synchronises the plan's last
 * stream).  The warp-specialised kernels (configurations 2 and 3 of cf_set_autotune / cf_set_choose) hand
 * work between their warps on shared-memory barriers whose waits are bounded (2 s); a wait that
 * gives up ends its launch early and records it in the plan.  Returns AWG_ERR_TIMEOUT (and clears
 * the record) when a launch since the last plan_create / plan_update / plan_check did so - its
 * results are then incomplete - else AWG_OK.  Errors: INVALID_ARG, CUDA.
 */
awg_status plan_check(awg_plan plan);

/*
 * Gridding G (Eq. IMAGE-MOD): for every kept sample s and pol p,
 *   grid[p0y+ty][p0x+tx][p] += conj(CF_cf[oy][ox][ty][tx]) * weight[s][p] * vis[s][p] (* phasor),
 * accumulated (+=) into the caller's grid; sumwt[p] += sum of weight[s][p] over kept samples (FP64).
 * vis: device c64 [R][C][P]; weight: device f32 [R][C][P] (0 = flagged); grid: device c64
 * [N][N][P] (complex128 with AWG_GRID_FP64); grid_lo: device c64 [N][N][P] compensation grid with
 * AWG_GRID_KAHAN (the true sum is grid + grid_lo), else NULL; sumwt: device f64 [P].
 * Accumulation is FP32 in registers and shared memory with one atomic flush per tile pixel;
 * the summation order is not fixed, so results agree with an FP64 sum to FP32 rounding.
 * Errors: INVALID_ARG (NULL pointer, P not in {1,2,4}, bad flags), CUDA.
 */
awg_status grid_visibilities(awg_cf_set cf, awg_plan plan, const void* vis, const float* weight,
                             int32_t n_pol, void* grid, void* grid_lo, double* sumwt, int32_t flags,
                             void* stream);

/*
 * Degridding D (Eq. ME-MOD-GRIDDED, Eq. VMod): for every sample s and pol p,
 *   vis_out[s][p] = sum_{ty,tx} CF_cf[oy][ox][ty][tx] * grid[p0y+ty][p0x+tx][p] (* conj(phasor)),
 * overwritten; dropped samples get 0.  grid: device c64 [N][N][P]; vis_out: device c64 [R][C][P].
 * With flags = AWG_DEGRID_SUBTRACT the call forms the residual of Eq. ResIm in place: vis_out
 * holds the observed visibilities on entry and each kept sample receives vis_out - D(grid), the
 * difference taken where the model value is formed (no second pass over the visibilities);
 * dropped samples keep their input.  D is the adjoint of G with unit weights: <G V, X> = <V, D X>.
 * Errors: INVALID_ARG (including unknown flags), CUDA.
 */
awg_status degrid_visibilities(awg_cf_set cf, awg_plan plan, const void* grid, void* vis_out,
                               int32_t n_pol, int32_t flags, void* stream);

/*
 * Taper correction around the caller's FFT (Eq. IMAGE-MOD, PS term of Tab. AWP-CFSETUP):
 * direction 0 (after F^dagger of a gridded grid): image[y][x][p] /= (sumwt[p] T(x - N/2) T(y - N/2));
 * direction 1 (a model image before F and degridding): image[y][x][p] /= (T(x - N/2) T(y - N/2)).
 * image: device c64 [N][N][P], in place; sumwt: device f64 [P] (direction 0; NULL means 1).
 * Errors: INVALID_ARG, CUDA.
 */
awg_status grid_normalize(awg_cf_set cf, void* image, int32_t n_pol, const double* sumwt,
                          int32_t direction, void* stream);

/*
 * Gridding without any device allocation (the paper has no counterpart: this is a service for
 * callers of the library).  Some callers cannot allocate device memory once they are running:
 * real-time pipelines that reserve all of the GPU's memory at start-up and forbid allocation
 * afterwards, and hosts whose own allocator owns the device, where a raw cudaMalloc would fail or
 * break that allocator's pool.  This call does what plan_create followed by grid_visibilities
 * (flags 0, no phase shift) does, but keeps the plan in one fixed array of about 4.7 MB of device
 * memory that belongs to the loaded library (every GPU that loads the library holds it until the
 * process exits); it calls no cudaMalloc, cudaFree or allocating library routine.
 * Limits: at most 65536 samples (n_rows x n_chan) per call and at most 65536 (support, tile)
 * buckets for the CF set and grid size (small grids, e.g. N = 512 with a few supports); larger
 * requests return AWG_ERR_INVALID_ARG with the limit in awg_last_error() and launch nothing.
 * Arguments: as plan_create (uvw_m, freq_hz, pa_bin, chan_subband: device) and grid_visibilities
 * (vis, weight, grid, sumwt: device, accumulated).
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture on the device.  The address
 * is kept per device and CUDA context: after a cudaDeviceReset the next call looks it up again in
 * the new context (where the array starts over with unspecified contents).  The call leaves the
 * caller's current device as it found it.
 * Every call on a device shares the one array and it keeps what the last call left there; each
 * call clears what it accumulates into before use, so sequential calls are independent, but calls
 * whose work overlaps on the GPU (different streams, not ordered by events) race and corrupt each
 * other's results: order them on one stream.
 */
awg_status grid_visibilities_noalloc(awg_cf_set cf, const double* uvw_m, int64_t n_rows, const double* freq_hz,
                                     int32_t n_chan, const int32_t* pa_bin, const int32_t* chan_subband,
                                     const void* vis, const float* weight, int32_t n_pol, void* grid,
                                     double* sumwt, void* stream);

/*
 * Plain FP64 baseline of G and D (the straightforward port the batched kernels are measured
 * against): one launch per channel in [chan_begin, chan_end), one thread per row, the index rules
 * of plan_create evaluated inline, FP32 table values widened to FP64, FP64 multiply-adds, and for
 * G one FP64 atomic per tap and pol into a complex128 grid.  No plan, no sort, no allocation.
 * The CF set must hold full FP32 tables (created with separable = 0).  freq_hz_host and
 * chan_subband_host are HOST arrays [n_chan]; uvw_m, pa_bin, vis, weight: device as above;
 * grid64: device complex128 [N][N][P] (accumulated); sumwt: device f64 [P] (accumulated);
 * vis_out: device c64 [R][C][P], written for the channels in range (dropped samples get 0).
 * Errors: INVALID_ARG, UNSUPPORTED (separable or BF16 CF set), CUDA.
 */
awg_status grid_visibilities_plain_fp64(awg_cf_set cf, const double* uvw_m, int64_t n_rows, const double* freq_hz_host,
                                        int32_t n_chan, int32_t chan_begin, int32_t chan_end, const int32_t* pa_bin,
                                        const int32_t* chan_subband_host, const void* vis, const float* weight,
                                        int32_t n_pol, void* grid64, double* sumwt, void* stream);
awg_status degrid_visibilities_plain_fp64(awg_cf_set cf, const double* uvw_m, int64_t n_rows,
                                          const double* freq_hz_host, int32_t n_chan, int32_t chan_begin,
                                          int32_t chan_end, const int32_t* pa_bin, const int32_t* chan_subband_host,
                                          const void* grid64, void* vis_out, int32_t n_pol, void* stream);

/*
 * FP32 FMA probe (a measurement utility; the paper has no counterpart): launches n_blocks CTAs
 * of 256 threads on `stream`, each thread running `iters` iterations of 8 independent FP32
 * fused multiply-adds, and writes one float per thread to out (device, n_blocks * 256 floats,
 * caller-owned) so the work cannot be elided.  *flop (host) receives the FLOP count of the
 * launch (2 per FMA).  The caller times the launch on `stream`; FLOP / time is the rate of the
 * non-tensor FP32 pipe that bounds gridding and degridding.  Asynchronous.
 * Errors: INVALID_ARG, CUDA.
 */
awg_status awg_fp32_fma_probe(float* out, int32_t n_blocks, int64_t iters, void* stream, double* flop);

/* The same probe in FP64 (out: device, n_blocks * 256 doubles): the FP64 FMA rate that bounds the
 * plain FP64 baseline (grid_visibilities_plain_fp64 / degrid_visibilities_plain_fp64).
 * Asynchronous.  Errors: INVALID_ARG, CUDA. */
awg_status awg_fp64_fma_probe(double* out, int32_t n_blocks, int64_t iters, void* stream, double* flop);

/*
 * Hogbom CLEAN minor cycle (the deconvolution step of the major cycle, Sec. 5.2; Eq. ModelUpdate
 * with point components).  n_iter iterations, each: find the pixel p of largest |residual| inside
 * the search window (ties: the lowest linear index y N + x), stop for good once that value is
 * below `threshold`; else g = gain * residual[p] (FP32), model[p] += g, and residual[y][x] -=
 * g * psf[y - py + psf_n/2][x - px + psf_n/2] wherever that PSF pixel exists.  Products and sums
 * are separately rounded FP32 operations (no fused multiply-add).
 * residual, model: device f32 [N][N] (row y, column x), updated in place; psf: device f32
 * [psf_n][psf_n], peak at (psf_n/2, psf_n/2) (psf_n = 2N covers every shift); window: host
 * int32 {x0, x1, y0, y1} (half-open) or NULL for the whole image; gain in (0, 1]; threshold >= 0.
 * workspace: device, clean_hogbom_workspace_bytes() bytes, 16-byte aligned, caller-owned.
 * Asynchronous on `stream` (3 launches per iteration, no host synchronisation, graph-capturable).
 * Errors: INVALID_ARG, UNSUPPORTED (N^2 >= 2^31), CUDA.
 */
int64_t clean_hogbom_workspace_bytes(void);
awg_status clean_hogbom(float* residual, float* model, int32_t N, const float* psf, int32_t psf_n, int32_t n_iter,
                        float gain, float threshold, const int32_t* window, void* workspace, void* stream);
/* Number of components the last clean_hogbom on this workspace found (synchronises). */
awg_status clean_hogbom_components(const void* workspace, int32_t* n_done);

/*
 * Direction-independent G-Jones calibration (Sec. 5.1): Eq. VAvg, then Eq. CalUpdateDir and
 * Eq. CalUpdateModel iterated to the exit test of the same section, for every solution interval.
 * vis (observed, corrected), model (Eq. VMod, e.g. from degrid_visibilities): device c64
 * [n_rows][n_chan][n_pol]; weight: device f32, same shape (<= 0: flagged).  Rows are time-major:
 * row = t n_bl + b, baseline b joining antennas ant1[b] and ant2[b] (device int32 [n_bl], values in
 * [0, n_ant)).  The parallel hands are pols 0 and n_pol - 1 (one product when n_pol = 1).
 * A solution interval is sol_int integrations x sol_chan channels (the last ones may be shorter);
 * per interval, hand and baseline X = sum w V conj(M) / sum w |M|^2 with weight sum w |M|^2 (the
 * weighted average of V / M), then from g = 1: g_i <- (1 - alpha) g_i + alpha sum_{j != i} g_j
 * X_ij w_ij / sum_{j != i} |g_j|^2 w_ij (X_ji = conj(X_ij)) until max_i |change| < delta or
 * max_iter iterations; finally every g_i is multiplied by conj(g_ref) / |g_ref| (ref_ant's phase
 * is zero).  Precision: the data pass forms N = sum w V conj(M) and D = sum w |M|^2 (so that
 * X w = N, w = D) in FP32 - products rounded once, Kahan-compensated per-thread sums, an FP32 tree
 * over 32 threads - to within ~10 u (u = 2^-24) of sum w |V| |M|.  The iteration runs in FP32
 * while the largest change exceeds 3e-5 of the largest |g|, then in FP64 to the exit test (a
 * delta coarser than that is tested in the FP32 phase); iterations counts both phases.
 * gains: device c128 [n_ts][n_fs][n_hands][n_ant] with n_ts =
 * ceil(n_int / sol_int), n_fs = ceil(n_chan / sol_chan); iterations: device int32
 * [n_ts][n_fs][n_hands], the iterations run.  workspace: device, gcal_workspace_bytes(...) bytes,
 * 16-byte aligned.  Asynchronous (two launches).  Errors: INVALID_ARG, UNSUPPORTED (> 128
 * antennas), CUDA.
 */
int64_t gcal_workspace_bytes(int64_t n_rows, int32_t n_chan, int32_t n_pol, int32_t n_bl, int32_t sol_int,
                             int32_t sol_chan);
awg_status gcal_solve(const void* vis, const void* model, const float* weight, int64_t n_rows, int32_t n_chan,
                      int32_t n_pol, int32_t n_bl, const int32_t* ant1, const int32_t* ant2, int32_t n_ant,
                      int32_t sol_int, int32_t sol_chan, double alpha, double delta, int32_t max_iter, int32_t ref_ant,
                      void* gains, int32_t* iterations, void* workspace, void* stream);

/*
 * Failure injection for tests (host side; no device fault).  After awg_debug_fail_allocations(n)
 * the next n device allocations of this library succeed and the one after fails as out of memory
 * (without reaching the driver), and so does every later one until the hook is reset with -1.  A
 * call that meets the failure returns AWG_ERR_OOM and frees what it had allocated:
 * awg_debug_live_allocations() (the library's live device allocations) is then what it was
 * before the call.  Errors: INVALID_ARG (n < -1).
 */
awg_status awg_debug_fail_allocations(int64_t after);
int64_t awg_debug_live_allocations(void);

/*
 * Failure injection for tests of the bounded waits (no device fault, trap or endless wait): after
 * awg_debug_ws_withhold(1) the next grid_visibilities or degrid_visibilities call withholds,
 * in every CTA of its warp-specialised launches (configurations 2 and 3), the hand-over of the first
 * chunk from the producer warp to the consumer warps.  Their bounded waits give up after 2 s, the
 * launch ends early with incomplete results, and plan_check reports AWG_ERR_TIMEOUT; the CUDA
 * context stays usable.  awg_debug_ws_withhold(0) disarms it.  Errors: INVALID_ARG.
 */
awg_status awg_debug_ws_withhold(int32_t on);

/* Thread-local message describing the last non-OK status of this thread. */
const char* awg_last_error(void);

/* Number of kernels this library has launched in the process so far (all threads, all devices).
 * A diagnostic for benchmarks and tests; reading it has no side effect. */
int64_t awg_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* AWGRID_H */

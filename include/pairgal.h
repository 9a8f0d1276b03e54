/*
 * pairgal.h -- C ABI of libpairgal.so, the GB300 (sm_103a) pair-galaxy
 * cross-correlation library after Yuan, Eisenstein & Garrison (2017),
 * "Using galaxy pairs to investigate the three-point correlation function in
 * the squeezed limit".
 *
 * The method (Sec. 2.1-2.2): close galaxy pairs, binned by separation s and
 * line-of-sight cosine mu, are objects at their midpoints; each bin's pair
 * field is deposited on a periodic mesh and cross-correlated with the galaxy
 * mesh by 3D FFTs. Binning the correlation by (r, mu_r) gives
 *   xi_pg(s, mu; r, mu_r), xi_gg(r, mu_r), b_pg = xi_pg / xi_gg   (eq. bpg_initial,
 *   with W the indicator of one (r, mu_r) shell; eq. bpg_final is the same
 *   estimator written in real space),
 *   xi(d_w) = sum C_gg^2 / sum C_gg over the shell                  (eq. xi_dw),
 *   Q_eff from eq. Qeff_notsq and the strict-squeezed form eq. Qeff, with
 *   xi(d_p) = xi(s, mu) = DD / RR - 1 from the pair counts           (eq. 2PCF_d_collapsed).
 * With pair_grid = 1 the pairs are binned instead on the (d_perp, d_par)
 * grid of the paper's b_pg and Q_eff maps (Sec. 5), d_perp = sqrt(dx^2 +
 * dy^2), d_par = |dz|, and the LOS-projected w(d_perp) of eq.
 * 2PCF_los_integrated_explicit is returned as well.
 *
 * Conventions for every entry point:
 *  - Positions are FP64, [n][3] row-major (x, y, z), Mpc/h, any real value
 *    (they are wrapped into [0, L)). The line of sight is z.
 *  - "device" pointers are CUDA device memory of the current device; "host"
 *    pointers are ordinary or pinned host memory. The caller owns every input
 *    and output buffer; the library never frees them.
 *  - Mesh arrays are [z][y][x] with x contiguous; mesh node i sits at i * L/N.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = the legacy
 *    default stream) unless it returns host results, in which case it
 *    synchronises that stream before returning.
 *  - No call throws; each returns a pg_status. A plan is not thread safe;
 *    separate plans may run on separate streams.
 *  - Empty bins (no pairs, no galaxies, or no mesh cells) give NaN outputs
 *    with PG_OK; callers inspect dd and n_cells.
 */
#ifndef PAIRGAL_H
#define PAIRGAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PG_OK = 0,
  PG_ERR_INVALID_ARG = 1,   /* bad sizes, edges, NaN/Inf input, NULL where required */
  PG_ERR_UNSUPPORTED = 2,   /* valid request this build does not handle (e.g. mesh_n) */
  PG_ERR_OOM = 3,           /* device allocation failed */
  PG_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed */
  PG_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
  PG_ERR_UNIMPLEMENTED = 6,
  PG_ERR_CAPACITY = 7       /* an output buffer is smaller than the result */
} pg_status;

/* Returns a static, NUL-terminated description of a status code. */
const char* pg_status_string(pg_status s);

/* Problem statement (Sec. 2.1, Sec. 3.3-3.6). Edge arrays are HOST memory and
 * are copied by pg_plan_create. */
typedef struct pg_params {
  double box_L;             /* periodic box side, Mpc/h, > 0 */
  int32_t mesh_n;           /* N: power of two, 32..1024 (Sec. 3.5 mesh) */
  int32_t assign;           /* 0 = NGP, 1 = CIC, 2 = TSC (the paper's) mass assignment (Sec. 3.5) */
  int32_t n_s;              /* pair separation bins, 1..64 */
  const double* s_edges;    /* [n_s+1] ascending, s_edges[0] >= 0, s_edges[n_s] < L/2 */
  int32_t n_mu;             /* equal bins of mu = |dz|/s on [0, 1], 1..64 */
  int32_t n_r;              /* correlation radius bins, 1..64 */
  const double* r_edges;    /* [n_r+1] ascending, r_edges[0] >= 0, r_edges[n_r] < L/2 */
  int32_t n_mur;            /* equal bins of mu_r = |r_z|/r on [0, 1], 1..64 */
  double rsd_factor;        /* Mpc/h per km/s: z' = z + rsd_factor * v_z (eq. RSD); 0 = real space */
  double r_perp_cut;        /* aggregates exclude cells with r_perp < cut (Sec. 3.6(b)); 0 = off */
  int32_t precision;        /* 0 = FP32 FFT + FP64 reductions, 1 = FP64 throughout */
  int32_t bins_per_batch;   /* pair meshes resident at once; 0 = chosen from N */
  int32_t pair_grid;        /* 0 = (s, mu) pair bins; 1 = (d_perp, d_par) grid: s_edges are then
                               the d_perp edges (n_s bins) and par_edges the |d_par| edges (n_mu
                               bins); the largest separation sqrt(d_perp,max^2 + d_par,max^2)
                               must be < L/2 */
  const double* par_edges;  /* [n_mu+1] ascending, par_edges[0] >= 0 (pair_grid = 1; else unused) */
} pg_params;

typedef struct pg_plan pg_plan;

/* Host output buffers (caller-owned; any pointer may be NULL to skip it).
 * P = n_s*n_mu pair bins (index s_bin*n_mu + mu_bin); Q = n_r*n_mur
 * correlation bins (index r_bin*n_mur + mur_bin). */
typedef struct pg_result {
  int64_t* dd;          /* [P] number of pairs per (s, mu) bin */
  double* dd_w;         /* [P] sum of w_i*w_j (exact: summed as Q32.32 integers) */
  double* xi_ss;        /* [P] xi(s, mu) = DD/RR - 1, RR = ((sum w)^2 - sum w^2)/2 * V_bin/L^3 with
                           V_bin = (4 pi/3)(s_hi^3 - s_lo^3)/n_mu, or on the (d_perp, d_par) grid
                           V_bin = pi (p_hi^2 - p_lo^2) * 2 (l_hi - l_lo) (both signs of d_par) */
  double* xi_pg;        /* [P][Q] mean of C_pg over the bin's cells */
  double* xi_gg;        /* [Q] mean of C_gg */
  double* b_pg;         /* [P][Q] xi_pg / xi_gg */
  double* q_eff;        /* [P][Q] eq. Qeff_notsq with xi(d_p) = xi_ss, xi(d_w) = xi_dw */
  double* q_eff_sq;     /* [P][Q] eq. Qeff (strictly squeezed) */
  double* xi_dw;        /* [Q] sum C_gg^2 / sum C_gg over the bin (eq. xi_dw) */
  double* b_pg_agg;     /* [P] sum C_pg / sum C_gg over all cells with r in [r_0, r_nr), r_perp >= cut */
  double* q_eff_agg;    /* [P] eq. Qeff_notsq with b_pg_agg and xi_dw_agg */
  double* xi_dw_agg;    /* [1] */
  int64_t* n_cells;     /* [Q] mesh offsets in each (r, mu_r) bin */
  int64_t* n_cells_agg; /* [1] */
  double* sum_pg;       /* [P][Q] sum of C_pg over the bin (raw) */
  double* sum_pg_agg;   /* [P] */
  double* sum_gg;       /* [Q] */
  double* sum2_gg;      /* [Q] sum of C_gg^2 */
  double* sum_gg_agg;   /* [2] sum C_gg, sum C_gg^2 over the aggregate cells */
  double* w_perp;       /* [n_s] pair_grid = 1: w(d_perp) = sum over the d_par bins of
                           2 (l_hi - l_lo) xi(d_perp, d_par) (eq. 2PCF_los_integrated_explicit,
                           first line, with d_par,max = the last par edge); NaN otherwise */
} pg_result;

/* Validates *params, copies the edges and builds the data-independent plan
 * state (FFT twiddles, the (r, mu_r) cell lists of the offset window) on the
 * current device. Device workspace grows on first use (see pg_plan_reserve).
 * Errors: PG_ERR_INVALID_ARG, PG_ERR_UNSUPPORTED, PG_ERR_OOM, PG_ERR_CUDA. */
pg_status pg_plan_create(const pg_params* params, pg_plan** out);

/* pg_plan_create whose mesh-sized scratch (line buffers, spectra, windows,
 * adjoint spectra: the bulk of the device memory at large N) is shared with
 * `share_with`, a plan of the same mesh_n and precision on the same device;
 * its other parameters (box, bins, batch size) may differ. Shared scratch
 * grows to the largest need. Plans that share scratch must not run
 * concurrently (one stream, or one call at a time). Errors as
 * pg_plan_create, plus PG_ERR_INVALID_ARG if share_with is NULL or differs
 * in mesh_n, precision or device. */
pg_status pg_plan_create_shared(const pg_params* params, const pg_plan* share_with, pg_plan** out);

/* Frees the plan and its device workspace (synchronises the device first);
 * shared scratch is freed with the last plan that uses it. */
void pg_plan_destroy(pg_plan* plan);

/* Allocates workspace for catalogues up to n_gal_max galaxies and
 * n_pairs_max pairs so that later calls allocate nothing. */
pg_status pg_plan_reserve(pg_plan* plan, int64_t n_gal_max, int64_t n_pairs_max);

/* Device bytes currently held by the plan, including the scratch it may
 * share with other plans. */
size_t pg_workspace_bytes(const pg_plan* plan);

/* The full forward path (Sec. 2.1-2.2, 3.2-3.6) for one catalogue:
 * positions -> (s, mu) pairs -> per-bin midpoint meshes and the galaxy mesh
 * -> FFT cross-correlation -> (r, mu_r) binning -> ratios.
 *   d_pos [n_gal][3] FP64 device; d_vel [n_gal][3] FP32 km/s device or NULL
 *   (needed when rsd_factor != 0); d_w [n_gal] FP32 device or NULL (unit
 *   weights; weights must be >= 0). Results are written to *host_out; the
 *   stream is synchronised before return.
 * Errors: PG_ERR_INVALID_ARG (n_gal < 0, NULL positions, non-finite
 * positions), PG_ERR_OOM, PG_ERR_CUDA. n_gal = 0 gives NaN outputs. */
pg_status pg_forward(pg_plan* plan, int64_t n_gal, const double* d_pos,
                     const float* d_vel, const float* d_w,
                     pg_result* host_out, void* stream);

/* pg_forward with HOST inputs: copies them to plan-owned device buffers on
 * `stream` first (pinned host memory makes the copies asynchronous). */
pg_status pg_forward_host(pg_plan* plan, int64_t n_gal, const double* h_pos,
                          const float* h_vel, const float* h_w,
                          pg_result* host_out, void* stream);

/* The Gauss-sigmoid weighting function of Sec. 3.6 (eq. weighting):
 * W(r_perp, r_par) = 1 / (1 + exp(-s0 (r_perp - r_s))) *
 * exp(-(r_perp^2 + r_par^2) / (2 sigma^2)) for r_perp >= r_cut and 0 inside
 * that cylinder around the line of sight (z); r_perp, r_par are the offsets
 * perpendicular and parallel to z. The paper's normalisation cancels and is
 * taken as 1. Table tab:weightings: (30, 20, 0.8, 10) for d_p,max = 10 Mpc/h,
 * (50, 35, 0.5, 20) for 30 Mpc/h. */
typedef struct pg_smooth_params {
  double sigma;   /* Mpc/h, > 0 */
  double r_s;     /* Mpc/h */
  double s0;      /* h/Mpc */
  double r_cut;   /* Mpc/h, >= 0 */
} pg_smooth_params;

/* Host outputs of pg_forward_smooth, P = n_s * n_mu pair bins. */
typedef struct pg_smooth_result {
  int64_t* dd;     /* [P] pairs per (s, mu) bin */
  double* xi_ss;   /* [P] xi(s, mu) = DD/RR - 1 */
  double* num;     /* [P] weighted mean of (W * delta_g) over the bin's pair midpoints (weights w_i w_j) */
  double* b_pg;    /* [P] num / den (eq. bpg_final); NaN for an empty bin */
  double* q_eff;   /* [P] eq. Qeff_notsq with xi(d_p) = xi_ss and xi(d_w) below */
  double* den;     /* [1] weighted mean of (W * delta_g) over the galaxies (weights w_j) */
  double* xi_dw;   /* [1] eq. xi_dw: sum_r W C_gg^2 / sum_r W C_gg over the mesh offsets */
} pg_smooth_result;

/* The paper's own estimator (Sec. 2.1 eq. bpg_final) with the smooth W of
 * Sec. 3.6: the galaxy overdensity is assigned to the plan's mesh (its NGP /
 * CIC / TSC choice), convolved once with W by FFT (G = W * delta_g, k = 0
 * removed), and G is interpolated with the same assignment weights at every
 * pair midpoint and every galaxy. For each (s, mu) pair bin of the plan,
 * b_pg is the ratio of the weighted means of G over the bin's pairs and over
 * the galaxies (the mean times the volume is the sum divided by the number
 * density), so all pair bins cost O(1) FFTs. xi(d_w) is eq. xi_dw with the
 * measured galaxy auto-correlation C_gg; Q_eff is eq. Qeff_notsq. The plan's
 * correlation bins are not used. Inputs as pg_forward (device positions,
 * optional velocities and weights); W's spectrum is computed on the first
 * call and kept in the plan while *w stays the same. Errors:
 * PG_ERR_INVALID_ARG (NULL plan, parameters, outputs or positions, sigma
 * <= 0, r_cut < 0, non-finite values, RSD without velocities),
 * PG_ERR_UNSUPPORTED, PG_ERR_OOM, PG_ERR_CUDA, PG_ERR_TIMEOUT. Synchronises
 * the stream. A pg_backward after this call returns PG_ERR_INVALID_ARG. */
pg_status pg_forward_smooth(pg_plan* plan, const pg_smooth_params* w, int64_t n_gal, const double* d_pos,
                            const float* d_vel, const float* d_w, pg_smooth_result* host_out,
                            void* stream);

/* Adjoint of the last successful pg_forward_smooth call on this plan (same
 * catalogue, still held in the plan's buffers): with the upstream gradients
 * in *grad_out (HOST arrays in the pg_smooth_result layout; the fields
 * xi_ss, num, b_pg, q_eff [P], den, xi_dw [1] are read, NULL means zero, dd is
 * ignored), writes d_grad_w[n_gal] (device FP64) = dL/dw_i for L = sum over
 * fields and bins of grad * output, outputs that are NaN contributing
 * nothing. The reverse sweep follows the forward's steps backwards (Sec. 2.1
 * eq. bpg_final, Sec. 3.6 eq. weighting, eqs. xi_dw, Qeff_notsq,
 * 2PCF_d_collapsed): ratio outputs -> the bin means and xi -> the adjoint
 * weights of G = W * delta_g at the pair midpoints and galaxies, deposited on
 * the mesh (the transpose of the interpolation) -> the W convolution (W is
 * real and even, so the operator is its own adjoint) together with the xi_w
 * term delta_bar += (2 / N^3) Cbar * delta (Cbar = d xi_w / d C_gg) in one
 * k-space combination -> the rho / Q normalisation at the galaxies and the
 * pair-weight chain w_p = w_i w_j. Without weights in the forward call the
 * gradient is taken at w = 1. The Q32.32 rounding of the deposit is treated
 * as exact. Errors: PG_ERR_INVALID_ARG if no smooth forward call preceded
 * (or another entry point reused the plan since), PG_ERR_UNSUPPORTED,
 * PG_ERR_OOM, PG_ERR_CUDA, PG_ERR_TIMEOUT. Synchronises the stream. */
pg_status pg_backward_smooth(pg_plan* plan, const pg_smooth_result* grad_out, double* d_grad_w, void* stream);

/* Adjoint of the last successful pg_forward / pg_forward_host call on this
 * plan (same catalogue, still held in the plan's buffers): with the upstream
 * gradients in *grad_out (HOST arrays in the pg_result layout; the fields
 * xi_pg, xi_gg, b_pg, q_eff, q_eff_sq, xi_dw, b_pg_agg, q_eff_agg, xi_dw_agg,
 * xi_ss, dd_w and, on the (d_perp, d_par) grid, w_perp are read, NULL means
 * zero, other fields are ignored), writes
 * d_grad_w[n_gal] (device FP64) = dL/dw_i for L = sum over fields and bins of
 * grad * output, outputs that are NaN contributing nothing. The reverse sweep
 * follows the forward definitions (Sec. 2.1 eqs. bpg_initial /
 * bpg_intermediate, Sec. 2.2 eqs. xi_dw, Qeff, Qeff_notsq, Sec. 3.4): ratio
 * outputs -> bin sums -> window fields -> mesh adjoints by FFT correlation ->
 * pair and galaxy weights -> w_i through w_p = w_i w_j. The galaxy and pair
 * spectra are recomputed, not stored; pair meshes go in the forward's
 * batches. Without weights in the forward call the gradient is taken at
 * w = 1. Errors: PG_ERR_INVALID_ARG if no forward call preceded (or a stage
 * entry point reused the plan since), PG_ERR_UNSUPPORTED if the window side
 * 2w+1 (w = ceil(r_max / (L/N))) exceeds 256 or the batched adjoint's shared
 * tiles do not fit (FP64 at N = 1024: 2w+1 <= 151), PG_ERR_OOM, PG_ERR_CUDA,
 * PG_ERR_TIMEOUT. Synchronises the stream. */
pg_status pg_backward(pg_plan* plan, const pg_result* grad_out, double* d_grad_w, void* stream);

/* Soft occupation weights of candidate galaxies under the five-parameter HOD
 * of Sec. 3.3 (eq. hod), theta = (log10 M_cut, log10 M_1, sigma, alpha,
 * kappa) in h_theta[5] (host):
 *   kind 0 (central at the halo centre):  w = erfc(ln(M_cut/M)/(sqrt(2) sigma)) / 2
 *   kind 1 (one of K satellite candidates of the halo):
 *            w = ((M - kappa M_cut)/M_1)^alpha / K  for M > kappa M_cut, else 0
 * d_mass [n] FP64 halo mass (Msun/h), d_kind [n] int32, d_kh [n] FP32 K (any
 * value for centrals); writes d_w [n] FP32 and, if d_dw_dtheta is not NULL,
 * d_dw_dtheta [n][5] FP64 = dw/dtheta. All device. Errors: PG_ERR_INVALID_ARG
 * (sigma <= 0, NULL arrays). */
pg_status pg_hod_weights(int64_t n, const double* d_mass, const int32_t* d_kind, const float* d_kh,
                         const double* h_theta, float* d_w, double* d_dw_dtheta, void* stream);

/* h_grad_theta[5] (host) = sum_i d_wbar[i] * d_dw_dtheta[i][k]: the chain from
 * weight gradients (pg_backward) to the HOD parameters. Uses the plan's
 * workspace; synchronises the stream. */
pg_status pg_hod_chain(pg_plan* plan, int64_t n, const double* d_wbar, const double* d_dw_dtheta,
                       double* h_grad_theta, void* stream);

/* pg_hod_weights with the second derivatives as well: d_d2w_dtheta2 [n][15]
 * FP64 device, the upper triangle j <= k of d2w/dtheta_j dtheta_k in row
 * order (00 01 02 03 04 11 12 13 14 22 23 24 33 34 44), from the chain rule
 * through eq. hod's closed forms. The satellite weight's second derivatives
 * in log10 M_cut and kappa are unbounded at M = kappa M_cut when alpha < 2
 * (the weight is not twice differentiable there). All outputs required. */
pg_status pg_hod_weights2(int64_t n, const double* d_mass, const int32_t* d_kind, const float* d_kh,
                          const double* h_theta, float* d_w, double* d_dw_dtheta,
                          double* d_d2w_dtheta2, void* stream);

/* Sec. 5, eqs. 2pf_emulate_1st and 2pf_emulate_2nd: the first and second
 * derivatives of the pair-count statistics with respect to the HOD
 * parameters, which the paper solves for from 14 separate evaluations, here
 * exact from the soft weights' derivatives in one pass over the pairs. The
 * call enumerates the pairs of the catalogue (positions d_pos [n][3] FP64,
 * d_vel [n][3] FP32 for RSD plans, else NULL) with the plan's pair binning,
 * then, with w = d_w [n] FP32 (the weights the forward would use, widened),
 * dw = d_dw_dtheta [n][5] and d2w = d_d2w_dtheta2 [n][15] (pg_hod_weights2):
 *   DD_b = sum over the pairs of bin b of w_i w_j (FP64 products), R =
 *   ((sum w)^2 - sum w^2)/2, xi_b = DD_b / (R V_b / L^3) - 1 (eq.
 *   2PCF_d_collapsed), and on the (d_perp, d_par) grid w(d_perp)_k =
 *   sum_m 2 (l_hi - l_lo) xi_{k,m} (eq. 2PCF_los_integrated_explicit),
 * each with its derivatives by the product and quotient rules. Outputs
 * (host): h_xi [P][21] per pair bin and h_w_perp [n_s][21] (may be NULL;
 * NaN unless the plan bins on the grid), each row [value, d/dtheta_j (5),
 * d2/dtheta_j dtheta_k (15, upper triangle as above)]. Sums are FP64 in a
 * fixed order. The plan's pair buffers are reused, so a following
 * pg_backward needs a new pg_forward. Synchronises the stream. Errors:
 * PG_ERR_INVALID_ARG for NULL arguments, RSD without velocities, or
 * positions holding NaN or Inf. */
pg_status pg_hod_pair_derivs(pg_plan* plan, int64_t n, const double* d_pos, const float* d_vel,
                             const float* d_w, const double* d_dw_dtheta, const double* d_d2w_dtheta2,
                             double* h_xi, double* h_w_perp, void* stream);

/* Low-level form of the estimator for two arbitrary point sets (Sec. 2.1,
 * eq. bpg_initial): deposits set a and set b, correlates them, and bins
 * C_ab(r) = (1/N^3) sum_x delta_b(x) delta_a(x + r) by (r, mu_r).
 * Positions are device [n][3] FP64 already inside [0, L); weights device FP64
 * or NULL. Writes host arrays h_sum[Q], h_sum2[Q] (sum C, sum C^2 per bin),
 * h_agg[2] (over the aggregate cells) and h_ncells[Q]; any may be NULL. */
pg_status pg_correlate_points(pg_plan* plan,
                              int64_t n_a, const double* d_pts_a, const double* d_w_a,
                              int64_t n_b, const double* d_pts_b, const double* d_w_b,
                              double* h_sum, double* h_sum2, double* h_agg,
                              int64_t* h_ncells, void* stream);

/* ---- stage entry points (each row of the path on its own) -------------- */

/* Sec. 3.2, eq. RSD: wraps positions into [0, L) and, when rsd_factor != 0,
 * shifts z to wrap(z + rsd_factor * v_z). d_in [n][3] FP64, d_vel [n][3]
 * FP32 or NULL, d_out [n][3] FP64 (may alias d_in). */
pg_status pg_transform_positions(int64_t n, double box_L, double rsd_factor,
                                 const double* d_in, const float* d_vel,
                                 double* d_out, void* stream);

/* Sec. 3.3 (all pairs closer than s_max, every pair of a triplet kept) and
 * Sec. 2.1 (a pair sits at its midpoint): cell-list enumeration of all
 * unordered pairs of the wrapped positions d_pos [n][3] with s in
 * [s_edges[0], s_edges[n_s]), binned by (s, mu). For a pair of input indices
 * i < j: d = min-image(x_j - x_i), midpoint wrap(x_i + d/2), weight w_i*w_j.
 * Outputs (device, caller-owned): d_dd[P] int64 pair counts, d_ddq[P] int64
 * sums of llrint(w_i w_j 2^32). If capacity > 0 the pairs are also written,
 * grouped by bin in ascending bin order (order inside a bin unspecified):
 * d_bin[cap] int32, d_i[cap], d_j[cap] int32, d_mid[cap][3] FP64,
 * d_wp[cap] FP64. *h_n_pairs (host) receives the total; PG_ERR_CAPACITY if it
 * exceeds capacity (counts are still valid). Uses `plan` for its binning and
 * box; the plan's mesh is not used. Synchronises the stream. */
pg_status pg_find_pairs(pg_plan* plan, int64_t n, const double* d_pos,
                        const float* d_w, int64_t* d_dd, int64_t* d_ddq,
                        int64_t capacity, int32_t* d_bin, int32_t* d_i,
                        int32_t* d_j, double* d_mid, double* d_wp,
                        int64_t* h_n_pairs, void* stream);

/* Sec. 3.5: NGP/CIC/TSC mass assignment of n points (device [n][3] FP64 in
 * [0, L)) with weights (device FP64 or NULL = 1) into a dense device mesh
 * d_mesh[N][N][N] int64 of Q32.32 node weights llrint(((w wx) wy) wz 2^32),
 * ADDED to its current contents (zero it first for a fresh mesh). Exact and
 * order independent. */
pg_status pg_deposit_dense(int64_t n, const double* d_pts, const double* d_w,
                           double box_L, int32_t mesh_n, int32_t assign,
                           int64_t* d_mesh, void* stream);

/* Sec. 3.5 as the estimator itself deposits: the compact-line mass
 * assignment the forward path runs on each batch of pair meshes (line
 * flags, their scan, the line numbering and the Q32.32 int64 atomics into
 * the touched x-lines), with the plan's mesh and assignment, exposed so that
 * its integer meshes can be compared bit for bit. d_pts [n][3] FP64 device
 * (inside [0, L)), d_w [n] FP64 device or NULL (= 1); d_bin [n] int32 device,
 * the mesh of each point in [0, nb), or NULL for one mesh (nb = 1);
 * 1 <= nb <= the plan's pair meshes per batch. Writes d_mesh[nb][N][N][N]
 * int64 (device, caller-owned, overwritten): the compact lines scattered
 * back to dense meshes (untouched lines are zero); h_qsum[nb] (host, may be
 * NULL): each mesh's total; *h_n_lines (host, may be NULL): the number of
 * touched lines. Uses the plan's workspace; synchronises the stream.
 * Errors: PG_ERR_INVALID_ARG for a NULL plan, mesh or points, nb out of
 * range, d_bin NULL with nb != 1, or a d_bin entry outside [0, nb) (checked
 * on the device before the deposit). */
pg_status pg_deposit_lines(pg_plan* plan, int64_t n, const double* d_pts, const double* d_w,
                           const int32_t* d_bin, int32_t nb, int64_t* d_mesh, int64_t* h_qsum,
                           int64_t* h_n_lines, void* stream);

/* Sec. 3.6 (the transforms the estimator is built on): forward real-to-
 * complex 3D DFT F(k) = sum_x f(x) exp(-2 pi i k.x / N) of a dense mesh
 * d_in[N][N][N] (FP32 if precision 0, FP64 if 1) into the half spectrum
 * d_out[N][N][N/2+1] (complex64 / complex128 interleaved, kx contiguous),
 * through the same pass kernels as the estimator. Needs a plan with this
 * mesh_n and precision (its workspace is used). Synchronises the stream;
 * PG_ERR_TIMEOUT if a bounded device wait of a column pass gave up. */
pg_status pg_fft_r2c_3d(pg_plan* plan, const void* d_in, void* d_out, void* stream);

/* Inverse of the above, unnormalised: f(x) = sum_k F(k) exp(+2 pi i k.x / N)
 * over the Hermitian-completed spectrum. d_in is not modified. Synchronises
 * the stream; PG_ERR_TIMEOUT as above. */
pg_status pg_fft_c2r_3d(pg_plan* plan, const void* d_in, void* d_out, void* stream);

/* Pair counts DD(s, mu) of one catalogue, like the counts of pg_find_pairs,
 * for callers that cannot allocate device memory: code running under a
 * framework whose caching allocator owns the whole device budget, or a
 * latency-critical host thread that must not take the device-wide
 * synchronisation cudaMalloc / cudaFree can cause. This call allocates
 * nothing and needs no plan: its cell-list scratch is a fixed array of about
 * 8.4 MB compiled into the library, which every GPU that loads the library
 * holds until the process exits. (The paper has no counterpart; this is a
 * deployment variant of the pair enumeration.)
 *   n <= 131072 galaxies, else PG_ERR_CAPACITY. d_pos [n][3] FP64 device,
 *   already inside [0, L); d_w [n] FP32 device or NULL; s_edges [n_s+1] host,
 *   ascending, s_edges[n_s] < box_L/2; d_dd, d_ddq [n_s*n_mu] int64 device
 *   outputs (zeroed by the call): pair counts and sums of
 *   llrint(w_i w_j 2^32). Positions holding NaN or Inf give
 *   PG_ERR_INVALID_ARG (as in pg_forward): the call synchronises `stream`
 *   once to read that check back, then launches the rest asynchronously.
 * The first call on a device looks up the scratch array's device address for
 * that device; make that first call before any stream capture. The address is
 * kept for the life of the process and does not survive a reset of the
 * device (cudaDeviceReset): do not call this entry point on a device after
 * resetting it. All calls share the one array, so calls that overlap on the
 * GPU (different streams or host threads) race and must be serialised by the
 * caller. */
pg_status pg_pair_counts_static(int64_t n, const double* d_pos, const float* d_w,
                                double box_L, int32_t n_s, const double* s_edges,
                                int32_t n_mu, int64_t* d_dd, int64_t* d_ddq, void* stream);

/* ---- measurement ---------------------------------------------------------- */

/* Kernel families of the path, in the order of pg_plan_last_stats. */
enum {
  PG_FAM_POSITIONS = 0,   /* wrap, RSD, finiteness check, weight sums */
  PG_FAM_CELLS,           /* cell-list counting sort */
  PG_FAM_PAIRS,           /* pair counting, pair list, grouping by bin */
  PG_FAM_DEPOSIT,         /* line flags, line numbering, Q32.32 deposit */
  PG_FAM_FFT_X_R2C,       /* x pass, real to complex */
  PG_FAM_FFT_Y_FWD,       /* y pass forward (writes the dense spectra) */
  PG_FAM_FFT_Z_FWD,       /* z pass forward of the galaxy spectrum */
  PG_FAM_FFT_Z_CORR,      /* z pass: forward, times conj(F_g), inverse, window */
  PG_FAM_FFT_Y_INV,       /* y pass inverse on the window */
  PG_FAM_FFT_X_C2R,       /* x pass complex to real on the window */
  PG_FAM_BIN,             /* (r, mu_r) sums */
  PG_FAM_RATIOS,          /* xi, b_pg, Q_eff */
  PG_FAM_ADJ_RATIOS,      /* adjoint: ratios -> bin-sum adjoints */
  PG_FAM_ADJ_WINDOW,      /* adjoint: window fields, their x and y passes */
  PG_FAM_ADJ_Z,           /* adjoint z pass: A += F_b conj(X_b), z inverse of X_b F_g */
  PG_FAM_ADJ_Y_INV,       /* adjoint: y inverse at the pair lines */
  PG_FAM_ADJ_X_C2R,       /* adjoint: x C2R of the pair lines */
  PG_FAM_ADJ_GATHER,      /* adjoint: interpolation at the pairs, chain to w_i */
  PG_FAM_ADJ_GALAXY,      /* adjoint: galaxy side (inverse of A, gather, final) */
  PG_FAM_SMOOTH,          /* smooth-W estimator: W spectrum, convolutions, interpolation, sums */
  PG_N_FAMILIES
};

typedef struct pg_kernel_stat {
  char name[24];          /* family name */
  int64_t launches;       /* kernel launches in the last profiled call */
  double ms;              /* their summed duration: CUDA events on the call's stream */
  double bytes;           /* algorithmic bytes they must move (reads + writes) */
} pg_kernel_stat;

/* One mock of a many-mock batch: its own problem and HOST catalogue (as in
 * pg_forward_host) and host outputs laid out for its params. */
typedef struct pg_mock {
  pg_params params;     /* edge arrays must stay valid during the call */
  int64_t n_gal;
  const double* h_pos;  /* [n_gal][3] */
  const float* h_vel;   /* [n_gal][3] or NULL */
  const float* h_w;     /* [n_gal] or NULL */
  pg_result* out;
} pg_mock;

typedef struct pg_batch_stats {
  double wall_ms;       /* the whole call, host clock */
  double mocks_per_s;   /* completed mocks / wall */
  double p50_ms;        /* per-mock latency, median: from the mock's turn (waiting */
  double p99_ms;        /*   for its plan included) to its results on the host */
  int32_t n_plans;      /* plans built (one per distinct problem) */
  int32_t n_workspaces; /* shared mesh scratch built (one per mesh_n x precision) */
  int64_t gpu_launches; /* kernels launched by the mocks' forward calls */
} pg_batch_stats;

/* Many mocks of uneven size (box, mesh, catalogue; the batching pattern of a
 * survey-scale HOD study, Sec. 3.3) through the forward path, in order, on
 * `stream`. Plans are built per distinct problem by a host thread that runs
 * up to two mocks ahead of the GPU, and share mesh scratch per (mesh_n,
 * precision), so the device holds one scratch per mesh size; the plans are
 * freed before return. A non-blocking stream lets plan building overlap the
 * GPU work. latency_ms [n_mocks] (host, may be NULL) receives each mock's
 * latency (NaN if it failed); *stats (may be NULL) the batch statistics.
 * Returns the first failing mock's status (the others still run). Errors:
 * PG_ERR_INVALID_ARG for a NULL mock array, a NULL output or positions. */
pg_status pg_run_batch(const pg_mock* mocks, int32_t n_mocks, double* latency_ms,
                       pg_batch_stats* stats, void* stream);

/* pg_run_batch with n_streams runners (1..8; 1 is pg_run_batch): runner
 * threads, each with its own non-blocking stream, plans and mesh scratch (one
 * per mesh size and precision: the device holds n_streams times the scratch
 * of pg_run_batch), claim the next mock from one work queue and run its
 * forward, so one mock's host work (plan building, the readbacks of pair and
 * line counts that size its launches) overlaps another's GPU work. The
 * runners start after the work queued on `stream` and `stream` waits for
 * them. Outputs, latency and stats as in pg_run_batch (latency from a mock's
 * claim to its results on the host); a mock that fails leaves the others
 * running. Errors: those of pg_run_batch, PG_ERR_INVALID_ARG for n_streams
 * out of range, PG_ERR_CUDA if a stream or event cannot be created. */
pg_status pg_run_batch_streams(const pg_mock* mocks, int32_t n_mocks, int32_t n_streams, double* latency_ms,
                               pg_batch_stats* stats, void* stream);

/* Batch-size autotuner: times one forward (after one warm-up) of the given
 * problem and HOST catalogue for each candidate bins_per_batch and writes the
 * fastest to *best (ms_out [n_cand], host, may be NULL: each candidate's
 * time, CUDA events on `stream`). Candidate plans share scratch, which grows
 * to the largest candidate. Errors: PG_ERR_INVALID_ARG (NULL params,
 * candidates or best, n_cand <= 0, a candidate <= 0), those of
 * pg_plan_create and pg_forward_host. */
pg_status pg_autotune(const pg_params* params, int64_t n_gal, const double* h_pos,
                      const float* h_vel, const float* h_w, const int32_t* candidates,
                      int32_t n_cand, int32_t* best, double* ms_out, void* stream);

/* Failure-detection test of the device waits: one CTA waits on an mbarrier
 * that nothing completes, with the same bounded wait the TMA-fed kernels use
 * (there 2 s), here limit_ms (0 < limit_ms <= 5000). Returns PG_ERR_TIMEOUT
 * when the wait gives up, which is the expected outcome; the context stays
 * usable. PG_ERR_INVALID_ARG for a NULL plan or a limit out of range. */
pg_status pg_selftest_wait(pg_plan* plan, double limit_ms, void* stream);

/* Enables (1) or disables (0) per-family event timing on later calls of
 * pg_forward / pg_forward_host / pg_backward on this plan. */
pg_status pg_plan_set_profiling(pg_plan* plan, int32_t enable);

/* Statistics of the last pg_forward / pg_forward_host / pg_backward call
 * (pg_backward's include the recomputed forward passes): out[PG_N_FAMILIES]
 * (host; times are 0 unless profiling was enabled) and *total_launches, the
 * number of kernels that call launched (always counted). Either may be NULL. */
pg_status pg_plan_last_stats(const pg_plan* plan, pg_kernel_stat* out, int64_t* total_launches);

#ifdef __cplusplus
}
#endif

#endif /* PAIRGAL_H */

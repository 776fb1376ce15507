/* libpolybin -- binned power spectrum and bispectrum estimators on a periodic 3D grid, one GB300 (sm_103a).
 *
 * Method: PolyBin3D, O. H. E. Philcox & T. Floss, arXiv 2404.07249.  The library computes, with hand-written
 * CUDA kernels:
 *   - the shell-filtered maps g_b = IFT[Theta_b FT[delta]] (Sec. 4.3.1, eq. g-ell-def, global line of sight);
 *   - the triplet sums S_abc = sum_x g_a g_b g_c and their normalisation N_abc from unit fields
 *     (eqs. beta-def, N-ell-def) and the ideal bispectrum (Sec. 4.4.1, eqs. bk-num-ideal, bk-fish-ideal2);
 *   - the Legendre-weighted power spectrum multipoles along the last grid axis (Sec. 3.4.1, eq. pk-limit,
 *     eq. fish-ideal-continuous).
 *
 * Conventions shared by every entry point:
 *   - Grids are C-order arrays [N0][N1][N2]; the line of sight is the last (fastest) axis.  Every N_i must be
 *     even and have no prime factor other than 2, 3, 5, with N_i <= 1024.  The box is cubic (one side L for all
 *     axes); boxsize[0..2] must be equal.
 *   - k-bins are half-open [e_b, e_{b+1}) in |k| (h/Mpc), k = 0 never binned; 1 <= n_kbins <= 64, ascending edges.
 *   - Inputs are float32 real fields.  A field pointer may be device memory (read in place) or host memory
 *     (pinned or pageable; copied to the device inside the call).  Outputs are float64 on the host.
 *   - The caller owns every input and output buffer; the context owns its device workspace, plans and caches.
 *   - All work runs on the CUDA stream given to polybin_init (borrowed, not owned); each call synchronises that
 *     stream before returning, so outputs are valid on return.  A context must not be used by two host threads
 *     at once.
 *   - Every int-returning function returns a polybin_status; on failure polybin_last_error() describes it.
 *     Nothing throws across this interface.
 */
#ifndef POLYBIN_H
#define POLYBIN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct polybin_ctx polybin_ctx;

typedef enum {
    POLYBIN_OK = 0,
    POLYBIN_EINVAL = -1,    /* bad argument: null pointer, unsupported grid, bad edges, ... */
    POLYBIN_ENOMEM = -2,    /* device or host allocation failed */
    POLYBIN_ECUDA = -3,     /* a CUDA call or kernel launch failed */
    POLYBIN_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
    POLYBIN_ENOTREADY = -5, /* a prerequisite (e.g. a Fisher matrix) has not been computed */
    POLYBIN_ETOL = -6       /* a self-check exceeded its tolerance */
} polybin_status;

typedef enum {
    POLYBIN_FP64 = 0,         /* FP64 FFTs and FP64 contraction: the plain double-precision GPU path        */
    POLYBIN_FP32 = 1,         /* FP32 FFTs, FP32 SIMT contraction with FP64 flushes and FP64 cross-CTA sums  */
    POLYBIN_SPLIT_TF32X3 = 2  /* FP32 FFTs, tensor-core contraction with 3-term split TF32 products          */
} polybin_prec;

/* Create a context for one grid and one set of k-bins.
 * grid[3]      : N0, N1, N2 (see conventions).
 * boxsize[3]   : box side in Mpc/h (all three equal).
 * k_edges      : n_kbins + 1 ascending edges in h/Mpc (host memory, copied).
 * l_max        : largest even Legendre order of the power spectrum (0, 2 or 4).
 * prec         : a polybin_prec value.
 * cuda_stream  : cudaStream_t to run on (NULL = legacy default stream).
 * The first POLYBIN_SPLIT_TF32X3 context on a device runs a one-MMA self-check on known operands: the split scheme
 * takes the tensor core's reading of an FP32 operand (its 13 low bits dropped) as the high part of the maps; if the
 * device reads it otherwise, polybin_init returns POLYBIN_ETOL (for this and every later split context there).
 * On success *out receives the context (destroy with polybin_destroy); on failure *out is NULL and
 * polybin_last_error(NULL) describes the error. */
int polybin_init(polybin_ctx** out, const int grid[3], const double boxsize[3], const double* k_edges,
                 int n_kbins, int l_max, int prec, void* cuda_stream);

/* Release the context and all its device memory.  NULL is accepted. */
void polybin_destroy(polybin_ctx* ctx);

/* Message of the last failure on ctx (or of the last failed polybin_init on this thread when ctx is NULL).
 * The string is owned by the library and valid until the next call on the same context. */
const char* polybin_last_error(const polybin_ctx* ctx);

/* ---- bispectrum (Sec. 4.4.1) ------------------------------------------------------------------------------ */

/* Number of closed triplets a <= b <= c (N_abc > 0).  The first call computes N_abc on the GPU in FP64
 * (eq. N-ell-def via unit-field shell maps) and caches it in the context. */
int polybin_num_triplets(polybin_ctx* ctx, int* n);

/* The closed triplets in lexicographic (a, b, c) order (abc: [n][3] ints, host) and, if n_abc is not NULL,
 * their closed-triangle counts N_abc = N^2 T_abc (host, [n] doubles; exact integers). */
int polybin_get_triplets(polybin_ctx* ctx, int* abc, double* n_abc);

/* Ideal bispectrum monopole of `batch` fields delta ([batch][N0][N1][N2] float32, device or host):
 * B_abc = (V^2 / N^3) S_abc / T_abc in (Mpc/h)^6 for every closed triplet (Sec. 4.4.1: b_num = S / Delta and
 * F = N_abc / (N Delta) in pixel units, so Delta cancels).  bk_out: host [batch][n_triplets]. */
int polybin_bk_ideal(polybin_ctx* ctx, const float* delta, int batch, double* bk_out);

/* Ideal bispectrum multipoles ell = 0, 2, .., lmax_b (lmax_b = 0, 2 or 4) about the global line of sight (the last
 * grid axis), Sec. 4.1 eqs. Bk-Yam and ideal-bk with the ideal continuous Fisher of Sec. 4.4.1 (eq. bk-fish-ideal2,
 * under which Delta_alpha cancels):
 *   B_ell(a, b, c) = (2 ell + 1) (V^2 / N^3) S^ell_abc / T_abc,  S^ell_abc = sum_x g_a g_b g_{c,ell},
 *   g_{c,ell} = IFT[Theta_c L_ell(mu) D]  (eq. g-ell-def, global line of sight; mu = k_z / |k| of the mode in the
 *   third bin c, the largest, as eq. ideal-bk places it),
 * over the closed triplets of polybin_get_triplets (N_0 = N_abc).  ell = 0 is polybin_bk_ideal.  delta: as
 * polybin_bk_ideal; bk_out: host [batch][lmax_b / 2 + 1][n_triplets].  The Legendre-weighted maps take a second
 * set of contraction-grid maps (allocated on the first call with lmax_b > 0). */
int polybin_bk_ideal_multipoles(polybin_ctx* ctx, const float* delta, int batch, int lmax_b, double* bk_out);

/* The same multipoles with a local line of sight (Sec. 4.3.1, eq. g-ell-def and its expansion in normalised real
 * spherical harmonics): g_{c,ell} = IFT[Theta_c sum_m Ybar_lm(k) FT[Ybar_lm(x) delta]], the direction x / |x| from
 * the observer of polybin_set_observer at every cell (cell centres as for the local P estimator), 2 ell + 1 forward
 * transforms per ell > 0 and field; normalised as polybin_bk_ideal_multipoles.  Same arguments and layout.  Not part
 * of the paper's printed estimator set (its ideal estimator, eq. ideal-bk, takes a global line of sight); the local
 * maps are those its unwindowed estimators use. */
int polybin_bk_ideal_multipoles_local(polybin_ctx* ctx, const float* delta, int batch, int lmax_b, double* bk_out);

/* Ideal bispectra of n_fields fields on possibly different grids (e.g. a batch of 96^3, 128^3 and 160^3
 * realisations).  ctxs[i] is the context of field i (fields on one grid share a context; all contexts must use
 * one stream, that of ctxs[0]); fields[i]: device float32 [N0][N1][N2] of ctxs[i]; bk_out[i]: host
 * [n_triplets(ctxs[i])], as polybin_bk_ideal.  The whole batch is captured into one CUDA graph on a private
 * stream and replayed with a single graph launch, ordered after the work already queued on the contexts' stream;
 * the graph is cached in ctxs[0] for repeated calls with the same contexts and field pointers (a call with other
 * arguments re-captures).  Profiling must be off. */
int polybin_bk_ideal_multi(polybin_ctx* const* ctxs, const float* const* fields, int n_fields, double* const* bk_out);

/* ---- power spectrum (Sec. 3.4.1) ------------------------------------------------------------------------- */

/* Ideal P_ell (ell = 0, 2, .., l_max) with the continuous-limit Fisher normalisation (eq. fish-ideal-continuous):
 * P_ell(b) = (2 ell + 1) (V / N^2) sum_{k in b} L_ell(mu) |D(k)|^2 / N_b, mu = k_z / |k|, D = DFT(delta).
 * pk_out: host [batch][l_max/2 + 1][n_kbins] in (Mpc/h)^3. */
int polybin_pk(polybin_ctx* ctx, const float* delta, int batch, double* pk_out);

/* Same numerator with the discrete ideal Fisher of eq. pk-limit, F_{ell ell'}(b) = (1/2) sum_{k in b} L_ell L_ell',
 * solved per bin (couples the multipoles through grid discreteness).  Same output layout as polybin_pk. */
int polybin_pk_discrete(polybin_ctx* ctx, const float* delta, int batch, double* pk_out);

/* Mode counts N_b of the full k-grid (host [n_kbins] doubles). */
int polybin_mode_counts(const polybin_ctx* ctx, double* counts);

/* Both statistics of the same fields from one forward transform: bk_out as polybin_bk_ideal, pk_out as
 * polybin_pk (continuous normalisation).  Either output may be NULL to skip that statistic.  With host memory and
 * batch > 1 the fields are staged through two device buffers on a copy stream, the copy of field f + 1 overlapping
 * the transforms of field f (pinned memory overlaps; pageable memory is copied synchronously by the driver). */
int polybin_bk_pk_ideal(polybin_ctx* ctx, const float* delta, int batch, double* bk_out, double* pk_out);

/* ---- masked ("unwindowed") estimators, global line of sight ------------------------------------------------
 * Data model (Sec. 2.3, eqs. data-model, pointing; pixel window m = 1, no noise): d = n delta with background
 * density n(x) (the pointing matrix P = n).  Weighting S^-1 = w(x) (Sec. 2.4), e.g. FKP w = 1 / (1 + n P_FKP).
 * Fields n, w, d and mocks are float32 DEVICE arrays [N0][N1][N2] owned by the caller.  Monte Carlo maps are
 * unit Gaussian white noise (A = I) from Philox4x32-10 + Box-Muller: map `draw` of `stream` holds at flat cell
 * i the value z_{i mod 4} of Philox block j = i / 4 with key (seed mod 2^32, seed / 2^32) and counter
 * (j mod 2^32, j / 2^32, draw, stream); z0, z1 = sqrt(-2 ln u0) (cos, sin)(2 pi u1), z2, z3 likewise from
 * u2, u3, u_q = (x_q + 1/2) 2^-32.  Streams 0 and 1 give the bispectrum Fisher pairs (a1, a2), stream 2 the
 * power-spectrum Fisher draws.  Parameter index alpha: power spectrum (ell, b) ell-major, index
 * (ell / 2) * n_kbins + b; bispectrum the closed triplets in polybin_get_triplets order. */

enum { POLYBIN_FISHER_PK = 0, POLYBIN_FISHER_BK = 1, POLYBIN_FISHER_PK_LOCAL = 2, POLYBIN_FISHER_PK_OPT = 3 };

/* w = 1 / (n P_FKP + 1) (Sec. 2.4, eq. Sinv-fkp), evaluated in FP64 and stored as float32 (device arrays). */
int polybin_fkp_weights(polybin_ctx* ctx, const float* n_dev, double p_fkp, float* w_dev);

/* The Monte Carlo map `draw` of `stream` (float32 device array [N]), as defined above. */
int polybin_mc_draw(polybin_ctx* ctx, unsigned long long seed, int draw, int stream, float* out_dev);

/* Monte Carlo Fisher matrix averaged over draws 0 .. n_mc-1 and its FP64 inverse (LU with partial pivoting on the
 * GPU), cached in the context for polybin_pk_unwindowed / polybin_bk_unwindowed.
 *   which = POLYBIN_FISHER_PK: F_ab = 1/2 <(P^T S^-T Q_a[S^-1 P a]) . Q^asym_b[a]> (Sec. 3.3.2, eq. fish-from-Q);
 *   which = POLYBIN_FISHER_BK: F_ab = 1/24 <(Q_a[S^-1 P a1] - Q_a[S^-1 P a2]) . S^-1 P . (Q_b[a1] - Q_b[a2])>
 *                              (Sec. 4.3.4, eqs. bk-fish-def, Q-bis-global), pixel units.
 * fisher_out, fisher_inv_out: host [n_alpha][n_alpha] row major, may be NULL.  checkpoint_path (may be NULL): the
 * running FP64 sum is saved after every draw and a matching file is resumed from (same grid, bins, mode, seed and
 * mask; the result is bit-identical to an uninterrupted run); a corrupted or mismatched file gives POLYBIN_EINVAL. */
int polybin_fisher(polybin_ctx* ctx, const float* n_dev, const float* w_dev, int n_mc, unsigned long long seed,
                   int which, double* fisher_out, double* fisher_inv_out, const char* checkpoint_path);

/* The per-draw Fisher terms of draws draw_begin .. draw_end-1 (host [draw_end - draw_begin][n_alpha][n_alpha]); the
 * mean over all draws is the Fisher matrix.  Independent replicas can each compute a range of draws. */
int polybin_fisher_draws(polybin_ctx* ctx, const float* n_dev, const float* w_dev, unsigned long long seed, int which,
                         int draw_begin, int draw_end, double* per_draw_out);

/* Install a Fisher matrix computed elsewhere (host [n_alpha][n_alpha]); its inverse is computed in FP64 on the GPU. */
int polybin_set_fisher(polybin_ctx* ctx, int which, const double* fisher);

/* ---- local (Yamamoto) line of sight, Sec. 3.1 eqs. cf-pk-def, xi-p-alpha-deriv and Sec. 3.3 ----------------------
 * The line of sight of a pair is taken at each end point, x / |x| from the observer, symmetrised; the Legendre
 * polynomials are expanded in normalised real spherical harmonics, sum_m Ybar_lm(a) Ybar_lm(b) = L_l(a.b) (the set of
 * the footnote of Sec. 3.3.1 up to signs within each l, which cancel in every sum the estimators take).  Cell centres
 * are at (i + 1/2) L / N_a - L / 2 (the box centred on the origin).  Even multipoles ell = 0 .. l_max. */

/* Observer position in box coordinates (Mpc/h, box centred on the origin; default (0, 0, 0), the box centre).  A
 * local Fisher matrix computed for another observer is discarded. */
int polybin_set_observer(polybin_ctx* ctx, const double pos[3]);

/* which = POLYBIN_FISHER_PK_LOCAL in polybin_fisher / polybin_fisher_draws / polybin_set_fisher: the P Fisher matrix
 * with the local line of sight (Sec. 3.3.2, eq. fish-from-Q with Q_alpha of eq. Q-alpha-local and the asymmetric
 * Q^asym_alpha[a](k) = Theta_b sum_m Ybar_lm(k) FT[Ybar_lm a](k)), alpha as for POLYBIN_FISHER_PK.  Per draw it takes
 * (l_max + 1)^2 forward transforms of the draw, as many of S^-1 P a, 2 l + 2 sets of n_kbins inverse transforms per
 * ell > 0 and one forward transform per alpha. */

/* Unwindowed P_ell with a local line of sight: p_num_alpha = 1/2 (1/N) sum_{k in b} sum_m Ybar_lm(k)
 * Re(conj(FT[Ybar_lm w d](k)) FT[w d](k)) (Sec. 3.3.1, eq. pk-num-fft, pixel units), p = F^-1 p_num with the local
 * Fisher matrix, pk_out = p V / N (host [n_alpha], may be NULL; needs polybin_fisher(POLYBIN_FISHER_PK_LOCAL) or
 * polybin_set_fisher first).  pnum_out: host [n_alpha] or NULL.  d, w: device arrays as for polybin_pk_unwindowed. */
int polybin_pk_unwindowed_local(polybin_ctx* ctx, const float* d_dev, const float* w_dev, double* pk_out,
                                double* pnum_out);

/* Unwindowed P_ell (Sec. 3.2, eq. pk-estimator-def):
 * p_num_alpha = 1/2 (1/N) sum_{k in b} L_ell |FT[w d]|^2 (pixel units), p = F^-1 (p_num - p_bias), pk_out = p V / N
 * (host [n_alpha]; needs polybin_fisher(POLYBIN_FISHER_PK) or polybin_set_fisher first, may be NULL).  p_bias is the
 * shot-noise bias last computed by polybin_pk_bias for POLYBIN_FISHER_PK (zero if none).  pnum_out: host [n_alpha] or
 * NULL (the numerator without the bias). */
int polybin_pk_unwindowed(polybin_ctx* ctx, const float* d_dev, const float* w_dev, double* pk_out, double* pnum_out);

/* Unwindowed bispectrum (Sec. 4.2, eq. bk-estimator-def, with the numerator of eq. b-numerator-practical):
 * b_num_abc = (S_abc[w d] - lin_abc) / Delta_abc, lin_abc = mean over the n_mocks mocks of
 * sum_x (g_a[u] g_b[v] g_c[v] + g_a[v] g_b[u] g_c[v] + g_a[v] g_b[v] g_c[u]), u = w d, v = w mock;
 * b = F^-1 b_num, bk_out = b (V/N)^2 (host [n_triplets]; needs the BK Fisher, may be NULL).  mocks_dev: device
 * [n_mocks][N] or NULL when n_mocks = 0.  bnum_out, lin_out: host [n_triplets] or NULL. */
int polybin_bk_unwindowed(polybin_ctx* ctx, const float* d_dev, const float* w_dev, const float* mocks_dev, int n_mocks,
                          double* bk_out, double* bnum_out, double* lin_out);

/* The closed-triplet plan of the split-TF32 contraction (after the first estimate; -1 before) and the autotuner's
 * choice.  info: [0] tile cost of the tile-cutting DP, [1] tiles a row group may take, [2] cell split (0: one CTA per
 * SM and row group; 1: one wave of SMs / groups CTAs a group; 2: two CTAs per SM and group), [3] row groups, [4] CTAs
 * per group, [5] candidates timed (0: not tuned).  ms: the chosen plan's time per launch on the tuning inputs.  The
 * autotuner runs on the first contraction outside stream capture: every distinct valid candidate is launched twice
 * on the caller's inputs and the fastest kept (POLYBIN_AUTOTUNE=0 in the environment keeps the default plan).  Not
 * part of the paper's interface. */
int polybin_contract_plan_info(polybin_ctx* ctx, int info[6], float* ms);

/* ---- optimal weighting by preconditioned conjugate gradients ------------------------------------------------------
 * Sec. 2.4, eq. cgd-operation-eqn and the transpose equation beside it; Sec. 3.3.3, eq. Sinv-optimal in the
 * distant-observer limit.  Data model d = n delta + eps, C = P xi P^T + N with P = diag(n), N = diag(n2) (pixel window
 * m = 1) and xi = IFT[P(k) FT[.]], P(k) = sum_ell P_ell(k) L_ell(mu) about the global line of sight.  On the cells
 * with n_w > 0 (Phi = 1) S^-1 solves n_w IFT[P FT[Phi S^-1 v]] + (n2_w / n_w) Phi S^-1 v = v: with
 * A = Phi (IFT[P FT[.]] + n2_w / n_w^2) Phi (symmetric positive definite there) and G = A^-1 on that subspace,
 *     S^-1 v = G (v / n_w),    S^-T v = G (v) / n_w,
 * zero where n_w = 0.  IFT[P FT[u]] is taken with the unnormalised forward DFT and the 1/N inverse (the exact
 * discretisation of int dy int_k e^{ik(x-y)} P(k) u(y)): n_w, n2_w are densities and P_ell powers in matching units.
 * G comes from conjugate gradients preconditioned with the ideal weighting of eq. Sinv-ideal (the exact inverse for a
 * uniform density), M^-1 r = Phi IFT[FT[Phi r] / (P(k) + sigma)], sigma = mean of n2_w / n_w^2 over the cells with
 * n_w > 0.  Each iteration costs two pruned forward and two pruned inverse transforms plus four map passes; dot
 * products accumulate in FP64.  Not part of the paper's interface: the weighting is configured once per context. */

/* The largest binned |n|^2 (integer wave numbers): fiducial tables may have up to smax + 1 entries. */
int polybin_max_shell(polybin_ctx* ctx, int* smax);

/* Configure the optimal weighting.  n_w_dev, n2_w_dev: float32 device arrays [N] (copied; n2_w_dev = NULL takes
 * n2_w = n_w, the Poisson noise of a unit-weight catalogue).  pfid: host [nell_fid][n_s] FP64, pfid[l][s] the fiducial
 * multipole ell = 2 l on the shell |n|^2 = s (|k| = k_F sqrt(s)), zero for s >= n_s; 1 <= nell_fid <= 3,
 * 1 <= n_s <= smax + 1 (P vanishes beyond the binned range, so both Fourier operators act on the pruned box of
 * binned wave numbers).  P(k, mu) + sigma must be > 0 on every box mode (POLYBIN_EINVAL otherwise).  The iteration
 * stops when ||r|| <= tol ||b|| (tol > 0: one host read-back per iteration) or after max_iter iterations (tol = 0:
 * exactly max_iter iterations, no read-back inside the loop).  Replaces any earlier configuration; a Fisher matrix of
 * POLYBIN_FISHER_PK_OPT computed with another configuration is no longer used. */
int polybin_set_optimal(polybin_ctx* ctx, const float* n_w_dev, const float* n2_w_dev, const double* pfid, int nell_fid,
                        int n_s, int max_iter, double tol);

/* out = S^-1 v (transpose = 0) or S^-T v (transpose = 1).  v_dev: float32 device [N]; out_dev: device [N] of the
 * context's working type (double for POLYBIN_FP64, float otherwise), zero where n_w = 0.  iters_out, relres_out (may
 * be NULL): iterations taken and the final ||r|| / ||b|| of the recursively updated residual.  POLYBIN_ENOTREADY
 * without polybin_set_optimal; POLYBIN_ETOL if the iteration breaks down (a non-finite residual: the operator was not
 * positive definite). */
int polybin_sinv_optimal(polybin_ctx* ctx, const float* v_dev, int transpose, void* out_dev, int* iters_out,
                         double* relres_out);

/* which = POLYBIN_FISHER_PK_OPT in polybin_fisher / polybin_fisher_draws / polybin_set_fisher: the P Fisher matrix of
 * eq. fish-from-Q with the optimal weighting, S^-1 P a = G (n a / n_w) and P^T S^-T u = n G (u) / n_w for the
 * pointing density n = n_dev (w_dev is not used and may be NULL); 1 + n_alpha solves per draw.  alpha as for
 * POLYBIN_FISHER_PK. */

/* Unwindowed P_ell with the optimal weighting: p_num_alpha = 1/2 (1/N) sum_{k in b} L_ell |FT[S^-1 d]|^2, p = F^-1
 * (p_num - p_bias) with the POLYBIN_FISHER_PK_OPT Fisher matrix and bias (polybin_pk_bias), pk_out = p V / N (host [n_alpha], may be NULL; POLYBIN_ENOTREADY
 * if that Fisher matrix is missing or belongs to another configuration).  pnum_out: host [n_alpha] or NULL. */
int polybin_pk_unwindowed_opt(polybin_ctx* ctx, const float* d_dev, double* pk_out, double* pnum_out);

/* ---- Poisson shot noise of the P numerator ----------------------------------------------------------------------
 * Data model d = n delta + eps with <eps eps^T> = diag(n2 / V_cell) (eq. two-point-noise, m = 1; n2 the density of the
 * doubly-weighted sample, n2 = n for unit weights).  p_bias_alpha = 1/2 <(S^-1 N a) . Q^asym_alpha[S^-1 a]>_a (Sec.
 * 3.3.2, first line of eq. fish-from-Q, A = I, global line of sight), averaged over the Monte Carlo maps r = 0 ..
 * n_mc-1 of stream 3: one Monte Carlo term is 1/2 (1/N) sum_{k in b} L_ell Re conj(FT[S^-1 N a]) FT[S^-1 a] (pixel
 * units, as p_num).  which = POLYBIN_FISHER_PK: S^-1 = w (w_dev); which = POLYBIN_FISHER_PK_OPT: the optimal weighting
 * of polybin_set_optimal (w_dev unused; two solves per map).  The result is cached for that mode and subtracted by
 * polybin_pk_unwindowed / polybin_pk_unwindowed_opt until replaced; n_mc = 0 clears it (n2_dev may then be NULL).
 * bias_out: host [n_alpha] or NULL. */
int polybin_pk_bias(polybin_ctx* ctx, const float* n2_dev, const float* w_dev, int which, int n_mc,
                    unsigned long long seed, double* bias_out);

/* ---- Poisson shot noise of the B numerator ----------------------------------------------------------------------
 * Sec. 4.3.3 (eq. three-point-noise and the Monte Carlo form after it), FKP weighting S^-1 = w, ell = 0, global line
 * of sight.  The noise is split as N_ijk = -2 N3_ijk + (d_i N2_jk + 2 perms), N3[u, v] = n3 u v / V_cell^2 and
 * N2 u = d2 u / V_cell (n3: the three-point noise density; d2: the doubly-weighted data minus randoms; n3 = n and
 * d2 = d for unit weights), and
 *     b_bias = -1/3 <beta[w N3[a1, a2], w a1, w a2]> + 1/2 <beta[w N2 a1, w a1, w d]>
 * over the Monte Carlo pairs r = 0 .. n_mc-1 of streams 4 and 5, beta of eq. beta-def (six assignments of the maps to
 * the bins, 1 / Delta), in the units of b_num.  Each pair costs six forward transforms, six sets of shell maps and
 * six contractions of 2 n_kbins by n_kbins maps (n_kbins <= 32).  Fields are float32 device arrays [N].
 * bias_out: host [n_triplets]. */
int polybin_bk_bias(polybin_ctx* ctx, const float* n3_dev, const float* d2_dev, const float* d_dev, const float* w_dev,
                    int n_mc, unsigned long long seed, double* bias_out);

/* polybin_bk_unwindowed with the shot noise removed: b = F^-1 (b_num - b_bias), b_bias of polybin_bk_bias for this d
 * (the bias depends on the data through its second term, so it is computed with the estimate).  bk_out, bnum_out
 * (without the bias), bias_out: host [n_triplets] or NULL. */
int polybin_bk_unwindowed_shot(polybin_ctx* ctx, const float* d_dev, const float* w_dev, const float* mocks_dev,
                               int n_mocks, const float* n3_dev, const float* d2_dev, int n_mc, unsigned long long seed,
                               double* bk_out, double* bnum_out, double* bias_out);

/* X = A^-1 B in FP64 on the GPU (dense LU with partial pivoting).  A: host [n][n], B, X: host [n][nrhs], row major.
 * POLYBIN_EINVAL if A is exactly singular. */
int polybin_solve(polybin_ctx* ctx, const double* A, int n, const double* B, int nrhs, double* X);

/* ---- instrumentation -------------------------------------------------------------------------------------- */

/* Enable (on != 0) or disable per-stage timing.  When enabled, each pipeline stage is bracketed by a pair of CUDA
 * events on the context stream.  Recording does not block the host: the elapsed times are read back when
 * polybin_get_stage_times is called, or when 64 brackets have accumulated.  Stages enqueued during a stream
 * capture are not timed.  The first enable creates 128 events (POLYBIN_ECUDA if that fails). */
int polybin_set_profiling(polybin_ctx* ctx, int on);

/* Accumulated device milliseconds and call counts of the stages since the last reset (reset != 0 clears them
 * after reading); waits for the stop events of brackets still in flight.  Stage order: 0 forward transform (a1), 1 shell filter + inverse transforms (a2),
 * 2 triplet contraction (a3), 3 P_ell binning (a4).  ms and calls: host arrays of 4 (calls may be NULL). */
int polybin_get_stage_times(polybin_ctx* ctx, double* ms, long long* calls, int reset);

/* Number of kernels this context has launched so far. */
int polybin_launch_count(const polybin_ctx* ctx, long long* n);

/* The contraction kernel that ran last on this context: POLYBIN_SPLIT_TF32X3 contexts use the tensor-core kernel
 * whenever the shape allows it (<= 512 pairs, <= 32 singles a call, 16-byte aligned maps) and the FP32 SIMT kernel
 * otherwise; this call tells which one produced the last result.  *path = -1 before the first contraction. */
enum { POLYBIN_PATH_SIMT_FP64 = 0, POLYBIN_PATH_SIMT_FP32 = 1, POLYBIN_PATH_TENSOR_SPLIT_TF32X3 = 2 };
int polybin_last_path(const polybin_ctx* ctx, int* path);

/* Lengths of the grid the bispectrum's triplet sums are evaluated on (host int[3]).  Every shell map has wave
 * numbers |n_i| <= m on each axis (m: the largest component of a binned mode), so the product of three maps has
 * |n_i| <= 3m and its sum over the cells of any grid with more than 3m points per axis is the same up to the factor
 * (cells of the data grid) / (cells of that grid).  The library evaluates the maps g_b = IFT[Theta_b D] (with the
 * data grid's 1/N) and the triplet sums on the smallest such grid whose lengths have no prime factor other than 2,
 * 3, 5 (the data grid's length on an axis where 3m + 1 would not be shorter), and rescales: the outputs are those
 * of the data grid (Sec. 4.3.1, eq. beta-def, and Sec. 4.4.1 on the data grid).  Outputs of polybin_shell_maps and
 * polybin_contract stay on the data grid. */
int polybin_contraction_grid(const polybin_ctx* ctx, int dims[3]);

/* Failure-detection self-test: one kernel waits on an mbarrier phase that nothing completes, using the same bounded
 * poll as the tensor-core pipeline, and another on a barrier armed for a bulk staging copy that is never issued,
 * using the bounded wait of the transform passes' staging; each wait gives up after 2^14 polls and sets its device
 * error flag, the kernels return and the context stays usable (the flags are cleared afterwards).
 * *timed_out = 1 when both bounded waits gave up (the expected outcome). */
int polybin_selftest_wait(polybin_ctx* ctx, int* timed_out);

/* ---- individual steps, for testing and composition (device pointers only) --------------------------------- */

/* Dimensions [Bx][By][Bz] of the pruned half-spectrum box: all wave numbers n with |n_x|, |n_y| <= m and
 * 0 <= n_z <= m, where m is the largest |n_i| of any binned mode (full axis when 2m + 1 > N_i). */
int polybin_spectrum_shape(const polybin_ctx* ctx, int dims[3], int lo[3]);

/* Step a1: forward real-to-complex DFT of one field, pruned to the box.  delta: device float32 [N0][N1][N2];
 * spec_out: device [Bx][By][Bz] complex (interleaved re, im) of float (FP32 modes) or double (FP64 mode);
 * element (ix, iy, iz) holds D(n = (lo[0] + ix, lo[1] + iy, lo[2] + iz)) = sum_x e^{-i k.x} delta(x). */
int polybin_forward(polybin_ctx* ctx, const float* delta, void* spec_out);

/* Step a2: shell maps g_b(x) = IFT[Theta_b D](x) (with the 1/N of the inverse DFT) for every bin, from a box
 * spectrum laid out as polybin_forward writes it.  g_out: device [n_kbins][N0][N1][N2] float (FP32 modes) or
 * double (FP64 mode). */
int polybin_shell_maps(polybin_ctx* ctx, const void* spec, void* g_out);

/* Step a3: M[p][i] = sum_x g_{j_p}(x) g_{k_p}(x) h_i(x) for all pairs p = (j <= k) in lexicographic order and all
 * i.  g: device [n_g][N] maps, h: device [n_h][N] maps or NULL (h = g, n_h = n_g); element type as for
 * polybin_shell_maps.  m_out: host [n_g (n_g + 1) / 2][n_h] doubles.  n_g, n_h <= 64. */
int polybin_contract(polybin_ctx* ctx, const void* g, int n_g, const void* h, int n_h, double* m_out);

/* ---- allocation-free contraction -----------------------------------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that cannot allocate device memory (code
 * running inside a caller-managed memory pool or arena, plugins whose host application owns every allocation,
 * threads that must not call cudaMalloc/cudaFree because those can synchronise the device).
 * It computes the same M[p][i] = sum_x g_{j_p}(x) g_{k_p}(x) h_i(x) as polybin_contract (FP32 SIMT kernel) without a
 * context and without allocating: its scratch (FP64 per-block partial sums and the pair tables of every n <= 64) is
 * a fixed file-scope device array of 2^21 doubles (16 MiB) plus 179 KiB, held by every GPU that loads the library
 * until the process exits.
 *   g: device float32 [n_g][ncell]; h: device float32 [n_h][ncell] or NULL (h = g); 1 <= n_g, n_h <= 64 and
 *   n_g (n_g + 1) / 2 * n_h <= 2^21 (larger requests return POLYBIN_EINVAL, as do pointers that are not device
 *   memory).  m_out_dev: device float64 [n_g (n_g + 1) / 2][n_h], written on cuda_stream (a cudaStream_t; NULL =
 *   legacy default stream).
 * Asynchronous: the call returns after enqueueing; synchronise the stream before reading m_out_dev.  The first call
 * on a device looks up the scratch address (cudaGetSymbolAddress), fills the pair tables with a kernel and waits for
 * it: make that first call before any stream capture.  Every call on a device shares the scratch, which keeps the
 * last call's contents (each call overwrites all it reads, so nothing needs clearing): calls that overlap on the
 * GPU (other streams, or other host threads) race and must be serialised by the caller.
 * Errors: polybin_contract_noalloc_error() describes the last failure on the calling host thread. */
int polybin_contract_noalloc(const float* g, int n_g, const float* h, int n_h, long long ncell, double* m_out_dev,
                             void* cuda_stream);
const char* polybin_contract_noalloc_error(void);

#ifdef __cplusplus
}
#endif

#endif /* POLYBIN_H */

/*
 * pr.h -- C ABI of the micro-macro parareal hot path on one GB300 (sm_103a).
 *
 * Method: Legoll, Lelievre, Myerscough, Samaey, "Parareal computation of
 * stochastic differential equations with time-scale separation: a numerical
 * study" (arXiv:1912.09240).  Section numbers below refer to that paper.
 *
 * Conventions shared by every call
 *  - Pointers marked (device) are caller-owned device memory; pointers marked
 *    (host) are caller-owned host memory.  No call keeps a pointer after it
 *    returns, except the handles created by pr_coarse_create.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous on that stream unless stated otherwise.
 *  - Arguments are validated on the host before anything is launched; a bad
 *    argument returns PR_ERR_INVALID_ARG and launches nothing.  A failed
 *    launch returns PR_ERR_CUDA.  Conditions found on the device (a NaN in the
 *    FP64 update, an empty macroscopic state) are written to a caller-provided
 *    int32 status word (device) and read by the caller after synchronising.
 *  - Every device array must be aligned to its element size (4 bytes for
 *    float, uint32 and int32, 8 for double and int64); a misaligned pointer
 *    returns PR_ERR_INVALID_ARG.  Workspaces state their own alignment.
 *  - Ensembles are stored as structure of arrays, slice-major:
 *      x[n_slices][n]            slow variable X^p
 *      y[n_slices][fast_dim][n]  fast variable Y^p (component-major)
 *    in float (PR_F32) or double (PR_F64).  Weights are uniform, W^p = 1/n,
 *    except where a call takes them (Section 5.2 calls, pr_moments).
 *  - A macroscopic state (a histogram of the slow variable on a uniform grid
 *    x_lo = e_0 < ... < e_I = x_hi, Section 2.2.2) is passed as its
 *    piecewise-linear CDF sampled at the I+1 edges (Eq. discr_cdf), double,
 *    C_0 = 0, C_I = 1, bin masses rho_i = C_{i+1} - C_i.
 *  - No call allocates device memory except pr_coarse_create; calls that need
 *    scratch take it from the caller (workspace arguments), except
 *    pr_fine_adjoint_noalloc, which uses a fixed array inside the library.
 *  - Calls on distinct handles are thread-safe.
 */
#ifndef PR_H
#define PR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PR_OK = 0,
    PR_ERR_INVALID_ARG = 1,
    PR_ERR_CUDA = 2,
    PR_ERR_TIMEOUT = 3,
    PR_ERR_UNSUPPORTED = 4,
    PR_ERR_NOMEM = 5,
    PR_ERR_NUMERIC = 6
} pr_status;

typedef enum { PR_F32 = 0, PR_F64 = 1 } pr_precision;

/* Drift families of the slow-fast SDE (Section 2.1.1, Eqs. SDEx/SDEy), tau_x
 * the slow time scale, D = 1/beta, fast potential G = |y - x|^2/2 per
 * component, E = 1:
 *   PR_MODEL_OU          d_x F = x - lambda*y             (fast_dim = 1)
 *   PR_MODEL_DOUBLE_WELL d_x F = x^3 - x + lambda*y       (fast_dim = 1)
 *   PR_MODEL_DW_MULTI    d_x F = x^3 - x + lambda*mean(y) (fast_dim 1..16)
 *   PR_MODEL_ADVECTION   no microscopic model (pr_coarse_create only): the coarse
 *                        potential Fbar(x) = x/eps, diffusion 1/beta -- the linear
 *                        advection case of Section 6
 * and the chemically reacting system of Section 2.1.2 (fast_dim = 1, rates
 * k0..k5 in pr_model.rate; lambda and beta unused), with
 *   D = (k4 y + k5 x)/2,  E = (k0 + k1 y + k2 y(y-1) + k3 y(y-1)(y-2))/2
 * (half the total propensities of the reactions 0 -> Y, Y -> 0, 2Y -> 3Y,
 * 3Y -> 2Y, Y -> Y + X, X -> 0), the square roots taking max(2D, 0) and
 * max(2E, 0), and the drifts
 *   PR_MODEL_CHEM         the net rates of those reactions (chemical Langevin
 *                         form): -d_x F = k4 y - k5 x,
 *                         -d_y G = k0 - k1 y + k2 y(y-1) - k3 y(y-1)(y-2)
 *   PR_MODEL_CHEM_PRINTED the derivatives of the potentials as printed
 *                         (Eqs. F_Bruna, G_Bruna): d_x F = -k4 y - k5 x,
 *                         d_y G = -k0 - k1 y + k2 y(y-1) - k3 y(y-1)(y-2).
 * Its coarse model (Section 2.2.3) averages over the fast equilibrium
 * phi(y) ~ exp(-int_0^y G'/E) / E through its mean ybar, taken by the
 * trapezoidal rule on y = 0, 1/2, ..., 2000 (pr_coarse_create). */
typedef enum {
    PR_MODEL_OU = 0,
    PR_MODEL_DOUBLE_WELL = 1,
    PR_MODEL_DW_MULTI = 2,
    PR_MODEL_ADVECTION = 3,
    PR_MODEL_CHEM = 4,
    PR_MODEL_CHEM_PRINTED = 5
} pr_model_kind;

/* Iterators of Section 4: quantile (4.4), additive (4.1), multiplicative
 * (4.2), rotation (4.3); PR_ITER_NONE keeps the coarse result (the serial
 * coarse sweep of the zeroth iteration, Section 3.2.4). */
typedef enum {
    PR_ITER_QUANTILE = 0, PR_ITER_ADD = 1, PR_ITER_MULT = 2, PR_ITER_ROT = 3, PR_ITER_NONE = 4
} pr_iterator;

/* Quantile of a CDF at a level it takes on a flat stretch (Section 4.4):
 * TWO_SIDED keeps both ends of the stretch as knots (J(a,b,a) = b holds
 * exactly); MIDPOINT takes the midpoint, as the paper prints it. */
typedef enum { PR_QMODE_TWO_SIDED = 0, PR_QMODE_MIDPOINT = 1 } pr_quantile_mode;

/* Resampling of Section 5.2: stratified points u_j = (j + u~_j)/N with u~_j
 * uniform (Eq. stratified), or the deterministic variant u~_j = 1/2. */
typedef enum { PR_RESAMPLE_STRATIFIED = 0, PR_RESAMPLE_DETERMINISTIC = 1 } pr_resample_mode;

typedef struct {
    int32_t kind;       /* pr_model_kind */
    int32_t fast_dim;   /* d, the dimension of Y */
    double lambda;      /* coupling strength */
    double beta;        /* inverse temperature of the slow variable, D = 1/beta */
    double eps;         /* fast time scale */
    double tau_x;       /* slow time scale */
    double rate[6];     /* k0..k5 of the chemical system (other kinds ignore them) */
} pr_model;

typedef struct {
    int32_t bins;       /* I, 1 .. 4096 */
    double x_lo, x_hi;  /* x_lo < x_hi */
} pr_grid;

typedef struct {
    uint64_t seed;        /* Philox4x32-10 key (low word, high word) */
    uint32_t problem_id;  /* < 2^24, selects an independent family of streams */
} pr_rng;

/* Human-readable name of a status code (static storage). */
const char* pr_status_string(pr_status s);

/* Library version, e.g. "0.1.0". */
const char* pr_version(void);

/*
 * Fine propagator F_dT (Section 3.2.1; Euler-Maruyama, Section 2.1.3,
 * Eqs. EMx/EMy) over the slices slice_begin .. slice_begin + n_slices - 1 at
 * once, each advanced by `steps` steps of size dt.
 *
 * Random numbers: slice n, particle p, step m draw their 1 + fast_dim standard
 * normals (Box-Muller) from Philox4x32-10 with key = seed and counter
 *   fast_dim == 1 : (m >> 1, p, n, problem_id << 8), step m taking words
 *                   2(m&1), 2(m&1)+1 (one block serves two steps);
 *   fast_dim  > 1 : with Q = 1 + fast_dim, F = Q / 4, t = Q mod 4: normals
 *                   4g .. 4g+3 of step m (g < F) from (m, p, n,
 *                   (problem_id << 8) | g), words in pairs, each pair giving
 *                   a cosine and a sine normal; the last t normals of the
 *                   steps 4k .. 4k+3 share t blocks (k, p, n,
 *                   (problem_id << 8) | (F + j)), normal i of step 4k + s
 *                   being number s t + i of their 4t normals in order;
 * so a slice reuses the same numbers in every parareal iteration (Section 6).
 *
 *   x_in, y_in   (device) start states, [n_slices][n] and [n_slices][d][n];
 *                with broadcast_input != 0 a single ensemble [n], [d][n] is
 *                the start of every slice (the zeroth iteration).
 *   x_out, y_out (device) end states, same layout as the non-broadcast input;
 *                may alias x_in / y_in exactly (in-place), not partially, and
 *                not at all with broadcast_input (PR_ERR_INVALID_ARG).
 *   grid         needed when any of the fused outputs below is requested.
 *   cdf_prior, cdf_target (device, [n_slices][bins+1]) or both NULL: fused
 *                matching (pr_match) applied to the start state first; its
 *                table shares the CTA's shared memory with the histograms
 *                (about 76 bins bytes in binary32, 44 bins in binary64).  In
 *                binary32 on a grid whose table does not fit (more than
 *                about 3050 bins on GB300) the call runs the same steps in
 *                turn: pr_match into x_out, the restriction of the matched
 *                states, y copied to y_out, the propagation in place; every
 *                grid up to 4096 bins is served in both precisions.
 *   counts_start, cdf_start (device, [n_slices][bins], [n_slices][bins+1]) or
 *                NULL: restriction (pr_restrict) of the start state after the
 *                matching.  cdf_start needs counts_start.
 *   counts_end, cdf_end: restriction of the end state.  cdf_end needs counts_end.
 * Counts are overwritten (the call zeroes them first).
 * Precision PR_F32: float state, FP32 arithmetic; PR_F64: double throughout.
 */
pr_status pr_fine_propagate(const pr_model* model, pr_precision precision, const pr_rng* rng,
                            const void* x_in, const void* y_in, int32_t broadcast_input,
                            void* x_out, void* y_out,
                            int64_t n, int32_t slice_begin, int32_t n_slices,
                            int32_t steps, double dt,
                            const pr_grid* grid,
                            const double* cdf_prior, const double* cdf_target,
                            uint32_t* counts_start, double* cdf_start,
                            uint32_t* counts_end, double* cdf_end,
                            void* stream);

/*
 * Raw Philox4x32-10 blocks (Salmon et al., SC'11) with key = rng->seed:
 * out[i] = Philox(ctr[i]) for n counters.  The generator behind the EM
 * increments dU_m, dV_m ~ N(0, dt) (Eqs. EMx/EMy), exposed for checking.
 *   ctr (device) [n][4] uint32, out (device) [n][4] uint32, both 16-byte aligned.
 */
pr_status pr_rng_words(const pr_rng* rng, const uint32_t* ctr, int64_t n, uint32_t* out, void* stream);

/*
 * Tuning knob of the binary32 fine propagator with fast_dim = 1: particles
 * carried per thread.  1, 2 or 4 force that value; any other value (0, the
 * default) chooses per launch: 4, or 2 or 1 where a launch over
 * n x n_slices particles would otherwise have fewer threads than the device
 * holds resident (2048 per SM).  Process-wide.  Results do not depend on it.
 */
void pr_set_particles_per_thread(int32_t ppt);

/* Tuning knob of the same kernel: the most consecutive particle tiles one CTA
 * processes (1..64, default 8); the launch also keeps ~16 waves of CTAs.
 * Process-wide; results do not depend on it. */
void pr_set_tiles_per_cta(int32_t tiles);

/*
 * Restriction R = R2 o R1 (Section 3.2.2, Eq. binning): drop Y, bin X.
 * A particle belongs to the bin i with e_i <= x < e_{i+1}, decided by exact
 * comparison with the double edges e_i = x_lo + i*(x_hi - x_lo)/I; particles
 * below x_lo count in bin 0 and at or above x_hi in bin I-1.
 *   x      (device) [n_slices][n], float or double per `precision`
 *   counts (device) [n_slices][bins] uint32, overwritten
 *   cdf    (device) [n_slices][bins+1] or NULL: C_i = (#particles in bins < i)/n
 */
pr_status pr_restrict(pr_precision precision, const void* x, int64_t n, int32_t n_slices,
                      const pr_grid* grid, uint32_t* counts, double* cdf, void* stream);

/* CDF at the edges from counts: cdf[s][0] = 0, cdf[s][i+1] = sum_{j<=i} counts[s][j] / n. */
pr_status pr_counts_to_cdf(const uint32_t* counts, int64_t n, int32_t n_slices, int32_t bins,
                           double* cdf, void* stream);

/*
 * Matching that preserves the fast marginal (Section 5.1, Eq. transformation):
 * X = c^{-1}(cbar(Xbar)) with cbar the piecewise-linear CDF of the prior
 * histogram and c that of the target; Y is untouched (not an argument).
 * The inverse takes the lowest non-empty target bin whose upper CDF value
 * reaches cbar(Xbar).  On a bin where prior and target CDF agree at both
 * edges the map is the identity (strong projection, Eq. projection, holds bit
 * for bit).  Particles outside [x_lo, x_hi] move by the displacement of the
 * nearest edge.
 *   x_prior (device) [n_slices][n]; x_out (device) [n_slices][n], may alias x_prior
 *   cdf_prior, cdf_target (device) [n_slices][bins+1]
 * Each CTA holds the map's table in shared memory: about 76 bins bytes in
 * binary32 and 32 bins bytes in binary64.  In binary32 on a grid whose table
 * exceeds the shared memory one CTA can have (227 KB on GB300: about 3050
 * bins), each particle takes the binary64 map and its image is rounded to
 * binary32 (bound by the FP64 pipe); binary64 keeps no binary32 table and
 * covers every grid up to 4096 bins.
 */
pr_status pr_match(pr_precision precision, const void* x_prior, void* x_out, int64_t n,
                   int32_t n_slices, const pr_grid* grid,
                   const double* cdf_prior, const double* cdf_target, void* stream);

/*
 * Matching that preserves the conditional distribution (Section 5.2), step
 * one: reweighting, W^p = Wbar^p rho'_i / rhobar_i with i the bin of Xbar^p,
 * rhobar and rho the bin masses of cdf_prior and cdf_target.  Target mass in
 * bins without prior mass moves half to the nearest bin with prior mass on
 * each side (all of it to the only side that has one); a particle in a bin
 * without prior mass gets weight 0.  Positions are not touched.  Equal CDFs
 * leave the weights unchanged bit for bit.
 *   x_prior    (device) [n_slices][n] (binary32 or binary64), or [n] shared by
 *              all slices when broadcast_input is non-zero
 *   w_prior    (device) same layout as x_prior, double, or NULL (1/n each)
 *   cdf_prior, cdf_target (device) [n_slices][bins+1]
 *   w_out      (device) [n_slices][n] double
 */
pr_status pr_reweight(pr_precision precision, const void* x_prior, int32_t broadcast_input,
                      const double* w_prior, int64_t n, int32_t n_slices, const pr_grid* grid,
                      const double* cdf_prior, const double* cdf_target, double* w_out, void* stream);

/*
 * Step two: stratified resampling (Section 5.2, Eq. stratified) of n
 * weighted particles into n equally weighted ones.  Output j takes the
 * particle p with C_{p-1} <= U_j < C_p, where C_p are the cumulative weights
 * in fixed point (round(W 2^61) as 64-bit integers: exact in any summation
 * order), T = C_{n-1} and U_j = floor(T (j 2^24 + a_j) / (n 2^24)): a_j the
 * odd 24-bit integer of the uniform of word j mod 4 of Philox block
 * (floor(j/4), 0xFFFFFFFF, slice, problem_id << 8 | 0xFE) for PR_RESAMPLE_STRATIFIED,
 * 2^23 (u~ = 1/2) for PR_RESAMPLE_DETERMINISTIC; slice = slice_begin + s.
 * Equal weights give output j = particle j (strong projection).  T = 0 (no
 * weight) gives the identity as well.  Weights are probability weights: their
 * sum must stay below 8.
 *   x_in, y_in (device) [n_slices][n], [n_slices][fast_dim][n] (or one slice
 *              with broadcast_input), precision as given; may be NULL when the
 *              matching output is NULL
 *   w          (device) [n_slices][n] double
 *   index_out  (device) [n_slices][n] uint32 or NULL: the particle each output takes
 *   x_out, y_out (device) gathered states, same layouts as the inputs without
 *              broadcast, or NULL; not aliasing the inputs
 *   workspace  (device) >= pr_resample_workspace(n, n_slices) bytes, 256-byte aligned
 */
size_t pr_resample_workspace(int64_t n, int32_t n_slices);
pr_status pr_resample(pr_precision precision, int32_t fast_dim, const void* x_in, const void* y_in,
                      int32_t broadcast_input, const double* w, int64_t n, int32_t n_slices,
                      int32_t slice_begin, pr_resample_mode mode, const pr_rng* rng, uint32_t* index_out,
                      void* x_out, void* y_out, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Restriction with weights (Section 3.2.2, Eq. binning with weights W^p):
 * bin sums of the weights in the fixed point above (exact, any order), then
 * the CDF at the edges, C_i = (sum over bins < i) / (total) with C_0 = 0 and
 * C_bins = 1 (the uniform CDF i / bins when no particle has weight).
 *   x (device) [n_slices][n], or [n] shared by all slices when broadcast_input is non-zero
 *   w (device) [n_slices][n] double (probability weights)
 *   cdf (device) [n_slices][bins+1]
 *   workspace (device) >= pr_restrict_weighted_workspace(n_slices, bins) bytes, 8-byte aligned
 */
size_t pr_restrict_weighted_workspace(int32_t n_slices, int32_t bins);
pr_status pr_restrict_weighted(pr_precision precision, const void* x, int32_t broadcast_input, const double* w,
                               int64_t n, int32_t n_slices, const pr_grid* grid, double* cdf, void* workspace,
                               size_t workspace_bytes, void* stream);

/*
 * Monte Carlo estimator (Section 2.1.3, Eq. MCestimator) of the power
 * observables M = v^q, q = 1..max_order (max_order <= 4), of one coordinate v
 * of each slice's ensemble (the slow variable, or one fast component):
 *   out[s][q-1] = sum_p W^p (v^p)^q,
 * W^p = w[s][p] when w is given, else 1/n (taken as the sum divided by n).
 * Binary64 accumulation (each term added by one fused multiply-add) in a
 * fixed order that depends only on n and n_slices, so repeated calls return
 * the same bits.
 *   v (device) precision as given; slice s starts slice_stride elements after
 *     slice s-1 (n for x[n_slices][n]; fast_dim * n for component c of
 *     y[n_slices][fast_dim][n], passing y + c * n); slice_stride >= n when
 *     n_slices > 1
 *   w (device) [n_slices][n] double, or NULL for uniform weights
 *   out (device) [n_slices][max_order] double
 *   workspace (device) >= pr_moments_workspace(n, n_slices, max_order) bytes,
 *     8-byte aligned
 * PR_ERR_INVALID_ARG for max_order outside 1..4, a short or misaligned
 * workspace, or a stride that makes slices overlap.
 */
size_t pr_moments_workspace(int64_t n, int32_t n_slices, int32_t max_order);
pr_status pr_moments(pr_precision precision, const void* v, int64_t slice_stride, const double* w, int64_t n,
                     int32_t n_slices, int32_t max_order, double* out, void* workspace, size_t workspace_bytes,
                     void* stream);

/*
 * Coarse propagator C_dT (Section 2.2.2): finite volumes on the detailed-
 * balance form of the averaged Fokker-Planck equation (Eq. FPz_rewritten),
 * central differences for the fluxes, zero flux at x_lo and x_hi, and an
 * exact time integrator P = exp(A dT) (matrix exponential by scaling and
 * squaring, FP64, built on the device).  The averaged coefficients are those
 * of the fast OU equilibrium Y | x ~ N(x, 1): Fbar' = (1-lambda) x (PR_MODEL_OU),
 * x^3 - (1-lambda) x (double-well families), Dbar = 1/beta.
 * Allocates the I x I matrix on the current device; synchronises `stream`.
 *   handle (host) receives an opaque pointer; release with pr_coarse_destroy.
 */
pr_status pr_coarse_create(const pr_model* model, const pr_grid* grid, double slice_dt,
                           void** handle, void* stream);
pr_status pr_coarse_destroy(void* handle);

/* Copy P = exp(A dT) (row-major I x I doubles) into out (device). */
pr_status pr_coarse_matrix(void* handle, double* out, void* stream);

/*
 * Apply C_dT to n_vec macroscopic states: masses = diff(cdf_in), P @ masses
 * with masses <= 1e-10 set to 0 (below that level they are rounding noise of
 * the matrix exponential, and negative round-off goes with them), cumulative
 * sum normalised to unit mass.  With few states each one is spread over a
 * thread-block cluster of up to 8 CTAs (rows of P split between them); the
 * result does not depend on that split.
 *   cdf_in, cdf_out (device) [n_vec][bins+1]; must not overlap.
 */
pr_status pr_coarse_fp(void* handle, const double* cdf_in, double* cdf_out, int32_t n_vec,
                       void* stream);

/*
 * Serial update of Section 3.2.3 (Eq. mm_sequential), on one thread-block
 * cluster (8 CTAs by default, one CTA below 64 bins) that splits the FP64
 * work of each slice; the result does not depend on the cluster size:
 *   rho^0 = cdf0,
 *   rho^{n+1} = J(C_dT(rho^n), rho_f*[n], rho_c*[n]),  n = 0 .. n_slices-1,
 * with J the chosen iterator (Section 4; PR_ITER_NONE: rho^{n+1} = C_dT(rho^n)).
 * C_dT is evaluated exactly as pr_coarse_fp does, bit for bit, so that
 * equal arguments give equal coarse results (the exactness theorem,
 * Section 3.3.3, needs that).
 *   cdf0       (device) [bins+1]
 *   cdf_f_star (device) [n_slices][bins+1], R F(X_k^n)   (NULL for PR_ITER_NONE)
 *   cdf_c_star (device) [n_slices][bins+1], C(R X_k^n)   (NULL for PR_ITER_NONE)
 *   cdf_next   (device) [n_slices+1][bins+1], receives rho_{k+1}^0 .. rho_{k+1}^{n_slices}
 *   status     (device) int32 or NULL: 0 on success, PR_ERR_NUMERIC if a
 *              non-finite value or an empty state appeared, or if an input
 *              of the quantile iterator was not a CDF (a value outside
 *              [0, 1], or decreasing); the results are then unspecified.
 */
pr_status pr_parareal_update(void* coarse, pr_iterator iterator, pr_quantile_mode qmode,
                             int32_t n_slices, const double* cdf0, const double* cdf_f_star,
                             const double* cdf_c_star, double* cdf_next, int32_t* status,
                             void* stream);

/* CTAs of the cluster running pr_parareal_update: 1, 2, 4 or 8 (default);
 * other values select 8.  Process-wide; affects later calls only. */
void pr_set_update_cluster(int32_t ctas);

/*
 * One iterator J(a, b, c) on n_vec independent triples (Section 4), no coarse
 * step: out[v] = J(a[v], b[v], c[v]).  a = rho_c^{n+1}, b = rho_f^*, c = rho_c^*.
 *   a, b, c, out (device) [n_vec][bins+1]; status as for pr_parareal_update.
 */
pr_status pr_iterate(pr_iterator iterator, pr_quantile_mode qmode, const pr_grid* grid,
                     int32_t n_vec, const double* a, const double* b, const double* c,
                     double* out, int32_t* status, void* stream);

/*
 * Pathwise adjoint of the binary32 fine propagator with fixed noise (not in
 * the paper; the EM recursion of Section 2.1.3 differentiated backwards).
 * fast_dim = 1, families PR_MODEL_OU and PR_MODEL_DOUBLE_WELL.  The forward
 * pass takes exactly the steps and random numbers of pr_fine_propagate over
 * slices slice_begin .. slice_begin + n_slices - 1 in sequence (slice s + 1
 * starting where slice s ended), storing (x, y) every ckpt_every steps in
 * the workspace.  The backward pass runs the adjoint recursion from the last
 * step to the first, accumulating in FP64, with the states of each
 * checkpoint segment of L = min(ckpt_every, n_slices steps) steps obtained
 * in one of two ways:
 *  - reverse walk, when (1/(1 - dt/eps))^L (1/(1 - dt/tau_x))^L <= 2: from
 *    the exact state at the segment's end, each state is reconstructed from
 *    the next by inverting the Euler step with the same noise (drawn again);
 *    the reconstruction's rounding grows by at most that factor over a
 *    segment, giving sensitivities within about 1e-4 of the ensemble RMS of
 *    the exact replay's (measured 1e-5 .. 6e-5);
 *  - otherwise, exact replay: each segment is replayed up to the start of its
 *    last 12-step block (leaving sub-checkpoints every 12 steps in the
 *    workspace), each 12-step block replayed once more into shared memory;
 *    ckpt_every = 12 then trades memory (8 n B per 12 steps) for one replay
 *    less.
 *   x0, y0      (device) [n] float start states
 *   x_T, y_T    (device) [n] float end states, or NULL
 *   xbar_T      (device) [n] double dL/dX_T per particle, or NULL
 *   ybar_T      (device) [n] double dL/dY_T per particle, or NULL (= 0; needs xbar_T)
 *   grad        (device) with xbar_T: [3] = dL/d(lambda, beta, eps), summed over
 *               particles in a fixed order; without: [n][3] = dX_T^p/d(lambda, beta, eps)
 *   xbar_0, ybar_0 (device) [n] double dL/dX_0, dL/dY_0 (per particle: dX_T/dX_0, dX_T/dY_0
 *               without seeds), or NULL
 *   workspace   (device) >= pr_fine_adjoint_workspace(...) bytes, 256-byte aligned,
 *               caller-owned scratch: 8 n B per checkpoint, 8 n B per sub-checkpoint
 *               of one segment, 24 B per 128 particles of partial sums
 */
size_t pr_fine_adjoint_workspace(int64_t n, int32_t n_slices, int32_t steps, int32_t ckpt_every);
pr_status pr_fine_adjoint(const pr_model* model, const pr_rng* rng, const float* x0, const float* y0,
                          int64_t n, int32_t slice_begin, int32_t n_slices, int32_t steps, double dt,
                          int32_t ckpt_every, float* x_T, float* y_T, const double* xbar_T,
                          const double* ybar_T, double* grad, double* xbar_0, double* ybar_0,
                          void* workspace, size_t workspace_bytes, void* stream);

/*
 * pr_fine_adjoint for an observable L = sum_p (seed_scale / 2 (X_T^p)^2 +
 * seed_shift X_T^p), whose seed dL/dX_T^p = seed_scale X_T^p + seed_shift
 * depends only on the particle's own end state (not in the paper; the second
 * moment E[X_T^2] = (1/n) sum_p (X_T^p)^2 is seed_scale = 2/n, seed_shift = 0,
 * the mean is seed_scale = 0, seed_shift = 1/n).  The seed is taken inside the
 * adjoint after its forward pass, in binary64 and then rounded to binary32
 * as pr_fine_adjoint rounds a given xbar_T: the gradient is bit for bit that
 * of pr_fine_adjoint with xbar_T computed from the end states, without the
 * separate forward pass that computing them would take.  dL/dY_T = 0.
 *   seed_scale, seed_shift  finite (PR_ERR_INVALID_ARG otherwise)
 *   grad        (device) [3] = dL/d(lambda, beta, eps), fixed summation order
 *   other arguments as pr_fine_adjoint (same workspace size)
 */
pr_status pr_fine_adjoint_affine(const pr_model* model, const pr_rng* rng, const float* x0, const float* y0,
                                 int64_t n, int32_t slice_begin, int32_t n_slices, int32_t steps, double dt,
                                 int32_t ckpt_every, double seed_scale, double seed_shift, float* x_T,
                                 float* y_T, double* grad, double* xbar_0, double* ybar_0, void* workspace,
                                 size_t workspace_bytes, void* stream);

/*
 * pr_fine_adjoint without any device allocation by the library or the
 * caller.  The paper has no counterpart: this serves callers that cannot
 * allocate device memory while they run -- a real-time control loop that
 * forbids cudaMalloc/cudaFree after start-up because they can block and
 * synchronise the device, or a host whose device memory belongs to another
 * allocator.  Arguments and results are those of pr_fine_adjoint; the
 * checkpoints, sub-checkpoints and partial sums live instead in a fixed 32 MiB device array
 * inside the library, which every GPU that loads the library holds until the
 * process exits (pr_fine_adjoint_noalloc_capacity() gives its size).
 *  - A problem whose pr_fine_adjoint_workspace(n, n_slices, steps, ckpt_every)
 *    exceeds the capacity is rejected with PR_ERR_NOMEM before anything runs.
 *  - The first call on a device looks up the array's device address there
 *    (the device must be current); make that first call before any stream
 *    capture.  The address is kept for the life of the process: after a
 *    cudaDeviceReset (or any other teardown of the device's primary context)
 *    it is stale, and this entry point must not be called on that device
 *    again in the same process.
 *  - All calls share the one array and it keeps the last call's contents.
 *    Every word a call reads it has written first, so nothing needs clearing;
 *    calls that overlap on the GPU (other streams, other threads) race on the
 *    array and must be serialised by the caller.
 */
size_t pr_fine_adjoint_noalloc_capacity(void);
pr_status pr_fine_adjoint_noalloc(const pr_model* model, const pr_rng* rng, const float* x0, const float* y0,
                                  int64_t n, int32_t slice_begin, int32_t n_slices, int32_t steps, double dt,
                                  int32_t ckpt_every, float* x_T, float* y_T, const double* xbar_T,
                                  const double* ybar_T, double* grad, double* xbar_0, double* ybar_0,
                                  void* stream);

/*
 * Order statistics of n floats: index_out[r] = the index of the particle of
 * rank ranks[r] (0-based, ascending; ties broken by particle index), -1 for a
 * rank outside [0, n).  Used for the pathwise derivative of the empirical
 * quantile function, Q(p) = X_(ceil(p n)).
 *   x (device) [n]; ranks (device) [n_ranks] int64; index_out (device) [n_ranks] int64
 *   workspace (device) >= pr_order_statistics_workspace(n) bytes, 8-byte aligned.
 * The ranks are selected, not sorted for: the values are binned into 8192
 * equal-width buckets of [min, max], and only the buckets holding a requested
 * rank are gathered and sorted (by value, then index).  Where a value is not
 * finite or such a bucket holds more than 4096 particles (many equal values,
 * far outliers), every key is sorted instead; the result is the same.  The
 * call synchronises `stream` once (the host reads which of the two applies).
 */
size_t pr_order_statistics_workspace(int64_t n);
pr_status pr_order_statistics(const float* x, int64_t n, const int64_t* ranks, int32_t n_ranks,
                              int64_t* index_out, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Batched serving: many independent micro-macro parareal problems advanced
 * together, one parareal iteration of the whole batch per pr_batch_iterate.
 * Problem p draws its random numbers with problem_id = p (so a batch run of
 * problem p equals a single-problem run with pr_rng{seed, p}, bit for bit).
 * FP32 state, fast_dim = 1, families PR_MODEL_OU and PR_MODEL_DOUBLE_WELL,
 * bins <= 1024.  The plan owns every buffer (allocated by pr_batch_create):
 * ensembles, CDFs, one coarse propagator per problem, the work list.
 *
 * One iteration = a persistent fine kernel whose CTAs take work items
 * (problem, slice, particle range of about `item_work` particle-steps) from
 * an atomic counter, largest first; counts -> CDFs; the coarse step on every
 * start state; the serial update, one CTA per problem.  From the second
 * iteration on it is replayed as a CUDA graph.  Calls on one plan must not
 * overlap.
 */
typedef struct {
    pr_model model;
    pr_grid grid;
    int64_t n;          /* particles */
    int32_t n_slices;   /* K */
    int32_t steps;      /* EM steps per slice */
    double dt;          /* EM step */
    uint64_t seed;      /* Philox key */
} pr_problem;

/* Creates the plan (synchronises `stream`). */
pr_status pr_batch_create(const pr_problem* problems, int32_t n_problems, pr_iterator iterator,
                          pr_quantile_mode qmode, void** plan, void* stream);
pr_status pr_batch_destroy(void* plan);

/* Particle-steps of one iteration of the whole batch. */
int64_t pr_batch_particle_steps(void* plan);

/* Initial ensembles, packed: problem p occupies [off_p, off_p + n_p) of x0 and
 * y0 (device, float), off_p = n_0 + ... + n_{p-1}.  Runs the restriction of
 * X_0 and the zeroth iteration (serial coarse sweep). */
pr_status pr_batch_set_initial(void* plan, const float* x0, const float* y0, void* stream);

/* One parareal iteration of every problem. */
pr_status pr_batch_iterate(void* plan, void* stream);

/* Copies of a problem's state: rho_k^n as CDFs [K+1][bins+1] (device double);
 * the latest fine end states Xbar^{n+1}, n = 0..K-1, [K][n] each (device float). */
pr_status pr_batch_rho(void* plan, int32_t problem, double* out, void* stream);
pr_status pr_batch_fine_state(void* plan, int32_t problem, float* x_out, float* y_out, void* stream);

/* Largest status word over the problems (0 = PR_OK, else PR_ERR_NUMERIC);
 * synchronises `stream`. */
pr_status pr_batch_status(void* plan, int32_t* worst, void* stream);

/* Scheduling knobs: particles per thread (1, 2, 4) and the work per item in
 * particle-steps.  pr_batch_tune times the fine kernel for a grid of both
 * (each trial at ceil(steps / steps_div) steps per item, after
 * pr_batch_set_initial; trials do not disturb the iteration state), keeps
 * the fastest, and reports its time.  Results do not depend on the knobs. */
pr_status pr_batch_set_config(void* plan, int32_t ppt, double item_work);
pr_status pr_batch_get_config(void* plan, int32_t* ppt, double* item_work, int32_t* n_items);
pr_status pr_batch_tune(void* plan, int32_t steps_div, double* best_ms, void* stream);

/*
 * W1 distance between pairs of macroscopic states on the same grid, each read
 * as its piecewise-linear CDF: integral of |C1 - C2| over [x_lo, x_hi].
 *   c1, c2 (device) [n_vec][bins+1]; w1 (device) [n_vec] doubles.
 */
pr_status pr_w1(const pr_grid* grid, int32_t n_vec, const double* c1, const double* c2,
                double* w1, void* stream);

/*
 * L2 distance between the piecewise-constant densities (Eq.
 * piecewise_constant_pdf: bin mass / h) of pairs of macroscopic states, the
 * histogram error of the experiments of Section 6:
 * sqrt(sum_i (m1_i - m2_i)^2 / h) with m_i = C_{i+1} - C_i.
 *   c1, c2 (device) [n_vec][bins+1]; l2 (device) [n_vec] doubles.
 */
pr_status pr_l2_density(const pr_grid* grid, int32_t n_vec, const double* c1, const double* c2,
                        double* l2, void* stream);

/*
 * Transfers for callers that keep the initial ensemble X_0 and the resulting
 * macroscopic states in host memory (no counterpart in the paper: plumbing of
 * the boundary).  pr_copy_to_device copies `bytes` from src (host) to dst
 * (device); pr_copy_to_host from src (device) to dst (host).  Both are
 * asynchronous on `stream` when the host buffer is page-locked (otherwise the
 * CUDA runtime may return before or after the copy, as it documents for
 * cudaMemcpyAsync); bytes == 0 is a no-op.  pr_stream_synchronize waits for
 * everything enqueued on `stream`.  A failed CUDA call returns PR_ERR_CUDA.
 */
pr_status pr_copy_to_device(void* dst, const void* src, size_t bytes, void* stream);
pr_status pr_copy_to_host(void* dst, const void* src, size_t bytes, void* stream);
pr_status pr_stream_synchronize(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PR_H */

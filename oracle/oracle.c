/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the micro-macro parareal hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py do.  It shares no code with the
 * CUDA library (paper_1912_09240_gb300/csrc): every formula here is written
 * out again from the paper (Legoll, Lelievre, Myerscough, Samaey,
 * "Parareal computation of stochastic differential equations with time-scale
 * separation: a numerical study", arXiv:1912.09240) in its own order and
 * notation, in double precision, with no blocking, fusion or reordering.
 *
 * Where the paper is silent or garbled, the reading taken is stated at the
 * function it affects.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused: every
 * operation below is one IEEE-754 double operation, identical on x86-64 and
 * aarch64.
 *
 * Pins (tests/test_oracle_*.py): Philox words against Triton's independent
 * Philox4x32-10, normal statistics, EM moment recursion of the linear
 * family, brute-force restriction and CDF-at-edge exactness, strong
 * projection of the matching, Gaussian quantile arithmetic and the iterator
 * property of J_q, the parareal exactness theorem.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Threads the OpenMP loops below use. */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Cap the threads of the OpenMP loops (timing at one core and at all cores). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Random numbers.  The paper draws the EM increments dU_m, dV_m ~ N(0, dt)  */
/* independently (Section 2.1.3, Eqs. EMx/EMy) and reuses the same numbers  */
/* in every parareal iteration within a subinterval (Section 6).  Both are   */
/* met by a counter-based generator keyed by (seed) and counted by           */
/* (step, particle, slice, problem): Philox4x32-10 as published by Salmon,   */
/* Moraes, Dror and Shaw (SC'11).                                            */
/* ------------------------------------------------------------------------ */

/* Philox4x32 round multipliers and Weyl key increments (SC'11, Table 2). */
static const uint32_t OR_PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t OR_PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t OR_PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t OR_PHILOX_WEYL_B = 0xBB67AE85u;

/* One Philox4x32-10 block: 10 rounds of the S-box, key bumped in between. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += OR_PHILOX_WEYL_A;
            k1 += OR_PHILOX_WEYL_B;
        }
        uint64_t prod_a = (uint64_t)OR_PHILOX_MUL_A * (uint64_t)c0;
        uint64_t prod_b = (uint64_t)OR_PHILOX_MUL_B * (uint64_t)c2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t n0 = hi_b ^ c1 ^ k0;
        uint32_t n1 = lo_b;
        uint32_t n2 = hi_a ^ c3 ^ k1;
        uint32_t n3 = lo_a;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Batch form for tests: n counters in ctr[n][4], one key. */
void or_philox_batch(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    for (int64_t i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Uniform on (0,1) from one 32-bit word: the odd 24-bit integer
 * 2*(w >> 9) + 1 times 2^-24.  Exactly representable in binary32 and
 * binary64, never 0 or 1. */
double or_uniform(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Box-Muller: two uniforms to two independent standard normals. */
static void or_box_muller(uint32_t w0, uint32_t w1, double* z0, double* z1)
{
    double u0 = or_uniform(w0);
    double u1 = or_uniform(w1);
    double r = sqrt(-2.0 * log(u0));
    double theta = 2.0 * M_PI * u1;
    *z0 = r * cos(theta);
    *z1 = r * sin(theta);
}

/* The Q = 1 + d standard normals of fine step m of particle p in slice n of
 * problem `problem`.  Counter layout (a reading: the paper fixes only that
 * numbers are reused across iterations):
 *   Q <= 2 : one block serves two steps, ctr = (m >> 1, p, n, problem << 8);
 *            step m takes words 2*(m & 1) and 2*(m & 1) + 1.
 *   Q  > 2 : with F = Q / 4 and t = Q mod 4, normals 4g .. 4g + 3 of step m
 *            (g < F) come from ctr = (m, p, n, (problem << 8) | g), words
 *            taken in pairs in order, each pair giving its cosine and sine
 *            normals.  The last t normals of the four steps 4k .. 4k + 3
 *            share t blocks, ctr = (k, p, n, (problem << 8) | (F + j)),
 *            j < t: normal i < t of step 4k + s is number s t + i of the 4t
 *            normals those blocks give in order.  No word is dropped (in a
 *            slice whose step count is not a multiple of four, the last
 *            group's spare normals are).
 * z[0] drives the slow variable, z[1 + j] the fast component j. */
void or_step_normals(uint64_t seed, uint32_t problem, uint32_t p, uint32_t n,
                     uint32_t m, int Q, double* z)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    uint32_t ctr[4], w[4];
    if (Q <= 2) {
        ctr[0] = m >> 1; ctr[1] = p; ctr[2] = n; ctr[3] = problem << 8;
        or_philox4x32_10(ctr, key, w);
        int off = 2 * (int)(m & 1u);
        double a, b;
        or_box_muller(w[off], w[off + 1], &a, &b);
        z[0] = a;
        if (Q == 2) z[1] = b;
        return;
    }
    const int F = Q / 4, t = Q % 4;
    for (int g = 0; g < F; ++g) {
        ctr[0] = m; ctr[1] = p; ctr[2] = n; ctr[3] = (problem << 8) | (uint32_t)g;
        or_philox4x32_10(ctr, key, w);
        or_box_muller(w[0], w[1], &z[4 * g], &z[4 * g + 1]);
        or_box_muller(w[2], w[3], &z[4 * g + 2], &z[4 * g + 3]);
    }
    for (int i = 0; i < t; ++i) {
        const int idx = (int)(m & 3u) * t + i;   /* within the group's 4t normals */
        ctr[0] = m >> 2; ctr[1] = p; ctr[2] = n; ctr[3] = (problem << 8) | (uint32_t)(F + idx / 4);
        or_philox4x32_10(ctr, key, w);
        const int pair = (idx % 4) / 2;
        double a, b;
        or_box_muller(w[2 * pair], w[2 * pair + 1], &a, &b);
        z[4 * F + i] = (idx % 2) ? b : a;
    }
}

/* Normals of steps m0 .. m0+n_steps-1 for particles p0 .. p0+n_part-1 of
 * slice n: out[particle][step][Q] (for statistical tests). */
void or_normals_block(uint64_t seed, uint32_t problem, uint32_t p0, int64_t n_part,
                      uint32_t n, uint32_t m0, int n_steps, int Q, double* out)
{
    for (int64_t i = 0; i < n_part; ++i)
        for (int m = 0; m < n_steps; ++m)
            or_step_normals(seed, problem, p0 + (uint32_t)i, n, m0 + (uint32_t)m, Q,
                            out + (i * n_steps + m) * Q);
}

/* ------------------------------------------------------------------------ */
/* Slow-fast SDE (Section 2.1.1, Eqs. SDEx/SDEy) and its Euler-Maruyama      */
/* discretisation (Section 2.1.3, Eqs. EMx/EMy).  Three drift families:      */
/*   kind 0 (linear OU):  d_x F = x - lambda*y,          D = 1/beta          */
/*   kind 1 (double well): d_x F = x^3 - x + lambda*y,   D = 1/beta          */
/*   kind 2 (double well, d-dim fast OU): d_x F = x^3 - x + lambda*mean(y)   */
/* and in every family the fast potential G = |y - x|^2 / 2 (per component), */
/* E = 1.                                                                    */
/* ------------------------------------------------------------------------ */

enum { OR_MODEL_OU = 0, OR_MODEL_DOUBLE_WELL = 1, OR_MODEL_DW_MULTI = 2 };

static double or_dFdx(int kind, int d, double lambda, double x, const double* y)
{
    if (kind == OR_MODEL_OU) return x - lambda * y[0];
    if (kind == OR_MODEL_DOUBLE_WELL) return x * x * x - x + lambda * y[0];
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += y[j];
    return x * x * x - x + lambda * (s / (double)d);
}

/* Advance slices slice_begin .. slice_begin + n_slices - 1 in place.
 * x: [n_slices][N], y: [n_slices][d][N] (structure of arrays).  Each slice
 * takes S Euler-Maruyama steps of size dt; slice n uses the random numbers
 * of (seed, problem, particle, n, step). */
/* ids: the particle index p that keys each column's random numbers
 * (NULL: column p is particle p), so that a sample of an ensemble can be
 * advanced on its own. */
void or_fine_propagate_ids(int kind, int d, double lambda, double beta, double eps, double tau_x,
                           uint64_t seed, uint32_t problem,
                           double* x, double* y, int64_t N, const uint32_t* ids,
                           int slice_begin, int n_slices, int S, double dt)
{
    const int Q = 1 + d;
    const double D = 1.0 / beta;     /* slow diffusion D(x, y) */
    const double E = 1.0;            /* fast diffusion E(x, y) */
    const double sqrt_dt = sqrt(dt);
    for (int s = 0; s < n_slices; ++s) {
        const uint32_t n = (uint32_t)(slice_begin + s);
        double* xs = x + (int64_t)s * N;
        double* ys = y + (int64_t)s * d * N;
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < N; ++p) {
            double X = xs[p];
            double Y[64], Ynew[64], z[65];
            for (int j = 0; j < d; ++j) Y[j] = ys[(int64_t)j * N + p];
            for (int m = 0; m < S; ++m) {
                const uint32_t pid = ids ? ids[p] : (uint32_t)p;
                or_step_normals(seed, problem, pid, n, (uint32_t)m, Q, z);
                double dU = sqrt_dt * z[0];
                double Xnew = X - (1.0 / tau_x) * or_dFdx(kind, d, lambda, X, Y) * dt
                                + sqrt(2.0 * D / tau_x) * dU;
                for (int j = 0; j < d; ++j) {
                    double dV = sqrt_dt * z[1 + j];
                    double dGdy = Y[j] - X;
                    Ynew[j] = Y[j] - (1.0 / eps) * dGdy * dt + sqrt(2.0 * E / eps) * dV;
                }
                X = Xnew;
                for (int j = 0; j < d; ++j) Y[j] = Ynew[j];
            }
            xs[p] = X;
            for (int j = 0; j < d; ++j) ys[(int64_t)j * N + p] = Y[j];
        }
    }
}

void or_fine_propagate(int kind, int d, double lambda, double beta, double eps, double tau_x,
                       uint64_t seed, uint32_t problem,
                       double* x, double* y, int64_t N,
                       int slice_begin, int n_slices, int S, double dt)
{
    or_fine_propagate_ids(kind, d, lambda, beta, eps, tau_x, seed, problem, x, y, N, NULL,
                          slice_begin, n_slices, S, dt);
}

/* ------------------------------------------------------------------------ */
/* The chemically reacting system of Section 2.1.2 (Eqs. F_Bruna, G_Bruna,   */
/* D, E_Bruna) under Euler-Maruyama (Eqs. EMx/EMy), one fast variable.       */
/* Rates k[0..5] = k0 .. k5.  The paper prints                              */
/*   F(x,y) = -k4 x y - k5 x^2 / 2,                                         */
/*   G(x,y) = -k0 y - k1 y^2 / 2 + k2 y^2 (y/3 - 1/2) - k3 y^2 (y/2 - 1)^2,  */
/*   D = (k4 y + k5 x) / 2,  E = (k0 + k1 y + k2 y(y-1) + k3 y(y-1)(y-2)) / 2 */
/* whose D and E are half the total propensities of the reactions            */
/* Y -> Y + X (k4 y), X -> 0 (k5 x), 0 -> Y (k0), Y -> 0 (k1 y),             */
/* 2Y -> 3Y (k2 y(y-1)), 3Y -> 2Y (k3 y(y-1)(y-2)): the chemical Langevin   */
/* form.  Two readings of the drifts:                                        */
/*   reading 0 (chemical Langevin; the default): -d_x F = k4 y - k5 x and    */
/*     -d_y G = k0 - k1 y + k2 y(y-1) - k3 y(y-1)(y-2), the net rates of     */
/*     those reactions;                                                      */
/*   reading 1 (as printed): d_x F = -k4 y - k5 x and                        */
/*     d_y G = -k0 - k1 y + k2 y(y-1) - k3 y(y-1)(y-2), the derivatives of   */
/*     the printed F and G.                                                  */
/* 2D and 2E are sums of propensities, non-negative for x, y >= 0; where an  */
/* Euler step leaves that range the square root takes max(2D, 0) and         */
/* max(2E, 0) (a reading: the paper is silent).                             */
/* ------------------------------------------------------------------------ */

static double or_chem_dFdx(int reading, const double* k, double x, double y)
{
    if (reading == 0) return -(k[4] * y - k[5] * x);
    return -k[4] * y - k[5] * x;
}

static double or_chem_dGdy(int reading, const double* k, double y)
{
    const double net = k[0] - k[1] * y + k[2] * y * (y - 1.0) - k[3] * y * (y - 1.0) * (y - 2.0);
    if (reading == 0) return -net;
    return -k[0] - k[1] * y + k[2] * y * (y - 1.0) - k[3] * y * (y - 1.0) * (y - 2.0);
}

static double or_chem_D(const double* k, double x, double y)
{
    return 0.5 * (k[4] * y + k[5] * x);
}

static double or_chem_E(const double* k, double y)
{
    return 0.5 * (k[0] + k[1] * y + k[2] * y * (y - 1.0) + k[3] * y * (y - 1.0) * (y - 2.0));
}

/* d_x F, d_y G, D and E at (x, y): out[0..3]. */
void or_chem_coefficients(int reading, const double* k, double x, double y, double* out)
{
    out[0] = or_chem_dFdx(reading, k, x, y);
    out[1] = or_chem_dGdy(reading, k, y);
    out[2] = or_chem_D(k, x, y);
    out[3] = or_chem_E(k, y);
}

/* As or_fine_propagate_ids, for the chemical system (d = 1, two normals per
 * step: z[0] drives X, z[1] drives Y). */
void or_fine_propagate_chem(int reading, const double* k, double eps, double tau_x,
                            uint64_t seed, uint32_t problem,
                            double* x, double* y, int64_t N, const uint32_t* ids,
                            int slice_begin, int n_slices, int S, double dt)
{
    const double sqrt_dt = sqrt(dt);
    for (int s = 0; s < n_slices; ++s) {
        const uint32_t n = (uint32_t)(slice_begin + s);
        double* xs = x + (int64_t)s * N;
        double* ys = y + (int64_t)s * N;
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < N; ++p) {
            double X = xs[p], Y = ys[p], z[2];
            const uint32_t pid = ids ? ids[p] : (uint32_t)p;
            for (int m = 0; m < S; ++m) {
                or_step_normals(seed, problem, pid, n, (uint32_t)m, 2, z);
                const double dU = sqrt_dt * z[0];
                const double dV = sqrt_dt * z[1];
                const double D = or_chem_D(k, X, Y);
                const double E = or_chem_E(k, Y);
                const double Xnew = X - (1.0 / tau_x) * or_chem_dFdx(reading, k, X, Y) * dt
                                      + sqrt(fmax(2.0 * D, 0.0) / tau_x) * dU;
                const double Ynew = Y - (1.0 / eps) * or_chem_dGdy(reading, k, Y) * dt
                                      + sqrt(fmax(2.0 * E, 0.0) / eps) * dV;
                X = Xnew;
                Y = Ynew;
            }
            xs[p] = X;
            ys[p] = Y;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Tangent-linear (forward-mode) derivatives of the EM recursion with fixed   */
/* noise (pathwise sensitivities; the paper has no adjoint, this checks one). */
/* One particle per column, one slow and one fast variable (d = 1), drift     */
/* families 0 (OU) and 1 (double well).  Tangent directions, in order:        */
/* theta = (lambda, beta, eps), then the initial state x0 and y0.  ids as in  */
/* or_fine_propagate_ids (NULL: column p is particle p).                      */
/*   x_out, y_out   : [N]  states after n_slices * S steps                    */
/*   dx_out, dy_out : [N][5] d(X_T, Y_T)/d(lambda, beta, eps, x0, y0)         */
/* ------------------------------------------------------------------------ */

void or_fine_tangent(int kind, double lambda, double beta, double eps, double tau_x,
                     uint64_t seed, uint32_t problem, const double* x0, const double* y0,
                     int64_t N, const uint32_t* ids, int slice_begin, int n_slices, int S, double dt,
                     double* x_out, double* y_out, double* dx_out, double* dy_out)
{
    const double D = 1.0 / beta, E = 1.0;
    const double sqrt_dt = sqrt(dt);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        double X = x0[p], Y = y0[p];
        double dX[5] = {0, 0, 0, 1, 0}, dY[5] = {0, 0, 0, 0, 1};
        double z[2];
        for (int s = 0; s < n_slices; ++s) {
            const uint32_t n = (uint32_t)(slice_begin + s);
            for (int m = 0; m < S; ++m) {
                or_step_normals(seed, problem, ids ? ids[p] : (uint32_t)p, n, (uint32_t)m, 2, z);
                const double dU = sqrt_dt * z[0], dV = sqrt_dt * z[1];
                const double sX = sqrt(2.0 * D / tau_x), sY = sqrt(2.0 * E / eps);
                /* d_x F and its partial derivatives */
                double F, Fx, Fy, Fl;
                if (kind == OR_MODEL_OU) { F = X - lambda * Y; Fx = 1.0; Fy = -lambda; Fl = -Y; }
                else { F = X * X * X - X + lambda * Y; Fx = 3.0 * X * X - 1.0; Fy = lambda; Fl = Y; }
                const double Xn = X - (1.0 / tau_x) * F * dt + sX * dU;
                const double Yn = Y - (1.0 / eps) * (Y - X) * dt + sY * dV;
                /* Jacobian of the step */
                const double Jxx = 1.0 - Fx * dt / tau_x, Jxy = -Fy * dt / tau_x;
                const double Jyx = dt / eps, Jyy = 1.0 - dt / eps;
                /* explicit parameter derivatives of the step */
                double px[5] = { -Fl * dt / tau_x,                       /* lambda */
                                 -0.5 * sX / beta * dU,                  /* beta: d sqrt(2/(beta tau))/d beta */
                                 0.0, 0.0, 0.0 };
                double py[5] = { 0.0, 0.0,
                                 (Y - X) * dt / (eps * eps) - 0.5 * sY / eps * dV,   /* eps */
                                 0.0, 0.0 };
                for (int k = 0; k < 5; ++k) {
                    const double a = Jxx * dX[k] + Jxy * dY[k] + px[k];
                    const double b = Jyx * dX[k] + Jyy * dY[k] + py[k];
                    dX[k] = a;
                    dY[k] = b;
                }
                X = Xn;
                Y = Yn;
            }
        }
        x_out[p] = X;
        y_out[p] = Y;
        for (int k = 0; k < 5; ++k) {
            dx_out[p * 5 + k] = dX[k];
            dy_out[p * 5 + k] = dY[k];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Uniform grid x_lo = e_0 < e_1 < ... < e_I = x_hi (Section 2.2.2).         */
/* ------------------------------------------------------------------------ */

double or_edge(int i, int I, double lo, double hi)
{
    double h = (hi - lo) / (double)I;
    return lo + (double)i * h;
}

/* Bin of x: the i with e_i <= x < e_{i+1}, decided by exact comparison with
 * the edges, and clamped into [0, I-1] (a reading: the paper's strict
 * inequalities in Eq. binning leave edge points and escaped particles
 * unassigned; clamping keeps unit mass like the zero-flux coarse model). */
int or_bin(double x, int I, double lo, double hi)
{
    if (!(x >= lo)) return 0;          /* also catches NaN */
    if (x >= hi) return I - 1;
    double h = (hi - lo) / (double)I;
    int i = (int)floor((x - lo) / h);
    if (i < 0) i = 0;
    if (i > I - 1) i = I - 1;
    while (i > 0 && x < or_edge(i, I, lo, hi)) --i;
    while (i < I - 1 && x >= or_edge(i + 1, I, lo, hi)) ++i;
    return i;
}

/* Restriction R = R2 o R1 (Section 3.2.2, Eq. binning) with uniform weights
 * W = 1/N: counts per bin, and the piecewise-linear CDF at the edges
 * (Eq. discr_cdf), C_0 = 0, C_i = (number of particles in bins < i) / N. */
void or_restrict(const double* x, int64_t N, int n_slices, int I, double lo, double hi,
                 uint32_t* counts, double* cdf)
{
    for (int s = 0; s < n_slices; ++s) {
        const double* xs = x + (int64_t)s * N;
        uint32_t* cs = counts + (int64_t)s * I;
        double* Cs = cdf + (int64_t)s * (I + 1);
        for (int i = 0; i < I; ++i) cs[i] = 0;
        for (int64_t p = 0; p < N; ++p) cs[or_bin(xs[p], I, lo, hi)] += 1;
        uint64_t below = 0;
        Cs[0] = 0.0;
        for (int i = 0; i < I; ++i) {
            below += cs[i];
            Cs[i + 1] = (double)below / (double)N;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Matching that preserves the fast marginal (Section 5.1, Eq.              */
/* transformation): X = c^{-1}(cbar(Xbar)), Y = Ybar, with both CDFs the     */
/* piecewise-linear ones of the histograms.  Readings (the printed formulas  */
/* swap rho and rhobar): the prior's bin mass enters cbar, the posterior's   */
/* bin mass enters the inversion; the inverse bin is the lowest non-empty    */
/* bin whose upper CDF value reaches u; where prior and target CDF agree at  */
/* both edges of the particle's bin the map is the identity there (this is  */
/* the strong projection property, Eq. projection, held exactly); particles  */
/* outside [x_lo, x_hi] move by the displacement of the nearest edge.        */
/* ------------------------------------------------------------------------ */

static double or_match_one(double xbar, int I, double lo, double hi,
                           const double* Cp, const double* Ct)
{
    const double h = (hi - lo) / (double)I;
    int i = or_bin(xbar, I, lo, hi);
    if (Cp[i] == Ct[i] && Cp[i + 1] == Ct[i + 1]) return xbar;
    double ei = or_edge(i, I, lo, hi);
    double frac = (xbar - ei) / h;
    int below = 0, above = 0;
    if (frac < 0.0) { frac = 0.0; below = 1; }
    if (frac > 1.0) { frac = 1.0; above = 1; }
    double rho_prior = Cp[i + 1] - Cp[i];
    double u = Cp[i] + frac * rho_prior;
    int j = -1, last_nonempty = -1;
    for (int k = 0; k < I; ++k) {
        double rho_k = Ct[k + 1] - Ct[k];
        if (rho_k > 0.0) {
            last_nonempty = k;
            if (Ct[k + 1] >= u) { j = k; break; }
        }
    }
    if (j < 0) j = last_nonempty;
    if (j < 0) return xbar;            /* empty target: nothing to match */
    double rho_j = Ct[j + 1] - Ct[j];
    double t = (u - Ct[j]) / rho_j;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double xnew = or_edge(j, I, lo, hi) + t * h;
    if (below) return xbar + (xnew - lo);
    if (above) return xbar + (xnew - hi);
    return xnew;
}

void or_match(const double* x_prior, double* x_out, int64_t N, int n_slices,
              int I, double lo, double hi, const double* cdf_prior, const double* cdf_target)
{
    for (int s = 0; s < n_slices; ++s) {
        const double* Cp = cdf_prior + (int64_t)s * (I + 1);
        const double* Ct = cdf_target + (int64_t)s * (I + 1);
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < N; ++p)
            x_out[(int64_t)s * N + p] = or_match_one(x_prior[(int64_t)s * N + p], I, lo, hi, Cp, Ct);
    }
}

/* ------------------------------------------------------------------------ */
/* Quantile iterator J_q (Section 4.4, Eqs. quantile_reconstruction,        */
/* discr_cdf).  All three states are given as CDFs at the I+1 edges.         */
/*   a = rho_c^{n+1} (qhat), b = rho_f^* (qbar), c = rho_c^* (q).            */
/* mode 0 ("two-sided", default reading): at a level p that a CDF takes on a */
/* flat stretch, both ends of the stretch are kept as knots, so that         */
/* J(a, b, a) = b holds exactly.  mode 1 ("midpoint", the paper's literal    */
/* rule): the midpoint of the stretch.  Both modes use q(0) = max{x: c = 0}  */
/* and q(1) = min{x: c = 1}.  qtilde = qbar + (qhat - q) in that order.  The  */
/* monotonicity repair averages violating neighbours until none is left      */
/* (pool-adjacent-violators with equal weights).                             */
/* ------------------------------------------------------------------------ */

/* A level strictly between two edge values of a CDF has its quantile
 * strictly inside that bin: e0 + t*h, kept off the edges e0, e1 when the
 * rounding of the interpolation would land on one.  (Without this a tiny
 * level could round onto an edge and lift the CDF read back there.) */
static double or_inside(double e0, double e1, double t, double h)
{
    double q = e0 + t * h;
    if (q <= e0) q = nextafter(e0, e1);
    if (q >= e1) q = nextafter(e1, e0);
    return q;
}

/* q^-(p) = min{x : F(x) >= p} */
static double or_q_minus(const double* F, int I, double lo, double hi, double p)
{
    const double h = (hi - lo) / (double)I;
    int a = 0;
    while (a < I && F[a] < p) ++a;
    if (F[a] == p || a == 0) return or_edge(a, I, lo, hi);
    double t = (p - F[a - 1]) / (F[a] - F[a - 1]);
    return or_inside(or_edge(a - 1, I, lo, hi), or_edge(a, I, lo, hi), t, h);
}

/* q^+(p) = max{x : F(x) <= p} */
static double or_q_plus(const double* F, int I, double lo, double hi, double p)
{
    const double h = (hi - lo) / (double)I;
    int b = I;
    while (b > 0 && F[b] > p) --b;
    if (F[b] == p || b == I) return or_edge(b, I, lo, hi);
    double t = (p - F[b]) / (F[b + 1] - F[b]);
    return or_inside(or_edge(b, I, lo, hi), or_edge(b + 1, I, lo, hi), t, h);
}

static int or_cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Returns the number of knots used (for tests); out[I+1] is the new CDF. */
int or_quantile_update(int I, double lo, double hi, int mode,
                       const double* A, const double* B, const double* C, double* out)
{
    const int M = 3 * (I + 1);
    double* levels = (double*)malloc(sizeof(double) * M);
    for (int i = 0; i <= I; ++i) {
        levels[i] = A[i];
        levels[I + 1 + i] = B[i];
        levels[2 * (I + 1) + i] = C[i];
    }
    for (int k = 0; k < M; ++k) {
        if (levels[k] < 0.0) levels[k] = 0.0;
        if (levels[k] > 1.0) levels[k] = 1.0;
    }
    qsort(levels, M, sizeof(double), or_cmp_double);
    int L = 0;
    for (int k = 0; k < M; ++k)
        if (L == 0 || levels[k] != levels[L - 1]) levels[L++] = levels[k];

    double* kq = (double*)malloc(sizeof(double) * 2 * L);
    double* kp = (double*)malloc(sizeof(double) * 2 * L);
    int nk = 0;
    for (int l = 0; l < L; ++l) {
        double p = levels[l];
        int first = (l == 0), last = (l == L - 1);
        double am = or_q_minus(A, I, lo, hi, p), ap = or_q_plus(A, I, lo, hi, p);
        double bm = or_q_minus(B, I, lo, hi, p), bp = or_q_plus(B, I, lo, hi, p);
        double cm = or_q_minus(C, I, lo, hi, p), cp = or_q_plus(C, I, lo, hi, p);
        if (mode == 0) {
            if (!first) { kq[nk] = bm + (am - cm); kp[nk] = p; ++nk; }
            if (!last)  { kq[nk] = bp + (ap - cp); kp[nk] = p; ++nk; }
            if (first && last) { kq[nk] = bp + (ap - cp); kp[nk] = p; ++nk; }
        } else {
            double qa, qb, qc;
            if (first) { qa = ap; qb = bp; qc = cp; }
            else if (last) { qa = am; qb = bm; qc = cm; }
            else { qa = 0.5 * (am + ap); qb = 0.5 * (bm + bp); qc = 0.5 * (cm + cp); }
            kq[nk] = qb + (qa - qc); kp[nk] = p; ++nk;
        }
    }

    /* pool adjacent violators on kq (equal weights) */
    double* bsum = (double*)malloc(sizeof(double) * nk);
    int* bcnt = (int*)malloc(sizeof(int) * nk);
    int nb = 0;
    for (int k = 0; k < nk; ++k) {
        bsum[nb] = kq[k]; bcnt[nb] = 1; ++nb;
        /* mean of the left block > mean of the right block, compared as
         * sum_l * n_r > sum_r * n_l (counts are positive) */
        while (nb >= 2 && bsum[nb - 2] * (double)bcnt[nb - 1] > bsum[nb - 1] * (double)bcnt[nb - 2]) {
            bsum[nb - 2] += bsum[nb - 1];
            bcnt[nb - 2] += bcnt[nb - 1];
            --nb;
        }
    }
    int k = 0;
    for (int b = 0; b < nb; ++b) {
        if (bcnt[b] == 1) { ++k; continue; }       /* untouched knot keeps its bits */
        double mean = bsum[b] / bcnt[b];
        for (int c = 0; c < bcnt[b]; ++c) kq[k++] = mean;
    }

    /* PL CDF through (kq, kp), right-continuous, evaluated at the edges */
    out[0] = 0.0;
    out[I] = 1.0;
    for (int i = 1; i < I; ++i) {
        double x = or_edge(i, I, lo, hi);
        int jmax = -1;
        for (int j = 0; j < nk; ++j)
            if (kq[j] <= x) jmax = j;
        double v;
        if (jmax < 0) v = 0.0;
        else if (jmax == nk - 1) v = kp[nk - 1];
        else {
            double t = (x - kq[jmax]) / (kq[jmax + 1] - kq[jmax]);
            v = kp[jmax] + t * (kp[jmax + 1] - kp[jmax]);
        }
        if (v < 0.0) v = 0.0;
        if (v > 1.0) v = 1.0;
        out[i] = v;
    }
    free(levels); free(kq); free(kp); free(bsum); free(bcnt);
    return nk;
}

/* ------------------------------------------------------------------------ */
/* The other iterators of Section 4 on bin masses (rho_i = C_{i+1} - C_i),  */
/* results returned as CDFs.                                                 */
/* ------------------------------------------------------------------------ */

static void or_cdf_from_mass(int I, const double* m, double* out)
{
    double total = 0.0;
    for (int i = 0; i < I; ++i) total += m[i];
    double run = 0.0;
    out[0] = 0.0;
    for (int i = 0; i < I; ++i) {
        run += m[i];
        out[i + 1] = run / total;
    }
    out[I] = 1.0;
}

/* kind 1: additive (Section 4.1), negatives to zero then rescale.
 * kind 2: multiplicative (Section 4.2), unsupported bins to zero then rescale.
 * kind 3: rotation on the L2 sphere (Section 4.3).
 * Reading: when the corrected masses sum to zero (the multiplicative
 * iterator when the supports of a b and c do not meet) there is nothing to
 * rescale; the correction is dropped and the result is b, the fine result. */
void or_iterator_mass(int kind, int I, const double* A, const double* B, const double* C, double* out)
{
    double* a = (double*)malloc(sizeof(double) * I);
    double* b = (double*)malloc(sizeof(double) * I);
    double* c = (double*)malloc(sizeof(double) * I);
    double* r = (double*)malloc(sizeof(double) * I);
    for (int i = 0; i < I; ++i) {
        a[i] = A[i + 1] - A[i];
        b[i] = B[i + 1] - B[i];
        c[i] = C[i + 1] - C[i];
    }
    if (kind == 1) {
        for (int i = 0; i < I; ++i) {
            r[i] = a[i] + b[i] - c[i];
            if (r[i] < 0.0) r[i] = 0.0;
        }
    } else if (kind == 2) {
        for (int i = 0; i < I; ++i) r[i] = (c[i] > 0.0) ? a[i] * (b[i] / c[i]) : 0.0;
    } else {
        double u = 0.0, v = 0.0, w = 0.0;
        for (int i = 0; i < I; ++i) {
            u += sqrt(b[i] * c[i]);
            v += sqrt(b[i] * a[i]);
            w += sqrt(c[i] * a[i]);
        }
        double ca = (u + 2.0 * u * w - v) / (1.0 + w);
        double cc = (u + v) / (1.0 + w);
        for (int i = 0; i < I; ++i) {
            double s = ca * sqrt(a[i]) + sqrt(b[i]) - cc * sqrt(c[i]);
            r[i] = s * s;
        }
    }
    double total = 0.0;
    for (int i = 0; i < I; ++i) total += r[i];
    if (total > 0.0) {
        or_cdf_from_mass(I, r, out);
    } else {
        for (int i = 0; i <= I; ++i) out[i] = B[i];
    }
    free(a); free(b); free(c); free(r);
}

/* ------------------------------------------------------------------------ */
/* W1 distance between two histograms on the same grid, each read as its    */
/* piecewise-linear CDF: integral of |C1 - C2| over [x_lo, x_hi], exact for */
/* the linear difference on every bin.                                       */
/* ------------------------------------------------------------------------ */

double or_w1(int I, double lo, double hi, const double* C1, const double* C2)
{
    const double h = (hi - lo) / (double)I;
    double acc = 0.0;
    for (int i = 0; i < I; ++i) {
        double d0 = C1[i] - C2[i], d1 = C1[i + 1] - C2[i + 1];
        double a0 = fabs(d0), a1 = fabs(d1);
        if ((d0 >= 0.0 && d1 >= 0.0) || (d0 <= 0.0 && d1 <= 0.0)) acc += 0.5 * h * (a0 + a1);
        else acc += h * (d0 * d0 + d1 * d1) / (2.0 * (a0 + a1));
    }
    return acc;
}

/* L2 distance between the piecewise-constant densities of two histograms on
 * the same uniform grid (Eq. piecewise_constant_pdf: density rho_i / h on bin
 * i), the error measure of the experiments of Section 6:
 * sqrt( int (rho1_pc - rho2_pc)^2 dx ) = sqrt( sum_i (m1_i - m2_i)^2 / h ),
 * with the bin masses m_i = C_{i+1} - C_i read from the CDFs at the edges. */
double or_l2_density(int I, double lo, double hi, const double* C1, const double* C2)
{
    const double h = (hi - lo) / (double)I;
    double acc = 0.0;
    for (int i = 0; i < I; ++i) {
        const double m1 = C1[i + 1] - C1[i];
        const double m2 = C2[i + 1] - C2[i];
        acc += (m1 - m2) * (m1 - m2) / h;
    }
    return sqrt(acc);
}

/* ------------------------------------------------------------------------ */
/* Matching that preserves the conditional distribution (Section 5.2):      */
/* mu = mubar f(x) with f = rho / rhobar, sampled by reweighting the prior  */
/* ensemble, W^p = Wbar^p rho_i / rhobar_i with i the bin of Xbar^p, and    */
/* optionally by stratified resampling after it (Eq. stratified), or its     */
/* deterministic variant u~ = 1/2.  Positions are not moved.                 */
/* Readings: rhobar and rho are the bin masses of the given prior and target */
/* CDFs.  A target bin with mass where the prior has none gives half of it   */
/* to the nearest bin with prior mass on its left and half to the nearest    */
/* one on its right, or all of it to the only side that has one; the bins    */
/* are visited from left to right, each adding to the running masses.  A     */
/* particle in a bin without prior mass (possible only with a prior CDF that */
/* is not this ensemble's) gets weight 0.                                    */
/* ------------------------------------------------------------------------ */

/* Per-bin factors r_i = rho'_i / rhobar_i (0 where rhobar_i = 0), with rho'
 * the target masses after the relocation above. */
void or_reweight_factors(int I, const double* Cp, const double* Ct, double* r)
{
    double* rb = (double*)malloc(sizeof(double) * I);
    double* rt = (double*)malloc(sizeof(double) * I);
    double* rn = (double*)malloc(sizeof(double) * I);
    for (int i = 0; i < I; ++i) {
        rb[i] = Cp[i + 1] - Cp[i];
        rt[i] = Ct[i + 1] - Ct[i];
        rn[i] = rb[i] > 0.0 ? rt[i] : 0.0;
    }
    for (int i = 0; i < I; ++i) {
        if (rb[i] > 0.0 || !(rt[i] > 0.0)) continue;
        int L = i - 1, R = i + 1;
        while (L >= 0 && !(rb[L] > 0.0)) --L;
        while (R < I && !(rb[R] > 0.0)) ++R;
        if (L >= 0 && R < I) {
            rn[L] += 0.5 * rt[i];
            rn[R] += 0.5 * rt[i];
        } else if (L >= 0) {
            rn[L] += rt[i];
        } else if (R < I) {
            rn[R] += rt[i];
        }
    }
    for (int i = 0; i < I; ++i) r[i] = rb[i] > 0.0 ? rn[i] / rb[i] : 0.0;
    free(rb); free(rt); free(rn);
}

/* W^p = Wbar^p r_{bin(Xbar^p)}; wbar NULL means the uniform weight 1/N.
 * x, wbar, w: [n_slices][N]; cdf_prior, cdf_target: [n_slices][I+1]. */
void or_reweight(const double* x, const double* wbar, int64_t N, int n_slices, int I, double lo, double hi,
                 const double* cdf_prior, const double* cdf_target, double* w)
{
    double* r = (double*)malloc(sizeof(double) * I);
    const double w0 = 1.0 / (double)N;
    for (int s = 0; s < n_slices; ++s) {
        or_reweight_factors(I, cdf_prior + (int64_t)s * (I + 1), cdf_target + (int64_t)s * (I + 1), r);
        for (int64_t p = 0; p < N; ++p) {
            const int64_t k = (int64_t)s * N + p;
            const double wb = wbar ? wbar[k] : w0;
            w[k] = wb * r[or_bin(x[k], I, lo, hi)];
        }
    }
    free(r);
}

/* Weights in fixed point: round(W 2^61) as a 64-bit integer (W >= 0; the
 * scaling by a power of two is exact and the rounding is to nearest, ties
 * to even).  Sums of these are exact in any order.  The weights are
 * probability weights (Section 5.2: they sum to one); sums up to 8 fit. */
uint64_t or_weight_fixed(double w)
{
    if (!(w > 0.0)) return 0;
    return (uint64_t)llrint(ldexp(w, 61));
}

/* Stratified resampling (Section 5.2, Eq. stratified) of N weighted
 * particles into N equally weighted ones: output j takes the particle p
 * whose cumulative-weight interval [sum_{q<p} W^q, sum_{q<=p} W^q) holds
 * u_j = (j + u~_j) / N, the points scaled by the total weight T.
 * Readings: the cumulative weights are taken in the fixed point above, so
 * that the selection is exact and independent of the order of summation;
 * u~_j = a_j / 2^24 with a_j the odd 24-bit integer of the uniform of word
 * j mod 4 of Philox block (floor(j / 4), 0xFFFFFFFF, slice, problem << 8 |
 * 0xFE) (stratified, mode 0: one block serves four consecutive outputs) or
 * a_j = 2^23 (u~ = 1/2, deterministic, mode 1); the point is
 * U_j = floor(T (j 2^24 + a_j) / (N 2^24)); a point on a boundary goes to the
 * particle on its right (the paper's strict inequalities leave it to none).
 * With T = 0 (no weight at all) output j takes particle j.
 * w: [n_slices][N]; idx: [n_slices][N], the particle of each output. */
void or_resample(const double* w, int64_t N, int n_slices, int mode, uint64_t seed, uint32_t problem,
                 uint32_t slice_begin, uint32_t* idx)
{
    uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
    const uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    for (int s = 0; s < n_slices; ++s) {
        const double* ws = w + (int64_t)s * N;
        uint32_t* is = idx + (int64_t)s * N;
        uint64_t run = 0;
        for (int64_t p = 0; p < N; ++p) {
            run += or_weight_fixed(ws[p]);
            C[p] = run;
        }
        const uint64_t T = run;
        int64_t p = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (T == 0) { is[j] = (uint32_t)j; continue; }
            uint64_t a = (uint64_t)1 << 23;
            if (mode == 0) {
                const uint32_t ctr[4] = {(uint32_t)(j >> 2), 0xFFFFFFFFu, slice_begin + (uint32_t)s,
                                         (problem << 8) | 0xFEu};
                uint32_t out[4];
                or_philox4x32_10(ctr, key, out);
                a = 2 * (uint64_t)(out[j & 3] >> 9) + 1;
            }
            const unsigned __int128 num = (unsigned __int128)T * (((uint64_t)j << 24) + a);
            const uint64_t U = (uint64_t)(num / ((unsigned __int128)N << 24));
            /* the points increase with j, so the search resumes where it stopped */
            while (C[p] <= U) ++p;
            is[j] = (uint32_t)p;
        }
    }
    free(C);
}

/* Restriction with weights (the general form of Section 3.2.2, Eq. binning,
 * rho_i = sum of the weights in bin i), in the fixed point above:
 * C_0 = 0, C_i = (sum of fixed weights in bins < i) / (total), both sums
 * exact integers converted to double once.  With no weight at all the CDF
 * is that of an empty histogram read as uniform (C_i = i / I). */
void or_restrict_weighted(const double* x, const double* w, int64_t N, int n_slices, int I, double lo,
                          double hi, double* cdf)
{
    uint64_t* h = (uint64_t*)malloc(sizeof(uint64_t) * I);
    for (int s = 0; s < n_slices; ++s) {
        for (int i = 0; i < I; ++i) h[i] = 0;
        for (int64_t p = 0; p < N; ++p) {
            const int64_t k = (int64_t)s * N + p;
            h[or_bin(x[k], I, lo, hi)] += or_weight_fixed(w[k]);
        }
        uint64_t T = 0;
        for (int i = 0; i < I; ++i) T += h[i];
        double* Cs = cdf + (int64_t)s * (I + 1);
        uint64_t below = 0;
        Cs[0] = 0.0;
        for (int i = 0; i < I; ++i) {
            below += h[i];
            Cs[i + 1] = T > 0 ? (double)below / (double)T : (double)(i + 1) / (double)I;
        }
        Cs[I] = 1.0;
    }
    free(h);
}

/* Monte Carlo estimator (Section 2.1.3, Eq. MCestimator) of the observables
 * M = v^q, q = 1..Q: out[s][q-1] = sum over p, in order, of W^p (v^p)^q, the
 * term built as W^p multiplied by v^p q times.  Without weights (w NULL)
 * W^p = 1/n, read as the sum of (v^p)^q divided by n.
 * v: slice s at v + s * stride; w: [n_slices][n]; out: [n_slices][Q]. */
void or_moments(const double* v, int64_t stride, const double* w, int64_t n, int n_slices, int Q, double* out)
{
    for (int s = 0; s < n_slices; ++s) {
        for (int q = 1; q <= Q; ++q) {
            double sum = 0.0;
            for (int64_t p = 0; p < n; ++p) {
                const double x = v[(int64_t)s * stride + p];
                double t = w ? w[(int64_t)s * n + p] : 1.0;
                for (int r = 0; r < q; ++r) t = t * x;
                sum = sum + t;
            }
            out[s * Q + q - 1] = w ? sum : sum / (double)n;
        }
    }
}

// adjoint.cu -- pathwise adjoint of the binary32 Euler-Maruyama propagator
// with fixed noise (the EM recursion of Section 2.1.3, Eqs. EMx/EMy, run
// backwards), for gradients of ensemble observables with respect to
// theta = (lambda, beta, eps) and to the initial state; and order statistics
// (sorting) for the derivative of the quantile function.
//
// Forward: each thread advances one particle over the whole horizon
// (n_slices x steps), drawing exactly the random numbers pr_fine_propagate
// draws and taking exactly its steps (em_step_f32), and stores (x, y) every
// `ckpt_every` steps in the caller's workspace.
// Backward, where a segment's reconstruction stays accurate (see
// adjoint_reverse_ok): the reverse walk (adjoint_rev_kernel), which
// reconstructs the states by inverting the Euler steps.  Otherwise, exact
// replay, for each checkpoint segment from the last: the segment is
// replayed once from its checkpoint to leave sub-checkpoints every 12 steps in
// a scratch area of the workspace (16 B per particle per 12 steps); each
// 12-step block is then replayed once more, keeping its states and noise
// increments in shared memory (the first replay stops at the start of the
// segment's last block, whose end state is never needed: with checkpoints
// every 12 steps the backward pass is a single replay), and the adjoint
// recursion
//   lbar_t = J_t^T lbar_{t+1},  g += lbar_{t+1} . d(step_t)/d theta
// runs backwards over the block.  Per-block partial sums are binary32; they
// are added into binary64 accumulators per particle, and the ensemble sum is
// reduced in a fixed order (deterministic).
// When every slice has an even number of steps and the checkpoint interval is
// even, each Philox block serves a pair of steps that never straddles a slice
// or a replay block (adjoint_paired_kernel); otherwise the steps are walked
// one by one (adjoint_kernel).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "pr_common.cuh"

namespace pr {

constexpr int kAdjThreads = 128;
constexpr int kSub = 12;   // steps per replay block (even: pairs never straddle one)

struct AdjArgs {
    const float* x0;
    const float* y0;
    int64_t n;
    int slice_begin;
    int steps;        // per slice
    int64_t total;    // n_slices * steps
    int ckpt;         // checkpoint interval
    int64_t n_ckpt;
    float lam, ddt, rel, sxk, syk;               // forward constants, as pr_fine_propagate
    float inv2beta, inv2eps, rel_over_eps;       // derivative factors: 1/(2 beta), 1/(2 eps), dt/eps^2
    float ia, ib, ic, id;     // inverse of the OU step's matrix [[1-ddt, lam ddt], [rel, 1-rel]]
    float inv1mrel;           // 1 / (1 - rel)
    uint32_t k0, k1, chi;
    float* ckpt_buf;          // [n_ckpt][2][n]
    float* sub_buf;           // [ceil(min(ckpt, total) / kSub)][2][n]
    double* partial;          // [gridDim.x][3] (ensemble-sum mode)
    float* xT;
    float* yT;
    const double* xbar;       // seeds dL/dX_T (NULL: per-particle mode with seed 1)
    const double* ybar;       // seeds dL/dY_T or NULL
    double* grad_pp;          // [n][3] in per-particle mode
    double* xbar0;
    double* ybar0;
    int seed_affine;          // seeds dL/dX_T = seed_scale X_T + seed_shift from the particle's own end state
    double seed_scale, seed_shift;
};

// dL/dX_T of particle p with end state xT: given per particle, affine in xT,
// or 1 (per-particle mode)
__device__ __forceinline__ float seed_of(const AdjArgs& a, int64_t p, float xT)
{
    if (a.seed_affine) return (float)__dadd_rn(__dmul_rn(a.seed_scale, (double)xT), a.seed_shift);
    return a.xbar ? (float)a.xbar[p] : 1.0f;
}

// Walks the steps in order; step m of slice s uses words 2(m&1), 2(m&1)+1 of
// the Philox block (m >> 1, p, slice_begin + s, problem << 8).
struct NoiseWalker {
    int slice, m, cached_mp, cached_slice;
    uint4 w;

    __device__ void seek(int64_t t, int S)
    {
        slice = (int)(t / S);
        m = (int)(t - (int64_t)slice * S);
        cached_mp = -1;
        cached_slice = -1;
    }

    __device__ __forceinline__ void draw(const AdjArgs& a, uint32_t pid, float& q, float& c, float& s)
    {
        const int mp = m >> 1;
        if (mp != cached_mp || slice != cached_slice) {
            w = philox4x32_10(make_uint4((uint32_t)mp, pid, (uint32_t)(a.slice_begin + slice), a.chi), a.k0, a.k1);
            cached_mp = mp;
            cached_slice = slice;
        }
        if (m & 1) box_muller_qcs(w.z, w.w, q, c, s);
        else box_muller_qcs(w.x, w.y, q, c, s);
    }

    __device__ __forceinline__ void advance(int S)
    {
        if (++m == S) {
            m = 0;
            ++slice;
        }
    }
};

// One block of the adjoint recursion, backwards over `len` steps whose states
// and noise increments are in shared memory:
//   lbar_t = J_t^T lbar_{t+1},  g += lbar_{t+1} . d(step_t)/d theta.
// LEN > 0: a full block of LEN steps, the loop unrolled (fixed shared-memory
// offsets); LEN = 0: `len` steps.
template <int KIND, int LEN = 0>
__device__ __forceinline__ void backward_block(const AdjArgs& a, int len, int T, int tid, const float* bx,
                                               const float* by, const float* bnx, const float* bny, float& lx,
                                               float& ly, double& g0, double& g1, double& g2)
{
    if (LEN > 0) {
        len = LEN;
        T = kAdjThreads;
    }
    float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f;
#pragma unroll
    for (int i = len - 1; i >= 0; --i) {
        const float xi = bx[i * T + tid], yi = by[i * T + tid];
        const float nx = bnx[i * T + tid], ny = bny[i * T + tid];
        float jxx, jxy, dxdl;
        if (KIND == PR_MODEL_OU) {          // d_x F = x - lam y
            jxx = 1.0f - a.ddt;
            jxy = a.lam * a.ddt;
            dxdl = a.ddt * yi;
        } else {                            // d_x F = x^3 - x + lam y
            jxx = 1.0f - a.ddt * (3.0f * xi * xi - 1.0f);
            jxy = -a.lam * a.ddt;
            dxdl = -a.ddt * yi;
        }
        const float jyx = a.rel, jyy = 1.0f - a.rel;
        p0 = fmaf(lx, dxdl, p0);                                   // d/d lambda
        p1 = fmaf(lx, -nx * a.inv2beta, p1);                       // d/d beta (noise amplitude)
        p2 = fmaf(ly, -a.rel_over_eps * (xi - yi) - ny * a.inv2eps, p2);   // d/d eps
        const float nlx = lx * jxx + ly * jyx;
        const float nly = lx * jxy + ly * jyy;
        lx = nlx;
        ly = nly;
    }
    g0 += (double)p0;
    g1 += (double)p1;
    g2 += (double)p2;
}

// Fixed-order block reduction of the three per-particle sums into partial[block].
__device__ __forceinline__ void block_partials(const AdjArgs& a, double g0, double g1, double g2)
{
    __shared__ double red[3][kAdjThreads / 32];
    double v[3] = {g0, g1, g2};
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        if (lane == 0) red[k][warp] = v[k];
    }
    __syncthreads();
    if (tid < 3) {
        double s = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) s += red[tid][w];
        a.partial[(size_t)blockIdx.x * 3 + tid] = s;
    }
}

__device__ __forceinline__ void store_outputs(const AdjArgs& a, int64_t p, float lx, float ly, double g0, double g1,
                                              double g2)
{
    if (a.xbar0) a.xbar0[p] = (double)lx;
    if (a.ybar0) a.ybar0[p] = (double)ly;
    if (a.grad_pp) {
        a.grad_pp[p * 3 + 0] = g0;
        a.grad_pp[p * 3 + 1] = g1;
        a.grad_pp[p * 3 + 2] = g2;
    }
}

// Any step count: steps walked one by one, the Philox block of a pair cached.
template <int KIND>
__global__ void __launch_bounds__(kAdjThreads, 8)
adjoint_kernel(AdjArgs a)
{
    extern __shared__ float asm_[];
    const int T = blockDim.x, tid = threadIdx.x;
    float* bx = asm_;
    float* by = bx + kSub * T;
    float* bnx = by + kSub * T;
    float* bny = bnx + kSub * T;
    const int64_t p = (int64_t)blockIdx.x * T + tid;
    const bool ok = p < a.n;
    const uint32_t pid = (uint32_t)p;
    const int S = a.steps;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    float lx = 0.0f, ly = 0.0f;

    if (ok) {
        // ---- forward with checkpoints ----
        float x = a.x0[p], y = a.y0[p];
        NoiseWalker nw;
        nw.seek(0, S);
        int64_t next_ck = 0, ck = 0;
        for (int64_t t = 0; t < a.total; ++t) {
            if (t == next_ck) {
                a.ckpt_buf[(ck * 2) * a.n + p] = x;
                a.ckpt_buf[(ck * 2 + 1) * a.n + p] = y;
                ++ck;
                next_ck += a.ckpt;
            }
            float q, c, s;
            nw.draw(a, pid, q, c, s);
            em_step_f32<KIND>(x, y, q * a.sxk, c, q * a.syk, s, a.lam, a.ddt, a.rel);
            nw.advance(S);
        }
        if (a.total == 0) {
            a.ckpt_buf[p] = x;
            a.ckpt_buf[a.n + p] = y;
        }
        if (a.xT) a.xT[p] = x;
        if (a.yT) a.yT[p] = y;

        // ---- backward ----
        lx = seed_of(a, p, x);
        ly = a.ybar ? (float)a.ybar[p] : 0.0f;
        for (int64_t c = a.n_ckpt - 1; c >= 0; --c) {
            const int64_t t0 = c * a.ckpt;
            const int L = (int)min((int64_t)a.ckpt, a.total - t0);
            const int nsub = (L + kSub - 1) / kSub;
            x = a.ckpt_buf[(c * 2) * a.n + p];
            y = a.ckpt_buf[(c * 2 + 1) * a.n + p];
            nw.seek(t0, S);
            for (int j = 0; j < nsub; ++j) {
                a.sub_buf[(int64_t)(2 * j) * a.n + p] = x;
                a.sub_buf[(int64_t)(2 * j + 1) * a.n + p] = y;
                if (j == nsub - 1) break;   // the last block's end state is not needed
                const int len = min(kSub, L - j * kSub);
                for (int i = 0; i < len; ++i) {
                    float q, cc, s;
                    nw.draw(a, pid, q, cc, s);
                    em_step_f32<KIND>(x, y, q * a.sxk, cc, q * a.syk, s, a.lam, a.ddt, a.rel);
                    nw.advance(S);
                }
            }
            for (int j = nsub - 1; j >= 0; --j) {
                const int len = min(kSub, L - j * kSub);
                x = a.sub_buf[(int64_t)(2 * j) * a.n + p];
                y = a.sub_buf[(int64_t)(2 * j + 1) * a.n + p];
                nw.seek(t0 + (int64_t)j * kSub, S);
                for (int i = 0; i < len; ++i) {
                    float q, cc, s;
                    nw.draw(a, pid, q, cc, s);
                    const float ax = q * a.sxk, ay = q * a.syk;
                    bx[i * T + tid] = x;
                    by[i * T + tid] = y;
                    bnx[i * T + tid] = ax * cc;
                    bny[i * T + tid] = ay * s;
                    em_step_f32<KIND>(x, y, ax, cc, ay, s, a.lam, a.ddt, a.rel);
                    nw.advance(S);
                }
                backward_block<KIND>(a, len, T, tid, bx, by, bnx, bny, lx, ly, g0, g1, g2);
            }
        }
        store_outputs(a, p, lx, ly, g0, g1, g2);
    }
    if (a.partial) block_partials(a, g0, g1, g2);
}

// Even steps per slice and an even checkpoint interval: every replay starts
// at an even step of a slice, so each Philox block serves the pair of steps
// (m, m+1) with words (x, y) and (z, w), as in pr_fine_propagate.
template <int KIND>
__global__ void __launch_bounds__(kAdjThreads, 8)
adjoint_paired_kernel(AdjArgs a)
{
    extern __shared__ float asm_[];
    const int T = blockDim.x, tid = threadIdx.x;
    float* bx = asm_;
    float* by = bx + kSub * T;
    float* bnx = by + kSub * T;
    float* bny = bnx + kSub * T;
    const int64_t p = (int64_t)blockIdx.x * T + tid;
    const bool ok = p < a.n;
    const uint32_t pid = (uint32_t)p;
    const int S = a.steps;
    const float lam = a.lam, ddt = a.ddt, rel = a.rel, sxk = a.sxk, syk = a.syk;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    float lx = 0.0f, ly = 0.0f;

    auto pair = [&](int slice, int m, float& x, float& y) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(m >> 1), pid, (uint32_t)(a.slice_begin + slice), a.chi),
                                      a.k0, a.k1);
        float q0, c0, s0, q1, c1, s1;
        box_muller_qcs(w.x, w.y, q0, c0, s0);
        box_muller_qcs(w.z, w.w, q1, c1, s1);
        em_step_f32<KIND>(x, y, q0 * sxk, c0, q0 * syk, s0, lam, ddt, rel);
        em_step_f32<KIND>(x, y, q1 * sxk, c1, q1 * syk, s1, lam, ddt, rel);
    };

    if (ok) {
        // ---- forward with checkpoints ----
        float x = a.x0[p], y = a.y0[p];
        int slice = 0, m = 0;
        for (int64_t c = 0; c < a.n_ckpt; ++c) {
            a.ckpt_buf[(c * 2) * a.n + p] = x;
            a.ckpt_buf[(c * 2 + 1) * a.n + p] = y;
            const int L = (int)min((int64_t)a.ckpt, a.total - c * a.ckpt);
            for (int i = 0; i < L; i += 2) {
                pair(slice, m, x, y);
                m += 2;
                if (m == S) { m = 0; ++slice; }
            }
        }
        if (a.xT) a.xT[p] = x;
        if (a.yT) a.yT[p] = y;

        // ---- backward ----
        lx = seed_of(a, p, x);
        ly = a.ybar ? (float)a.ybar[p] : 0.0f;
        for (int64_t c = a.n_ckpt - 1; c >= 0; --c) {
            const int64_t t0 = c * a.ckpt;
            const int L = (int)min((int64_t)a.ckpt, a.total - t0);
            const int nsub = (L + kSub - 1) / kSub;
            x = a.ckpt_buf[(c * 2) * a.n + p];
            y = a.ckpt_buf[(c * 2 + 1) * a.n + p];
            int slice = (int)(t0 / S), m = (int)(t0 - (int64_t)slice * S);
            for (int j = 0; j < nsub; ++j) {
                a.sub_buf[(int64_t)(2 * j) * a.n + p] = x;
                a.sub_buf[(int64_t)(2 * j + 1) * a.n + p] = y;
                if (j == nsub - 1) break;   // the last block's end state is not needed
                const int len = min(kSub, L - j * kSub);
                for (int i = 0; i < len; i += 2) {
                    pair(slice, m, x, y);
                    m += 2;
                    if (m == S) { m = 0; ++slice; }
                }
            }
            for (int j = nsub - 1; j >= 0; --j) {
                const int len = min(kSub, L - j * kSub);
                x = a.sub_buf[(int64_t)(2 * j) * a.n + p];
                y = a.sub_buf[(int64_t)(2 * j + 1) * a.n + p];
                const int64_t tb = t0 + (int64_t)j * kSub;
                slice = (int)(tb / S);
                m = (int)(tb - (int64_t)slice * S);
                // steps i, i + 1 of the block: states and noise increments to shared memory
                auto replay_pair = [&](int i, int Ts) {
                    const uint4 w = philox4x32_10(
                        make_uint4((uint32_t)(m >> 1), pid, (uint32_t)(a.slice_begin + slice), a.chi), a.k0, a.k1);
                    float q0, c0, s0, q1, c1, s1;
                    box_muller_qcs(w.x, w.y, q0, c0, s0);
                    box_muller_qcs(w.z, w.w, q1, c1, s1);
                    const float ax0 = q0 * sxk, ay0 = q0 * syk, ax1 = q1 * sxk, ay1 = q1 * syk;
                    bx[i * Ts + tid] = x;
                    by[i * Ts + tid] = y;
                    bnx[i * Ts + tid] = ax0 * c0;
                    bny[i * Ts + tid] = ay0 * s0;
                    em_step_f32<KIND>(x, y, ax0, c0, ay0, s0, lam, ddt, rel);
                    bx[(i + 1) * Ts + tid] = x;
                    by[(i + 1) * Ts + tid] = y;
                    bnx[(i + 1) * Ts + tid] = ax1 * c1;
                    bny[(i + 1) * Ts + tid] = ay1 * s1;
                    em_step_f32<KIND>(x, y, ax1, c1, ay1, s1, lam, ddt, rel);
                    m += 2;
                    if (m == S) { m = 0; ++slice; }
                };
                if (len == kSub) {
#pragma unroll
                    for (int i = 0; i < kSub; i += 2) replay_pair(i, kAdjThreads);
                    backward_block<KIND, kSub>(a, len, T, tid, bx, by, bnx, bny, lx, ly, g0, g1, g2);
                } else {
                    for (int i = 0; i < len; i += 2) replay_pair(i, T);
                    backward_block<KIND>(a, len, T, tid, bx, by, bnx, bny, lx, ly, g0, g1, g2);
                }
            }
        }
        store_outputs(a, p, lx, ly, g0, g1, g2);
    }
    if (a.partial) block_partials(a, g0, g1, g2);
}

// Reverse-walk adjoint.  The backward pass does not replay the forward: it
// reconstructs each state from the next by inverting the Euler step with the
// same noise increments, which it draws again, and runs the adjoint recursion
// on the fly:
//   OU:          (x, y) = M^{-1} (x' - dU, y' - dV), M = [[1-ddt, lam ddt], [rel, 1-rel]]
//   double well: y = (y' - dV - rel x) / (1 - rel), x the fixed point of
//                x = x' - dU + ddt (x^3 - x + lam y(x)), two iterations from
//                x' - dU (each shrinks the error by ddt |3x^2 - 1 - lam rel/(1-rel)|)
// Each checkpoint segment starts again from the stored exact state at its
// end, so the rounding of the reconstruction grows over one segment only, by
// at most (1/(1-rel))^ckpt / (1-ddt)^ckpt, which the host bounds before it
// picks this kernel.  Cost: the forward pass and one backward pass with its
// Philox blocks, no sub-checkpoints, no shared memory.
template <int KIND>
__device__ __forceinline__ void inverse_step(const AdjArgs& a, float& x, float& y, float nx, float ny)
{
    const float bx = x - nx, by = y - ny;
    if (KIND == PR_MODEL_OU) {
        x = fmaf(a.ia, bx, a.ib * by);
        y = fmaf(a.ic, bx, a.id * by);
    } else {
        float u = bx;
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const float v = (by - a.rel * u) * a.inv1mrel;
            u = fmaf(a.ddt, fmaf(u * u, u, -u) + a.lam * v, bx);
        }
        x = u;
        y = (by - a.rel * u) * a.inv1mrel;
    }
}

// Adjoint of step t at its start state (x, y), given lbar_{t+1} in (lx, ly):
// the parameter sums and lbar_t.
template <int KIND>
__device__ __forceinline__ void adjoint_step(const AdjArgs& a, float x, float y, float nx, float ny, float& lx,
                                             float& ly, float& p0, float& p1, float& p2)
{
    float jxx, jxy, dxdl;
    if (KIND == PR_MODEL_OU) {
        jxx = 1.0f - a.ddt;
        jxy = a.lam * a.ddt;
        dxdl = a.ddt * y;
    } else {
        jxx = 1.0f - a.ddt * (3.0f * x * x - 1.0f);
        jxy = -a.lam * a.ddt;
        dxdl = -a.ddt * y;
    }
    p0 = fmaf(lx, dxdl, p0);
    p1 = fmaf(lx, -nx * a.inv2beta, p1);
    p2 = fmaf(ly, -a.rel_over_eps * (x - y) - ny * a.inv2eps, p2);
    const float nlx = lx * jxx + ly * a.rel;
    const float nly = lx * jxy + ly * (1.0f - a.rel);
    lx = nlx;
    ly = nly;
}

// PAIRED: every slice has an even number of steps and the checkpoint
// interval is even, so each Philox block serves the pair (m, m+1) of one
// segment, forwards and backwards.
template <int KIND, bool PAIRED>
__global__ void __launch_bounds__(kAdjThreads, 8)
adjoint_rev_kernel(AdjArgs a)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = p < a.n;
    const uint32_t pid = (uint32_t)p;
    const int S = a.steps;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    float lx = 0.0f, ly = 0.0f;
    if (ok) {
        // ---- forward with checkpoints (pr_fine_propagate's steps) ----
        float x = a.x0[p], y = a.y0[p];
        NoiseWalker nw;
        nw.seek(0, S);
        int slice = 0, m = 0;
        for (int64_t c = 0; c < a.n_ckpt; ++c) {
            a.ckpt_buf[(c * 2) * a.n + p] = x;
            a.ckpt_buf[(c * 2 + 1) * a.n + p] = y;
            const int L = (int)min((int64_t)a.ckpt, a.total - c * a.ckpt);
            if (PAIRED) {
                for (int i = 0; i < L; i += 2) {
                    const uint4 w = philox4x32_10(
                        make_uint4((uint32_t)(m >> 1), pid, (uint32_t)(a.slice_begin + slice), a.chi), a.k0, a.k1);
                    float q0, c0, s0, q1, c1, s1;
                    box_muller_qcs(w.x, w.y, q0, c0, s0);
                    box_muller_qcs(w.z, w.w, q1, c1, s1);
                    em_step_f32<KIND>(x, y, q0 * a.sxk, c0, q0 * a.syk, s0, a.lam, a.ddt, a.rel);
                    em_step_f32<KIND>(x, y, q1 * a.sxk, c1, q1 * a.syk, s1, a.lam, a.ddt, a.rel);
                    m += 2;
                    if (m == S) { m = 0; ++slice; }
                }
            } else {
                for (int i = 0; i < L; ++i) {
                    float q, cc, sn;
                    nw.draw(a, pid, q, cc, sn);
                    em_step_f32<KIND>(x, y, q * a.sxk, cc, q * a.syk, sn, a.lam, a.ddt, a.rel);
                    nw.advance(S);
                }
            }
        }
        if (a.xT) a.xT[p] = x;
        if (a.yT) a.yT[p] = y;
        const float xe = x, ye = y;

        // ---- backward, segment by segment from the last ----
        lx = seed_of(a, p, xe);
        ly = a.ybar ? (float)a.ybar[p] : 0.0f;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        int cached_mp = -1, cached_slice = -1;
        for (int64_t c = a.n_ckpt - 1; c >= 0; --c) {
            const int64_t t0 = c * a.ckpt;
            const int L = (int)min((int64_t)a.ckpt, a.total - t0);
            if (c + 1 < a.n_ckpt) {   // the exact state at the segment's end
                x = a.ckpt_buf[((c + 1) * 2) * a.n + p];
                y = a.ckpt_buf[((c + 1) * 2 + 1) * a.n + p];
            } else {
                x = xe;
                y = ye;
            }
            const int64_t tl = t0 + L - 1;
            slice = (int)(tl / S);
            m = (int)(tl - (int64_t)slice * S);
            // blocks of at most 4 kSub steps, backwards; binary32 partial sums
            // per block (48 terms at most), added into the binary64 sums after it
            for (int left = L; left > 0; left -= 4 * kSub) {
                const int len = min(4 * kSub, left);
                float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f;
                if (PAIRED) {   // m is odd here: steps m and m - 1 from one block
                    for (int i = 0; i < len; i += 2) {
                        const uint4 wp = philox4x32_10(
                            make_uint4((uint32_t)(m >> 1), pid, (uint32_t)(a.slice_begin + slice), a.chi), a.k0,
                            a.k1);
                        float q0, c0, s0, q1, c1, s1;
                        box_muller_qcs(wp.z, wp.w, q1, c1, s1);
                        box_muller_qcs(wp.x, wp.y, q0, c0, s0);
                        float nx = (q1 * a.sxk) * c1, ny = (q1 * a.syk) * s1;
                        inverse_step<KIND>(a, x, y, nx, ny);
                        adjoint_step<KIND>(a, x, y, nx, ny, lx, ly, p0, p1, p2);
                        nx = (q0 * a.sxk) * c0;
                        ny = (q0 * a.syk) * s0;
                        inverse_step<KIND>(a, x, y, nx, ny);
                        adjoint_step<KIND>(a, x, y, nx, ny, lx, ly, p0, p1, p2);
                        m -= 2;
                        if (m < 0) { --slice; m = S - 1; }
                    }
                } else {
                    for (int i = 0; i < len; ++i) {
                        const int mp = m >> 1;
                        if (mp != cached_mp || slice != cached_slice) {
                            w = philox4x32_10(
                                make_uint4((uint32_t)mp, pid, (uint32_t)(a.slice_begin + slice), a.chi), a.k0, a.k1);
                            cached_mp = mp;
                            cached_slice = slice;
                        }
                        float q, cc, sn;
                        if (m & 1) box_muller_qcs(w.z, w.w, q, cc, sn);
                        else box_muller_qcs(w.x, w.y, q, cc, sn);
                        const float nx = (q * a.sxk) * cc, ny = (q * a.syk) * sn;
                        inverse_step<KIND>(a, x, y, nx, ny);
                        adjoint_step<KIND>(a, x, y, nx, ny, lx, ly, p0, p1, p2);
                        if (--m < 0) { --slice; m = S - 1; }
                    }
                }
                g0 += (double)p0;
                g1 += (double)p1;
                g2 += (double)p2;
            }
        }
        store_outputs(a, p, lx, ly, g0, g1, g2);
    }
    if (a.partial) block_partials(a, g0, g1, g2);
}

__global__ void reduce_partials_kernel(const double* __restrict__ partial, int64_t blocks, double* __restrict__ grad)
{
    __shared__ double red[3][256];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t b = threadIdx.x; b < blocks; b += blockDim.x) {
        s0 += partial[b * 3 + 0];
        s1 += partial[b * 3 + 1];
        s2 += partial[b * 3 + 2];
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) s += red[threadIdx.x][i];
        grad[threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Order statistics: the requested ranks of (orderable float bits << 32 |
// index), by bucket selection, or by a bitonic sort of all keys
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t float_order_bits(float v)
{
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void make_keys_kernel(const float* __restrict__ x, int64_t n, int64_t padded, unsigned long long* keys)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < padded; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = i < n ? (((unsigned long long)float_order_bits(x[i]) << 32) | (unsigned long long)i)
                        : ~0ull;
}

__global__ void bitonic_step_kernel(unsigned long long* keys, int64_t padded, int64_t j, int64_t k)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < padded; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = i ^ j;
        if (l > i) {
            const unsigned long long a = keys[i], b = keys[l];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
                keys[i] = b;
                keys[l] = a;
            }
        }
    }
}

__global__ void gather_ranks_kernel(const unsigned long long* __restrict__ keys, const int64_t* __restrict__ ranks,
                                    int n_ranks, int64_t n, int64_t* __restrict__ idx)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_ranks) return;
    const int64_t rk = ranks[r];
    idx[r] = (rk >= 0 && rk < n) ? (int64_t)(keys[rk] & 0xFFFFFFFFull) : -1;   // -1: rank out of range
}

// Selection of the requested ranks without sorting everything: the values
// are binned into kSelBuckets equal-width buckets of [min, max] (a monotone
// map, so the sorted order is bucket by bucket), the buckets holding a
// requested rank are found from the bucket counts' prefix sums, their
// particles are gathered, and each such bucket (at most kSelCap particles) is
// sorted by (value, index) in shared memory by one CTA per rank.  Non-finite
// values or a bucket beyond kSelCap fall back to the full sort.
constexpr int kSelBuckets = 8192;
constexpr int kSelCap = 4096;

struct SelWs {
    unsigned* counts;    // [kSelBuckets]
    unsigned* starts;    // [kSelBuckets + 1] exclusive prefix sums of counts
    unsigned* seg;       // [kSelBuckets] offset of a wanted bucket's particles in cand, or ~0u
    unsigned* cursor;    // [kSelBuckets]
    unsigned* mm;        // [2] orderable min, max
    unsigned* flag;      // [1] 1: fall back to the full sort
    unsigned long long* cand;
};

__device__ __forceinline__ float float_from_order_bits(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ int sel_bucket(float v, float vmin, float scale)
{
    const float t = (v - vmin) * scale;
    return t >= (float)(kSelBuckets - 1) ? kSelBuckets - 1 : (int)t;
}

__device__ __forceinline__ void sel_range(const SelWs& w, float& vmin, float& scale)
{
    vmin = float_from_order_bits(w.mm[0]);
    const float vmax = float_from_order_bits(w.mm[1]);
    scale = vmax > vmin ? (float)kSelBuckets / (vmax - vmin) : 0.0f;
}

__global__ void sel_minmax_kernel(const float* __restrict__ x, int64_t n, SelWs w)
{
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = float_order_bits(x[i]);
        lo = min(lo, k);
        hi = max(hi, k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&w.mm[0], lo);
        atomicMax(&w.mm[1], hi);
    }
}

__global__ void __launch_bounds__(1024) sel_hist_kernel(const float* __restrict__ x, int64_t n, SelWs w)
{
    __shared__ unsigned h[kSelBuckets];
    for (int b = threadIdx.x; b < kSelBuckets; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    float vmin, scale;
    sel_range(w, vmin, scale);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[sel_bucket(x[i], vmin, scale)], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBuckets; b += blockDim.x)
        if (h[b]) atomicAdd(&w.counts[b], h[b]);
}

// One CTA: prefix sums of the counts, the wanted buckets and their offsets in
// cand, and the fallback flag.
__global__ void __launch_bounds__(1024) sel_plan_kernel(const int64_t* __restrict__ ranks, int n_ranks, int64_t n,
                                                        SelWs w)
{
    __shared__ unsigned part[1024];
    __shared__ unsigned char want[kSelBuckets];
    const int T = blockDim.x, t = threadIdx.x;
    constexpr int per = kSelBuckets / 1024;
    unsigned s = 0;
    for (int k = 0; k < per; ++k) s += w.counts[t * per + k];
    part[t] = s;
    for (int b = t; b < kSelBuckets; b += T) want[b] = 0;
    __syncthreads();
    if (t == 0) {   // exclusive scan of the per-thread sums (1024 values)
        unsigned run = 0;
        for (int i = 0; i < T; ++i) {
            const unsigned v = part[i];
            part[i] = run;
            run += v;
        }
        w.starts[kSelBuckets] = run;
    }
    __syncthreads();
    unsigned run = part[t];
    for (int k = 0; k < per; ++k) {
        w.starts[t * per + k] = run;
        run += w.counts[t * per + k];
    }
    __syncthreads();
    // the bucket of each requested rank: the last b with starts[b] <= rank
    for (int r = t; r < n_ranks; r += T) {
        const int64_t rk = ranks[r];
        if (rk < 0 || rk >= n) continue;
        int lo = 0, hi = kSelBuckets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)w.starts[mid] <= rk) lo = mid; else hi = mid - 1;
        }
        want[lo] = 1;
    }
    __syncthreads();
    if (t == 0) {
        const float vmin = float_from_order_bits(w.mm[0]), vmax = float_from_order_bits(w.mm[1]);
        unsigned fb = (isfinite(vmin) && isfinite(vmax)) ? 0u : 1u;
        unsigned off = 0;
        for (int b = 0; b < kSelBuckets; ++b) {
            const unsigned c = w.counts[b];
            if (want[b]) {
                if (c > (unsigned)kSelCap) fb = 1u;
                w.seg[b] = off;
                off += c;
            } else {
                w.seg[b] = 0xFFFFFFFFu;
            }
        }
        *w.flag = fb;
    }
}

__global__ void sel_gather_kernel(const float* __restrict__ x, int64_t n, SelWs w)
{
    float vmin, scale;
    sel_range(w, vmin, scale);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        const int b = sel_bucket(v, vmin, scale);
        const unsigned o = w.seg[b];
        if (o != 0xFFFFFFFFu) {
            const unsigned pos = atomicAdd(&w.cursor[b], 1u);
            w.cand[o + pos] = ((unsigned long long)float_order_bits(v) << 32) | (unsigned long long)i;
        }
    }
}

// One CTA per requested rank: sort its bucket's (value, index) keys in shared
// memory and read the rank's index.
__global__ void __launch_bounds__(512) sel_rank_kernel(const int64_t* __restrict__ ranks, int64_t n, SelWs w,
                                                       int64_t* __restrict__ idx)
{
    __shared__ unsigned long long k[kSelCap];
    __shared__ int bucket;
    const int64_t rk = ranks[blockIdx.x];
    if (rk < 0 || rk >= n) {
        if (threadIdx.x == 0) idx[blockIdx.x] = -1;   // rank out of range
        return;
    }
    if (threadIdx.x == 0) {
        int lo = 0, hi = kSelBuckets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)w.starts[mid] <= rk) lo = mid; else hi = mid - 1;
        }
        bucket = lo;
    }
    __syncthreads();
    const int b = bucket;
    const int c = (int)w.counts[b];
    int P = 1;
    while (P < c) P <<= 1;
    const unsigned long long* src = w.cand + w.seg[b];
    for (int i = threadIdx.x; i < P; i += blockDim.x) k[i] = i < c ? src[i] : ~0ull;
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = k[i], bb = k[l];
                    if ((a > bb) == ((i & kk) == 0)) {
                        k[i] = bb;
                        k[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) idx[blockIdx.x] = (int64_t)(k[rk - (int64_t)w.starts[b]] & 0xFFFFFFFFull);
}

inline int64_t next_pow2(int64_t v)
{
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace pr

using namespace pr;

namespace pr {

struct AdjLayout {
    int64_t total, n_ckpt, nsub, blocks;
    size_t ckpt_bytes, sub_bytes, partial_bytes;
};

static AdjLayout adjoint_layout(int64_t n, int32_t n_slices, int32_t steps, int32_t ckpt_every)
{
    AdjLayout l{};
    l.total = (int64_t)n_slices * steps;
    l.n_ckpt = std::max<int64_t>(1, (l.total + ckpt_every - 1) / ckpt_every);
    l.nsub = std::max<int64_t>(1, (std::min<int64_t>(ckpt_every, l.total) + kSub - 1) / kSub);
    l.blocks = (n + kAdjThreads - 1) / kAdjThreads;
    l.ckpt_bytes = align256((size_t)l.n_ckpt * 2 * n * sizeof(float));
    l.sub_bytes = align256((size_t)l.nsub * 2 * n * sizeof(float));
    l.partial_bytes = align256((size_t)l.blocks * 3 * sizeof(double));
    return l;
}

// The reverse walk is taken when the reconstruction over one checkpoint
// segment of L steps cannot amplify rounding by more than a factor 2:
// (1/(1-rel))^L (1/(1-ddt))^L <= 2 (the inverse step's growth in y, and its
// bound in x for the double well).  Otherwise the backward pass replays the
// forward exactly from sub-checkpoints.
static bool adjoint_reverse_ok(double drift_dt, double relax, int32_t ckpt_every, int64_t total)
{
    const double seg = (double)std::min<int64_t>(ckpt_every, std::max<int64_t>(total, 1));
    return relax < 0.5 && drift_dt < 0.5 &&
           seg * (-std::log1p(-relax) - std::log1p(-drift_dt)) <= std::log(2.0);
}

static pr_status adjoint_check(const pr_model* model, const pr_rng* rng, const float* x0, const float* y0,
                               int64_t n, int32_t slice_begin, int32_t n_slices, int32_t steps, double dt,
                               int32_t ckpt_every, const double* xbar_T, const double* ybar_T, const double* grad)
{
    if (!model || !rng || !x0 || !y0 || !grad) return PR_ERR_INVALID_ARG;
    if (model->kind != PR_MODEL_OU && model->kind != PR_MODEL_DOUBLE_WELL) return PR_ERR_UNSUPPORTED;
    if (model->fast_dim != 1) return PR_ERR_UNSUPPORTED;
    if (!(model->beta > 0.0) || !(model->eps > 0.0) || !(model->tau_x > 0.0)) return PR_ERR_INVALID_ARG;
    if (n < 1 || n > 0xFFFFFFFFll || n_slices < 1 || slice_begin < 0 || steps < 0 || ckpt_every < 1) return PR_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !isfinite(dt) || rng->problem_id >= (1u << 24)) return PR_ERR_INVALID_ARG;
    if (ybar_T && !xbar_T) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(x0, 4) || !elem_aligned(y0, 4) || !elem_aligned(xbar_T, 8) || !elem_aligned(ybar_T, 8) ||
        !elem_aligned(grad, 8))
        return PR_ERR_INVALID_ARG;
    return PR_OK;
}

// Fills the arguments and launches; `ws` holds checkpoints, sub-checkpoints
// and per-block partial sums, in that order (every word is written before it
// is read in the same call, so nothing is cleared).
static pr_status adjoint_launch(const pr_model* model, const pr_rng* rng, const float* x0, const float* y0,
                                int64_t n, int32_t slice_begin, int32_t n_slices, int32_t steps, double dt,
                                int32_t ckpt_every, float* x_T, float* y_T, const double* xbar_T,
                                const double* ybar_T, double* grad, double* xbar_0, double* ybar_0, void* ws,
                                cudaStream_t st, int seed_affine = 0, double seed_scale = 0.0,
                                double seed_shift = 0.0)
{
    const AdjLayout l = adjoint_layout(n, n_slices, steps, ckpt_every);
    AdjArgs a{};
    a.x0 = x0;
    a.y0 = y0;
    a.n = n;
    a.slice_begin = slice_begin;
    a.steps = steps;
    a.total = l.total;
    a.ckpt = ckpt_every;
    a.n_ckpt = l.n_ckpt;
    const double drift_dt = dt / model->tau_x, relax = dt / model->eps;
    const double sx = sqrt(2.0 * (1.0 / model->beta) / model->tau_x) * sqrt(dt);
    const double sy = sqrt(2.0 / model->eps) * sqrt(dt);
    a.lam = (float)model->lambda;
    a.ddt = (float)drift_dt;
    a.rel = (float)relax;
    a.sxk = (float)(sx * 1.1774100225154746910);
    a.syk = (float)(sy * 1.1774100225154746910);
    a.inv2beta = (float)(0.5 / model->beta);
    a.inv2eps = (float)(0.5 / model->eps);
    a.rel_over_eps = (float)(dt / (model->eps * model->eps));
    {
        const double m00 = 1.0 - drift_dt, m01 = model->lambda * drift_dt, m10 = relax, m11 = 1.0 - relax;
        const double det = m00 * m11 - m01 * m10;
        a.ia = (float)(m11 / det);
        a.ib = (float)(-m01 / det);
        a.ic = (float)(-m10 / det);
        a.id = (float)(m00 / det);
        a.inv1mrel = (float)(1.0 / (1.0 - relax));
    }
    a.k0 = (uint32_t)(rng->seed & 0xFFFFFFFFull);
    a.k1 = (uint32_t)(rng->seed >> 32);
    a.chi = rng->problem_id << 8;
    char* base = static_cast<char*>(ws);
    a.ckpt_buf = reinterpret_cast<float*>(base);
    a.sub_buf = reinterpret_cast<float*>(base + l.ckpt_bytes);
    const bool sum_mode = xbar_T != nullptr || seed_affine;
    a.seed_affine = seed_affine;
    a.seed_scale = seed_scale;
    a.seed_shift = seed_shift;
    a.partial = sum_mode ? reinterpret_cast<double*>(base + l.ckpt_bytes + l.sub_bytes) : nullptr;
    a.xT = x_T;
    a.yT = y_T;
    a.xbar = xbar_T;
    a.ybar = ybar_T;
    a.grad_pp = sum_mode ? nullptr : grad;
    a.xbar0 = xbar_0;
    a.ybar0 = ybar_0;
    const size_t smem = (size_t)4 * kSub * kAdjThreads * sizeof(float);
    const bool paired = steps > 0 && (steps % 2) == 0 && (ckpt_every % 2) == 0;
    const unsigned grid = (unsigned)l.blocks;
    if (adjoint_reverse_ok(drift_dt, relax, ckpt_every, l.total)) {
        if (model->kind == PR_MODEL_OU) {
            if (paired) adjoint_rev_kernel<PR_MODEL_OU, true><<<grid, kAdjThreads, 0, st>>>(a);
            else adjoint_rev_kernel<PR_MODEL_OU, false><<<grid, kAdjThreads, 0, st>>>(a);
        } else {
            if (paired) adjoint_rev_kernel<PR_MODEL_DOUBLE_WELL, true><<<grid, kAdjThreads, 0, st>>>(a);
            else adjoint_rev_kernel<PR_MODEL_DOUBLE_WELL, false><<<grid, kAdjThreads, 0, st>>>(a);
        }
    } else if (model->kind == PR_MODEL_OU) {
        if (paired) adjoint_paired_kernel<PR_MODEL_OU><<<grid, kAdjThreads, smem, st>>>(a);
        else adjoint_kernel<PR_MODEL_OU><<<grid, kAdjThreads, smem, st>>>(a);
    } else {
        if (paired) adjoint_paired_kernel<PR_MODEL_DOUBLE_WELL><<<grid, kAdjThreads, smem, st>>>(a);
        else adjoint_kernel<PR_MODEL_DOUBLE_WELL><<<grid, kAdjThreads, smem, st>>>(a);
    }
    PR_CHECK_LAUNCH();
    if (sum_mode) {
        reduce_partials_kernel<<<1, 256, 0, st>>>(a.partial, l.blocks, grad);
        PR_CHECK_LAUNCH();
    }
    return PR_OK;
}

}  // namespace pr

extern "C" size_t pr_fine_adjoint_workspace(int64_t n, int32_t n_slices, int32_t steps, int32_t ckpt_every)
{
    if (n < 1 || n_slices < 1 || steps < 0 || ckpt_every < 1) return 0;
    const AdjLayout l = adjoint_layout(n, n_slices, steps, ckpt_every);
    return l.ckpt_bytes + l.sub_bytes + l.partial_bytes;
}

extern "C" pr_status pr_fine_adjoint(const pr_model* model, const pr_rng* rng, const float* x0, const float* y0,
                                     int64_t n, int32_t slice_begin, int32_t n_slices, int32_t steps, double dt,
                                     int32_t ckpt_every, float* x_T, float* y_T, const double* xbar_T,
                                     const double* ybar_T, double* grad, double* xbar_0, double* ybar_0,
                                     void* workspace, size_t workspace_bytes, void* stream)
{
    const pr_status chk = adjoint_check(model, rng, x0, y0, n, slice_begin, n_slices, steps, dt, ckpt_every,
                                        xbar_T, ybar_T, grad);
    if (chk != PR_OK) return chk;
    if (!elem_aligned(x_T, 4) || !elem_aligned(y_T, 4) || !elem_aligned(xbar_0, 8) || !elem_aligned(ybar_0, 8))
        return PR_ERR_INVALID_ARG;
    if (!workspace) return PR_ERR_INVALID_ARG;
    const size_t need = pr_fine_adjoint_workspace(n, n_slices, steps, ckpt_every);
    if (workspace_bytes < need || ((uintptr_t)workspace & 255)) return PR_ERR_INVALID_ARG;
    return adjoint_launch(model, rng, x0, y0, n, slice_begin, n_slices, steps, dt, ckpt_every, x_T, y_T, xbar_T,
                          ybar_T, grad, xbar_0, ybar_0, workspace, static_cast<cudaStream_t>(stream));
}

extern "C" pr_status pr_fine_adjoint_affine(const pr_model* model, const pr_rng* rng, const float* x0,
                                            const float* y0, int64_t n, int32_t slice_begin, int32_t n_slices,
                                            int32_t steps, double dt, int32_t ckpt_every, double seed_scale,
                                            double seed_shift, float* x_T, float* y_T, double* grad,
                                            double* xbar_0, double* ybar_0, void* workspace,
                                            size_t workspace_bytes, void* stream)
{
    const pr_status chk = adjoint_check(model, rng, x0, y0, n, slice_begin, n_slices, steps, dt, ckpt_every,
                                        nullptr, nullptr, grad);
    if (chk != PR_OK) return chk;
    if (!elem_aligned(x_T, 4) || !elem_aligned(y_T, 4) || !elem_aligned(xbar_0, 8) || !elem_aligned(ybar_0, 8))
        return PR_ERR_INVALID_ARG;
    if (!isfinite(seed_scale) || !isfinite(seed_shift) || !workspace) return PR_ERR_INVALID_ARG;
    const size_t need = pr_fine_adjoint_workspace(n, n_slices, steps, ckpt_every);
    if (workspace_bytes < need || ((uintptr_t)workspace & 255)) return PR_ERR_INVALID_ARG;
    return adjoint_launch(model, rng, x0, y0, n, slice_begin, n_slices, steps, dt, ckpt_every, x_T, y_T, nullptr,
                          nullptr, grad, xbar_0, ybar_0, workspace, static_cast<cudaStream_t>(stream), 1, seed_scale,
                          seed_shift);
}

static size_t sel_tables_bytes() { return align256((size_t)(4 * kSelBuckets + 8) * sizeof(unsigned)); }

extern "C" size_t pr_order_statistics_workspace(int64_t n)
{
    return n < 1 ? 0 : align256((size_t)next_pow2(n) * sizeof(unsigned long long)) + sel_tables_bytes();
}

extern "C" pr_status pr_order_statistics(const float* x, int64_t n, const int64_t* ranks, int32_t n_ranks,
                                         int64_t* index_out, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!x || !ranks || !index_out || !workspace || n < 1 || n > 0xFFFFFFFFll || n_ranks < 1) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(x, 4) || !elem_aligned(ranks, 8) || !elem_aligned(index_out, 8)) return PR_ERR_INVALID_ARG;
    if (workspace_bytes < pr_order_statistics_workspace(n) || ((uintptr_t)workspace & 7)) return PR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t padded = next_pow2(n);
    auto* keys = static_cast<unsigned long long*>(workspace);
    // selection first
    {
        unsigned* tab = reinterpret_cast<unsigned*>(static_cast<char*>(workspace) +
                                                    align256((size_t)padded * sizeof(unsigned long long)));
        SelWs w;
        w.counts = tab;
        w.starts = tab + kSelBuckets;
        w.seg = w.starts + kSelBuckets + 1;
        w.cursor = w.seg + kSelBuckets;
        w.mm = w.cursor + kSelBuckets;
        w.flag = w.mm + 2;
        w.cand = keys;
        PR_TRY_CUDA(cudaMemsetAsync(w.counts, 0, kSelBuckets * sizeof(unsigned), st));
        PR_TRY_CUDA(cudaMemsetAsync(w.cursor, 0, kSelBuckets * sizeof(unsigned), st));
        PR_TRY_CUDA(cudaMemsetAsync(w.mm, 0xFF, sizeof(unsigned), st));
        PR_TRY_CUDA(cudaMemsetAsync(w.mm + 1, 0, sizeof(unsigned), st));
        const int sb = (int)std::min<int64_t>((n + 1023) / 1024, 2 * (int64_t)num_sms());
        sel_minmax_kernel<<<sb, 1024, 0, st>>>(x, n, w);
        sel_hist_kernel<<<sb, 1024, 0, st>>>(x, n, w);
        sel_plan_kernel<<<1, 1024, 0, st>>>(ranks, n_ranks, n, w);
        unsigned fb = 1u;
        PR_TRY_CUDA(cudaMemcpyAsync(&fb, w.flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        PR_TRY_CUDA(cudaStreamSynchronize(st));
        if (fb == 0u) {
            sel_gather_kernel<<<sb, 1024, 0, st>>>(x, n, w);
            sel_rank_kernel<<<n_ranks, 512, 0, st>>>(ranks, n, w, index_out);
            PR_CHECK_LAUNCH();
            return PR_OK;
        }
    }
    // full sort: bitonic network over (value, index) keys
    const int blocks = (int)std::min<int64_t>((padded + 255) / 256, 16 * (int64_t)num_sms());
    make_keys_kernel<<<blocks, 256, 0, st>>>(x, n, padded, keys);
    for (int64_t k = 2; k <= padded; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1)
            bitonic_step_kernel<<<blocks, 256, 0, st>>>(keys, padded, j, k);
    gather_ranks_kernel<<<(n_ranks + 255) / 256, 256, 0, st>>>(keys, ranks, n_ranks, n, index_out);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

// ---------------------------------------------------------------------------
// Adjoint without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// real-time control loop (the paper's motivating setting of model-predictive
// control) that forbids cudaMalloc/cudaFree after start-up because they can
// block and synchronise the device, or a host application whose device memory
// is owned by another allocator.  pr_fine_adjoint_noalloc serves them: its
// checkpoints and partial sums live in the fixed array below, which every GPU
// that loads this library holds until the process exits.
// ---------------------------------------------------------------------------

namespace pr {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_adjoint_scratch[kNoAllocScratchBytes];

// The array's device address on the current device.  Looked up once per
// device (with that device current) and kept for the life of the process; a
// reset of the device's primary context makes it stale (stated in pr.h).
static pr_status adjoint_scratch_address(void** out)
{
    static std::mutex mu;
    static void* addr[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return PR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_adjoint_scratch) != cudaSuccess || !p) return PR_ERR_CUDA;
        addr[dev] = p;
    }
    *out = addr[dev];
    return PR_OK;
}

}  // namespace pr

extern "C" size_t pr_fine_adjoint_noalloc_capacity(void) { return kNoAllocScratchBytes; }

extern "C" pr_status pr_fine_adjoint_noalloc(const pr_model* model, const pr_rng* rng, const float* x0,
                                             const float* y0, int64_t n, int32_t slice_begin, int32_t n_slices,
                                             int32_t steps, double dt, int32_t ckpt_every, float* x_T, float* y_T,
                                             const double* xbar_T, const double* ybar_T, double* grad,
                                             double* xbar_0, double* ybar_0, void* stream)
{
    const pr_status chk = adjoint_check(model, rng, x0, y0, n, slice_begin, n_slices, steps, dt, ckpt_every,
                                        xbar_T, ybar_T, grad);
    if (chk != PR_OK) return chk;
    if (!elem_aligned(x_T, 4) || !elem_aligned(y_T, 4) || !elem_aligned(xbar_0, 8) || !elem_aligned(ybar_0, 8))
        return PR_ERR_INVALID_ARG;
    // the problem must fit the fixed array (checked before anything else runs)
    if (pr_fine_adjoint_workspace(n, n_slices, steps, ckpt_every) > kNoAllocScratchBytes) return PR_ERR_NOMEM;
    void* scratch = nullptr;
    const pr_status got = adjoint_scratch_address(&scratch);
    if (got != PR_OK) return got;
    return adjoint_launch(model, rng, x0, y0, n, slice_begin, n_slices, steps, dt, ckpt_every, x_T, y_T, xbar_T,
                          ybar_T, grad, xbar_0, ybar_0, scratch, static_cast<cudaStream_t>(stream));
}

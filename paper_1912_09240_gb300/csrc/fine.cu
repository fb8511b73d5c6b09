// fine.cu -- fine propagator F_dT (Euler-Maruyama on a particle ensemble,
// Section 2.1.3, Eqs. EMx/EMy) for every parareal slice at once, with the
// restriction (Section 3.2.2, Eq. binning) fused into its epilogue and the
// matching (Section 5.1) optionally fused into its prologue; plus the
// standalone restriction, matching and counts-to-CDF kernels.
//
// Work decomposition: blockIdx.y is the slice, blockIdx.x a tile of
// blockDim.x * PPT particles of that slice; each thread carries PPT particles
// in registers through all `steps` steps of the slice.  State is read once
// and written once per slice (structure of arrays, coalesced).  The step loop
// draws its normals from Philox4x32-10 keyed by the seed and counted by
// (step, particle, slice, problem), so nothing random is stored.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fine_dev.cuh"
#include "match.cuh"
#include "pr_common.cuh"

namespace pr {

int num_sms()
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) {
        int v = 1;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

int smem_optin_max()
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cache[dev] = v > 0 ? v : 48 * 1024;
    }
    return cache[dev];
}

// Arguments of one fine launch, after host-side validation.
struct FineArgs {
    const void* x_in;
    const void* y_in;
    void* x_out;
    void* y_out;
    int64_t n;
    int64_t in_slice_stride;   // elements of x between input slices (0 = broadcast)
    int slice_begin;
    int steps;
    int fast_dim;
    // model constants
    double lam;
    double drift_dt;   // dt / tau_x
    double relax;      // dt / eps
    double sx;         // sqrt(2 D / tau_x) sqrt(dt), D = 1/beta
    double sy;         // sqrt(2 E / eps) sqrt(dt), E = 1
    float lam_f, drift_dt_f, relax_f, sx_f, sy_f;   // the same, rounded once on the host
    float sxk_f, syk_f;                             // sx, sy times sqrt(2 ln 2)
    ChemConsts<float> chem_f;                       // the chemical system (kinds CHEM, CHEM_PRINTED)
    ChemConsts<double> chem_d;
    int tiles_per_cta;  // binary32 d = 1 kernel: consecutive tiles handled by one CTA
    // random numbers
    uint32_t k0, k1, ctr_hi;   // key words; (problem_id << 8)
    // fused restriction / matching
    GridDev g;
    float lo_f, inv_h_f;
    const double* cdf_prior;
    const double* cdf_target;
    uint32_t* counts_start;
    uint32_t* counts_end;
};

// Dynamic shared memory of the fine kernels: [thresholds | hist_start |
// hist_end | match table], each section 16-byte aligned.
struct FineSmem {
    size_t thr, hs, he, match, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Binary32 with matching: thresholds, the matching table, then its build
// scratch, which the two histograms reuse once the table is built.  Binary64
// (or no matching): thresholds, histograms, then the full matching scratch.
inline FineSmem fine_smem_layout(int bins, bool any_grid, bool match, bool f32)
{
    FineSmem L{0, 0, 0, 0, 0};
    if (!any_grid) return L;
    size_t off = 0;
    L.thr = off;
    off += align16((size_t)(bins + 1) * sizeof(float));
    const size_t hb = align16((size_t)bins * sizeof(uint32_t));
    if (match && f32) {
        L.match = off;
        off += match_table_bytes(bins);
        L.hs = off;
        L.he = off + hb;
        off += std::max(match_build_bytes_f32(bins), 2 * hb);
    } else {
        L.hs = off;
        off += hb;
        L.he = off;
        off += hb;
        L.match = off;
        if (match) off += match_smem_bytes(bins);
    }
    L.total = off;
    return L;
}

struct FineSmemOffsets {
    unsigned thr, hs, he, match;
};

// ---------------------------------------------------------------------------
// Drift of the slow variable, d_x F (Section 2.1.1)
// ---------------------------------------------------------------------------

template <int KIND, typename T>
__device__ __forceinline__ T slow_force(T x, T ymean, T lam)
{
    if (KIND == PR_MODEL_OU) return x - lam * ymean;
    return x * x * x - x + lam * ymean;
}

// ---------------------------------------------------------------------------
// binary32 kernel, fast_dim = 1
// ---------------------------------------------------------------------------

template <int KIND, int PPT>
__global__ void __launch_bounds__(256)
fine_f32_d1_kernel(FineArgs a, FineSmemOffsets so, int flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const bool any_grid = flags & 1, do_match = flags & 2, do_hs = flags & 4, do_he = flags & 8;
    const int s = blockIdx.y;
    const uint32_t slice = (uint32_t)(a.slice_begin + s);
    const int bins = a.g.bins;
    float* thr = reinterpret_cast<float*>(smem + so.thr);
    uint32_t* hist_s = reinterpret_cast<uint32_t*>(smem + so.hs);
    uint32_t* hist_e = reinterpret_cast<uint32_t*>(smem + so.he);
    MatchSmem ms;
    if (any_grid) {
        build_thresholds(a.g, thr);
        if (do_match) {   // the histograms reuse the table's build scratch afterwards
            ms = carve_match_smem_f32(smem + so.match, bins, a.cdf_prior + (size_t)s * (bins + 1),
                                      a.cdf_target + (size_t)s * (bins + 1));
            build_match_table(a.g, thr, ms);
        }
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            hist_s[i] = 0u;
            hist_e[i] = 0u;
        }
        __syncthreads();
    }
    const BinF32 bf = any_grid ? make_bin_f32(thr, bins, a.lo_f, a.inv_h_f) : BinF32{};

    const int64_t N = a.n;
    const float* __restrict__ xin = static_cast<const float*>(a.x_in) + (int64_t)s * a.in_slice_stride;
    const float* __restrict__ yin = static_cast<const float*>(a.y_in) + (int64_t)s * a.in_slice_stride;
    float* __restrict__ xout = static_cast<float*>(a.x_out) + (int64_t)s * N;
    float* __restrict__ yout = static_cast<float*>(a.y_out) + (int64_t)s * N;
    D1Consts cst{a.lam_f, a.drift_dt_f, a.relax_f, a.sxk_f, a.syk_f, a.k0, a.k1, a.ctr_hi, a.chem_f};
    D1Smem sm{thr, hist_s, hist_e, &ms, bf, do_match, do_hs, do_he};
    const int64_t span = (int64_t)a.tiles_per_cta * blockDim.x * PPT;
    const int64_t p_begin = (int64_t)blockIdx.x * span;
    fine_d1_range<KIND, PPT>(xin, yin, xout, yout, p_begin, min(N, p_begin + span), slice, a.steps, cst, sm);
    if (do_hs || do_he) {
        __syncthreads();
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            if (do_hs && hist_s[i]) atomicAdd(&a.counts_start[(size_t)s * bins + i], hist_s[i]);
            if (do_he && hist_e[i]) atomicAdd(&a.counts_end[(size_t)s * bins + i], hist_e[i]);
        }
    }
}

// ---------------------------------------------------------------------------
// binary32 kernel, fast_dim = D > 1 (coupling through mean(y)), one particle
// per thread.  Normals: (1+D)/4 whole Philox blocks per step, the last
// (1+D) mod 4 from blocks shared by four consecutive steps.
// ---------------------------------------------------------------------------

template <int KIND, int D>
__global__ void __launch_bounds__(512)
fine_f32_dn_kernel(FineArgs a, FineSmemOffsets so, int flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const bool any_grid = flags & 1, do_match = flags & 2, do_hs = flags & 4, do_he = flags & 8;
    const int s = blockIdx.y;
    const uint32_t slice = (uint32_t)(a.slice_begin + s);
    const int bins = a.g.bins;
    float* thr = reinterpret_cast<float*>(smem + so.thr);
    uint32_t* hist_s = reinterpret_cast<uint32_t*>(smem + so.hs);
    uint32_t* hist_e = reinterpret_cast<uint32_t*>(smem + so.he);
    MatchSmem ms;
    if (any_grid) {
        build_thresholds(a.g, thr);
        if (do_match) {   // the histograms reuse the table's build scratch afterwards
            ms = carve_match_smem_f32(smem + so.match, bins, a.cdf_prior + (size_t)s * (bins + 1),
                                      a.cdf_target + (size_t)s * (bins + 1));
            build_match_table(a.g, thr, ms);
        }
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            hist_s[i] = 0u;
            hist_e[i] = 0u;
        }
        __syncthreads();
    }
    const BinF32 bf = any_grid ? make_bin_f32(thr, bins, a.lo_f, a.inv_h_f) : BinF32{};
    const int64_t N = a.n;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = p < N;
    const float* __restrict__ xin = static_cast<const float*>(a.x_in) + (int64_t)s * a.in_slice_stride;
    const float* __restrict__ yin = static_cast<const float*>(a.y_in) + (int64_t)s * a.in_slice_stride * D;
    float* __restrict__ xout = static_cast<float*>(a.x_out) + (int64_t)s * N;
    float* __restrict__ yout = static_cast<float*>(a.y_out) + (int64_t)s * N * D;

    float x = ok ? xin[p] : 0.0f;
    float y[D];
#pragma unroll
    for (int j = 0; j < D; ++j) y[j] = ok ? yin[(int64_t)j * N + p] : 0.0f;
    if (do_match && ok) x = match_one_f32(ms, thr, bf, x);
    if (do_hs && ok) atomicAdd(&hist_s[bin_fast_f32(bf, thr, x)], 1u);

    const float lam = a.lam_f, ddt = a.drift_dt_f, rel = a.relax_f;
    const float sxk = a.sxk_f, syk = a.syk_f, omr = 1.0f - rel;
    const float invD = 1.0f / (float)D;
    // Normals of a step: 4 per full block (F of them), and the last T = Q mod 4
    // from tail blocks shared by the four steps 4k .. 4k + 3 (normal i of
    // step 4k + s is number s T + i of the group's 4T), so no word is wasted.
    // With Q = 2 (D = 1) one block serves two steps, as in the d = 1 kernel.
    constexpr int Q = 1 + D;
    constexpr int F = Q > 2 ? Q / 4 : 0;
    constexpr int T = Q > 2 ? Q % 4 : 0;
    constexpr int FP = F > 0 ? 2 * F : 1;   // Box-Muller pairs of the full blocks
    constexpr int TP = T > 0 ? 2 * T : 1;   // pairs of a group's tail blocks
    const uint32_t k0 = a.k0, k1 = a.k1, chi = a.ctr_hi, pid = (uint32_t)p;
    // normal 2i of a pair is sqrt(2 ln 2) q_i cos(theta_i), normal 2i + 1 the
    // sine; sqrt(2 ln 2) is folded into the amplitudes sxk, syk
    float tq[TP], tc[TP], ts[TP], tamp[TP];
    // the tail blocks of the group of four steps from step m on
    auto tail_blocks = [&](int m) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)(m >> 2), pid, slice, chi | (uint32_t)(F + j)),
                                          k0, k1);
            box_muller_qcs(w.x, w.y, tq[2 * j], tc[2 * j], ts[2 * j]);
            box_muller_qcs(w.z, w.w, tq[2 * j + 1], tc[2 * j + 1], ts[2 * j + 1]);
        }
#pragma unroll
        for (int i = 0; i < TP; ++i) tamp[i] = syk * tq[i];
    };
    // step m, the s4-th of its group (a constant where the loop below is unrolled)
    auto step = [&](int m, int s4) {
        float pq = 0.0f, pc = 0.0f, ps = 0.0f;   // Q = 2: this step's pair
        if (Q <= 2) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)(m >> 1), pid, slice, chi), k0, k1);
            if (m & 1) box_muller_qcs(w.z, w.w, pq, pc, ps);
            else box_muller_qcs(w.x, w.y, pq, pc, ps);
        }
        float q[FP], c[FP], sn[FP], amp[FP];
#pragma unroll
        for (int gi = 0; gi < F; ++gi) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)m, pid, slice, chi | (uint32_t)gi), k0, k1);
            box_muller_qcs(w.x, w.y, q[2 * gi], c[2 * gi], sn[2 * gi]);
            box_muller_qcs(w.z, w.w, q[2 * gi + 1], c[2 * gi + 1], sn[2 * gi + 1]);
        }
#pragma unroll
        for (int i = 0; i < 2 * F; ++i) amp[i] = syk * q[i];
        // normal k of this step as (q, trig) of its pair, q scaled by syk for
        // the fast components (scaled = true)
        auto normal = [&](int k, bool scaled, float& qq, float& tt) {
            if (Q <= 2) {
                qq = scaled ? syk * pq : pq;
                tt = k ? ps : pc;
            } else if (k < 4 * F) {
                qq = scaled ? amp[k >> 1] : q[k >> 1];
                tt = (k & 1) ? sn[k >> 1] : c[k >> 1];
            } else {
                const int idx = s4 * T + (k - 4 * F);
                const int pr = idx >> 1;
                const bool odd = idx & 1;
                qq = scaled ? tamp[0] : tq[0];
                tt = odd ? ts[0] : tc[0];
#pragma unroll
                for (int cc = 1; cc < TP; ++cc)
                    if (pr == cc) {
                        qq = scaled ? tamp[cc] : tq[cc];
                        tt = odd ? ts[cc] : tc[cc];
                    }
            }
        };
        float ysum = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) ysum += y[j];
        const float f = slow_force<KIND>(x, ysum * invD, lam);
        float q0, t0;
        normal(0, false, q0, t0);
        const float xn = fmaf(sxk * q0, t0, fmaf(-f, ddt, x));
        // y_j <- y_j + (x - y_j) rel + sy dV_j, as y_j (1 - rel) + x rel + sy dV_j
        const float xr = x * rel;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float aj, tj;
            normal(1 + j, true, aj, tj);   // the normal of component j
            y[j] = fmaf(aj, tj, fmaf(y[j], omr, xr));
        }
        x = xn;
    };
    int m0 = 0;
    if (T > 0) {
        for (; m0 + 4 <= a.steps; m0 += 4) {
            tail_blocks(m0);
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) step(m0 + s4, s4);
        }
        if (m0 < a.steps) tail_blocks(m0);
    }
    for (int m = m0; m < a.steps; ++m) step(m, m & 3);
    if (ok) {
        xout[p] = x;
#pragma unroll
        for (int j = 0; j < D; ++j) yout[(int64_t)j * N + p] = y[j];
        if (do_he) atomicAdd(&hist_e[bin_fast_f32(bf, thr, x)], 1u);
    }
    if (do_hs || do_he) {
        __syncthreads();
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            if (do_hs && hist_s[i]) atomicAdd(&a.counts_start[(size_t)s * bins + i], hist_s[i]);
            if (do_he && hist_e[i]) atomicAdd(&a.counts_end[(size_t)s * bins + i], hist_e[i]);
        }
    }
}

// ---------------------------------------------------------------------------
// binary64 kernel (the plain FP64 path), any fast_dim <= 16, one particle per
// thread, FP64 normals and arithmetic.
// ---------------------------------------------------------------------------

template <int KIND>
__global__ void __launch_bounds__(128)
fine_f64_kernel(FineArgs a, FineSmemOffsets so, int flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const bool any_grid = flags & 1, do_match = flags & 2, do_hs = flags & 4, do_he = flags & 8;
    const int s = blockIdx.y;
    const uint32_t slice = (uint32_t)(a.slice_begin + s);
    const int bins = a.g.bins;
    uint32_t* hist_s = reinterpret_cast<uint32_t*>(smem + so.hs);
    uint32_t* hist_e = reinterpret_cast<uint32_t*>(smem + so.he);
    MatchSmem ms;
    if (any_grid) {
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            hist_s[i] = 0u;
            hist_e[i] = 0u;
        }
        if (do_match) {
            ms = carve_match_smem(smem + so.match, bins);
            build_match_index(a.g, a.cdf_prior + (size_t)s * (bins + 1),
                              a.cdf_target + (size_t)s * (bins + 1), ms);
        }
        __syncthreads();
    }
    const int D = a.fast_dim;
    const int64_t N = a.n;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = p < N;
    const double* __restrict__ xin = static_cast<const double*>(a.x_in) + (int64_t)s * a.in_slice_stride;
    const double* __restrict__ yin = static_cast<const double*>(a.y_in) + (int64_t)s * a.in_slice_stride * D;
    double* __restrict__ xout = static_cast<double*>(a.x_out) + (int64_t)s * N;
    double* __restrict__ yout = static_cast<double*>(a.y_out) + (int64_t)s * N * D;

    double x = ok ? xin[p] : 0.0;
    double y[PR_MAX_FAST_DIM];
    for (int j = 0; j < D; ++j) y[j] = ok ? yin[(int64_t)j * N + p] : 0.0;
    if (do_match && ok) x = match_one_f64(ms, a.g, x);
    if (do_hs && ok) atomicAdd(&hist_s[bin_of_f64(a.g, x)], 1u);

    const uint32_t k0 = a.k0, k1 = a.k1, chi = a.ctr_hi, pid = (uint32_t)p;
    const int Q = 1 + D;
    for (int m = 0; m < a.steps; ++m) {
        double z[PR_MAX_FAST_DIM + 3];
        if (Q <= 2) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)(m >> 1), pid, slice, chi), k0, k1);
            if (m & 1) box_muller_f64(w.z, w.w, z[0], z[1]);
            else box_muller_f64(w.x, w.y, z[0], z[1]);
        } else {
            // F full blocks per step, then the step's T = Q mod 4 normals from
            // the tail blocks shared by its group of four steps
            const int F = Q / 4, T = Q % 4;
            for (int gi = 0; gi < F; ++gi) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)m, pid, slice, chi | (uint32_t)gi), k0, k1);
                box_muller_f64(w.x, w.y, z[4 * gi], z[4 * gi + 1]);
                box_muller_f64(w.z, w.w, z[4 * gi + 2], z[4 * gi + 3]);
            }
            for (int i = 0; i < T; ++i) {
                const int idx = (m & 3) * T + i;
                const uint4 w = philox4x32_10(make_uint4((uint32_t)(m >> 2), pid, slice, chi | (uint32_t)(F + idx / 4)),
                                              k0, k1);
                double za, zb;
                if ((idx & 2) != 0) box_muller_f64(w.z, w.w, za, zb);
                else box_muller_f64(w.x, w.y, za, zb);
                z[4 * F + i] = (idx & 1) ? zb : za;
            }
        }
        if (KIND == PR_MODEL_CHEM) {   // sx = sy = 1: the amplitudes depend on the state
            em_step_chem_f64(x, y[0], a.sx * z[0], a.sy * z[1], a.chem_d);
            continue;
        }
        double ysum = 0.0;
        for (int j = 0; j < D; ++j) ysum += y[j];
        const double ym = (KIND == PR_MODEL_DW_MULTI) ? ysum / (double)D : y[0];
        const double f = slow_force<KIND == PR_MODEL_OU ? 0 : 1>(x, ym, a.lam);
        const double xn = x - f * a.drift_dt + a.sx * z[0];
        for (int j = 0; j < D; ++j) y[j] = y[j] - (y[j] - x) * a.relax + a.sy * z[1 + j];
        x = xn;
    }
    if (ok) {
        xout[p] = x;
        for (int j = 0; j < D; ++j) yout[(int64_t)j * N + p] = y[j];
        if (do_he) atomicAdd(&hist_e[bin_of_f64(a.g, x)], 1u);
    }
    if (do_hs || do_he) {
        __syncthreads();
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            if (do_hs && hist_s[i]) atomicAdd(&a.counts_start[(size_t)s * bins + i], hist_s[i]);
            if (do_he && hist_e[i]) atomicAdd(&a.counts_end[(size_t)s * bins + i], hist_e[i]);
        }
    }
}

// ---------------------------------------------------------------------------
// counts -> CDF at the edges (exact integer prefix sums, one division each)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256)
counts_to_cdf_kernel(const uint32_t* __restrict__ counts, int64_t n, int bins, double* __restrict__ cdf)
{
    __shared__ unsigned long long warp_tot[8];
    const int s = blockIdx.x;
    const uint32_t* c = counts + (size_t)s * bins;
    double* C = cdf + (size_t)s * (bins + 1);
    const int T = blockDim.x;
    const int chunk = (bins + T - 1) / T;
    const int b = threadIdx.x * chunk, e = min(bins, b + chunk);
    unsigned long long loc = 0;
    for (int i = b; i < e; ++i) loc += c[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned long long off = 0;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    unsigned long long run = off + incl - loc;
    const double dn = (double)n;
    for (int i = b; i < e; ++i) {
        run += c[i];
        C[i + 1] = (double)run / dn;
    }
    if (threadIdx.x == 0) C[0] = 0.0;
}

// ---------------------------------------------------------------------------
// standalone restriction: histogram per slice, binary32 or binary64 input
// ---------------------------------------------------------------------------

// Streams the elements [b, e) of one slice: `op1(value)` on a scalar head up
// to the next 16-byte boundary and on a scalar tail, `op8(u0, u1)` on pairs
// of 16-byte vectors (two loads in flight per thread) and `op4(u)` on a last
// single vector.
template <typename Op1, typename Op4, typename Op8>
__device__ __forceinline__ void for_each_f32(const float* __restrict__ xs, int64_t b, int64_t e, Op1 op1, Op4 op4,
                                             Op8 op8)
{
    const int T = blockDim.x, t = threadIdx.x;
    const int64_t mis = (int64_t)(((uintptr_t)(xs + b) >> 2) & 3);
    const int64_t hb = min(e, b + ((4 - mis) & 3));
    for (int64_t p = b + t; p < hb; p += T) op1(xs[p]);
    const int64_t nv = (e - hb) >> 2;
    const float4* __restrict__ v = reinterpret_cast<const float4*>(xs + hb);
    int64_t q = t;
    for (; q + 3 * T < nv; q += 4 * T) {   // four loads in flight per thread
        const float4 u0 = __ldcs(v + q), u1 = __ldcs(v + q + T), u2 = __ldcs(v + q + 2 * T),
                     u3 = __ldcs(v + q + 3 * T);
        op8(u0, u1);
        op8(u2, u3);
    }
    for (; q + T < nv; q += 2 * T) op8(__ldcs(v + q), __ldcs(v + q + T));
    if (q < nv) op4(__ldcs(v + q));
    for (int64_t p = hb + 4 * nv + t; p < e; p += T) op1(xs[p]);
}

template <typename T>
__global__ void __launch_bounds__(512)
restrict_kernel(const T* __restrict__ x, int64_t n, GridDev g, float lo_f, float inv_h_f,
                uint32_t* __restrict__ counts, int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int bins = g.bins;
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem);
    float* thr = reinterpret_cast<float*>(hist + bins);   // binary32 thresholds, bins + 1
    const int s = blockIdx.y;
    if (sizeof(T) == 4) build_thresholds(g, thr);
    for (int i = threadIdx.x; i < bins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const T* xs = x + (int64_t)s * n;
    const int64_t b = (int64_t)blockIdx.x * per_block;
    const int64_t e = min(n, b + per_block);
    if (sizeof(T) == 4) {
        // the thresholds (built once per CTA, binary64 edges rounded up to
        // binary32) are read only for the few particles near an edge, decided
        // once per group of values so that the common case has no divergent
        // branch and no binary64 arithmetic
        const BinF32 bf = make_bin_f32(thr, bins, lo_f, inv_h_f);
        const auto thr_of = [thr](int k) { return thr[k]; };
        auto group4 = [&](float4 u, int m) {
            int i0 = bin_try_f32(bf, u.x);
            int i1 = m > 1 ? bin_try_f32(bf, u.y) : 0;
            int i2 = m > 2 ? bin_try_f32(bf, u.z) : 0;
            int i3 = m > 3 ? bin_try_f32(bf, u.w) : 0;
            if ((i0 | i1 | i2 | i3) < 0) {
                if (i0 < 0) i0 = bin_slow_f32(bf, thr_of, u.x);
                if (i1 < 0) i1 = bin_slow_f32(bf, thr_of, u.y);
                if (i2 < 0) i2 = bin_slow_f32(bf, thr_of, u.z);
                if (i3 < 0) i3 = bin_slow_f32(bf, thr_of, u.w);
            }
            atomicAdd(&hist[i0], 1u);
            if (m > 1) atomicAdd(&hist[i1], 1u);
            if (m > 2) atomicAdd(&hist[i2], 1u);
            if (m > 3) atomicAdd(&hist[i3], 1u);
        };
        for_each_f32(
            reinterpret_cast<const float*>(xs), b, e, [&](float v) { group4(make_float4(v, v, v, v), 1); },
            [&](float4 u) { group4(u, 4); },
            [&](float4 u0, float4 u1) {
                group4(u0, 4);
                group4(u1, 4);
            });
    } else {
        for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x)
            atomicAdd(&hist[bin_of_f64(g, (double)xs[p])], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < bins; i += blockDim.x)
        if (hist[i]) atomicAdd(&counts[(size_t)s * bins + i], hist[i]);
}

// ---------------------------------------------------------------------------
// standalone matching
// ---------------------------------------------------------------------------

// two CTAs of 1024 threads per SM (32 registers): the gathers of the
// matching table need every warp the SM can hold
__global__ void __launch_bounds__(1024, 2)
match_f32_kernel(const float* __restrict__ xp, float* __restrict__ xo, int64_t n, GridDev g,
                 float lo_f, float inv_h_f, const double* __restrict__ cp,
                 const double* __restrict__ ct, int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int bins = g.bins;
    float* thr = reinterpret_cast<float*>(smem);
    const int s = blockIdx.y;
    MatchSmem ms = carve_match_smem_f32(smem + align16((size_t)(bins + 1) * sizeof(float)), bins,
                                        cp + (size_t)s * (bins + 1), ct + (size_t)s * (bins + 1));
    build_thresholds(g, thr);
    build_match_table(g, thr, ms);
    const BinF32 bf = make_bin_f32(thr, bins, lo_f, inv_h_f);
    const int64_t b = (int64_t)blockIdx.x * per_block;
    const int64_t e = min(n, b + per_block);
    const float* xs = xp + (int64_t)s * n;
    float* os = xo + (int64_t)s * n;
    // vector stores need the output at the same offset from a 16-byte boundary
    if ((((uintptr_t)xs ^ (uintptr_t)os) & 15) == 0) {
        const int T = blockDim.x, t = threadIdx.x;
        const int64_t mis = (int64_t)(((uintptr_t)(xs + b) >> 2) & 3);
        const int64_t hb = min(e, b + ((4 - mis) & 3));
        for (int64_t p = b + t; p < hb; p += T) os[p] = match_one_f32(ms, thr, bf, xs[p]);
        const int64_t nv = (e - hb) >> 2;
        const float4* __restrict__ v = reinterpret_cast<const float4*>(xs + hb);
        float4* __restrict__ w = reinterpret_cast<float4*>(os + hb);
        auto map4 = [&](float4 u) {
            u.x = match_one_f32(ms, thr, bf, u.x);
            u.y = match_one_f32(ms, thr, bf, u.y);
            u.z = match_one_f32(ms, thr, bf, u.z);
            u.w = match_one_f32(ms, thr, bf, u.w);
            return u;
        };
        int64_t q = t;
        for (; q + T < nv; q += 2 * T) {
            const float4 u0 = __ldcs(v + q);
            const float4 u1 = __ldcs(v + q + T);
            __stcs(w + q, map4(u0));
            __stcs(w + q + T, map4(u1));
        }
        if (q < nv) __stcs(w + q, map4(__ldcs(v + q)));
        for (int64_t p = hb + 4 * nv + t; p < e; p += T) os[p] = match_one_f32(ms, thr, bf, xs[p]);
    } else {
        for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x)
            os[p] = match_one_f32(ms, thr, bf, xs[p]);
    }
}

__global__ void __launch_bounds__(256)
match_f64_kernel(const double* __restrict__ xp, double* __restrict__ xo, int64_t n, GridDev g,
                 const double* __restrict__ cp, const double* __restrict__ ct, int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int bins = g.bins;
    MatchSmem ms = carve_match_smem(smem, bins);
    const int s = blockIdx.y;
    build_match_index(g, cp + (size_t)s * (bins + 1), ct + (size_t)s * (bins + 1), ms);
    const int64_t b = (int64_t)blockIdx.x * per_block;
    const int64_t e = min(n, b + per_block);
    const double* xs = xp + (int64_t)s * n;
    double* os = xo + (int64_t)s * n;
    for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) os[p] = match_one_f64(ms, g, xs[p]);
}

// Binary32 matching on grids whose binary32 table does not fit one CTA's
// shared memory: the binary64 map of each widened particle (the same
// operations as match_f64_kernel), its image rounded to binary32.  Bound by
// the FP64 pipe; it serves only grids of more than about 3050 bins.
// `in_stride` = 0 maps one input ensemble into every slice.
__global__ void __launch_bounds__(256)
match_f32_wide_kernel(const float* __restrict__ xp, float* __restrict__ xo, int64_t n, int64_t in_stride,
                      GridDev g, const double* __restrict__ cp, const double* __restrict__ ct, int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int bins = g.bins;
    MatchSmem ms = carve_match_smem(smem, bins);
    const int s = blockIdx.y;
    build_match_index(g, cp + (size_t)s * (bins + 1), ct + (size_t)s * (bins + 1), ms);
    const int64_t b = (int64_t)blockIdx.x * per_block;
    const int64_t e = min(n, b + per_block);
    const float* xs = xp + (int64_t)s * in_stride;
    float* os = xo + (int64_t)s * n;
    for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x)
        os[p] = __double2float_rn(match_one_f64(ms, g, (double)xs[p]));
}

// dst[s][j] = src[j] for every slice s (one ensemble's values copied into
// every slice of a slice-major array of `per_slice` floats per slice).
__global__ void broadcast_slices_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t per_slice,
                                        int n_slices)
{
    const int64_t total = per_slice * n_slices;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i % per_slice];
}

// raw Philox blocks for caller-given counters
__global__ void rng_words_kernel(const uint4* __restrict__ ctr, int64_t n, uint32_t k0, uint32_t k1,
                                 uint4* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = philox4x32_10(ctr[i], k0, k1);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static bool is_chem(int kind) { return kind == PR_MODEL_CHEM || kind == PR_MODEL_CHEM_PRINTED; }

static bool model_ok(const pr_model* m)
{
    if (!m) return false;
    if (is_chem(m->kind)) {   // rates finite and non-negative, one fast variable
        if (m->fast_dim != 1 || !(m->eps > 0.0) || !(m->tau_x > 0.0)) return false;
        for (int i = 0; i < 6; ++i)
            if (!isfinite(m->rate[i]) || m->rate[i] < 0.0) return false;
        return true;
    }
    if (m->kind < PR_MODEL_OU || m->kind > PR_MODEL_DW_MULTI) return false;
    if (m->fast_dim < 1 || m->fast_dim > PR_MAX_FAST_DIM) return false;
    if (m->kind != PR_MODEL_DW_MULTI && m->fast_dim != 1) return false;
    if (!(m->beta > 0.0) || !(m->eps > 0.0) || !(m->tau_x > 0.0)) return false;
    if (!isfinite(m->lambda)) return false;
    return true;
}

// Elements per CTA for a streaming pass over n_slices x n elements: as many
// CTAs per slice as fit one wave (per_sm CTAs per SM) over all slices, at
// least min_per elements each, a multiple of 4 (whole vectors).
static int64_t stream_range(int64_t n, int n_slices, int64_t min_per, int per_sm)
{
    const int64_t slots = (int64_t)num_sms() * per_sm;
    int64_t bps = std::max<int64_t>(1, slots / n_slices);
    bps = std::min<int64_t>(bps, std::max<int64_t>(1, n / min_per));
    int64_t per = (n + bps - 1) / bps;
    return (per + 3) & ~(int64_t)3;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static int g_tiles_max = 8;   // upper bound of tiles per CTA (binary32 d = 1 kernel)

template <int KIND, int PPT>
static pr_status launch_f32_d1(const FineArgs& a, FineSmemOffsets so, int flags, size_t smem,
                               int n_slices, cudaStream_t st)
{
    const int threads = a.n >= 4096 ? 256 : 64;
    const int64_t per = (int64_t)threads * PPT;
    const int64_t tiles = (a.n + per - 1) / per;
    // Several consecutive tiles per CTA amortise the per-CTA prologue (edge
    // thresholds, matching table), while keeping >= ~16 waves of CTAs so the
    // last wave costs little.
    FineArgs b = a;
    const int64_t target_ctas = (int64_t)num_sms() * 6 * 16;
    int64_t tpc = (tiles * n_slices) / std::max<int64_t>(1, target_ctas);
    b.tiles_per_cta = (int)std::max<int64_t>(1, std::min<int64_t>(tpc, g_tiles_max));
    dim3 grid((unsigned)((tiles + b.tiles_per_cta - 1) / b.tiles_per_cta), (unsigned)n_slices);
    auto k = fine_f32_d1_kernel<KIND, PPT>;
    PR_TRY_CUDA(set_smem(k, smem));
    k<<<grid, threads, smem, st>>>(b, so, flags);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

template <int KIND, int D>
static pr_status launch_f32_dn(const FineArgs& a, FineSmemOffsets so, int flags, size_t smem,
                               int n_slices, cudaStream_t st)
{
    // 512 threads: the matching table (up to ~90 KB at 1024 bins) allows two
    // CTAs per SM, so larger CTAs keep more warps resident
    const int threads = a.n >= 16384 ? 512 : (a.n >= 4096 ? 256 : 64);
    dim3 grid((unsigned)((a.n + threads - 1) / threads), (unsigned)n_slices);
    auto k = fine_f32_dn_kernel<KIND, D>;
    PR_TRY_CUDA(set_smem(k, smem));
    k<<<grid, threads, smem, st>>>(a, so, flags);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

static pr_status launch_f32_multi(int D, const FineArgs& a, FineSmemOffsets so, int flags,
                                  size_t smem, int n_slices, cudaStream_t st)
{
    switch (D) {
#define PR_DN_CASE(d) \
    case d: return launch_f32_dn<PR_MODEL_DW_MULTI, d>(a, so, flags, smem, n_slices, st);
    PR_DN_CASE(1) PR_DN_CASE(2) PR_DN_CASE(3) PR_DN_CASE(4) PR_DN_CASE(5) PR_DN_CASE(6) PR_DN_CASE(7)
    PR_DN_CASE(8) PR_DN_CASE(9) PR_DN_CASE(10) PR_DN_CASE(11) PR_DN_CASE(12) PR_DN_CASE(13) PR_DN_CASE(14)
    PR_DN_CASE(15) PR_DN_CASE(16)
#undef PR_DN_CASE
    default: return PR_ERR_UNSUPPORTED;
    }
}

static int g_ppt = 0;   // particles per thread of the binary32 d = 1 kernel (0: per launch)

// Particles per thread of a binary32 d = 1 launch over n x n_slices
// particles: 4 unless the launch would then have fewer threads than the
// device holds resident (2048 per SM), then 2, else 1, so that a small
// launch still fills the SMs; a value forced by pr_set_particles_per_thread
// wins.
static int pick_ppt(int64_t n, int n_slices)
{
    if (g_ppt) return g_ppt;
    const int64_t resident = (int64_t)num_sms() * 2048;
    const int64_t total = n * (int64_t)n_slices;
    if (total / 4 >= resident) return 4;
    if (total / 2 >= resident) return 2;
    return 1;
}

}  // namespace pr

using namespace pr;

extern "C" void pr_set_particles_per_thread(int32_t ppt) { g_ppt = (ppt == 1 || ppt == 2 || ppt == 4) ? ppt : 0; }

extern "C" void pr_set_tiles_per_cta(int32_t tiles) { g_tiles_max = tiles < 1 ? 1 : (tiles > 64 ? 64 : tiles); }

// The wide binary32 matching of n_slices slices (see match_f32_wide_kernel).
static pr_status launch_match_f32_wide(const float* xp, float* xo, int64_t n, int64_t in_stride, int n_slices,
                                       const GridDev& g, const double* cp, const double* ct, cudaStream_t st)
{
    const size_t smem = match_smem_bytes(g.bins);
    if (smem > (size_t)smem_optin_max()) return PR_ERR_UNSUPPORTED;
    // one wave of as many CTAs per SM as their shared memory allows (at most 8)
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(228 * 1024) / (smem + 1024)));
    const int64_t per_block = stream_range(n, n_slices, 4096, per_sm);
    const int64_t blocks_per_slice = (n + per_block - 1) / per_block;
    PR_TRY_CUDA(set_smem(match_f32_wide_kernel, smem));
    match_f32_wide_kernel<<<dim3((unsigned)blocks_per_slice, (unsigned)n_slices), 256, smem, st>>>(
        xp, xo, n, in_stride, g, cp, ct, per_block);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" pr_status pr_fine_propagate(const pr_model* model, pr_precision precision, const pr_rng* rng,
                                       const void* x_in, const void* y_in, int32_t broadcast_input,
                                       void* x_out, void* y_out, int64_t n, int32_t slice_begin,
                                       int32_t n_slices, int32_t steps, double dt, const pr_grid* grid,
                                       const double* cdf_prior, const double* cdf_target,
                                       uint32_t* counts_start, double* cdf_start,
                                       uint32_t* counts_end, double* cdf_end, void* stream)
{
    if (!model_ok(model) || !rng) return PR_ERR_INVALID_ARG;
    {
        const size_t es = elem_bytes(precision);
        if (!elem_aligned(x_in, es) || !elem_aligned(y_in, es) || !elem_aligned(x_out, es) ||
            !elem_aligned(y_out, es) || !elem_aligned(cdf_prior, 8) || !elem_aligned(cdf_target, 8) ||
            !elem_aligned(counts_start, 4) || !elem_aligned(cdf_start, 8) || !elem_aligned(counts_end, 4) ||
            !elem_aligned(cdf_end, 8))
            return PR_ERR_INVALID_ARG;
    }
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
    if (!x_in || !y_in || !x_out || !y_out) return PR_ERR_INVALID_ARG;
    if (n < 1 || n > 0xFFFFFFFFll || n_slices < 1 || n_slices > 65535 || slice_begin < 0) return PR_ERR_INVALID_ARG;
    if (steps < 0 || !(dt > 0.0) || !isfinite(dt)) return PR_ERR_INVALID_ARG;
    if (rng->problem_id >= (1u << 24)) return PR_ERR_INVALID_ARG;
    if ((cdf_prior == nullptr) != (cdf_target == nullptr)) return PR_ERR_INVALID_ARG;
    if (cdf_start && !counts_start) return PR_ERR_INVALID_ARG;
    if (cdf_end && !counts_end) return PR_ERR_INVALID_ARG;
    const bool do_match = cdf_prior != nullptr;
    const bool any_grid = do_match || counts_start || counts_end;
    if (any_grid && !grid_ok(grid)) return PR_ERR_INVALID_ARG;
    const int D = model->fast_dim;
    const size_t esz = precision == PR_F32 ? 4 : 8;
    // in-place is allowed only as exact aliasing of whole arrays, and not
    // from a broadcast input (every slice reads the one input ensemble)
    if (x_in == x_out && (broadcast_input || y_in != y_out)) return PR_ERR_INVALID_ARG;
    if (broadcast_input && y_in == y_out) return PR_ERR_INVALID_ARG;
    (void)esz;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    FineArgs a{};
    a.x_in = x_in;
    a.y_in = y_in;
    a.x_out = x_out;
    a.y_out = y_out;
    a.n = n;
    a.in_slice_stride = broadcast_input ? 0 : n;
    a.slice_begin = slice_begin;
    a.steps = steps;
    a.fast_dim = D;
    a.lam = model->lambda;
    a.drift_dt = dt / model->tau_x;
    a.relax = dt / model->eps;
    a.sx = sqrt(2.0 * (1.0 / model->beta) / model->tau_x) * sqrt(dt);
    a.sy = sqrt(2.0 * 1.0 / model->eps) * sqrt(dt);
    a.lam_f = (float)a.lam;
    a.drift_dt_f = (float)a.drift_dt;
    a.relax_f = (float)a.relax;
    a.sx_f = (float)a.sx;
    a.sy_f = (float)a.sy;
    a.sxk_f = (float)(a.sx * 1.1774100225154746910);
    a.syk_f = (float)(a.sy * 1.1774100225154746910);
    if (is_chem(model->kind)) {
        // state-dependent amplitudes: dt is folded into the variance
        // polynomials, so the binary64 normals enter unscaled and the
        // binary32 ones scaled by sqrt(2 ln 2) alone
        const bool printed = model->kind == PR_MODEL_CHEM_PRINTED;
        a.chem_d = make_chem_consts<double>(model->rate, printed, dt, model->tau_x, model->eps);
        a.chem_f = make_chem_consts<float>(model->rate, printed, dt, model->tau_x, model->eps);
        a.sx = a.sy = 1.0;
        a.sxk_f = a.syk_f = 1.1774100225154746910f;
    }
    a.tiles_per_cta = 1;
    a.k0 = (uint32_t)(rng->seed & 0xFFFFFFFFull);
    a.k1 = (uint32_t)(rng->seed >> 32);
    a.ctr_hi = rng->problem_id << 8;
    if (any_grid) {
        a.g = make_grid(*grid);
        a.lo_f = (float)grid->x_lo;
        a.inv_h_f = (float)(1.0 / a.g.h);
    } else {
        a.g = GridDev{1, 0.0, 1.0, 1.0};
    }
    a.cdf_prior = cdf_prior;
    a.cdf_target = cdf_target;
    a.counts_start = counts_start;
    a.counts_end = counts_end;
    const int bins = any_grid ? grid->bins : 1;
    if (counts_start) PR_TRY_CUDA(cudaMemsetAsync(counts_start, 0, (size_t)n_slices * bins * 4, st));
    if (counts_end) PR_TRY_CUDA(cudaMemsetAsync(counts_end, 0, (size_t)n_slices * bins * 4, st));

    const FineSmem L = fine_smem_layout(bins, any_grid, do_match, precision == PR_F32);
    if (L.total > (size_t)smem_optin_max()) {
        if (precision != PR_F32 || !do_match) return PR_ERR_UNSUPPORTED;
        // Binary32 on a grid whose matching table does not fit beside the
        // histograms: the same steps in turn.  The start states are matched
        // into x_out by the wide matching, restricted there, and propagated
        // in place (y brought to y_out first).
        const size_t ybytes = (size_t)D * n * sizeof(float);
        if (y_in != y_out) {
            if (broadcast_input) {
                const int64_t per = (int64_t)D * n;
                const int blocks = (int)std::min<int64_t>((per * n_slices + 255) / 256, 8 * (int64_t)num_sms());
                broadcast_slices_kernel<<<blocks, 256, 0, st>>>(static_cast<const float*>(y_in),
                                                                static_cast<float*>(y_out), per, n_slices);
                PR_CHECK_LAUNCH();
            } else {
                PR_TRY_CUDA(cudaMemcpyAsync(y_out, y_in, ybytes * n_slices, cudaMemcpyDeviceToDevice, st));
            }
        }
        const pr_status m = launch_match_f32_wide(static_cast<const float*>(x_in), static_cast<float*>(x_out), n,
                                                  broadcast_input ? 0 : n, n_slices, a.g, cdf_prior, cdf_target, st);
        if (m != PR_OK) return m;
        if (counts_start) {
            const pr_status r = pr_restrict(PR_F32, x_out, n, n_slices, grid, counts_start, cdf_start, stream);
            if (r != PR_OK) return r;
        }
        return pr_fine_propagate(model, precision, rng, x_out, y_out, 0, x_out, y_out, n, slice_begin, n_slices,
                                 steps, dt, grid, nullptr, nullptr, nullptr, nullptr, counts_end, cdf_end, stream);
    }
    FineSmemOffsets so{(unsigned)L.thr, (unsigned)L.hs, (unsigned)L.he, (unsigned)L.match};
    const int flags = (any_grid ? 1 : 0) | (do_match ? 2 : 0) | (counts_start ? 4 : 0) | (counts_end ? 8 : 0);
    pr_status rc = PR_OK;
    if (precision == PR_F32) {
        if (model->kind == PR_MODEL_DW_MULTI && D > 1) {
            rc = launch_f32_multi(D, a, so, flags, L.total, n_slices, st);
        } else if (is_chem(model->kind)) {
            switch (pick_ppt(n, n_slices)) {
            case 2: rc = launch_f32_d1<PR_MODEL_CHEM, 2>(a, so, flags, L.total, n_slices, st); break;
            case 4: rc = launch_f32_d1<PR_MODEL_CHEM, 4>(a, so, flags, L.total, n_slices, st); break;
            default: rc = launch_f32_d1<PR_MODEL_CHEM, 1>(a, so, flags, L.total, n_slices, st);
            }
        } else {
            // (the multi-component family with one component is the double well)
            const bool ou = model->kind == PR_MODEL_OU;
            switch (pick_ppt(n, n_slices)) {
            case 2:
                rc = ou ? launch_f32_d1<PR_MODEL_OU, 2>(a, so, flags, L.total, n_slices, st)
                        : launch_f32_d1<PR_MODEL_DOUBLE_WELL, 2>(a, so, flags, L.total, n_slices, st);
                break;
            case 4:
                rc = ou ? launch_f32_d1<PR_MODEL_OU, 4>(a, so, flags, L.total, n_slices, st)
                        : launch_f32_d1<PR_MODEL_DOUBLE_WELL, 4>(a, so, flags, L.total, n_slices, st);
                break;
            default:
                rc = ou ? launch_f32_d1<PR_MODEL_OU, 1>(a, so, flags, L.total, n_slices, st)
                        : launch_f32_d1<PR_MODEL_DOUBLE_WELL, 1>(a, so, flags, L.total, n_slices, st);
            }
        }
    } else {
        const int threads = 128;
        dim3 g((unsigned)((n + threads - 1) / threads), (unsigned)n_slices);
        switch (model->kind) {
        case PR_MODEL_OU: {
            auto k = fine_f64_kernel<PR_MODEL_OU>;
            PR_TRY_CUDA(set_smem(k, L.total));
            k<<<g, threads, L.total, st>>>(a, so, flags);
            break;
        }
        case PR_MODEL_DOUBLE_WELL: {
            auto k = fine_f64_kernel<PR_MODEL_DOUBLE_WELL>;
            PR_TRY_CUDA(set_smem(k, L.total));
            k<<<g, threads, L.total, st>>>(a, so, flags);
            break;
        }
        case PR_MODEL_CHEM:
        case PR_MODEL_CHEM_PRINTED: {
            auto k = fine_f64_kernel<PR_MODEL_CHEM>;
            PR_TRY_CUDA(set_smem(k, L.total));
            k<<<g, threads, L.total, st>>>(a, so, flags);
            break;
        }
        default: {
            auto k = fine_f64_kernel<PR_MODEL_DW_MULTI>;
            PR_TRY_CUDA(set_smem(k, L.total));
            k<<<g, threads, L.total, st>>>(a, so, flags);
        }
        }
        PR_CHECK_LAUNCH();
    }
    if (rc != PR_OK) return rc;
    if (cdf_start) {
        counts_to_cdf_kernel<<<n_slices, 256, 0, st>>>(counts_start, n, bins, cdf_start);
        PR_CHECK_LAUNCH();
    }
    if (cdf_end) {
        counts_to_cdf_kernel<<<n_slices, 256, 0, st>>>(counts_end, n, bins, cdf_end);
        PR_CHECK_LAUNCH();
    }
    return PR_OK;
}

extern "C" pr_status pr_rng_words(const pr_rng* rng, const uint32_t* ctr, int64_t n, uint32_t* out, void* stream)
{
    if (!rng || !ctr || !out || n < 1) return PR_ERR_INVALID_ARG;
    if (((uintptr_t)ctr & 15) || ((uintptr_t)out & 15)) return PR_ERR_INVALID_ARG;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4 * (int64_t)num_sms());
    rng_words_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4*>(ctr), n, (uint32_t)(rng->seed & 0xFFFFFFFFull), (uint32_t)(rng->seed >> 32),
        reinterpret_cast<uint4*>(out));
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" pr_status pr_counts_to_cdf(const uint32_t* counts, int64_t n, int32_t n_slices, int32_t bins,
                                      double* cdf, void* stream)
{
    if (!counts || !cdf || n < 1 || n_slices < 1 || bins < 1 || bins > PR_MAX_BINS) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(counts, 4) || !elem_aligned(cdf, 8)) return PR_ERR_INVALID_ARG;
    counts_to_cdf_kernel<<<n_slices, 256, 0, static_cast<cudaStream_t>(stream)>>>(counts, n, bins, cdf);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" pr_status pr_restrict(pr_precision precision, const void* x, int64_t n, int32_t n_slices,
                                 const pr_grid* grid, uint32_t* counts, double* cdf, void* stream)
{
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(x, elem_bytes(precision)) || !elem_aligned(counts, 4) || !elem_aligned(cdf, 8))
        return PR_ERR_INVALID_ARG;
    if (!x || !counts || n < 1 || n_slices < 1 || n_slices > 65535 || !grid_ok(grid)) return PR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int bins = grid->bins;
    PR_TRY_CUDA(cudaMemsetAsync(counts, 0, (size_t)n_slices * bins * 4, st));
    const GridDev g = make_grid(*grid);
    const float lo_f = (float)grid->x_lo, inv_h_f = (float)(1.0 / g.h);
    // one wave of 512-thread CTAs (4 per SM), each a contiguous range of one slice
    const int64_t per_block = stream_range(n, n_slices, 4096, 4);
    const int64_t blocks_per_slice = (n + per_block - 1) / per_block;
    const size_t smem = align16((size_t)bins * 4 + (size_t)(bins + 1) * 4);
    dim3 gr((unsigned)blocks_per_slice, (unsigned)n_slices);
    if (precision == PR_F32) {
        restrict_kernel<float><<<gr, 512, smem, st>>>(static_cast<const float*>(x), n, g, lo_f, inv_h_f, counts, per_block);
    } else {
        restrict_kernel<double><<<gr, 512, smem, st>>>(static_cast<const double*>(x), n, g, lo_f, inv_h_f, counts, per_block);
    }
    PR_CHECK_LAUNCH();
    if (cdf) {
        counts_to_cdf_kernel<<<n_slices, 256, 0, st>>>(counts, n, bins, cdf);
        PR_CHECK_LAUNCH();
    }
    return PR_OK;
}

extern "C" pr_status pr_match(pr_precision precision, const void* x_prior, void* x_out, int64_t n,
                              int32_t n_slices, const pr_grid* grid, const double* cdf_prior,
                              const double* cdf_target, void* stream)
{
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(x_prior, elem_bytes(precision)) || !elem_aligned(x_out, elem_bytes(precision)) ||
        !elem_aligned(cdf_prior, 8) || !elem_aligned(cdf_target, 8))
        return PR_ERR_INVALID_ARG;
    if (!x_prior || !x_out || !cdf_prior || !cdf_target) return PR_ERR_INVALID_ARG;
    if (n < 1 || n_slices < 1 || n_slices > 65535 || !grid_ok(grid)) return PR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int bins = grid->bins;
    const GridDev g = make_grid(*grid);
    // two 1024-thread CTAs per SM, each building its table once (a few
    // microseconds of FP64 work) and streaming its share of the particles
    const int64_t per_block = stream_range(n, n_slices, 16384, 2);
    const int64_t blocks_per_slice = (n + per_block - 1) / per_block;
    dim3 gr((unsigned)blocks_per_slice, (unsigned)n_slices);
    // the per-CTA binary32 table must fit in shared memory; beyond, the wide
    // matching (binary64 map per particle, rounded to binary32)
    const size_t smem = precision == PR_F32 ? align16((size_t)(bins + 1) * 4) + match_smem_bytes_f32(bins)
                                            : match_smem_bytes(bins);
    if (precision == PR_F32 && smem > (size_t)smem_optin_max())
        return launch_match_f32_wide(static_cast<const float*>(x_prior), static_cast<float*>(x_out), n, n, n_slices,
                                     g, cdf_prior, cdf_target, st);
    if (smem > (size_t)smem_optin_max()) return PR_ERR_UNSUPPORTED;
    if (precision == PR_F32) {
        PR_TRY_CUDA(set_smem(match_f32_kernel, smem));
        match_f32_kernel<<<gr, 1024, smem, st>>>(static_cast<const float*>(x_prior), static_cast<float*>(x_out), n, g,
                                                (float)grid->x_lo, (float)(1.0 / g.h), cdf_prior, cdf_target, per_block);
    } else {
        PR_TRY_CUDA(set_smem(match_f64_kernel, smem));
        match_f64_kernel<<<gr, 256, smem, st>>>(static_cast<const double*>(x_prior), static_cast<double*>(x_out), n, g,
                                                cdf_prior, cdf_target, per_block);
    }
    PR_CHECK_LAUNCH();
    return PR_OK;
}

// match.cuh -- quantile-transport matching (Section 5.1, Eq. transformation)
// as device code shared by the standalone matching kernel and the prologue of
// the fine propagator.
//
// The map X = c^{-1}(cbar(Xbar)) composes two piecewise-linear CDFs, so on
// each prior bin i it is piecewise affine in the bin fraction
// f = (Xbar - e_i)/h, with one piece per non-empty target bin j that the
// prior level interval [Cbar_i, Cbar_{i+1}] reaches:
//     X = e_j + (Cbar_i - C_j) h/rho_j + f rhobar_i h/rho_j.
// The binary32 path builds that table of pieces once per CTA (FP64 where CDF
// values are subtracted, then rounded) and maps every particle with binary32
// arithmetic only: the FP64 units of GB300 run at a small fraction of the
// FP32 rate, and per-particle FP64 would make this memory-bound pass
// compute-bound.  The binary64 path evaluates the map per particle in FP64.
#pragma once

#include "pr_common.cuh"

namespace pr {

// Shared-memory layout of the binary32 table (bins = I):
//   Cp, Ct      : double [I+1]     prior / target CDF
//   nzpre       : int    [I+1]     number of non-empty target bins below j
//   nzlist      : int    [I]       non-empty target bins in order
//   jfirst      : int    [I]       first piece's target bin of prior bin i
//   pstart      : int    [I+1]     first piece of prior bin i (pstart[i] == pstart[i+1]: identity)
//   fend, alpha, beta : float [2I+1]
//   jp          : int    [2I+1]    target bin of each piece (the result is clamped into it)
struct MatchSmem {
    double* Cp;
    double* Ct;
    int* nzpre;
    int* nzlist;
    int* jfirst;
    int* pstart;
    float* fend;
    float* alpha;
    float* beta;
    int* jp;
    int* scratch;   // [blockDim.x / 32 + 1] for scans
};

__host__ __device__ inline size_t match_smem_bytes(int bins)
{
    const size_t I = (size_t)bins;
    size_t b = 2 * (I + 1) * sizeof(double);
    b += (I + 1 + I + I + I + 1) * sizeof(int);
    b += 3 * (2 * I + 1) * sizeof(float);
    b += (2 * I + 1) * sizeof(int);
    b += 64 * sizeof(int);
    return (b + 15) & ~(size_t)15;
}

__device__ inline MatchSmem carve_match_smem(unsigned char* base, int bins)
{
    const int I = bins;
    MatchSmem m;
    m.Cp = reinterpret_cast<double*>(base);
    m.Ct = m.Cp + (I + 1);
    int* ip = reinterpret_cast<int*>(m.Ct + (I + 1));
    m.nzpre = ip;
    m.nzlist = m.nzpre + (I + 1);
    m.jfirst = m.nzlist + I;
    m.pstart = m.jfirst + I;
    float* fp = reinterpret_cast<float*>(m.pstart + (I + 1));
    m.fend = fp;
    m.alpha = m.fend + (2 * I + 1);
    m.beta = m.alpha + (2 * I + 1);
    m.jp = reinterpret_cast<int*>(m.beta + (2 * I + 1));
    m.scratch = m.jp + (2 * I + 1);
    return m;
}

// Block-wide exclusive scan of v[0..n) (ints) into out[0..n], out[n] = total.
// Deterministic; every thread of the block must call it; v may equal out.
__device__ inline void block_exclusive_scan_int(const int* v, int* out, int n, int* scratch)
{
    const int T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int b = threadIdx.x * chunk;
    const int e = min(n, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += v[i];
    // warp inclusive scan of per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = T >> 5;
        int w = lane < nw ? scratch[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) scratch[lane] = wi - w;   // exclusive warp offsets
        if (lane == nw - 1) scratch[32] = wi;    // total
    }
    __syncthreads();
    int run = scratch[warp] + incl - s;
    for (int i = b; i < e; ++i) {
        const int vi = v[i];
        out[i] = run;
        run += vi;
    }
    if (threadIdx.x == 0) out[n] = scratch[32];
    __syncthreads();
}

// Lowest j with Ct[j+1] >= u among all bins (u <= Ct[I] assumed; else I-1).
__device__ __forceinline__ int lowest_reaching(const double* Ct, int I, double u)
{
    const long long ku = dkey(u);
    int lo = 0, hi = I - 1;   // answer in [lo, hi]
    if (dkey(Ct[I]) < ku) return I - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (dkey(Ct[mid + 1]) >= ku) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Lowest non-empty target bin with Ct[j+1] >= u, else the last non-empty one.
__device__ __forceinline__ int target_bin(const double* Ct, const int* nzpre, const int* nzlist,
                                          int I, double u)
{
    const int nnz = nzpre[I];
    const int j = lowest_reaching(Ct, I, u);
    const int r = nzpre[j];   // non-empty bins below j; the r-th is the first at or after j
    return r < nnz ? nzlist[r] : nzlist[nnz - 1];
}

// Build the binary32 table for one slice.  All threads of the block call it.
__device__ inline void build_match_table(const GridDev& g, const double* __restrict__ cp_g,
                                         const double* __restrict__ ct_g, MatchSmem& m)
{
    const int I = g.bins;
    for (int i = threadIdx.x; i <= I; i += blockDim.x) {
        m.Cp[i] = cp_g[i];
        m.Ct[i] = ct_g[i];
    }
    __syncthreads();
    // non-empty target bins (jfirst used as a temporary flag array)
    for (int j = threadIdx.x; j < I; j += blockDim.x)
        m.jfirst[j] = dkey(m.Ct[j + 1]) > dkey(m.Ct[j]) ? 1 : 0;
    __syncthreads();
    block_exclusive_scan_int(m.jfirst, m.nzpre, I, m.scratch);
    for (int j = threadIdx.x; j < I; j += blockDim.x)
        if (m.jfirst[j]) m.nzlist[m.nzpre[j]] = j;
    __syncthreads();
    const int nnz = m.nzpre[I];
    // pieces per prior bin (pstart used as the count array)
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        int cnt = 0;
        const bool ident = (m.Cp[i] == m.Ct[i]) && (m.Cp[i + 1] == m.Ct[i + 1]);
        if (!ident && nnz > 0) {
            const int j0 = target_bin(m.Ct, m.nzpre, m.nzlist, I, m.Cp[i]);
            const int j1 = target_bin(m.Ct, m.nzpre, m.nzlist, I, m.Cp[i + 1]);
            m.jfirst[i] = m.nzpre[j0];
            cnt = max(1, m.nzpre[j1] - m.nzpre[j0] + 1);
        } else {
            m.jfirst[i] = 0;
        }
        m.pstart[i] = cnt;
    }
    __syncthreads();
    // in place: each thread reads an element of its own chunk before writing it
    block_exclusive_scan_int(m.pstart, m.pstart, I, m.scratch);
    // Monotone CDFs give at most 2I - 1 pieces.  A prior that is not a CDF
    // could ask for more than the table holds: map nothing (identity) then.
    if (m.pstart[I] > 2 * I + 1) {
        __syncthreads();
        for (int i = threadIdx.x; i <= I; i += blockDim.x) m.pstart[i] = 0;
        __syncthreads();
    }
    const int npieces = m.pstart[I];
    const double h = g.h;
    // one thread per piece: its prior bin by binary search over pstart
    for (int k = threadIdx.x; k < npieces; k += blockDim.x) {
        int lo = 0, hi = I - 1;
        while (lo < hi) {   // last i with pstart[i] <= k
            const int mid = (lo + hi + 1) >> 1;
            if (m.pstart[mid] <= k) lo = mid; else hi = mid - 1;
        }
        const int i = lo;
        const int r = m.jfirst[i] + (k - m.pstart[i]);
        const int j = m.nzlist[min(r, nnz - 1)];
        const double rho_bar = __dsub_rn(m.Cp[i + 1], m.Cp[i]);
        const double rho_j = __dsub_rn(m.Ct[j + 1], m.Ct[j]);
        const double hr = __ddiv_rn(h, rho_j);
        const double a = __dadd_rn(edge(g, j), __dmul_rn(__dsub_rn(m.Cp[i], m.Ct[j]), hr));
        const double b = __dmul_rn(rho_bar, hr);
        float fe = 2.0f;
        if (k + 1 < m.pstart[i + 1] && rho_bar > 0.0)
            fe = (float)__ddiv_rn(__dsub_rn(m.Ct[j + 1], m.Cp[i]), rho_bar);
        m.fend[k] = fe;
        // a target bin of negligible mass makes the slope huge; saturate so
        // that the clamp into the bin below never sees inf - inf
        m.alpha[k] = (float)fmax(fmin(a, 1e30), -1e30);
        m.beta[k] = (float)fmin(b, 1e30);
        m.jp[k] = j;
    }
    __syncthreads();
}

// Map one binary32 particle through the table.
__device__ __forceinline__ float match_one_f32(const MatchSmem& m, const float* __restrict__ thr,
                                               int bins, float lo_f, float inv_h_f, float x)
{
    const int i = bin_of_f32(thr, bins, lo_f, inv_h_f, x);
    const int k0 = m.pstart[i], k1 = m.pstart[i + 1];
    if (k0 == k1) return x;   // identity on this bin
    const bool below = !(x >= thr[0]);
    const bool above = x >= thr[bins];
    float f = (x - thr[i]) * inv_h_f;
    f = fminf(fmaxf(f, 0.0f), 1.0f);
    if (below) f = 0.0f;
    if (above) f = 1.0f;
    int k = k0;
    while (k < k1 - 1 && f > m.fend[k]) ++k;
    const int j = m.jp[k];
    const float xn = fminf(fmaxf(fmaf(m.beta[k], f, m.alpha[k]), thr[j]), thr[j + 1]);
    if (below) return x + (xn - thr[0]);
    if (above) return x + (xn - thr[bins]);
    return xn;
}

// Binary64: the map evaluated per particle, in the same operations as the
// CPU reference (each rounded on its own).  Needs Cp, Ct, nzpre, nzlist of
// the table (the binary32 pieces are not used).
__device__ inline void build_match_index(const GridDev& g, const double* __restrict__ cp_g,
                                         const double* __restrict__ ct_g, MatchSmem& m)
{
    const int I = g.bins;
    for (int i = threadIdx.x; i <= I; i += blockDim.x) {
        m.Cp[i] = cp_g[i];
        m.Ct[i] = ct_g[i];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < I; j += blockDim.x)
        m.jfirst[j] = dkey(m.Ct[j + 1]) > dkey(m.Ct[j]) ? 1 : 0;
    __syncthreads();
    block_exclusive_scan_int(m.jfirst, m.nzpre, I, m.scratch);
    for (int j = threadIdx.x; j < I; j += blockDim.x)
        if (m.jfirst[j]) m.nzlist[m.nzpre[j]] = j;
    __syncthreads();
}

__device__ inline double match_one_f64(const MatchSmem& m, const GridDev& g, double x)
{
    const int I = g.bins;
    const int i = bin_of_f64(g, x);
    if (m.Cp[i] == m.Ct[i] && m.Cp[i + 1] == m.Ct[i + 1]) return x;
    if (m.nzpre[I] == 0) return x;
    const double ei = edge(g, i);
    double frac = __ddiv_rn(__dsub_rn(x, ei), g.h);
    bool below = false, above = false;
    if (frac < 0.0) { frac = 0.0; below = true; }
    if (frac > 1.0) { frac = 1.0; above = true; }
    const double rho_prior = __dsub_rn(m.Cp[i + 1], m.Cp[i]);
    const double u = __dadd_rn(m.Cp[i], __dmul_rn(frac, rho_prior));
    const int j = target_bin(m.Ct, m.nzpre, m.nzlist, I, u);
    const double rho_j = __dsub_rn(m.Ct[j + 1], m.Ct[j]);
    double t = __ddiv_rn(__dsub_rn(u, m.Ct[j]), rho_j);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    const double xn = __dadd_rn(edge(g, j), __dmul_rn(t, g.h));
    if (below) return __dadd_rn(x, __dsub_rn(xn, g.lo));
    if (above) return __dadd_rn(x, __dsub_rn(xn, g.hi));
    return xn;
}

}  // namespace pr

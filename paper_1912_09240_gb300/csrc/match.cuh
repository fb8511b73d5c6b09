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

// Shared-memory layout (bins = I).  The table, live while particles are mapped:
//   rec    : float4 [I]     one record per prior bin i.  Where the bin's map
//            has one piece, or two pieces whose target bins j, j+1 meet at
//            the edge e_{j+1}, the record is (m, fs, b1, b2): the map is
//            X = m + b (f - fs), b = b1 for f < fs and b2 beyond, with
//            m = thr[j+1] (two pieces: they meet there at fs; one piece: the
//            line of the piece reaches it at fs >= 1), the particle's target
//            bin jm - 1 below fs and jm from fs on (jm the index of the edge
//            m), so that such a particle reads one 16-byte record; b2 is
//            stored negated where an image could leave those bins by
//            rounding (the general path then checks it).  Otherwise b1 = -2
//            (identity) or -1 and m holds the bits of start | end << 16: the
//            pieces [start, end) of the bin in the arrays below (at most
//            2I+1 <= 8193 pieces).
//   piece  : float4 [2I+1]  (alpha, beta, thr[j], thr[j+1]) of target bin j:
//            on prior bin i the map is X = clamp(alpha + beta f, thr[j], thr[j+1])
//            for the first piece of the bin whose f_end >= f (or its last piece)
//   fend   : float  [2I+1]  f_end of each piece
// Build scratch, dead once the table is built:
//   Cp, Ct : double [I+1]   prior / target CDF
//   nzpre  : int    [I+1]   number of non-empty target bins below j
//   nzlist : int    [I]     non-empty target bins in order
//   jfirst : int    [I]     first piece's target bin of prior bin i
//   pstart : int    [I+1]   first piece of prior bin i
// The binary64 path (carve_match_smem) has no table: it keeps Cp, Ct, nzpre
// and nzlist and maps every particle from them.
struct MatchSmem {
    float4* rec;
    float4* piece;
    float* fend;
    double* Cp;
    double* Ct;
    int* nzpre;
    int* nzlist;
    int* jfirst;
    int* pstart;
    int* scratch;   // [blockDim.x / 32 + 1] for scans
};

__host__ __device__ inline size_t match_table_bytes(int bins)
{
    const size_t I = (size_t)bins;
    return ((I * 16 + (2 * I + 1) * 16 + (2 * I + 1) * 4) + 15) & ~(size_t)15;
}

__host__ __device__ inline size_t match_build_bytes(int bins)
{
    const size_t I = (size_t)bins;
    size_t b = 2 * (I + 1) * sizeof(double);
    b += (I + 1 + I + I + I + 1) * sizeof(int);
    b += 64 * sizeof(int);
    return (b + 15) & ~(size_t)15;
}

// The binary64 path maps every particle from the CDFs and their index arrays
// (no binary32 pieces), so its shared memory is the build scratch alone.
__host__ __device__ inline size_t match_smem_bytes(int bins) { return match_build_bytes(bins); }

// The binary32 table reads the CDFs from global memory while it is built, so
// its scratch holds only the integer arrays (nzpre, nzlist, jfirst, pstart,
// scan scratch); callers may reuse that scratch once the table is built.
__host__ __device__ inline size_t match_build_bytes_f32(int bins)
{
    const size_t I = (size_t)bins;
    return ((I + 1 + I + I + I + 1 + 64) * sizeof(int) + 15) & ~(size_t)15;
}

__host__ __device__ inline size_t match_smem_bytes_f32(int bins)
{
    return match_table_bytes(bins) + match_build_bytes_f32(bins);
}

// `base` 16-byte aligned; the build scratch starts match_table_bytes(bins) after it.
// Binary32 layout: the table, then the integer scratch; Cp and Ct point to
// the CDFs in global memory.
__device__ inline MatchSmem carve_match_smem_f32(unsigned char* base, int bins, const double* cp_g, const double* ct_g)
{
    const int I = bins;
    MatchSmem m;
    m.rec = reinterpret_cast<float4*>(base);
    m.piece = m.rec + I;
    m.fend = reinterpret_cast<float*>(m.piece + (2 * I + 1));
    m.Cp = const_cast<double*>(cp_g);
    m.Ct = const_cast<double*>(ct_g);
    int* ip = reinterpret_cast<int*>(base + match_table_bytes(bins));
    m.nzpre = ip;
    m.nzlist = m.nzpre + (I + 1);
    m.jfirst = m.nzlist + I;
    m.pstart = m.jfirst + I;
    m.scratch = m.pstart + (I + 1);
    return m;
}

__device__ inline MatchSmem carve_match_smem(unsigned char* base, int bins)
{
    const int I = bins;
    MatchSmem m;
    m.rec = nullptr;
    m.piece = nullptr;
    m.fend = nullptr;
    m.Cp = reinterpret_cast<double*>(base);
    m.Ct = m.Cp + (I + 1);
    int* ip = reinterpret_cast<int*>(m.Ct + (I + 1));
    m.nzpre = ip;
    m.nzlist = m.nzpre + (I + 1);
    m.jfirst = m.nzlist + I;
    m.pstart = m.jfirst + I;
    m.scratch = m.pstart + (I + 1);
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
// thr[] (the binary32 thresholds of the grid) must be written by the block
// before the call; it is read after the first barrier inside.
// m from carve_match_smem_f32: the CDFs are read where they are (global
// memory, through the read-only cache).
__device__ inline void build_match_table(const GridDev& g, const float* thr, MatchSmem& m)
{
    const int I = g.bins;
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
        const bool ident = deq(m.Cp[i], m.Ct[i]) && deq(m.Cp[i + 1], m.Ct[i + 1]);
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
    const float h_f = (float)g.h;
    // one thread per piece: its prior bin by binary search over pstart.  CDF
    // values are subtracted in FP64 (they cancel); the quotients, which end
    // up rounded to binary32 anyway, are taken in binary32, and the target
    // bin's left edge is its binary32 threshold, so the table costs four FP64
    // subtractions per piece and no FP64 division.
    for (int k = threadIdx.x; k < npieces; k += blockDim.x) {
        int lo = 0, hi = I - 1;
        while (lo < hi) {   // last i with pstart[i] <= k
            const int mid = (lo + hi + 1) >> 1;
            if (m.pstart[mid] <= k) lo = mid; else hi = mid - 1;
        }
        const int i = lo;
        const int r = m.jfirst[i] + (k - m.pstart[i]);
        const int j = m.nzlist[min(r, nnz - 1)];
        const double dij = __dsub_rn(m.Cp[i], m.Ct[j]);
        const float rbf = (float)__dsub_rn(m.Cp[i + 1], m.Cp[i]);
        const float rho_j = fmaxf((float)__dsub_rn(m.Ct[j + 1], m.Ct[j]), 1e-30f);
        const float hr = __fdiv_rn(h_f, rho_j);
        const float a = __fadd_rn(thr[j], __fmul_rn((float)dij, hr));
        const float b = __fmul_rn(rbf, hr);
        float fe = 2.0f;
        if (k + 1 < m.pstart[i + 1] && rbf > 0.0f)
            fe = __fdiv_rn((float)__dsub_rn(m.Ct[j + 1], m.Cp[i]), rbf);
        // a target bin of negligible mass makes the slope huge; saturate so
        // that the clamp into the bin below never sees inf - inf
        m.piece[k] = make_float4(fmaxf(fminf(a, 1e30f), -1e30f), fminf(b, 1e30f), thr[j], thr[j + 1]);
        m.fend[k] = fe;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const int k0 = m.pstart[i], k1 = m.pstart[i + 1];
        // general (-1) or identity (-2) unless one of the anchored forms applies
        float4 r = make_float4(__uint_as_float((uint32_t)k0 | ((uint32_t)k1 << 16)), 0.0f,
                               k0 == k1 ? -2.0f : -1.0f, 0.0f);
        float lo_j = 0.0f, hi_j = 0.0f;   // outer thresholds of the record's target bins
        if (k1 == k0 + 1) {
            // one piece X = alpha + beta f on [thr_j, thr_{j+1}]: anchored at
            // the right edge, reached at fs = (thr_{j+1} - alpha) / beta
            const float4 pc = m.piece[k0];
            if (pc.y > 0.0f && pc.y < 1e30f) {
                const float fs = (float)(((double)pc.w - (double)pc.x) / (double)pc.y);
                if (fs >= 1.0f && fs < 1e30f) {
                    r = make_float4(pc.w, fs, pc.y, pc.y);
                    lo_j = pc.z;
                    hi_j = pc.w;
                }
            }
        } else if (k1 == k0 + 2) {
            // two pieces meeting at the edge thr_{j+1} = hi of the first = lo of the second
            const float4 p1 = m.piece[k0], p2 = m.piece[k0 + 1];
            if (p1.w == p2.z && p1.y > 0.0f && p2.y > 0.0f && p1.y < 1e30f && p2.y < 1e30f) {
                r = make_float4(p1.w, m.fend[k0], p1.y, p2.y);
                lo_j = p1.z;
                hi_j = p2.w;
            }
        }
        if (r.z >= 0.0f) {
            // Safe when every image the fast path can compute lies in its
            // target bins: the fast path's f lies in [0, 1] and its image
            // fmaf(b, f - fs, m) is monotone in f, so the images at f = 0
            // and f = 1, taken with the same operations, bound them all.
            const float x0 = fmaf(r.z, 0.0f - r.y, r.x);
            const float x1 = fmaf(1.0f >= r.y ? r.w : r.z, 1.0f - r.y, r.x);
            if (!(x0 >= lo_j && x1 <= hi_j)) r.w = -r.w;   // unsafe: the general path checks
        }
        m.rec[i] = r;
    }
    __syncthreads();
}

// Map one binary32 particle through the table.
// General path: any particle, any bin.  The bin fraction f = (x - e_i)/h
// takes the left edge as lo + i h in binary32 (one fma, within half an ulp
// of x's magnitude of the edge).  An anchored record's image is checked
// against its target bin by the fast binning and clamped into it by the
// bin's thresholds where that check does not confirm it.
__device__ __forceinline__ float match_one_f32_general(const MatchSmem& m, const float* __restrict__ thr,
                                                       const BinF32& bf, float x)
{
    float fi;
    const int i = bin_fast_f32(bf, thr, x, fi);
    const float4 r = m.rec[i];
    const bool below = !(x >= bf.thr0);
    const bool above = x >= bf.thrI;
    float f = (x - fmaf(fi, bf.h, bf.lo)) * bf.inv_h;
    f = fminf(fmaxf(f, 0.0f), 1.0f);
    if (below) f = 0.0f;
    if (above) f = 1.0f;
    float xn;
    if (r.z >= 0.0f) {
        const bool second = f >= r.y;
        xn = fmaf(second ? fabsf(r.w) : r.z, f - r.y, r.x);
        const int jm = __float2int_rn((r.x - bf.lo) * bf.inv_h);
        const int j = min(second ? jm : jm - 1, bf.bins - 1);
        if (bin_try_f32(bf, xn) != j) xn = fminf(fmaxf(xn, thr[j]), thr[j + 1]);
    } else {
        const uint32_t kk = __float_as_uint(r.x);
        const int k0 = (int)(kk & 0xFFFFu), k1 = (int)(kk >> 16);
        if (k0 == k1) return x;   // identity on this bin
        int k = k0;
        while (k < k1 - 1 && f > m.fend[k]) ++k;
        const float4 pc = m.piece[k];
        xn = fminf(fmaxf(fmaf(pc.y, f, pc.x), pc.z), pc.w);
    }
    if (below) return x + (xn - bf.thr0);
    if (above) return x + (xn - bf.thrI);
    return xn;
}

// Map one binary32 particle through the table.  Fast path (most particles:
// inside the grid, away from their bin's edges by the binning's error
// margin, on an identity bin or a safe anchored record): the bin and the
// fraction f = d + 1/2 come from one rounding (d the signed distance to the
// bin's middle, in bins), one 16-byte record gives the image, and no
// threshold is read.  Everything else takes the general path.
__device__ __forceinline__ float match_one_f32(const MatchSmem& m, const float* __restrict__ thr, const BinF32& bf,
                                               float x)
{
    const float g = fmaf(x, bf.inv_h, bf.c);
    const float t = g + 12582912.0f;
    const float d = g - (t - 12582912.0f);
    const int i = __float_as_int(t) - 0x4B400000;
    if ((unsigned)i < (unsigned)bf.bins && fabsf(d) <= bf.half_m) {
        const float4 r = m.rec[i];
        if (r.z >= 0.0f && r.w >= 0.0f) {
            const float f = d + 0.5f;
            return fmaf(f >= r.y ? r.w : r.z, f - r.y, r.x);
        }
        if (r.z == -2.0f) return x;   // identity on this bin
    }
    return match_one_f32_general(m, thr, bf, x);
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
    if (deq(m.Cp[i], m.Ct[i]) && deq(m.Cp[i + 1], m.Ct[i + 1])) return x;
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

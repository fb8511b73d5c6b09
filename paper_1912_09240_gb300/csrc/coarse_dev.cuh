// coarse_dev.cuh -- FP64 block-level pieces of the coarse propagator and the
// serial update (Sections 2.2.2, 3.2.3, 4): deterministic scans, the coarse
// step on one state, the iterators, and the serial sweep over the slices;
// shared by the single-problem and the batched kernels.
#pragma once

#include <cooperative_groups.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "pr_common.cuh"

namespace pr {

namespace cg = cooperative_groups;

// Work split over the CL CTAs of a thread-block cluster (CL = 1: one CTA).
// Each CTA computes its share [lo(n), hi(n)) of an index range into an
// array in its shared memory; share() copies that part into the same array
// of every other CTA of the cluster (the arrays sit at the same offsets in
// every CTA, distributed shared memory) and synchronises the cluster, so
// that every CTA then holds the whole array.  Each element is computed by
// one CTA with the arithmetic of the single-CTA code, so the results do not
// depend on CL.
template <int CL>
struct Dist {
    int rank;
    __device__ static Dist make()
    {
        Dist d;
        d.rank = CL > 1 ? (int)cg::this_cluster().block_rank() : 0;
        return d;
    }
    __device__ int lo(int n) const { return (int)(((long long)n * rank) / CL); }
    __device__ int hi(int n) const { return (int)(((long long)n * (rank + 1)) / CL); }
    template <typename T>
    __device__ void share(T* arr, int b, int e) const
    {
        __syncthreads();
        if constexpr (CL > 1) {
            cg::cluster_group cl = cg::this_cluster();
            for (int q = 1; q < CL; ++q) {
                T* dst = cl.map_shared_rank(arr, (unsigned)((rank + q) % CL));
                for (int i = b + (int)threadIdx.x; i < e; i += (int)blockDim.x) dst[i] = arr[i];
            }
            cl.sync();
        }
    }
    __device__ void sync() const
    {
        if constexpr (CL > 1) cg::this_cluster().sync();
        else __syncthreads();
    }
};

constexpr int kCoarseThreads = 512;   // every coarse apply uses this block size
constexpr int kUpdateMaxBins = 1024;
// Bin masses of a coarse result at or below this are dropped: below it the
// entries of P @ m are rounding noise of the matrix exponential (absolute
// error ~1e-15), which would otherwise decide where the support of the
// result ends, and with it the quantile iterator's q(0) and q(1).
constexpr double kTailMass = 1e-10;

// ---------------------------------------------------------------------------
// Block-level FP64 helpers (deterministic order for a fixed blockDim)
// ---------------------------------------------------------------------------

// Inclusive scan of v[0..n) into out[0..n) (out may equal v); wsum >= 33 doubles.
__device__ inline void block_scan_f64(const double* v, double* out, int n, double* wsum)
{
    const int T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int b = threadIdx.x * chunk, e = min(n, b + chunk);
    double loc = 0.0;
    for (int i = b; i < e; ++i) loc = __dadd_rn(loc, v[i]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl = __dadd_rn(t, incl);
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        const int nw = T >> 5;
        for (int w = 0; w < nw; ++w) {
            const double t = wsum[w];
            wsum[w] = run;
            run = __dadd_rn(run, t);
        }
        wsum[32] = run;
    }
    __syncthreads();
    // exclusive prefix of this thread: the warp's offset plus the inclusive
    // prefix of the previous lane
    const double prev = __shfl_up_sync(0xffffffffu, incl, 1);
    double run = lane > 0 ? __dadd_rn(wsum[warp], prev) : wsum[warp];
    double lmax = -INFINITY;
    for (int i = b; i < e; ++i) {
        run = __dadd_rn(run, v[i]);
        lmax = fmax(lmax, run);
        out[i] = lmax;
    }
    // The prefix of a thread's first element and the last prefix of the
    // thread before it are rounded in different orders, so for non-negative
    // inputs they can step back by an ulp.  A prefix maximum (exact in any
    // order) makes the scan non-decreasing again.
    double imax = lmax;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, imax, o);
        if (lane >= o) imax = fmax(imax, t);
    }
    __syncthreads();   // everyone is done reading wsum
    if (lane == 31) wsum[warp] = imax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = -INFINITY;
        const int nw = T >> 5;
        for (int w = 0; w < nw; ++w) {
            const double t = wsum[w];
            wsum[w] = m;
            m = fmax(m, t);
        }
    }
    __syncthreads();
    const double pmax_lane = __shfl_up_sync(0xffffffffu, imax, 1);
    const double before = lane > 0 ? fmax(wsum[warp], pmax_lane) : wsum[warp];
    for (int i = b; i < e; ++i) out[i] = fmax(out[i], before);
    __syncthreads();
}

// Block sum of one value per thread (deterministic); wsum >= 33 doubles.
__device__ inline double block_sum_f64(double v, double* wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = __dadd_rn(s, wsum[w]);
        wsum[32] = s;
    }
    __syncthreads();
    const double r = wsum[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// C_dT on one state: masses, P @ masses (masses <= kTailMass dropped), CDF of
// the result normalised to unit mass.  cdf_in, out: [I+1]; mass, mp: [I].
// All in shared memory; every thread of a kCoarseThreads block calls it.
// ---------------------------------------------------------------------------

template <int CL = 1>
__device__ inline void coarse_apply_block(const double* __restrict__ P, int I, const double* cdf_in,
                                          double* out, double* mass, double* mp, double* wsum,
                                          const Dist<CL> d = Dist<CL>{0})
{
    for (int c = threadIdx.x; c < I; c += blockDim.x) mass[c] = __dsub_rn(cdf_in[c + 1], cdf_in[c]);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int r0 = d.lo(I), r1 = d.hi(I);
    for (int r = r0 + warp; r < r1; r += nw) {
        const double* row = P + (size_t)r * I;
        double acc = 0.0;
        for (int c = lane; c < I; c += 32) acc = fma(row[c], mass[c], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if (lane == 0) mp[r] = acc > kTailMass ? acc : 0.0;
    }
    d.share(mp, r0, r1);
    block_scan_f64(mp, mp, I, wsum);
    const double total = mp[I - 1];
    const int q0 = d.lo(I - 1), q1 = d.hi(I - 1);
    for (int r = q0 + threadIdx.x; r < q1; r += blockDim.x) {
        double v = total > 0.0 ? __ddiv_rn(mp[r], total) : 0.0;
        out[r + 1] = v < 1.0 ? v : 1.0;
    }
    if (threadIdx.x == 0) {
        out[0] = 0.0;
        out[I] = 1.0;
    }
    d.share(out, 1 + q0, 1 + q1);
}

// ---------------------------------------------------------------------------
// Quantile iterator J_q (Section 4.4) on CDFs in shared memory.
// ---------------------------------------------------------------------------

// Ordered 64-bit key of a non-NaN double: signed comparison of keys is
// numeric comparison, and -0 and +0 both map to 0.
__device__ __forceinline__ long long okey(double v)
{
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll) + 1;
}

__device__ __forceinline__ int count_lt(const double* F, int n, double v)   // #F < v
{
    const long long kv = dkey(v);
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (dkey(F[mid]) < kv) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int count_le(const double* F, int n, double v)   // #F <= v
{
    const long long kv = dkey(v);
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (dkey(F[mid]) <= kv) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Interior quantile: strictly inside bin b (never rounded onto an edge).
__device__ __forceinline__ double inside(const GridDev& g, int b, double t)
{
    const double e0 = edge(g, b), e1 = edge(g, b + 1);
    double q = __dadd_rn(e0, __dmul_rn(t, g.h));
    if (q <= e0) q = nextafter(e0, e1);
    if (q >= e1) q = nextafter(e1, e0);
    return q;
}

// Both one-sided quantiles of a CDF F at level p:
//   q^-(p) = min{x : F(x) >= p},  q^+(p) = max{x : F(x) <= p}.
// They differ only where F is flat at p; otherwise one interpolation serves both.
__device__ __forceinline__ void quantiles(const GridDev& g, const double* F, double p, double& qm, double& qp)
{
    const int I = g.bins;
    const int a = count_lt(F, I + 1, p);   // lowest index with F[a] >= p (F[I] = 1 >= p)
    if (a == 0 || F[a] == p) {
        const int b = count_le(F, I + 1, p) - 1;   // highest index with F[b] <= p
        qm = edge(g, a);
        qp = edge(g, b);
        return;
    }
    const double t = __ddiv_rn(__dsub_rn(p, F[a - 1]), __dsub_rn(F[a], F[a - 1]));
    qm = qp = inside(g, a - 1, t);
}

struct JqSmem {
    double* levels;   // [3(I+1)]
    double* kq;       // [6(I+1)]  knots
    double* bsum;     // [6(I+1)]  merged levels, then sums of pooled blocks
    int* ibuf;        // [6(I+1)]  (distinct flags, then the descent list)
    int* bpos;        // [6(I+1)]  pooled blocks: start | end << 16
    int* flag;        // [0]: level count, [1]: input not a CDF, [2]: knots need repair
    double* wsum;     // [40]
};

__host__ __device__ inline size_t jq_smem_bytes(int bins)
{
    const size_t M = 3 * (size_t)(bins + 1);
    return (M + 2 * M + 2 * M + 40) * sizeof(double) + (4 * M + 4) * sizeof(int);
}

__device__ inline JqSmem carve_jq(unsigned char* base, int bins)
{
    const int M = 3 * (bins + 1);
    JqSmem j;
    j.levels = reinterpret_cast<double*>(base);
    j.kq = j.levels + M;
    j.bsum = j.kq + 2 * M;
    j.wsum = j.bsum + 2 * M;
    j.ibuf = reinterpret_cast<int*>(j.wsum + 40);
    j.bpos = j.ibuf + 2 * M;
    j.flag = j.bpos + 2 * M;
    return j;
}

// out = J_q(A, B, C).  A, B, C, out: [I+1] in shared memory (out distinct).
// Returns through flag[1] a non-zero value if an input was not a CDF.  With a
// cluster (CL > 1) the quantiles at the levels and the read-back at the edges
// are split over its CTAs; the rest runs in every CTA on identical data.
template <int CL = 1>
__device__ inline void quantile_iterate_block(const GridDev& g, int qmode, const double* A, const double* B,
                                              const double* C, double* out, JqSmem& s,
                                              const Dist<CL> d = Dist<CL>{0})
{
    const int I = g.bins;
    const int n1 = I + 1;
    const int M = 3 * n1;
    if (threadIdx.x == 0) s.flag[2] = 0;
    // validity: in [0, 1] (NaN fails) and non-decreasing, by ordered keys
    const long long k0 = okey(0.0), k1 = okey(1.0);
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        const double* Fs[3] = {A, B, C};
        for (int f = 0; f < 3; ++f) {
            const long long kv = okey(Fs[f][i]);
            bool bad = kv < k0 || kv > k1;
            if (i > 0 && okey(Fs[f][i - 1]) > kv) bad = true;
            if (bad) s.flag[1] = 1;
        }
    }
    // 1. sorted union of the 3(I+1) levels (stable merge by rank) into bsum
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        const int f = k / n1, i = k - f * n1;
        double v;
        int r;
        if (f == 0) { v = A[i]; r = i + count_lt(B, n1, v) + count_lt(C, n1, v); }
        else if (f == 1) { v = B[i]; r = i + count_le(A, n1, v) + count_lt(C, n1, v); }
        else { v = C[i]; r = i + count_le(A, n1, v) + count_le(B, n1, v); }
        s.bsum[r] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < M; k += blockDim.x)
        s.ibuf[k] = (k == 0 || !deq(s.bsum[k], s.bsum[k - 1])) ? 1 : 0;
    __syncthreads();
    // exclusive scan of the distinct flags -> positions (ints, deterministic)
    {
        const int T = blockDim.x;
        const int chunk = (M + T - 1) / T;
        const int b = threadIdx.x * chunk, e = min(M, b + chunk);
        int loc = 0;
        for (int i = b; i < e; ++i) loc += s.ibuf[i];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int incl = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int* wtot = reinterpret_cast<int*>(s.wsum);
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        int off = 0;
        for (int w = 0; w < warp; ++w) off += wtot[w];
        int run = off + incl - loc;
        for (int i = b; i < e; ++i) {
            if (s.ibuf[i]) s.levels[run] = s.bsum[i];
            run += s.ibuf[i];
        }
        if (threadIdx.x == T - 1) s.flag[0] = run;   // number of levels L
    }
    __syncthreads();
    const int L = s.flag[0];
    __syncthreads();
    // 2-3. quantiles of A, B, C at every level and the combined knots
    const bool two = qmode == PR_QMODE_TWO_SIDED;
    const int nk = two ? 2 * L - 2 : L;
    const int l0 = d.lo(L), l1 = d.hi(L);
    for (int l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
        const double p = s.levels[l];
        const bool first = l == 0, last = l == L - 1;
        double am, ap, bm, bp, cm, cp;
        quantiles(g, A, p, am, ap);
        quantiles(g, B, p, bm, bp);
        quantiles(g, C, p, cm, cp);
        if (two) {
            if (!first) s.kq[2 * l - 1] = __dadd_rn(__dadd_rn(bm, __dsub_rn(am, cm)), 0.0);
            if (!last) s.kq[2 * l] = __dadd_rn(__dadd_rn(bp, __dsub_rn(ap, cp)), 0.0);
        } else {
            double qa, qb, qc;
            if (first) { qa = ap; qb = bp; qc = cp; }
            else if (last) { qa = am; qb = bm; qc = cm; }
            else {
                qa = __dmul_rn(0.5, __dadd_rn(am, ap));
                qb = __dmul_rn(0.5, __dadd_rn(bm, bp));
                qc = __dmul_rn(0.5, __dadd_rn(cm, cp));
            }
            s.kq[l] = __dadd_rn(__dadd_rn(qb, __dsub_rn(qa, qc)), 0.0);
        }
    }
    // knots of levels [l0, l1): 2l - 1 and 2l (two-sided), l (midpoint)
    if (two) d.share(s.kq, max(2 * l0 - 1, 0), min(2 * l1 - 1, nk));
    else d.share(s.kq, l0, l1);
    // 4. monotone repair: pool adjacent violators (PAV) with equal weights.
    //    A boundary between knots k-1 and k where max(q[0..k-1]) <= min(q[k..])
    //    is never crossed by a pooled block, and the left-to-right stack
    //    algorithm does the same merges, with the same additions in the same
    //    order, on each side of it as it does on the whole.  So the knots are
    //    cut at every such boundary (exact integer max/min scans on ordered
    //    keys) and each segment is pooled by its own thread with that
    //    algorithm; the bits are those of the single sequential pass.
    {
        long long* pm = reinterpret_cast<long long*>(s.bsum);   // prefix max of the keys
        long long* wl = reinterpret_cast<long long*>(s.wsum);
        const int T = blockDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int chunk = (nk + T - 1) / T;
        // prefix maximum, chunks in index order
        {
            const int b0 = threadIdx.x * chunk, e0 = min(nk, b0 + chunk);
            long long loc = LLONG_MIN;
            for (int i = b0; i < e0; ++i) loc = max(loc, okey(s.kq[i]));
            long long incl = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl = max(incl, t);
            }
            if (lane == 31) wl[warp] = incl;
            __syncthreads();
            long long run = LLONG_MIN;
            for (int w = 0; w < warp; ++w) run = max(run, wl[w]);
            const long long prev = __shfl_up_sync(0xffffffffu, incl, 1);
            if (lane > 0) run = max(run, prev);
            for (int i = b0; i < e0; ++i) {
                run = max(run, okey(s.kq[i]));
                pm[i] = run;
            }
            __syncthreads();
        }
        // suffix minimum, chunks in reverse index order; segment starts into ibuf
        {
            const int r0 = threadIdx.x * chunk, r1 = min(nk, r0 + chunk);   // reversed positions
            long long loc = LLONG_MAX;
            for (int r = r0; r < r1; ++r) loc = min(loc, okey(s.kq[nk - 1 - r]));
            long long incl = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl = min(incl, t);
            }
            if (lane == 31) wl[warp] = incl;
            __syncthreads();
            long long run = LLONG_MAX;
            for (int w = 0; w < warp; ++w) run = min(run, wl[w]);
            const long long prev = __shfl_up_sync(0xffffffffu, incl, 1);
            if (lane > 0) run = min(run, prev);
            for (int r = r0; r < r1; ++r) {
                const int k = nk - 1 - r;
                run = min(run, okey(s.kq[k]));
                s.ibuf[k] = (k == 0 || pm[k - 1] <= run) ? 1 : 0;
            }
        }
        __syncthreads();
        // segment starts -> sorted list in bpos (deterministic compaction)
        {
            const int b0 = threadIdx.x * chunk, e0 = min(nk, b0 + chunk);
            int loc = 0;
            for (int i = b0; i < e0; ++i) loc += s.ibuf[i];
            int incl = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            int* wtot = reinterpret_cast<int*>(s.wsum);
            if (lane == 31) wtot[warp] = incl;
            __syncthreads();
            int off = 0;
            for (int w = 0; w < warp; ++w) off += wtot[w];
            int run = off + incl - loc;
            for (int i = b0; i < e0; ++i) {
                if (s.ibuf[i]) s.bpos[run] = i;
                run += s.ibuf[i];
            }
            if (threadIdx.x == T - 1) {
                s.flag[2] = run;      // number of segments
                s.bpos[run] = nk;     // end of the last one
            }
        }
        __syncthreads();
        const int nseg = s.flag[2];
        // each segment [a, e) by one thread: the stack of pooled blocks below
        // the top lives in bsum[a..] (sums) and ibuf[a..] (counts), the top
        // block in registers
        for (int j = threadIdx.x; j < nseg; j += T) {
            const int a = s.bpos[j], e = s.bpos[j + 1];
            if (e - a < 2) continue;   // one knot: nothing to pool
            double R = s.kq[a];
            int nr = 1, nb = 0;
            for (int k = a + 1; k < e; ++k) {
                s.bsum[a + nb] = R;
                s.ibuf[a + nb] = nr;
                ++nb;
                R = s.kq[k];
                nr = 1;
                while (nb > 0) {
                    const double Ls = s.bsum[a + nb - 1];
                    const int nl = s.ibuf[a + nb - 1];
                    // mean(left) > mean(right) as sum_l * n_r > sum_r * n_l
                    if (!(__dmul_rn(Ls, (double)nr) > __dmul_rn(R, (double)nl))) break;
                    R = __dadd_rn(Ls, R);
                    nr += nl;
                    --nb;
                }
            }
            s.bsum[a + nb] = R;
            s.ibuf[a + nb] = nr;
            ++nb;
            int k = a;
            for (int t = 0; t < nb; ++t) {
                const int c = s.ibuf[a + t];
                if (c >= 2) {   // a knot that pooled with nothing keeps its bits
                    const double mean = __dadd_rn(__ddiv_rn(s.bsum[a + t], (double)c), 0.0);
                    for (int u = 0; u < c; ++u) s.kq[k + u] = mean;
                }
                k += c;
            }
        }
    }
    __syncthreads();
    // 5. PL CDF through the knots, right-continuous, read at the interior edges
    const int e0 = 1 + d.lo(I - 1), e1 = 1 + d.hi(I - 1);
    for (int i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
        const double x = edge(g, i);
        const long long kx = okey(x);
        int lo = 0, hi = nk;   // first knot with kq > x
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (okey(s.kq[mid]) <= kx) lo = mid + 1; else hi = mid;
        }
        const int j = lo - 1;
        double v;
        if (j < 0) v = 0.0;
        else {
            const double pj = s.levels[two ? (j + 1) >> 1 : j];
            if (j == nk - 1) v = pj;
            else {
                const double pn = s.levels[two ? (j + 2) >> 1 : j + 1];
                const double t = __ddiv_rn(__dsub_rn(x, s.kq[j]), __dsub_rn(s.kq[j + 1], s.kq[j]));
                v = __dadd_rn(pj, __dmul_rn(t, __dsub_rn(pn, pj)));
            }
        }
        if (v < 0.0) v = 0.0;
        if (v > 1.0) v = 1.0;
        out[i] = v;
    }
    if (threadIdx.x == 0) {
        out[0] = 0.0;
        out[I] = 1.0;
    }
    d.share(out, e0, e1);
}

// Additive (4.1), multiplicative (4.2) and rotation (4.3) iterators on masses.
__device__ inline void mass_iterate_block(int kind, int I, const double* A, const double* B, const double* C,
                                   double* out, double* r, double* wsum)
{
    double pu = 0.0, pv = 0.0, pw = 0.0;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const double a = __dsub_rn(A[i + 1], A[i]), b = __dsub_rn(B[i + 1], B[i]), c = __dsub_rn(C[i + 1], C[i]);
        if (kind == PR_ITER_ADD) {
            const double v = __dsub_rn(__dadd_rn(a, b), c);
            r[i] = v < 0.0 ? 0.0 : v;
        } else if (kind == PR_ITER_MULT) {
            r[i] = c > 0.0 ? __dmul_rn(a, __ddiv_rn(b, c)) : 0.0;
        } else {
            pu = __dadd_rn(pu, sqrt(__dmul_rn(b, c)));
            pv = __dadd_rn(pv, sqrt(__dmul_rn(b, a)));
            pw = __dadd_rn(pw, sqrt(__dmul_rn(c, a)));
        }
    }
    if (kind == PR_ITER_ROT) {
        const double u = block_sum_f64(pu, wsum);
        const double v = block_sum_f64(pv, wsum);
        const double w = block_sum_f64(pw, wsum);
        const double ca = __ddiv_rn(__dsub_rn(__dadd_rn(u, __dmul_rn(__dmul_rn(2.0, u), w)), v), __dadd_rn(1.0, w));
        const double cc = __ddiv_rn(__dadd_rn(u, v), __dadd_rn(1.0, w));
        for (int i = threadIdx.x; i < I; i += blockDim.x) {
            const double a = __dsub_rn(A[i + 1], A[i]), b = __dsub_rn(B[i + 1], B[i]), c = __dsub_rn(C[i + 1], C[i]);
            const double sv = __dsub_rn(__dadd_rn(__dmul_rn(ca, sqrt(a)), sqrt(b)), __dmul_rn(cc, sqrt(c)));
            r[i] = __dmul_rn(sv, sv);
        }
    }
    __syncthreads();
    block_scan_f64(r, r, I, wsum);
    const double total = r[I - 1];
    if (!(total > 0.0)) {   // no mass to normalise (the multiplicative iterator
        // when the supports of a b and c do not meet): the correction is
        // dropped and the update keeps the fine result b
        for (int i = threadIdx.x; i <= I; i += blockDim.x) out[i] = B[i];
        __syncthreads();
        return;
    }
    for (int i = threadIdx.x; i < I - 1; i += blockDim.x) {
        const double v = __ddiv_rn(r[i], total);
        out[i + 1] = v < 1.0 ? v : 1.0;
    }
    if (threadIdx.x == 0) {
        out[0] = 0.0;
        out[I] = 1.0;
    }
    __syncthreads();
}

__host__ __device__ inline size_t coarse_apply_smem(int bins)
{
    return ((size_t)2 * (bins + 1) + 2 * (size_t)bins + 40) * sizeof(double);
}

__host__ __device__ inline size_t update_smem(int bins)
{
    return (size_t)5 * (bins + 1) * sizeof(double) + jq_smem_bytes(bins);
}

// The serial update of Section 3.2.3 (Eq. mm_sequential) for one problem on
// the calling CTA, or on the CL CTAs of a cluster (kCoarseThreads threads,
// update_smem(bins) bytes at usm in each):
//   rho^0 = cdf0, rho^{n+1} = J(C(rho^n), fstar[n], cstar[n]), n < K.
// Every CTA of the cluster holds the whole state; the matrix-vector product,
// the normalisation, the quantiles and the read-back are split between them
// (Dist), so the FP64 work per slice spreads over CL SMs.  Results do not
// depend on CL.
template <int CL = 1>
__device__ inline void serial_sweep(unsigned char* usm, const double* __restrict__ P, const GridDev& g,
                                    int iterator, int qmode, int K, const double* __restrict__ cdf0,
                                    const double* __restrict__ fstar, const double* __restrict__ cstar,
                                    double* __restrict__ next, int32_t* status)
{
    const Dist<CL> d = Dist<CL>::make();
    const bool writer = d.rank == 0;
    const int I = g.bins;
    double* cur = reinterpret_cast<double*>(usm);
    double* Ab = cur + (I + 1);
    double* Bb = Ab + (I + 1);
    double* Cb = Bb + (I + 1);
    double* Ob = Cb + (I + 1);
    JqSmem js = carve_jq(reinterpret_cast<unsigned char*>(Ob + (I + 1)), I);
    double* mass = js.levels;       // coarse scratch aliases the level list
    double* mp = js.levels + I;
    if (threadIdx.x == 0) js.flag[1] = 0;
    for (int i = threadIdx.x; i <= I; i += blockDim.x) {
        cur[i] = cdf0[i];
        if (writer) next[i] = cdf0[i];
    }
    d.sync();   // every CTA of the cluster runs before any writes into its shared memory
    for (int n = 0; n < K; ++n) {
        coarse_apply_block<CL>(P, I, cur, Ab, mass, mp, js.wsum, d);
        double* res = Ab;
        if (iterator != PR_ITER_NONE) {
            for (int i = threadIdx.x; i <= I; i += blockDim.x) {
                Bb[i] = fstar[(size_t)n * (I + 1) + i];
                Cb[i] = cstar[(size_t)n * (I + 1) + i];
            }
            __syncthreads();
            if (iterator == PR_ITER_QUANTILE) quantile_iterate_block<CL>(g, qmode, Ab, Bb, Cb, Ob, js, d);
            else mass_iterate_block(iterator, I, Ab, Bb, Cb, Ob, js.kq, js.wsum);
            res = Ob;
        }
        for (int i = threadIdx.x; i <= I; i += blockDim.x) {
            const double v = res[i];
            if (!isfinite(v)) js.flag[1] = 1;
            cur[i] = v;
            if (writer) next[(size_t)(n + 1) * (I + 1) + i] = v;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && status && writer) *status = js.flag[1] ? PR_ERR_NUMERIC : PR_OK;
    d.sync();   // no CTA leaves while another may still write into its shared memory
}

}  // namespace pr

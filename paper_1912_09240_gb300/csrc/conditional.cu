// conditional.cu -- matching that preserves the conditional distribution
// (Section 5.2): reweighting of the prior ensemble to the target histogram,
// W^p = Wbar^p rho'_i / rhobar_i, with the mass of target bins the prior
// does not support moved half to the nearest supported bin on each side (all
// of it to the only side that has one); stratified resampling of weighted
// ensembles (Eq. stratified) and its deterministic variant u~ = 1/2; and the
// restriction with weights.
//
// Weights enter sums in fixed point, round(W 2^61) as 64-bit integers, so
// that cumulative weights -- and with them the particle each resampled slot
// takes and the weighted histograms -- are exact and independent of the
// order in which threads add them.  The strata points are exact integers too:
// U_j = floor(T (j 2^24 + a_j) / (N 2^24)), T the total fixed weight and
// a_j / 2^24 = u~_j (a_j the odd 24-bit integer of a Philox uniform, or
// 2^23).  Equal weights therefore reproduce the ensemble exactly (the strong
// projection property).
//
// The per-particle passes are HBM streams; none of them does binary64
// arithmetic per particle (GB300's FP64 pipe is narrow): the fixed point is
// taken in integer arithmetic on the encoding, and the reweighting factors
// are multiplied out per bin.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "pr_common.cuh"

namespace pr {

constexpr int kCondThreads = 512;

// Fixed point of a probability weight: round(w 2^61) to nearest, ties to
// even (0 for w <= 0 or NaN; saturated at 2^64 - 1 from w >= 8 on), in
// integer arithmetic on the binary64 encoding: w = M 2^(E - 1075) with the
// 53-bit significand M, so w 2^61 = M 2^(E - 1014).  Below 1 the shift right
// by k rounds to nearest-even by adding 2^(k-1) - 1 plus the lowest kept bit.
__device__ __forceinline__ uint64_t weight_fixed(double w)
{
    const uint64_t b = (uint64_t)__double_as_longlong(w);
    const uint32_t hi = (uint32_t)(b >> 32);
    if ((int32_t)hi < 0) return 0ull;                       // the sign bit set (negative, -0, NaN with sign)
    const int k = 1014 - (int)(hi >> 20);                    // w 2^61 = M 2^-k
    if (k > 53) return 0ull;                                 // below 1/2, +0 and subnormals included
    if (k < -11) return (b << 12) && (hi >> 20) == 2047 ? 0ull : ~0ull;   // w >= 8 saturates; NaN -> 0
    const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    if (k <= 0) return M << -k;                              // exact below 2^64
    return (M + ((1ull << (k - 1)) - 1ull) + ((M >> k) & 1ull)) >> k;
}

// In-place inclusive scan of a[0..I) with an associative `op` (identity
// `ident`), by the whole block, from the right end when `reverse`: each thread
// scans a run of consecutive elements, and the run totals are combined by a
// warp scan and a scan of the warp totals (wtmp: 32 ints).
template <typename Op>
__device__ void block_scan_int(int* a, int I, int ident, Op op, bool reverse, int* wtmp)
{
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int c = (I + T - 1) / T, b = min(I, t * c), e = min(I, b + c);
    auto at = [&](int i) -> int& { return a[reverse ? I - 1 - i : i]; };
    int run = ident;
    for (int i = b; i < e; ++i) run = op(run, at(i));
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl = op(v, incl);
    }
    if (lane == 31) wtmp[warp] = incl;
    __syncthreads();
    int acc = ident;
    for (int k = 0; k < warp; ++k) acc = op(acc, wtmp[k]);
    const int prev = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane > 0) acc = op(acc, prev);
    for (int i = b; i < e; ++i) {
        acc = op(acc, at(i));
        at(i) = acc;
    }
    __syncthreads();
}

struct ReweightSmem {
    double *r, *rb, *rt;
    int *left, *right, *next;   // nearest supported bin <= i, >= i; next contributing bin >= i
    int* wtmp;
};

__host__ __device__ inline size_t reweight_smem_bytes(int I)
{
    return (size_t)I * 24 + (size_t)I * 12 + 32 * 4;
}

// r[i] = rho'_i / rhobar_i for one prior/target pair, by the whole block.
// Bin b with prior mass collects its own target mass, then that of the
// unsupported bins between it and the previous supported bin (left to right),
// then that of those up to the next supported bin, each halved where both
// sides have a supported bin: the additions of the left-to-right visit of the
// unsupported bins, in the same order.  The gaps come from block scans (the
// nearest supported bin on each side, the next unsupported bin with target
// mass), so each bin's loops visit only the bins that add to it.
__device__ void reweight_factors_block(int I, const double* __restrict__ Cp, const double* __restrict__ Ct,
                                       const ReweightSmem& m)
{
    for (int b = threadIdx.x; b < I; b += blockDim.x) {
        const double mb = __dsub_rn(Cp[b + 1], Cp[b]), mt = __dsub_rn(Ct[b + 1], Ct[b]);
        const bool sup = mb > 0.0;
        m.rb[b] = mb;
        m.rt[b] = mt;
        m.left[b] = sup ? b : -1;
        m.right[b] = sup ? b : I;
        m.next[b] = (!sup && mt > 0.0) ? b : I;
    }
    __syncthreads();
    const auto mx = [](int u, int v) { return max(u, v); };
    const auto mn = [](int u, int v) { return min(u, v); };
    block_scan_int(m.left, I, -1, mx, false, m.wtmp);
    block_scan_int(m.right, I, I, mn, true, m.wtmp);
    block_scan_int(m.next, I, I, mn, true, m.wtmp);
    for (int b = threadIdx.x; b < I; b += blockDim.x) {
        const double mb = m.rb[b];
        if (!(mb > 0.0)) {
            m.r[b] = 0.0;
            continue;
        }
        double rn = m.rt[b];
        const int L = b > 0 ? m.left[b - 1] : -1;
        for (int i = m.next[L + 1]; i < b; i = m.next[i + 1])
            rn = __dadd_rn(rn, L >= 0 ? __dmul_rn(0.5, m.rt[i]) : m.rt[i]);
        const int R = b + 1 < I ? m.right[b + 1] : I;
        for (int i = b + 1 < I ? m.next[b + 1] : I; i < R; i = i + 1 < I ? m.next[i + 1] : I)
            rn = __dadd_rn(rn, R < I ? __dmul_rn(0.5, m.rt[i]) : m.rt[i]);
        m.r[b] = __ddiv_rn(rn, mb);
    }
}

// W^p = Wbar^p r_{bin(Xbar^p)}; one CTA per (range, slice), the factors built
// per CTA in shared memory.  Without prior weights W = (1/n) r_i is taken once
// per bin (the same rounding as per particle).  Binary32 positions stream as
// 16-byte vectors (two in flight per thread), binary64 ones four at a time.
template <typename T>
__global__ void __launch_bounds__(kCondThreads)
reweight_kernel(const T* __restrict__ x, int64_t in_stride, const double* __restrict__ wbar, int64_t n,
                GridDev g, float lo_f, float inv_h_f, const double* __restrict__ cp, const double* __restrict__ ct,
                double* __restrict__ w, int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int I = g.bins;
    ReweightSmem m;
    m.r = reinterpret_cast<double*>(smem);
    m.rb = m.r + I;
    m.rt = m.rb + I;
    m.left = reinterpret_cast<int*>(m.rt + I);
    m.right = m.left + I;
    m.next = m.right + I;
    m.wtmp = m.next + I;
    double* r = m.r;
    float* thr = reinterpret_cast<float*>(smem + ((reweight_smem_bytes(I) + 15) & ~(size_t)15));
    const int s = blockIdx.y;
    if (sizeof(T) == 4) build_thresholds(g, thr);
    reweight_factors_block(I, cp + (size_t)s * (I + 1), ct + (size_t)s * (I + 1), m);
    __syncthreads();
    if (!wbar) {
        const double w0 = __ddiv_rn(1.0, (double)n);
        for (int i = threadIdx.x; i < I; i += blockDim.x) r[i] = __dmul_rn(w0, r[i]);
    }
    __syncthreads();
    const T* xs = x + (int64_t)s * in_stride;
    const double* wbs = wbar ? wbar + (int64_t)s * in_stride : nullptr;
    double* ws = w + (int64_t)s * n;
    const int64_t b = (int64_t)blockIdx.x * per_block, e = min(n, b + per_block);
    const int Tn = blockDim.x, t = threadIdx.x;
    auto put = [&](int64_t p, int i) { __stcs(ws + p, wbs ? __dmul_rn(__ldcs(wbs + p), r[i]) : r[i]); };
    if (sizeof(T) == 4) {
        const float* xf = reinterpret_cast<const float*>(xs);
        const BinF32 bf = make_bin_f32(thr, I, lo_f, inv_h_f);
        const int64_t mis = (int64_t)(((uintptr_t)(xf + b) >> 2) & 3);
        const int64_t hb = min(e, b + ((4 - mis) & 3));
        for (int64_t p = b + t; p < hb; p += Tn) put(p, bin_fast_f32(bf, thr, xf[p]));
        const int64_t nv = (e - hb) >> 2;
        const float4* __restrict__ v = reinterpret_cast<const float4*>(xf + hb);
        const bool pair_out = !wbs && ((reinterpret_cast<uintptr_t>(ws + hb) & 15) == 0);
        auto four = [&](int64_t q, float4 u) {
            int i0 = bin_try_f32(bf, u.x), i1 = bin_try_f32(bf, u.y);
            int i2 = bin_try_f32(bf, u.z), i3 = bin_try_f32(bf, u.w);
            if ((i0 | i1 | i2 | i3) < 0) {
                const auto th = [thr](int k) { return thr[k]; };
                if (i0 < 0) i0 = bin_slow_f32(bf, th, u.x);
                if (i1 < 0) i1 = bin_slow_f32(bf, th, u.y);
                if (i2 < 0) i2 = bin_slow_f32(bf, th, u.z);
                if (i3 < 0) i3 = bin_slow_f32(bf, th, u.w);
            }
            const int64_t p = hb + 4 * q;
            if (pair_out) {
                double2* o = reinterpret_cast<double2*>(ws + p);
                __stcs(o, make_double2(r[i0], r[i1]));
                __stcs(o + 1, make_double2(r[i2], r[i3]));
            } else {
                put(p, i0);
                put(p + 1, i1);
                put(p + 2, i2);
                put(p + 3, i3);
            }
        };
        int64_t q = t;
        for (; q + Tn < nv; q += 2 * Tn) {
            const float4 u0 = __ldcs(v + q), u1 = __ldcs(v + q + Tn);
            four(q, u0);
            four(q + Tn, u1);
        }
        if (q < nv) four(q, __ldcs(v + q));
        for (int64_t p = hb + 4 * nv + t; p < e; p += Tn) put(p, bin_fast_f32(bf, thr, xf[p]));
    } else {
        const double* xd = reinterpret_cast<const double*>(xs);
        for (int64_t p = b + t; p < e; p += 4 * Tn) {
            double u[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) u[k] = p + k * Tn < e ? __ldcs(xd + p + k * Tn) : 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (p + k * Tn < e) put(p + k * Tn, bin_of_f64(g, u[k]));
        }
    }
}

// ---------------------------------------------------------------------------
// Resampling: cumulative fixed weights C_p = sum_{q <= p} round(W^q 2^61)
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;                              // elements per thread
constexpr int kScanBlock = kScanThreads * kScanPer;      // elements per block

// Sum of the fixed weights of each block of kScanBlock elements, one warp
// per block (kScanWarps blocks per CTA, no block-wide synchronisation).
constexpr int kScanWarps = kScanThreads / 32;

__global__ void __launch_bounds__(kScanThreads)
fixed_blocksum_kernel(const double* __restrict__ w, int64_t n, int64_t nblk, uint64_t* __restrict__ bsum)
{
    const int s = blockIdx.y, lane = threadIdx.x & 31;
    const int64_t blk = (int64_t)blockIdx.x * kScanWarps + (threadIdx.x >> 5);
    if (blk >= nblk) return;
    const double* ws = w + (int64_t)s * n;
    const int64_t b0 = blk * kScanBlock;
    uint64_t loc = 0;
    for (int c = 0; c < kScanBlock; c += 8 * 32) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t p = b0 + c + k * 32 + lane;
            v[k] = p < n ? __ldcs(ws + p) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) loc += weight_fixed(v[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if (lane == 0) bsum[(int64_t)s * nblk + blk] = loc;
}

// Exclusive scan of the block sums of each slice (one CTA per slice); the
// total of slice s goes to total[s].
__global__ void __launch_bounds__(1024)
scan_blocks_kernel(uint64_t* __restrict__ bsum, int64_t nblk, uint64_t* __restrict__ total)
{
    __shared__ uint64_t wtot[32];
    const int s = blockIdx.x;
    uint64_t* b = bsum + (int64_t)s * nblk;
    const int T = blockDim.x;
    const int64_t chunk = (nblk + T - 1) / T;
    const int64_t b0 = (int64_t)threadIdx.x * chunk, e0 = min(nblk, b0 + chunk);
    uint64_t loc = 0;
    for (int64_t i = b0; i < e0; ++i) loc += b[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    uint64_t off = 0;
    for (int k = 0; k < warp; ++k) off += wtot[k];
    uint64_t run = off + incl - loc;
    for (int64_t i = b0; i < e0; ++i) {
        const uint64_t v = b[i];
        b[i] = run;
        run += v;
    }
    if (threadIdx.x == T - 1) total[s] = run;
}

// C_p: the weights are read again and each block's inclusive scan is added
// to its offset, one warp per block in chunks of 256 elements.  In a chunk,
// lane l scans the 8 consecutive elements 8l .. 8l+7; loads and stores stay
// coalesced through a warp-private stage in shared memory (one pad word per 8,
// so that a lane's run and its neighbours' sit in distinct banks).
constexpr int kScanChunk = 8 * 32;

__device__ __forceinline__ int scan_pad(int i) { return i + i / 8; }

__global__ void __launch_bounds__(kScanThreads)
scan_within_kernel(const double* __restrict__ w, uint64_t* __restrict__ C, int64_t n, int64_t nblk,
                   const uint64_t* __restrict__ boff)
{
    __shared__ uint64_t stage_all[kScanWarps][kScanChunk + kScanChunk / 8];
    const int s = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t blk = (int64_t)blockIdx.x * kScanWarps + warp;
    if (blk >= nblk) return;
    uint64_t* stage = stage_all[warp];
    const double* ws = w + (int64_t)s * n;
    uint64_t* Cs = C + (int64_t)s * n;
    uint64_t carry = boff[(int64_t)s * nblk + blk];
    for (int64_t c0 = blk * kScanBlock; c0 < min(n, (blk + 1) * kScanBlock); c0 += kScanChunk) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t p = c0 + k * 32 + lane;
            v[k] = p < n ? __ldcs(ws + p) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) stage[scan_pad(k * 32 + lane)] = weight_fixed(v[k]);
        __syncwarp();
        uint64_t r[8], loc = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            r[k] = stage[lane * 9 + k];
            loc += r[k];
        }
        uint64_t incl = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        uint64_t run = carry + incl - loc;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            run += r[k];
            stage[lane * 9 + k] = run;
        }
        carry += __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t p = c0 + k * 32 + lane;
            if (p < n) Cs[p] = stage[scan_pad(k * 32 + lane)];
        }
        __syncwarp();
    }
}

// Output j of slice s takes the particle p with C_{p-1} <= U_j < C_p and
// copies its state, with U_j = floor(T A_j / D), A_j = j 2^24 + a_j,
// D = n 2^24, evaluated without a 128-bit division: with T = Q n + R,
// Q a_j = P1 2^24 + m1 and R j = q2 n + r2,
//   T A_j / D = Q j + P1 + q2 + (m1 n + r2 2^24 + R a_j) / D,
// where the last numerator is below 3 D < 2^58 -- so U_j is Q j + P1 + q2
// plus 0, 1 or 2, found by comparison.  R, r2 < n < 2^32, q2 < j < 2^32 and
// a_j < 2^24, so every product but Q j is a 32 x 32-bit one; (q2, r2) follow
// j by additions.
struct StrataPoint {
    uint64_t Q, D;
    uint32_t R, n, Ql, Qh;
    int mode;
    uint32_t k0, k1, chi, slice;

    // a_j of the stratified mode is the odd 24-bit integer of the uniform of
    // word j mod 4 of Philox block floor(j / 4): one block serves four
    // consecutive outputs.
    __device__ __forceinline__ uint4 block_of(uint32_t jq) const
    {
        return philox4x32_10(make_uint4(jq, 0xFFFFFFFFu, slice, chi | 0xFEu), k0, k1);
    }

    __device__ __forceinline__ static uint32_t odd24(uint32_t w) { return 2u * (w >> 9) + 1u; }

    __device__ __forceinline__ uint32_t a_of(uint32_t j) const
    {
        if (mode != PR_RESAMPLE_STRATIFIED) return 1u << 23;
        const uint4 wd = block_of(j >> 2);
        const uint32_t r = j & 3u;
        return odd24(r == 0 ? wd.x : r == 1 ? wd.y : r == 2 ? wd.z : wd.w);
    }

    // U_j given a_j, q2 = floor(R j / n) and r2 = R j - q2 n
    __device__ __forceinline__ uint64_t at_a(uint32_t j, uint32_t q2, uint32_t r2, uint32_t a) const
    {
        const uint64_t la = (uint64_t)Ql * a;                          // below 2^56
        const uint64_t P1 = (((uint64_t)Qh * a) << 8) + (la >> 24);   // floor(Q a / 2^24)
        const uint32_t m1 = (uint32_t)la & 0xFFFFFFu;
        const uint64_t W = (uint64_t)m1 * n + ((uint64_t)r2 << 24) + (uint64_t)R * a;
        const uint64_t f = W < D ? 0ull : (W < 2 * D ? 1ull : 2ull);
        return Q * (uint64_t)j + P1 + (uint64_t)q2 + f;
    }

    __device__ __forceinline__ uint64_t at(uint32_t j, uint32_t q2, uint32_t r2) const
    {
        return at_a(j, q2, r2, a_of(j));
    }

    __device__ __forceinline__ void divmod_Rj(uint32_t j, uint32_t& q2, uint32_t& r2) const
    {
        const uint64_t Rj = (uint64_t)R * j;
        const uint64_t q = Rj / n;
        q2 = (uint32_t)q;
        r2 = (uint32_t)(Rj - q * n);
    }

    // (q2, r2) of j + 1 from those of j
    __device__ __forceinline__ void step(uint32_t& q2, uint32_t& r2) const
    {
        if (r2 >= n - R) {
            r2 -= n - R;
            ++q2;
        } else {
            r2 += R;
        }
    }

    __device__ __forceinline__ uint64_t operator()(uint32_t j) const
    {
        uint32_t q2, r2;
        divmod_Rj(j, q2, r2);
        return at(j, q2, r2);
    }
};

__device__ __forceinline__ StrataPoint make_strata(uint64_t Q, uint32_t R, int64_t n, int mode, uint32_t k0,
                                                   uint32_t k1, uint32_t chi, uint32_t slice)
{
    StrataPoint U;
    U.n = (uint32_t)n;
    U.Q = Q;
    U.R = R;
    U.Ql = (uint32_t)Q;
    U.Qh = (uint32_t)(Q >> 32);
    U.D = (uint64_t)n << 24;
    U.mode = mode;
    U.k0 = k0;
    U.k1 = k1;
    U.chi = chi;
    U.slice = slice;
    return U;
}

// smallest p in [lo, hi] with C[p] > U, given C[hi] > U
__device__ __forceinline__ int64_t first_above(const uint64_t* __restrict__ C, int64_t lo, int64_t hi, uint64_t U)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (C[mid] > U) hi = mid; else lo = mid + 1;
    }
    return lo;
}

constexpr int kSelThreads = 256;
constexpr int kSelPer = 8;
constexpr int kSelOut = kSelThreads * kSelPer;   // consecutive outputs per CTA
static_assert(kSelPer % 4 == 0, "a thread's outputs start on a Philox block of the strata draws");
constexpr int kSelStage = 4096;                  // cumulative weights staged per CTA

// The particles of the first and last output of every selection CTA: one
// thread per bound, all at once.  The block offsets of the scan locate the
// kScanBlock elements that hold the answer (the last block whose offset is
// <= U), and the search ends inside that block.
__global__ void __launch_bounds__(256)
select_bounds_kernel(const uint64_t* __restrict__ C, const uint64_t* __restrict__ boff,
                     const uint64_t* __restrict__ total, int64_t n, int64_t nblk, int64_t nsel, int mode,
                     uint32_t k0, uint32_t k1, uint32_t chi, uint32_t slice0, int64_t* __restrict__ bounds)
{
    const int s = blockIdx.y;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * nsel) return;
    const uint64_t Tw = total[s];
    int64_t* out = bounds + (int64_t)s * nsel * 2 + q;
    if (Tw == 0) {
        *out = 0;
        return;
    }
    const int64_t c = q >> 1;
    const int64_t j = (q & 1) ? min(n, (c + 1) * kSelOut) - 1 : c * kSelOut;
    const uint64_t Q = Tw / (uint64_t)n;
    const StrataPoint U = make_strata(Q, (uint32_t)(Tw - Q * (uint64_t)n), n, mode, k0, k1, chi, slice0 + (uint32_t)s);
    const uint64_t u = U((uint32_t)j);
    const uint64_t* bo = boff + (int64_t)s * nblk;
    int64_t lo = 0, hi = nblk - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (bo[mid] <= u) lo = mid; else hi = mid - 1;
    }
    const int64_t p0 = lo * kScanBlock, p1 = min(n, p0 + kScanBlock) - 1;
    *out = first_above(C + (int64_t)s * n, p0, p1, u);
}

// Searches over cumulative weights given by an accessor v (index -> C):
// the smallest index in [a, b] with C > u, given C_b > u; and the same from a
// known lower bound a, in steps 1, 2, 4, .. and then a search of the last
// step (C_hi > u).
template <typename V, typename Idx>
__device__ __forceinline__ Idx sel_search(const V& v, Idx a, Idx b, uint64_t u)
{
    while (a < b) {
        const Idx mid = (a + b) >> 1;
        if (v(mid) > u) b = mid; else a = mid + 1;
    }
    return a;
}

template <typename V, typename Idx>
__device__ __forceinline__ Idx sel_gallop(const V& v, Idx a, Idx hi, uint64_t u)
{
    if (v(a) > u) return a;
    Idx step = 1;
    for (;;) {                          // C_a <= u < C_hi, so a < hi
        const Idx nx = a + step;
        if (nx >= hi) return sel_search(v, a + 1, hi, u);
        if (v(nx) > u) return sel_search(v, a + 1, nx, u);
        a = nx;
        step <<= 1;
    }
}

__device__ __forceinline__ int sel_pad(int i) { return i + (i >> 5); }

// A thread's kSelPer consecutive outputs from jj0 on (j0 + jj0 a multiple of
// kSelPer, so they take whole Philox blocks of four draws): their strata
// points first (independent blocks, all in flight), then a search for the
// first particle and a gallop from the previous one for the rest; the
// particles, relative to `base`, go to sp.
template <typename V, typename Idx>
__device__ __forceinline__ void select_run(const V& v, Idx base, Idx hi, const StrataPoint& U, uint32_t j0,
                                           int jj0, int cnt, uint32_t* sp)
{
    const uint32_t j = j0 + (uint32_t)jj0;
    uint32_t q2, r2;
    U.divmod_Rj(j, q2, r2);
    uint32_t a[kSelPer];
    if (U.mode == PR_RESAMPLE_STRATIFIED) {
#pragma unroll
        for (int b = 0; b < kSelPer / 4; ++b) {
            const uint4 wd = U.block_of((j >> 2) + (uint32_t)b);
            a[4 * b] = StrataPoint::odd24(wd.x);
            a[4 * b + 1] = StrataPoint::odd24(wd.y);
            a[4 * b + 2] = StrataPoint::odd24(wd.z);
            a[4 * b + 3] = StrataPoint::odd24(wd.w);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kSelPer; ++k) a[k] = 1u << 23;
    }
    uint64_t u[kSelPer];
#pragma unroll
    for (int k = 0; k < kSelPer; ++k) {
        u[k] = U.at_a(j + (uint32_t)k, q2, r2, a[k]);   // past the end: unused
        U.step(q2, r2);
    }
    const int m = min(kSelPer, cnt - jj0);
    Idx p = sel_search(v, base, hi, u[0]);
    sp[sel_pad(jj0)] = (uint32_t)(p - base);
#pragma unroll
    for (int k = 1; k < kSelPer; ++k) {
        if (k < m) {
            p = sel_gallop(v, p, hi, u[k]);
            sp[sel_pad(jj0 + k)] = (uint32_t)(p - base);
        }
    }
}

// Copies dst[k kSelThreads] = src[pr[k]] for the kSelPer outputs of this
// thread (src starting at the CTA's first particle, dst at the thread's first
// output), all loads issued before the stores.
template <typename T>
__device__ __forceinline__ void gather_rows(const T* __restrict__ src, T* __restrict__ dst, const uint32_t* pr,
                                            int valid)
{
    T v[kSelPer];
#pragma unroll
    for (int k = 0; k < kSelPer; ++k) v[k] = k < valid ? src[pr[k]] : T(0);
#pragma unroll
    for (int k = 0; k < kSelPer; ++k)
        if (k < valid) dst[k * kSelThreads] = v[k];
}

// One CTA takes kSelOut consecutive outputs, whose particles lie between
// those of its first and last output (U and C both increase).  Their
// cumulative weights are staged in shared memory (up to kSelStage of them;
// beyond, they are read from global memory).  Each thread finds the particles
// of kSelPer consecutive outputs into shared memory; the indices and the
// gathered states are then written with consecutive outputs on consecutive
// threads.
template <typename T>
__global__ void __launch_bounds__(kSelThreads)
select_gather_kernel(const uint64_t* __restrict__ C, const uint64_t* __restrict__ total,
                     const int64_t* __restrict__ bounds, int64_t n, int mode, uint32_t k0, uint32_t k1, uint32_t chi,
                     uint32_t slice0, const T* __restrict__ x_in, const T* __restrict__ y_in, int broadcast, int d,
                     uint32_t* __restrict__ idx, T* __restrict__ x_out, T* __restrict__ y_out)
{
    __shared__ uint64_t cs[kSelStage];
    __shared__ uint32_t sp[kSelOut + kSelOut / 32];
    __shared__ uint64_t s_Q;
    const int s = blockIdx.y;
    const int64_t j0 = (int64_t)blockIdx.x * kSelOut, j1 = min(n, j0 + kSelOut);
    const int cnt = (int)(j1 - j0);
    const uint64_t Tw = total[s];
    int64_t lo = j0;
    if (Tw > 0) {
        const int64_t* bd = bounds + ((int64_t)s * gridDim.x + blockIdx.x) * 2;
        lo = bd[0];
        const int64_t hi = bd[1];
        const uint64_t* Cs = C + (int64_t)s * n;
        const int64_t span = hi - lo + 1;
        const int m = (int)min(span, (int64_t)kSelStage);
        if (threadIdx.x == 0) s_Q = Tw / (uint64_t)n;
        for (int k = threadIdx.x; k < m; k += kSelThreads) cs[k] = Cs[lo + k];
        __syncthreads();
        const uint64_t Q = s_Q;
        const StrataPoint U = make_strata(Q, (uint32_t)(Tw - Q * (uint64_t)n), n, mode, k0, k1, chi,
                                          slice0 + (uint32_t)s);
        const int jj0 = threadIdx.x * kSelPer;
        if (jj0 < cnt) {
            if (span <= kSelStage) {        // the whole range staged: 32-bit indices into it
                const auto v = [&](int i) { return cs[i]; };
                select_run(v, 0, (int)span - 1, U, (uint32_t)j0, jj0, cnt, sp);
            } else {
                const auto v = [&](int64_t p) { return p - lo < m ? cs[p - lo] : Cs[p]; };
                select_run(v, lo, hi, U, (uint32_t)j0, jj0, cnt, sp);
            }
        }
    } else {
        for (int jj = threadIdx.x; jj < cnt; jj += kSelThreads) sp[sel_pad(jj)] = (uint32_t)jj;
    }
    __syncthreads();
    // output jj = threadIdx.x + k kSelThreads of this CTA
    // particles relative to lo (below 2^32: p < n <= 2^32 - 1), outputs at
    // j0 + threadIdx.x + k kSelThreads
    const int valid = max(0, min(kSelPer, (cnt - (int)threadIdx.x + kSelThreads - 1) / kSelThreads));
    uint32_t pr[kSelPer];
#pragma unroll
    for (int k = 0; k < kSelPer; ++k) pr[k] = k < valid ? sp[sel_pad(threadIdx.x + k * kSelThreads)] : 0u;
    const int64_t si = broadcast ? 0 : s;   // the input slice (one shared by all with broadcast)
    const int64_t jt = j0 + threadIdx.x;
    if (idx) {
        uint32_t* o = idx + (int64_t)s * n + jt;
#pragma unroll
        for (int k = 0; k < kSelPer; ++k)
            if (k < valid) o[k * kSelThreads] = (uint32_t)lo + pr[k];
    }
    if (x_out) gather_rows(x_in + si * n + lo, x_out + (int64_t)s * n + jt, pr, valid);
    if (y_out)
        for (int c = 0; c < d; ++c)
            gather_rows(y_in + (si * d + c) * n + lo, y_out + ((int64_t)s * d + c) * n + jt, pr, valid);
}

// ---------------------------------------------------------------------------
// Restriction with weights: fixed-point bin sums, then the CDF
// ---------------------------------------------------------------------------

// Each bin's 64-bit sum is kept as two 32-bit words in shared memory: the low
// word takes the low halves (its wrap-arounds, seen from the value returned
// by the atomic, go into the high word with the high halves), so the sum is
// exact and independent of the order of the additions.
template <typename T>
__global__ void __launch_bounds__(kCondThreads)
restrict_weighted_kernel(const T* __restrict__ x, int64_t in_stride, const double* __restrict__ w, int64_t n,
                         GridDev g, float lo_f, float inv_h_f, unsigned long long* __restrict__ hist_g,
                         int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int I = g.bins;
    uint32_t* hl = reinterpret_cast<uint32_t*>(smem);
    uint32_t* hh = hl + I;
    float* thr = reinterpret_cast<float*>(hh + I);
    const int s = blockIdx.y;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        hl[i] = 0u;
        hh[i] = 0u;
    }
    if (sizeof(T) == 4) build_thresholds(g, thr);
    __syncthreads();
    const BinF32 bf = make_bin_f32(thr, I, lo_f, inv_h_f);
    const T* xs = x + (int64_t)s * in_stride;
    const double* ws = w + (int64_t)s * n;
    const int64_t b = (int64_t)blockIdx.x * per_block, e = min(n, b + per_block);
    const int Tn = blockDim.x;
    // four particles per thread and round: eight loads in flight
    for (int64_t p = b + threadIdx.x; p < e; p += 4 * Tn) {
        T xv[4];
        double wv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool in = p + k * Tn < e;
            xv[k] = in ? __ldcs(xs + p + k * Tn) : T(0);
            wv[k] = in ? __ldcs(ws + p + k * Tn) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t v = weight_fixed(wv[k]);
            if (v) {
                const int i = sizeof(T) == 4 ? bin_fast_f32(bf, thr, (float)xv[k]) : bin_of_f64(g, (double)xv[k]);
                const uint32_t vl = (uint32_t)v;
                const uint32_t old = atomicAdd(&hl[i], vl);
                const uint32_t up = (uint32_t)(v >> 32) + ((uint32_t)(old + vl) < old ? 1u : 0u);
                if (up) atomicAdd(&hh[i], up);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const unsigned long long v = ((unsigned long long)hh[i] << 32) | hl[i];
        if (v) atomicAdd(&hist_g[(size_t)s * I + i], v);
    }
}

// C_0 = 0, C_i = (fixed weight in bins < i) / (total), C_I = 1; with no weight
// the uniform CDF i / I.  One CTA per slice, integer prefix sums (exact).
__global__ void __launch_bounds__(256)
weighted_cdf_kernel(const unsigned long long* __restrict__ hist_g, int I, double* __restrict__ cdf)
{
    __shared__ unsigned long long wtot[8];
    __shared__ unsigned long long s_total;
    const int s = blockIdx.x;
    const unsigned long long* h = hist_g + (size_t)s * I;
    double* C = cdf + (size_t)s * (I + 1);
    const int T = blockDim.x;
    const int chunk = (I + T - 1) / T;
    const int b0 = threadIdx.x * chunk, e0 = min(I, b0 + chunk);
    unsigned long long loc = 0;
    for (int i = b0; i < e0; ++i) loc += h[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < T / 32; ++k) t += wtot[k];
        s_total = t;
    }
    __syncthreads();
    const unsigned long long total = s_total;
    unsigned long long run = incl - loc;
    for (int k = 0; k < warp; ++k) run += wtot[k];
    const double dt = __ull2double_rn(total);
    for (int i = b0; i < e0; ++i) {
        run += h[i];
        C[i + 1] = total ? __ddiv_rn(__ull2double_rn(run), dt) : __ddiv_rn((double)(i + 1), (double)I);
    }
    if (threadIdx.x == 0) {
        C[0] = 0.0;
        C[I] = 1.0;
    }
}

}  // namespace pr

namespace pr {

static inline size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
static inline size_t al16c(size_t v) { return (v + 15) & ~(size_t)15; }

// Elements per CTA: one wave of CTAs (per_sm per SM) over all slices, at
// least min_per elements each.
static int64_t cond_range(int64_t n, int n_slices, int64_t min_per, int per_sm)
{
    const int64_t slots = (int64_t)num_sms() * per_sm;
    int64_t bps = std::max<int64_t>(1, slots / n_slices);
    bps = std::min<int64_t>(bps, std::max<int64_t>(1, n / min_per));
    return (n + bps - 1) / bps;
}

template <typename K>
static cudaError_t cond_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

struct ResampleLayout {
    int64_t nblk, nsel;
    size_t c_bytes, b_bytes, t_bytes, s_bytes;
};

static ResampleLayout resample_layout(int64_t n, int32_t n_slices)
{
    ResampleLayout l;
    l.nblk = (n + kScanBlock - 1) / kScanBlock;
    l.nsel = (n + kSelOut - 1) / kSelOut;
    l.c_bytes = al256((size_t)n_slices * n * sizeof(uint64_t));
    l.b_bytes = al256((size_t)n_slices * l.nblk * sizeof(uint64_t));
    l.t_bytes = al256((size_t)n_slices * sizeof(uint64_t));
    l.s_bytes = al256((size_t)n_slices * l.nsel * 2 * sizeof(int64_t));
    return l;
}

}  // namespace pr

using namespace pr;

extern "C" pr_status pr_reweight(pr_precision precision, const void* x_prior, int32_t broadcast_input,
                                 const double* w_prior, int64_t n, int32_t n_slices, const pr_grid* grid,
                                 const double* cdf_prior, const double* cdf_target, double* w_out, void* stream)
{
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(x_prior, elem_bytes(precision)) || !elem_aligned(w_prior, 8) || !elem_aligned(cdf_prior, 8) ||
        !elem_aligned(cdf_target, 8) || !elem_aligned(w_out, 8))
        return PR_ERR_INVALID_ARG;
    if (!x_prior || !cdf_prior || !cdf_target || !w_out || !grid_ok(grid)) return PR_ERR_INVALID_ARG;
    if (n < 1 || n_slices < 1 || n_slices > 65535) return PR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GridDev g = make_grid(*grid);
    const int I = grid->bins;
    const float lo_f = (float)grid->x_lo, inv_h_f = (float)(1.0 / g.h);
    const size_t smem = al16c(reweight_smem_bytes(I)) + al16c((size_t)(I + 1) * 4);
    const int64_t per = cond_range(n, n_slices, 16384, 2);
    dim3 gr((unsigned)((n + per - 1) / per), (unsigned)n_slices);
    const int64_t stride = broadcast_input ? 0 : n;
    if (precision == PR_F32) {
        PR_TRY_CUDA(cond_smem(reweight_kernel<float>, smem));
        reweight_kernel<float><<<gr, kCondThreads, smem, st>>>(static_cast<const float*>(x_prior), stride, w_prior, n, g,
                                                               lo_f, inv_h_f, cdf_prior, cdf_target, w_out, per);
    } else {
        PR_TRY_CUDA(cond_smem(reweight_kernel<double>, smem));
        reweight_kernel<double><<<gr, kCondThreads, smem, st>>>(static_cast<const double*>(x_prior), stride, w_prior, n,
                                                                g, lo_f, inv_h_f, cdf_prior, cdf_target, w_out, per);
    }
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" size_t pr_resample_workspace(int64_t n, int32_t n_slices)
{
    if (n < 1 || n_slices < 1) return 0;
    const ResampleLayout l = resample_layout(n, n_slices);
    return l.c_bytes + l.b_bytes + l.t_bytes + l.s_bytes;
}

extern "C" pr_status pr_resample(pr_precision precision, int32_t fast_dim, const void* x_in, const void* y_in,
                                 int32_t broadcast_input, const double* w, int64_t n, int32_t n_slices,
                                 int32_t slice_begin, pr_resample_mode mode, const pr_rng* rng, uint32_t* index_out,
                                 void* x_out, void* y_out, void* workspace, size_t workspace_bytes, void* stream)
{
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(x_in, elem_bytes(precision)) || !elem_aligned(y_in, elem_bytes(precision)) ||
        !elem_aligned(w, 8) || !elem_aligned(index_out, 4) || !elem_aligned(x_out, elem_bytes(precision)) ||
        !elem_aligned(y_out, elem_bytes(precision)))
        return PR_ERR_INVALID_ARG;
    if (mode != PR_RESAMPLE_STRATIFIED && mode != PR_RESAMPLE_DETERMINISTIC) return PR_ERR_INVALID_ARG;
    if (!w || !rng || !workspace || n < 1 || n > 0xFFFFFFFFll || n_slices < 1 || n_slices > 65535) return PR_ERR_INVALID_ARG;
    if (slice_begin < 0 || rng->problem_id >= (1u << 24)) return PR_ERR_INVALID_ARG;
    if ((x_out && !x_in) || (y_out && !y_in) || (y_out && (fast_dim < 1 || fast_dim > PR_MAX_FAST_DIM)))
        return PR_ERR_INVALID_ARG;
    if ((x_out && x_out == x_in) || (y_out && y_out == y_in)) return PR_ERR_INVALID_ARG;   // a gather, not in place
    if (workspace_bytes < pr_resample_workspace(n, n_slices) || ((uintptr_t)workspace & 255)) return PR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ResampleLayout l = resample_layout(n, n_slices);
    char* base = static_cast<char*>(workspace);
    uint64_t* C = reinterpret_cast<uint64_t*>(base);
    uint64_t* bsum = reinterpret_cast<uint64_t*>(base + l.c_bytes);
    uint64_t* total = reinterpret_cast<uint64_t*>(base + l.c_bytes + l.b_bytes);
    int64_t* bounds = reinterpret_cast<int64_t*>(base + l.c_bytes + l.b_bytes + l.t_bytes);
    dim3 gb((unsigned)((l.nblk + kScanWarps - 1) / kScanWarps), (unsigned)n_slices);
    fixed_blocksum_kernel<<<gb, kScanThreads, 0, st>>>(w, n, l.nblk, bsum);
    PR_CHECK_LAUNCH();
    scan_blocks_kernel<<<n_slices, 1024, 0, st>>>(bsum, l.nblk, total);
    PR_CHECK_LAUNCH();
    scan_within_kernel<<<gb, kScanThreads, 0, st>>>(w, C, n, l.nblk, bsum);
    PR_CHECK_LAUNCH();
    const uint32_t k0 = (uint32_t)(rng->seed & 0xFFFFFFFFull), k1 = (uint32_t)(rng->seed >> 32);
    const uint32_t chi = rng->problem_id << 8;
    dim3 gbd((unsigned)((2 * l.nsel + 255) / 256), (unsigned)n_slices);
    select_bounds_kernel<<<gbd, 256, 0, st>>>(C, bsum, total, n, l.nblk, l.nsel, (int)mode, k0, k1, chi,
                                              (uint32_t)slice_begin, bounds);
    PR_CHECK_LAUNCH();
    dim3 gs((unsigned)l.nsel, (unsigned)n_slices);
    const int d = y_out ? fast_dim : 0;
    if (precision == PR_F32)
        select_gather_kernel<float><<<gs, kSelThreads, 0, st>>>(C, total, bounds, n, (int)mode, k0, k1, chi, (uint32_t)slice_begin,
                                                        static_cast<const float*>(x_in), static_cast<const float*>(y_in),
                                                        broadcast_input ? 1 : 0, d, index_out,
                                                        static_cast<float*>(x_out), static_cast<float*>(y_out));
    else
        select_gather_kernel<double><<<gs, kSelThreads, 0, st>>>(C, total, bounds, n, (int)mode, k0, k1, chi, (uint32_t)slice_begin,
                                                         static_cast<const double*>(x_in), static_cast<const double*>(y_in),
                                                         broadcast_input ? 1 : 0, d, index_out,
                                                         static_cast<double*>(x_out), static_cast<double*>(y_out));
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" size_t pr_restrict_weighted_workspace(int32_t n_slices, int32_t bins)
{
    if (n_slices < 1 || bins < 1) return 0;
    return al256((size_t)n_slices * bins * sizeof(unsigned long long));
}

extern "C" pr_status pr_restrict_weighted(pr_precision precision, const void* x, int32_t broadcast_input,
                                          const double* w, int64_t n, int32_t n_slices, const pr_grid* grid,
                                          double* cdf, void* workspace, size_t workspace_bytes, void* stream)
{
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(x, elem_bytes(precision)) || !elem_aligned(w, 8) || !elem_aligned(cdf, 8))
        return PR_ERR_INVALID_ARG;
    if (!x || !w || !cdf || !workspace || !grid_ok(grid) || n < 1 || n_slices < 1 || n_slices > 65535)
        return PR_ERR_INVALID_ARG;
    if (workspace_bytes < pr_restrict_weighted_workspace(n_slices, grid->bins) || ((uintptr_t)workspace & 7))
        return PR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int I = grid->bins;
    auto* hist = static_cast<unsigned long long*>(workspace);
    PR_TRY_CUDA(cudaMemsetAsync(hist, 0, (size_t)n_slices * I * sizeof(unsigned long long), st));
    const GridDev g = make_grid(*grid);
    const float lo_f = (float)grid->x_lo, inv_h_f = (float)(1.0 / g.h);
    const size_t smem = al16c((size_t)I * 8) + al16c((size_t)(I + 1) * 4);
    const int64_t per = cond_range(n, n_slices, 16384, 2);
    dim3 gr((unsigned)((n + per - 1) / per), (unsigned)n_slices);
    const int64_t stride = broadcast_input ? 0 : n;
    if (precision == PR_F32) {
        PR_TRY_CUDA(cond_smem(restrict_weighted_kernel<float>, smem));
        restrict_weighted_kernel<float><<<gr, kCondThreads, smem, st>>>(static_cast<const float*>(x), stride, w, n, g,
                                                                        lo_f, inv_h_f, hist, per);
    } else {
        PR_TRY_CUDA(cond_smem(restrict_weighted_kernel<double>, smem));
        restrict_weighted_kernel<double><<<gr, kCondThreads, smem, st>>>(static_cast<const double*>(x), stride, w, n,
                                                                         g, lo_f, inv_h_f, hist, per);
    }
    PR_CHECK_LAUNCH();
    weighted_cdf_kernel<<<n_slices, 256, 0, st>>>(hist, I, cdf);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

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
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "pr_common.cuh"

namespace pr {

constexpr int kCondThreads = 512;

// Fixed point of a probability weight (0 for w <= 0 or NaN).
__device__ __forceinline__ uint64_t weight_fixed(double w)
{
    if (!(w > 0.0)) return 0ull;
    return __double2ull_rn(__dmul_rn(w, 2305843009213693952.0));   // w 2^61, exact scaling
}

// r[i] = rho'_i / rhobar_i for one prior/target pair, by the whole block.
// Bin b with prior mass collects its own target mass, then that of the
// unsupported bins between it and the previous supported bin (left to right),
// then that of those up to the next supported bin, each halved where both
// sides have a supported bin: the additions of the left-to-right visit of the
// unsupported bins, in the same order.
__device__ void reweight_factors_block(int I, const double* __restrict__ Cp, const double* __restrict__ Ct,
                                       double* r)
{
    for (int b = threadIdx.x; b < I; b += blockDim.x) {
        const double rb = __dsub_rn(Cp[b + 1], Cp[b]);
        if (!(rb > 0.0)) {
            r[b] = 0.0;
            continue;
        }
        double rn = __dsub_rn(Ct[b + 1], Ct[b]);
        // gap on the left: bins L+1 .. b-1 without prior mass
        int L = b - 1;
        while (L >= 0 && !(__dsub_rn(Cp[L + 1], Cp[L]) > 0.0)) --L;
        for (int i = L + 1; i < b; ++i) {
            const double rt = __dsub_rn(Ct[i + 1], Ct[i]);
            if (rt > 0.0) rn = __dadd_rn(rn, L >= 0 ? __dmul_rn(0.5, rt) : rt);
        }
        // gap on the right: bins b+1 .. R-1
        int R = b + 1;
        while (R < I && !(__dsub_rn(Cp[R + 1], Cp[R]) > 0.0)) ++R;
        for (int i = b + 1; i < R; ++i) {
            const double rt = __dsub_rn(Ct[i + 1], Ct[i]);
            if (rt > 0.0) rn = __dadd_rn(rn, R < I ? __dmul_rn(0.5, rt) : rt);
        }
        r[b] = __ddiv_rn(rn, rb);
    }
}

// W^p = Wbar^p r_{bin(Xbar^p)}; one CTA per (range, slice), the factors built
// per CTA in shared memory.
template <typename T>
__global__ void __launch_bounds__(kCondThreads)
reweight_kernel(const T* __restrict__ x, int64_t in_stride, const double* __restrict__ wbar, int64_t n,
                GridDev g, float lo_f, float inv_h_f, const double* __restrict__ cp, const double* __restrict__ ct,
                double* __restrict__ w, int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int I = g.bins;
    double* r = reinterpret_cast<double*>(smem);
    float* thr = reinterpret_cast<float*>(r + I);
    const int s = blockIdx.y;
    reweight_factors_block(I, cp + (size_t)s * (I + 1), ct + (size_t)s * (I + 1), r);
    if (sizeof(T) == 4) build_thresholds(g, thr);
    __syncthreads();
    const BinF32 bf = make_bin_f32(thr, I, lo_f, inv_h_f);
    const double w0 = __ddiv_rn(1.0, (double)n);
    const T* xs = x + (int64_t)s * in_stride;
    const double* wbs = wbar ? wbar + (int64_t)s * in_stride : nullptr;
    double* ws = w + (int64_t)s * n;
    const int64_t b = (int64_t)blockIdx.x * per_block, e = min(n, b + per_block);
    for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
        const int i = sizeof(T) == 4 ? bin_fast_f32(bf, thr, (float)xs[p]) : bin_of_f64(g, (double)xs[p]);
        ws[p] = __dmul_rn(wbs ? wbs[p] : w0, r[i]);
    }
}

// ---------------------------------------------------------------------------
// Resampling: cumulative fixed weights C_p = sum_{q <= p} round(W^q 2^61)
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;                              // elements per thread
constexpr int kScanBlock = kScanThreads * kScanPer;      // elements per block

// Fixed weights into C (per element) and their sum per block.
__global__ void __launch_bounds__(kScanThreads)
fixed_blocksum_kernel(const double* __restrict__ w, int64_t n, int64_t nblk, uint64_t* __restrict__ C,
                      uint64_t* __restrict__ bsum)
{
    __shared__ uint64_t wsum[kScanThreads / 32];
    const int s = blockIdx.y;
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
    const double* ws = w + (int64_t)s * n;
    uint64_t* Cs = C + (int64_t)s * n;
    uint64_t loc = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int64_t p = base + k;
        if (p < n) {
            const uint64_t v = weight_fixed(ws[p]);
            Cs[p] = v;
            loc += v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_down_sync(0xffffffffu, loc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int k = 0; k < kScanThreads / 32; ++k) t += wsum[k];
        bsum[(int64_t)s * nblk + blockIdx.x] = t;
    }
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

// Inclusive scan within each block plus the block's offset: C_p.
__global__ void __launch_bounds__(kScanThreads)
scan_within_kernel(uint64_t* __restrict__ C, int64_t n, int64_t nblk, const uint64_t* __restrict__ boff)
{
    __shared__ uint64_t wtot[kScanThreads / 32];
    const int s = blockIdx.y;
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanPer;
    uint64_t* Cs = C + (int64_t)s * n;
    uint64_t v[kScanPer];
    uint64_t loc = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int64_t p = base + k;
        v[k] = p < n ? Cs[p] : 0ull;
        loc += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    uint64_t run = boff[(int64_t)s * nblk + blockIdx.x] + incl - loc;
    for (int k = 0; k < warp; ++k) run += wtot[k];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int64_t p = base + k;
        run += v[k];
        if (p < n) Cs[p] = run;
    }
}

// Output j of slice s takes the particle p with C_{p-1} <= U_j < C_p and
// copies its state.  U_j = floor(T (j 2^24 + a_j) / (n 2^24)) < T.
template <typename T>
__global__ void __launch_bounds__(256)
select_gather_kernel(const uint64_t* __restrict__ C, const uint64_t* __restrict__ total, int64_t n, int mode,
                     uint32_t k0, uint32_t k1, uint32_t chi, uint32_t slice0, const T* __restrict__ x_in,
                     const T* __restrict__ y_in, int broadcast, int d, uint32_t* __restrict__ idx,
                     T* __restrict__ x_out, T* __restrict__ y_out)
{
    const int s = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint64_t Tw = total[s];
    int64_t p = j;
    if (Tw > 0) {
        uint64_t a = 1ull << 23;
        if (mode == PR_RESAMPLE_STRATIFIED) {
            const uint4 wd = philox4x32_10(make_uint4((uint32_t)j, 0xFFFFFFFFu, slice0 + (uint32_t)s, chi | 0xFEu),
                                           k0, k1);
            a = 2ull * (uint64_t)(wd.x >> 9) + 1ull;
        }
        const unsigned __int128 num = (unsigned __int128)Tw * (((uint64_t)j << 24) + a);
        const uint64_t U = (uint64_t)(num / ((unsigned __int128)n << 24));
        const uint64_t* Cs = C + (int64_t)s * n;
        int64_t lo = 0, hi = n - 1;   // smallest p with C_p > U (C_{n-1} = T > U)
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (Cs[mid] > U) hi = mid; else lo = mid + 1;
        }
        p = lo;
    }
    const int64_t si = broadcast ? 0 : s;   // the input slice (one shared by all with broadcast)
    if (idx) idx[(int64_t)s * n + j] = (uint32_t)p;
    if (x_out) x_out[(int64_t)s * n + j] = x_in[si * n + p];
    if (y_out)
        for (int c = 0; c < d; ++c) y_out[((int64_t)s * d + c) * n + j] = y_in[(si * d + c) * n + p];
}

// ---------------------------------------------------------------------------
// Restriction with weights: fixed-point bin sums, then the CDF
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kCondThreads)
restrict_weighted_kernel(const T* __restrict__ x, int64_t in_stride, const double* __restrict__ w, int64_t n,
                         GridDev g, float lo_f, float inv_h_f, unsigned long long* __restrict__ hist_g,
                         int64_t per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int I = g.bins;
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(smem);
    float* thr = reinterpret_cast<float*>(hist + I);
    const int s = blockIdx.y;
    for (int i = threadIdx.x; i < I; i += blockDim.x) hist[i] = 0ull;
    if (sizeof(T) == 4) build_thresholds(g, thr);
    __syncthreads();
    const BinF32 bf = make_bin_f32(thr, I, lo_f, inv_h_f);
    const T* xs = x + (int64_t)s * in_stride;
    const double* ws = w + (int64_t)s * n;
    const int64_t b = (int64_t)blockIdx.x * per_block, e = min(n, b + per_block);
    for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
        const int i = sizeof(T) == 4 ? bin_fast_f32(bf, thr, (float)xs[p]) : bin_of_f64(g, (double)xs[p]);
        const uint64_t v = weight_fixed(ws[p]);
        if (v) atomicAdd(&hist[i], (unsigned long long)v);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < I; i += blockDim.x)
        if (hist[i]) atomicAdd(&hist_g[(size_t)s * I + i], hist[i]);
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
    int64_t nblk;
    size_t c_bytes, b_bytes, t_bytes;
};

static ResampleLayout resample_layout(int64_t n, int32_t n_slices)
{
    ResampleLayout l;
    l.nblk = (n + kScanBlock - 1) / kScanBlock;
    l.c_bytes = al256((size_t)n_slices * n * sizeof(uint64_t));
    l.b_bytes = al256((size_t)n_slices * l.nblk * sizeof(uint64_t));
    l.t_bytes = al256((size_t)n_slices * sizeof(uint64_t));
    return l;
}

}  // namespace pr

using namespace pr;

extern "C" pr_status pr_reweight(pr_precision precision, const void* x_prior, int32_t broadcast_input,
                                 const double* w_prior, int64_t n, int32_t n_slices, const pr_grid* grid,
                                 const double* cdf_prior, const double* cdf_target, double* w_out, void* stream)
{
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
    if (!x_prior || !cdf_prior || !cdf_target || !w_out || !grid_ok(grid)) return PR_ERR_INVALID_ARG;
    if (n < 1 || n_slices < 1 || n_slices > 65535) return PR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GridDev g = make_grid(*grid);
    const int I = grid->bins;
    const float lo_f = (float)grid->x_lo, inv_h_f = (float)(1.0 / g.h);
    const size_t smem = al16c((size_t)I * 8) + al16c((size_t)(I + 1) * 4);
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
    return l.c_bytes + l.b_bytes + l.t_bytes;
}

extern "C" pr_status pr_resample(pr_precision precision, int32_t fast_dim, const void* x_in, const void* y_in,
                                 int32_t broadcast_input, const double* w, int64_t n, int32_t n_slices,
                                 int32_t slice_begin, pr_resample_mode mode, const pr_rng* rng, uint32_t* index_out,
                                 void* x_out, void* y_out, void* workspace, size_t workspace_bytes, void* stream)
{
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
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
    dim3 gb((unsigned)l.nblk, (unsigned)n_slices);
    fixed_blocksum_kernel<<<gb, kScanThreads, 0, st>>>(w, n, l.nblk, C, bsum);
    PR_CHECK_LAUNCH();
    scan_blocks_kernel<<<n_slices, 1024, 0, st>>>(bsum, l.nblk, total);
    PR_CHECK_LAUNCH();
    scan_within_kernel<<<gb, kScanThreads, 0, st>>>(C, n, l.nblk, bsum);
    PR_CHECK_LAUNCH();
    const uint32_t k0 = (uint32_t)(rng->seed & 0xFFFFFFFFull), k1 = (uint32_t)(rng->seed >> 32);
    const uint32_t chi = rng->problem_id << 8;
    dim3 gs((unsigned)((n + 255) / 256), (unsigned)n_slices);
    const int d = y_out ? fast_dim : 0;
    if (precision == PR_F32)
        select_gather_kernel<float><<<gs, 256, 0, st>>>(C, total, n, (int)mode, k0, k1, chi, (uint32_t)slice_begin,
                                                        static_cast<const float*>(x_in), static_cast<const float*>(y_in),
                                                        broadcast_input ? 1 : 0, d, index_out,
                                                        static_cast<float*>(x_out), static_cast<float*>(y_out));
    else
        select_gather_kernel<double><<<gs, 256, 0, st>>>(C, total, n, (int)mode, k0, k1, chi, (uint32_t)slice_begin,
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

// estimator.cu -- the Monte Carlo estimator of Section 2.1.3 (Eq. MCestimator),
// M_hat = sum_p M(X^p, Y^p) W^p, for the power observables M = v^q of one
// coordinate v of the ensemble (the slow variable x, or one fast component),
// q = 1..max_order, with the weights W^p given or uniform (1/n).
//
// Each thread accumulates its particles in binary64 registers; a CTA reduces
// its threads in a fixed tree (warp shuffles, then the warps in order) to one
// partial per order, and a second kernel adds a slice's partials in block
// order.  The grid depends only on n and the slice count, so a call returns
// the same bits every time on any device.  Each order's term enters its sum
// through one fused multiply-add (W v^(q-1) times v, added with one rounding),
// and the running power takes one multiply: per particle 2 max_order - 1
// binary64 operations with weights, 2 max_order - 2 without (the first order
// adds v itself).  On GB300's narrow FP64 pipe that, not HBM,
// bounds the pass; it is meant for observables at the end of a run, not for
// every step.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pr_common.cuh"

namespace pr {

constexpr int kMomThreads = 256;
constexpr int kMomMaxOrder = 4;
constexpr int kMomUnroll = 8;              // loads in flight per thread
constexpr int64_t kMomPerBlock = 4096;     // particles per CTA at least (then fewer CTAs)
constexpr int64_t kMomMaxBlocks = 2432;    // CTAs over all slices at most (16 per SM of 152)

static int64_t moments_blocks(int64_t n, int32_t n_slices)
{
    const int64_t cap = std::max<int64_t>(1, kMomMaxBlocks / n_slices);
    return std::min<int64_t>(cap, std::max<int64_t>(1, (n + kMomPerBlock - 1) / kMomPerBlock));
}

template <typename T, int Q, bool W>
__global__ void __launch_bounds__(kMomThreads)
moments_kernel(const T* __restrict__ v, int64_t stride, const double* __restrict__ w, int64_t n, int64_t per_block,
               double* __restrict__ partial)
{
    const int s = blockIdx.y;
    const T* vs = v + (int64_t)s * stride;
    const double* ws = W ? w + (int64_t)s * n : nullptr;
    const int64_t b = (int64_t)blockIdx.x * per_block, e = min(n, b + per_block);
    double acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = 0.0;
    // kMomUnroll particles per thread and round, their loads issued first
    for (int64_t p0 = b + threadIdx.x; p0 < e; p0 += kMomUnroll * kMomThreads) {
        T xv[kMomUnroll];
        double wv[kMomUnroll];
#pragma unroll
        for (int k = 0; k < kMomUnroll; ++k) {
            const int64_t p = p0 + (int64_t)k * kMomThreads;
            xv[k] = p < e ? vs[p] : T(0);
            wv[k] = W ? (p < e ? ws[p] : 0.0) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < kMomUnroll; ++k) {
            if (p0 + (int64_t)k * kMomThreads >= e) break;
            const double x = widen(xv[k]);
            double t;                     // W x^q before order q + 1
            int q0;
            if (W) {
                t = wv[k];
                q0 = 0;
            } else {
                acc[0] += x;
                t = x;
                q0 = 1;
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if (q < q0) continue;
                acc[q] = fma(t, x, acc[q]);
                if (q + 1 < Q) t *= x;
            }
        }
    }
    __shared__ double red[Q][kMomThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        double a = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[q][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < Q) {
        double t = 0.0;
        for (int k = 0; k < kMomThreads / 32; ++k) t += red[threadIdx.x][k];
        partial[((int64_t)s * gridDim.x + blockIdx.x) * Q + threadIdx.x] = t;
    }
}

// out[s][q] = sum of slice s's partials in block order (divided by n without weights)
__global__ void moments_finish_kernel(const double* __restrict__ partial, int64_t nblk, int32_t n_slices, int Q,
                                      int64_t n, int weighted, double* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_slices * Q) return;
    const int64_t s = i / Q, q = i - s * Q;
    double t = 0.0;
    for (int64_t b = 0; b < nblk; ++b) t += partial[(s * nblk + b) * Q + q];
    out[i] = weighted ? t : t / (double)n;
}

template <typename T, int Q>
static void launch_moments(const void* v, int64_t stride, const double* w, int64_t n, int32_t n_slices, int64_t nblk,
                           double* partial, cudaStream_t st)
{
    const int64_t per = (n + nblk - 1) / nblk;
    const dim3 grid((unsigned)nblk, (unsigned)n_slices);
    if (w)
        moments_kernel<T, Q, true><<<grid, kMomThreads, 0, st>>>(static_cast<const T*>(v), stride, w, n, per, partial);
    else
        moments_kernel<T, Q, false><<<grid, kMomThreads, 0, st>>>(static_cast<const T*>(v), stride, w, n, per, partial);
}

template <typename T>
static void launch_moments_q(int Q, const void* v, int64_t stride, const double* w, int64_t n, int32_t n_slices,
                             int64_t nblk, double* partial, cudaStream_t st)
{
    switch (Q) {
    case 1: launch_moments<T, 1>(v, stride, w, n, n_slices, nblk, partial, st); break;
    case 2: launch_moments<T, 2>(v, stride, w, n, n_slices, nblk, partial, st); break;
    case 3: launch_moments<T, 3>(v, stride, w, n, n_slices, nblk, partial, st); break;
    default: launch_moments<T, 4>(v, stride, w, n, n_slices, nblk, partial, st); break;
    }
}

}  // namespace pr

using namespace pr;

extern "C" size_t pr_moments_workspace(int64_t n, int32_t n_slices, int32_t max_order)
{
    if (n < 1 || n_slices < 1 || n_slices > 65535 || max_order < 1 || max_order > kMomMaxOrder) return 0;
    return (size_t)(moments_blocks(n, n_slices) * n_slices * max_order) * sizeof(double);
}

extern "C" pr_status pr_moments(pr_precision precision, const void* v, int64_t slice_stride, const double* w,
                                int64_t n, int32_t n_slices, int32_t max_order, double* out, void* workspace,
                                size_t workspace_bytes, void* stream)
{
    if (precision != PR_F32 && precision != PR_F64) return PR_ERR_INVALID_ARG;
    if (!v || !out || !workspace || n < 1 || n_slices < 1 || n_slices > 65535) return PR_ERR_INVALID_ARG;
    if (max_order < 1 || max_order > kMomMaxOrder || slice_stride < 0 || (n_slices > 1 && slice_stride < n))
        return PR_ERR_INVALID_ARG;
    if (!elem_aligned(workspace, 8) || !elem_aligned(v, elem_bytes(precision)) || !elem_aligned(w, 8) ||
        !elem_aligned(out, 8))
        return PR_ERR_INVALID_ARG;
    if (workspace_bytes < pr_moments_workspace(n, n_slices, max_order)) return PR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nblk = moments_blocks(n, n_slices);
    double* partial = static_cast<double*>(workspace);
    if (precision == PR_F32)
        launch_moments_q<float>(max_order, v, slice_stride, w, n, n_slices, nblk, partial, st);
    else
        launch_moments_q<double>(max_order, v, slice_stride, w, n, n_slices, nblk, partial, st);
    PR_CHECK_LAUNCH();
    const int64_t tot = (int64_t)n_slices * max_order;
    moments_finish_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(partial, nblk, n_slices, max_order, n,
                                                                        w ? 1 : 0, out);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

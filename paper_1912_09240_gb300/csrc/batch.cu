// batch.cu -- many independent micro-macro parareal problems served together.
//
// A plan holds every problem's ensembles and macroscopic states in packed
// device buffers.  One parareal iteration of the whole batch is four launches:
//   1. a persistent fine kernel: CTAs pull work items (problem, slice,
//      particle range) from an atomic counter, largest first, and run the
//      same fused matching / Euler-Maruyama / restriction code as
//      pr_fine_propagate (fine_dev.cuh), bit for bit;
//   2. counts -> CDFs for every (problem, slice);
//   3. the coarse step on every start state (each problem its own P);
//   4. the serial update of Section 3.2.3, one CTA per problem.
// From the second iteration on, an iteration is replayed as a CUDA graph
// (one per parity of the ping-pong buffers).  Items are sized by an amount of
// work (particle-steps) so that problems with 10^4x different costs balance;
// pr_batch_tune picks the particles per thread and the item size by timing.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "coarse_dev.cuh"
#include "fine_dev.cuh"
#include "match.cuh"
#include "pr_common.cuh"

namespace pr {

struct BatchProblemDev {
    float lam, ddt, rel, sxk, syk;
    uint32_t k0, k1, chi;
    int32_t kind, steps, bins, K;
    GridDev g;
    float lo_f, inv_h_f;
    int64_t n;
    int64_t x0_off;   // into [sum n]            (X_0)
    int64_t x_off;    // into [sum K n]          (slice-major within the problem)
    int64_t h_off;    // into [sum K I]          (counts)
    int64_t c_off;    // into [sum K (I+1)]      (per-slice CDFs)
    int64_t r_off;    // into [sum (K+1)(I+1)]   (rho)
    int64_t c0_off;   // into [sum (I+1)]        (R X_0)
    const double* P;
};

struct BatchItemDev {
    int32_t problem, slice;
    int64_t begin, end;
};

struct BatchRowDev {   // one (problem, slice)
    int32_t problem, slice;
};

struct BatchFineArgs {
    const BatchProblemDev* probs;
    const BatchItemDev* items;
    int n_items;
    unsigned int* counter;
    const float* x0;
    const float* y0;
    const float* xa;
    const float* ya;
    float* xb;
    float* yb;
    const double* cdf0;
    const double* fprev;
    const double* rho;
    uint32_t* counts_s;
    uint32_t* counts_e;
    int first;
    int max_bins;
    int steps_div;   // > 1: every item runs ceil(steps / steps_div) steps (timing trials only)
};

__host__ __device__ inline size_t batch_fine_smem(int max_bins)
{
    const size_t a = ((size_t)(max_bins + 1) * 4 + 15) & ~(size_t)15;
    const size_t b = ((size_t)max_bins * 4 + 15) & ~(size_t)15;
    return a + 2 * b + match_smem_bytes_f32(max_bins);
}

template <int PPT>
__global__ void __launch_bounds__(256)
batch_fine_kernel(BatchFineArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    const int MB = a.max_bins;
    const size_t off_h = ((size_t)(MB + 1) * 4 + 15) & ~(size_t)15;
    const size_t hb = ((size_t)MB * 4 + 15) & ~(size_t)15;
    float* thr = reinterpret_cast<float*>(smem);
    uint32_t* hs = reinterpret_cast<uint32_t*>(smem + off_h);
    uint32_t* he = reinterpret_cast<uint32_t*>(smem + off_h + hb);
    unsigned char* mbase = smem + off_h + 2 * hb;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.n_items) break;
        const BatchItemDev it = a.items[item];
        const BatchProblemDev& P = a.probs[it.problem];
        const int s = it.slice, bins = P.bins;
        const int64_t n = P.n;
        build_thresholds(P.g, thr);
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            hs[i] = 0u;
            he[i] = 0u;
        }
        const bool do_match = s >= 1;
        const float* xin;
        const float* yin;
        const double* prior = nullptr;
        if (s == 0 || a.first) {
            xin = a.x0 + P.x0_off;
            yin = a.y0 + P.x0_off;
            if (s >= 1) prior = a.cdf0 + P.c0_off;
        } else {
            xin = a.xa + P.x_off + (int64_t)(s - 1) * n;
            yin = a.ya + P.x_off + (int64_t)(s - 1) * n;
            prior = a.fprev + P.c_off + (int64_t)(s - 1) * (bins + 1);
        }
        MatchSmem ms = carve_match_smem_f32(mbase, bins, prior, a.rho + P.r_off + (int64_t)s * (bins + 1));
        if (do_match) build_match_table(P.g, thr, ms);
        __syncthreads();
        const BinF32 bf = make_bin_f32(thr, bins, P.lo_f, P.inv_h_f);
        float* xout = a.xb + P.x_off + (int64_t)s * n;
        float* yout = a.yb + P.x_off + (int64_t)s * n;
        const int steps = a.steps_div > 1 ? (P.steps + a.steps_div - 1) / a.steps_div : P.steps;
        const D1Consts c{P.lam, P.ddt, P.rel, P.sxk, P.syk, P.k0, P.k1, P.chi};
        const D1Smem sm{thr, hs, he, &ms, bf, do_match, true, true};
        if (P.kind == PR_MODEL_OU)
            fine_d1_range<PR_MODEL_OU, PPT>(xin, yin, xout, yout, it.begin, it.end, (uint32_t)s, steps, c, sm);
        else
            fine_d1_range<PR_MODEL_DOUBLE_WELL, PPT>(xin, yin, xout, yout, it.begin, it.end, (uint32_t)s, steps, c, sm);
        __syncthreads();
        uint32_t* cs = a.counts_s + P.h_off + (int64_t)s * bins;
        uint32_t* ce = a.counts_e + P.h_off + (int64_t)s * bins;
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            if (hs[i]) atomicAdd(&cs[i], hs[i]);
            if (he[i]) atomicAdd(&ce[i], he[i]);
        }
        __syncthreads();
    }
}

// counts -> CDF per (problem, slice); blockIdx.y selects start (0) or end (1)
__global__ void __launch_bounds__(256)
batch_cdf_kernel(const BatchProblemDev* __restrict__ probs, const BatchRowDev* __restrict__ rows,
                 const uint32_t* __restrict__ counts_s, const uint32_t* __restrict__ counts_e,
                 double* __restrict__ start, double* __restrict__ fstar)
{
    __shared__ unsigned long long warp_tot[8];
    const BatchRowDev r = rows[blockIdx.x];
    const BatchProblemDev& P = probs[r.problem];
    const int bins = P.bins;
    const uint32_t* c = (blockIdx.y == 0 ? counts_s : counts_e) + P.h_off + (int64_t)r.slice * bins;
    double* C = (blockIdx.y == 0 ? start : fstar) + P.c_off + (int64_t)r.slice * (bins + 1);
    const int T = blockDim.x;
    const int chunk = (bins + T - 1) / T;
    const int b = threadIdx.x * chunk, e = min(bins, b + chunk);
    unsigned long long loc = 0;
    for (int i = b; i < e; ++i) loc += c[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned long long off = 0;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    unsigned long long run = off + incl - loc;
    const double dn = (double)P.n;
    for (int i = b; i < e; ++i) {
        run += c[i];
        C[i + 1] = (double)run / dn;
    }
    if (threadIdx.x == 0) C[0] = 0.0;
}

__global__ void __launch_bounds__(kCoarseThreads)
batch_coarse_kernel(const BatchProblemDev* __restrict__ probs, const BatchRowDev* __restrict__ rows,
                    const double* __restrict__ cin, double* __restrict__ cout)
{
    extern __shared__ __align__(16) double dsm[];
    const BatchRowDev r = rows[blockIdx.x];
    const BatchProblemDev& P = probs[r.problem];
    const int I = P.bins;
    double* in = dsm;
    double* out = in + (I + 1);
    double* mass = out + (I + 1);
    double* mp = mass + I;
    double* wsum = mp + I;
    const double* src = cin + P.c_off + (int64_t)r.slice * (I + 1);
    for (int i = threadIdx.x; i <= I; i += blockDim.x) in[i] = src[i];
    __syncthreads();
    coarse_apply_block(P.P, I, in, out, mass, mp, wsum);
    double* dst = cout + P.c_off + (int64_t)r.slice * (I + 1);
    for (int i = threadIdx.x; i <= I; i += blockDim.x) dst[i] = out[i];
}

__global__ void __launch_bounds__(kCoarseThreads)
batch_update_kernel(const BatchProblemDev* __restrict__ probs, int iterator, int qmode,
                    const double* __restrict__ cdf0, const double* __restrict__ fstar,
                    const double* __restrict__ cstar, double* __restrict__ rho, int32_t* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char usm[];
    const BatchProblemDev& P = probs[blockIdx.x];
    serial_sweep(usm, P.P, P.g, iterator, qmode, P.K, cdf0 + P.c0_off, fstar ? fstar + P.c_off : nullptr,
                 cstar ? cstar + P.c_off : nullptr, rho + P.r_off, status + blockIdx.x);
}

__global__ void batch_restrict0_kernel(const BatchProblemDev* __restrict__ probs, const float* __restrict__ x0,
                                       uint32_t* __restrict__ counts0, double* __restrict__ cdf0)
{
    // restriction of X_0 for one problem per block (set-up only)
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long warp_tot[8];
    const BatchProblemDev& P = probs[blockIdx.x];
    const int bins = P.bins;
    float* thr = reinterpret_cast<float*>(smem);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + (((size_t)(bins + 1) * 4 + 15) & ~(size_t)15));
    build_thresholds(P.g, thr);
    for (int i = threadIdx.x; i < bins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const float* x = x0 + P.x0_off;
    for (int64_t p = threadIdx.x; p < P.n; p += blockDim.x) atomicAdd(&hist[bin_of_f32(thr, bins, P.lo_f, P.inv_h_f, x[p])], 1u);
    __syncthreads();
    // exclusive prefix -> CDF (one chunk per thread)
    const int T = blockDim.x;
    const int chunk = (bins + T - 1) / T;
    const int b = threadIdx.x * chunk, e = min(bins, b + chunk);
    unsigned long long loc = 0;
    for (int i = b; i < e; ++i) loc += hist[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned long long off = 0;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    unsigned long long run = off + incl - loc;
    double* C = cdf0 + P.c0_off;
    const int64_t h0 = P.c0_off - blockIdx.x;   // sum of I over the problems before: counts0 is [sum I]
    for (int i = b; i < e; ++i) {
        counts0[h0 + i] = hist[i];
        run += hist[i];
        C[i + 1] = (double)run / (double)P.n;
    }
    if (threadIdx.x == 0) C[0] = 0.0;
}

struct BatchPlan {
    int device = 0;
    int np = 0;
    pr_iterator iterator = PR_ITER_QUANTILE;
    pr_quantile_mode qmode = PR_QMODE_TWO_SIDED;
    std::vector<pr_problem> probs;
    std::vector<void*> coarse;
    std::vector<BatchProblemDev> hp;
    std::vector<BatchRowDev> hrows;
    int max_bins = 1;
    int64_t sumN = 0, sumKN = 0, sumKI = 0, sumKI1 = 0, sumK1I1 = 0, sumI1 = 0, sumK = 0;
    int64_t work = 0;   // particle-steps per iteration
    // device
    BatchProblemDev* d_probs = nullptr;
    BatchRowDev* d_rows = nullptr;
    BatchItemDev* d_items = nullptr;
    int n_items = 0;
    size_t items_cap = 0;
    unsigned int* d_counter = nullptr;
    float *x0 = nullptr, *y0 = nullptr, *xa = nullptr, *ya = nullptr, *xb = nullptr, *yb = nullptr;
    double *cdf0 = nullptr, *rho = nullptr, *fstar = nullptr, *fprev = nullptr, *start = nullptr, *cstar = nullptr;
    // the ping-pong buffers as allocated: every run starts from these roles,
    // so the graphs captured for the two parities stay valid across runs
    float *xa0 = nullptr, *ya0 = nullptr, *xb0 = nullptr, *yb0 = nullptr;
    double *fstar0 = nullptr, *fprev0 = nullptr;
    uint32_t *counts = nullptr, *counts0 = nullptr;
    int32_t* status = nullptr;
    int k = -1;
    int ppt = 4;
    double item_work = 0.0;
    int grid_ctas = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

template <int PPT>
static int batch_resident(size_t smem)
{
    int per_sm = 0;
    cudaFuncSetAttribute(batch_fine_kernel<PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fine_kernel<PPT>, 256, smem) != cudaSuccess)
        per_sm = 1;
    return std::max(1, per_sm) * num_sms();
}

static int resident_ctas(const BatchPlan& pl)
{
    const size_t smem = batch_fine_smem(pl.max_bins);
    switch (pl.ppt) {
    case 1: return batch_resident<1>(smem);
    case 2: return batch_resident<2>(smem);
    default: return batch_resident<4>(smem);
    }
}

// Work items: each problem's slices cut into particle ranges of about
// item_work particle-steps (whole tiles), sorted by cost, largest first.
static pr_status build_items(BatchPlan& pl)
{
    const int64_t tile = 256LL * pl.ppt;
    std::vector<BatchItemDev> items;
    std::vector<double> cost;
    for (int p = 0; p < pl.np; ++p) {
        const pr_problem& q = pl.probs[p];
        const int64_t S = std::max(1, q.steps);
        int64_t chunk = (int64_t)std::ceil(pl.item_work / (double)S);
        chunk = ((chunk + tile - 1) / tile) * tile;
        chunk = std::max<int64_t>(tile, std::min<int64_t>(chunk, q.n));
        for (int s = 0; s < q.n_slices; ++s)
            for (int64_t b = 0; b < q.n; b += chunk) {
                items.push_back(BatchItemDev{p, s, b, std::min<int64_t>(q.n, b + chunk)});
                cost.push_back((double)(std::min<int64_t>(q.n, b + chunk) - b) * S);
            }
    }
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<BatchItemDev> sorted;
    sorted.reserve(items.size());
    for (size_t i : order) sorted.push_back(items[i]);
    if (sorted.size() > pl.items_cap) {
        if (pl.d_items) cudaFree(pl.d_items);
        pl.d_items = nullptr;
        pl.items_cap = 0;
        if (cudaMalloc(&pl.d_items, sorted.size() * sizeof(BatchItemDev)) != cudaSuccess) return PR_ERR_NOMEM;
        pl.items_cap = sorted.size();
    }
    if (cudaMemcpy(pl.d_items, sorted.data(), sorted.size() * sizeof(BatchItemDev), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return PR_ERR_CUDA;
    pl.n_items = (int)sorted.size();
    pl.grid_ctas = resident_ctas(pl);
    return PR_OK;
}

static void drop_graphs(BatchPlan& pl)
{
    for (auto& g : pl.graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

static pr_status launch_fine(BatchPlan& pl, int first, int steps_div, cudaStream_t st)
{
    BatchFineArgs a{};
    a.probs = pl.d_probs;
    a.items = pl.d_items;
    a.n_items = pl.n_items;
    a.counter = pl.d_counter;
    a.x0 = pl.x0;
    a.y0 = pl.y0;
    a.xa = pl.xa;
    a.ya = pl.ya;
    a.xb = pl.xb;
    a.yb = pl.yb;
    a.cdf0 = pl.cdf0;
    a.fprev = pl.fprev;
    a.rho = pl.rho;
    a.counts_s = pl.counts;
    a.counts_e = pl.counts + pl.sumKI;
    a.first = first;
    a.max_bins = pl.max_bins;
    a.steps_div = steps_div;
    const size_t smem = batch_fine_smem(pl.max_bins);
    PR_TRY_CUDA(cudaMemsetAsync(pl.d_counter, 0, sizeof(unsigned int), st));
    PR_TRY_CUDA(cudaMemsetAsync(pl.counts, 0, (size_t)2 * pl.sumKI * sizeof(uint32_t), st));
    switch (pl.ppt) {
    case 1: batch_fine_kernel<1><<<pl.grid_ctas, 256, smem, st>>>(a); break;
    case 2: batch_fine_kernel<2><<<pl.grid_ctas, 256, smem, st>>>(a); break;
    default: batch_fine_kernel<4><<<pl.grid_ctas, 256, smem, st>>>(a); break;
    }
    PR_CHECK_LAUNCH();
    return PR_OK;
}

static pr_status enqueue_iteration(BatchPlan& pl, int first, cudaStream_t st)
{
    pr_status rc = launch_fine(pl, first, 1, st);
    if (rc != PR_OK) return rc;
    batch_cdf_kernel<<<dim3((unsigned)pl.sumK, 2), 256, 0, st>>>(pl.d_probs, pl.d_rows, pl.counts,
                                                                 pl.counts + pl.sumKI, pl.start, pl.fstar);
    PR_CHECK_LAUNCH();
    const size_t csm = ((size_t)2 * (pl.max_bins + 1) + 2 * (size_t)pl.max_bins + 40) * sizeof(double);
    batch_coarse_kernel<<<(unsigned)pl.sumK, kCoarseThreads, csm, st>>>(pl.d_probs, pl.d_rows, pl.start, pl.cstar);
    PR_CHECK_LAUNCH();
    batch_update_kernel<<<pl.np, kCoarseThreads, update_smem(pl.max_bins), st>>>(
        pl.d_probs, (int)pl.iterator, (int)pl.qmode, pl.cdf0, pl.fstar, pl.cstar, pl.rho, pl.status);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

static void swap_buffers(BatchPlan& pl)
{
    std::swap(pl.xa, pl.xb);
    std::swap(pl.ya, pl.yb);
    std::swap(pl.fstar, pl.fprev);
}

static void free_plan(BatchPlan* pl)
{
    drop_graphs(*pl);
    for (auto& d : pl->hp)
        if (d.P) cudaFree(const_cast<double*>(d.P));
    if (pl->xa0) {   // restore the allocation roles before freeing
        pl->xa = pl->xa0;
        pl->ya = pl->ya0;
        pl->xb = pl->xb0;
        pl->yb = pl->yb0;
        pl->fstar = pl->fstar0;
        pl->fprev = pl->fprev0;
    }
    for (void* h : pl->coarse)
        if (h) pr_coarse_destroy(h);
    void* bufs[] = {pl->d_probs, pl->d_rows, pl->d_items, pl->d_counter, pl->x0, pl->y0, pl->xa, pl->ya, pl->xb,
                    pl->yb, pl->cdf0, pl->rho, pl->fstar, pl->fprev, pl->start, pl->cstar, pl->counts,
                    pl->counts0, pl->status};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete pl;
}

}  // namespace pr

using namespace pr;

extern "C" pr_status pr_batch_create(const pr_problem* problems, int32_t n_problems, pr_iterator iterator,
                                     pr_quantile_mode qmode, void** plan, void* stream)
{
    if (!problems || n_problems < 1 || n_problems > (1 << 24) || !plan) return PR_ERR_INVALID_ARG;
    if (iterator < PR_ITER_QUANTILE || iterator > PR_ITER_ROT) return PR_ERR_INVALID_ARG;
    if (qmode != PR_QMODE_TWO_SIDED && qmode != PR_QMODE_MIDPOINT) return PR_ERR_INVALID_ARG;
    for (int p = 0; p < n_problems; ++p) {
        const pr_problem& q = problems[p];
        if (q.model.kind != PR_MODEL_OU && q.model.kind != PR_MODEL_DOUBLE_WELL) return PR_ERR_UNSUPPORTED;
        if (q.model.fast_dim != 1) return PR_ERR_UNSUPPORTED;
        if (!(q.model.beta > 0.0) || !(q.model.eps > 0.0) || !(q.model.tau_x > 0.0)) return PR_ERR_INVALID_ARG;
        if (!grid_ok(&q.grid) || q.grid.bins > kUpdateMaxBins) return PR_ERR_INVALID_ARG;
        if (q.n < 1 || q.n > 0xFFFFFFFFll || q.n_slices < 1 || q.steps < 0) return PR_ERR_INVALID_ARG;
        if (!(q.dt > 0.0) || !std::isfinite(q.dt)) return PR_ERR_INVALID_ARG;
    }
    *plan = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto* pl = new BatchPlan;
    cudaGetDevice(&pl->device);
    pl->np = n_problems;
    pl->iterator = iterator;
    pl->qmode = qmode;
    pl->probs.assign(problems, problems + n_problems);
    pl->hp.resize(n_problems);
    for (int p = 0; p < n_problems; ++p) {
        const pr_problem& q = problems[p];
        BatchProblemDev& d = pl->hp[p];
        const double drift_dt = q.dt / q.model.tau_x, relax = q.dt / q.model.eps;
        const double sx = std::sqrt(2.0 * (1.0 / q.model.beta) / q.model.tau_x) * std::sqrt(q.dt);
        const double sy = std::sqrt(2.0 / q.model.eps) * std::sqrt(q.dt);
        d.lam = (float)q.model.lambda;
        d.ddt = (float)drift_dt;
        d.rel = (float)relax;
        d.sxk = (float)(sx * 1.1774100225154746910);
        d.syk = (float)(sy * 1.1774100225154746910);
        d.k0 = (uint32_t)(q.seed & 0xFFFFFFFFull);
        d.k1 = (uint32_t)(q.seed >> 32);
        d.chi = (uint32_t)p << 8;
        d.kind = q.model.kind;
        d.steps = q.steps;
        d.bins = q.grid.bins;
        d.K = q.n_slices;
        d.g = make_grid(q.grid);
        d.lo_f = (float)q.grid.x_lo;
        d.inv_h_f = (float)(1.0 / d.g.h);
        d.n = q.n;
        d.x0_off = pl->sumN;
        d.x_off = pl->sumKN;
        d.h_off = pl->sumKI;
        d.c_off = pl->sumKI1;
        d.r_off = pl->sumK1I1;
        d.c0_off = pl->sumI1;
        pl->sumN += q.n;
        pl->sumKN += (int64_t)q.n_slices * q.n;
        pl->sumKI += (int64_t)q.n_slices * q.grid.bins;
        pl->sumKI1 += (int64_t)q.n_slices * (q.grid.bins + 1);
        pl->sumK1I1 += (int64_t)(q.n_slices + 1) * (q.grid.bins + 1);
        pl->sumI1 += q.grid.bins + 1;
        pl->sumK += q.n_slices;
        pl->max_bins = std::max(pl->max_bins, q.grid.bins);
        pl->work += q.n * (int64_t)q.n_slices * q.steps;
        for (int s = 0; s < q.n_slices; ++s) pl->hrows.push_back(BatchRowDev{p, s});
        void* h = nullptr;
        const pr_status rc = pr_coarse_create(&q.model, &q.grid, q.steps * q.dt, &h, stream);
        if (rc != PR_OK) {
            free_plan(pl);
            return rc;
        }
        pl->coarse.push_back(h);
        d.P = nullptr;
    }
    // the coarse matrices: copy each handle's P into its own buffer owned by the handle
    for (int p = 0; p < n_problems; ++p) {
        double* Pd = nullptr;
        // pr_coarse_matrix copies; the handle's pointer is reached through a copy-out buffer
        const size_t bytes = (size_t)pl->probs[p].grid.bins * pl->probs[p].grid.bins * sizeof(double);
        if (cudaMalloc(&Pd, bytes) != cudaSuccess) {
            free_plan(pl);
            return PR_ERR_NOMEM;
        }
        if (pr_coarse_matrix(pl->coarse[p], Pd, stream) != PR_OK) {
            cudaFree(Pd);
            free_plan(pl);
            return PR_ERR_CUDA;
        }
        pr_coarse_destroy(pl->coarse[p]);
        pl->coarse[p] = nullptr;
        pl->hp[p].P = Pd;
    }
    auto alloc = [&](void** ptr, size_t bytes) { return cudaMalloc(ptr, std::max<size_t>(bytes, 16)) == cudaSuccess; };
    bool ok = alloc((void**)&pl->d_probs, n_problems * sizeof(BatchProblemDev)) &&
              alloc((void**)&pl->d_rows, pl->hrows.size() * sizeof(BatchRowDev)) &&
              alloc((void**)&pl->d_counter, sizeof(unsigned int)) && alloc((void**)&pl->x0, pl->sumN * 4) &&
              alloc((void**)&pl->y0, pl->sumN * 4) && alloc((void**)&pl->xa, pl->sumKN * 4) &&
              alloc((void**)&pl->ya, pl->sumKN * 4) && alloc((void**)&pl->xb, pl->sumKN * 4) &&
              alloc((void**)&pl->yb, pl->sumKN * 4) && alloc((void**)&pl->cdf0, pl->sumI1 * 8) &&
              alloc((void**)&pl->rho, pl->sumK1I1 * 8) && alloc((void**)&pl->fstar, pl->sumKI1 * 8) &&
              alloc((void**)&pl->fprev, pl->sumKI1 * 8) && alloc((void**)&pl->start, pl->sumKI1 * 8) &&
              alloc((void**)&pl->cstar, pl->sumKI1 * 8) && alloc((void**)&pl->counts, 2 * pl->sumKI * 4) &&
              alloc((void**)&pl->counts0, pl->sumI1 * 4) && alloc((void**)&pl->status, n_problems * 4);
    if (!ok) {
        free_plan(pl);
        return PR_ERR_NOMEM;
    }
    pl->xa0 = pl->xa;
    pl->ya0 = pl->ya;
    pl->xb0 = pl->xb;
    pl->yb0 = pl->yb;
    pl->fstar0 = pl->fstar;
    pl->fprev0 = pl->fprev;
    // the P pointers are device pointers owned by the plan (freed in free_plan via hp)
    if (cudaMemcpyAsync(pl->d_probs, pl->hp.data(), n_problems * sizeof(BatchProblemDev), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(pl->d_rows, pl->hrows.data(), pl->hrows.size() * sizeof(BatchRowDev), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemsetAsync(pl->status, 0, n_problems * 4, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        free_plan(pl);
        return PR_ERR_CUDA;
    }
    const size_t fsm = batch_fine_smem(pl->max_bins);
    cudaFuncSetAttribute(batch_fine_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    cudaFuncSetAttribute(batch_fine_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    cudaFuncSetAttribute(batch_fine_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    cudaFuncSetAttribute(batch_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)update_smem(pl->max_bins));
    cudaFuncSetAttribute(batch_coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(((size_t)2 * (pl->max_bins + 1) + 2 * (size_t)pl->max_bins + 40) * sizeof(double)));
    cudaFuncSetAttribute(batch_restrict0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((((size_t)(pl->max_bins + 1) * 4 + 15) & ~(size_t)15) + (size_t)pl->max_bins * 4));
    pl->ppt = 4;
    pl->item_work = 0.0;
    {
        const int slots = resident_ctas(*pl);
        pl->item_work = std::max(1.0, (double)pl->work / ((double)slots * 8.0));
    }
    const pr_status rc = build_items(*pl);
    if (rc != PR_OK) {
        free_plan(pl);
        return rc;
    }
    *plan = pl;
    return PR_OK;
}

extern "C" pr_status pr_batch_destroy(void* plan)
{
    if (!plan) return PR_ERR_INVALID_ARG;
    free_plan(static_cast<BatchPlan*>(plan));
    return PR_OK;
}

extern "C" int64_t pr_batch_particle_steps(void* plan)
{
    return plan ? static_cast<BatchPlan*>(plan)->work : 0;
}

extern "C" pr_status pr_batch_set_initial(void* plan, const float* x0, const float* y0, void* stream)
{
    if (!plan || !x0 || !y0 || !elem_aligned(x0, 4) || !elem_aligned(y0, 4)) return PR_ERR_INVALID_ARG;
    auto* pl = static_cast<BatchPlan*>(plan);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pl->xa = pl->xa0;
    pl->ya = pl->ya0;
    pl->xb = pl->xb0;
    pl->yb = pl->yb0;
    pl->fstar = pl->fstar0;
    pl->fprev = pl->fprev0;
    PR_TRY_CUDA(cudaMemcpyAsync(pl->x0, x0, pl->sumN * 4, cudaMemcpyDeviceToDevice, st));
    PR_TRY_CUDA(cudaMemcpyAsync(pl->y0, y0, pl->sumN * 4, cudaMemcpyDeviceToDevice, st));
    const size_t rsm = (((size_t)(pl->max_bins + 1) * 4 + 15) & ~(size_t)15) + (size_t)pl->max_bins * 4;
    batch_restrict0_kernel<<<pl->np, 256, rsm, st>>>(pl->d_probs, pl->x0, pl->counts0, pl->cdf0);
    PR_CHECK_LAUNCH();
    // zeroth iteration: serial coarse sweep from R X_0
    batch_update_kernel<<<pl->np, kCoarseThreads, update_smem(pl->max_bins), st>>>(
        pl->d_probs, (int)PR_ITER_NONE, (int)pl->qmode, pl->cdf0, nullptr, nullptr, pl->rho, pl->status);
    PR_CHECK_LAUNCH();
    pl->k = 0;
    return PR_OK;
}

extern "C" pr_status pr_batch_iterate(void* plan, void* stream)
{
    if (!plan) return PR_ERR_INVALID_ARG;
    auto* pl = static_cast<BatchPlan*>(plan);
    if (pl->k < 0) return PR_ERR_INVALID_ARG;   // no initial ensemble yet
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (pl->k == 0) {
        const pr_status rc = enqueue_iteration(*pl, 1, st);
        if (rc != PR_OK) return rc;
    } else {
        const int par = pl->k & 1;
        if (!pl->graph[par]) {
            cudaStream_t cap = nullptr;
            PR_TRY_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            pr_status rc = PR_OK;
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PR_ERR_CUDA;
            if (rc == PR_OK) rc = enqueue_iteration(*pl, 0, cap);
            const cudaError_t ec = cudaStreamEndCapture(cap, &g);
            if (rc == PR_OK && ec != cudaSuccess) rc = PR_ERR_CUDA;
            if (rc == PR_OK && cudaGraphInstantiate(&pl->graph[par], g, 0) != cudaSuccess) rc = PR_ERR_CUDA;
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
            if (rc != PR_OK) return rc;
        }
        PR_TRY_CUDA(cudaGraphLaunch(pl->graph[par], st));
    }
    swap_buffers(*pl);
    pl->k += 1;
    return PR_OK;
}

extern "C" pr_status pr_batch_rho(void* plan, int32_t problem, double* out, void* stream)
{
    if (!plan || !out || !elem_aligned(out, 8)) return PR_ERR_INVALID_ARG;
    auto* pl = static_cast<BatchPlan*>(plan);
    if (problem < 0 || problem >= pl->np) return PR_ERR_INVALID_ARG;
    const BatchProblemDev& d = pl->hp[problem];
    const size_t bytes = (size_t)(d.K + 1) * (d.bins + 1) * sizeof(double);
    PR_TRY_CUDA(cudaMemcpyAsync(out, pl->rho + d.r_off, bytes, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
    return PR_OK;
}

extern "C" pr_status pr_batch_fine_state(void* plan, int32_t problem, float* x_out, float* y_out, void* stream)
{
    if (!plan || !x_out || !y_out || !elem_aligned(x_out, 4) || !elem_aligned(y_out, 4)) return PR_ERR_INVALID_ARG;
    auto* pl = static_cast<BatchPlan*>(plan);
    if (problem < 0 || problem >= pl->np) return PR_ERR_INVALID_ARG;
    const BatchProblemDev& d = pl->hp[problem];
    const size_t bytes = (size_t)d.K * d.n * sizeof(float);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PR_TRY_CUDA(cudaMemcpyAsync(x_out, pl->xa + d.x_off, bytes, cudaMemcpyDeviceToDevice, st));
    PR_TRY_CUDA(cudaMemcpyAsync(y_out, pl->ya + d.x_off, bytes, cudaMemcpyDeviceToDevice, st));
    return PR_OK;
}

extern "C" pr_status pr_batch_status(void* plan, int32_t* worst, void* stream)
{
    if (!plan || !worst) return PR_ERR_INVALID_ARG;
    auto* pl = static_cast<BatchPlan*>(plan);
    std::vector<int32_t> h(pl->np);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PR_TRY_CUDA(cudaMemcpyAsync(h.data(), pl->status, pl->np * 4, cudaMemcpyDeviceToHost, st));
    PR_TRY_CUDA(cudaStreamSynchronize(st));
    int32_t w = 0;
    for (int32_t v : h) w = std::max(w, v);
    *worst = w;
    return PR_OK;
}

extern "C" pr_status pr_batch_set_config(void* plan, int32_t ppt, double item_work)
{
    if (!plan || (ppt != 1 && ppt != 2 && ppt != 4) || !(item_work >= 1.0)) return PR_ERR_INVALID_ARG;
    auto* pl = static_cast<BatchPlan*>(plan);
    pl->ppt = ppt;
    pl->item_work = item_work;
    drop_graphs(*pl);
    return build_items(*pl);
}

extern "C" pr_status pr_batch_get_config(void* plan, int32_t* ppt, double* item_work, int32_t* n_items)
{
    if (!plan) return PR_ERR_INVALID_ARG;
    auto* pl = static_cast<BatchPlan*>(plan);
    if (ppt) *ppt = pl->ppt;
    if (item_work) *item_work = pl->item_work;
    if (n_items) *n_items = pl->n_items;
    return PR_OK;
}

extern "C" pr_status pr_batch_tune(void* plan, int32_t steps_div, double* best_ms, void* stream)
{
    if (!plan || steps_div < 1) return PR_ERR_INVALID_ARG;
    auto* pl = static_cast<BatchPlan*>(plan);
    if (pl->k < 0) return PR_ERR_INVALID_ARG;   // needs the initial ensemble (the trials read it)
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ppts[3] = {1, 2, 4};
    const double per_slot[4] = {2.0, 8.0, 32.0, 128.0};
    cudaEvent_t e0, e1;
    PR_TRY_CUDA(cudaEventCreate(&e0));
    PR_TRY_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_ppt = pl->ppt;
    double best_work = pl->item_work;
    pr_status rc = PR_OK;
    for (int pi = 0; pi < 3 && rc == PR_OK; ++pi) {
        pl->ppt = ppts[pi];
        const int slots = resident_ctas(*pl);
        for (int wi = 0; wi < 4 && rc == PR_OK; ++wi) {
            pl->item_work = std::max(1.0, (double)pl->work / ((double)slots * per_slot[wi]));
            if ((rc = build_items(*pl)) != PR_OK) break;
            // a trial writes only the work buffers of the next iteration, so the state is kept
            if ((rc = launch_fine(*pl, 1, steps_div, st)) != PR_OK) break;
            cudaEventRecord(e0, st);
            if ((rc = launch_fine(*pl, 1, steps_div, st)) != PR_OK) break;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = PR_ERR_CUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_ppt = pl->ppt;
                best_work = pl->item_work;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->ppt = best_ppt;
    pl->item_work = best_work;
    drop_graphs(*pl);
    const pr_status rb = build_items(*pl);
    if (best_ms) *best_ms = best;
    return rc != PR_OK ? rc : rb;
}

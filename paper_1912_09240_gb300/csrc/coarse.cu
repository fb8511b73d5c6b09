// coarse.cu -- coarse propagator C_dT (Section 2.2.2), the serial parareal
// update rho^{n+1} = J(C(rho^n), rho_f*, rho_c*) (Section 3.2.3, Eq.
// mm_sequential) with the iterators of Section 4, and the W1 distance.
//
// Everything here is FP64.  The macroscopic states are short (I <= 4096 bins,
// the serial update I <= 1024), so the work is latency-bound: one CTA per
// state vector, and one CTA for the serial sweep over the slices.  Operations
// that decide exactness (edges, quantile interpolation, the monotone repair,
// reading the CDF back at the edges) are written with explicitly rounded
// intrinsics so that no multiply-add is fused.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "coarse_dev.cuh"
#include "pr_common.cuh"

namespace pr {

struct ChemRates {
    double k[6];
    bool printed;
};

struct CoarseHandle {
    GridDev g;
    double* P;   // row-major I x I
    int device;
};

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Mean ybar of the chemical system's fast equilibrium (Section 2.2.3),
// phi(y) ~ exp(-int_0^y G'(s)/E(s) ds) / E(y), by the trapezoidal rule on
// y_j = j/2, j = 0..4000 (the inner integral cumulatively on the same grid).
// One thread walks the grid twice in order (the maximum of log phi, then the
// weighted sums); set-up work of a few milliseconds.
constexpr double kChemDy = 0.5;
constexpr int kChemJ = 4000;

__device__ __forceinline__ void chem_fast_terms(const double* k, bool printed, double y, double& ratio,
                                                double& log_e)
{
    const double y1 = y * (y - 1.0), y2 = y1 * (y - 2.0);
    const double net = k[0] - k[1] * y + k[2] * y1 - k[3] * y2;              // -G' (net rates)
    const double dg = printed ? -k[0] - k[1] * y + k[2] * y1 - k[3] * y2 : -net;
    const double e = 0.5 * (k[0] + k[1] * y + k[2] * y1 + k[3] * y2);
    ratio = dg / e;
    log_e = log(e);
}

__global__ void chem_ybar_kernel(ChemRates r, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double top = -INFINITY;
    for (int pass = 0; pass < 2; ++pass) {
        double integral = 0.0, prev = 0.0, num = 0.0, den = 0.0;
        for (int j = 0; j <= kChemJ; ++j) {
            const double y = j * kChemDy;
            double ratio, log_e;
            chem_fast_terms(r.k, r.printed, y, ratio, log_e);
            if (j) integral += 0.5 * kChemDy * (prev + ratio);
            prev = ratio;
            const double log_phi = -integral - log_e;
            if (pass == 0) {
                top = fmax(top, log_phi);
            } else {
                const double w = (j == 0 || j == kChemJ) ? 0.5 : 1.0;
                const double phi = exp(log_phi - top);
                num += w * y * phi;
                den += w * phi;
            }
        }
        if (pass == 1) *out = num / den;
    }
}

__global__ void assemble_generator_kernel(GridDev g, int kind, double lam, double beta, double eps, double tau_x,
                                          double k4, double k5, const double* __restrict__ ybar_ptr,
                                          double slice_dt, double* __restrict__ A)
{
    const int I = g.bins;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= I) return;
    const bool chem = kind == PR_MODEL_CHEM || kind == PR_MODEL_CHEM_PRINTED;
    const double a = chem ? k4 * *ybar_ptr : 0.0;   // k4 ybar
    // Dbar(x): 1/beta, or (k4 ybar + k5 x)/2 for the chemical system
    auto dbar = [&](double x) { return chem ? 0.5 * (a + k5 * x) : 1.0 / beta; };
    // log rho_inf(x) = log(1/Dbar(x)) - int_0^x Fbar'/Dbar: Fbar(x)/Dbar for a
    // constant Dbar; for the chemical system 2x - (4a/k5) log(1 + k5 x/a)
    // (Fbar' = k5 x - a, net rates) or -2x (Fbar' = -(a + k5 x), as printed)
    auto fbar = [&](double x) {
        if (kind == PR_MODEL_ADVECTION) return x / eps;   // given directly (linear advection case)
        return kind == PR_MODEL_OU ? 0.5 * (1.0 - lam) * x * x
                                   : 0.25 * x * x * x * x - 0.5 * (1.0 - lam) * x * x;
    };
    auto log_rho_inf = [&](double x) {
        if (!chem) return log(1.0 / dbar(x)) - fbar(x) / dbar(x);
        const double integral = kind == PR_MODEL_CHEM ? 2.0 * x - (4.0 * a / k5) * log1p(k5 * x / a) : -2.0 * x;
        return log(1.0 / dbar(x)) - integral;
    };
    auto centre = [&](int k) { return 0.5 * (edge(g, k) + edge(g, k + 1)); };
    auto width = [&](int k) { return edge(g, k + 1) - edge(g, k); };
    double* row = A + (size_t)c * I;
    for (int k = 0; k < I; ++k) row[k] = 0.0;
    double diag = 0.0;
    // left edge e = c: cell c loses phi_c
    if (c >= 1) {
        const int e = c;
        const double xe = edge(g, e);
        const double coef = dbar(xe) / (centre(e) - centre(e - 1));
        const double rr = exp(log_rho_inf(xe) - log_rho_inf(centre(e))) / width(e);
        const double rl = exp(log_rho_inf(xe) - log_rho_inf(centre(e - 1))) / width(e - 1);
        diag -= coef * rr / tau_x;
        row[c - 1] += coef * rl / tau_x;
    }
    // right edge e = c+1: cell c gains phi_{c+1}
    if (c + 1 <= I - 1) {
        const int e = c + 1;
        const double xe = edge(g, e);
        const double coef = dbar(xe) / (centre(e) - centre(e - 1));
        const double rr = exp(log_rho_inf(xe) - log_rho_inf(centre(e))) / width(e);
        const double rl = exp(log_rho_inf(xe) - log_rho_inf(centre(e - 1))) / width(e - 1);
        row[c + 1] += coef * rr / tau_x;
        diag -= coef * rl / tau_x;
    }
    row[c] = diag;
    for (int k = 0; k < I; ++k) row[k] *= slice_dt;
}

__global__ void norm1_kernel(const double* __restrict__ A, int n, double* out)
{
    // max over columns of the absolute column sum; one block
    __shared__ double best[256];
    double m = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < n; ++r) s += fabs(A[(size_t)r * n + c]);
        m = fmax(m, s);
    }
    best[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) v = fmax(v, best[i]);
        *out = v;
    }
}

__global__ void scale_kernel(double* A, size_t n, double s)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        A[i] *= s;
}

__global__ void identity_kernel(double* A, int n)
{
    const size_t nn = (size_t)n * n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
        A[i] = (i / n == i % n) ? 1.0 : 0.0;
}

// C = alpha * A B + beta * I   (n x n, row-major), 64x64 tiles, 256 threads x 4x4.
__global__ void __launch_bounds__(256) dgemm_kernel(int n, const double* __restrict__ A,
                                                    const double* __restrict__ B, double* __restrict__ C,
                                                    double alpha, double beta_identity)
{
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < n; k0 += 16) {
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int kk = t / 64, rr = t % 64;
            const int ar = row0 + rr, ak = k0 + kk;
            As[kk][rr] = (ar < n && ak < n) ? A[(size_t)ar * n + ak] : 0.0;
            const int bk = k0 + kk, bc = col0 + rr;
            Bs[kk][rr] = (bk < n && bc < n) ? B[(size_t)bk * n + bc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty * 4 + i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx * 4 + j;
            if (c >= n) continue;
            C[(size_t)r * n + c] = alpha * acc[i][j] + (r == c ? beta_identity : 0.0);
        }
    }
}

// C_dT on n_vec states, one state per cluster of CL CTAs (the rows of P @ m
// split between them; the bits do not depend on CL): on GB300's narrow FP64
// pipe one CTA takes ~60 us for 512^2 FMAs, so a few states fill the GPU only
// when each is spread over several SMs.
template <int CL>
__global__ void __launch_bounds__(kCoarseThreads)
coarse_fp_kernel(const double* __restrict__ P, int I, const double* __restrict__ cin, double* __restrict__ cout)
{
    extern __shared__ __align__(16) double dsm[];
    double* in = dsm;
    double* out = in + (I + 1);
    double* mass = out + (I + 1);
    double* mp = mass + I;
    double* wsum = mp + I;
    const Dist<CL> d = Dist<CL>::make();
    const size_t v = blockIdx.x / CL;
    const double* src = cin + v * (I + 1);
    for (int i = threadIdx.x; i <= I; i += blockDim.x) in[i] = src[i];
    __syncthreads();
    coarse_apply_block<CL>(P, I, in, out, mass, mp, wsum, d);
    double* dst = cout + v * (I + 1);
    const int q0 = d.lo(I - 1), q1 = d.hi(I - 1);
    for (int r = q0 + (int)threadIdx.x; r < q1; r += blockDim.x) dst[r + 1] = out[r + 1];
    if (d.rank == 0 && threadIdx.x == 0) {
        dst[0] = out[0];
        dst[I] = out[I];
    }
}

// The serial sweep of Section 3.2.3 on one CTA (CL = 1) or on a cluster of
// CL CTAs (launched with that cluster size).
template <int CL>
__global__ void __launch_bounds__(kCoarseThreads)
parareal_update_kernel(const double* __restrict__ P, GridDev g, int iterator, int qmode, int K,
                       const double* __restrict__ cdf0, const double* __restrict__ fstar,
                       const double* __restrict__ cstar, double* __restrict__ next, int32_t* status)
{
    extern __shared__ __align__(16) unsigned char usm[];
    serial_sweep<CL>(usm, P, g, iterator, qmode, K, cdf0, fstar, cstar, next, status);
}

__global__ void __launch_bounds__(kCoarseThreads)
iterate_kernel(GridDev g, int iterator, int qmode, const double* __restrict__ a, const double* __restrict__ b,
               const double* __restrict__ c, double* __restrict__ out, int32_t* status)
{
    extern __shared__ __align__(16) unsigned char usm[];
    const int I = g.bins;
    double* Ab = reinterpret_cast<double*>(usm);
    double* Bb = Ab + (I + 1);
    double* Cb = Bb + (I + 1);
    double* Ob = Cb + (I + 1);
    JqSmem js = carve_jq(reinterpret_cast<unsigned char*>(Ob + (I + 1)), I);
    if (threadIdx.x == 0) js.flag[1] = 0;
    const size_t off = (size_t)blockIdx.x * (I + 1);
    for (int i = threadIdx.x; i <= I; i += blockDim.x) {
        Ab[i] = a[off + i];
        Bb[i] = b[off + i];
        Cb[i] = c[off + i];
    }
    __syncthreads();
    if (iterator == PR_ITER_QUANTILE) quantile_iterate_block(g, qmode, Ab, Bb, Cb, Ob, js);
    else mass_iterate_block(iterator, I, Ab, Bb, Cb, Ob, js.kq, js.wsum);
    for (int i = threadIdx.x; i <= I; i += blockDim.x) out[off + i] = Ob[i];
    if (threadIdx.x == 0 && status && js.flag[1]) atomicExch(status, (int32_t)PR_ERR_NUMERIC);
}

__global__ void __launch_bounds__(256)
w1_kernel(GridDev g, const double* __restrict__ c1, const double* __restrict__ c2, double* __restrict__ w1)
{
    __shared__ double wsum[40];
    const int I = g.bins;
    const size_t off = (size_t)blockIdx.x * (I + 1);
    double acc = 0.0;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const double d0 = c1[off + i] - c2[off + i], d1 = c1[off + i + 1] - c2[off + i + 1];
        const double a0 = fabs(d0), a1 = fabs(d1);
        if ((d0 >= 0.0 && d1 >= 0.0) || (d0 <= 0.0 && d1 <= 0.0)) acc += 0.5 * g.h * (a0 + a1);
        else acc += g.h * (d0 * d0 + d1 * d1) / (2.0 * (a0 + a1));
    }
    const double s = block_sum_f64(acc, wsum);
    if (threadIdx.x == 0) w1[blockIdx.x] = s;
}

// L2 distance of the piecewise-constant densities (bin mass / h) of two CDFs:
// sqrt(sum_i (m1_i - m2_i)^2 / h), one CTA per pair.
__global__ void __launch_bounds__(256)
l2_density_kernel(GridDev g, const double* __restrict__ c1, const double* __restrict__ c2, double* __restrict__ out)
{
    __shared__ double wsum[40];
    const int I = g.bins;
    const size_t off = (size_t)blockIdx.x * (I + 1);
    double acc = 0.0;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        const double d = (c1[off + i + 1] - c1[off + i]) - (c2[off + i + 1] - c2[off + i]);
        acc += d * d / g.h;
    }
    const double s = block_sum_f64(acc, wsum);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
}

// CTAs of the cluster that runs the serial sweep (1, 2, 4 or 8; portable sizes).
static int g_update_cluster = 8;

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace pr

using namespace pr;

extern "C" pr_status pr_coarse_create(const pr_model* model, const pr_grid* grid, double slice_dt,
                                      void** handle, void* stream)
{
    if (!model || !grid_ok(grid) || !handle || !(slice_dt > 0.0) || !std::isfinite(slice_dt)) return PR_ERR_INVALID_ARG;
    const bool chem = model->kind == PR_MODEL_CHEM || model->kind == PR_MODEL_CHEM_PRINTED;
    if (chem) {
        // rates finite and non-negative, k4 and k5 positive (Dbar > 0 needs a
        // positive ybar and x_lo >= 0)
        if (!(model->tau_x > 0.0) || !(grid->x_lo >= 0.0)) return PR_ERR_INVALID_ARG;
        for (int i = 0; i < 6; ++i)
            if (!std::isfinite(model->rate[i]) || model->rate[i] < 0.0) return PR_ERR_INVALID_ARG;
        if (!(model->rate[4] > 0.0) || !(model->rate[5] > 0.0) || !(model->rate[0] > 0.0)) return PR_ERR_INVALID_ARG;
    } else {
        if (model->kind < PR_MODEL_OU || model->kind > PR_MODEL_ADVECTION) return PR_ERR_INVALID_ARG;
        if (!(model->beta > 0.0) || !(model->tau_x > 0.0) || !std::isfinite(model->lambda)) return PR_ERR_INVALID_ARG;
        if (model->kind == PR_MODEL_ADVECTION && !(model->eps > 0.0)) return PR_ERR_INVALID_ARG;
    }
    *handle = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int I = grid->bins;
    const size_t nn = (size_t)I * I;
    double *B = nullptr, *X = nullptr, *Y = nullptr, *nrm = nullptr;
    auto release = [&]() {
        if (B) cudaFree(B);
        if (X) cudaFree(X);
        if (Y) cudaFree(Y);
        if (nrm) cudaFree(nrm);
    };
    if (cudaMalloc(&B, nn * 8) != cudaSuccess || cudaMalloc(&X, nn * 8) != cudaSuccess ||
        cudaMalloc(&Y, nn * 8) != cudaSuccess || cudaMalloc(&nrm, 16) != cudaSuccess) {
        release();
        return PR_ERR_NOMEM;
    }
    const GridDev g = make_grid(*grid);
    if (chem) {   // ybar (nrm[1]) first; it must be positive and finite
        ChemRates r;
        for (int i = 0; i < 6; ++i) r.k[i] = model->rate[i];
        r.printed = model->kind == PR_MODEL_CHEM_PRINTED;
        chem_ybar_kernel<<<1, 32, 0, st>>>(r, nrm + 1);
        double ybar = 0.0;
        if (cudaMemcpyAsync(&ybar, nrm + 1, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            release();
            return PR_ERR_CUDA;
        }
        if (!std::isfinite(ybar) || !(ybar > 0.0)) {
            release();
            return PR_ERR_NUMERIC;
        }
    }
    assemble_generator_kernel<<<(I + 127) / 128, 128, 0, st>>>(g, model->kind, model->lambda, model->beta,
                                                               model->eps, model->tau_x, model->rate[4],
                                                               model->rate[5], nrm + 1, slice_dt, B);
    norm1_kernel<<<1, 256, 0, st>>>(B, I, nrm);
    double norm = 0.0;
    if (cudaMemcpyAsync(&norm, nrm, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess || !std::isfinite(norm)) {
        release();
        return PR_ERR_CUDA;
    }
    // scaling and squaring: ||B / 2^s||_1 <= 1/4, Taylor polynomial of degree 18
    int s = 0;
    while (norm / std::ldexp(1.0, s) > 0.25 && s < 1000) ++s;
    const int blocks = 4 * num_sms();
    scale_kernel<<<blocks, 256, 0, st>>>(B, nn, std::ldexp(1.0, -s));
    double* T = X;   // current iterate
    double* W = Y;   // work
    identity_kernel<<<blocks, 256, 0, st>>>(T, I);
    dim3 gg((I + 63) / 64, (I + 63) / 64);
    const int degree = 18;
    for (int k = degree; k >= 1; --k) {   // T <- I + (B T)/k  (Horner)
        dgemm_kernel<<<gg, 256, 0, st>>>(I, B, T, W, 1.0 / k, 1.0);
        std::swap(T, W);
    }
    for (int q = 0; q < s; ++q) {         // T <- T T
        dgemm_kernel<<<gg, 256, 0, st>>>(I, T, T, W, 1.0, 0.0);
        std::swap(T, W);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        release();
        return PR_ERR_CUDA;
    }
    // keep T as P, free the rest
    double* P = T;
    if (T == X) X = nullptr; else Y = nullptr;
    release();
    auto* h = new CoarseHandle;
    h->g = g;
    h->P = P;
    cudaGetDevice(&h->device);
    *handle = h;
    return PR_OK;
}

extern "C" pr_status pr_coarse_destroy(void* handle)
{
    if (!handle) return PR_ERR_INVALID_ARG;
    auto* h = static_cast<CoarseHandle*>(handle);
    cudaFree(h->P);
    delete h;
    return PR_OK;
}

extern "C" pr_status pr_coarse_matrix(void* handle, double* out, void* stream)
{
    if (!handle || !out || !elem_aligned(out, 8)) return PR_ERR_INVALID_ARG;
    auto* h = static_cast<CoarseHandle*>(handle);
    const size_t bytes = (size_t)h->g.bins * h->g.bins * sizeof(double);
    PR_TRY_CUDA(cudaMemcpyAsync(out, h->P, bytes, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
    return PR_OK;
}

extern "C" pr_status pr_coarse_fp(void* handle, const double* cdf_in, double* cdf_out, int32_t n_vec, void* stream)
{
    if (!handle || !cdf_in || !cdf_out || n_vec < 1 || cdf_in == cdf_out) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(cdf_in, 8) || !elem_aligned(cdf_out, 8)) return PR_ERR_INVALID_ARG;
    auto* h = static_cast<CoarseHandle*>(handle);
    const int I = h->g.bins;
    const size_t smem = coarse_apply_smem(I);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the largest cluster that keeps the launch within two CTAs per SM
    int cl = 1;
    if (I >= 64)
        for (int c : {8, 4, 2})
            if ((int64_t)n_vec * c <= 2 * (int64_t)num_sms()) {
                cl = c;
                break;
            }
    if (cl == 1) {
        PR_TRY_CUDA(allow_smem(coarse_fp_kernel<1>, smem));
        coarse_fp_kernel<1><<<n_vec, kCoarseThreads, smem, st>>>(h->P, I, cdf_in, cdf_out);
        PR_CHECK_LAUNCH();
        return PR_OK;
    }
    auto launch = [&](auto kernel) -> cudaError_t {
        cudaError_t e = allow_smem(kernel, smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(n_vec * cl));
        cfg.blockDim = dim3(kCoarseThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, (const double*)h->P, I, cdf_in, cdf_out);
    };
    cudaError_t e;
    switch (cl) {
    case 2: e = launch(coarse_fp_kernel<2>); break;
    case 4: e = launch(coarse_fp_kernel<4>); break;
    default: e = launch(coarse_fp_kernel<8>); break;
    }
    if (e != cudaSuccess) return PR_ERR_CUDA;
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" pr_status pr_parareal_update(void* coarse, pr_iterator iterator, pr_quantile_mode qmode, int32_t n_slices,
                                        const double* cdf0, const double* cdf_f_star, const double* cdf_c_star,
                                        double* cdf_next, int32_t* status, void* stream)
{
    if (!coarse || !cdf0 || !cdf_next || n_slices < 1) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(cdf0, 8) || !elem_aligned(cdf_f_star, 8) || !elem_aligned(cdf_c_star, 8) ||
        !elem_aligned(cdf_next, 8) || !elem_aligned(status, 4))
        return PR_ERR_INVALID_ARG;
    if (iterator < PR_ITER_QUANTILE || iterator > PR_ITER_NONE) return PR_ERR_INVALID_ARG;
    if (qmode != PR_QMODE_TWO_SIDED && qmode != PR_QMODE_MIDPOINT) return PR_ERR_INVALID_ARG;
    if (iterator != PR_ITER_NONE && (!cdf_f_star || !cdf_c_star)) return PR_ERR_INVALID_ARG;
    auto* h = static_cast<CoarseHandle*>(coarse);
    if (h->g.bins > kUpdateMaxBins) return PR_ERR_UNSUPPORTED;
    const size_t smem = update_smem(h->g.bins);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int cl = h->g.bins >= 64 ? g_update_cluster : 1;
    if (cl == 1) {
        PR_TRY_CUDA(allow_smem(parareal_update_kernel<1>, smem));
        parareal_update_kernel<1><<<1, kCoarseThreads, smem, st>>>(h->P, h->g, (int)iterator, (int)qmode, n_slices,
                                                                  cdf0, cdf_f_star, cdf_c_star, cdf_next, status);
        PR_CHECK_LAUNCH();
        return PR_OK;
    }
    auto launch = [&](auto kernel) -> cudaError_t {
        cudaError_t e = allow_smem(kernel, smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)cl);
        cfg.blockDim = dim3(kCoarseThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, (const double*)h->P, h->g, (int)iterator, (int)qmode, (int)n_slices,
                                  cdf0, cdf_f_star, cdf_c_star, cdf_next, status);
    };
    cudaError_t e;
    switch (cl) {
    case 2: e = launch(parareal_update_kernel<2>); break;
    case 4: e = launch(parareal_update_kernel<4>); break;
    default: e = launch(parareal_update_kernel<8>); break;
    }
    if (e != cudaSuccess) return PR_ERR_CUDA;
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" void pr_set_update_cluster(int32_t ctas)
{
    g_update_cluster = (ctas == 1 || ctas == 2 || ctas == 4) ? ctas : 8;
}

extern "C" pr_status pr_iterate(pr_iterator iterator, pr_quantile_mode qmode, const pr_grid* grid, int32_t n_vec,
                                const double* a, const double* b, const double* c, double* out, int32_t* status,
                                void* stream)
{
    if (!grid_ok(grid) || n_vec < 1 || !a || !b || !c || !out) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(a, 8) || !elem_aligned(b, 8) || !elem_aligned(c, 8) || !elem_aligned(out, 8) ||
        !elem_aligned(status, 4))
        return PR_ERR_INVALID_ARG;
    if (iterator < PR_ITER_QUANTILE || iterator > PR_ITER_ROT) return PR_ERR_INVALID_ARG;
    if (qmode != PR_QMODE_TWO_SIDED && qmode != PR_QMODE_MIDPOINT) return PR_ERR_INVALID_ARG;
    if (grid->bins > kUpdateMaxBins) return PR_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (status) PR_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    const GridDev g = make_grid(*grid);
    const size_t smem = (size_t)4 * (grid->bins + 1) * sizeof(double) + jq_smem_bytes(grid->bins);
    PR_TRY_CUDA(allow_smem(iterate_kernel, smem));
    iterate_kernel<<<n_vec, kCoarseThreads, smem, st>>>(g, (int)iterator, (int)qmode, a, b, c, out, status);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" pr_status pr_w1(const pr_grid* grid, int32_t n_vec, const double* c1, const double* c2, double* w1,
                           void* stream)
{
    if (!grid_ok(grid) || n_vec < 1 || !c1 || !c2 || !w1) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(c1, 8) || !elem_aligned(c2, 8) || !elem_aligned(w1, 8)) return PR_ERR_INVALID_ARG;
    const GridDev g = make_grid(*grid);
    w1_kernel<<<n_vec, 256, 0, static_cast<cudaStream_t>(stream)>>>(g, c1, c2, w1);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" pr_status pr_l2_density(const pr_grid* grid, int32_t n_vec, const double* c1, const double* c2,
                                   double* l2, void* stream)
{
    if (!grid_ok(grid) || n_vec < 1 || !c1 || !c2 || !l2) return PR_ERR_INVALID_ARG;
    if (!elem_aligned(c1, 8) || !elem_aligned(c2, 8) || !elem_aligned(l2, 8)) return PR_ERR_INVALID_ARG;
    const GridDev g = make_grid(*grid);
    l2_density_kernel<<<n_vec, 256, 0, static_cast<cudaStream_t>(stream)>>>(g, c1, c2, l2);
    PR_CHECK_LAUNCH();
    return PR_OK;
}

extern "C" const char* pr_status_string(pr_status s)
{
    switch (s) {
    case PR_OK: return "PR_OK";
    case PR_ERR_INVALID_ARG: return "PR_ERR_INVALID_ARG";
    case PR_ERR_CUDA: return "PR_ERR_CUDA";
    case PR_ERR_TIMEOUT: return "PR_ERR_TIMEOUT";
    case PR_ERR_UNSUPPORTED: return "PR_ERR_UNSUPPORTED";
    case PR_ERR_NOMEM: return "PR_ERR_NOMEM";
    case PR_ERR_NUMERIC: return "PR_ERR_NUMERIC";
    }
    return "PR_ERR_UNKNOWN";
}

extern "C" const char* pr_version(void) { return "0.1.0"; }

/* Host <-> device transfers of caller buffers, for callers that hold their
 * inputs and results in host memory (no method arithmetic: one
 * cudaMemcpyAsync each, ordered on `stream`). */
extern "C" pr_status pr_copy_to_device(void* dst, const void* src, size_t bytes, void* stream)
{
    if (bytes == 0) return PR_OK;
    if (!dst || !src) return PR_ERR_INVALID_ARG;
    PR_TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream)));
    return PR_OK;
}

extern "C" pr_status pr_copy_to_host(void* dst, const void* src, size_t bytes, void* stream)
{
    if (bytes == 0) return PR_OK;
    if (!dst || !src) return PR_ERR_INVALID_ARG;
    PR_TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)));
    return PR_OK;
}

extern "C" pr_status pr_stream_synchronize(void* stream)
{
    PR_TRY_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return PR_OK;
}

// pr_common.cuh -- device helpers shared by the kernels of libpr.so:
// counter-based random numbers, uniform/normal conversion, grid edges and
// bin lookup, launch bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pr.h"

#define PR_MAX_BINS 4096
#define PR_MAX_FAST_DIM 16

// ---------------------------------------------------------------------------
// Host-side helpers
// ---------------------------------------------------------------------------

#define PR_CHECK_LAUNCH()                                   \
    do {                                                    \
        cudaError_t _e = cudaGetLastError();                \
        if (_e != cudaSuccess) return PR_ERR_CUDA;          \
    } while (0)

#define PR_TRY_CUDA(call)                                   \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) return PR_ERR_CUDA;          \
    } while (0)

namespace pr {

inline bool grid_ok(const pr_grid* g)
{
    return g && g->bins >= 1 && g->bins <= PR_MAX_BINS && g->x_lo < g->x_hi &&
           g->x_hi - g->x_lo < 1e300;
}

// A device pointer aligned to its element size (NULL counts as aligned: the
// optional arguments); entry points reject misaligned data on the host.
inline bool elem_aligned(const void* p, size_t bytes)
{
    return (reinterpret_cast<uintptr_t>(p) & (bytes - 1)) == 0;
}

inline size_t elem_bytes(pr_precision p) { return p == PR_F64 ? 8 : 4; }

int num_sms();   // of the current device, cached per device
int smem_optin_max();   // shared memory one CTA may opt in to, current device, cached per device

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor S-box, the key advanced by the Weyl constants between rounds.
// ---------------------------------------------------------------------------

constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

// One Philox4x32 round keyed by (k0, k1); each 32 x 32 -> 64-bit product
// gives both its high and low words.
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1)
{
    const unsigned long long pa = (unsigned long long)kPhiloxMulA * c.x;
    const unsigned long long pb = (unsigned long long)kPhiloxMulB * c.z;
    return make_uint4((uint32_t)(pb >> 32) ^ c.y ^ k0, (uint32_t)pb, (uint32_t)(pa >> 32) ^ c.w ^ k1,
                      (uint32_t)pa);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        c = philox_round(c, k0, k1);
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return c;
}

// Uniform in (0,1): the odd 24-bit integer 2*(w >> 9) + 1 times 2^-24.
// In binary32 this is built from the exponent bits of 1.0: the float
// 1 + (w>>9) 2^-23 minus (1 - 2^-24), an exact subtraction (Sterbenz).
__device__ __forceinline__ float uniform_f32(uint32_t w)
{
    return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994039535522461f;
}

__device__ __forceinline__ double uniform_f64(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

// Box-Muller in binary32 on the special-function unit: r = sqrt(-2 ln u0),
// theta = 2 pi u1.  -2 ln u0 = -2 ln2 * log2(u0).
__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ void box_muller_f32(uint32_t w0, uint32_t w1, float& z0, float& z1)
{
    const float u0 = uniform_f32(w0);
    const float u1 = uniform_f32(w1);
    const float r = sqrt_approx(-1.38629436111989061883f * __log2f(u0));
    const float th = 6.28318530717958647693f * u1;
    float s, c;
    __sincosf(th, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// Box-Muller split for the EM kernels: with L = log2(u0), the normals are
// z0 = K q cos(theta), z1 = K q sin(theta), q = sqrt(-L), K = sqrt(2 ln 2);
// K is folded into the noise amplitudes on the host.  The angle is built with
// one FMA from the float 1 + (w1 >> 9) 2^-23: theta = 2 pi (u1) with
// u1 = that float - (1 - 2^-24).
constexpr float kSqrt2Ln2 = 1.17741002251547469101f;   // sqrt(2 ln 2)

__device__ __forceinline__ void box_muller_qcs(uint32_t w0, uint32_t w1, float& q, float& c, float& s)
{
    const float u0 = uniform_f32(w0);
    const float f1 = __uint_as_float(0x3F800000u | (w1 >> 9));
    const float th = fmaf(6.28318530717958647693f, f1, -6.283185107518108f);   // 2 pi_f (1 - 2^-24)
    q = sqrt_approx(-__log2f(u0));
    __sincosf(th, &s, &c);
}

// One binary32 Euler-Maruyama step of the d = 1 families (Eqs. EMx/EMy with
// tau_x folded into ddt = dt/tau_x, rel = dt/eps), the noise increments given
// as products: sx dU = ax * cx, sy dV = ay * cy.  Written with explicit FMAs so
// that every kernel taking this step produces the same bits.
//   OU:          d_x F = x - lam y
//   double well: d_x F = x^3 - x + lam y
template <int KIND>
__device__ __forceinline__ float slow_force_f32(float x, float y, float lam)
{
    if (KIND == PR_MODEL_OU) return fmaf(-lam, y, x);
    return fmaf(lam, y, fmaf(x * x, x, -x));
}

template <int KIND>
__device__ __forceinline__ void em_step_f32(float& x, float& y, float ax, float cx, float ay, float cy, float lam,
                                            float ddt, float rel)
{
    const float f = slow_force_f32<KIND>(x, y, lam);
    const float xn = fmaf(ax, cx, fmaf(-f, ddt, x));
    const float yn = fmaf(ay, cy, fmaf(x - y, rel, y));
    x = xn;
    y = yn;
}

// The chemically reacting system (Section 2.1.2, Eqs. EMx/EMy), both
// readings of its drifts, with every constant folded on the host:
//   x' = x + a4 y + a5 x + sqrt(max(a4 y + v5 x, 0)) zx
//   y' = y + ((f3 y + f2) y + f1) y + f0 + sqrt(max(((e3 y + e2) y + e1) y + e0, 0)) zy
// a4 = k4 dt/tau_x, v5 = k5 dt/tau_x, a5 = -v5 (net reaction rates) or +v5
// (printed potential); f_i the coefficients of the cubic -d_y G and e_i those
// of 2E = k0 + k1 y + k2 y(y-1) + k3 y(y-1)(y-2), both times dt/eps.  The
// noise is given as products zx = ax * cx, zy = ay * cy (ax, ay = q sqrt(2 ln 2)).
template <typename T>
struct ChemConsts {
    T a4, a5, v5, f0, f1, f2, f3, e0, e1, e2, e3;
};

__device__ __forceinline__ void em_step_chem_f32(float& x, float& y, float ax, float cx, float ay, float cy,
                                                 const ChemConsts<float>& k)
{
    const float vx = fmaxf(fmaf(k.a4, y, k.v5 * x), 0.0f);
    const float vy = fmaxf(fmaf(fmaf(fmaf(k.e3, y, k.e2), y, k.e1), y, k.e0), 0.0f);
    const float fy = fmaf(fmaf(fmaf(k.f3, y, k.f2), y, k.f1), y, k.f0);
    const float xn = fmaf(ax * sqrt_approx(vx), cx, fmaf(k.a4, y, fmaf(k.a5, x, x)));
    const float yn = fmaf(ay * sqrt_approx(vy), cy, y + fy);
    x = xn;
    y = yn;
}

__device__ __forceinline__ void em_step_chem_f64(double& x, double& y, double zx, double zy,
                                                 const ChemConsts<double>& k)
{
    const double vx = fmax(k.a4 * y + k.v5 * x, 0.0);
    const double vy = fmax(((k.e3 * y + k.e2) * y + k.e1) * y + k.e0, 0.0);
    const double fy = ((k.f3 * y + k.f2) * y + k.f1) * y + k.f0;
    const double xn = x + (k.a4 * y + k.a5 * x) + sqrt(vx) * zx;
    const double yn = y + fy + sqrt(vy) * zy;
    x = xn;
    y = yn;
}

// Host-side folding of the rates (k[0..5]) into ChemConsts; `printed` selects
// the drifts of the printed potentials.
template <typename T>
inline ChemConsts<T> make_chem_consts(const double* k, bool printed, double dt, double tau_x, double eps)
{
    const double ax = dt / tau_x, ay = dt / eps;
    // -d_y G (net rates) = k0 - (k1 + k2 + 2 k3) y + (k2 + 3 k3) y^2 - k3 y^3;
    // the printed reading flips the sign of the terms in y, y^2, y^3
    const double sg = printed ? -1.0 : 1.0;
    ChemConsts<T> c;
    c.a4 = (T)(k[4] * ax);
    c.v5 = (T)(k[5] * ax);
    c.a5 = (T)((printed ? 1.0 : -1.0) * k[5] * ax);
    c.f0 = (T)(k[0] * ay);
    c.f1 = (T)(sg * -(k[1] + k[2] + 2.0 * k[3]) * ay);
    c.f2 = (T)(sg * (k[2] + 3.0 * k[3]) * ay);
    c.f3 = (T)(sg * -k[3] * ay);
    // 2E = k0 + (k1 - k2 + 2 k3) y + (k2 - 3 k3) y^2 + k3 y^3
    c.e0 = (T)(k[0] * ay);
    c.e1 = (T)((k[1] - k[2] + 2.0 * k[3]) * ay);
    c.e2 = (T)((k[2] - 3.0 * k[3]) * ay);
    c.e3 = (T)(k[3] * ay);
    return c;
}

__device__ __forceinline__ void box_muller_f64(uint32_t w0, uint32_t w1, double& z0, double& z1)
{
    const double u0 = uniform_f64(w0);
    const double u1 = uniform_f64(w1);
    const double r = sqrt(-2.0 * log(u0));
    double s, c;
    sincospi(2.0 * u1, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// ---------------------------------------------------------------------------
// Uniform grid.  Edges are e_i = x_lo + i*h with h = (x_hi - x_lo)/I, each
// operation rounded on its own (no fused multiply-add) so that every edge is
// the same double on the host, in the CPU reference and on the device.
// ---------------------------------------------------------------------------

struct GridDev {
    int bins;
    double lo, hi, h;
};

__host__ __device__ inline GridDev make_grid(const pr_grid& g)
{
    GridDev d;
    d.bins = g.bins;
    d.lo = g.x_lo;
    d.hi = g.x_hi;
#ifdef __CUDA_ARCH__
    d.h = __ddiv_rn(__dsub_rn(g.x_hi, g.x_lo), (double)g.bins);
#else
    d.h = (g.x_hi - g.x_lo) / (double)g.bins;
#endif
    return d;
}

__device__ __forceinline__ double edge(const GridDev& g, int i)
{
    return __dadd_rn(g.lo, __dmul_rn((double)i, g.h));
}

// Bin of a double: e_i <= x < e_{i+1}, clamped into [0, I-1].
__device__ __forceinline__ int bin_of_f64(const GridDev& g, double x)
{
    if (!(x >= g.lo)) return 0;
    if (x >= g.hi) return g.bins - 1;
    int i = (int)floor(__ddiv_rn(__dsub_rn(x, g.lo), g.h));
    i = max(0, min(i, g.bins - 1));
    while (i > 0 && x < edge(g, i)) --i;
    while (i < g.bins - 1 && x >= edge(g, i + 1)) ++i;
    return i;
}

// Bin of a float with binary32 arithmetic only.  thr[i] is the smallest float
// not below e_i, so for a float x: x < e_i  <=>  x < thr[i].  A first guess
// from one multiply is corrected by those exact comparisons.
__device__ __forceinline__ int bin_of_f32(const float* __restrict__ thr, int bins, float lo_f,
                                          float inv_h_f, float x)
{
    if (!(x >= thr[0])) return 0;
    if (x >= thr[bins]) return bins - 1;
    int i = __float2int_rd((x - lo_f) * inv_h_f);
    i = max(0, min(i, bins - 1));
    while (i > 0 && x < thr[i]) --i;
    while (i < bins - 1 && x >= thr[i + 1]) ++i;
    return i;
}

// Binary32 binning with a fast path that reads no threshold.  With
// c = -(lo_f inv_h_f + 1/2) (binary32), g = fma(x, inv_h_f, c) differs from
// the exact (x - lo) / h - 1/2 by less than
// 2^-24 (max(|lo|, |hi|) / h + 3 |lo| / h + bins + 4) for x within a bin of
// the grid (rounding of inv_h, of lo, of c and of the fma).  r = round(g)
// comes from the low mantissa bits of g + 1.5 * 2^23 (exact for |g| < 2^22;
// larger |g| gives an index outside [0, bins) or fails the test below).  When
// |g - r| <= 1/2 - margin, margin at least twice that bound, (x - lo) / h lies
// at least the bound away from every integer, so r = floor((x - lo) / h) is
// the exact bin.  Elsewhere (near an edge, outside the grid, NaN) the
// thresholds decide as in bin_of_f32; the result equals bin_of_f32's for
// every x, and the common case needs one fma, three adds and no conversion.
struct BinF32 {
    float lo, inv_h, c, thr0, thrI, half_m, h;
    int bins;
};

__device__ __forceinline__ BinF32 make_bin_f32(float thr0, float thrI, int bins, float lo_f, float inv_h_f)
{
    BinF32 b;
    b.lo = lo_f;
    b.inv_h = inv_h_f;
    b.h = __frcp_rn(inv_h_f);
    b.bins = bins;
    b.thr0 = thr0;
    b.thrI = thrI;
    b.c = -(lo_f * inv_h_f + 0.5f);
    const float span = fmaxf(fabsf(thr0), fabsf(thrI)) * inv_h_f;
    const float m = 1.25e-7f * (span + 3.0f * fabsf(lo_f) * inv_h_f + (float)bins + 4.0f);
    b.half_m = m < 0.25f ? 0.5f - m : -1.0f;   // -1: never take the fast path
    return b;
}

// After thr[] is complete and visible to the calling thread.
__device__ __forceinline__ BinF32 make_bin_f32(const float* thr, int bins, float lo_f, float inv_h_f)
{
    return make_bin_f32(thr[0], thr[bins], bins, lo_f, inv_h_f);
}

// The fast path alone: the bin, or -1 when the thresholds must decide.
__device__ __forceinline__ int bin_try_f32(const BinF32& b, float x)
{
    const float g = fmaf(x, b.inv_h, b.c);
    const float t = g + 12582912.0f;
    const float r = t - 12582912.0f;
    const float d = g - r;
    const int i = __float_as_int(t) - 0x4B400000;
    return ((unsigned)i < (unsigned)b.bins && fabsf(d) <= b.half_m) ? i : -1;
}

// Exact bin by comparison with the thresholds thr(i) (bin_of_f32's rule).
template <typename Thr>
__device__ __forceinline__ int bin_slow_f32(const BinF32& b, Thr thr, float x)
{
    if (!(x >= b.thr0)) return 0;
    if (x >= b.thrI) return b.bins - 1;
    int i = __float2int_rd((x - b.lo) * b.inv_h);
    i = max(0, min(i, b.bins - 1));
    while (i > 0 && x < thr(i)) --i;
    while (i < b.bins - 1 && x >= thr(i + 1)) ++i;
    return i;
}

__device__ __forceinline__ int bin_fast_f32(const BinF32& b, const float* __restrict__ thr, float x)
{
    const int i = bin_try_f32(b, x);
    if (i >= 0) return i;
    return bin_slow_f32(b, [thr](int k) { return thr[k]; }, x);
}

// bin_fast_f32, also giving the bin index as a float (taken from the fast
// path's rounding, which already holds it, else converted).
__device__ __forceinline__ int bin_fast_f32(const BinF32& b, const float* __restrict__ thr, float x, float& fi)
{
    const float g = fmaf(x, b.inv_h, b.c);
    const float t = g + 12582912.0f;
    const float r = t - 12582912.0f;
    const float d = g - r;
    const int i = __float_as_int(t) - 0x4B400000;
    if ((unsigned)i < (unsigned)b.bins && fabsf(d) <= b.half_m) {
        fi = r;
        return i;
    }
    const int k = bin_slow_f32(b, [thr](int q) { return thr[q]; }, x);
    fi = (float)k;
    return k;
}

// thr[i] for i = 0..bins, cooperatively by the block.
__device__ __forceinline__ void build_thresholds(const GridDev& g, float* thr)
{
    for (int i = threadIdx.x; i <= g.bins; i += blockDim.x) thr[i] = __double2float_ru(edge(g, i));
}

// The binary64 value of a binary32 number, built from its encoding on the
// integer units (exponent rebiased by 1023 - 127, mantissa moved up by 29
// bits) for normal numbers and zeros; subnormals, infinities and NaNs take
// the conversion instruction.  Exact either way.  On GB300 the conversion
// instruction occupies the narrow binary64 pipe.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e - 1u < 254u) {
        const uint32_t hi = (u & 0x80000000u) | (((u & 0x7FFFFFFFu) >> 3) + 0x38000000u);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
}

__device__ __forceinline__ double widen(double d) { return d; }

// Equality of two non-NaN doubles by their bits (+0 and -0 equal), on the
// integer units.
__device__ __forceinline__ bool deq(double a, double b)
{
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    return x == y || ((x | y) << 1) == 0;
}

// Exact ordering of non-negative doubles through their bit patterns.
__device__ __forceinline__ long long dkey(double v) { return __double_as_longlong(v); }

}  // namespace pr

// fine_dev.cuh -- the binary32 Euler-Maruyama loop (fast_dim = 1) over a
// range of particles of one slice, with the fused matching prologue and
// restriction epilogue; shared by the single-problem and the batched kernels
// so that both take the same steps bit for bit.
#pragma once

#include "match.cuh"
#include "pr_common.cuh"

namespace pr {

struct D1Consts {
    float lam, ddt, rel, sxk, syk;   // EM constants; sxk, syk include sqrt(2 ln 2)
    uint32_t k0, k1, chi;            // Philox key words and (problem_id << 8)
    ChemConsts<float> chem;          // the chemical system's constants (KIND == PR_MODEL_CHEM)
};

// One step of the d = 1 families from a Box-Muller pair (q, cos, sin).
template <int KIND>
__device__ __forceinline__ void em_step_d1(float& x, float& y, float q, float c, float s, const D1Consts& k)
{
    if (KIND == PR_MODEL_CHEM)
        em_step_chem_f32(x, y, q * k.sxk, c, q * k.syk, s, k.chem);
    else
        em_step_f32<KIND>(x, y, q * k.sxk, c, q * k.syk, s, k.lam, k.ddt, k.rel);
}

struct D1Smem {
    const float* thr;                // edge thresholds [bins+1]
    uint32_t* hist_s;                // restriction of the start state [bins]
    uint32_t* hist_e;                // restriction of the end state [bins]
    const MatchSmem* ms;             // matching table (when do_match)
    BinF32 bf;                       // binning constants (after thr is built)
    bool do_match, do_hs, do_he;
};

// Particles [p_begin, p_end) of slice `slice` (global index, keys the random
// numbers) in tiles of blockDim.x * PPT, PPT per thread strided by blockDim.x.
template <int KIND, int PPT>
__device__ __forceinline__ void fine_d1_range(const float* __restrict__ xin, const float* __restrict__ yin,
                                              float* __restrict__ xout, float* __restrict__ yout,
                                              int64_t p_begin, int64_t p_end, uint32_t slice, int steps,
                                              const D1Consts& c, const D1Smem& sm)
{
    const uint32_t k0 = c.k0, k1 = c.k1, chi = c.chi;
    const int pairs = steps >> 1;
    const int64_t tile = (int64_t)blockDim.x * PPT;
    for (int64_t t0 = p_begin; t0 < p_end; t0 += tile) {
        const int64_t base = t0 + threadIdx.x;
        float x[PPT], y[PPT];
        uint32_t pid[PPT];
        bool ok[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int64_t p = base + (int64_t)k * blockDim.x;
            ok[k] = p < p_end;
            pid[k] = (uint32_t)p;
            x[k] = ok[k] ? xin[p] : 0.0f;
            y[k] = ok[k] ? yin[p] : 0.0f;
        }
        if (sm.do_match) {
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (ok[k]) x[k] = match_one_f32(*sm.ms, sm.thr, sm.bf, x[k]);
        }
        if (sm.do_hs) {
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (ok[k]) atomicAdd(&sm.hist_s[bin_fast_f32(sm.bf, sm.thr, x[k])], 1u);
        }
        for (int mp = 0; mp < pairs; ++mp) {
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)mp, pid[k], slice, chi), k0, k1);
                float q0, c0, s0, q1, c1, s1;
                box_muller_qcs(w.x, w.y, q0, c0, s0);
                box_muller_qcs(w.z, w.w, q1, c1, s1);
                // steps 2 mp and 2 mp + 1: sx z0 = (q sxk) cos, sy z1 = (q syk) sin
                em_step_d1<KIND>(x[k], y[k], q0, c0, s0, c);
                em_step_d1<KIND>(x[k], y[k], q1, c1, s1, c);
            }
        }
        if (steps & 1) {
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)pairs, pid[k], slice, chi), k0, k1);
                float q0, c0, s0;
                box_muller_qcs(w.x, w.y, q0, c0, s0);
                em_step_d1<KIND>(x[k], y[k], q0, c0, s0, c);
            }
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (!ok[k]) continue;
            const int64_t p = base + (int64_t)k * blockDim.x;
            xout[p] = x[k];
            yout[p] = y[k];
            if (sm.do_he) atomicAdd(&sm.hist_e[bin_fast_f32(sm.bf, sm.thr, x[k])], 1u);
        }
    }
}

}  // namespace pr

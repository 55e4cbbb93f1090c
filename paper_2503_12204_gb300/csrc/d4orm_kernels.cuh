// d4orm_kernels.cuh -- device functions shared by the single-problem kernels
// and the batched persistent solver: the per-sample rollout + fitness of one
// lane segment, the one-warp iteration end (apply, rollout, verdict), and the
// block-wide batch softmax with weight compaction.
#pragma once

#include <cmath>

#include "d4orm_device.cuh"
#include "d4orm.h"

namespace d4orm {

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

template <bool MAX>
__device__ float block_reduce(float v, float* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = MAX ? warp_max(v) : warp_sum(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sh[lane] : (MAX ? -INFINITY : 0.0f);
        v = MAX ? warp_max(v) : warp_sum(v);
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    const float r = sh[32];
    __syncthreads();
    return r;
}

// Samples whose unnormalised weight exp(l_j - max l) falls below 2^-30
// are left out of the weighted sum: together they move it by at most
// N * 2^-30 * max|eps| relative to the largest weight (max|eps| <= 5.77 for
// the 24-bit Box-Muller inputs: under 4.5e-5 for N <= 8192 and 3.5e-4 for
// N <= 65536, against the 1e-3 tolerance of the update), and typically a
// large share of a batch is that far below the best sample, so the noise
// those samples would need is never regenerated.
constexpr float kLogWeightCut = -20.794415f;  // -30 ln 2

// ---------------------------------------------------------------------------
// Batch normalisation (Sec. IV-C) + temperature softmax (Eq. (6)) of the N
// rewards in `fitness` (global or shared memory), by the whole thread block:
// writes the ordered (weight, index) list of the samples that carry weight
// and its length.  sh[kSoftmaxScratch], scan[33]: shared scratch.  VR > 0
// keeps each thread's (at most VR) values in registers.
//
// Two block-wide rounds, two barriers each:
//  1. sum and sum of squares of r - r_0 (shifted by the first reward, so the
//     population variance E[(r - r_0)^2] - E[r - r_0]^2 loses no precision
//     to a large common offset) and the largest reward -- the largest logit
//     is that reward's, (r - mu) * scale being monotone in r;
//  2. the sum of exp(l - max l) and an exclusive scan of the per-thread
//     counts of weights at or above the cut, which places each thread's
//     survivors in the list.
// ---------------------------------------------------------------------------
constexpr int kSoftmaxScratch = 100;

template <int VR>
__device__ __noinline__ void softmax_block(const float* __restrict__ fitness, int N, float inv_lambda,
                                              float2* __restrict__ list, int* __restrict__ count,
                                              float* __restrict__ stats, float* sh, int* scan)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    // contiguous ranges keep the compacted list in sample order
    const int per = (N + nt - 1) / nt;
    const int j0 = min(N, tid * per), j1 = min(N, j0 + per);
    const int cnt = j1 - j0;
    constexpr int R = VR > 0 ? VR : 1;
    float r[R];
    if constexpr (VR > 0) {
#pragma unroll
        for (int i = 0; i < VR; ++i) r[i] = i < cnt ? fitness[j0 + i] : 0.0f;
    }
    // apply f to every value of this thread's range, in order
    auto each = [&](auto&& f) {
        if constexpr (VR > 0) {
#pragma unroll
            for (int i = 0; i < VR; ++i)
                if (i < cnt) f(i, r[i]);
        } else {
            for (int i = 0; i < cnt; ++i) f(i, fitness[j0 + i]);
        }
    };
    // round 1: shifted sum, shifted sum of squares, maximum
    const float r0 = fitness[0];
    float s1 = 0.0f, s2 = 0.0f, mx = -INFINITY;
    each([&](int, float x) {
        const float d = x - r0;
        s1 += d;
        s2 = fmaf(d, d, s2);
        mx = fmaxf(mx, x);
    });
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    mx = warp_max(mx);
    if (lane == 0) {
        sh[warp] = s1;
        sh[32 + warp] = s2;
        sh[64 + warp] = mx;
    }
    __syncthreads();
    if (warp == 0) {
        float a = lane < nw ? sh[lane] : 0.0f;
        float b = lane < nw ? sh[32 + lane] : 0.0f;
        float c = lane < nw ? sh[64 + lane] : -INFINITY;
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_max(c);
        if (lane == 0) {
            sh[96] = a;
            sh[97] = b;
            sh[98] = c;
        }
    }
    __syncthreads();
    const float inv_n = 1.0f / (float)N;
    const float dm = sh[96] * inv_n;
    const float mu = r0 + dm;
    const float sd = sqrtf(fmaxf(fmaf(-dm, dm, sh[97] * inv_n), 0.0f));
    mx = sh[98];
    const bool degenerate = !(sd > 1e-12f * fmaxf(1.0f, fabsf(mu)));
    const float scale = degenerate ? 0.0f : inv_lambda / sd;
    const float m = (mx - mu) * scale;
    // round 2: sum of exp(l - m) and the survivors' exclusive scan
    float z = 0.0f;
    int kept = 0;
    each([&](int, float x) {
        const float l = (x - mu) * scale - m;
        z += expf(l);
        kept += l >= kLogWeightCut ? 1 : 0;
    });
    z = warp_sum(z);
    int incl = kept;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o;
    }
    // the scratch of round 1 is free: every thread has read its results
    if (lane == 31) scan[warp] = incl;
    if (lane == 0) sh[warp] = z;
    __syncthreads();
    if (warp == 0) {
        const int t = lane < nw ? scan[lane] : 0;
        int ti = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(kFull, ti, off);
            if (lane >= off) ti += o;
        }
        const float zz = warp_sum(lane < nw ? sh[lane] : 0.0f);
        if (lane < nw) scan[lane] = ti - t;
        if (lane == 31) scan[32] = ti;
        if (lane == 0) sh[99] = zz;
    }
    __syncthreads();
    const float Z = sh[99];
    const float invZ = 1.0f / Z;
    int pos = scan[warp] + incl - kept;
    each([&](int i, float x) {
        const float l = (x - mu) * scale - m;
        if (l >= kLogWeightCut) list[pos++] = make_float2(expf(l) * invZ, __int_as_float(j0 + i));
    });
    if (tid == 0) {
        *count = scan[32];
        if (stats) {
            stats[0] = mu;
            stats[1] = sd;
            stats[2] = m;
            stats[3] = Z;
        }
    }
}

// ---------------------------------------------------------------------------
// One sample per aligned segment of SEG lanes (robot k = lane % SEG), all 32
// lanes of the warp calling together: Eq. (12) sample, Eq. (1) rollout and
// Eq. (3)-(5) fitness of sample j.  sM holds the mean controls
// M[t][k][d] = u_base + c_i dU_i.  Returns the sample's fitness (already
// divided by nT) on every lane of the segment.  Shared by the single-problem
// kernel and the batched solver.  OBS compiles in the obstacle penalty
// (problems without obstacles run the variant without it: a runtime loop
// in the unrolled time loop costs about 6 %).
// ---------------------------------------------------------------------------
template <int DYN, int SEG, bool OBS>
__device__ __forceinline__ float sample_fitness_segment(const DevProblem& P, const DevStep& S,
                                                        const float* __restrict__ sM, uint32_t c3, int j)
{
    using D = DynDims<DYN>;
    constexpr int DX = D::DX, DU = D::DU, DP = D::DP;
    const int lane = threadIdx.x & 31;
    const int k = lane & (SEG - 1);
    const int seg_base = lane & ~(SEG - 1);
    const bool robot = k < P.n;
    const int kr = robot ? k : P.n - 1;

    float x[DX];
    load_start<DYN>(x, P, k);
    // padding robots park far away and far apart, so no pair test involving
    // them can hit and the Eq. (5) test needs no validity mask
    if (!robot) {
#pragma unroll
        for (int d = 0; d < DP; ++d) x[d] = 1.0e15f * (float)(1 + k);
    }
    float g[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) g[d] = P.goal[kr * 3 + d];
    const float inv_d0 = P.inv_d0[kr];
    const float w_safe = S.w_safe;
    const int rowM = P.n * DU;
    const float* Mk = sM + kr * DU;
    float acc = 0.0f;
    // bit of the lane that tests pair (k - s, k), for s = 1..SEG/2 - 1
    uint32_t back[SEG / 2 > 1 ? SEG / 2 - 1 : 1];
#pragma unroll
    for (int s = 1; s < SEG / 2; ++s) back[s - 1] = (uint32_t)(seg_base + ((k - s) & (SEG - 1)));

    // one time step t with its noise eps[d]
    auto step = [&](int t, const float* eps) {
        float u[DU];
#pragma unroll
        for (int d = 0; d < DU; ++d)
            u[d] = clampf(fmaf(S.sigma, eps[d], Mk[t * rowM + d]), P.u_lo[d], P.u_hi[d]);
        integrate<DYN>(x, u, P);
        // Eq. (4): goal term, accumulated before the pair tests so that it
        // does not wait for their shuffle chain (on the latency-bound
        // unicycle workload this ordering took the kernel from 15.9 to
        // 15.0 us inside the solve's CUDA graph)
        float dg2 = 0.0f;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const float e = x[d] - g[d];
            dg2 = fmaf(e, e, dg2);
        }
        if (robot) acc += 1.0f - sqrt_approx(dg2) * inv_d0;
        // Eq. (5): any partner inside 2R+eps.  Each unordered pair is
        // evaluated once: lane k tests partner k+s (mod SEG) for
        // s = 1..SEG/2, and hands the result to the partner (for s = SEG/2
        // both lanes of the pair test it).  Up to 8 lanes a ballot hands
        // back the flag; with 16 lanes the partner receives the squared
        // distance itself by a shuffle and the test becomes "nearest partner
        // within 2R+eps" -- the same decision on the same binary32 values,
        // fewer instructions per offset (measured faster at 16 lanes,
        // slower at 8, where the per-step latency dominates).
        bool hit = false;
        if constexpr (SEG == 16) {
            float m = INFINITY;
#pragma unroll
            for (int s = 1; s <= SEG / 2; ++s) {
                const int src = seg_base + ((k + s) & (SEG - 1));
                float d2 = 0.0f;
#pragma unroll
                for (int d = 0; d < DP; ++d) {
                    const float e = x[d] - __shfl_sync(kFull, x[d], src);
                    d2 = fmaf(e, e, d2);
                }
                m = fminf(m, d2);
                if (2 * s != SEG) m = fminf(m, __shfl_sync(kFull, d2, seg_base + ((k - s) & (SEG - 1))));
            }
            hit = m <= P.thr2;
        } else {
#pragma unroll
            for (int s = 1; s <= SEG / 2; ++s) {
                const int src = seg_base + ((k + s) & (SEG - 1));
                float d2 = 0.0f;
#pragma unroll
                for (int d = 0; d < DP; ++d) {
                    const float e = x[d] - __shfl_sync(kFull, x[d], src);
                    d2 = fmaf(e, e, d2);
                }
                const bool h = d2 <= P.thr2;
                hit |= h;
                if (2 * s != SEG) {
                    const unsigned m = __ballot_sync(kFull, h);
                    hit |= (m >> back[s - 1]) & 1u;
                }
            }
        }
        if (robot && hit) acc -= w_safe;
        // Appendix: binary obstacle penalty with the same weight
        if constexpr (OBS)
            if (robot && obstacle_hit<DP>(P, x)) acc -= w_safe;
    };
    // the noise of four time steps, d_u Philox quads
    auto noise4 = [&](int t0, float* eps) {
        const uint32_t q0 = (uint32_t)(t0 * DU) >> 2;
#pragma unroll
        for (int c = 0; c < DU; ++c) noise_quad(S, c3, q0 + c, (uint32_t)j, (uint32_t)k, &eps[4 * c]);
    };

    const int T4 = P.T & ~3;
    for (int t0 = 0; t0 < T4; t0 += 4) {  // whole groups of four: no per-step bound test
        float eps[4 * DU];
        noise4(t0, eps);
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) step(t0 + tt, &eps[tt * DU]);
    }
    if (T4 < P.T) {  // ragged tail, uniform across the warp
        float eps[4 * DU];
        noise4(T4, eps);
#pragma unroll
        for (int tt = 0; tt < 3; ++tt)
            if (T4 + tt < P.T) step(T4 + tt, &eps[tt * DU]);
    }
    acc = seg_sum<SEG>(acc);
    return acc * P.inv_nT;
}

// ---------------------------------------------------------------------------
// Iteration end of Algorithm 2 on one warp (robots in lanes): u = clip(u_base
// + dU_0) (du0 nullable; u_out nullable, may alias u_base), rollout from S
// (states nullable, [T+1][n][d_x]), and the Eq. (1)/(2) verdict written by
// lane 0 to *verdict (nullable).
// ---------------------------------------------------------------------------
template <int DYN>
__device__ __forceinline__ void apply_rollout_verdict_warp(const DevProblem& P, float w_safe, const float* u_base,
                                                           const float* du0, float* u_out, float* states,
                                                           d4orm_verdict* verdict)
{
    using D = DynDims<DYN>;
    constexpr int DX = D::DX, DU = D::DU, DP = D::DP;
    const int k = threadIdx.x & 31;
    const bool robot = k < P.n;
    const int kr = robot ? k : P.n - 1;
    float x[DX];
    load_start<DYN>(x, P, k);
    float g[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) g[d] = P.goal[kr * 3 + d];
    const float inv_d0 = P.inv_d0[kr];

    auto pair_min = [&](float cur) {
        float m = cur;
        for (int s = 1; s < 32; ++s) {
            float d2 = 0.0f;
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                const float e = x[d] - __shfl_xor_sync(kFull, x[d], s);
                d2 = fmaf(e, e, d2);
            }
            if (((k ^ s) < P.n) && robot) m = fminf(m, d2);
        }
        return m;
    };
    if (states && robot)
        for (int c = 0; c < DX; ++c) states[(size_t)k * DX + c] = x[c];
    float min_d2 = pair_min(INFINITY);
    float obs_clear = robot ? obstacle_clearance<DP>(P, x) : INFINITY;
    float acc = 0.0f;
    int at_goal = 0;
    float dg2 = 0.0f;
    for (int t = 0; t < P.T; ++t) {
        float u[DU];
#pragma unroll
        for (int d = 0; d < DU; ++d) {
            const size_t idx = ((size_t)t * P.n + kr) * DU + d;
            const float v = clampf(u_base[idx] + (du0 ? du0[idx] : 0.0f), P.u_lo[d], P.u_hi[d]);
            u[d] = v;
            if (u_out && robot) u_out[idx] = v;
        }
        integrate<DYN>(x, u, P);
        if (states && robot)
            for (int c = 0; c < DX; ++c) states[((size_t)(t + 1) * P.n + k) * DX + c] = x[c];
        dg2 = 0.0f;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const float e = x[d] - g[d];
            dg2 = fmaf(e, e, dg2);
        }
        bool hit = false;
        float m = INFINITY;
        for (int s = 1; s < 32; ++s) {
            float d2 = 0.0f;
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                const float e = x[d] - __shfl_xor_sync(kFull, x[d], s);
                d2 = fmaf(e, e, d2);
            }
            if ((k ^ s) < P.n) {
                hit |= d2 <= P.thr2;
                m = fminf(m, d2);
            }
        }
        if (robot) {
            min_d2 = fminf(min_d2, m);
            obs_clear = fminf(obs_clear, obstacle_clearance<DP>(P, x));
            const bool obs = obstacle_hit<DP>(P, x);
            acc += (1.0f - sqrtf(dg2) * inv_d0) - (hit ? w_safe : 0.0f) - (obs ? w_safe : 0.0f);
            at_goal += dg2 <= P.tol2 ? 1 : 0;
        }
    }
    int reached = (!robot || dg2 <= P.tol2) ? 1 : 0;
    float acc_s = acc;
    int goal_s = at_goal;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc_s += __shfl_xor_sync(kFull, acc_s, off);
        goal_s += __shfl_xor_sync(kFull, goal_s, off);
        min_d2 = fminf(min_d2, __shfl_xor_sync(kFull, min_d2, off));
        obs_clear = fminf(obs_clear, __shfl_xor_sync(kFull, obs_clear, off));
        reached &= __shfl_xor_sync(kFull, reached, off);
    }
    if (k == 0) {
        if (verdict) {
            d4orm_verdict v;
            v.collision_free = ((P.n < 2 || min_d2 > P.safe2) && obs_clear > 0.0f) ? 1 : 0;
            v.goal_reached = reached;
            v.reward = acc_s * P.inv_nT;
            v.objective = (float)goal_s * P.inv_nT;
            v.min_pair_dist = P.n < 2 ? 1e30f : sqrtf(min_d2);
            *verdict = v;
        }
    }
}

}  // namespace d4orm

// d4orm_paired.cuh -- the per-sample rollout + fitness with two robots per
// lane, for batches large enough that halving the number of warps still
// keeps every scheduler busy (the 16-robot 3D workload: 2048 warps).
//
// Same arithmetic as sample_fitness_segment (Eq. (12) samples, Eq. (1)
// rollout, Eq. (3)-(5) fitness), laid out differently: a sample occupies an
// aligned segment of L lanes, lane a holding robots a and a + L.  The two
// robots' values of each state component share one 64-bit register, so the
// control update, the holonomic integration, the goal term and every pair
// distance run as packed f32x2 instructions (fma/add/sub/mul.rn.f32x2,
// sm_100+): one issue slot for two robots.
//
// Eq. (5) indicator: a robot is penalised when its nearest partner lies
// within 2R + eps, i.e. when the smallest squared pair distance is at most
// (2R + eps)^2 -- the same decision, on the same binary32 distances, as
// testing every partner.  Each unordered pair is evaluated once: lane a
// takes its own pair and the robot pairs of lanes a + s (mod L) for
// s = 1..L/2, and returns the minima it found for the partner's robots to
// lane a + s with one shuffle (for s = L/2 both lanes of a pair evaluate it).
// The partners' positions come from a per-warp shared-memory buffer that
// every lane writes once per step: one 64-bit load brings both robots of a
// partner lane already packed, where shuffles need two per coordinate and
// a repack (with shuffles the stand-alone kernel took 87.2 us instead of
// 86.5 on the 16-robot 3D workload, and the batched solver ran 167.7
// instead of 170.2 M sample-rollouts/s on 512 ragged teams).
#pragma once

#include "d4orm_kernels.cuh"

namespace d4orm {

// Two binary32 values in one 64-bit register: lo = robot a, hi = robot a + L.
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(f2 v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f2_hi(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 f2_clamp(f2 v, float lo, float hi)
{
    return f2_pack(clampf(f2_lo(v), lo, hi), clampf(f2_hi(v), lo, hi));
}
// xbuf: this warp's position buffer in shared memory, 2 x DP x 32 packed
// pairs (double-buffered by step parity), 8-byte aligned.
template <int DYN, int L, bool OBS>
__device__ __forceinline__ float sample_fitness_paired(const DevProblem& P, const DevStep& S,
                                                       const float* __restrict__ sM, uint32_t c3, int j,
                                                       f2* __restrict__ xbuf)
{
    using D = DynDims<DYN>;
    constexpr int DX = D::DX, DU = D::DU, DP = D::DP;
    constexpr bool HOLO = DYN == HOLO2D || DYN == HOLO3D;
    const int lane = threadIdx.x & 31;
    const int a = lane & (L - 1);
    const int seg_base = lane & ~(L - 1);
    const int k0 = a, k1 = a + L;
    const bool real0 = k0 < P.n, real1 = k1 < P.n;
    const int kr0 = real0 ? k0 : P.n - 1, kr1 = real1 ? k1 : P.n - 1;

    // state component c of both robots; padding robots park far away and
    // far apart, so no pair test involving them can hit
    f2 x[DX];
    {
        float s0[DX], s1[DX];
        load_start<DYN>(s0, P, k0);
        load_start<DYN>(s1, P, k1);
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            if (!real0) s0[d] = 1.0e15f * (float)(1 + k0);
            if (!real1) s1[d] = 1.0e15f * (float)(1 + k1);
        }
#pragma unroll
        for (int c = 0; c < DX; ++c) x[c] = f2_pack(s0[c], s1[c]);
    }
    f2 g[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) g[d] = f2_pack(P.goal[kr0 * 3 + d], P.goal[kr1 * 3 + d]);
    const f2 neg_inv_d0 = f2_pack(-P.inv_d0[kr0], -P.inv_d0[kr1]);
    const f2 mask = f2_pack(real0 ? 1.0f : 0.0f, real1 ? 1.0f : 0.0f);
    const f2 one2 = f2_pack(1.0f, 1.0f);
    const f2 sigma2 = f2_pack(S.sigma, S.sigma);
    const f2 dt2 = f2_pack(P.dt, P.dt), half_dt2 = f2_pack(P.half_dt2, P.half_dt2);
    const float* M0 = sM + kr0 * DU;
    const float* M1 = sM + kr1 * DU;
    const int rowM = P.n * DU;
    f2 acc = f2_pack(0.0f, 0.0f);
    float hits = 0.0f;  // penalised robot-steps (Eq. (5) and the obstacle term), real robots only

    auto step = [&](int t, const float* e0, const float* e1) {
        // Eq. (12) sample, clipped to the control box
        f2 u[DU];
#pragma unroll
        for (int d = 0; d < DU; ++d)
            u[d] = f2_clamp(f2_fma(sigma2, f2_pack(e0[d], e1[d]), f2_pack(M0[t * rowM + d], M1[t * rowM + d])),
                            P.u_lo[d], P.u_hi[d]);
        // Eq. (1): one integration step of both robots
        if constexpr (HOLO) {
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                x[d] = P.integ == 1 ? f2_fma(x[DP + d], dt2, f2_fma(half_dt2, u[d], x[d])) : f2_fma(x[DP + d], dt2, x[d]);
                x[DP + d] = f2_clamp(f2_fma(u[d], dt2, x[DP + d]), -P.v_max, P.v_max);
            }
        } else {
            float s0[DX], s1[DX], u0[DU], u1[DU];
#pragma unroll
            for (int c = 0; c < DX; ++c) {
                s0[c] = f2_lo(x[c]);
                s1[c] = f2_hi(x[c]);
            }
#pragma unroll
            for (int d = 0; d < DU; ++d) {
                u0[d] = f2_lo(u[d]);
                u1[d] = f2_hi(u[d]);
            }
            integrate<DYN>(s0, u0, P);
            integrate<DYN>(s1, u1, P);
#pragma unroll
            for (int c = 0; c < DX; ++c) x[c] = f2_pack(s0[c], s1[c]);
        }
        // Eq. (4): goal term of both robots
        f2 dg2;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const f2 e = f2_sub(x[d], g[d]);
            dg2 = d == 0 ? f2_mul(e, e) : f2_fma(e, e, dg2);
        }
        const f2 dist = f2_pack(sqrt_approx(f2_lo(dg2)), sqrt_approx(f2_hi(dg2)));
        acc = f2_fma(mask, f2_fma(dist, neg_inv_d0, one2), acc);
        // Eq. (5): nearest partner of each robot
        float m0, m1;
        {
            float d2 = 0.0f;
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                const float e = f2_lo(x[d]) - f2_hi(x[d]);
                d2 = fmaf(e, e, d2);
            }
            m0 = d2;
            m1 = d2;
        }
        // own positions to the buffer of this step's parity; the lane's
        // two robots swapped once, so that (k1, k0) - (p0, p1) gives the
        // cross pairs of every offset
        f2* buf = xbuf + (t & 1) * (DP * 32);
        f2 xs[DP];
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            buf[d * 32 + lane] = x[d];
            xs[d] = f2_pack(f2_hi(x[d]), f2_lo(x[d]));
        }
        __syncwarp();
#pragma unroll
        for (int s = 1; s <= L / 2; ++s) {
            const int src = seg_base + ((a + s) & (L - 1));
            f2 dd, dx;  // (k0, p0), (k1, p1) and (k1, p0), (k0, p1)
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                const f2 q = buf[d * 32 + src];
                const f2 e = f2_sub(x[d], q), es = f2_sub(xs[d], q);
                dd = d == 0 ? f2_mul(e, e) : f2_fma(e, e, dd);
                dx = d == 0 ? f2_mul(es, es) : f2_fma(es, es, dx);
            }
            m0 = fminf(m0, fminf(f2_lo(dd), f2_hi(dx)));
            m1 = fminf(m1, fminf(f2_hi(dd), f2_lo(dx)));
            if (2 * s != L) {
                // the partner lane's minima over this lane's two robots
                const float p0 = fminf(f2_lo(dd), f2_lo(dx));
                const float p1 = fminf(f2_hi(dd), f2_hi(dx));
                const int back = seg_base + ((a - s) & (L - 1));
                m0 = fminf(m0, __shfl_sync(kFull, p0, back));
                m1 = fminf(m1, __shfl_sync(kFull, p1, back));
            }
        }
        float h = (real0 && m0 <= P.thr2 ? 1.0f : 0.0f) + (real1 && m1 <= P.thr2 ? 1.0f : 0.0f);
        // Appendix: binary obstacle penalty with the same weight
        if constexpr (OBS) {
            float p0[DP], p1[DP];
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                p0[d] = f2_lo(x[d]);
                p1[d] = f2_hi(x[d]);
            }
            h += (real0 && obstacle_hit<DP>(P, p0) ? 1.0f : 0.0f) + (real1 && obstacle_hit<DP>(P, p1) ? 1.0f : 0.0f);
        }
        hits += h;
    };
    // the noise of four time steps of both robots, d_u Philox quads each
    auto noise4 = [&](int t0, float* e0, float* e1) {
        const uint32_t q0 = (uint32_t)(t0 * DU) >> 2;
#pragma unroll
        for (int c = 0; c < DU; ++c) {
            noise_quad(S, c3, q0 + c, (uint32_t)j, (uint32_t)k0, &e0[4 * c]);
            noise_quad(S, c3, q0 + c, (uint32_t)j, (uint32_t)k1, &e1[4 * c]);
        }
    };

    const int T4 = P.T & ~3;
    for (int t0 = 0; t0 < T4; t0 += 4) {  // whole groups of four: no per-step bound test
        float e0[4 * DU], e1[4 * DU];
        noise4(t0, e0, e1);
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) step(t0 + tt, &e0[tt * DU], &e1[tt * DU]);
    }
    if (T4 < P.T) {  // ragged tail, uniform across the warp
        float e0[4 * DU], e1[4 * DU];
        noise4(T4, e0, e1);
#pragma unroll
        for (int tt = 0; tt < 3; ++tt)
            if (T4 + tt < P.T) step(T4 + tt, &e0[tt * DU], &e1[tt * DU]);
    }
    float total = f2_lo(acc) + f2_hi(acc) - S.w_safe * hits;
    total = seg_sum<L>(total);
    return total * P.inv_nT;
}

}  // namespace d4orm

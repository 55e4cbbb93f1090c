// d4orm_device.cuh -- device-side building blocks of the D4orm step kernels:
// the by-value problem/step constants, Philox4x32-10, Box-Muller, the
// dynamics integrators and warp helpers.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace d4orm {

constexpr int kMaxRobots = 32;
constexpr int kMaxObstacles = 16;
constexpr unsigned kFull = 0xffffffffu;

enum Dyn : int { HOLO2D = 0, HOLO3D = 1, UNICYCLE = 2, DIFFDRIVE4 = 3 };

template <int DYN> struct DynDims;
template <> struct DynDims<HOLO2D>     { static constexpr int DX = 4, DU = 2, DP = 2; };
template <> struct DynDims<HOLO3D>     { static constexpr int DX = 6, DU = 3, DP = 3; };
template <> struct DynDims<UNICYCLE>   { static constexpr int DX = 3, DU = 2, DP = 2; };
template <> struct DynDims<DIFFDRIVE4> { static constexpr int DX = 4, DU = 2, DP = 2; };

// Problem constants, passed by value as a kernel parameter (constant bank):
// no device allocation is needed for a problem.
struct DevProblem {
    int n, T, dyn, integ;     // integ: 0 Euler, 1 RK4
    int d_x, d_u, d_p;
    int Q;                    // Philox quads per robot stream: ceil(T*d_u/4)
    float dt, half_dt2, dt6;  // dt, dt^2/2, dt/6
    float v_max;              // +inf when unbounded
    float thr2;               // (2 R_a + eps)^2  : Eq. (5) penalty radius
    float safe2;              // (2 R_a)^2        : Eq. (1) safety
    float tol2;               // goal_tol^2       : terminal condition
    float inv_nT;             // 1 / (n T)        : Eq. (3) normaliser
    float u_lo[3], u_hi[3];
    float start[kMaxRobots * 6];
    float goal[kMaxRobots * 3];   // goal positions
    float inv_d0[kMaxRobots];     // 1 / max(|p0 - g|, R_a)  (Eq. (4))
    // spherical obstacles (Appendix): centres, penalty radius^2 (r_o + R_a + eps)^2,
    // safety radius^2 (r_o + R_a)^2
    int n_obs;
    float obs_c[kMaxObstacles * 3];
    float obs_pen2[kMaxObstacles];
    float obs_safe2[kMaxObstacles];
};

// Appendix obstacle term: does the robot at position p lie within the
// penalty radius of any obstacle?
template <int DP>
__device__ __forceinline__ bool obstacle_hit(const DevProblem& P, const float* p)
{
    bool h = false;
    for (int o = 0; o < P.n_obs; ++o) {
        float d2 = 0.0f;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const float e = p[d] - P.obs_c[o * 3 + d];
            d2 = fmaf(e, e, d2);
        }
        h |= d2 <= P.obs_pen2[o];
    }
    return h;
}

// Smallest (d^2 - safety radius^2) over obstacles; > 0 means clear.
template <int DP>
__device__ __forceinline__ float obstacle_clearance(const DevProblem& P, const float* p)
{
    float m = INFINITY;
    for (int o = 0; o < P.n_obs; ++o) {
        float d2 = 0.0f;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const float e = p[d] - P.obs_c[o * 3 + d];
            d2 = fmaf(e, e, d2);
        }
        m = fminf(m, d2 - P.obs_safe2[o]);
    }
    return m;
}

// Per-step constants of step i in iteration it.
struct DevStep {
    uint32_t key0, key1;      // Philox key (seed lo, hi)
    uint32_t rk0[10], rk1[10];// Philox round keys: key + r * Weyl constant
    uint32_t c2_step;         // step_i << 8 (robot index fills the low byte)
    uint32_t c3_tag;          // tag << 12   (iteration fills the low 12 bits)
    int it;                   // iteration (used when no device counter given)
    int N;                    // samples
    float c;                  // 1 / sqrt(abar_i)
    float sigma;              // sqrt(1 / abar_i - 1)
    float g;                  // sqrt(abar_{i-1})
    float w_safe;             // w of Eq. (3)
    float inv_lambda;         // 1 / lambda of Eq. (6)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// 4x32 bijection with multipliers 0xD2511F53 / 0xCD9E8D57 and a Weyl key
// schedule 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox_round(U4 c, uint32_t k0, uint32_t k1)
{
    // one 32x32 -> 64 wide multiply per product: high and low words together
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    return U4{(uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0};
}

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        c = philox_round(c, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Same function with the ten round keys precomputed on the host (uniform
// kernel parameters: the key schedule costs no instructions per call).
__device__ __forceinline__ U4 philox4x32_10(U4 c, const DevStep& S)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) c = philox_round(c, S.rk0[r], S.rk1[r]);
    return c;
}

// Square root on the special-function unit (relative error ~2^-23): used
// for the Eq. (4) distance, which enters a sum checked to 1e-3.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Box-Muller: u1 = ((a >> 8) + 1) 2^-24 in (0, 1], u2 = (b >> 8) 2^-24 in
// [0, 1) (both exact in binary32); z0 = r cos(2 pi u2), z1 = r sin(2 pi u2),
// r = sqrt(-2 ln u1).  Evaluated on the special-function unit: r^2 =
// -2 ln 2 log2(u1) (hardware log2, absolute error <= 2^-22 on [0.5, 2], 2 ulp
// elsewhere), approximate square root, and sin/cos of the angle shifted to
// [-pi, pi) (2 pi u2 - pi; hardware sin/cos, absolute error <= 2^-21.41
// there), with the signs flipped back.  Resulting bound on each normal:
// |dz| <= 1e-6 r + min(2e-7 / r, 6e-4) -- a few 1e-7 for typical r, and at
// most 6e-4 in the rare draws with r below 1e-3 -- far inside the rollout
// and update tolerances.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1)
{
    const float u1 = (float)((a >> 8) + 1u) * 0x1.0p-24f;
    const float r = sqrt_approx(fmaxf(-1.3862943611198906f * __log2f(u1), 0.0f));
    const float ang = ((float)(b >> 8) * 0x1.0p-24f - 0.5f) * 6.283185307179586f;
    float s, c;
    __sincosf(ang, &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}

// Four standard normals: elements 4q..4q+3 of robot k's stream of sample j.
__device__ __forceinline__ void noise_quad(const DevStep& S, uint32_t c3, uint32_t q, uint32_t j, uint32_t k,
                                           float z[4])
{
    const U4 w = philox4x32_10(U4{q, j, (k & 0xffu) | S.c2_step, c3}, S);
    box_muller(w.x, w.y, z[0], z[1]);
    box_muller(w.z, w.w, z[2], z[3]);
}

__device__ __forceinline__ uint32_t iter_word(const DevStep& S, const int* it_dev)
{
    const int it = it_dev ? *it_dev : S.it;
    return (uint32_t)it | S.c3_tag;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// Device-wide nanosecond clock.
__device__ __forceinline__ long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// sin/cos of an arbitrary heading: Cody-Waite reduction by 2*pi (Cody and
// Waite, 1980; 2*pi split into 6.28125 + a binary32 tail, the first part
// with few enough bits that k * 6.28125 is exact), then the hardware
// sin/cos on [-pi, pi] (absolute error below 4e-7 there).
__device__ __forceinline__ void sincos_heading(float th, float* s, float* c)
{
    const float k = rintf(th * 0.15915494309189535f);
    float r = fmaf(-k, 6.28125f, th);
    r = fmaf(-k, 1.9353071795864769e-3f, r);
    __sincosf(r, s, c);
}

// ---------------------------------------------------------------------------
// One integration step (Sec. III Eq. (1) feasibility; dynamics of Sec. V).
// RK4 with the control held over the step is evaluated in closed form:
//  * double integrator: RK4 is exact, p += v dt + a dt^2/2, v += a dt;
//  * unicycle: theta is linear in time, so the four stages only need the
//    headings theta, theta + h, theta + 2h (h = omega dt / 2):
//    p += dt/6 v [c(theta) + 4 c(theta+h) + c(theta+2h)];
//  * differential drive: the same three headings with the stage speeds
//    v, v + a dt/2, v + a dt.
// The speed bound is applied after the step.
// ---------------------------------------------------------------------------
template <int DYN>
__device__ __forceinline__ void integrate(float* x, const float* u, const DevProblem& P)
{
    if constexpr (DYN == HOLO2D || DYN == HOLO3D) {
        constexpr int DP = DynDims<DYN>::DP;
        if (P.integ == 1) {
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                x[d] = fmaf(x[DP + d], P.dt, fmaf(P.half_dt2, u[d], x[d]));
                x[DP + d] = clampf(fmaf(u[d], P.dt, x[DP + d]), -P.v_max, P.v_max);
            }
        } else {
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                x[d] = fmaf(x[DP + d], P.dt, x[d]);
                x[DP + d] = clampf(fmaf(u[d], P.dt, x[DP + d]), -P.v_max, P.v_max);
            }
        }
    } else if constexpr (DYN == UNICYCLE) {
        const float v = u[0], w = u[1];
        float s0, c0;
        sincos_heading(x[2], &s0, &c0);
        if (P.integ == 1) {
            float sh, ch;
            sincos_heading(0.5f * w * P.dt, &sh, &ch);
            const float c1 = c0 * ch - s0 * sh, s1 = s0 * ch + c0 * sh;
            const float c2 = c1 * ch - s1 * sh, s2 = s1 * ch + c1 * sh;
            const float k = P.dt6 * v;
            x[0] = fmaf(k, c0 + 4.0f * c1 + c2, x[0]);
            x[1] = fmaf(k, s0 + 4.0f * s1 + s2, x[1]);
        } else {
            x[0] = fmaf(P.dt * v, c0, x[0]);
            x[1] = fmaf(P.dt * v, s0, x[1]);
        }
        x[2] = fmaf(w, P.dt, x[2]);
    } else {  // DIFFDRIVE4: x = [px, py, theta, v], u = [omega, a]
        const float w = u[0], a = u[1], v = x[3];
        float s0, c0;
        sincos_heading(x[2], &s0, &c0);
        if (P.integ == 1) {
            float sh, ch;
            sincos_heading(0.5f * w * P.dt, &sh, &ch);
            const float c1 = c0 * ch - s0 * sh, s1 = s0 * ch + c0 * sh;
            const float c2 = c1 * ch - s1 * sh, s2 = s1 * ch + c1 * sh;
            const float vm = fmaf(0.5f * P.dt, a, v), ve = fmaf(P.dt, a, v);
            x[0] = fmaf(P.dt6, v * c0 + 4.0f * vm * c1 + ve * c2, x[0]);
            x[1] = fmaf(P.dt6, v * s0 + 4.0f * vm * s1 + ve * s2, x[1]);
        } else {
            x[0] = fmaf(P.dt * v, c0, x[0]);
            x[1] = fmaf(P.dt * v, s0, x[1]);
        }
        x[2] = fmaf(w, P.dt, x[2]);
        x[3] = clampf(fmaf(a, P.dt, v), -P.v_max, P.v_max);
    }
}

template <int DYN>
__device__ __forceinline__ void load_start(float* x, const DevProblem& P, int k)
{
    constexpr int DX = DynDims<DYN>::DX;
    const int kk = k < P.n ? k : P.n - 1;
#pragma unroll
    for (int c = 0; c < DX; ++c) x[c] = P.start[kk * DX + c];
}

// M = base + c dU into shared memory by the whole CTA.  Every thread issues
// up to four 128-bit loads of each input before it stores, so the array
// arrives in one or two round trips to L2 instead of one per element; a
// scalar tail covers lengths that are not a multiple of four, and unaligned
// inputs take the scalar path.  NC: the inputs are read-only for the whole
// kernel, so the non-coherent read path may be used.
template <bool NC>
__device__ __forceinline__ float ld_in(const float* p)
{
    if constexpr (NC) return __ldg(p);
    else return *p;
}
template <bool NC>
__device__ __forceinline__ float4 ld_in4(const float4* p)
{
    if constexpr (NC) return __ldg(p);
    else return *p;
}

template <bool NC>
__device__ __forceinline__ void stage_mean(float* sM, const float* du, const float* base, float c, int total)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool vec = ((((uintptr_t)du) | ((uintptr_t)base) | ((uintptr_t)sM)) & 15u) == 0;
    if (!vec) {
        for (int e = tid; e < total; e += nt) sM[e] = fmaf(c, ld_in<NC>(du + e), ld_in<NC>(base + e));
        return;
    }
    const int n4 = total >> 2;
    const float4* d4 = reinterpret_cast<const float4*>(du);
    const float4* b4 = reinterpret_cast<const float4*>(base);
    float4* m4 = reinterpret_cast<float4*>(sM);
    for (int e0 = tid; e0 < n4; e0 += 4 * nt) {
        float4 a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = e0 + r * nt;
            if (e < n4) {
                a[r] = ld_in4<NC>(d4 + e);
                b[r] = ld_in4<NC>(b4 + e);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = e0 + r * nt;
            if (e < n4)
                m4[e] = make_float4(fmaf(c, a[r].x, b[r].x), fmaf(c, a[r].y, b[r].y), fmaf(c, a[r].z, b[r].z),
                                    fmaf(c, a[r].w, b[r].w));
        }
    }
    for (int e = 4 * n4 + tid; e < total; e += nt) sM[e] = fmaf(c, ld_in<NC>(du + e), ld_in<NC>(base + e));
}

// Warp-wide sums within aligned segments of SEG lanes.
template <int SEG>
__device__ __forceinline__ float seg_sum(float v)
{
#pragma unroll
    for (int off = SEG / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

}  // namespace d4orm

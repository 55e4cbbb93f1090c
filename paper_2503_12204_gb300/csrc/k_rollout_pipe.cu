// k_rollout_pipe.cu -- K2p, the warp-specialised rollout + fitness kernel
// for batches too small to fill the GPU with the register kernel (K2).
//
// Computes exactly what K2 computes (Eq. (12) samples, Eq. (1) rollout,
// Eq. (3)-(5) fitness) for the 32/SEG samples of one rollout warp, but only
// the dynamics recurrence stays on that warp.  The horizon is cut into
// chunks of CT steps and the CTA runs a three-stage software pipeline with
// one CTA barrier per stage:
//
//   helper warps : Philox noise + clipped controls of chunk c   -> U[c % 2]
//                  Eq. (4)/(5) terms of chunk c - 2 from Pos[(c - 2) % 2]
//   rollout warp : integrate chunk c - 1 from U[(c - 1) % 2]    -> Pos[(c - 1) % 2]
//
// so noise generation and the O(n^2) pair tests (both independent along
// time) run on the helpers while the recurrence advances.  There are
// CT * d_u / 4 helper warps: each helper lane owns one (sample, robot) pair
// and generates exactly one Philox quad of it per chunk, and scores the
// time steps h, h + H, ... of the chunk.  Per-row sums (one row = one sample
// at one time step) are reduced inside lane segments in a fixed order and
// added per sample at the end, so the result is deterministic.
//
// Shared memory: positions Pos[2][CT][SPC][SEG][PD] (PD = 2 in the plane,
// 4 in space, so a partner pair or a 3D position is one 128-bit load; rows
// are not padded: every warp access pattern below is conflict-free), the
// controls U[2][CT][SPC][n][d_u], the mean controls M = u_base + c dU
// [T][n][d_u] and the per-row terms [SPC][T].  Lanes of padding robots
// (k >= n) store a far-away sentinel position, so the Eq. (5) indicator of
// a real robot is "at least two robots (itself included) within 2R + eps".
#include <cmath>
#include <cstdint>

#include "d4orm_internal.h"

namespace d4orm {

constexpr int kPipeCT = 16;  // time steps per chunk (a multiple of 4: chunks are Philox-quad aligned)

template <int SEG, int DU>
struct PipeShape {
    static constexpr int SPC = 32 / SEG;                   // samples per CTA
    static constexpr int HELPERS = kPipeCT * DU / 4;       // helper warps: one quad per lane per chunk
    static constexpr int THREADS = 32 * (1 + HELPERS);
};

template <int DP>
struct PosSlot { static constexpr int PD = DP == 2 ? 2 : 4; };  // floats per robot position

template <int DYN, int SEG>
size_t pipe_smem_bytes(const DevProblem& P)
{
    using D = DynDims<DYN>;
    constexpr int SPC = PipeShape<SEG, D::DU>::SPC;
    const size_t pos = 2ull * kPipeCT * SPC * SEG * PosSlot<D::DP>::PD;
    const size_t u = 2ull * kPipeCT * SPC * P.n * D::DU;
    const size_t mean = (size_t)P.T * P.n * D::DU;
    const size_t rows = (size_t)SPC * P.T;
    return (pos + u + mean + rows) * sizeof(float);
}

template <int DYN, int SEG, bool OBS>
__global__ void __launch_bounds__(PipeShape<SEG, DynDims<DYN>::DU>::THREADS)
k_rollout_fitness_pipe(const DevProblem P, const DevStep S, const float* __restrict__ u_base,
                       const float* __restrict__ du_in, float* __restrict__ fitness, const int* __restrict__ it_dev)
{
    using D = DynDims<DYN>;
    constexpr int DX = D::DX, DU = D::DU, DP = D::DP;
    constexpr int SPC = PipeShape<SEG, DU>::SPC;
    constexpr int H = PipeShape<SEG, DU>::HELPERS;
    constexpr int CT = kPipeCT;
    constexpr int QPC = CT * DU / 4;                       // quads per robot per chunk (= H)
    constexpr int PD = PosSlot<DP>::PD;
    constexpr int RS = SEG * PD;                           // floats per position row
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    const int n = P.n, T = P.T;
    const int rowM = n * DU;
    float* sPos = smem;                                    // [2][CT][SPC][SEG][PD]
    float* sU = sPos + 2 * CT * SPC * RS;                  // [2][CT][SPC][n][DU]
    float* sM = sU + 2 * CT * SPC * rowM;                  // [T][n][DU]
    float* sRows = sM + T * rowM;                          // [SPC][T]
    const int pos_slot = CT * SPC * RS;
    const int u_slot = CT * SPC * rowM;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j_base = blockIdx.x * SPC;
    const uint32_t c3 = iter_word(S, it_dev);
    const int nchunks = (T + CT - 1) / CT;
    stage_mean<true>(sM, du_in, u_base, S.c, T * rowM);
    __syncthreads();

    // every lane owns one (sample, robot) pair: s = lane / SEG, k = lane % SEG
    const int k = lane & (SEG - 1);
    const int s = lane / SEG;
    const bool robot = k < n;
    const int kr = robot ? k : n - 1;

    // rollout-warp state
    float x[DX];
    load_start<DYN>(x, P, k);
    const float far = 1.0e15f * (float)(1 + k);   // padding robots park far away and far apart
    // helper constants: control box, Philox counter words, goal, Eq. (4) normaliser
    const int h = warp - 1;
    float lo[DU], hi[DU];
#pragma unroll
    for (int d = 0; d < DU; ++d) {
        lo[d] = P.u_lo[d];
        hi[d] = P.u_hi[d];
    }
    const uint32_t c2 = ((uint32_t)k & 0xffu) | S.c2_step;
    const uint32_t jj = (uint32_t)(j_base + s);
    float g[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) g[d] = P.goal[kr * 3 + d];
    const float inv_d0 = P.inv_d0[kr];

    for (int c = 0; c < nchunks + 2; ++c) {
        if (warp == 0) {
            // ---------------- rollout warp: integrate chunk c - 1
            if (c >= 1 && c <= nchunks) {
                const int cr = c - 1;
                const float* U = sU + (cr & 1) * u_slot;
                float* Pos = sPos + (cr & 1) * pos_slot;
                const int steps = min(CT, T - cr * CT);
#pragma unroll 4
                for (int tl = 0; tl < steps; ++tl) {
                    float u[DU];
                    const float* ur = U + (tl * SPC + s) * rowM + kr * DU;
                    if constexpr (DU == 2) {
                        const float2 v = *reinterpret_cast<const float2*>(ur);
                        u[0] = v.x;
                        u[1] = v.y;
                    } else {
#pragma unroll
                        for (int d = 0; d < DU; ++d) u[d] = ur[d];
                    }
                    integrate<DYN>(x, u, P);
                    float* pr = Pos + (tl * SPC + s) * RS + k * PD;
                    if constexpr (PD == 2)
                        *reinterpret_cast<float2*>(pr) = robot ? make_float2(x[0], x[1]) : make_float2(far, far);
                    else
                        *reinterpret_cast<float4*>(pr) =
                            robot ? make_float4(x[0], x[1], x[2], 0.0f) : make_float4(far, far, far, 0.0f);
                }
            }
        } else {
            // ---------------- helpers (1): noise and clipped controls of chunk c;
            // lane (s, k) generates quad h of its robot's stream
            if (c < nchunks && robot) {
                const int q = c * QPC + h;
                if (4 * q < T * DU) {
                    float z[4];
                    const U4 w = philox4x32_10(U4{(uint32_t)q, jj, c2, c3}, S);
                    box_muller(w.x, w.y, z[0], z[1]);
                    box_muller(w.z, w.w, z[2], z[3]);
                    float* U = sU + (c & 1) * u_slot;
                    if constexpr (DU == 2) {
                        // the quad is time steps 2q, 2q + 1 of controls (0, 1)
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const int t = 2 * q + r;
                            if (t < T) {
                                const float2 m = *reinterpret_cast<const float2*>(sM + t * rowM + k * 2);
                                const float2 v = make_float2(clampf(fmaf(S.sigma, z[2 * r], m.x), lo[0], hi[0]),
                                                             clampf(fmaf(S.sigma, z[2 * r + 1], m.y), lo[1], hi[1]));
                                *reinterpret_cast<float2*>(U + ((t - c * CT) * SPC + s) * rowM + k * 2) = v;
                            }
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int e = 4 * q + r;     // element of robot k's stream
                            const int t = e / DU, d = e - t * DU;
                            if (t < T) {
                                float lod = lo[0], hid = hi[0];
#pragma unroll
                                for (int dd = 1; dd < DU; ++dd)
                                    if (d == dd) {
                                        lod = lo[dd];
                                        hid = hi[dd];
                                    }
                                U[((t - c * CT) * SPC + s) * rowM + k * DU + d] =
                                    clampf(fmaf(S.sigma, z[r], sM[t * rowM + k * DU + d]), lod, hid);
                            }
                        }
                    }
                }
            }
            // ---------------- helpers (2): Eq. (4)/(5) terms of chunk c - 2,
            // time steps h, h + H, ... of the chunk
            const int ce = c - 2;
            if (ce >= 0) {
                const float* Pos = sPos + (ce & 1) * pos_slot;
                for (int tl = h; tl < CT; tl += H) {
                    const int t = ce * CT + tl;
                    if (t >= T) break;                   // uniform across the warp
                    const float* pr = Pos + (tl * SPC + s) * RS;
                    float term = 0.0f;
                    if (robot) {
                        float p[DP];
                        if constexpr (PD == 2) {
                            const float2 v = *reinterpret_cast<const float2*>(pr + k * 2);
                            p[0] = v.x;
                            p[1] = v.y;
                        } else {
                            const float4 v = *reinterpret_cast<const float4*>(pr + k * 4);
                            p[0] = v.x;
                            p[1] = v.y;
                            p[2] = v.z;
                        }
                        float dg2 = 0.0f;
#pragma unroll
                        for (int d = 0; d < DP; ++d) {
                            const float e = p[d] - g[d];
                            dg2 = fmaf(e, e, dg2);
                        }
                        // Eq. (5): robots within 2R + eps, itself included
                        int cnt = 0;
                        if constexpr (PD == 2 && SEG >= 2) {
#pragma unroll
                            for (int m = 0; m < SEG / 2; ++m) {
                                const float4 v = *reinterpret_cast<const float4*>(pr + 4 * m);
                                const float ax = p[0] - v.x, ay = p[1] - v.y;
                                const float bx = p[0] - v.z, by = p[1] - v.w;
                                cnt += fmaf(ay, ay, ax * ax) <= P.thr2;
                                cnt += fmaf(by, by, bx * bx) <= P.thr2;
                            }
                        } else if constexpr (PD == 2) {
                            cnt = 1;                      // a single robot
                        } else {
#pragma unroll
                            for (int l = 0; l < SEG; ++l) {
                                const float4 v = *reinterpret_cast<const float4*>(pr + 4 * l);
                                const float ax = p[0] - v.x, ay = p[1] - v.y, az = p[2] - v.z;
                                cnt += fmaf(az, az, fmaf(ay, ay, ax * ax)) <= P.thr2;
                            }
                        }
                        term = (1.0f - sqrt_approx(dg2) * inv_d0) - (cnt > 1 ? S.w_safe : 0.0f);
                        // Appendix: binary obstacle penalty with the same weight
                        if constexpr (OBS)
                            if (obstacle_hit<DP>(P, p)) term -= S.w_safe;
                    }
                    term = seg_sum<SEG>(term);
                    if (k == 0) sRows[s * T + t] = term;
                }
            }
        }
        __syncthreads();
    }
    // per-sample sum of the row terms, fixed order
    if (warp == 0) {
        for (int ss = 0; ss < SPC; ++ss) {
            float a = 0.0f;
            for (int t = lane; t < T; t += 32) a += sRows[ss * T + t];
            a = seg_sum<32>(a);
            if (lane == 0 && j_base + ss < S.N) fitness[j_base + ss] = a * P.inv_nT;
        }
    }
}

template <int DYN, int SEG, bool OBS>
static cudaError_t prepare_pipe()
{
    return cudaFuncSetAttribute(k_rollout_fitness_pipe<DYN, SEG, OBS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
}

template <int DYN, int SEG, bool OBS>
static cudaError_t launch_pipe(const DevProblem& P, const DevStep& S, const float* u_base, const float* du_in,
                               float* fitness, const int* it_dev, cudaStream_t st)
{
    using Shape = PipeShape<SEG, DynDims<DYN>::DU>;
    const int grid = (S.N + Shape::SPC - 1) / Shape::SPC;
    k_rollout_fitness_pipe<DYN, SEG, OBS><<<grid, Shape::THREADS, pipe_smem_bytes<DYN, SEG>(P), st>>>(
        P, S, u_base, du_in, fitness, it_dev);
    return cudaGetLastError();
}

template <int DYN, int SEG, bool OBS>
static cudaError_t pipe_one(const DevProblem& P, const DevStep* S, const float* u_base, const float* du_in,
                            float* fitness, const int* it_dev, cudaStream_t st)
{
    // S == nullptr: set the kernel attributes only
    return S ? launch_pipe<DYN, SEG, OBS>(P, *S, u_base, du_in, fitness, it_dev, st) : prepare_pipe<DYN, SEG, OBS>();
}

template <int DYN, bool OBS>
static cudaError_t pipe_seg(const DevProblem& P, const DevStep* S, const float* u_base, const float* du_in,
                            float* fitness, const int* it_dev, cudaStream_t st)
{
    if (P.n <= 1) return pipe_one<DYN, 1, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    if (P.n <= 2) return pipe_one<DYN, 2, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    if (P.n <= 4) return pipe_one<DYN, 4, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    if (P.n <= 8) return pipe_one<DYN, 8, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    if (P.n <= 16) return pipe_one<DYN, 16, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    return pipe_one<DYN, 32, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
}

template <bool OBS>
static cudaError_t pipe_dyn(const DevProblem& P, const DevStep* S, const float* u_base, const float* du_in,
                            float* fitness, const int* it_dev, cudaStream_t st)
{
    switch (P.dyn) {
    case HOLO2D: return pipe_seg<HOLO2D, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    case HOLO3D: return pipe_seg<HOLO3D, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    case UNICYCLE: return pipe_seg<UNICYCLE, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    case DIFFDRIVE4: return pipe_seg<DIFFDRIVE4, OBS>(P, S, u_base, du_in, fitness, it_dev, st);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t pipe_dispatch(const DevProblem& P, const DevStep* S, const float* u_base, const float* du_in,
                                 float* fitness, const int* it_dev, cudaStream_t st)
{
    return P.n_obs > 0 ? pipe_dyn<true>(P, S, u_base, du_in, fitness, it_dev, st)
                       : pipe_dyn<false>(P, S, u_base, du_in, fitness, it_dev, st);
}

cudaError_t prepare_rollout_fitness_pipe(const DevProblem& P)
{
    return pipe_dispatch(P, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

cudaError_t launch_rollout_fitness_pipe(const DevProblem& P, const DevStep& S, const float* u_base,
                                        const float* du_in, float* fitness, const int* it_dev, cudaStream_t st)
{
    return pipe_dispatch(P, &S, u_base, du_in, fitness, it_dev, st);
}

size_t rollout_fitness_pipe_smem(const DevProblem& P)
{
    const int seg = P.n <= 1 ? 1 : P.n <= 2 ? 2 : P.n <= 4 ? 4 : P.n <= 8 ? 8 : P.n <= 16 ? 16 : 32;
    const int spc = 32 / seg;
    const int pd = P.d_p == 2 ? 2 : 4;
    const size_t pos = 2ull * kPipeCT * spc * seg * pd;
    const size_t u = 2ull * kPipeCT * spc * P.n * P.d_u;
    const size_t mean = (size_t)P.T * P.n * P.d_u;
    return (pos + u + mean + (size_t)spc * P.T) * sizeof(float);
}

}  // namespace d4orm

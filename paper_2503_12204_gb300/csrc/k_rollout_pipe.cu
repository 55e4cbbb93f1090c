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
// time) run on the helpers while the recurrence advances.  Per-row sums
// (one row = one sample at one time step) are reduced inside lane segments
// in a fixed order and added per sample at the end, so the result is
// deterministic.  Shared memory holds the mean controls u_base + c dU, two
// chunks of controls and positions (time-major, rows padded, so that warp
// accesses are conflict-free) and the per-row terms.
#include <cmath>

#include "d4orm_internal.h"

namespace d4orm {

constexpr int kPipeCT = 16;  // time steps per chunk (a multiple of 4: chunks are Philox-quad aligned)

template <int SEG>
struct PipeShape {
    static constexpr int SPC = 32 / SEG;                   // samples per CTA
    static constexpr int HELPERS = SEG <= 8 ? 3 : 7;       // helper warps
    static constexpr int THREADS = 32 * (1 + HELPERS);
};

// Shared memory, time-major so that one warp access touches consecutive
// words: U[2][CT][SPC][n][DU] (controls), Pos[2][CT*SPC][RS] (positions, row
// stride RS = SEG*DP + 1 so the rows a warp reads fall in different banks),
// rows[SPC][T] (per-row fitness terms).
template <int SEG, int DP>
struct PosStride { static constexpr int RS = SEG * DP + 1; };

template <int DYN, int SEG>
size_t pipe_smem_bytes(const DevProblem& P)
{
    using D = DynDims<DYN>;
    constexpr int SPC = PipeShape<SEG>::SPC;
    const size_t u = 2ull * SPC * kPipeCT * P.n * D::DU;
    const size_t pos = 2ull * SPC * kPipeCT * PosStride<SEG, D::DP>::RS;
    const size_t rows = (size_t)SPC * P.T;
    const size_t mean = (size_t)P.T * P.n * D::DU;
    return (u + pos + rows + mean) * sizeof(float);
}

template <int DYN, int SEG, bool OBS>
__global__ void __launch_bounds__(PipeShape<SEG>::THREADS)
k_rollout_fitness_pipe(const DevProblem P, const DevStep S, const float* __restrict__ u_base,
                       const float* __restrict__ du_in, float* __restrict__ fitness, const int* __restrict__ it_dev)
{
    using D = DynDims<DYN>;
    constexpr int DX = D::DX, DU = D::DU, DP = D::DP;
    constexpr int SPC = PipeShape<SEG>::SPC;
    constexpr int HELPERS = PipeShape<SEG>::HELPERS;
    constexpr int CT = kPipeCT;
    constexpr int RS = PosStride<SEG, DP>::RS;
    extern __shared__ float smem[];
    const int n = P.n, T = P.T;
    float* sU = smem;                                   // [2][CT][SPC][n][DU]
    float* sPos = sU + 2 * SPC * CT * n * DU;           // [2][CT*SPC][RS]
    float* sRows = sPos + 2 * SPC * CT * RS;            // [SPC][T]
    float* sM = sRows + SPC * T;                         // [T][n][DU] mean controls
    const int u_slot = SPC * CT * n * DU;
    const int pos_slot = SPC * CT * RS;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j_base = blockIdx.x * SPC;
    const uint32_t c3 = iter_word(S, it_dev);
    const int nchunks = (T + CT - 1) / CT;
    const int rowM = n * DU;
    for (int e = threadIdx.x; e < T * rowM; e += blockDim.x) sM[e] = fmaf(S.c, du_in[e], u_base[e]);
    __syncthreads();
    const int quads_per_chunk = CT * DU / 4;

    // rollout-warp state (warp 0)
    const int rk = lane & (SEG - 1);
    const int rs = lane / SEG;
    float x[DX];
    load_start<DYN>(x, P, rk);
    const int rkr = rk < n ? rk : n - 1;

    for (int c = 0; c < nchunks + 2; ++c) {
        if (warp > 0) {
            const int h = threadIdx.x - 32;  // helper thread index
            // (1) noise and clipped controls of chunk c
            if (c < nchunks) {
                // items over (quad, sample, lane-robot) with the robot
                // fastest (neighbouring threads touch neighbouring words of U
                // and of the mean controls); SEG and SPC are powers of two,
                // so the index split is shifts and masks
                constexpr int ITEMS = SPC * SEG * (CT * DU / 4);
                float* U = sU + (c & 1) * u_slot;
#pragma unroll 1
                for (int it = h; it < ITEMS; it += 32 * HELPERS) {
                    const int k = it & (SEG - 1);
                    const int s = (it / SEG) & (SPC - 1);
                    const int qq = it / (SEG * SPC);
                    if (k >= n) continue;
                    const uint32_t q = (uint32_t)(c * quads_per_chunk + qq);
                    float z[4];
                    noise_quad(S, c3, q, (uint32_t)(j_base + s), (uint32_t)k, z);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int e = 4 * (int)q + r;          // element of robot k's stream
                        const int t = e / DU, d = e - t * DU;
                        if (t < T) {
                            U[(((t - c * CT) * SPC + s) * n + k) * DU + d] =
                                clampf(fmaf(S.sigma, z[r], sM[t * rowM + k * DU + d]), P.u_lo[d], P.u_hi[d]);
                        }
                    }
                }
            }
            // (2) Eq. (4)/(5) terms of chunk c - 2: one row per lane segment
            const int ce = c - 2;
            if (ce >= 0) {
                const float* Pos = sPos + (ce & 1) * pos_slot;
                const int hw = warp - 1;
                const int k = lane & (SEG - 1);
                const bool robot = k < n;
                const int kr = robot ? k : n - 1;
                float g[DP];
#pragma unroll
                for (int d = 0; d < DP; ++d) g[d] = P.goal[kr * 3 + d];
                const float inv_d0 = P.inv_d0[kr];
                const int rows = SPC * CT;
                for (int rb = hw * (32 / SEG); rb < rows; rb += HELPERS * (32 / SEG)) {
                    const int row = rb + lane / SEG;  // row = tl * SPC + s; warp-uniform loop bound
                    const int tl = row / SPC, s = row - tl * SPC;
                    const int t = ce * CT + tl;
                    float term = 0.0f;
                    if (row < rows && t < T && robot) {
                        const float* pr = Pos + row * RS;
                        float p[DP];
#pragma unroll
                        for (int d = 0; d < DP; ++d) p[d] = pr[k * DP + d];
                        float dg2 = 0.0f;
#pragma unroll
                        for (int d = 0; d < DP; ++d) {
                            const float e = p[d] - g[d];
                            dg2 = fmaf(e, e, dg2);
                        }
                        bool hit = false;
#pragma unroll
                        for (int l = 0; l < SEG; ++l) {
                            float d2 = 0.0f;
#pragma unroll
                            for (int d = 0; d < DP; ++d) {
                                const float e = p[d] - pr[l * DP + d];
                                d2 = fmaf(e, e, d2);
                            }
                            hit |= (l != k) & (l < n) & (d2 <= P.thr2);
                        }
                        term = (1.0f - sqrt_approx(dg2) * inv_d0) - (hit ? S.w_safe : 0.0f);
                        // Appendix: binary obstacle penalty with the same weight
                        if constexpr (OBS)
                            if (obstacle_hit<DP>(P, p)) term -= S.w_safe;
                    }
                    term = seg_sum<SEG>(term);
                    if (k == 0 && row < rows && t < T) sRows[s * T + t] = term;
                }
            }
        } else if (c >= 1 && c <= nchunks) {
            // (3) rollout of chunk c - 1
            const int cr = c - 1;
            const float* U = sU + (cr & 1) * u_slot;
            float* Pos = sPos + (cr & 1) * pos_slot;
            const int steps = min(CT, T - cr * CT);
#pragma unroll 4
            for (int tl = 0; tl < steps; ++tl) {
                float u[DU];
#pragma unroll
                for (int d = 0; d < DU; ++d) u[d] = U[((tl * SPC + rs) * n + rkr) * DU + d];
                integrate<DYN>(x, u, P);
#pragma unroll
                for (int d = 0; d < DP; ++d) Pos[(tl * SPC + rs) * RS + rk * DP + d] = x[d];
            }
        }
        __syncthreads();
    }
    // per-sample sum of the row terms, fixed order
    if (warp == 0) {
        for (int s = 0; s < SPC; ++s) {
            float a = 0.0f;
            for (int t = lane; t < T; t += 32) a += sRows[s * T + t];
            a = seg_sum<32>(a);
            if (lane == 0 && j_base + s < S.N) fitness[j_base + s] = a * P.inv_nT;
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
    constexpr int SPC = PipeShape<SEG>::SPC;
    const int grid = (S.N + SPC - 1) / SPC;
    k_rollout_fitness_pipe<DYN, SEG, OBS><<<grid, PipeShape<SEG>::THREADS, pipe_smem_bytes<DYN, SEG>(P), st>>>(
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
    const size_t u = 2ull * spc * kPipeCT * P.n * P.d_u;
    const size_t pos = 2ull * spc * kPipeCT * (seg * P.d_p + 1);
    const size_t mean = (size_t)P.T * P.n * P.d_u;
    return (u + pos + (size_t)spc * P.T + mean) * sizeof(float);
}

}  // namespace d4orm

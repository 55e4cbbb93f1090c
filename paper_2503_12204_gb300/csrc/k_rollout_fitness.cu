// k_rollout_fitness.cu -- K2, the fused sample rollout + fitness kernel.
//
// One denoising step evaluates N deformation samples (Eq. (12), Algorithm 1
// sampling + rollout lines).  Each sample is one whole robot team, rolled
// out over T steps and scored by the team reward of Eq. (3)-(5):
//
//   u_{t,k}  = clip(M_{t,k} + sigma_i eps_{j,t,k}),  M = u_base + c_i dU_i
//   x_{t+1}  = integrate(x_t, u_t)                    (Sec. III Eq. (1), Sec. V)
//   r_j      = 1/(nT) sum_{t=1..T} sum_k [1 - |p_k - g_k| / d0_k
//                                         - w Ind(exists l: |p_k - p_l| <= 2R+eps)]
//
// Mapping: robots in lanes.  A warp holds 32/SEG samples, one per aligned
// segment of SEG lanes (SEG = next power of two >= n); the robot state lives
// in registers for the whole horizon.  Pairwise distances of Eq. (5) are
// read from the partner lanes with shuffles inside the segment, each
// unordered pair once (a ballot returns the flag to the partner), and the
// per-sample fitness is reduced with segment shuffles: nothing but
// the final float per sample leaves the SM.  The mean controls M are staged
// once per CTA in shared memory.  The noise eps is regenerated from Philox in
// registers, four time steps at a time (d_u Philox calls), never stored.
#include <cmath>

#include "d4orm_internal.h"
#include "d4orm_kernels.cuh"

namespace d4orm {

constexpr int kK2Threads = 256;

template <int DYN, int SEG, bool OBS>
__global__ void __launch_bounds__(kK2Threads)
k_rollout_fitness(const DevProblem P, const DevStep S, const float* __restrict__ u_base,
                  const float* __restrict__ du_in, float* __restrict__ fitness, const int* __restrict__ it_dev)
{
    constexpr int DU = DynDims<DYN>::DU;
    constexpr int SPW = 32 / SEG;  // samples per warp
    extern __shared__ float sM[];  // M[t][k][d]

    const int nctrl = P.T * P.n * DU;
    stage_mean<true>(sM, du_in, u_base, S.c, nctrl);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int j = warp * SPW + lane / SEG;
    const float f = sample_fitness_segment<DYN, SEG, OBS>(P, S, sM, iter_word(S, it_dev), j);
    if ((lane & (SEG - 1)) == 0 && j < S.N) fitness[j] = f;
}

// Opt in to up to 200 KB of dynamic shared memory (mean controls of the
// largest problems).  Called outside any stream capture.
template <int DYN, int SEG, bool OBS>
static cudaError_t prepare_k2()
{
    return cudaFuncSetAttribute(k_rollout_fitness<DYN, SEG, OBS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
}

template <int DYN, bool OBS>
static cudaError_t prepare_dyn(int n)
{
    if (n <= 1) return prepare_k2<DYN, 1, OBS>();
    if (n <= 2) return prepare_k2<DYN, 2, OBS>();
    if (n <= 4) return prepare_k2<DYN, 4, OBS>();
    if (n <= 8) return prepare_k2<DYN, 8, OBS>();
    if (n <= 16) return prepare_k2<DYN, 16, OBS>();
    return prepare_k2<DYN, 32, OBS>();
}

template <bool OBS>
static cudaError_t prepare_k2_variant(const DevProblem& P)
{
    switch (P.dyn) {
    case HOLO2D: return prepare_dyn<HOLO2D, OBS>(P.n);
    case HOLO3D: return prepare_dyn<HOLO3D, OBS>(P.n);
    case UNICYCLE: return prepare_dyn<UNICYCLE, OBS>(P.n);
    case DIFFDRIVE4: return prepare_dyn<DIFFDRIVE4, OBS>(P.n);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_rollout_fitness(const DevProblem& P)
{
    cudaError_t e = prepare_rollout_fitness_pipe(P);
    if (e != cudaSuccess) return e;
    e = prepare_rollout_fitness_paired(P);
    if (e != cudaSuccess) return e;
    return P.n_obs > 0 ? prepare_k2_variant<true>(P) : prepare_k2_variant<false>(P);
}

// Warps per CTA: every sample is the same amount of work, so the launch
// that minimises the most-loaded SM (all CTAs resident in one wave) wins;
// ties go to wider CTAs (fewer shared-memory loads of the mean controls).
static int pick_warps_per_cta(int total_warps, int sm_count)
{
    int best_w = 1;
    long long best_cost = -1;
    for (int w = 1; w <= kK2Threads / 32; ++w) {
        const long long ctas = (total_warps + w - 1) / w;
        const long long per_sm = (ctas + sm_count - 1) / sm_count;
        const long long cost = per_sm * w;
        if (best_cost < 0 || cost <= best_cost) {
            best_cost = cost;
            best_w = w;
        }
    }
    return best_w;
}

template <int DYN, int SEG, bool OBS>
static cudaError_t launch_k2(const DevProblem& P, const DevStep& S, const float* u_base, const float* du_in,
                             float* fitness, const int* it_dev, int sm_count, cudaStream_t st)
{
    constexpr int spw = 32 / SEG;
    const int total_warps = (S.N + spw - 1) / spw;
    const int w = pick_warps_per_cta(total_warps, sm_count);
    const size_t smem = (size_t)P.T * P.n * DynDims<DYN>::DU * sizeof(float);
    const int grid = (total_warps + w - 1) / w;
    k_rollout_fitness<DYN, SEG, OBS><<<grid, 32 * w, smem, st>>>(P, S, u_base, du_in, fitness, it_dev);
    return cudaGetLastError();
}

template <int DYN, bool OBS>
static cudaError_t dispatch_seg(const DevProblem& P, const DevStep& S, const float* u_base, const float* du_in,
                                float* fitness, const int* it_dev, int sms, cudaStream_t st)
{
    if (P.n <= 1) return launch_k2<DYN, 1, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    if (P.n <= 2) return launch_k2<DYN, 2, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    if (P.n <= 4) return launch_k2<DYN, 4, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    if (P.n <= 8) return launch_k2<DYN, 8, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    if (P.n <= 16) return launch_k2<DYN, 16, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    return launch_k2<DYN, 32, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
}

template <bool OBS>
static cudaError_t dispatch_dyn(const DevProblem& P, const DevStep& S, const float* u_base, const float* du_in,
                                float* fitness, const int* it_dev, int sms, cudaStream_t st)
{
    switch (P.dyn) {
    case HOLO2D: return dispatch_seg<HOLO2D, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case HOLO3D: return dispatch_seg<HOLO3D, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case UNICYCLE: return dispatch_seg<UNICYCLE, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case DIFFDRIVE4: return dispatch_seg<DIFFDRIVE4, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    default: return cudaErrorInvalidValue;
    }
}

int resolve_rollout_kernel(const DevProblem& P, int N, int sm_count, int requested)
{
    const bool pipe_fits = rollout_fitness_pipe_smem(P) <= 200 * 1024;
    if (requested == D4ORM_ROLLOUT_PAIRED) return D4ORM_ROLLOUT_PAIRED;
    if (requested == D4ORM_ROLLOUT_PIPELINE && pipe_fits) return D4ORM_ROLLOUT_PIPELINE;
    if (requested == D4ORM_ROLLOUT_REGISTER) return D4ORM_ROLLOUT_REGISTER;
    const int seg = P.n <= 1 ? 1 : P.n <= 2 ? 2 : P.n <= 4 ? 4 : P.n <= 8 ? 8 : P.n <= 16 ? 16 : 32;
    const long long warps = ((long long)N * seg + 31) / 32;
    // automatic: two robots per lane for holonomic teams of 5 or more robots
    // once the paired kernel keeps 6 warps per SM busy (12 with obstacles,
    // whose test does not pack).  Measured on GB300 inside CUDA graphs, us,
    // register vs paired: 3D n = 16, N = 2048 / 3072 / 4096 / 8192 ->
    // 33.2/34.4, 45.0/48.6, 55.1/48.9, 93.0/86.6; 2D n = 16, N = 4096:
    // 40.6/36.0; 3D n = 8, N = 4096 / 8192: 27.1/28.1, 46.0/38.9; 2D n = 16
    // with 4 obstacles, N = 4096 / 8192: 56.7/67.6, 96.4/96.5; unicycle
    // n = 8, N = 2048 / 8192: 15.1/33.5, 37.6/42.3 (never paired).
    const long long paired_warps = ((long long)N * paired_lanes(P.n) + 31) / 32;
    const bool holonomic = P.dyn == HOLO2D || P.dyn == HOLO3D;
    const long long paired_need = (P.n_obs > 0 ? 12LL : 6LL) * sm_count;
    if (holonomic && P.n >= 5 && paired_warps >= paired_need) return D4ORM_ROLLOUT_PAIRED;
    if (!pipe_fits) return D4ORM_ROLLOUT_REGISTER;
    // below about 2.5 warps per SM the register kernel leaves the SMs too
    // idle and the pipelined kernel's parallelism along time wins (measured
    // whole solves on GB300: unicycle, 8 robots, N = 1024 / 1.7 warps per
    // SM: pipelined 12.6 vs register 13.4 ms; N = 2048 / 3.4 warps per SM:
    // register 14.3 vs pipelined 16.7 ms)
    return 2 * warps < 5LL * sm_count ? D4ORM_ROLLOUT_PIPELINE : D4ORM_ROLLOUT_REGISTER;
}

cudaError_t launch_rollout_fitness(const DevProblem& P, const DevStep& S, const float* u_base, const float* du_in,
                                   float* fitness, const int* it_dev, int sm_count, int kernel, cudaStream_t st)
{
    const int kind = resolve_rollout_kernel(P, S.N, sm_count, kernel);
    if (kind == D4ORM_ROLLOUT_PIPELINE) return launch_rollout_fitness_pipe(P, S, u_base, du_in, fitness, it_dev, st);
    if (kind == D4ORM_ROLLOUT_PAIRED)
        return launch_rollout_fitness_paired(P, S, u_base, du_in, fitness, it_dev, sm_count, st);
    return P.n_obs > 0 ? dispatch_dyn<true>(P, S, u_base, du_in, fitness, it_dev, sm_count, st)
                       : dispatch_dyn<false>(P, S, u_base, du_in, fitness, it_dev, sm_count, st);
}

}  // namespace d4orm

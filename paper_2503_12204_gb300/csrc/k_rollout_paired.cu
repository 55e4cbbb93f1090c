// k_rollout_paired.cu -- K2b, the fused sample rollout + fitness kernel with
// two robots per lane (sample_fitness_paired): the same Eq. (12) samples,
// Eq. (1) rollout and Eq. (3)-(5) fitness as K2, for batches whose
// register-kernel warps are plentiful enough that half as many still keep
// every scheduler busy.  A warp holds 32/L samples (L = SEG/2 lanes each);
// the mean controls M = u_base + c dU are staged once per CTA in shared
// memory, followed by each warp's position-exchange buffer; nothing but one
// float per sample leaves the SM.
#include <cmath>

#include "d4orm_internal.h"
#include "d4orm_paired.cuh"

namespace d4orm {

constexpr int kK2bThreads = 256;
// per-warp position buffers of sample_fitness_paired, after the mean controls
template <int DYN>
__host__ __device__ constexpr size_t k2b_xbuf_bytes_per_warp()
{
    return 2 * DynDims<DYN>::DP * 32 * sizeof(f2);
}

template <int DYN, int L, bool OBS>
__global__ void __launch_bounds__(kK2bThreads)
k_rollout_fitness_paired(const DevProblem P, const DevStep S, const float* __restrict__ u_base,
                         const float* __restrict__ du_in, float* __restrict__ fitness, const int* __restrict__ it_dev)
{
    constexpr int DU = DynDims<DYN>::DU;
    constexpr int SPW = 32 / L;  // samples per warp
    extern __shared__ float sM[];  // M[t][k][d]

    stage_mean<true>(sM, du_in, u_base, S.c, P.T * P.n * DU);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int j = warp * SPW + lane / L;
    // per-warp position buffers after the mean controls (8-byte aligned)
    f2* xbuf = reinterpret_cast<f2*>(sM + ((P.T * P.n * DU + 1) & ~1)) +
               (threadIdx.x >> 5) * (k2b_xbuf_bytes_per_warp<DYN>() / sizeof(f2));
    const float f = sample_fitness_paired<DYN, L, OBS>(P, S, sM, iter_word(S, it_dev), j, xbuf);
    if ((lane & (L - 1)) == 0 && j < S.N) fitness[j] = f;
}

// Lanes per sample: half the register kernel's segment (at least 1).
int paired_lanes(int n)
{
    const int seg = n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32;
    return seg > 1 ? seg / 2 : 1;
}

// Warps per CTA: as for K2, the width that least loads the busiest SM
// (all CTAs resident in one wave), ties to wider CTAs.
static int paired_warps_per_cta(int total_warps, int sm_count)
{
    int best_w = 1;
    long long best_cost = -1;
    for (int w = 1; w <= kK2bThreads / 32; ++w) {
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

template <int DYN, int L, bool OBS>
static cudaError_t paired_one(const DevProblem& P, const DevStep* S, const float* u_base, const float* du_in,
                              float* fitness, const int* it_dev, int sm_count, cudaStream_t st)
{
    auto kern = k_rollout_fitness_paired<DYN, L, OBS>;
    if (!S) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    constexpr int spw = 32 / L;
    const int total_warps = (S->N + spw - 1) / spw;
    const int w = paired_warps_per_cta(total_warps, sm_count);
    const size_t smem = (size_t)((P.T * P.n * DynDims<DYN>::DU + 1) & ~1) * sizeof(float) +
                        (size_t)w * k2b_xbuf_bytes_per_warp<DYN>();
    const int grid = (total_warps + w - 1) / w;
    kern<<<grid, 32 * w, smem, st>>>(P, *S, u_base, du_in, fitness, it_dev);
    return cudaGetLastError();
}

template <int DYN, bool OBS>
static cudaError_t paired_lanes_dispatch(const DevProblem& P, const DevStep* S, const float* u_base,
                                         const float* du_in, float* fitness, const int* it_dev, int sms,
                                         cudaStream_t st)
{
    switch (paired_lanes(P.n)) {
    case 1: return paired_one<DYN, 1, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case 2: return paired_one<DYN, 2, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case 4: return paired_one<DYN, 4, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case 8: return paired_one<DYN, 8, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    default: return paired_one<DYN, 16, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    }
}

template <bool OBS>
static cudaError_t paired_dyn(const DevProblem& P, const DevStep* S, const float* u_base, const float* du_in,
                              float* fitness, const int* it_dev, int sms, cudaStream_t st)
{
    switch (P.dyn) {
    case HOLO2D: return paired_lanes_dispatch<HOLO2D, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case HOLO3D: return paired_lanes_dispatch<HOLO3D, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case UNICYCLE: return paired_lanes_dispatch<UNICYCLE, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    case DIFFDRIVE4: return paired_lanes_dispatch<DIFFDRIVE4, OBS>(P, S, u_base, du_in, fitness, it_dev, sms, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_rollout_fitness_paired(const DevProblem& P)
{
    return P.n_obs > 0 ? paired_dyn<true>(P, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr)
                       : paired_dyn<false>(P, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr);
}

cudaError_t launch_rollout_fitness_paired(const DevProblem& P, const DevStep& S, const float* u_base,
                                          const float* du_in, float* fitness, const int* it_dev, int sm_count,
                                          cudaStream_t st)
{
    return P.n_obs > 0 ? paired_dyn<true>(P, &S, u_base, du_in, fitness, it_dev, sm_count, st)
                       : paired_dyn<false>(P, &S, u_base, du_in, fitness, it_dev, sm_count, st);
}

}  // namespace d4orm

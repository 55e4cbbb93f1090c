// k_update.cu -- K3, the softmax weights and the weighted-mean update.
//
// Pass 1 (k_softmax_weights, one CTA): batch normalisation of the rewards
// (Sec. IV-C: z = (r - mean) / std, population std) and the temperature
// softmax of Eq. (6), as a two-pass log-sum-exp (maximum logit first).
//
// Pass 1 also compacts the samples that carry weight into an ordered
// (weight, index) list; weights below 2^-30 of the largest are dropped.
//
// Pass 2 (k_weighted_mean): S = sum_j w_j eps_j over the listed samples, with
// eps regenerated from the same Philox counters K2 used (no sample is
// stored), and dU_{i-1} = g_i (c_i dU_i + sigma_i S), the weighted mean of
// the samples of Eq. (12) scaled as in Eq. (13).  Every sum runs in a fixed
// order, so the result is deterministic.
#include <algorithm>
#include <cmath>

#include "d4orm_internal.h"
#include "d4orm_kernels.cuh"

namespace d4orm {

constexpr int kSoftmaxThreads = 1024;

// VR > 0: each thread keeps its (at most VR) fitness values in registers;
// VR == 0: the values are re-read from global memory (L1) on every pass.
template <int VR>
__global__ void __launch_bounds__(kSoftmaxThreads)
k_softmax_weights(const float* __restrict__ fitness, int N, float inv_lambda, float2* __restrict__ list,
                  int* __restrict__ count, float* __restrict__ stats)
{
    __shared__ float sh[kSoftmaxScratch];
    __shared__ int scan[33];
    softmax_block<VR>(fitness, N, inv_lambda, list, count, stats, sh, scan);
}

// K3b: the weighted noise sum and the Eq. (13) update in one pass.  A CTA
// owns QC noise quads and all the listed samples: its 256 threads form QC
// quads x (256 / QC) sample slices, the list dealt round-robin over the
// slices; slices are reduced by warp shuffles, then across the eight warps
// in shared memory, both in a fixed order.  The CTA then writes its quads'
// controls of dU_{i-1} = g_i (c_i dU_i + sigma_i S) itself.  (Splitting the
// samples over CTAs instead needs per-chunk partial sums and a second
// pass over them; on the 8-robot unicycle solve that form took 6 % longer,
// on the 16-robot 3D solve 1.3 %.)
constexpr int kWMThreads = 256;

template <int QC>
__global__ void __launch_bounds__(kWMThreads, 8)
k_weighted_mean(const DevProblem P, const DevStep S, const float2* __restrict__ list,
                const int* __restrict__ count, const float* __restrict__ du_in, float* __restrict__ du_out,
                const int* __restrict__ it_dev)
{
    constexpr int SL = kWMThreads / QC;  // sample slices
    __shared__ float4 red[kWMThreads / 32][QC];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int qi = tid % QC, slice = tid / QC;
    const int nQ = P.n * P.Q;
    const int gq = blockIdx.x * QC + qi;
    const bool valid = gq < nQ;
    const int k = valid ? gq / P.Q : 0;
    const int q = valid ? gq - k * P.Q : 0;
    const uint32_t c3 = iter_word(S, it_dev);
    const int n_list = *count;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    // two entries per trip: their Philox chains are independent, so one
    // thread keeps two in flight; they are added in list order
    int e = slice;
    for (; e + SL < n_list; e += 2 * SL) {
        const float2 w0 = list[e], w1 = list[e + SL];
        float z[4], y[4];
        noise_quad(S, c3, (uint32_t)q, (uint32_t)__float_as_int(w0.y), (uint32_t)k, z);
        noise_quad(S, c3, (uint32_t)q, (uint32_t)__float_as_int(w1.y), (uint32_t)k, y);
        a0 = fmaf(w1.x, y[0], fmaf(w0.x, z[0], a0));
        a1 = fmaf(w1.x, y[1], fmaf(w0.x, z[1], a1));
        a2 = fmaf(w1.x, y[2], fmaf(w0.x, z[2], a2));
        a3 = fmaf(w1.x, y[3], fmaf(w0.x, z[3], a3));
    }
    if (e < n_list) {
        const float2 w0 = list[e];
        float z[4];
        noise_quad(S, c3, (uint32_t)q, (uint32_t)__float_as_int(w0.y), (uint32_t)k, z);
        a0 = fmaf(w0.x, z[0], a0);
        a1 = fmaf(w0.x, z[1], a1);
        a2 = fmaf(w0.x, z[2], a2);
        a3 = fmaf(w0.x, z[3], a3);
    }
    // lanes lane and lane ^ off (off >= QC) hold the same quad
#pragma unroll
    for (int off = 16; off >= QC; off >>= 1) {
        a0 += __shfl_xor_sync(kFull, a0, off);
        a1 += __shfl_xor_sync(kFull, a1, off);
        a2 += __shfl_xor_sync(kFull, a2, off);
        a3 += __shfl_xor_sync(kFull, a3, off);
    }
    if (lane < QC) red[warp][lane] = make_float4(a0, a1, a2, a3);
    __syncthreads();
    // thread r * QC + qi finishes element r of quad qi
    if (tid < 4 * QC) {
        const int r = tid / QC, qo = tid % QC;
        const int go = blockIdx.x * QC + qo;
        if (go < nQ) {
            float s = 0.0f;
#pragma unroll
            for (int w = 0; w < kWMThreads / 32; ++w) {
                const float4 v = red[w][qo];
                s += r == 0 ? v.x : r == 1 ? v.y : r == 2 ? v.z : v.w;
            }
            const int ko = go / P.Q;
            const int el = (go - ko * P.Q) * 4 + r;  // t * d_u + d
            if (el < P.T * P.d_u) {
                const int t = el / P.d_u, d = el - t * P.d_u;
                const int idx = (t * P.n + ko) * P.d_u + d;
                du_out[idx] = S.g * fmaf(S.sigma, s, S.c * du_in[idx]);
            }
        }
    }
}

// Quads per CTA of k_weighted_mean: the fewest that keep the grid within one
// wave of eight CTAs per SM (at most 32).
int weighted_mean_qc(const DevProblem& P, int sm_count)
{
    const int nQ = P.n * P.Q;
    int qc = 1;
    while (qc < 32 && (nQ + qc - 1) / qc > 8 * sm_count) qc *= 2;
    return qc;
}

cudaError_t launch_weighted_mean(const DevProblem& P, const DevStep& S, const float2* list, const int* count,
                                 const float* du_in, float* du_out, const int* it_dev, int sm_count, cudaStream_t st)
{
    const int nQ = P.n * P.Q;
    const int qc = weighted_mean_qc(P, sm_count);
    const int grid = (nQ + qc - 1) / qc;
#define D4_WM(QCV)                                                                                          \
    case QCV:                                                                                               \
        k_weighted_mean<QCV><<<grid, kWMThreads, 0, st>>>(P, S, list, count, du_in, du_out, it_dev);      \
        break
    switch (qc) {
        D4_WM(1);
        D4_WM(2);
        D4_WM(4);
        D4_WM(8);
        D4_WM(16);
        default:
            k_weighted_mean<32><<<grid, kWMThreads, 0, st>>>(P, S, list, count, du_in, du_out, it_dev);
            break;
    }
#undef D4_WM
    return cudaGetLastError();
}

cudaError_t launch_softmax_weights(const float* fitness, int N, float inv_lambda, float2* list, int* count,
                                   float* stats, cudaStream_t st)
{
    if (N <= 8 * kSoftmaxThreads) {
        // eight rewards per thread: fewer warps, cheaper block reductions
        const int threads = std::min(kSoftmaxThreads, std::max(128, ((N + 7) / 8 + 31) / 32 * 32));
        k_softmax_weights<8><<<1, threads, 0, st>>>(fitness, N, inv_lambda, list, count, stats);
    } else {
        k_softmax_weights<0><<<1, kSoftmaxThreads, 0, st>>>(fitness, N, inv_lambda, list, count, stats);
    }
    return cudaGetLastError();
}

}  // namespace d4orm

// k_update.cu -- K3, the softmax weights and the weighted-mean update.
//
// Pass 1 (k_softmax_weights, one CTA): batch normalisation of the rewards
// (Sec. IV-C: z = (r - mean) / std, population std) and the temperature
// softmax of Eq. (6), as a two-pass log-sum-exp (maximum logit first).
//
// Pass 1 also compacts the samples that carry weight into an ordered
// (weight, index) list; weights below 2^-30 of the largest are dropped.
//
// Pass 2 (k_weighted_sum): S = sum_j w_j eps_j over the listed samples, with
// eps regenerated from the same Philox counters K2 used (no sample is
// stored).  The grid splits the n*Q noise quads over CTA columns and deals
// the list round-robin over CTA rows; each CTA reduces its 8 sample rows in
// shared memory and writes one float4 partial per quad and chunk.
//
// Pass 3 (k_finalize): dU_{i-1} = g_i (c_i dU_i + sigma_i sum_chunks S_c),
// the weighted mean of the samples of Eq. (12) scaled as in Eq. (13); chunk
// partials are added in a fixed order, so the result is deterministic.
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
    __shared__ float sh[66];
    __shared__ int scan[33];
    softmax_block<VR>(fitness, N, inv_lambda, list, count, stats, sh, scan);
}

constexpr int kWSRows = 8;

__global__ void __launch_bounds__(32 * kWSRows)
k_weighted_sum(const DevProblem P, const DevStep S, const float2* __restrict__ list,
               const int* __restrict__ count, float* __restrict__ partial, const int* __restrict__ it_dev)
{
    __shared__ float4 red[kWSRows][32];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int nQ = P.n * P.Q;
    const int gq = blockIdx.x * 32 + lane;
    const bool valid = gq < nQ;
    const int k = valid ? gq / P.Q : 0;
    const int q = valid ? gq - k * P.Q : 0;
    const uint32_t c3 = iter_word(S, it_dev);
    // the compacted (weight, sample) list is dealt round-robin over the
    // gridDim.y * 8 sample rows, so every CTA gets an equal share whatever
    // the survivor count; the order of accumulation is fixed.
    const int n_list = *count;
    const int stride = gridDim.y * kWSRows;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    // the next entry is loaded while the current sample's noise is
    // regenerated (the Philox counter needs the sample index first)
    int e = blockIdx.y * kWSRows + row;
    float2 next = e < n_list ? list[e] : make_float2(0.0f, 0.0f);
    for (; e < n_list; e += stride) {
        const float2 wj = next;  // warp-uniform
        if (e + stride < n_list) next = list[e + stride];
        float z[4];
        noise_quad(S, c3, (uint32_t)q, (uint32_t)__float_as_int(wj.y), (uint32_t)k, z);
        a0 = fmaf(wj.x, z[0], a0);
        a1 = fmaf(wj.x, z[1], a1);
        a2 = fmaf(wj.x, z[2], a2);
        a3 = fmaf(wj.x, z[3], a3);
    }
    red[row][lane] = make_float4(a0, a1, a2, a3);
    __syncthreads();
    if (row == 0 && valid) {
        float4 s = red[0][lane];
#pragma unroll
        for (int r = 1; r < kWSRows; ++r) {
            const float4 o = red[r][lane];
            s.x += o.x; s.y += o.y; s.z += o.z; s.w += o.w;
        }
        reinterpret_cast<float4*>(partial)[(size_t)blockIdx.y * nQ + gq] = s;
    }
}

constexpr int kFinRows = 8;

__global__ void __launch_bounds__(32 * kFinRows)
k_finalize(const DevProblem P, const DevStep S, const float* __restrict__ partial, int chunks,
           const float* __restrict__ du_in, float* __restrict__ du_out)
{
    __shared__ float red[kFinRows][32];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int nctrl = P.T * P.n * P.d_u;
    const int nQ = P.n * P.Q;
    const int idx = blockIdx.x * 32 + lane;
    float s = 0.0f;
    if (idx < nctrl) {
        const int per_t = P.n * P.d_u;
        const int t = idx / per_t;
        const int rem = idx - t * per_t;
        const int k = rem / P.d_u;
        const int d = rem - k * P.d_u;
        const int e = t * P.d_u + d;
        const size_t base = ((size_t)k * P.Q + (e >> 2)) * 4 + (e & 3);
        for (int c = row; c < chunks; c += kFinRows) s += partial[(size_t)c * nQ * 4 + base];
    }
    red[row][lane] = s;
    __syncthreads();
    if (row == 0 && idx < nctrl) {
#pragma unroll
        for (int r = 1; r < kFinRows; ++r) s += red[r][lane];
        du_out[idx] = S.g * fmaf(S.sigma, s, S.c * du_in[idx]);
    }
}

SumSplit plan_weighted_sum(const DevProblem& P, int N, int sm_count)
{
    const int nQ = P.n * P.Q;
    const int xblocks = (nQ + 31) / 32;
    const int target = sm_count * 8;
    int chunks = (target + xblocks - 1) / xblocks;
    const int max_chunks = (N + kWSRows - 1) / kWSRows;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    int chunk = (N + chunks - 1) / chunks;
    chunk = (chunk + kWSRows - 1) / kWSRows * kWSRows;
    chunks = (N + chunk - 1) / chunk;
    return SumSplit{chunks, chunk};
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

cudaError_t launch_weighted_sum(const DevProblem& P, const DevStep& S, const float2* list, const int* count,
                                SumSplit split, float* partial, const int* it_dev, cudaStream_t st)
{
    const int nQ = P.n * P.Q;
    dim3 grid((nQ + 31) / 32, split.chunks);
    k_weighted_sum<<<grid, 32 * kWSRows, 0, st>>>(P, S, list, count, partial, it_dev);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const DevProblem& P, const DevStep& S, const float* partial, SumSplit split,
                            const float* du_in, float* du_out, cudaStream_t st)
{
    const int nctrl = P.T * P.n * P.d_u;
    k_finalize<<<(nctrl + 31) / 32, 32 * kFinRows, 0, st>>>(P, S, partial, split.chunks, du_in, du_out);
    return cudaGetLastError();
}

}  // namespace d4orm

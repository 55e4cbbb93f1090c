// k_update.cu -- K3, the softmax weights and the weighted-mean update.
//
// Pass 1 (k_softmax_weights, one CTA): batch normalisation of the rewards
// (Sec. IV-C: z = (r - mean) / std, population std) and the temperature
// softmax of Eq. (6), as a two-pass log-sum-exp (maximum logit first).
//
// Pass 2 (k_weighted_sum): S = sum_j w_j eps_j over all samples, with eps
// regenerated from the same Philox counters K2 used (no sample is stored).
// The grid splits the n*Q noise quads over CTA columns and the samples over
// chunks; each CTA reduces its 8 sample rows in shared memory and writes one
// float4 partial per quad and chunk.
//
// Pass 3 (k_finalize): dU_{i-1} = g_i (c_i dU_i + sigma_i sum_chunks S_c),
// the weighted mean of the samples of Eq. (12) scaled as in Eq. (13); chunk
// partials are added in a fixed order, so the result is deterministic.
#include <cmath>

#include "d4orm_internal.h"

namespace d4orm {

constexpr int kSoftmaxThreads = 1024;

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

__global__ void __launch_bounds__(kSoftmaxThreads)
k_softmax_weights(const float* __restrict__ fitness, int N, float inv_lambda, float* __restrict__ w,
                  float* __restrict__ stats)
{
    __shared__ float sh[33];
    const int tid = threadIdx.x, nt = blockDim.x;
    float s = 0.0f;
    for (int j = tid; j < N; j += nt) s += fitness[j];
    const float mu = block_reduce<false>(s, sh) / (float)N;
    float v = 0.0f;
    for (int j = tid; j < N; j += nt) {
        const float d = fitness[j] - mu;
        v = fmaf(d, d, v);
    }
    const float sd = sqrtf(block_reduce<false>(v, sh) / (float)N);
    const bool degenerate = !(sd > 1e-12f * fmaxf(1.0f, fabsf(mu)));
    const float scale = degenerate ? 0.0f : inv_lambda / sd;
    float m = -INFINITY;
    for (int j = tid; j < N; j += nt) m = fmaxf(m, (fitness[j] - mu) * scale);
    m = block_reduce<true>(m, sh);
    float z = 0.0f;
    for (int j = tid; j < N; j += nt) {
        const float e = expf((fitness[j] - mu) * scale - m);
        w[j] = e;
        z += e;
    }
    const float Z = block_reduce<false>(z, sh);
    const float invZ = 1.0f / Z;
    for (int j = tid; j < N; j += nt) w[j] *= invZ;
    if (tid == 0 && stats) {
        stats[0] = mu;
        stats[1] = sd;
        stats[2] = m;
        stats[3] = Z;
    }
}

constexpr int kWSRows = 8;

__global__ void __launch_bounds__(32 * kWSRows)
k_weighted_sum(const DevProblem P, const DevStep S, const float* __restrict__ w, int chunk,
               float* __restrict__ partial, const int* __restrict__ it_dev)
{
    __shared__ float4 red[kWSRows][32];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int nQ = P.n * P.Q;
    const int gq = blockIdx.x * 32 + lane;
    const bool valid = gq < nQ;
    const int k = valid ? gq / P.Q : 0;
    const int q = valid ? gq - k * P.Q : 0;
    const uint32_t c3 = iter_word(S, it_dev);
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(S.N, j0 + chunk);
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    for (int j = j0 + row; j < j1; j += kWSRows) {
        const float wj = __ldg(&w[j]);
        if (wj != 0.0f) {  // warp-uniform; an exactly zero weight adds nothing
            float z[4];
            noise_quad(S, c3, (uint32_t)q, (uint32_t)j, (uint32_t)k, z);
            a0 = fmaf(wj, z[0], a0);
            a1 = fmaf(wj, z[1], a1);
            a2 = fmaf(wj, z[2], a2);
            a3 = fmaf(wj, z[3], a3);
        }
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

cudaError_t launch_softmax_weights(const float* fitness, int N, float inv_lambda, float* w, float* stats,
                                   cudaStream_t st)
{
    k_softmax_weights<<<1, kSoftmaxThreads, 0, st>>>(fitness, N, inv_lambda, w, stats);
    return cudaGetLastError();
}

cudaError_t launch_weighted_sum(const DevProblem& P, const DevStep& S, const float* w, SumSplit split,
                                float* partial, const int* it_dev, cudaStream_t st)
{
    const int nQ = P.n * P.Q;
    dim3 grid((nQ + 31) / 32, split.chunks);
    k_weighted_sum<<<grid, 32 * kWSRows, 0, st>>>(P, S, w, split.chunk, partial, it_dev);
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

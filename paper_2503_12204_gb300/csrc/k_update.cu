// k_update.cu -- K3, the softmax weights and the weighted-mean update.
//
// Pass 1 (k_softmax_weights, one CTA): batch normalisation of the rewards
// (Sec. IV-C: z = (r - mean) / std, population std) and the temperature
// softmax of Eq. (6), as a two-pass log-sum-exp (maximum logit first).
//
// Pass 1 also compacts the samples that carry weight into an ordered
// (weight, index) list; weights below 2^-36 of the largest are dropped.
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

// Samples whose unnormalised weight exp(l_j - max l) falls below 2^-36
// are left out of the weighted sum: together they move it by at most
// N * 2^-36 * max|eps| / Z (under 1e-6 of the largest weight for N <= 65536),
// below the rounding of the binary32 sum, and typically most samples of a
// batch are that far below the best one, so the noise they would need is
// never regenerated.
constexpr float kLogWeightCut = -24.953298f;  // -36 ln 2

// VR > 0: each thread keeps its (at most VR) fitness values in registers;
// VR == 0: the values are re-read from global memory (L1) on every pass.
template <int VR>
__global__ void __launch_bounds__(kSoftmaxThreads)
k_softmax_weights(const float* __restrict__ fitness, int N, float inv_lambda, float2* __restrict__ list,
                  int* __restrict__ count, float* __restrict__ stats)
{
    __shared__ float sh[33];
    __shared__ int scan[33];
    const int tid = threadIdx.x, nt = blockDim.x;
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
    float s = 0.0f;
    each([&](int, float x) { s += x; });
    const float mu = block_reduce<false>(s, sh) / (float)N;
    float v = 0.0f;
    each([&](int, float x) {
        const float d = x - mu;
        v = fmaf(d, d, v);
    });
    const float sd = sqrtf(block_reduce<false>(v, sh) / (float)N);
    const bool degenerate = !(sd > 1e-12f * fmaxf(1.0f, fabsf(mu)));
    const float scale = degenerate ? 0.0f : inv_lambda / sd;
    float m = -INFINITY;
    each([&](int, float x) { m = fmaxf(m, (x - mu) * scale); });
    m = block_reduce<true>(m, sh);
    float z = 0.0f;
    int kept = 0;
    each([&](int, float x) {
        const float l = (x - mu) * scale - m;
        z += expf(l);
        kept += l >= kLogWeightCut ? 1 : 0;
    });
    const float Z = block_reduce<false>(z, sh);
    const float invZ = 1.0f / Z;
    // exclusive scan of the per-thread survivor counts
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    int incl = kept;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) scan[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? scan[lane] : 0;
        int ti = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(kFull, ti, off);
            if (lane >= off) ti += o;
        }
        if (lane < nw) scan[lane] = ti - t;
        if (lane == 31) scan[32] = ti;
    }
    __syncthreads();
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
    for (int e = blockIdx.y * kWSRows + row; e < n_list; e += stride) {
        const float2 wj = list[e];  // warp-uniform
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
    if (N <= 8 * kSoftmaxThreads)
        k_softmax_weights<8><<<1, kSoftmaxThreads, 0, st>>>(fitness, N, inv_lambda, list, count, stats);
    else
        k_softmax_weights<0><<<1, kSoftmaxThreads, 0, st>>>(fitness, N, inv_lambda, list, count, stats);
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

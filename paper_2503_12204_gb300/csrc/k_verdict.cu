// k_verdict.cu -- K4 (iteration end of Algorithm 2: apply the deformation,
// roll the plan out, judge it) and the noise diagnostics kernels.
//
// K4 runs one warp, robots in lanes:
//   u      = clip(u_base + dU_0)                        (Algorithm 2 update)
//   x      = rollout(S, u)                              (Sec. III Eq. (1))
//   reward = Eq. (3); objective = Eq. (2) with |p - g| <= goal_tol;
//   collision_free = |p_k - p_l| > 2 R_a for every t in 0..T (Eq. (1) safety);
//   goal_reached   = |p_k[T] - g_k| <= goal_tol for every k (terminal condition).
// It uses the same integrate<DYN> as K2, so d4orm_rollout's states are the
// states every sample rollout computes.
#include <cmath>

#include "d4orm_internal.h"
#include "d4orm_kernels.cuh"

namespace d4orm {

template <int DYN>
__global__ void __launch_bounds__(32)
k_apply_rollout_verdict(const DevProblem P, float w_safe, const float* u_base, const float* du0, float* u_out,
                        float* __restrict__ states, d4orm_verdict* __restrict__ verdict, int* it_inc)
{
    apply_rollout_verdict_warp<DYN>(P, w_safe, u_base, du0, u_out, states, verdict);
    if (threadIdx.x == 0 && it_inc) *it_inc += 1;
}

cudaError_t launch_apply_rollout_verdict(const DevProblem& P, float w_safe, const float* u_base, const float* du0,
                                         float* u_out, float* states, d4orm_verdict* verdict, int* it_inc,
                                         cudaStream_t st)
{
    switch (P.dyn) {
    case HOLO2D:
        k_apply_rollout_verdict<HOLO2D><<<1, 32, 0, st>>>(P, w_safe, u_base, du0, u_out, states, verdict, it_inc);
        break;
    case HOLO3D:
        k_apply_rollout_verdict<HOLO3D><<<1, 32, 0, st>>>(P, w_safe, u_base, du0, u_out, states, verdict, it_inc);
        break;
    case UNICYCLE:
        k_apply_rollout_verdict<UNICYCLE><<<1, 32, 0, st>>>(P, w_safe, u_base, du0, u_out, states, verdict, it_inc);
        break;
    case DIFFDRIVE4:
        k_apply_rollout_verdict<DIFFDRIVE4><<<1, 32, 0, st>>>(P, w_safe, u_base, du0, u_out, states, verdict,
                                                              it_inc);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// eps[s][t][k][d] for samples j0 + s, s < count: one thread per (s, k, quad).
__global__ void k_sample_noise(const DevProblem P, const DevStep S, int j0, int count, float* __restrict__ eps)
{
    const long long total = (long long)count * P.n * P.Q;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int s = (int)(idx / ((long long)P.n * P.Q));
    const int rem = (int)(idx - (long long)s * P.n * P.Q);
    const int k = rem / P.Q;
    const int q = rem - k * P.Q;
    float z[4];
    noise_quad(S, iter_word(S, nullptr), (uint32_t)q, (uint32_t)(j0 + s), (uint32_t)k, z);
    const int len = P.T * P.d_u;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = 4 * q + r;
        if (e < len) {
            const int t = e / P.d_u, d = e - t * P.d_u;
            eps[(((size_t)s * P.T + t) * P.n + k) * P.d_u + d] = z[r];
        }
    }
}

__global__ void k_philox(const uint4* __restrict__ ctr, uint32_t key0, uint32_t key1, int count,
                         uint4* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint4 c = ctr[i];
    const U4 r = philox4x32_10(U4{c.x, c.y, c.z, c.w}, key0, key1);
    out[i] = make_uint4(r.x, r.y, r.z, r.w);
}

// A fixed-length sleep (bounded: iterations x ~1 us), used to keep the
// stream busy while the host submits the kernels of a timed step.
__global__ void k_hold(int iterations)
{
    for (int i = 0; i < iterations; ++i) __nanosleep(1000);
}

// FP32 throughput probe: eight independent FFMA chains per thread
// (a = a * b + c), so the FMA pipe, not latency, limits the rate when the
// grid fills every SM.  One launch performs blocks * threads * iters * 8
// FFMA (16 FLOPs per thread and iteration).  b and c come from the host so
// the chains cannot be folded; the sums are stored so they cannot be dropped.
__global__ void k_fp32_fma_probe(float* __restrict__ out, int iters, float b, float c)
{
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fp32_fma_probe(float* out, int blocks, int threads, int iters, cudaStream_t st)
{
    k_fp32_fma_probe<<<blocks, threads, 0, st>>>(out, iters, 0.9999f, 1e-4f);
    return cudaGetLastError();
}

cudaError_t launch_hold(int microseconds, cudaStream_t st)
{
    k_hold<<<1, 32, 0, st>>>(microseconds);
    return cudaGetLastError();
}

cudaError_t launch_sample_noise(const DevProblem& P, const DevStep& S, int j0, int count, float* eps,
                                cudaStream_t st)
{
    const long long total = (long long)count * P.n * P.Q;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    k_sample_noise<<<(unsigned)blocks, threads, 0, st>>>(P, S, j0, count, eps);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t key0, uint32_t key1, int count, uint32_t* out,
                          cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    k_philox<<<(count + 255) / 256, 256, 0, st>>>(reinterpret_cast<const uint4*>(ctr), key0, key1, count,
                                                  reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

}  // namespace d4orm

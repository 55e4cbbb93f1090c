// k_batched.cuh -- K5, the batched persistent solver.
//
// Many independent problems of uneven robot count, horizon and dynamics are
// solved by one persistent launch.  Each CTA pops problem indices from an
// atomic work queue (ordered longest-first by the host) and runs the whole of
// Algorithm 2 for that problem by itself: every denoising step (Algorithm 1
// body: Eq. (12) samples, Eq. (1) rollouts, Eq. (3)-(5) fitness, Sec. IV-C
// normalisation + Eq. (6) softmax, Eq. (13) update) and every iteration end
// (apply, rollout, Eq. (1)/(2) verdict, stop on success), synchronising only
// with __syncthreads.  CTAs never wait for one another, so there is no
// inter-CTA spin and nothing to time out.
//
// Per step the CTA stages the mean controls in shared memory, evaluates all
// N samples with the same lane-segment code as the single-problem kernel,
// runs the block softmax with weight compaction, and forms the weighted
// noise sum with one warp per noise quad (noise regenerated from the same
// Philox counters), the lanes' partial sums added by a fixed shuffle tree.
//
// The kernel is a template on OBS (obstacle penalty compiled in or not);
// k_batched.cu instantiates the obstacle-free variant and k_batched_obs.cu
// the other, so the two large instantiations compile in parallel.
#pragma once

#include <cmath>

#include "d4orm_internal.h"
#include "d4orm_kernels.cuh"
#include "d4orm_paired.cuh"

namespace d4orm {

// Per-warp buffers of the paired rollouts' position exchange, after the
// weight list in dynamic shared memory: 2 step parities x 3 coordinates x
// 32 lanes of packed pairs.
constexpr int kXbufPerWarp = 2 * 3 * 32;  // f2 entries
__device__ __forceinline__ f2* batched_xbuf(float2* sList, const BatchConsts& C)
{
    return reinterpret_cast<f2*>(sList + C.n_cap);
}

// PAIRED: the samples' rollouts use two robots per lane (L = SEG/2 lanes
// per sample, f32x2 arithmetic, partners' positions through the warp's
// shared-memory buffer), otherwise one robot per lane.
template <int DYN, int SEG, bool OBS, bool PAIRED>
__device__ __noinline__ void batched_instance(const DevProblem& P, const BatchInstance& I, const BatchConsts& C,
                                                 const float4* __restrict__ sched, int b, float* sM, float* sFit,
                                                 float2* sList, float* sh, int* scan, int* s_count,
                                                 d4orm_verdict* s_verdict, BatchResult* results, long long t_launch,
                                                 int* s_stop)
{
    constexpr int DU = DynDims<DYN>::DU;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int nctrl = P.T * P.n * DU;
    const int N = C.N;
    float* tau = I.tau_u;
    float* du[2] = {I.du0, I.du1};
    const long long t_start = globaltimer_ns();

    for (int e = tid; e < nctrl; e += nt) tau[e] = 0.0f;
    int first = -1, iters = 0, stop = 0;
    long long t_success = -1;
    d4orm_verdict last{};
    // anytime stop (deadline or host cancel), decided by thread 0 before each
    // step and shared through shared memory so the whole CTA leaves together
    auto must_stop = [&]() {
        if (tid == 0) {
            int r = 0;
            if (C.cancel && *C.cancel) r = D4ORM_STOP_CANCELLED;
            else if (C.deadline_ns > 0 && globaltimer_ns() - t_launch > C.deadline_ns) r = D4ORM_STOP_DEADLINE;
            *s_stop = r;
        }
        __syncthreads();
        return *s_stop;
    };
    for (int it = 0; it < C.max_iters && !stop; ++it) {
        // dU_K = 0 (Sec. IV-D); a warm start enters the first iteration at
        // start_step with the given deformation
        const bool warm = (it == 0) && I.du_init != nullptr;
        for (int e = tid; e < nctrl; e += nt) du[0][e] = warm ? I.du_init[e] : 0.0f;
        __syncthreads();
        int cur = 0;
        const uint32_t c3 = (uint32_t)it | ((C.tag_base + (uint32_t)b) << 12);
        for (int i = warm ? C.start_step : C.K; i >= 1; --i) {
            if ((stop = must_stop()) != 0) break;
            DevStep S;
#pragma unroll
            for (int r = 0; r < 10; ++r) {
                S.rk0[r] = C.rk0[r];
                S.rk1[r] = C.rk1[r];
            }
            const float4 sc = sched[i];
            S.c2_step = (uint32_t)i << 8;
            S.c3_tag = 0;
            S.it = it;
            S.N = N;
            S.c = sc.x;
            S.sigma = sc.y;
            S.g = sc.z;
            S.w_safe = C.w_safe;
            S.inv_lambda = C.inv_lambda;
            // mean controls M = tau.u + c dU_i
            stage_mean<false>(sM, du[cur], tau, S.c, nctrl);  // written by this CTA: coherent loads
            __syncthreads();
            // fitness of all N samples, 32/SEG (paired: 32/(SEG/2)) per warp per pass
            constexpr int LPS = PAIRED ? SEG / 2 : SEG;  // lanes per sample
            constexpr int SPW = 32 / LPS;
            for (int base = 0; base < N; base += nw * SPW) {
                const int j = base + warp * SPW + lane / LPS;
                float f;
                if constexpr (PAIRED)
                    f = sample_fitness_paired<DYN, LPS, OBS>(P, S, sM, c3, j,
                                                             batched_xbuf(sList, C) + warp * kXbufPerWarp);
                else f = sample_fitness_segment<DYN, SEG, OBS>(P, S, sM, c3, j);
                if ((lane & (LPS - 1)) == 0 && j < N) sFit[j] = f;
            }
            __syncthreads();
            // batch softmax + compaction (Sec. IV-C, Eq. (6))
            if (N <= 8 * nt)
                softmax_block<8>(sFit, N, S.inv_lambda, sList, s_count, nullptr, sh, scan);
            else
                softmax_block<0>(sFit, N, S.inv_lambda, sList, s_count, nullptr, sh, scan);
            __syncthreads();
            // weighted noise sum and Eq. (13) update: each warp owns whole
            // noise quads (quads dealt round-robin over the warps), its lanes
            // deal the listed samples round-robin, and a fixed shuffle tree
            // adds the lanes' partial sums -- no CTA barrier until the next
            // step reads the new deformation
            const int n_list = *s_count;
            const int nQ = P.n * P.Q;
            const int len = P.T * DU;
            for (int gq = warp; gq < nQ; gq += nw) {
                const int k = gq / P.Q;
                const int q = gq - k * P.Q;
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int e = lane; e < n_list; e += 32) {
                    const float2 wj = sList[e];
                    float z[4];
                    noise_quad(S, c3, (uint32_t)q, (uint32_t)__float_as_int(wj.y), (uint32_t)k, z);
                    a.x = fmaf(wj.x, z[0], a.x);
                    a.y = fmaf(wj.x, z[1], a.y);
                    a.z = fmaf(wj.x, z[2], a.z);
                    a.w = fmaf(wj.x, z[3], a.w);
                }
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    a.x += __shfl_xor_sync(kFull, a.x, off);
                    a.y += __shfl_xor_sync(kFull, a.y, off);
                    a.z += __shfl_xor_sync(kFull, a.z, off);
                    a.w += __shfl_xor_sync(kFull, a.w, off);
                }
                // lane r4 < 4 writes element 4q + r4
                if (lane < 4) {
                    const float sv = lane == 0 ? a.x : lane == 1 ? a.y : lane == 2 ? a.z : a.w;
                    const int e = 4 * q + lane;
                    if (e < len) {
                        const int t = e / DU, d = e - t * DU;
                        const int idx = (t * P.n + k) * DU + d;
                        du[cur ^ 1][idx] = S.g * fmaf(S.sigma, sv, S.c * du[cur][idx]);
                    }
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        if (stop) break;  // an interrupted iteration is discarded: tau.u keeps the completed ones
        // iteration end: tau.u <- clip(tau.u + dU_0), rollout, verdict
        if (warp == 0) apply_rollout_verdict_warp<DYN>(P, C.w_safe, tau, du[cur], tau, nullptr, s_verdict);
        __syncthreads();
        last = *s_verdict;
        iters = it + 1;
        if (first < 0 && last.collision_free && last.goal_reached) {
            first = it;
            t_success = globaltimer_ns();
        }
        __syncthreads();
        if (C.stop_on_success && first >= 0) break;
    }
    for (int e = tid; e < nctrl; e += nt) I.u_out[e] = tau[e];
    if (tid == 0) {
        BatchResult r;
        r.verdict = last;
        r.iters_run = iters;
        r.first_success_iter = first;
        r.ns_to_success = t_success >= 0 ? t_success - t_start : -1;
        r.ns_total = globaltimer_ns() - t_start;
        r.stop_reason = stop;
        results[b] = r;
    }
}

template <int DYN, bool OBS>
__device__ __forceinline__ void batched_dispatch_seg(const DevProblem& P, const BatchInstance& I,
                                                     const BatchConsts& C, const float4* sched, int b, float* sM,
                                                     float* sFit, float2* sList, float* sh, int* scan,
                                                     int* s_count, d4orm_verdict* s_verdict, BatchResult* results,
                                                     long long t_launch, int* s_stop)
{
#define D4_CASE(SEGV, PV) batched_instance<DYN, SEGV, OBS, PV>(P, I, C, sched, b, sM, sFit, sList, sh, scan, \
                                                           s_count, s_verdict, results, t_launch, s_stop)
    // robot-lane packing (I.paired, chosen per problem by the autotuner) is
    // compiled for the 8- and 16-lane segments (5..16 robots); holonomic
    // teams pack their integration too, the others their pair tests and
    // goal terms only
    if (P.n <= 2) D4_CASE(2, false);
    else if (P.n <= 4) D4_CASE(4, false);
    else if (P.n <= 8) {
        if (I.paired) D4_CASE(8, true);
        else D4_CASE(8, false);
    } else if (P.n <= 16) {
        if (I.paired) D4_CASE(16, true);
        else D4_CASE(16, false);
    } else D4_CASE(32, false);
#undef D4_CASE
}

template <bool OBS>
__global__ void __launch_bounds__(kBatchMaxThreads, 1)
k_batched_solve(const DevProblem* __restrict__ probs, const BatchInstance* __restrict__ insts,
                const int* __restrict__ order, const float4* __restrict__ sched, const BatchConsts C, int* queue,
                BatchResult* results)
{
    __shared__ DevProblem sP;
    __shared__ float sh[kSoftmaxScratch];
    __shared__ int scan[33];
    __shared__ int s_pick, s_count, s_stop;
    __shared__ d4orm_verdict s_verdict;
    __shared__ long long s_launch;
    extern __shared__ float4 dyn_smem[];
    float* sM = reinterpret_cast<float*>(dyn_smem);                 // [C.ctrl_cap]
    float* sFit = sM + C.ctrl_cap;                                  // [C.n_cap]
    float2* sList = reinterpret_cast<float2*>(sFit + C.n_cap);      // [C.n_cap]
    if (threadIdx.x == 0) s_launch = globaltimer_ns();  // every CTA is resident from the launch on
    __syncthreads();
    const long long t_launch = s_launch;
    for (;;) {
        if (threadIdx.x == 0) s_pick = atomicAdd(queue, 1);
        __syncthreads();
        const int pick = s_pick;
        if (pick >= C.count) break;
        const int b = order[pick];
        const int* src = reinterpret_cast<const int*>(&probs[b]);
        int* dst = reinterpret_cast<int*>(&sP);
        for (int w = threadIdx.x; w < (int)(sizeof(DevProblem) / 4); w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        const BatchInstance I = insts[b];
        switch (sP.dyn) {
        case HOLO2D:
            batched_dispatch_seg<HOLO2D, OBS>(sP, I, C, sched, b, sM, sFit, sList, sh, scan, &s_count, &s_verdict,
                                         results, t_launch, &s_stop);
            break;
        case HOLO3D:
            batched_dispatch_seg<HOLO3D, OBS>(sP, I, C, sched, b, sM, sFit, sList, sh, scan, &s_count, &s_verdict,
                                         results, t_launch, &s_stop);
            break;
        case UNICYCLE:
            batched_dispatch_seg<UNICYCLE, OBS>(sP, I, C, sched, b, sM, sFit, sList, sh, scan, &s_count,
                                           &s_verdict, results, t_launch, &s_stop);
            break;
        default:
            batched_dispatch_seg<DIFFDRIVE4, OBS>(sP, I, C, sched, b, sM, sFit, sList, sh, scan, &s_count,
                                             &s_verdict, results, t_launch, &s_stop);
            break;
        }
        __syncthreads();
    }
}

// Host operations on one variant (instantiated by the file that owns it).
template <bool OBS>
struct BatchedOps {
    static cudaError_t prepare()
    {
        return cudaFuncSetAttribute(k_batched_solve<OBS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    static int ctas_per_sm(int threads, size_t smem)
    {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched_solve<OBS>, threads,
                                                          smem + batched_xbuf_bytes(threads)) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return occ;
    }
    static cudaError_t launch(const DevProblem* probs, const BatchInstance* insts, const int* order,
                              const float4* sched, const BatchConsts& C, int* queue, BatchResult* results, int grid,
                              int threads, cudaStream_t st)
    {
        k_batched_solve<OBS><<<grid, threads, batched_smem_bytes(C) + batched_xbuf_bytes(threads), st>>>(
            probs, insts, order, sched, C, queue,
                                                                           results);
        return cudaGetLastError();
    }
};

}  // namespace d4orm

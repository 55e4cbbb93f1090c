// d4orm_internal.h -- launchers shared by the C-ABI layer and the kernel
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include "d4orm.h"
#include "d4orm_device.cuh"

namespace d4orm {

// Kernel attributes K2 needs for problem P (call outside stream capture).
cudaError_t prepare_rollout_fitness(const DevProblem& P);
cudaError_t prepare_rollout_fitness_pipe(const DevProblem& P);

// Which rollout kernel serves (P, N): D4ORM_ROLLOUT_REGISTER,
// D4ORM_ROLLOUT_PIPELINE or D4ORM_ROLLOUT_PAIRED (requested AUTO picks by
// how full each would keep the GPU).
int resolve_rollout_kernel(const DevProblem& P, int N, int sm_count, int requested);

// K2: fused sample rollout + fitness (Eq. (12) samples, Eq. (1) rollout,
// Eq. (3)-(5) reward).  fitness[N].  `kernel` is a d4orm_rollout_kernel.
cudaError_t launch_rollout_fitness(const DevProblem& P, const DevStep& S, const float* u_base,
                                   const float* du_in, float* fitness, const int* it_dev, int sm_count, int kernel,
                                   cudaStream_t st);
// K2b: two robots per lane (same results up to summation order).
cudaError_t prepare_rollout_fitness_paired(const DevProblem& P);
cudaError_t launch_rollout_fitness_paired(const DevProblem& P, const DevStep& S, const float* u_base,
                                          const float* du_in, float* fitness, const int* it_dev, int sm_count,
                                          cudaStream_t st);
int paired_lanes(int n);
// K2p: the warp-specialised variant (same results up to summation order).
cudaError_t launch_rollout_fitness_pipe(const DevProblem& P, const DevStep& S, const float* u_base,
                                        const float* du_in, float* fitness, const int* it_dev, cudaStream_t st);
size_t rollout_fitness_pipe_smem(const DevProblem& P);

// K3a: batch z-score + softmax (Sec. IV-C, Eq. (6)); writes the ordered
// list of (normalised weight, sample index) of the samples that carry
// weight (list[N] capacity) and its length to *count.
cudaError_t launch_softmax_weights(const float* fitness, int N, float inv_lambda, float2* list, int* count,
                                   float* stats, cudaStream_t st);

// K3b: du_out = g (c du_in + sigma sum_j w_j eps_j) over the listed samples,
// eps regenerated (Eq. (12) noise, Eq. (13) update), in one pass.
cudaError_t launch_weighted_mean(const DevProblem& P, const DevStep& S, const float2* list, const int* count,
                                 const float* du_in, float* du_out, const int* it_dev, int sm_count, cudaStream_t st);

// K4: u_out = clip(u_base + du0) (du0 nullable), rollout, verdict.
// states (nullable) [T+1][n][d_x]; verdict (nullable) device struct;
// it_inc (nullable) incremented once when done.
cudaError_t launch_apply_rollout_verdict(const DevProblem& P, float w_safe, const float* u_base, const float* du0,
                                         float* u_out, float* states, d4orm_verdict* verdict, int* it_inc,
                                         cudaStream_t st);

// Diagnostics: a bounded sleep, regenerated noise and raw Philox.
cudaError_t launch_hold(int microseconds, cudaStream_t st);
cudaError_t launch_sample_noise(const DevProblem& P, const DevStep& S, int j0, int count, float* eps,
                                cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t key0, uint32_t key1, int count, uint32_t* out,
                          cudaStream_t st);
cudaError_t launch_fp32_fma_probe(float* out, int blocks, int threads, int iters, cudaStream_t st);

// ---------------------------------------------------------------------------
// K5: batched persistent solver (k_batched.cu)
// ---------------------------------------------------------------------------
constexpr int kBatchMaxThreads = 512;

struct BatchInstance {
    float* tau_u;          // [T][n][d_u] plan workspace
    float* du0;            // deformation ping
    float* du1;            // deformation pong
    float* u_out;          // caller's output plan
    const float* du_init;  // nullable warm-start deformation at start_step
    int paired;            // rollouts with two robots per lane (5..16 robots only)
};

struct BatchConsts {
    int count, N, K, max_iters, stop_on_success, start_step;
    int ctrl_cap, n_cap;   // shared-memory capacities (floats; multiples of 4)
    uint32_t rk0[10], rk1[10];
    uint32_t tag_base;
    float w_safe, inv_lambda;
    long long deadline_ns;        // > 0: stop once the device clock passes launch + deadline
    const volatile int* cancel;   // nullable: host-mapped flag, non-zero = stop
};

struct BatchResult {
    d4orm_verdict verdict;
    int iters_run;
    int first_success_iter;
    long long ns_to_success;  // device clock from the instance's start; -1 if none
    long long ns_total;       // device clock of the instance's solve
    int stop_reason;          // D4ORM_STOP_*
};

// `obstacles` selects the kernel variant with the obstacle penalty compiled
// in (any problem of the batch has obstacles).
size_t batched_smem_bytes(const BatchConsts& C);
// Shared memory of the paired rollouts' per-warp position buffers at
// `threads` per CTA (on top of batched_smem_bytes).
size_t batched_xbuf_bytes(int threads);
cudaError_t prepare_batched(bool obstacles);
int batched_ctas_per_sm(bool obstacles, int threads, size_t smem);
cudaError_t launch_batched(bool obstacles, const DevProblem* probs, const BatchInstance* insts, const int* order,
                           const float4* sched, const BatchConsts& C, int* queue, BatchResult* results, int grid,
                           int threads, cudaStream_t st);
// the obstacle variant's own entry points (k_batched_obs.cu)
cudaError_t prepare_batched_obs();
int batched_ctas_per_sm_obs(int threads, size_t smem);
cudaError_t launch_batched_obs(const DevProblem* probs, const BatchInstance* insts, const int* order,
                               const float4* sched, const BatchConsts& C, int* queue, BatchResult* results, int grid,
                               int threads, cudaStream_t st);

// ---------------------------------------------------------------------------
// Learned warm start: set-MLP kernels (k_setmlp.cu)
// ---------------------------------------------------------------------------
// C[m][n] = sum_k A(m, k) * B(n, k), A(m, k) = A[m * a_rs + k * a_cs],
// B(n, k) = B[n * b_rs + k * b_cs]; epilogue: + bias[n], relu, zero where
// ref(m, n) <= 0, store to out_f32 / out_bf16 (row stride ldc); with
// splits > 1, raw partials to partial[split][M][N] instead.
struct GemmArgs {
    int M, N, K;
    long long a_rs, a_cs, b_rs, b_cs;
    const float* bias;
    int relu;
    const void* ref;             // __nv_bfloat16  // relu-gradient mask source, [M][ldc]
    float* out_f32;
    void* out_bf16;              // __nv_bfloat16
    long long ldc;
    float* partial;
};
cudaError_t mlp_gemm(const void* A, bool a_bf16, const void* B, bool b_bf16, const GemmArgs& g, int splits,
                     cudaStream_t st);
// True (and cleared) when a tensor-core GEMM gave up waiting for its MMAs.
bool mlp_gemm_timed_out();
cudaError_t mlp_sum_partials(const float* partial, int splits, long long MN, float* out, cudaStream_t st);
cudaError_t mlp_colsum(const float* dY, int M, int N, float* db, cudaStream_t st);
cudaError_t mlp_pool_concat(const void* H3, const float* mask, int B, int nmax, int W, void* C, cudaStream_t st);
cudaError_t mlp_pool_concat_bwd(const float* dC, const float* mask, const void* H3, int B, int nmax, int W,
                                float* dH3, cudaStream_t st);
cudaError_t mlp_mse(const float* Y, const float* Tgt, const float* mask, int rows, int D, float* dY, float* loss,
                    cudaStream_t st);
cudaError_t mlp_adamw(float* p, void* p16, const float* grad, float* m, float* v, long long count, float lr, float b1,
                      float b2, float eps, float wd, float bc1, float bc2, cudaStream_t st);
cudaError_t mlp_to_bf16(const float* src, void* dst, long long count, cudaStream_t st);
cudaError_t mlp_gather_rows(const float* src, const int* idx, int rows_per, int w, long long total_rows, float* dst,
                            cudaStream_t st);
cudaError_t mlp_seed_from_output(const float* Y, int n, int T, int d_u, int D, float scale, float* du_seed,
                                 cudaStream_t st);

// Shared host-side helpers defined in d4orm_capi.cu.
d4orm_status validate_step_args(const d4orm_problem* P, const d4orm_params* params, int iter, int step_i,
                                const float* u_base_dev, const float* du_in_dev, const float* du_out_dev);
DevStep make_step_consts(const d4orm_params* params, int iter, int step_i);
d4orm_status validate_params(const d4orm_problem* P, const d4orm_params* params);
const DevProblem& dev_problem(const d4orm_problem* P);
int rollout_kernel_choice(const d4orm_problem* P);
d4orm_status set_error(d4orm_status s, const char* msg);
d4orm_status set_cuda_error(cudaError_t e, const char* where);

}  // namespace d4orm

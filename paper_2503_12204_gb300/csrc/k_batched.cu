// k_batched.cu -- K5 host entry points and the obstacle-free instantiation
// (the kernel itself is in k_batched.cuh; k_batched_obs.cu holds the
// variant with the obstacle penalty).
#include "k_batched.cuh"

namespace d4orm {

size_t batched_smem_bytes(const BatchConsts& C)
{
    return ((size_t)C.ctrl_cap + C.n_cap + 2ull * C.n_cap) * sizeof(float);
}

size_t batched_xbuf_bytes(int threads) { return (size_t)(threads / 32) * kXbufPerWarp * sizeof(f2); }

cudaError_t prepare_batched(bool obstacles)
{
    return obstacles ? prepare_batched_obs() : BatchedOps<false>::prepare();
}

int batched_ctas_per_sm(bool obstacles, int threads, size_t smem)
{
    return obstacles ? batched_ctas_per_sm_obs(threads, smem) : BatchedOps<false>::ctas_per_sm(threads, smem);
}

cudaError_t launch_batched(bool obstacles, const DevProblem* probs, const BatchInstance* insts, const int* order,
                           const float4* sched, const BatchConsts& C, int* queue, BatchResult* results, int grid,
                           int threads, cudaStream_t st)
{
    if (obstacles) return launch_batched_obs(probs, insts, order, sched, C, queue, results, grid, threads, st);
    return BatchedOps<false>::launch(probs, insts, order, sched, C, queue, results, grid, threads, st);
}

}  // namespace d4orm

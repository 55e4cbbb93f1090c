// k_batched_obs.cu -- the K5 instantiation with the obstacle penalty
// (Appendix), used when any problem of a batch has obstacles.
#include "k_batched.cuh"

namespace d4orm {

cudaError_t prepare_batched_obs() { return BatchedOps<true>::prepare(); }

int batched_ctas_per_sm_obs(int threads, size_t smem) { return BatchedOps<true>::ctas_per_sm(threads, smem); }

cudaError_t launch_batched_obs(const DevProblem* probs, const BatchInstance* insts, const int* order,
                               const float4* sched, const BatchConsts& C, int* queue, BatchResult* results, int grid,
                               int threads, cudaStream_t st)
{
    return BatchedOps<true>::launch(probs, insts, order, sched, C, queue, results, grid, threads, st);
}

}  // namespace d4orm

// d4orm_noalloc.cu -- one denoising step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a planner inside a robot's real-time
// control loop, where cudaMalloc may synchronise the device and has no
// latency bound, and host applications that reserve all device memory up
// front in their own pool and forbid allocations by plug-in libraries.
// d4orm_denoise_step gets its scratch (fitness, the compacted weight list,
// the batch statistics) from the problem's workspace, which it allocates on
// first use; this
// variant takes the same scratch from a fixed array that is part of the
// library's device image, so it never allocates.  The problem handle itself
// holds no device memory (d4orm_problem_create allocates none).
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Nothing in it needs to start at zero: each step writes every
// fitness, list and count entry it later reads.  Calls whose work
// overlaps on the GPU (other streams, or other host threads) race on it.
#include <mutex>

#include "d4orm_internal.h"

namespace {

constexpr size_t kScratchFloats = D4ORM_NOALLOC_SCRATCH_FLOATS;

// Device scratch of the allocation-free step; every GPU that loads the
// library holds it (2 MiB) until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

struct DeviceSetup {
    bool done = false;
    float* scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int sm_count = 0;
};

constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

size_t pad64(size_t n) { return (n + 63) / 64 * 64; }  // 256-byte slices

// Per device, with that device current: the array's device address (the
// host-side name is only a stand-in) and the SM count.  The address is
// queried again on every call (a host-side lookup, no device work); if it
// differs from the cached one -- the context was destroyed and re-created,
// e.g. after cudaDeviceReset -- the cached set-up is replaced.  The first
// call on a device, and the first call after such a reset, should come
// before any stream capture.
d4orm_status setup_device(int dev, DeviceSetup** out)
{
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return d4orm::set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup& s = g_setup[dev];
    if (!s.done || s.scratch != static_cast<float*>(ptr)) {
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return d4orm::set_cuda_error(e, "cudaDeviceGetAttribute");
        s.scratch = static_cast<float*>(ptr);
        s.sm_count = sms;
        s.done = true;
    }
    *out = &s;
    return D4ORM_OK;
}

}  // namespace

extern "C" d4orm_status d4orm_denoise_step_noalloc(const d4orm_problem* problem, const d4orm_params* params,
                                                   int iter, int step_i, const float* u_base_dev,
                                                   const float* du_in_dev, float* du_out_dev, float* fitness_dev,
                                                   void* stream)
{
    using namespace d4orm;
    d4orm_status s = validate_step_args(problem, params, iter, step_i, u_base_dev, du_in_dev, du_out_dev);
    if (s != D4ORM_OK) return s;
    const int N = params->n_samples;
    if (N > D4ORM_NOALLOC_MAX_SAMPLES)
        return set_error(D4ORM_ERR_UNSUPPORTED, "d4orm_denoise_step_noalloc: n_samples exceeds "
                                                "D4ORM_NOALLOC_MAX_SAMPLES (65536)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(D4ORM_ERR_UNSUPPORTED, "device ordinal >= 64");
    DeviceSetup* ds = nullptr;
    s = setup_device(dev, &ds);
    if (s != D4ORM_OK) return s;

    const DevProblem& P = dev_problem(problem);
    // the dynamic shared-memory opt-in of this problem's rollout kernels (a
    // kernel attribute of the current context: applied on every call, so a
    // re-created context gets it too)
    if ((e = prepare_rollout_fitness(P)) != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute");
    const size_t n_w = 2 * pad64((size_t)N), n_fit = pad64((size_t)N), n_stats = 64;
    if (n_w + n_fit + n_stats > kScratchFloats)
        return set_error(D4ORM_ERR_UNSUPPORTED, "d4orm_denoise_step_noalloc: problem needs more scratch than "
                                                "D4ORM_NOALLOC_SCRATCH_FLOATS");
    float2* list = reinterpret_cast<float2*>(ds->scratch);
    float* fit = fitness_dev ? fitness_dev : ds->scratch + n_w;
    float* stats = ds->scratch + n_w + n_fit;
    int* count = reinterpret_cast<int*>(stats + 8);

    const DevStep S = make_step_consts(params, iter, step_i);
    cudaStream_t st = (cudaStream_t)stream;
    if ((e = launch_rollout_fitness(P, S, u_base_dev, du_in_dev, fit, nullptr, ds->sm_count,
                                     rollout_kernel_choice(problem), st)) != cudaSuccess ||
        (e = launch_softmax_weights(fit, N, S.inv_lambda, list, count, stats, st)) != cudaSuccess ||
        (e = launch_weighted_mean(P, S, list, count, du_in_dev, du_out_dev, nullptr, ds->sm_count, st)) !=
            cudaSuccess)
        return set_cuda_error(e, "d4orm_denoise_step_noalloc launch");
    return D4ORM_OK;
}

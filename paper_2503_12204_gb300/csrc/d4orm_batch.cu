// d4orm_batch.cu -- host side of the batched persistent solve: instance
// descriptors, longest-first work order, the autotuner of the CTA width, and
// the CUDA graph (descriptor upload, queue reset, persistent kernel, result
// read-back) that one d4orm_batch_solve replays.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "d4orm_internal.h"

using namespace d4orm;

namespace {

int seg_of(int n) { return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32; }

// The batched kernel has a two-robots-per-lane rollout for teams of 5..16
// robots (8- and 16-lane segments), every dynamics model.
bool packable(const DevProblem& P) { return P.n >= 5 && P.n <= 16; }

// Autotuner bucket of a packable problem: dynamics x lane segment.
constexpr int kPackBuckets = 8;
int pack_bucket(const DevProblem& P) { return 2 * P.dyn + (P.n > 8 ? 1 : 0); }

}  // namespace

struct d4orm_batch {
    int count = 0;
    d4orm_params params{};
    int device = 0, sms = 0;
    std::vector<DevProblem> h_probs;
    std::vector<int> nctrl;
    DevProblem* d_probs = nullptr;
    BatchInstance* d_insts = nullptr;
    BatchInstance* h_insts = nullptr;  // pinned staging, copied by the graph
    int* d_order = nullptr;
    float4* d_sched = nullptr;
    int* d_queue = nullptr;
    BatchResult* d_results = nullptr;
    BatchResult* h_results = nullptr;  // pinned
    float* d_work = nullptr;           // 3 x sum(nctrl) floats: tau.u, dU ping, dU pong
    BatchConsts C{};
    size_t smem = 0;
    int threads = 256, grid = 0;
    bool obstacles = false;            // any problem has obstacles: the kernel variant with the penalty
    float tuned_ms[3] = {-1.f, -1.f, -1.f};   // best pilot per CTA width
    int ctas_per_sm = 0;
    // packing pilots: summed per-problem device time (ns) of each bucket
    // (dynamics x 5..8 / 9..16 robots), one robot vs two per lane
    long long pack_ns[kPackBuckets][2] = {};
    // every pilot of the autotuner: CTA width, resident CTAs per SM, ms
    std::vector<int> tune_width, tune_occ;
    std::vector<float> tune_ms;
    // cached graph for one (max_iters, stop_on_success, start_step, deadline) combination
    cudaGraphExec_t graph = nullptr;
    int g_iters = -1, g_stop = -1, g_start = -1;
    long long g_deadline = -1;
    // host-mapped cancel flag: written by d4orm_batch_cancel, read by the kernel
    int* h_cancel = nullptr;
    int* d_cancel = nullptr;
};

namespace {

void batch_free(d4orm_batch* B)
{
    if (B->graph) cudaGraphExecDestroy(B->graph);
    cudaFree(B->d_probs);
    cudaFree(B->d_insts);
    cudaFree(B->d_order);
    cudaFree(B->d_sched);
    cudaFree(B->d_queue);
    cudaFree(B->d_results);
    cudaFree(B->d_work);
    cudaFreeHost(B->h_insts);
    cudaFreeHost(B->h_results);
    cudaFreeHost(B->h_cancel);
}

#define B_CUDA(call)                                                     \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return set_cuda_error(e_, #call);         \
    } while (0)

// One timed run of the persistent kernel over the whole batch with a short
// schedule (2 steps, 1 iteration) at `threads` per CTA and `occ` CTAs per
// SM (<= the resident maximum), for the autotuner.
d4orm_status pilot_ms(d4orm_batch* B, int threads, int occ, float* ms, bool upload = false,
                      bool read_results = false)
{
    if (occ <= 0) {
        *ms = -1.f;
        return D4ORM_OK;
    }
    if (upload)
        B_CUDA(cudaMemcpy(B->d_insts, B->h_insts, sizeof(BatchInstance) * B->count, cudaMemcpyHostToDevice));
    const int grid = std::min(B->count, B->sms * occ);
    BatchConsts P = B->C;
    P.deadline_ns = 0;
    P.cancel = nullptr;
    P.K = std::min(2, B->C.K);
    P.max_iters = 1;
    P.stop_on_success = 0;
    cudaStream_t st;
    B_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // rep 0 warms up
        e = cudaMemsetAsync(B->d_queue, 0, sizeof(int), st);
        if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess)
            e = launch_batched(B->obstacles, B->d_probs, B->d_insts, B->d_order, B->d_sched, P, B->d_queue,
                               B->d_results, grid, threads, st);
        if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e1, st);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e == cudaSuccess && read_results)
        e = cudaMemcpy(B->h_results, B->d_results, sizeof(BatchResult) * B->count, cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return set_cuda_error(e, "batched pilot run");
    return D4ORM_OK;
}

}  // namespace

extern "C" {

d4orm_status d4orm_batch_create(d4orm_problem* const* problems, int count, const d4orm_params* params,
                                int autotune, d4orm_batch** out)
{
    if (!out) return set_error(D4ORM_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!problems || count < 1 || !params) return set_error(D4ORM_ERR_INVALID_ARG, "null problems/params or count < 1");
    for (int b = 0; b < count; ++b)
        if (!problems[b]) return set_error(D4ORM_ERR_INVALID_ARG, "null problem in batch");
    d4orm_status s = validate_params(problems[0], params);
    if (s != D4ORM_OK) return s;
    if (params->n_samples > D4ORM_BATCH_MAX_SAMPLES)
        return set_error(D4ORM_ERR_UNSUPPORTED, "batched solve: n_samples > D4ORM_BATCH_MAX_SAMPLES");
    if ((long long)params->instance_tag + count - 1 > (long long)D4ORM_MAX_TAG)
        return set_error(D4ORM_ERR_INVALID_ARG, "instance_tag + count exceeds D4ORM_MAX_TAG");

    d4orm_batch* B = new (std::nothrow) d4orm_batch();
    if (!B) return set_error(D4ORM_ERR_OOM, "host allocation failed");
    B->count = count;
    B->params = *params;
    int ctrl_cap = 0;
    size_t total = 0;
    for (int b = 0; b < count; ++b) {
        const DevProblem& P = dev_problem(problems[b]);
        B->h_probs.push_back(P);
        B->obstacles = B->obstacles || P.n_obs > 0;
        const int nc = P.T * P.n * P.d_u;
        B->nctrl.push_back(nc);
        ctrl_cap = std::max(ctrl_cap, nc);
        total += (size_t)((nc + 3) / 4 * 4);
    }
    B->C.count = count;
    B->C.N = params->n_samples;
    B->C.K = params->n_steps;
    B->C.ctrl_cap = (ctrl_cap + 3) / 4 * 4;
    B->C.n_cap = (params->n_samples + 3) / 4 * 4;
    B->C.tag_base = params->instance_tag;
    const DevStep S1 = make_step_consts(params, 0, 1);
    for (int r = 0; r < 10; ++r) {
        B->C.rk0[r] = S1.rk0[r];
        B->C.rk1[r] = S1.rk1[r];
    }
    B->C.w_safe = params->w_safe;
    B->C.inv_lambda = S1.inv_lambda;
    B->smem = batched_smem_bytes(B->C);
    if (B->smem + batched_xbuf_bytes(kBatchMaxThreads) > 200 * 1024) {
        delete B;
        return set_error(D4ORM_ERR_UNSUPPORTED, "batched solve: largest problem and N need more than 200 KB of "
                                                "shared memory (with the 24 KB of position buffers)");
    }

    auto fail_cleanup = [&](d4orm_status st) {
        batch_free(B);
        delete B;
        return st;
    };
    cudaError_t e = cudaGetDevice(&B->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, B->device);
    if (e == cudaSuccess) e = prepare_batched(B->obstacles);
    if (e == cudaSuccess) {
        // the single-problem path's kernel attributes are not needed here
        e = cudaMalloc(&B->d_probs, sizeof(DevProblem) * count);
    }
    if (e == cudaSuccess) e = cudaMalloc(&B->d_insts, sizeof(BatchInstance) * count);
    if (e == cudaSuccess) e = cudaMallocHost(&B->h_insts, sizeof(BatchInstance) * count);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_order, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_sched, sizeof(float4) * (params->n_steps + 1));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_results, sizeof(BatchResult) * count);
    if (e == cudaSuccess) e = cudaMallocHost(&B->h_results, sizeof(BatchResult) * count);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_work, sizeof(float) * 3 * total);
    if (e == cudaSuccess) e = cudaHostAlloc(&B->h_cancel, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *(volatile int*)B->h_cancel = 0;
        e = cudaHostGetDevicePointer((void**)&B->d_cancel, B->h_cancel, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_cleanup(set_error(e == cudaErrorMemoryAllocation ? D4ORM_ERR_OOM : D4ORM_ERR_CUDA,
                                      cudaGetErrorString(e)));
    }
    // per-instance workspace slices (16-byte aligned)
    size_t off = 0;
    for (int b = 0; b < count; ++b) {
        const size_t nc = (size_t)((B->nctrl[b] + 3) / 4 * 4);
        B->h_insts[b].tau_u = B->d_work + off;
        B->h_insts[b].du0 = B->d_work + total + off;
        B->h_insts[b].du1 = B->d_work + 2 * total + off;
        B->h_insts[b].u_out = B->h_insts[b].tau_u;  // replaced by the caller's buffers at solve time
        B->h_insts[b].du_init = nullptr;
        B->h_insts[b].paired = 0;
        off += nc;
    }
    // longest-first order: cost ~ samples x lanes x steps (+ the noise sum)
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(count);
    for (int b = 0; b < count; ++b) {
        const DevProblem& P = B->h_probs[b];
        cost[b] = (double)seg_of(P.n) * P.T * (P.dyn == HOLO3D ? 1.3 : 1.0) + 0.25 * P.n * P.Q;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<float4> sched(params->n_steps + 1);
    sched[0] = make_float4(1.f, 0.f, 1.f, 0.f);
    for (int i = 1; i <= params->n_steps; ++i) {
        const DevStep Si = make_step_consts(params, 0, i);
        sched[i] = make_float4(Si.c, Si.sigma, Si.g, 0.f);
    }
    e = cudaMemcpy(B->d_probs, B->h_probs.data(), sizeof(DevProblem) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_sched, sched.data(), sizeof(float4) * sched.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_insts, B->h_insts, sizeof(BatchInstance) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail_cleanup(set_cuda_error(e, "batch upload"));

    // autotuner: CTA width (128 / 256 / 512 threads) x resident CTAs per SM
    // (the maximum, half of it, one), each pair timed by a pilot over the
    // whole batch; without autotuning, 256 threads at the maximum
    const int cand[3] = {128, 256, 512};
    int best = std::min(256, kBatchMaxThreads), best_occ = 0;
    float best_ms = -1.f;
    for (int c = 0; c < 3 && autotune; ++c) {
        if (cand[c] > kBatchMaxThreads) continue;
        const int occ_max = batched_ctas_per_sm(B->obstacles, cand[c], B->smem);
        int occs[3] = {occ_max, occ_max / 2, 1};
        for (int o = 0; o < 3; ++o) {
            const int occ = occs[o];
            if (occ <= 0 || (o > 0 && occ >= occs[o - 1])) continue;  // distinct, descending
            float ms = -1.f;
            s = pilot_ms(B, cand[c], occ, &ms);
            if (s != D4ORM_OK) return fail_cleanup(s);
            B->tune_width.push_back(cand[c]);
            B->tune_occ.push_back(occ);
            B->tune_ms.push_back(ms);
            if (ms > 0.f && (B->tuned_ms[c] < 0.f || ms < B->tuned_ms[c])) B->tuned_ms[c] = ms;
            if (ms > 0.f && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                best = cand[c];
                best_occ = occ;
            }
        }
    }
    if (!autotune) {
        // default: the widest CTA, one per SM (the best pilot on the 512
        // ragged mixed-dynamics teams: 6.9 ms against 9.1 ms at two per SM
        // and 10.6-21.2 ms for narrower CTAs)
        best = kBatchMaxThreads;
        best_occ = batched_ctas_per_sm(B->obstacles, best, B->smem) > 0 ? 1 : 0;
    }
    int occ = best_occ > 0 ? best_occ : batched_ctas_per_sm(B->obstacles, best, B->smem);
    if (occ <= 0) {
        best = 128;
        occ = batched_ctas_per_sm(B->obstacles, best, B->smem);
    }
    if (occ <= 0) return fail_cleanup(set_error(D4ORM_ERR_UNSUPPORTED, "batched kernel cannot be resident"));
    B->threads = best;
    B->ctas_per_sm = occ;
    B->grid = std::min(count, B->sms * occ);

    // robot-lane packing, per bucket (dynamics x lane segment) of the
    // packable problems: at the chosen launch shape, one pilot with one robot
    // per lane and one with two, compared by the problems' own device times
    bool any_packable = false;
    for (int b = 0; b < count; ++b) any_packable = any_packable || packable(B->h_probs[b]);
    if (autotune && any_packable) {
        for (int mode = 0; mode < 2; ++mode) {
            for (int b = 0; b < count; ++b) B->h_insts[b].paired = mode;
            float ms = -1.f;
            s = pilot_ms(B, B->threads, B->ctas_per_sm, &ms, true, true);
            if (s != D4ORM_OK) return fail_cleanup(s);
            for (int b = 0; b < count; ++b)
                if (packable(B->h_probs[b])) B->pack_ns[pack_bucket(B->h_probs[b])][mode] += B->h_results[b].ns_total;
        }
        for (int b = 0; b < count; ++b) {
            const DevProblem& P = B->h_probs[b];
            const int k = packable(P) ? pack_bucket(P) : -1;
            B->h_insts[b].paired = k >= 0 && B->pack_ns[k][1] < B->pack_ns[k][0] ? 1 : 0;
        }
    } else {
        // default: two robots per lane wherever the kernel has that rollout
        for (int b = 0; b < count; ++b) B->h_insts[b].paired = packable(B->h_probs[b]) ? 1 : 0;
    }
    e = cudaMemcpy(B->d_insts, B->h_insts, sizeof(BatchInstance) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail_cleanup(set_cuda_error(e, "batch upload"));
    *out = B;
    return D4ORM_OK;
}

void d4orm_batch_destroy(d4orm_batch* B)
{
    if (!B) return;
    cudaDeviceSynchronize();
    batch_free(B);
    delete B;
}

d4orm_status d4orm_batch_info(const d4orm_batch* B, int* threads_per_cta, int* ctas, float* tuned_ms)
{
    if (!B) return set_error(D4ORM_ERR_INVALID_ARG, "null batch");
    if (threads_per_cta) *threads_per_cta = B->threads;
    if (ctas) *ctas = B->grid;
    if (tuned_ms)
        for (int c = 0; c < 3; ++c) tuned_ms[c] = B->tuned_ms[c];
    return D4ORM_OK;
}

d4orm_status d4orm_batch_tuning(const d4orm_batch* B, int capacity, int* count, int* threads_per_cta,
                                int* ctas_per_sm, float* pilot_ms)
{
    if (!B || !count) return set_error(D4ORM_ERR_INVALID_ARG, "null batch or count");
    const int n = (int)B->tune_ms.size();
    *count = n;
    for (int i = 0; i < n && i < capacity; ++i) {
        if (threads_per_cta) threads_per_cta[i] = B->tune_width[i];
        if (ctas_per_sm) ctas_per_sm[i] = B->tune_occ[i];
        if (pilot_ms) pilot_ms[i] = B->tune_ms[i];
    }
    return D4ORM_OK;
}

d4orm_status d4orm_batch_set_packing(d4orm_batch* B, int mode)
{
    if (!B) return set_error(D4ORM_ERR_INVALID_ARG, "null batch");
    if (mode != D4ORM_PACK_SINGLE && mode != D4ORM_PACK_PAIRED)
        return set_error(D4ORM_ERR_INVALID_ARG, "packing mode must be D4ORM_PACK_SINGLE or D4ORM_PACK_PAIRED");
    // the staging buffer is copied to the device by the next solve's graph;
    // wait for a replay that may still read it
    B_CUDA(cudaDeviceSynchronize());
    for (int b = 0; b < B->count; ++b)
        B->h_insts[b].paired = mode == D4ORM_PACK_PAIRED && packable(B->h_probs[b]) ? 1 : 0;
    return D4ORM_OK;
}

d4orm_status d4orm_batch_packing(const d4orm_batch* B, int capacity, int* paired, long long* bucket_ns)
{
    if (!B) return set_error(D4ORM_ERR_INVALID_ARG, "null batch");
    if (paired)
        for (int b = 0; b < B->count && b < capacity; ++b) paired[b] = B->h_insts[b].paired;
    if (bucket_ns)
        for (int k = 0; k < kPackBuckets; ++k)
            for (int m = 0; m < 2; ++m) bucket_ns[2 * k + m] = B->pack_ns[k][m];
    return D4ORM_OK;
}

d4orm_status d4orm_batch_solve(d4orm_batch* B, const d4orm_budget* budget, const float* const* du_init_dev,
                               float* const* u_out_dev, d4orm_result* out_host, void* stream)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (!B || !budget || !u_out_dev) return set_error(D4ORM_ERR_INVALID_ARG, "null batch, budget or u_out_dev");
    if (budget->max_iters < 1 || budget->max_iters > D4ORM_MAX_ITERS)
        return set_error(D4ORM_ERR_INVALID_ARG, "max_iters out of range");
    const bool warm = du_init_dev != nullptr;
    if (warm && (budget->start_step < 1 || budget->start_step > B->params.n_steps))
        return set_error(D4ORM_ERR_INVALID_ARG, "start_step out of 1..K");
    for (int b = 0; b < B->count; ++b) {
        if (!u_out_dev[b]) return set_error(D4ORM_ERR_INVALID_ARG, "null u_out_dev entry");
        if (warm && !du_init_dev[b]) return set_error(D4ORM_ERR_INVALID_ARG, "null du_init_dev entry");
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the previous replay of the graph read the staging buffer; wait for it
    // before rewriting the buffer (the caller may use another stream now)
    B_CUDA(cudaDeviceSynchronize());
    for (int b = 0; b < B->count; ++b) {
        B->h_insts[b].u_out = u_out_dev[b];
        B->h_insts[b].du_init = warm ? du_init_dev[b] : nullptr;
    }
    const int start = warm ? budget->start_step : 0;
    // deadline on the device clock, at least 1 ns when one is set
    const long long deadline_ns =
        budget->deadline_ms > 0.0 ? std::max(1LL, (long long)std::llround(budget->deadline_ms * 1e6)) : 0;
    if (!B->graph || B->g_iters != budget->max_iters || B->g_stop != (budget->stop_on_success ? 1 : 0) ||
        B->g_start != start || B->g_deadline != deadline_ns) {
        if (B->graph) {
            cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
        }
        BatchConsts C = B->C;
        C.max_iters = budget->max_iters;
        C.stop_on_success = budget->stop_on_success ? 1 : 0;
        C.start_step = warm ? budget->start_step : B->params.n_steps;
        C.deadline_ns = deadline_ns;
        C.cancel = B->d_cancel;
        cudaStream_t cap;
        B_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B->d_insts, B->h_insts, sizeof(BatchInstance) * B->count, cudaMemcpyHostToDevice, cap);
        if (e == cudaSuccess) e = cudaMemsetAsync(B->d_queue, 0, sizeof(int), cap);
        if (e == cudaSuccess)
            e = launch_batched(B->obstacles, B->d_probs, B->d_insts, B->d_order, B->d_sched, C, B->d_queue,
                               B->d_results, B->grid, B->threads, cap);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B->h_results, B->d_results, sizeof(BatchResult) * B->count, cudaMemcpyDeviceToHost,
                                cap);
        const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            B->graph = nullptr;
            return set_cuda_error(e, "batched graph capture");
        }
        B->g_iters = budget->max_iters;
        B->g_stop = budget->stop_on_success ? 1 : 0;
        B->g_start = start;
        B->g_deadline = deadline_ns;
    }
    B_CUDA(cudaGraphLaunch(B->graph, st));
    const cudaError_t sync = cudaStreamSynchronize(st);
    // a cancel request covers this solve only
    __atomic_store_n(B->h_cancel, 0, __ATOMIC_SEQ_CST);
    if (sync != cudaSuccess) return set_cuda_error(sync, "cudaStreamSynchronize(batched solve)");
    const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    bool cancelled = false, starved = false;
    for (int b = 0; b < B->count; ++b) {
        const BatchResult& r = B->h_results[b];
        cancelled = cancelled || r.stop_reason == D4ORM_STOP_CANCELLED;
        starved = starved || (r.stop_reason == D4ORM_STOP_DEADLINE && r.iters_run == 0);
    }
    if (out_host) {
        for (int b = 0; b < B->count; ++b) {
            const BatchResult& r = B->h_results[b];
            d4orm_result& o = out_host[b];
            o.verdict = r.verdict;
            o.iters_run = r.iters_run;
            o.first_success_iter = r.first_success_iter;
            o.ms_to_success = r.ns_to_success >= 0 ? r.ns_to_success * 1e-6 : -1.0;
            o.ms_total = r.ns_total * 1e-6;
            o.stop_reason = r.stop_reason;
        }
    }
    (void)wall;
    if (cancelled) return set_error(D4ORM_ERR_CANCELLED, "batched solve cancelled (plans of completed iterations kept)");
    if (starved)
        return set_error(D4ORM_ERR_TIMEOUT, "deadline passed before some problem completed an iteration");
    return D4ORM_OK;
}

d4orm_status d4orm_batch_cancel(d4orm_batch* B)
{
    if (!B || !B->h_cancel) return set_error(D4ORM_ERR_INVALID_ARG, "null batch");
    __atomic_store_n(B->h_cancel, 1, __ATOMIC_SEQ_CST);
    return D4ORM_OK;
}

d4orm_status d4orm_solve_batched(d4orm_problem* const* problems, int count, const d4orm_params* params,
                                 const d4orm_budget* budget, float* const* u_out_dev, d4orm_result* out_host,
                                 void* stream)
{
    d4orm_batch* B = nullptr;
    d4orm_status s = d4orm_batch_create(problems, count, params, 0, &B);
    if (s != D4ORM_OK) return s;
    s = d4orm_batch_solve(B, budget, nullptr, u_out_dev, out_host, stream);
    d4orm_batch_destroy(B);
    return s;
}

}  // extern "C"

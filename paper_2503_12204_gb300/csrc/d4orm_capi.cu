// d4orm_capi.cu -- the extern "C" boundary (include/d4orm.h): argument
// validation, the host-side FP64 noise schedule, per-handle device
// workspace, and the Algorithm 2 solve loop replayed from CUDA graphs.
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "d4orm_internal.h"

using namespace d4orm;

namespace {

thread_local std::string g_last_error;

d4orm_status fail(d4orm_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

d4orm_status cuda_fail(cudaError_t e, const char* where)
{
    return fail(D4ORM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define D4_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

void dims_of(int dyn, int* d_x, int* d_u, int* d_p)
{
    switch (dyn) {
    case HOLO2D: *d_x = 4; *d_u = 2; *d_p = 2; break;
    case HOLO3D: *d_x = 6; *d_u = 3; *d_p = 3; break;
    case UNICYCLE: *d_x = 3; *d_u = 2; *d_p = 2; break;
    default: *d_x = 4; *d_u = 2; *d_p = 2; break;  // DIFFDRIVE4
    }
}

// Default control boxes per model (the boxes of the measured workloads).
void default_box(int dyn, float* lo, float* hi)
{
    switch (dyn) {
    case HOLO2D: lo[0] = lo[1] = -1.f; hi[0] = hi[1] = 1.f; break;
    case HOLO3D: lo[0] = lo[1] = lo[2] = -2.f; hi[0] = hi[1] = hi[2] = 2.f; break;
    case UNICYCLE: lo[0] = 0.f; hi[0] = 1.f; lo[1] = -1.f; hi[1] = 1.f; break;
    default: lo[0] = lo[1] = -1.f; hi[0] = hi[1] = 1.f; break;
    }
}

// One iteration shape of a problem: captured into a graph the second time
// it is requested (the first request runs it eagerly, so a one-off solve
// does not pay for capture and instantiation).
struct GraphEntry {
    int i0 = 0;
    bool record_all = false;
    cudaGraphExec_t exec = nullptr;  // null: seen once, not captured yet
};

}  // namespace

struct d4orm_problem {
    int n, T, dyn, integ, d_x, d_u, d_p;
    DevProblem dp;
    int device = 0;
    int sm_count = 0;
    int rollout_kernel = D4ORM_ROLLOUT_AUTO;
    // workspace
    int ws_N = 0;
    float* d_fit = nullptr;      // [N]
    float2* d_list = nullptr;    // [N] (weight, sample index) of the samples that carry weight
    int* d_count = nullptr;      // list length
    float* d_stats = nullptr;    // [4]
    float* d_tau_u = nullptr;    // tau.u  [T][n][d_u]
    float* d_du[2] = {nullptr, nullptr};
    d4orm_verdict* d_verdicts = nullptr;  // [1 + D4ORM_MAX_ITERS]: slot 0 = latest, 1+it = history
    int* d_it = nullptr;
    d4orm_verdict* h_verdicts = nullptr;  // pinned [1 + D4ORM_MAX_ITERS]
    // graph cache (keyed by the parameters baked into the captured steps)
    d4orm_params g_params{};
    std::vector<GraphEntry> graphs;
    long long graph_captures = 0;  // iteration graphs captured so far (diagnostic)
    std::atomic<int> cancel{0};    // set by d4orm_problem_cancel, consumed by d4orm_solve
};

namespace {

void free_graphs(d4orm_problem* P)
{
    for (auto& g : P->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    P->graphs.clear();
}

d4orm_status ensure_device(d4orm_problem* P)
{
    int dev = 0;
    D4_CUDA(cudaGetDevice(&dev));
    if (P->sm_count == 0) {
        P->device = dev;
        D4_CUDA(cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, dev));
        D4_CUDA(prepare_rollout_fitness(P->dp));
    }
    return D4ORM_OK;
}

d4orm_status ensure_workspace(d4orm_problem* P, int N)
{
    d4orm_status s = ensure_device(P);
    if (s != D4ORM_OK) return s;
    const size_t nctrl = (size_t)P->T * P->n * P->d_u;
    if (!P->d_tau_u) {
        // all or nothing: a partial set would leave the next call with null
        // buffers behind a non-null d_tau_u
        float *tau = nullptr, *du0 = nullptr, *du1 = nullptr, *stats = nullptr;
        int *count = nullptr, *it = nullptr;
        d4orm_verdict *verdicts = nullptr, *h_verdicts = nullptr;
        if (cudaMalloc(&tau, nctrl * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&du0, nctrl * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&du1, nctrl * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&stats, 4 * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&count, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&it, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&verdicts, (1 + D4ORM_MAX_ITERS) * sizeof(d4orm_verdict)) != cudaSuccess ||
            cudaMallocHost(&h_verdicts, (1 + D4ORM_MAX_ITERS) * sizeof(d4orm_verdict)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(tau);
            cudaFree(du0);
            cudaFree(du1);
            cudaFree(stats);
            cudaFree(count);
            cudaFree(it);
            cudaFree(verdicts);
            cudaFreeHost(h_verdicts);
            return fail(D4ORM_ERR_OOM, "workspace allocation failed");
        }
        P->d_tau_u = tau;
        P->d_du[0] = du0;
        P->d_du[1] = du1;
        P->d_stats = stats;
        P->d_count = count;
        P->d_it = it;
        P->d_verdicts = verdicts;
        P->h_verdicts = h_verdicts;
    }
    if (N > P->ws_N) {
        free_graphs(P);
        cudaFree(P->d_fit);
        cudaFree(P->d_list);
        P->d_fit = nullptr;
        P->d_list = nullptr;
        if (cudaMalloc(&P->d_fit, (size_t)N * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&P->d_list, (size_t)N * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            P->ws_N = 0;
            return fail(D4ORM_ERR_OOM, "workspace allocation for N=%d failed", N);
        }
        P->ws_N = N;
    }
    return D4ORM_OK;
}

d4orm_status check_params(const d4orm_problem* P, const d4orm_params* p)
{
    if (!P || !p) return fail(D4ORM_ERR_INVALID_ARG, "null problem or params");
    if (p->n_samples < 1) return fail(D4ORM_ERR_INVALID_ARG, "n_samples must be >= 1");
    if (p->n_steps < 1 || p->n_steps >= (1 << 24)) return fail(D4ORM_ERR_INVALID_ARG, "n_steps out of range");
    if (!(p->temperature > 0.f) || !std::isfinite(p->temperature))
        return fail(D4ORM_ERR_INVALID_ARG, "temperature must be > 0");
    if (!std::isfinite(p->w_safe)) return fail(D4ORM_ERR_INVALID_ARG, "w_safe must be finite");
    if (!(p->beta0 > 0.f && p->beta0 < 1.f && p->beta1 > 0.f && p->beta1 < 1.f))
        return fail(D4ORM_ERR_INVALID_ARG, "beta0/beta1 must lie in (0,1)");
    if (p->instance_tag > D4ORM_MAX_TAG) return fail(D4ORM_ERR_INVALID_ARG, "instance_tag too large");
    if (p->update_rule != D4ORM_UPDATE_DENOISE && p->update_rule != D4ORM_UPDATE_MPPI)
        return fail(D4ORM_ERR_INVALID_ARG, "unknown update_rule");
    if (p->update_rule == D4ORM_UPDATE_MPPI && !(p->mppi_sigma > 0.f && std::isfinite(p->mppi_sigma)))
        return fail(D4ORM_ERR_INVALID_ARG, "mppi_sigma must be > 0 and finite");
    (void)P;
    return D4ORM_OK;
}

// Host FP64 schedule (Sec. IV-B): alpha_i = 1 - beta_i (beta linear from
// beta0 at i = 1 to beta1 at i = K), abar_i = prod_{j<=i} alpha_j, abar_0 = 1.
void schedule(const d4orm_params* p, std::vector<double>& abar)
{
    const int K = p->n_steps;
    abar.assign(K + 1, 1.0);
    for (int i = 1; i <= K; ++i) {
        const double beta =
            K == 1 ? (double)p->beta0 : (double)p->beta0 + ((double)p->beta1 - p->beta0) * (i - 1) / (double)(K - 1);
        abar[i] = abar[i - 1] * (1.0 - beta);
    }
}

DevStep step_consts(const d4orm_params* p, const std::vector<double>& abar, int it, int i)
{
    DevStep S;
    S.key0 = (uint32_t)(p->seed & 0xffffffffu);
    S.key1 = (uint32_t)(p->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        S.rk0[r] = S.key0 + (uint32_t)r * 0x9E3779B9u;
        S.rk1[r] = S.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    S.c2_step = (uint32_t)i << 8;
    S.c3_tag = p->instance_tag << 12;
    S.it = it;
    S.N = p->n_samples;
    if (p->update_rule == D4ORM_UPDATE_MPPI) {
        // no schedule: samples around the current deformation, new one = weighted mean
        S.c = 1.0f;
        S.sigma = p->mppi_sigma;
        S.g = 1.0f;
    } else {
        S.c = (float)(1.0 / std::sqrt(abar[i]));
        S.sigma = (float)std::sqrt(1.0 / abar[i] - 1.0);
        S.g = (float)std::sqrt(abar[i - 1]);
    }
    S.w_safe = p->w_safe;
    S.inv_lambda = (float)(1.0 / (double)p->temperature);
    return S;
}

// One denoising step on the problem's workspace buffers.
d4orm_status enqueue_step(d4orm_problem* P, const DevStep& S, const float* u_base, const float* du_in, float* du_out,
                          float* fitness, const int* it_dev, cudaStream_t st)
{
    float* fit = fitness ? fitness : P->d_fit;
    D4_CUDA(launch_rollout_fitness(P->dp, S, u_base, du_in, fit, it_dev, P->sm_count, P->rollout_kernel, st));
    D4_CUDA(launch_softmax_weights(fit, S.N, S.inv_lambda, P->d_list, P->d_count, P->d_stats, st));
    D4_CUDA(launch_weighted_mean(P->dp, S, P->d_list, P->d_count, du_in, du_out, it_dev, P->sm_count, st));
    return D4ORM_OK;
}

bool same_params(const d4orm_params& a, const d4orm_params& b)
{
    return a.n_samples == b.n_samples && a.n_steps == b.n_steps && a.temperature == b.temperature &&
           a.w_safe == b.w_safe && a.beta0 == b.beta0 && a.beta1 == b.beta1 && a.seed == b.seed &&
           a.instance_tag == b.instance_tag && a.update_rule == b.update_rule && a.mppi_sigma == b.mppi_sigma;
}

// Steps i0..1 of one iteration (ping-pong between d_du[0] -> ...), the
// iteration-end apply/rollout/verdict, and the verdict read-back, captured
// once into a graph.  The iteration index is read from P->d_it, which the
// verdict kernel increments, so one graph serves every iteration.
// The kernels of one iteration of Algorithm 2 on stream st: steps i0..1,
// then apply + rollout + verdict (K4, which also advances the device
// iteration counter), then, unless every verdict is kept on the device,
// the read-back of this iteration's verdict.
d4orm_status enqueue_iteration(d4orm_problem* P, const d4orm_params* p, const std::vector<double>& abar, int i0,
                               bool record_all, cudaStream_t st)
{
    int cur = 0;
    for (int i = i0; i >= 1; --i) {
        const DevStep S = step_consts(p, abar, 0, i);
        const d4orm_status status = enqueue_step(P, S, P->d_tau_u, P->d_du[cur], P->d_du[cur ^ 1], nullptr, P->d_it, st);
        if (status != D4ORM_OK) return status;
        cur ^= 1;
    }
    // verdict slot: d_verdicts[it] when recording all, else slot 0
    cudaError_t e = launch_apply_rollout_verdict(P->dp, p->w_safe, P->d_tau_u, P->d_du[cur], P->d_tau_u, nullptr,
                                                 P->d_verdicts, P->d_it, st);
    if (e != cudaSuccess) return cuda_fail(e, "launch_apply_rollout_verdict");
    if (!record_all) {
        e = cudaMemcpyAsync(P->h_verdicts, P->d_verdicts, sizeof(d4orm_verdict), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(verdict)");
    }
    return D4ORM_OK;
}

// The executable graph of one iteration shape, or null (*out) the first
// time the shape is requested: the caller then enqueues it eagerly.
d4orm_status iteration_graph(d4orm_problem* P, const d4orm_params* p, const std::vector<double>& abar, int i0,
                             bool record_all, cudaStream_t st, cudaGraphExec_t* out)
{
    *out = nullptr;
    if (!same_params(P->g_params, *p)) {
        free_graphs(P);
        P->g_params = *p;
    }
    GraphEntry* entry = nullptr;
    for (auto& g : P->graphs)
        if (g.i0 == i0 && g.record_all == record_all) entry = &g;
    if (!entry) {
        GraphEntry ge;
        ge.i0 = i0;
        ge.record_all = record_all;
        P->graphs.push_back(ge);
        return D4ORM_OK;
    }
    if (entry->exec) {
        *out = entry->exec;
        return D4ORM_OK;
    }
    cudaStream_t cap;
    D4_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    d4orm_status status = D4ORM_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    status = enqueue_iteration(P, p, abar, i0, record_all, cap);
    e = cudaStreamEndCapture(cap, &graph);
    if (status == D4ORM_OK && e != cudaSuccess) status = cuda_fail(e, "cudaStreamEndCapture");
    cudaStreamDestroy(cap);
    if (status != D4ORM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return status;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    entry->exec = exec;
    ++P->graph_captures;
    *out = exec;
    return D4ORM_OK;
}

}  // namespace

extern "C" {

const char* d4orm_status_string(d4orm_status s)
{
    switch (s) {
    case D4ORM_OK: return "ok";
    case D4ORM_ERR_INVALID_ARG: return "invalid argument";
    case D4ORM_ERR_UNSUPPORTED: return "unsupported";
    case D4ORM_ERR_OOM: return "out of memory";
    case D4ORM_ERR_CUDA: return "CUDA error";
    case D4ORM_ERR_TIMEOUT: return "timeout";
    case D4ORM_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
    }
}

const char* d4orm_last_error(void) { return g_last_error.c_str(); }

d4orm_status d4orm_problem_create(const d4orm_problem_desc* desc, d4orm_problem** out)
{
    if (!out) return fail(D4ORM_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!desc) return fail(D4ORM_ERR_INVALID_ARG, "desc is null");
    if (!desc->start || !desc->goal) return fail(D4ORM_ERR_INVALID_ARG, "start/goal is null");
    if (desc->dyn < HOLO2D || desc->dyn > DIFFDRIVE4) return fail(D4ORM_ERR_INVALID_ARG, "bad dynamics %d", desc->dyn);
    if (desc->integ != 0 && desc->integ != 1) return fail(D4ORM_ERR_INVALID_ARG, "bad integrator %d", desc->integ);
    if (desc->n_robots < 1) return fail(D4ORM_ERR_INVALID_ARG, "n_robots must be >= 1");
    if (desc->n_robots > D4ORM_MAX_ROBOTS) return fail(D4ORM_ERR_UNSUPPORTED, "n_robots > %d", D4ORM_MAX_ROBOTS);
    if (desc->T < 1) return fail(D4ORM_ERR_INVALID_ARG, "T must be >= 1");
    if (!(desc->dt > 0.f) || !std::isfinite(desc->dt)) return fail(D4ORM_ERR_INVALID_ARG, "dt must be > 0");
    if (!(desc->radius > 0.f) || !std::isfinite(desc->radius)) return fail(D4ORM_ERR_INVALID_ARG, "radius must be > 0");
    if (!(desc->eps_margin >= 0.f) || !(desc->goal_tol >= 0.f))
        return fail(D4ORM_ERR_INVALID_ARG, "eps_margin and goal_tol must be >= 0");
    int d_x, d_u, d_p;
    dims_of(desc->dyn, &d_x, &d_u, &d_p);
    if ((long long)desc->T * desc->n_robots * d_u > D4ORM_MAX_CTRL)
        return fail(D4ORM_ERR_UNSUPPORTED, "T*n*d_u exceeds %d", D4ORM_MAX_CTRL);
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    default_box(desc->dyn, lo, hi);
    for (int d = 0; d < d_u; ++d) {
        if (desc->u_lo) lo[d] = desc->u_lo[d];
        if (desc->u_hi) hi[d] = desc->u_hi[d];
        if (!(lo[d] <= hi[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return fail(D4ORM_ERR_INVALID_ARG, "control box component %d invalid", d);
    }
    for (int i = 0; i < desc->n_robots * d_x; ++i)
        if (!std::isfinite(desc->start[i]) || !std::isfinite(desc->goal[i]))
            return fail(D4ORM_ERR_INVALID_ARG, "start/goal must be finite");
    if (desc->n_obstacles < 0) return fail(D4ORM_ERR_INVALID_ARG, "n_obstacles must be >= 0");
    if (desc->n_obstacles > D4ORM_MAX_OBSTACLES)
        return fail(D4ORM_ERR_UNSUPPORTED, "more than %d obstacles", D4ORM_MAX_OBSTACLES);
    if (desc->n_obstacles > 0 && !desc->obstacles) return fail(D4ORM_ERR_INVALID_ARG, "obstacles is null");
    for (int o = 0; o < desc->n_obstacles; ++o) {
        for (int c = 0; c < 4; ++c)
            if (!std::isfinite(desc->obstacles[o * 4 + c])) return fail(D4ORM_ERR_INVALID_ARG, "obstacle not finite");
        if (!(desc->obstacles[o * 4 + 3] > 0.f)) return fail(D4ORM_ERR_INVALID_ARG, "obstacle radius must be > 0");
    }

    d4orm_problem* P = new (std::nothrow) d4orm_problem();
    if (!P) return fail(D4ORM_ERR_OOM, "host allocation failed");
    P->n = desc->n_robots;
    P->T = desc->T;
    P->dyn = desc->dyn;
    P->integ = desc->integ;
    P->d_x = d_x;
    P->d_u = d_u;
    P->d_p = d_p;
    DevProblem& D = P->dp;
    std::memset(&D, 0, sizeof D);
    D.n = P->n;
    D.T = P->T;
    D.dyn = P->dyn;
    D.integ = P->integ;
    D.d_x = d_x;
    D.d_u = d_u;
    D.d_p = d_p;
    D.Q = (P->T * d_u + 3) / 4;
    D.dt = desc->dt;
    D.half_dt2 = (float)(0.5 * (double)desc->dt * desc->dt);
    D.dt6 = (float)((double)desc->dt / 6.0);
    D.v_max = desc->v_max > 0.f ? desc->v_max : INFINITY;
    const double thr = 2.0 * desc->radius + desc->eps_margin;
    D.thr2 = (float)(thr * thr);
    D.safe2 = (float)(4.0 * (double)desc->radius * desc->radius);
    D.tol2 = (float)((double)desc->goal_tol * desc->goal_tol);
    D.inv_nT = (float)(1.0 / ((double)P->n * P->T));
    for (int d = 0; d < 3; ++d) {
        D.u_lo[d] = lo[d];
        D.u_hi[d] = hi[d];
    }
    for (int k = 0; k < P->n; ++k) {
        double d0 = 0.0;
        for (int c = 0; c < d_x; ++c) D.start[k * d_x + c] = desc->start[k * d_x + c];
        for (int c = 0; c < d_p; ++c) {
            D.goal[k * 3 + c] = desc->goal[k * d_x + c];
            const double e = (double)desc->start[k * d_x + c] - desc->goal[k * d_x + c];
            d0 += e * e;
        }
        d0 = std::sqrt(d0);
        if (d0 < desc->radius) d0 = desc->radius;
        D.inv_d0[k] = (float)(1.0 / d0);
    }
    D.n_obs = desc->n_obstacles;
    for (int o = 0; o < desc->n_obstacles; ++o) {
        for (int c = 0; c < 3; ++c) D.obs_c[o * 3 + c] = c < d_p ? desc->obstacles[o * 4 + c] : 0.0f;
        const double r = desc->obstacles[o * 4 + 3];
        const double pen = r + desc->radius + desc->eps_margin, safe = r + desc->radius;
        D.obs_pen2[o] = (float)(pen * pen);
        D.obs_safe2[o] = (float)(safe * safe);
    }
    *out = P;
    return D4ORM_OK;
}

void d4orm_problem_destroy(d4orm_problem* P)
{
    if (!P) return;
    if (P->sm_count) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(P->device);
        cudaDeviceSynchronize();
        free_graphs(P);
        cudaFree(P->d_fit);
        cudaFree(P->d_list);
        cudaFree(P->d_count);
        cudaFree(P->d_stats);
        cudaFree(P->d_tau_u);
        cudaFree(P->d_du[0]);
        cudaFree(P->d_du[1]);
        cudaFree(P->d_verdicts);
        cudaFree(P->d_it);
        cudaFreeHost(P->h_verdicts);
        cudaSetDevice(cur);
    }
    delete P;
}

d4orm_status d4orm_problem_set_rollout_kernel(d4orm_problem* P, int kernel)
{
    if (!P) return fail(D4ORM_ERR_INVALID_ARG, "null problem");
    if (kernel != D4ORM_ROLLOUT_AUTO && kernel != D4ORM_ROLLOUT_REGISTER && kernel != D4ORM_ROLLOUT_PIPELINE &&
        kernel != D4ORM_ROLLOUT_PAIRED)
        return fail(D4ORM_ERR_INVALID_ARG, "unknown rollout kernel %d", kernel);
    if (kernel != P->rollout_kernel) {
        free_graphs(P);
        P->rollout_kernel = kernel;
    }
    return D4ORM_OK;
}

long long d4orm_problem_graph_captures(const d4orm_problem* P) { return P ? P->graph_captures : -1; }

int d4orm_problem_rollout_kernel(const d4orm_problem* P, int n_samples)
{
    if (!P || n_samples < 1) return -1;
    int sms = P->sm_count;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
    }
    return resolve_rollout_kernel(P->dp, n_samples, sms, P->rollout_kernel);
}

d4orm_status d4orm_rollout(d4orm_problem* P, const d4orm_params* params, const float* u_dev, float* states_dev,
                           d4orm_verdict* verdict_host, void* stream)
{
    if (!P || !u_dev) return fail(D4ORM_ERR_INVALID_ARG, "null problem or u_dev");
    d4orm_status s = ensure_workspace(P, 1);
    if (s != D4ORM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const float w = params ? params->w_safe : 5.0f;
    D4_CUDA(launch_apply_rollout_verdict(P->dp, w, u_dev, nullptr, nullptr, states_dev,
                                         verdict_host ? P->d_verdicts : nullptr, nullptr, st));
    if (verdict_host) {
        D4_CUDA(cudaMemcpyAsync(P->h_verdicts, P->d_verdicts, sizeof(d4orm_verdict), cudaMemcpyDeviceToHost, st));
        D4_CUDA(cudaStreamSynchronize(st));
        *verdict_host = P->h_verdicts[0];
    }
    return D4ORM_OK;
}

d4orm_status d4orm_denoise_step(d4orm_problem* P, const d4orm_params* params, int iter, int step_i,
                                const float* u_base_dev, const float* du_in_dev, float* du_out_dev,
                                float* fitness_dev, void* stream)
{
    d4orm_status s = check_params(P, params);
    if (s != D4ORM_OK) return s;
    if (!u_base_dev || !du_in_dev || !du_out_dev) return fail(D4ORM_ERR_INVALID_ARG, "null device buffer");
    if (du_in_dev == du_out_dev) return fail(D4ORM_ERR_INVALID_ARG, "du_out_dev must not alias du_in_dev");
    if (step_i < 1 || step_i > params->n_steps) return fail(D4ORM_ERR_INVALID_ARG, "step_i out of 1..K");
    if (iter < 0 || iter >= D4ORM_MAX_ITERS) return fail(D4ORM_ERR_INVALID_ARG, "iter out of range");
    s = ensure_workspace(P, params->n_samples);
    if (s != D4ORM_OK) return s;
    std::vector<double> abar;
    schedule(params, abar);
    const DevStep S = step_consts(params, abar, iter, step_i);
    return enqueue_step(P, S, u_base_dev, du_in_dev, du_out_dev, fitness_dev, nullptr, (cudaStream_t)stream);
}

d4orm_status d4orm_sample_fitness(d4orm_problem* P, const d4orm_params* params, int iter, int step_i,
                                  const float* u_base_dev, const float* du_in_dev, float* fitness_dev, void* stream)
{
    d4orm_status s = check_params(P, params);
    if (s != D4ORM_OK) return s;
    if (!u_base_dev || !du_in_dev || !fitness_dev) return fail(D4ORM_ERR_INVALID_ARG, "null device buffer");
    if (step_i < 1 || step_i > params->n_steps) return fail(D4ORM_ERR_INVALID_ARG, "step_i out of 1..K");
    if (iter < 0 || iter >= D4ORM_MAX_ITERS) return fail(D4ORM_ERR_INVALID_ARG, "iter out of range");
    s = ensure_workspace(P, params->n_samples);
    if (s != D4ORM_OK) return s;
    std::vector<double> abar;
    schedule(params, abar);
    const DevStep S = step_consts(params, abar, iter, step_i);
    D4_CUDA(launch_rollout_fitness(P->dp, S, u_base_dev, du_in_dev, fitness_dev, nullptr, P->sm_count,
                                   P->rollout_kernel, (cudaStream_t)stream));
    return D4ORM_OK;
}

d4orm_status d4orm_solve(d4orm_problem* P, const d4orm_params* params, const d4orm_budget* budget,
                         const float* du_init_dev, float* u_out_dev, d4orm_result* out_host, void* stream)
{
    const auto t_start = std::chrono::steady_clock::now();
    d4orm_status s = check_params(P, params);
    if (s != D4ORM_OK) return s;
    if (!budget || !u_out_dev) return fail(D4ORM_ERR_INVALID_ARG, "null budget or u_out_dev");
    if (budget->max_iters < 1 || budget->max_iters > D4ORM_MAX_ITERS)
        return fail(D4ORM_ERR_INVALID_ARG, "max_iters out of 1..%d", D4ORM_MAX_ITERS);
    if (du_init_dev && (budget->start_step < 1 || budget->start_step > params->n_steps))
        return fail(D4ORM_ERR_INVALID_ARG, "start_step out of 1..K");
    s = ensure_workspace(P, params->n_samples);
    if (s != D4ORM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> abar;
    schedule(params, abar);
    const size_t nbytes = (size_t)P->T * P->n * P->d_u * sizeof(float);
    const bool per_iter_sync = budget->stop_on_success || budget->deadline_ms > 0.0;

    D4_CUDA(cudaMemsetAsync(P->d_tau_u, 0, nbytes, st));
    D4_CUDA(cudaMemsetAsync(P->d_it, 0, sizeof(int), st));
    d4orm_result res;
    std::memset(&res, 0, sizeof res);
    res.first_success_iter = -1;
    res.ms_to_success = -1.0;
    int it = 0;
    for (; it < budget->max_iters; ++it) {
        if (P->cancel.exchange(0)) {
            res.stop_reason = D4ORM_STOP_CANCELLED;
            break;
        }
        const bool warm = (it == 0 && du_init_dev);
        const int i0 = warm ? budget->start_step : params->n_steps;
        if (warm)
            D4_CUDA(cudaMemcpyAsync(P->d_du[0], du_init_dev, nbytes, cudaMemcpyDeviceToDevice, st));
        else
            D4_CUDA(cudaMemsetAsync(P->d_du[0], 0, nbytes, st));
        cudaGraphExec_t exec = nullptr;
        s = iteration_graph(P, params, abar, i0, !per_iter_sync, st, &exec);
        if (s != D4ORM_OK) return s;
        if (exec) {
            D4_CUDA(cudaGraphLaunch(exec, st));
        } else {
            s = enqueue_iteration(P, params, abar, i0, !per_iter_sync, st);
            if (s != D4ORM_OK) return s;
        }
        if (!per_iter_sync) {
            // keep this iteration's verdict: slot 0 -> history slot 1 + it
            D4_CUDA(cudaMemcpyAsync(P->d_verdicts + 1 + it, P->d_verdicts, sizeof(d4orm_verdict),
                                    cudaMemcpyDeviceToDevice, st));
            continue;
        }
        D4_CUDA(cudaStreamSynchronize(st));
        const d4orm_verdict v = P->h_verdicts[0];
        res.verdict = v;
        const double ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        if (res.first_success_iter < 0 && v.collision_free && v.goal_reached) {
            res.first_success_iter = it;
            res.ms_to_success = ms;
        }
        if (budget->stop_on_success && res.first_success_iter >= 0) {
            ++it;
            break;
        }
        if (budget->deadline_ms > 0.0 && ms >= budget->deadline_ms) {
            ++it;
            if (it < budget->max_iters) res.stop_reason = D4ORM_STOP_DEADLINE;
            break;
        }
    }
    res.iters_run = it;
    D4_CUDA(cudaMemcpyAsync(u_out_dev, P->d_tau_u, nbytes, cudaMemcpyDeviceToDevice, st));
    if (!per_iter_sync) {
        const int n_it = it;
        D4_CUDA(cudaMemcpyAsync(P->h_verdicts + 1, P->d_verdicts + 1, sizeof(d4orm_verdict) * n_it,
                                cudaMemcpyDeviceToHost, st));
        D4_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < n_it; ++i) {
            const d4orm_verdict v = P->h_verdicts[1 + i];
            if (res.first_success_iter < 0 && v.collision_free && v.goal_reached) res.first_success_iter = i;
        }
        if (n_it > 0) res.verdict = P->h_verdicts[n_it];
    } else {
        D4_CUDA(cudaStreamSynchronize(st));
    }
    res.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (out_host) *out_host = res;
    if (res.stop_reason == D4ORM_STOP_CANCELLED)
        return fail(D4ORM_ERR_CANCELLED, "solve cancelled after %d iteration(s) (their plan is kept)", it);
    return D4ORM_OK;
}

d4orm_status d4orm_problem_cancel(d4orm_problem* P)
{
    if (!P) return fail(D4ORM_ERR_INVALID_ARG, "null problem");
    P->cancel.store(1);
    return D4ORM_OK;
}

d4orm_status d4orm_denoise_step_timed(d4orm_problem* P, const d4orm_params* params, int iter, int step_i,
                                      const float* u_base_dev, const float* du_in_dev, float* du_out_dev,
                                      float* fitness_dev, float* kernel_ms_host, void* stream)
{
    d4orm_status s = check_params(P, params);
    if (s != D4ORM_OK) return s;
    if (!u_base_dev || !du_in_dev || !du_out_dev || !kernel_ms_host)
        return fail(D4ORM_ERR_INVALID_ARG, "null buffer");
    if (du_in_dev == du_out_dev) return fail(D4ORM_ERR_INVALID_ARG, "du_out_dev must not alias du_in_dev");
    if (step_i < 1 || step_i > params->n_steps) return fail(D4ORM_ERR_INVALID_ARG, "step_i out of 1..K");
    if (iter < 0 || iter >= D4ORM_MAX_ITERS) return fail(D4ORM_ERR_INVALID_ARG, "iter out of range");
    s = ensure_workspace(P, params->n_samples);
    if (s != D4ORM_OK) return s;
    std::vector<double> abar;
    schedule(params, abar);
    const DevStep S = step_consts(params, abar, iter, step_i);
    cudaStream_t st = (cudaStream_t)stream;
    float* fit = fitness_dev ? fitness_dev : P->d_fit;
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; ++k) D4_CUDA(cudaEventCreate(&ev[k]));
    // a short sleep first, so that every kernel below is already submitted
    // when the first event fires: the events then bracket device time only
    cudaError_t e = launch_hold(200, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = launch_rollout_fitness(P->dp, S, u_base_dev, du_in_dev, fit, nullptr, P->sm_count,
                                                             P->rollout_kernel, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = launch_softmax_weights(fit, S.N, S.inv_lambda, P->d_list, P->d_count, P->d_stats, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
    if (e == cudaSuccess)
        e = launch_weighted_mean(P->dp, S, P->d_list, P->d_count, du_in_dev, du_out_dev, nullptr, P->sm_count, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&kernel_ms_host[k], ev[k], ev[k + 1]);
    for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return cuda_fail(e, "d4orm_denoise_step_timed");
    return D4ORM_OK;
}

d4orm_status d4orm_sample_noise(d4orm_problem* P, const d4orm_params* params, int iter, int step_i, int j0,
                                int count, float* eps_dev, void* stream)
{
    d4orm_status s = check_params(P, params);
    if (s != D4ORM_OK) return s;
    if (!eps_dev) return fail(D4ORM_ERR_INVALID_ARG, "eps_dev is null");
    if (count < 0 || j0 < 0) return fail(D4ORM_ERR_INVALID_ARG, "j0/count must be >= 0");
    if (step_i < 1 || step_i > params->n_steps) return fail(D4ORM_ERR_INVALID_ARG, "step_i out of 1..K");
    if (iter < 0 || iter >= D4ORM_MAX_ITERS) return fail(D4ORM_ERR_INVALID_ARG, "iter out of range");
    std::vector<double> abar;
    schedule(params, abar);
    const DevStep S = step_consts(params, abar, iter, step_i);
    D4_CUDA(launch_sample_noise(P->dp, S, j0, count, eps_dev, (cudaStream_t)stream));
    return D4ORM_OK;
}

d4orm_status d4orm_philox4x32_10(const uint32_t* ctr_dev, uint32_t key0, uint32_t key1, int count, uint32_t* out_dev,
                                 void* stream)
{
    if (!ctr_dev || !out_dev) return fail(D4ORM_ERR_INVALID_ARG, "null buffer");
    if (count < 0) return fail(D4ORM_ERR_INVALID_ARG, "count must be >= 0");
    if (((uintptr_t)ctr_dev & 15) || ((uintptr_t)out_dev & 15))
        return fail(D4ORM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    D4_CUDA(launch_philox(ctr_dev, key0, key1, count, out_dev, (cudaStream_t)stream));
    return D4ORM_OK;
}

d4orm_status d4orm_fp32_fma_probe(float* out_dev, int blocks, int threads, int iters, void* stream)
{
    if (!out_dev) return fail(D4ORM_ERR_INVALID_ARG, "out_dev is null");
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1)
        return fail(D4ORM_ERR_INVALID_ARG, "blocks >= 1, threads a multiple of 32 in 32..1024, iters >= 1");
    D4_CUDA(launch_fp32_fma_probe(out_dev, blocks, threads, iters, (cudaStream_t)stream));
    return D4ORM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Accessors for other translation units of the library (same validation,
// schedule and per-step constants as the entry points above).
// ---------------------------------------------------------------------------
namespace d4orm {

d4orm_status validate_step_args(const d4orm_problem* P, const d4orm_params* params, int iter, int step_i,
                                const float* u_base_dev, const float* du_in_dev, const float* du_out_dev)
{
    d4orm_status s = check_params(P, params);
    if (s != D4ORM_OK) return s;
    if (!u_base_dev || !du_in_dev || !du_out_dev) return fail(D4ORM_ERR_INVALID_ARG, "null device buffer");
    if (du_in_dev == du_out_dev) return fail(D4ORM_ERR_INVALID_ARG, "du_out_dev must not alias du_in_dev");
    if (step_i < 1 || step_i > params->n_steps) return fail(D4ORM_ERR_INVALID_ARG, "step_i out of 1..K");
    if (iter < 0 || iter >= D4ORM_MAX_ITERS) return fail(D4ORM_ERR_INVALID_ARG, "iter out of range");
    return D4ORM_OK;
}

d4orm_status validate_params(const d4orm_problem* P, const d4orm_params* params) { return check_params(P, params); }

DevStep make_step_consts(const d4orm_params* params, int iter, int step_i)
{
    std::vector<double> abar;
    schedule(params, abar);
    return step_consts(params, abar, iter, step_i);
}

const DevProblem& dev_problem(const d4orm_problem* P) { return P->dp; }

int rollout_kernel_choice(const d4orm_problem* P) { return P->rollout_kernel; }

d4orm_status set_error(d4orm_status s, const char* msg) { return fail(s, "%s", msg); }

d4orm_status set_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }

}  // namespace d4orm

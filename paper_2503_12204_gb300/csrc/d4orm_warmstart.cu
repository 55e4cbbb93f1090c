// d4orm_warmstart.cu -- host side of the learned warm start (include/d4orm.h,
// d4orm_warmstart_*): parameter layout and initialisation, the forward /
// backward / AdamW sequence of the set-MLP, team features, and seeding a
// problem's deformation at an intermediate denoising step.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "d4orm_internal.h"

using namespace d4orm;

namespace {

constexpr int kFeat = 16;  // input features per robot (11 used, zero padded)

struct Layer {
    int out, in;
    size_t w, b;  // offsets into the flat parameter vector
};

}  // namespace

struct d4orm_warmstart {
    d4orm_warmstart_desc desc{};
    int nmax = 0, W = 0, D = 0, Bmax = 0;
    Layer L[6];
    size_t count = 0;
    int step = 0;
    float* d_p = nullptr;
    __nv_bfloat16* d_p16 = nullptr;
    float *d_m = nullptr, *d_v = nullptr, *d_g = nullptr;
    // activations for up to Bmax teams (M = Bmax * nmax rows)
    __nv_bfloat16 *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *C4 = nullptr, *H4 = nullptr, *H5 = nullptr;
    float *Y = nullptr, *dY = nullptr, *dH5 = nullptr, *dH4 = nullptr, *dC4 = nullptr, *dH3 = nullptr, *dH2 = nullptr,
          *dH1 = nullptr;
    float* partial = nullptr;
    size_t partial_cap = 0;
    float *Xb = nullptr, *Mb = nullptr, *Yb = nullptr;  // gathered batch
    float* d_loss = nullptr;
    float* h_loss = nullptr;  // pinned
    float *x1 = nullptr, *m1 = nullptr;  // single-team features for predict
};

namespace {

#define W_CUDA(call)                                                     \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return set_cuda_error(e_, #call);         \
    } while (0)

constexpr int kSplits = 8;

// splitmix64 (Steele, Lea, Flood 2014): seeded uniform initialisation
uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void ws_free(d4orm_warmstart* S)
{
    void* ptrs[] = {S->d_p, S->d_p16, S->d_m, S->d_v, S->d_g, S->H1, S->H2, S->H3, S->C4, S->H4, S->H5, S->Y, S->dY,
                    S->dH5, S->dH4, S->dC4, S->dH3, S->dH2, S->dH1, S->partial, S->Xb, S->Mb, S->Yb, S->d_loss,
                    S->x1, S->m1};
    for (void* p : ptrs) cudaFree(p);
    cudaFreeHost(S->h_loss);
}

// Y_rows = relu?(A W^T + b) with A: [M][in] (bf16 or f32), W = layer weights
cudaError_t fwd_layer(d4orm_warmstart* S, const void* A, bool a_bf16, int M, const Layer& l, bool relu,
                      __nv_bfloat16* out_bf16, float* out_f32, cudaStream_t st)
{
    GemmArgs g{};
    g.M = M;
    g.N = l.out;
    g.K = l.in;
    g.a_rs = l.in;
    g.a_cs = 1;
    g.b_rs = l.in;
    g.b_cs = 1;
    g.bias = S->d_p + l.b;
    g.relu = relu ? 1 : 0;
    g.out_bf16 = out_bf16;
    g.out_f32 = out_f32;
    g.ldc = l.out;
    return mlp_gemm(A, a_bf16, S->d_p16 + l.w, true, g, 1, st);
}

// dW = dY^T A (split reduction over M), db = column sums of dY
cudaError_t wgrad(d4orm_warmstart* S, const float* dYl, const void* A, bool a_bf16, int M, const Layer& l,
                  cudaStream_t st)
{
    GemmArgs g{};
    g.M = l.out;   // rows of dW
    g.N = l.in;    // cols of dW
    g.K = M;       // reduction over team rows
    g.a_rs = 1;    // dY^T(o, m) = dY[m][o]
    g.a_cs = l.out;
    g.b_rs = 1;    // A^T as B(n = i, k = m) = A[m][i]
    g.b_cs = l.in;
    g.partial = S->partial;
    cudaError_t e = mlp_gemm(dYl, false, A, a_bf16, g, kSplits, st);
    if (e == cudaSuccess) e = mlp_sum_partials(S->partial, kSplits, (long long)l.out * l.in, S->d_g + l.w, st);
    if (e == cudaSuccess) e = mlp_colsum(dYl, M, l.out, S->d_g + l.b, st);
    return e;
}

// dA = (dY W) (* (ref > 0)) : [M][in]
cudaError_t dgrad(d4orm_warmstart* S, const float* dYl, int M, const Layer& l, const __nv_bfloat16* ref, float* dA,
                  cudaStream_t st)
{
    GemmArgs g{};
    g.M = M;
    g.N = l.in;
    g.K = l.out;
    g.a_rs = l.out;
    g.a_cs = 1;
    g.b_rs = 1;       // B(n = i, k = o) = W[o][i]
    g.b_cs = l.in;
    g.ref = ref;
    g.out_f32 = dA;
    g.ldc = l.in;
    return mlp_gemm(dYl, false, S->d_p16 + l.w, true, g, 1, st);
}

cudaError_t forward(d4orm_warmstart* S, const float* X, const float* mask, int B, cudaStream_t st)
{
    const int M = B * S->nmax, W = S->W;
    cudaError_t e = fwd_layer(S, X, false, M, S->L[0], true, S->H1, nullptr, st);
    if (e == cudaSuccess) e = fwd_layer(S, S->H1, true, M, S->L[1], true, S->H2, nullptr, st);
    if (e == cudaSuccess) e = fwd_layer(S, S->H2, true, M, S->L[2], true, S->H3, nullptr, st);
    if (e == cudaSuccess) e = mlp_pool_concat(S->H3, mask, B, S->nmax, W, S->C4, st);
    if (e == cudaSuccess) e = fwd_layer(S, S->C4, true, M, S->L[3], true, S->H4, nullptr, st);
    if (e == cudaSuccess) e = fwd_layer(S, S->H4, true, M, S->L[4], true, S->H5, nullptr, st);
    if (e == cudaSuccess) e = fwd_layer(S, S->H5, true, M, S->L[5], false, nullptr, S->Y, st);
    return e;
}

cudaError_t backward(d4orm_warmstart* S, const float* X, const float* mask, int B, cudaStream_t st)
{
    const int M = B * S->nmax, W = S->W;
    cudaError_t e = wgrad(S, S->dY, S->H5, true, M, S->L[5], st);
    if (e == cudaSuccess) e = dgrad(S, S->dY, M, S->L[5], S->H5, S->dH5, st);
    if (e == cudaSuccess) e = wgrad(S, S->dH5, S->H4, true, M, S->L[4], st);
    if (e == cudaSuccess) e = dgrad(S, S->dH5, M, S->L[4], S->H4, S->dH4, st);
    if (e == cudaSuccess) e = wgrad(S, S->dH4, S->C4, true, M, S->L[3], st);
    if (e == cudaSuccess) e = dgrad(S, S->dH4, M, S->L[3], nullptr, S->dC4, st);
    if (e == cudaSuccess) e = mlp_pool_concat_bwd(S->dC4, mask, S->H3, B, S->nmax, W, S->dH3, st);
    if (e == cudaSuccess) e = wgrad(S, S->dH3, S->H2, true, M, S->L[2], st);
    if (e == cudaSuccess) e = dgrad(S, S->dH3, M, S->L[2], S->H2, S->dH2, st);
    if (e == cudaSuccess) e = wgrad(S, S->dH2, S->H1, true, M, S->L[1], st);
    if (e == cudaSuccess) e = dgrad(S, S->dH2, M, S->L[1], S->H1, S->dH1, st);
    if (e == cudaSuccess) e = wgrad(S, S->dH1, X, false, M, S->L[0], st);
    return e;
}

d4orm_status check_batch(const d4orm_warmstart* S, int B)
{
    if (!S) return set_error(D4ORM_ERR_INVALID_ARG, "null warm start");
    if (B < 1 || B > S->Bmax) return set_error(D4ORM_ERR_INVALID_ARG, "batch size out of 1..max_batch");
    return D4ORM_OK;
}

d4orm_status loss_grad(d4orm_warmstart* S, const float* X, const float* mask, const float* Yt, int B,
                       cudaStream_t st)
{
    const int M = B * S->nmax;
    cudaError_t e = forward(S, X, mask, B, st);
    if (e == cudaSuccess) e = mlp_mse(S->Y, Yt, mask, M, S->D, S->dY, S->d_loss, st);
    if (e == cudaSuccess) e = backward(S, X, mask, B, st);
    if (e != cudaSuccess) return set_cuda_error(e, "warm-start forward/backward");
    return D4ORM_OK;
}

d4orm_status adam_update(d4orm_warmstart* S, cudaStream_t st)
{
    S->step += 1;
    const double b1 = S->desc.beta1, b2 = S->desc.beta2;
    const float bc1 = (float)(1.0 - std::pow(b1, S->step)), bc2 = (float)(1.0 - std::pow(b2, S->step));
    W_CUDA(mlp_adamw(S->d_p, S->d_p16, S->d_g, S->d_m, S->d_v, (long long)S->count, S->desc.lr, S->desc.beta1,
                     S->desc.beta2, S->desc.eps, S->desc.weight_decay, bc1, bc2, st));
    return D4ORM_OK;
}

d4orm_status read_loss(d4orm_warmstart* S, float* loss_host, cudaStream_t st)
{
    if (!loss_host) return D4ORM_OK;
    W_CUDA(cudaMemcpyAsync(S->h_loss, S->d_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    W_CUDA(cudaStreamSynchronize(st));
    if (mlp_gemm_timed_out()) return set_error(D4ORM_ERR_TIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs");
    *loss_host = *S->h_loss;
    return D4ORM_OK;
}

}  // namespace

extern "C" {

d4orm_status d4orm_warmstart_create(const d4orm_warmstart_desc* desc, d4orm_warmstart** out)
{
    if (!out) return set_error(D4ORM_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!desc) return set_error(D4ORM_ERR_INVALID_ARG, "desc is null");
    if (desc->n_max < 1 || desc->n_max > D4ORM_MAX_ROBOTS || desc->T < 1 || desc->d_u < 1 || desc->d_u > 3 ||
        desc->width < 16 || desc->width > 1024 || desc->width % 16 != 0 || desc->max_batch < 1 ||
        !(desc->pos_scale > 0.f))
        return set_error(D4ORM_ERR_INVALID_ARG, "warm-start shape out of range");
    d4orm_warmstart* S = new (std::nothrow) d4orm_warmstart();
    if (!S) return set_error(D4ORM_ERR_OOM, "host allocation failed");
    S->desc = *desc;
    S->nmax = desc->n_max;
    S->W = desc->width;
    S->D = desc->T * desc->d_u;
    S->Bmax = desc->max_batch;
    const int W = S->W;
    const int shapes[6][2] = {{W, kFeat}, {W, W}, {W, W}, {W, 2 * W}, {W, W}, {S->D, W}};
    size_t off = 0;
    for (int l = 0; l < 6; ++l) {
        S->L[l].out = shapes[l][0];
        S->L[l].in = shapes[l][1];
        S->L[l].w = off;
        off += (size_t)shapes[l][0] * shapes[l][1];
        S->L[l].b = off;
        off += shapes[l][0];
    }
    S->count = off;
    // uniform(-1/sqrt(in), 1/sqrt(in)) weights, zero biases
    std::vector<float> p(S->count, 0.0f);
    uint64_t st = desc->seed;
    for (int l = 0; l < 6; ++l) {
        const float bound = 1.0f / std::sqrt((float)S->L[l].in);
        for (size_t i = 0; i < (size_t)S->L[l].out * S->L[l].in; ++i) {
            const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
            p[S->L[l].w + i] = (float)((2.0 * u - 1.0) * bound);
        }
    }
    const size_t M = (size_t)S->Bmax * S->nmax;
    size_t max_wgrad = 0;
    for (int l = 0; l < 6; ++l) max_wgrad = std::max(max_wgrad, (size_t)S->L[l].out * S->L[l].in);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    alloc((void**)&S->d_p, S->count * 4);
    alloc((void**)&S->d_p16, S->count * 2);
    alloc((void**)&S->d_m, S->count * 4);
    alloc((void**)&S->d_v, S->count * 4);
    alloc((void**)&S->d_g, S->count * 4);
    alloc((void**)&S->H1, M * W * 2);
    alloc((void**)&S->H2, M * W * 2);
    alloc((void**)&S->H3, M * W * 2);
    alloc((void**)&S->C4, M * 2 * W * 2);
    alloc((void**)&S->H4, M * W * 2);
    alloc((void**)&S->H5, M * W * 2);
    alloc((void**)&S->Y, M * S->D * 4);
    alloc((void**)&S->dY, M * S->D * 4);
    alloc((void**)&S->dH5, M * W * 4);
    alloc((void**)&S->dH4, M * W * 4);
    alloc((void**)&S->dC4, M * 2 * W * 4);
    alloc((void**)&S->dH3, M * W * 4);
    alloc((void**)&S->dH2, M * W * 4);
    alloc((void**)&S->dH1, M * W * 4);
    alloc((void**)&S->partial, (size_t)kSplits * max_wgrad * 4);
    alloc((void**)&S->Xb, M * kFeat * 4);
    alloc((void**)&S->Mb, M * 4);
    alloc((void**)&S->Yb, M * S->D * 4);
    alloc((void**)&S->d_loss, 4);
    alloc((void**)&S->x1, (size_t)S->nmax * kFeat * 4);
    alloc((void**)&S->m1, (size_t)S->nmax * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&S->h_loss, 4);
    if (e == cudaSuccess) e = cudaMemcpy(S->d_p, p.data(), S->count * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(S->d_m, 0, S->count * 4);
    if (e == cudaSuccess) e = cudaMemset(S->d_v, 0, S->count * 4);
    if (e == cudaSuccess) e = mlp_to_bf16(S->d_p, S->d_p16, (long long)S->count, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        ws_free(S);
        delete S;
        return set_error(e == cudaErrorMemoryAllocation ? D4ORM_ERR_OOM : D4ORM_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = S;
    return D4ORM_OK;
}

void d4orm_warmstart_destroy(d4orm_warmstart* S)
{
    if (!S) return;
    cudaDeviceSynchronize();
    ws_free(S);
    delete S;
}

int d4orm_warmstart_param_count(const d4orm_warmstart* S) { return S ? (int)S->count : -1; }

d4orm_status d4orm_warmstart_get_params(const d4orm_warmstart* S, float* host, int count)
{
    if (!S || !host || count != (int)S->count) return set_error(D4ORM_ERR_INVALID_ARG, "bad arguments");
    W_CUDA(cudaMemcpy(host, S->d_p, S->count * 4, cudaMemcpyDeviceToHost));
    return D4ORM_OK;
}

d4orm_status d4orm_warmstart_set_params(d4orm_warmstart* S, const float* host, int count)
{
    if (!S || !host || count != (int)S->count) return set_error(D4ORM_ERR_INVALID_ARG, "bad arguments");
    W_CUDA(cudaMemcpy(S->d_p, host, S->count * 4, cudaMemcpyHostToDevice));
    W_CUDA(mlp_to_bf16(S->d_p, S->d_p16, (long long)S->count, nullptr));
    W_CUDA(cudaMemset(S->d_m, 0, S->count * 4));
    W_CUDA(cudaMemset(S->d_v, 0, S->count * 4));
    W_CUDA(cudaDeviceSynchronize());
    S->step = 0;
    return D4ORM_OK;
}

d4orm_status d4orm_warmstart_forward(d4orm_warmstart* S, const float* x_dev, const float* mask_dev, int B,
                                     float* y_dev, void* stream)
{
    d4orm_status s = check_batch(S, B);
    if (s != D4ORM_OK) return s;
    if (!x_dev || !mask_dev || !y_dev) return set_error(D4ORM_ERR_INVALID_ARG, "null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = forward(S, x_dev, mask_dev, B, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y_dev, S->Y, (size_t)B * S->nmax * S->D * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return set_cuda_error(e, "warm-start forward");
    return D4ORM_OK;
}

d4orm_status d4orm_warmstart_loss_grad(d4orm_warmstart* S, const float* x_dev, const float* mask_dev,
                                       const float* y_dev, int B, float* loss_host, float* grad_dev, void* stream)
{
    d4orm_status s = check_batch(S, B);
    if (s != D4ORM_OK) return s;
    if (!x_dev || !mask_dev || !y_dev) return set_error(D4ORM_ERR_INVALID_ARG, "null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    s = loss_grad(S, x_dev, mask_dev, y_dev, B, st);
    if (s != D4ORM_OK) return s;
    if (grad_dev) W_CUDA(cudaMemcpyAsync(grad_dev, S->d_g, S->count * 4, cudaMemcpyDeviceToDevice, st));
    return read_loss(S, loss_host, st);
}

d4orm_status d4orm_warmstart_train_step(d4orm_warmstart* S, const float* x_all, const float* mask_all,
                                        const float* y_all, const int* idx_dev, int B, float* loss_host, void* stream)
{
    d4orm_status s = check_batch(S, B);
    if (s != D4ORM_OK) return s;
    if (!x_all || !mask_all || !y_all) return set_error(D4ORM_ERR_INVALID_ARG, "null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const float *X = x_all, *Mk = mask_all, *Yt = y_all;
    if (idx_dev) {
        const long long rows = (long long)B * S->nmax;
        W_CUDA(mlp_gather_rows(x_all, idx_dev, S->nmax, kFeat, rows, S->Xb, st));
        W_CUDA(mlp_gather_rows(mask_all, idx_dev, S->nmax, 1, rows, S->Mb, st));
        W_CUDA(mlp_gather_rows(y_all, idx_dev, S->nmax, S->D, rows, S->Yb, st));
        X = S->Xb;
        Mk = S->Mb;
        Yt = S->Yb;
    }
    s = loss_grad(S, X, Mk, Yt, B, st);
    if (s != D4ORM_OK) return s;
    s = adam_update(S, st);
    if (s != D4ORM_OK) return s;
    return read_loss(S, loss_host, st);
}

d4orm_status d4orm_warmstart_features(const d4orm_problem* problem, int n_max, float pos_scale, float* x_host,
                                      float* mask_host)
{
    if (!problem || !x_host || !mask_host || !(pos_scale > 0.f))
        return set_error(D4ORM_ERR_INVALID_ARG, "bad arguments");
    const DevProblem& P = dev_problem(problem);
    if (P.n > n_max) return set_error(D4ORM_ERR_INVALID_ARG, "problem has more robots than n_max");
    std::memset(x_host, 0, sizeof(float) * n_max * kFeat);
    for (int k = 0; k < n_max; ++k) mask_host[k] = k < P.n ? 1.0f : 0.0f;
    const float inv = 1.0f / pos_scale;
    for (int k = 0; k < P.n; ++k) {
        float* x = x_host + k * kFeat;
        double dist2 = 0.0;
        for (int c = 0; c < P.d_p; ++c) {
            const float s = P.start[k * P.d_x + c] * inv, g = P.goal[k * 3 + c] * inv;
            x[c] = s;
            x[3 + c] = g;
            x[6 + c] = g - s;
            dist2 += (double)(g - s) * (g - s);
        }
        x[9] = (float)std::sqrt(dist2);
        x[10] = 1.0f;
    }
    return D4ORM_OK;
}

d4orm_status d4orm_warmstart_predict(d4orm_warmstart* S, const d4orm_problem* problem, const d4orm_params* params,
                                     int start_step, float* du_seed_dev, void* stream)
{
    if (!S || !problem || !params || !du_seed_dev) return set_error(D4ORM_ERR_INVALID_ARG, "null argument");
    d4orm_status s = validate_params(problem, params);
    if (s != D4ORM_OK) return s;
    if (start_step < 1 || start_step > params->n_steps) return set_error(D4ORM_ERR_INVALID_ARG, "start_step out of 1..K");
    const DevProblem& P = dev_problem(problem);
    if (P.n > S->nmax || P.T != S->desc.T || P.d_u != S->desc.d_u)
        return set_error(D4ORM_ERR_INVALID_ARG, "problem shape does not match the network");
    std::vector<float> x((size_t)S->nmax * kFeat), m(S->nmax);
    s = d4orm_warmstart_features(problem, S->nmax, S->desc.pos_scale, x.data(), m.data());
    if (s != D4ORM_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    W_CUDA(cudaMemcpyAsync(S->x1, x.data(), x.size() * 4, cudaMemcpyHostToDevice, st));
    W_CUDA(cudaMemcpyAsync(S->m1, m.data(), m.size() * 4, cudaMemcpyHostToDevice, st));
    W_CUDA(forward(S, S->x1, S->m1, 1, st));
    // dU_{i0} = sqrt(abar_{i0}) U_hat, so that the sampling mean dU/sqrt(abar) is U_hat
    const DevStep Si = make_step_consts(params, 0, start_step);
    W_CUDA(mlp_seed_from_output(S->Y, P.n, P.T, P.d_u, S->D, 1.0f / Si.c, du_seed_dev, st));
    W_CUDA(cudaStreamSynchronize(st));  // x, m are host stack buffers
    if (mlp_gemm_timed_out()) return set_error(D4ORM_ERR_TIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs");
    return D4ORM_OK;
}

}  // extern "C"

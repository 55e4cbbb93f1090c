// k_setmlp.cu -- kernels of the learned warm start: a set-MLP trained on the
// method's own solutions.
//
// Network (per team, robots padded to n_max with a mask):
//   per-robot encoder  H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2),
//                      H3 = relu(H2 W3^T + b3)                 (width 256)
//   team context       Pbar = masked mean over robots of H3
//   head               C = [H3, Pbar], H4 = relu(C W4^T + b4),
//                      H5 = relu(H4 W5^T + b5), Y = H5 W6^T + b6 (T*d_u per robot)
//   loss               masked mean squared error against the method's plan
//
// GEMMs run on the fifth-generation tensor cores (tcgen05.mma, BF16
// operands, FP32 accumulation in tensor memory).  Operands are staged into
// shared memory as BF16 from either BF16 or FP32 global tensors with
// arbitrary (row, column) strides, so one kernel serves Y = A W^T
// (forward), dA = dY W (data gradient) and dW = dY^T A (weight gradient,
// split over the reduction with per-split partials summed in a fixed
// order).  Activations are stored in BF16, their
// gradients in FP32, the weights as FP32 masters with BF16 copies.
#include <cuda_bf16.h>

#include <cmath>

#include "d4orm_internal.h"
#include "d4orm_kernels.cuh"

namespace d4orm {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// C[m][n] = sum_k A(m, k) * B(n, k) over k in [k_begin, k_end), where
// A(m, k) = A[m * a_rs + k * a_cs] and B(n, k) = B[n * b_rs + k * b_cs].
// Epilogue (split == 1): + bias[n], relu, times (ref(m, n) > 0), then store
// to out_f32 and/or out_bf16 (row stride ldc).  Split-K (gridDim.z > 1):
// raw partial sums to partial[z][M][N].

// ---------------------------------------------------------------------------
// The GEMM runs on the fifth-generation tensor cores: tcgen05.mma (kind::f16,
// BF16 x BF16 -> FP32, one CTA, M = 128) with the accumulator in tensor
// memory.  The CTA (128 threads) stages each 128 x 64 (A) and 64 x 64 (B)
// K-slice into shared memory as BF16 in the canonical no-swizzle K-major
// layout -- 8-row x 16-byte core matrices, 128 B apart along K and 1 KB
// apart along rows -- converting from FP32 where needed and honouring the
// arbitrary strides (which is why the threads stage the operands rather
// than TMA).  One thread issues the four K = 16 MMAs of the slice and
// commits them to an mbarrier; the CTA waits on it (bounded) before the
// slice's shared memory is refilled.  The epilogue reads the accumulator
// back with tcgen05.ld (warp w owns rows 32w..32w+31) and applies the bias,
// ReLU, ReLU-gradient mask or split-K partial store.
// ---------------------------------------------------------------------------
constexpr int kTBM = 128, kTBN = 64, kTBK = 64;
// Dynamic shared memory requested per CTA: the staged operands (24 KB)
// plus padding that keeps at most 4 CTAs on an SM, so 4 x 64 tensor-memory
// columns never exceed the SM's 512 and tcgen05.alloc never waits.
constexpr int kTcSmemLaunch = 52 * 1024;
// set when an MMA completion wait gave up (read by mlp_gemm_timed_out)
__device__ int g_tc_timeout;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start address, leading (K) and
// stride (row-group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of a staged [rows][64] K-major slice
__device__ __forceinline__ uint32_t tc_off(int r, int k)
{
    return (uint32_t)((r >> 3) * (kTBK / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Stage rows [0, ROWS) x k [k0, k0 + 64) of X(r, k) = X[(r0 + r) * rs + k * cs]
// (zero outside [0, rmax) x [k0, ke)), 8 consecutive k per 16-byte store.
template <int ROWS, typename T>
__device__ __forceinline__ void tc_stage(uint8_t* s, const T* __restrict__ X, int r0, int rmax, long long rs,
                                         long long cs, int k0, int ke)
{
    for (int i = threadIdx.x; i < ROWS * (kTBK / 8); i += blockDim.x) {
        const int r = i % ROWS, j = i / ROWS;
        const int gr = r0 + r;
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int k = k0 + 8 * j + 2 * h;
            const float lo = (gr < rmax && k < ke) ? to_f(X[gr * rs + k * cs]) : 0.0f;
            const float hi = (gr < rmax && k + 1 < ke) ? to_f(X[gr * rs + (k + 1) * cs]) : 0.0f;
            w[h] = pack_bf16(__float2bfloat16_rn(lo), __float2bfloat16_rn(hi));
        }
        *reinterpret_cast<uint4*>(s + tc_off(r, 8 * j)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity)
{
    // bounded: 2^22 polls, far beyond the microseconds an MMA slice takes
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(128)
k_gemm_tc(const TA* __restrict__ A, const TB* __restrict__ B, const GemmArgs g)
{
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    uint8_t* sA = tc_smem;
    uint8_t* sB = tc_smem + kTBM * kTBK * 2;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTBM, n0 = blockIdx.x * kTBN;
    const int splits = gridDim.z;
    const int kchunk = ((g.K + splits - 1) / splits + kTBK - 1) / kTBK * kTBK;
    const int kb = blockIdx.z * kchunk, ke = min(g.K, kb + kchunk);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base, mb = smem_addr(&mbar);
    constexpr uint32_t idesc = tc_idesc(kTBM, kTBN);
    uint32_t parity = 0;
    bool ok = true, any = false;
    for (int k0 = kb; k0 < ke && ok; k0 += kTBK) {
        tc_stage<kTBM>(sA, A, m0, g.M, g.a_rs, g.a_cs, k0, ke);
        tc_stage<kTBN>(sB, B, n0, g.N, g.b_rs, g.b_cs, k0, ke);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < kTBK / 16; ++s) {
                const uint64_t da = tc_smem_desc(smem_addr(sA) + s * 256, 128, (kTBK / 8) * 128);
                const uint64_t db = tc_smem_desc(smem_addr(sB) + s * 256, 128, (kTBK / 8) * 128);
                const uint32_t accumulate = (any || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                         : "memory");
        }
        any = true;
        const bool mine = tc_wait(mb, parity);
        parity ^= 1u;
        ok = __syncthreads_and(mine) != 0;  // one verdict for the whole CTA
        if (!ok && tid == 0) atomicExch(&g_tc_timeout, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int m = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < kTBN; c += 8) {
            float v[8];
            if (any) {
                uint32_t r[8];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = 0.0f;  // an empty K range
            }
            if (m >= g.M) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int n = n0 + c + i;
                if (n >= g.N) continue;
                float x = v[i];
                if (splits > 1) {
                    g.partial[((long long)blockIdx.z * g.M + m) * g.N + n] = x;
                    continue;
                }
                if (g.bias) x += g.bias[n];
                if (g.relu) x = fmaxf(x, 0.0f);
                if (g.ref && !(__bfloat162float(static_cast<const __nv_bfloat16*>(g.ref)[m * g.ldc + n]) > 0.0f))
                    x = 0.0f;
                if (g.out_f32) g.out_f32[m * g.ldc + n] = x;
                if (g.out_bf16) static_cast<__nv_bfloat16*>(g.out_bf16)[m * g.ldc + n] = __float2bfloat16_rn(x);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTBN) : "memory");
}

// out[m][n] = sum_z partial[z][m][n]   (fixed order)
__global__ void k_sum_partials(const float* __restrict__ partial, int splits, long long MN, float* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN) return;
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += partial[z * MN + i];
    out[i] = s;
}

// db[n] = sum_m dY[m][n]  (fixed order per column)
__global__ void k_colsum(const float* __restrict__ dY, int M, int N, float* __restrict__ db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int m = 0; m < M; ++m) s += dY[(long long)m * N + n];
    db[n] = s;
}

// C[b, k] = [H3[b, k], Pbar[b]],  Pbar[b] = sum_k mask H3[b, k] / max(1, sum_k mask)
__global__ void k_pool_concat(const __nv_bfloat16* __restrict__ H3, const float* __restrict__ mask, int B, int nmax,
                              int W, __nv_bfloat16* __restrict__ C)
{
    const int b = blockIdx.x;
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        float s = 0.0f, cnt = 0.0f;
        for (int k = 0; k < nmax; ++k) {
            const float mk = mask[b * nmax + k];
            s += mk * __bfloat162float(H3[((long long)b * nmax + k) * W + c]);
            cnt += mk;
        }
        const __nv_bfloat16 p = __float2bfloat16_rn(s / fmaxf(cnt, 1.0f));
        for (int k = 0; k < nmax; ++k) {
            C[((long long)b * nmax + k) * 2 * W + c] = H3[((long long)b * nmax + k) * W + c];
            C[((long long)b * nmax + k) * 2 * W + W + c] = p;
        }
    }
}

// dH3[b, k] = (dC[b, k, :W] + mask_k / cnt * sum_k' dC[b, k', W:]) * (H3 > 0)
__global__ void k_pool_concat_bwd(const float* __restrict__ dC, const float* __restrict__ mask,
                                  const __nv_bfloat16* __restrict__ H3, int B, int nmax, int W, float* __restrict__ dH3)
{
    const int b = blockIdx.x;
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        float sp = 0.0f, cnt = 0.0f;
        for (int k = 0; k < nmax; ++k) {
            sp += dC[((long long)b * nmax + k) * 2 * W + W + c];
            cnt += mask[b * nmax + k];
        }
        const float share = sp / fmaxf(cnt, 1.0f);
        for (int k = 0; k < nmax; ++k) {
            const long long r = (long long)b * nmax + k;
            float v = dC[r * 2 * W + c] + mask[b * nmax + k] * share;
            if (!(__bfloat162float(H3[r * W + c]) > 0.0f)) v = 0.0f;
            dH3[r * W + c] = v;
        }
    }
}

// masked MSE: loss = sum mask (y - t)^2 / (sum mask * D);  dY = 2 mask (y - t) / (sum mask * D)
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ Tgt, const float* __restrict__ mask,
                      int rows, int D, float* __restrict__ dY, float* __restrict__ loss)
{
    __shared__ float sh[33];
    float cnt = 0.0f;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) cnt += mask[r];
    cnt = block_reduce<false>(cnt, sh);
    const float inv = 1.0f / (fmaxf(cnt, 1.0f) * D);
    float l = 0.0f;
    for (long long i = threadIdx.x; i < (long long)rows * D; i += blockDim.x) {
        const float mk = mask[i / D];
        const float e = (Y[i] - Tgt[i]) * mk;
        l = fmaf(e, e, l);
        dY[i] = 2.0f * e * inv;
    }
    l = block_reduce<false>(l, sh);
    if (threadIdx.x == 0 && loss) *loss = l * inv;
}

// AdamW on flat FP32 parameters; refreshes the BF16 copy.
__global__ void k_adamw(float* __restrict__ p, __nv_bfloat16* __restrict__ p16, const float* __restrict__ grad,
                        float* __restrict__ m, float* __restrict__ v, long long count, float lr, float b1, float b2,
                        float eps, float wd, float bc1, float bc2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = grad[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    const float pi = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
    p[i] = pi;
    p16[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, long long count)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = __float2bfloat16_rn(src[i]);
}

// dst[r] = src[idx[r / rows_per] * rows_per + r % rows_per], row width w (batch gather)
__global__ void k_gather_rows(const float* __restrict__ src, const int* __restrict__ idx, int rows_per, int w,
                              long long total_rows, float* __restrict__ dst)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total_rows * w) return;
    const long long r = i / w;
    const int c = (int)(i - r * w);
    const long long src_row = (long long)idx[r / rows_per] * rows_per + r % rows_per;
    dst[i] = src[src_row * w + c];
}

// du_seed[t][k][d] = scale * Y[k][t * d_u + d]  for k < n
__global__ void k_seed_from_output(const float* __restrict__ Y, int n, int T, int d_u, int D, float scale,
                                   float* __restrict__ du_seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T * n * d_u) return;
    const int t = i / (n * d_u), rem = i - t * n * d_u, k = rem / d_u, d = rem - k * d_u;
    du_seed[i] = scale * Y[(long long)k * D + t * d_u + d];
}

// ------------------------------------------------------------------ launchers

bool mlp_gemm_timed_out()
{
    int flag = 0;
    if (cudaMemcpyFromSymbol(&flag, g_tc_timeout, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (flag) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int));
    }
    return flag != 0;
}

template <typename TA, typename TB>
static cudaError_t gemm_launch(const TA* A, const TB* B, GemmArgs g, int splits, cudaStream_t st)
{
    static cudaError_t attr =
        cudaFuncSetAttribute(k_gemm_tc<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemLaunch);
    if (attr != cudaSuccess) return attr;
    dim3 grid((g.N + kTBN - 1) / kTBN, (g.M + kTBM - 1) / kTBM, splits);
    k_gemm_tc<TA, TB><<<grid, 128, kTcSmemLaunch, st>>>(A, B, g);
    return cudaGetLastError();
}

cudaError_t mlp_gemm(const void* A, bool a_bf16, const void* B, bool b_bf16, const GemmArgs& g, int splits,
                     cudaStream_t st)
{
    using bf = __nv_bfloat16;
    if (a_bf16 && b_bf16) return gemm_launch((const bf*)A, (const bf*)B, g, splits, st);
    if (a_bf16) return gemm_launch((const bf*)A, (const float*)B, g, splits, st);
    if (b_bf16) return gemm_launch((const float*)A, (const bf*)B, g, splits, st);
    return gemm_launch((const float*)A, (const float*)B, g, splits, st);
}

cudaError_t mlp_sum_partials(const float* partial, int splits, long long MN, float* out, cudaStream_t st)
{
    k_sum_partials<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(partial, splits, MN, out);
    return cudaGetLastError();
}

cudaError_t mlp_colsum(const float* dY, int M, int N, float* db, cudaStream_t st)
{
    k_colsum<<<(N + 127) / 128, 128, 0, st>>>(dY, M, N, db);
    return cudaGetLastError();
}

cudaError_t mlp_pool_concat(const void* H3, const float* mask, int B, int nmax, int W, void* C, cudaStream_t st)
{
    k_pool_concat<<<B, 256, 0, st>>>((const __nv_bfloat16*)H3, mask, B, nmax, W, (__nv_bfloat16*)C);
    return cudaGetLastError();
}

cudaError_t mlp_pool_concat_bwd(const float* dC, const float* mask, const void* H3, int B, int nmax, int W,
                                float* dH3, cudaStream_t st)
{
    k_pool_concat_bwd<<<B, 256, 0, st>>>(dC, mask, (const __nv_bfloat16*)H3, B, nmax, W, dH3);
    return cudaGetLastError();
}

cudaError_t mlp_mse(const float* Y, const float* Tgt, const float* mask, int rows, int D, float* dY, float* loss,
                    cudaStream_t st)
{
    k_mse<<<1, 1024, 0, st>>>(Y, Tgt, mask, rows, D, dY, loss);
    return cudaGetLastError();
}

cudaError_t mlp_adamw(float* p, void* p16, const float* grad, float* m, float* v, long long count, float lr, float b1,
                      float b2, float eps, float wd, float bc1, float bc2, cudaStream_t st)
{
    k_adamw<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(p, (__nv_bfloat16*)p16, grad, m, v, count, lr, b1, b2,
                                                             eps, wd, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t mlp_to_bf16(const float* src, void* dst, long long count, cudaStream_t st)
{
    k_to_bf16<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(src, (__nv_bfloat16*)dst, count);
    return cudaGetLastError();
}

cudaError_t mlp_gather_rows(const float* src, const int* idx, int rows_per, int w, long long total_rows, float* dst,
                            cudaStream_t st)
{
    const long long n = total_rows * w;
    k_gather_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, idx, rows_per, w, total_rows, dst);
    return cudaGetLastError();
}

cudaError_t mlp_seed_from_output(const float* Y, int n, int T, int d_u, int D, float scale, float* du_seed,
                                 cudaStream_t st)
{
    const int total = T * n * d_u;
    k_seed_from_output<<<(total + 255) / 256, 256, 0, st>>>(Y, n, T, d_u, D, scale, du_seed);
    return cudaGetLastError();
}

}  // namespace d4orm

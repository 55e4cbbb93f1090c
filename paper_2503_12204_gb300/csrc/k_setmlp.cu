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
// GEMMs run on the tensor cores with mma.sync m16n8k16 (BF16 operands, FP32
// accumulation).  Operands are staged into shared memory as BF16 from
// either BF16 or FP32 global tensors with arbitrary (row, column) strides,
// so one kernel serves Y = A W^T (forward), dA = dY W (data gradient) and
// dW = dY^T A (weight gradient, split over the reduction with per-split
// partials summed in a fixed order).  Activations are stored in BF16, their
// gradients in FP32, the weights as FP32 masters with BF16 copies.
#include <cuda_bf16.h>

#include <cmath>

#include "d4orm_internal.h"
#include "d4orm_kernels.cuh"

namespace d4orm {

constexpr int kGBM = 64, kGBN = 64, kGBK = 32;  // CTA tile
constexpr int kGPad = 8;                        // smem row padding (bf16)

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A(16x16, row) * B(16x8, col) + D, BF16 x BF16 -> FP32
__device__ __forceinline__ void mma_bf16_16816(float* d, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[m][n] = sum_k A(m, k) * B(n, k) over k in [k_begin, k_end), where
// A(m, k) = A[m * a_rs + k * a_cs] and B(n, k) = B[n * b_rs + k * b_cs].
// Epilogue (split == 1): + bias[n], relu, times (ref(m, n) > 0), then store
// to out_f32 and/or out_bf16 (row stride ldc).  Split-K (gridDim.z > 1):
// raw partial sums to partial[z][M][N].


template <typename TA, typename TB>
__global__ void __launch_bounds__(128)
k_gemm_bf16(const TA* __restrict__ A, const TB* __restrict__ B, const GemmArgs g)
{
    __shared__ __nv_bfloat16 sA[kGBM][kGBK + kGPad];
    __shared__ __nv_bfloat16 sB[kGBN][kGBK + kGPad];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kGBM, n0 = blockIdx.x * kGBN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // 2x2 warps, 32x32 each
    const int splits = gridDim.z;
    const int kchunk = ((g.K + splits - 1) / splits + kGBK - 1) / kGBK * kGBK;
    const int kb = blockIdx.z * kchunk, ke = min(g.K, kb + kchunk);
    float acc[2][4][4] = {};
    const int grp = lane >> 2, tig = lane & 3;
    for (int k0 = kb; k0 < ke; k0 += kGBK) {
        for (int i = tid; i < kGBM * kGBK; i += 128) {
            const int r = i / kGBK, c = i % kGBK;
            const int m = m0 + r, k = k0 + c;
            const float v = (m < g.M && k < ke) ? to_f(A[m * g.a_rs + k * g.a_cs]) : 0.0f;
            sA[r][c] = __float2bfloat16_rn(v);
        }
        for (int i = tid; i < kGBN * kGBK; i += 128) {
            const int r = i / kGBK, c = i % kGBK;
            const int n = n0 + r, k = k0 + c;
            const float v = (n < g.N && k < ke) ? to_f(B[n * g.b_rs + k * g.b_cs]) : 0.0f;
            sB[r][c] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGBK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm + mi * 16 + grp;
                const int c = kk + tig * 2;
                af[mi][0] = pack_bf16(sA[r][c], sA[r][c + 1]);
                af[mi][1] = pack_bf16(sA[r + 8][c], sA[r + 8][c + 1]);
                af[mi][2] = pack_bf16(sA[r][c + 8], sA[r][c + 9]);
                af[mi][3] = pack_bf16(sA[r + 8][c + 8], sA[r + 8][c + 9]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int n = wn + ni * 8 + grp;
                const int c = kk + tig * 2;
                bfr[ni][0] = pack_bf16(sB[n][c], sB[n][c + 1]);
                bfr[ni][1] = pack_bf16(sB[n][c + 8], sB[n][c + 9]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16_16816(acc[mi][ni], af[mi], bfr[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int m = m0 + wm + mi * 16 + grp + (h >= 2 ? 8 : 0);
                const int n = n0 + wn + ni * 8 + tig * 2 + (h & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[mi][ni][h];
                if (splits > 1) {
                    g.partial[((long long)blockIdx.z * g.M + m) * g.N + n] = v;
                    continue;
                }
                if (g.bias) v += g.bias[n];
                if (g.relu) v = fmaxf(v, 0.0f);
                if (g.ref && !(__bfloat162float(static_cast<const __nv_bfloat16*>(g.ref)[m * g.ldc + n]) > 0.0f))
                    v = 0.0f;
                if (g.out_f32) g.out_f32[m * g.ldc + n] = v;
                if (g.out_bf16) static_cast<__nv_bfloat16*>(g.out_bf16)[m * g.ldc + n] = __float2bfloat16_rn(v);
            }
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

template <typename TA, typename TB>
static cudaError_t gemm_launch(const TA* A, const TB* B, GemmArgs g, int splits, cudaStream_t st)
{
    dim3 grid((g.N + kGBN - 1) / kGBN, (g.M + kGBM - 1) / kGBM, splits);
    k_gemm_bf16<TA, TB><<<grid, 128, 0, st>>>(A, B, g);
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

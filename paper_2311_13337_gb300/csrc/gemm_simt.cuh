// Tiled FP32 SIMT matrix product with strided operands, used by the
// surrogate network and the FC principal components:
//   C(m, n) = sum_k A(m, k) B(n, k), A(m, k) = A[m sam + k sak],
//   B(n, k) = B[n sbn + k sbk], blockIdx.z = batch index (member strides),
// with optional epilogues (bias, bias + ReLU, mask). Operands are float or
// bf16 (converted to FP32 on load); accumulation is FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace tvbx {

constexpr int GT = 64;   // GEMM tile (M and N)
constexpr int GK = 16;   // GEMM tile K
enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_MASK = 3 };

// C(m, n) = sum_k A(m, k) B(n, k) with A(m, k) = A[m sam + k sak] and
// B(n, k) = B[n sbn + k sbk]; blockIdx.z selects the ensemble member.
struct GemmArgs {
    const void* A;
    int64_t sam, sak, a_mem;
    const void* B;
    int64_t sbn, sbk, b_mem;
    float* C;
    int64_t ldc, c_mem;
    const float* bias;        // [N] (EPI_BIAS*)
    int64_t bias_mem;
    const float* mask;        // mask[m ldm + n] > 0 keeps the entry (EPI_MASK)
    int64_t ldm, mask_mem;
    int M, N, K;
};

static __device__ __forceinline__ float ldf(const float* p, int64_t i) { return p[i]; }
static __device__ __forceinline__ float ldf(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

template <typename TA, typename TB, int EPI>
__global__ void __launch_bounds__(256) mlp_gemm_kernel(const GemmArgs g)
{
    __shared__ __align__(16) float As[GK][GT + 4];
    __shared__ __align__(16) float Bs[GK][GT + 4];
    const int64_t mem = blockIdx.z;
    const TA* A = static_cast<const TA*>(g.A) + mem * g.a_mem;
    const TB* B = static_cast<const TB*>(g.B) + mem * g.b_mem;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < g.K; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            int mm, kk;
            if (g.sak == 1) { kk = e % GK; mm = e / GK; } else { mm = e % GT; kk = e / GT; }
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < g.M && k < g.K) ? ldf(A, m * g.sam + k * g.sak) : 0.0f;
        }
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            int nn, kk;
            if (g.sbk == 1) { kk = e % GK; nn = e / GK; } else { nn = e % GT; kk = e / GT; }
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < g.N && k < g.K) ? ldf(B, n * g.sbn + k * g.sbk) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* C = g.C + mem * g.c_mem;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= g.N) continue;
            float v = acc[i][j];
            if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) v += g.bias[mem * g.bias_mem + n];
            if (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.0f);
            if (EPI == EPI_MASK && !(g.mask[mem * g.mask_mem + (int64_t)m * g.ldm + n] > 0.0f)) v = 0.0f;
            C[(int64_t)m * g.ldc + n] = v;
        }
    }
}


template <typename TA, typename TB, int EPI>
static inline cudaError_t gemm(const GemmArgs& g, int E, cudaStream_t s)
{
    dim3 grid((g.N + GT - 1) / GT, (g.M + GT - 1) / GT, E);
    note_launch();
    mlp_gemm_kernel<TA, TB, EPI><<<grid, 256, 0, s>>>(g);
    return cudaGetLastError();
}


}  // namespace tvbx

// Tensor-core (tcgen05) matrix product of the surrogate network, with the
// operands of gemm_simt.cuh:
//   C(m, n) = sum_k A(m, k) B(n, k),  A(m, k) = A[m sam + k sak],
//   B(n, k) = B[n sbn + k sbk],  blockIdx.z = ensemble member,
// and the same epilogues (bias, bias + ReLU, mask).
//
// Split precision. An FP32 operand X is split into BF16 parts X = H + L
// (H = bf16(X), L = bf16(X - H)); a BF16 operand (the network's weights) is
// its own H with L = 0. The product takes H_A H_B + L_A H_B (+ H_A L_B when
// both operands are FP32) on the tensor cores in kind::f16 (BF16 x BF16) with
// FP32 accumulation in tensor memory: the error of the split is about 2^-16
// of each operand, far below the FP32 reference product's own rounding over
// these K.
//
// Layout. A CTA of 128 threads owns a 128 x 128 tile of C. Per chunk of 64
// K (one 128-byte row of BF16) thread t reads row t of the A tile and row t
// of the B tile from global memory (any strides: the backward products read
// transposed operands), splits, and writes the parts to shared memory in the
// 128-byte swizzled K-major layout; one thread then issues the MMAs of the
// four 16-wide K slices and commits them to an mbarrier that every thread
// waits on (bounded) before the next chunk overwrites the operands. The
// accumulator (128 lanes x up to 128 FP32 columns) is read back by the four
// warps, each its 32 lanes (rows), and stored with the epilogue. Rows and
// columns beyond M, N and K are staged as zeros.
//
// Split K. A product with few output tiles and a long K (the weight
// gradients: K = the mini-batch rows) would occupy a handful of SMs, so its
// K chunks are divided among `splits` CTAs per tile; each writes its partial
// tile to a scratch array and a second kernel adds the partials in split
// order (deterministic), for the plain-store epilogue only.
#pragma once

#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gemm_simt.cuh"
#include "internal.h"
#include "ptx_async.cuh"

namespace tvbx {

constexpr int TCG_M = 128;       // rows of C per CTA (the MMA's M)
constexpr int TCG_N = 128;       // columns of C per CTA (MMA N <= 128, a multiple of 16)
constexpr int TCG_K = 64;        // K per staged chunk: 64 BF16 = one 128-byte row
constexpr int TCG_THREADS = 128;
constexpr int TCG_TILE_BYTES = TCG_M * TCG_K * 2;   // one operand part, 16 KB
constexpr size_t TCG_SMEM = 4 * (size_t)TCG_TILE_BYTES + 1024;   // A hi/lo, B hi/lo, slack for alignment

// Byte offset of element (r, k) (k < 64) of a 128-byte swizzled K-major tile.
static __device__ __forceinline__ uint32_t tcg_sw_off(int r, int k)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1));
}

static __device__ __forceinline__ uint32_t tcg_pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Row r (of R valid rows) of an operand tile, K chunk k0 (of K), split into
// BF16 parts and written to the swizzled tiles at sh (high) and sl (low).
template <typename T>
static __device__ __forceinline__ void tcg_stage_row(const T* X, int64_t s_row, int64_t s_k, int64_t row0, int r,
                                                     int R, int k0, int K, uint32_t sh, uint32_t sl)
{
    const bool rok = r < R;
#pragma unroll
    for (int c = 0; c < 8; ++c) {   // 16-byte chunks of 8 BF16
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __nv_bfloat16 hv[2], lv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int k = k0 + c * 8 + q * 2 + u;
                const float x = (rok && k < K) ? ldf(X, (row0 + r) * s_row + (int64_t)k * s_k) : 0.0f;
                hv[u] = __float2bfloat16_rn(x);
                lv[u] = __float2bfloat16_rn(x - __bfloat162float(hv[u]));
            }
            h[q] = tcg_pack2(hv[0], hv[1]);
            l[q] = tcg_pack2(lv[0], lv[1]);
        }
        const uint32_t off = tcg_sw_off(r, c * 8);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(sh + off), "r"(h[0]), "r"(h[1]), "r"(h[2]),
                     "r"(h[3])
                     : "memory");
        if (sl) {
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(sl + off), "r"(l[0]), "r"(l[1]),
                         "r"(l[2]), "r"(l[3])
                         : "memory");
        }
    }
}

template <typename TA, typename TB, int EPI>
__global__ void __launch_bounds__(TCG_THREADS) mlp_gemm_tc_kernel(const GemmArgs g, uint32_t* __restrict__ error,
                                                                  uint32_t wait_limit, int splits, int chunks_per_split,
                                                                  float* __restrict__ part)
{
    extern __shared__ __align__(1024) uint8_t tcg_smem_raw[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    // 1024-byte aligned operand tiles (the swizzle pattern is tied to address bits)
    const uint32_t raw = smem_u32(tcg_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sAh = base, sAl = base + TCG_TILE_BYTES, sBh = base + 2 * TCG_TILE_BYTES,
                   sBl = base + 3 * TCG_TILE_BYTES;
    constexpr bool B_SPLIT = !std::is_same<TB, __nv_bfloat16>::value;
    constexpr bool A_SPLIT = !std::is_same<TA, __nv_bfloat16>::value;

    const int64_t mem = blockIdx.z / splits;
    const int split = (int)(blockIdx.z % splits);
    const TA* A = static_cast<const TA*>(g.A) + mem * g.a_mem;
    const TB* B = static_cast<const TB*>(g.B) + mem * g.b_mem;
    const int m0 = blockIdx.y * TCG_M, n0 = blockIdx.x * TCG_N;
    const int nvalid = min(TCG_N, g.N - n0);
    const uint32_t nmma = (uint32_t)((nvalid + 15) / 16 * 16);   // MMA N: a multiple of 16
    const uint32_t idesc = tc_idesc(1u, (uint32_t)TCG_M, nmma);
    const int t = threadIdx.x;

    if (t == 0) {
        mbar_init(&mbar, 1);
        abort_flag = 0;
        fence_mbarrier_init();
    }
    if (t < 32) tmem_alloc(&tmem_slot, (uint32_t)TCG_N);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    uint32_t parity = 0;
    const int n_chunks = (g.K + TCG_K - 1) / TCG_K;
    const int ch0 = split * chunks_per_split, ch1 = min(n_chunks, ch0 + chunks_per_split);   // ch0 < ch1 (host)
    for (int ch = ch0; ch < ch1; ++ch) {
        const int k0 = ch * TCG_K;
        tcg_stage_row(A, g.sam, g.sak, m0, t, g.M - m0, k0, g.K, sAh, A_SPLIT ? sAl : 0u);
        tcg_stage_row(B, g.sbn, g.sbk, n0, t, g.N - n0, k0, g.K, sBh, B_SPLIT ? sBl : 0u);
        fence_proxy_async_shared();   // the operand writes, visible to the tensor cores
        __syncthreads();
        if (t == 0 && !abort_flag) {
            tc_fence_after();
#pragma unroll
            for (int sl = 0; sl < TCG_K / 16; ++sl) {
                const uint32_t koff = (uint32_t)(sl * 32);   // 16 BF16 = 32 bytes into each row
                const uint64_t ah = sw128_desc(sAh + koff), bh = sw128_desc(sBh + koff);
                tc_mma<0>(tmem, ah, bh, idesc, (ch > ch0 || sl > 0) ? 1u : 0u);
                if (A_SPLIT) tc_mma<0>(tmem, sw128_desc(sAl + koff), bh, idesc, 1u);
                if (B_SPLIT) tc_mma<0>(tmem, ah, sw128_desc(sBl + koff), idesc, 1u);
            }
            tc_commit(&mbar);
        }
        // every thread: wait (bounded) until the MMAs have read the operands
        if (!abort_flag && !mbar_wait_bounded(&mbar, parity, wait_limit)) {
            atomicOr(error, TVBX_DEVERR_TIMEOUT);
            abort_flag = 1;
        }
        parity ^= 1u;
        tc_fence_after();
        __syncthreads();
    }

    // epilogue: warp w drains accumulator lanes 32 w .. 32 w + 31 (rows of C)
    const int warp = t >> 5;
    const int m = m0 + t;   // = m0 + 32 warp + lane
    float* C = g.C + mem * g.c_mem;
    int64_t ldc = g.ldc;
    if (part) {   // split K: this split's partial tile, [split][member][M][N]
        const int64_t E = gridDim.z / splits;
        C = part + ((int64_t)split * E + mem) * (int64_t)g.M * g.N;
        ldc = g.N;
    }
    if (!abort_flag) {
        for (int cb = 0; cb * 16 < nvalid; ++cb) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16), v);
            if (m < g.M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = n0 + cb * 16 + i;
                    if (n >= g.N) continue;
                    float x = v[i];
                    if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) x += g.bias[mem * g.bias_mem + n];
                    if (EPI == EPI_BIAS_RELU) x = fmaxf(x, 0.0f);
                    if (EPI == EPI_MASK && !(g.mask[mem * g.mask_mem + (int64_t)m * g.ldm + n] > 0.0f)) x = 0.0f;
                    C[(int64_t)m * ldc + n] = x;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (t < 32) tmem_dealloc(tmem, (uint32_t)TCG_N);
}

// C(member) = sum over splits of the partial tiles, in split order.
__global__ void mlp_splitk_reduce_kernel(const float* __restrict__ part, int splits, int E, int M, int N,
                                         float* __restrict__ C, int64_t ldc, int64_t c_mem)
{
    const int64_t MN = (int64_t)M * N, total = (int64_t)E * MN;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t mem = i / MN, r = i % MN;
        float acc = 0.0f;
        for (int sp = 0; sp < splits; ++sp) acc += part[((int64_t)sp * E + mem) * MN + r];
        C[mem * c_mem + (r / N) * ldc + r % N] = acc;
    }
}

// Launch on E members; error: device word that receives TVBX_DEVERR_TIMEOUT
// when a bounded wait expires (the outputs are then invalid). part / part_cap
// (floats): scratch for split K (plain-store epilogue only; nullptr: none).
template <typename TA, typename TB, int EPI>
static inline cudaError_t gemm_tc(const GemmArgs& g, int E, uint32_t* error, uint32_t wait_limit, cudaStream_t s,
                                  float* part = nullptr, size_t part_cap = 0)
{
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
    auto kern = mlp_gemm_tc_kernel<TA, TB, EPI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TCG_SMEM);
    if (e != cudaSuccess) return e;
    const int tiles = ((g.N + TCG_N - 1) / TCG_N) * ((g.M + TCG_M - 1) / TCG_M) * E;
    const int n_chunks = (g.K + TCG_K - 1) / TCG_K;
    int splits = 1;
    if (EPI == EPI_STORE && part) {
        // about two CTAs per SM of the 152, as far as the chunks and the scratch allow
        splits = std::min(n_chunks, std::max(1, 304 / tiles));
        const size_t per_split = (size_t)E * g.M * g.N;
        splits = (int)std::min<size_t>((size_t)splits, part_cap / per_split);
        splits = std::max(splits, 1);
    }
    const int cps = (n_chunks + splits - 1) / splits;
    splits = (n_chunks + cps - 1) / cps;   // every split owns at least one chunk
    dim3 grid((g.N + TCG_N - 1) / TCG_N, (g.M + TCG_M - 1) / TCG_M, E * splits);
    note_launch();
    kern<<<grid, TCG_THREADS, TCG_SMEM, s>>>(g, error, wait_limit, splits, cps, splits > 1 ? part : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess || splits == 1) return e;
    const int64_t total = (int64_t)E * g.M * g.N;
    note_launch();
    mlp_splitk_reduce_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4 * 152), 256, 0, s>>>(
        part, splits, E, g.M, g.N, g.C, g.ldc, g.c_mem);
    return cudaGetLastError();
}

}  // namespace tvbx

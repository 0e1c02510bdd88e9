// Tensor-core FC block moments (arXiv 2311.13337, Sec. "Output" and Eq. 6:
// the FC is the Pearson correlation of the simulated E series).
//
// For each set the Gram matrix of the shifted series, G = Z Z^T with
// Z[k][t] = x_k(t) - m_k, is a dense contraction over time, so it runs on the
// fifth-generation tensor cores (tcgen05) with the accumulator in tensor
// memory. Z is split into a high part H and a low part L (Z = H + L up to the
// rounding of L) in BF16 or TF32; the "x3" modes form
//   D = H H^T + H (2L)^T,   G = (D + D^T) / 2 = H H^T + H L^T + L H^T,
// i.e. the three-product split-precision form with two MMAs (the L L^T term
// is below the FP32 rounding of G). The single modes use D = H H^T.
// Accumulation is FP32 throughout. The row sums s[k] = sum_t Z[k][t] use
// compensated (Kahan) FP32 summation in the loading threads.
//
// Output: the same block-moment format as the SIMT kernel,
// blocks[p][b][N*N + N] = (G_b, s_b) for the blocks of `blk` samples, so the
// finalize (Pearson, chi, mean FC) and FCD kernels are shared.
//
// Layout. A CTA owns SC consecutive sets (one 16- or 8-byte piece of every
// (t, k) row of the [T][N][P] series) and all their samples. Per chunk of 128
// bytes of K (64 BF16 or 32 TF32 samples) each thread (k, j) loads samples
// j*SPC .. j*SPC+SPC-1 of region k for the SC sets, subtracts the shift,
// splits, and writes one 16-byte piece of row k of each operand buffer in the
// 128-byte swizzled K-major layout the MMA reads. Two stages: the loads of
// chunk c+1 are in flight while chunk c is converted, and the MMAs of chunk c
// run while chunk c+1 is converted. Thread 0 issues the MMAs (M = 128 rows,
// of which the first N are regions; N_mma = N rounded up to 16) and commits
// them to the stage's mbarrier, which the loaders wait on (bounded) before
// overwriting the stage. After the last chunk of a block, warps 0-3 read the
// accumulator rows out of tensor memory (lane = region) into shared memory,
// and all threads write the symmetrised block moments.
//
// Rows N .. 127 of the A operand and N .. N_mma - 1 of the B operand are
// whatever follows the buffer in shared memory (in bounds by construction);
// they only reach accumulator rows and columns >= N, which are never read.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "ptx_async.cuh"

namespace tvbx {

namespace {

template <int SC> struct LoadVec;
template <> struct LoadVec<4> { using T = float4; };
template <> struct LoadVec<2> { using T = float2; };

static __device__ __forceinline__ float lv(const float4& v, int s)
{
    return s == 0 ? v.x : (s == 1 ? v.y : (s == 2 ? v.z : v.w));
}
static __device__ __forceinline__ float lv(const float2& v, int s) { return s == 0 ? v.x : v.y; }
static __device__ __forceinline__ void lset(float4& v, int s, float x)
{
    if (s == 0) v.x = x; else if (s == 1) v.y = x; else if (s == 2) v.z = x; else v.w = x;
}
static __device__ __forceinline__ void lset(float2& v, int s, float x)
{
    if (s == 0) v.x = x; else v.y = x;
}

static __device__ __forceinline__ void kahan(float& sum, float& comp, float x)
{
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

static __device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}

static __device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

}  // namespace

// PREC: 1 BF16, 2 BF16x3, 3 TF32, 4 TF32x3 (the TVBX_FC_* values).
template <int PREC, int SC, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
fc_tc_kernel(const __grid_constant__ FcArgs a, int32_t R, int32_t Ncols, uint32_t tmem_cols, int32_t vec_ok)
{
    constexpr int KIND = (PREC <= 2) ? 0 : 1;        // 0: kind::f16 (bf16), 1: kind::tf32
    constexpr bool SPLIT = (PREC == 2 || PREC == 4);
    constexpr int NBUF = SPLIT ? 2 : 1;
    constexpr int SPC = KIND == 0 ? 8 : 4;            // samples per 16-byte piece
    constexpr int KC = 8 * SPC;                       // samples per 128-byte chunk
    using V = typename LoadVec<SC>::T;

    extern __shared__ uint8_t dyn_smem[];
    __shared__ uint64_t s_mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int N = a.N;
    const int64_t P = a.P;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int k = tid >> 3, j = tid & 7;
    const bool loader = k < N;
    const int64_t p0 = (int64_t)blockIdx.x * SC;
    const int64_t Tn = a.t_end - a.t_begin;
    const int64_t blk = a.blk > 0 ? (int64_t)a.blk : Tn;
    const int64_t NP = (int64_t)N * P;
    const uint32_t buf_bytes = (uint32_t)R * 128u;
    const uint32_t stage_bytes = (uint32_t)SC * NBUF * buf_bytes;

    // 1024-byte aligned operand area
    const uint32_t raw = smem_u32(dyn_smem);
    const uint32_t base = (raw + 1023u) & ~1023u;
    float* dmat = reinterpret_cast<float*>(dyn_smem + (base - raw));   // drain area (overlaps the stages)

    if (warp == 0) tmem_alloc(&s_tmem, tmem_cols);
    if (tid == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        s_abort = 0;
        fence_mbarrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // shift of this thread's region for each set
    float sh[SC];
#pragma unroll
    for (int s = 0; s < SC; ++s) {
        float m = 0.0f;
        if (loader && p0 + s < P) {
            const int64_t o = (int64_t)k * P + p0 + s;
            if (a.state) m = Tn > 0 ? a.state[(int64_t)SV_SUM_E * NP + o] / (float)Tn : 0.0f;
            else if (a.shift) m = a.shift[o];
        }
        sh[s] = m;
    }

    // global chunk sequence: blocks b, chunks c of KC samples (last one partial)
    auto chunk_range = [&](int64_t b, int64_t c, int64_t& ts, int64_t& te) {
        const int64_t b0 = b * blk;
        const int64_t b1 = (b0 + blk < Tn) ? b0 + blk : Tn;
        ts = b0 + c * KC;
        te = (ts + KC < b1) ? ts + KC : b1;
    };
    auto load_chunk = [&](int64_t ts, int64_t te, V* v) {
#pragma unroll
        for (int i = 0; i < SPC; ++i) {
            const int64_t t = ts + j * SPC + i;
            V x;
#pragma unroll
            for (int s = 0; s < SC; ++s) lset(x, s, 0.0f);
            if (loader && t < te) {
                const float* src = a.series + (a.t_begin + t) * NP + (int64_t)k * P + p0;
                if (vec_ok) {
                    x = __ldcs(reinterpret_cast<const V*>(src));
                } else {
#pragma unroll
                    for (int s = 0; s < SC; ++s)
                        if (p0 + s < P) lset(x, s, __ldcs(src + s));
                }
            }
            v[i] = x;
        }
    };

    float S[SC], C[SC];
#pragma unroll
    for (int s = 0; s < SC; ++s) S[s] = C[s] = 0.0f;

    const uint32_t row_off = (uint32_t)(k >> 3) * 1024u + (uint32_t)(k & 7) * 128u +
                             (uint32_t)((j ^ (k & 7)) << 4);
    const uint32_t idesc = tc_idesc(KIND == 0 ? 1u : 2u, 128u, (uint32_t)Ncols);
    const int64_t n_blocks = a.n_blocks;

    V cur[SPC], nxt[SPC];
    int64_t gc = 0;      // chunks issued so far
    bool ok = true;
    {
        int64_t ts, te;
        chunk_range(0, 0, ts, te);
        load_chunk(ts, te, cur);
    }
    for (int64_t b = 0; b < n_blocks && ok; ++b) {
        int64_t bs, be;
        chunk_range(b, 0, bs, be);
        const int64_t blen = ((b * blk + blk < Tn) ? b * blk + blk : Tn) - b * blk;
        const int64_t nck = (blen + KC - 1) / KC;
        for (int64_t c = 0; c < nck; ++c) {
            int64_t ts, te;
            chunk_range(b, c, ts, te);
            // prefetch the next chunk (in this block or the next one)
            {
                int64_t nb = b, ncn = c + 1;
                if (ncn >= nck) { nb = b + 1; ncn = 0; }
                if (nb < n_blocks) {
                    int64_t nts, nte;
                    chunk_range(nb, ncn, nts, nte);
                    load_chunk(nts, nte, nxt);
                }
            }
            const int stage = (int)(gc & 1);
            if (gc >= 2 && !mbar_wait_bounded(&s_mbar[stage], (uint32_t)(((gc - 2) >> 1) & 1), a.wait_limit)) {
                atomicOr(a.error, TVBX_DEVERR_TIMEOUT);
                s_abort = 1;
            }
            // convert and store this thread's piece of every operand buffer
            if (loader) {
                const uint32_t sbase = base + (uint32_t)stage * stage_bytes;
#pragma unroll
                for (int s = 0; s < SC; ++s) {
                    float z[SPC];
#pragma unroll
                    for (int i = 0; i < SPC; ++i) {
                        const int64_t t = ts + j * SPC + i;
                        z[i] = (t < te && p0 + s < P) ? lv(cur[i], s) - sh[s] : 0.0f;
                        kahan(S[s], C[s], z[i]);
                    }
                    uint32_t hw[4], lw[4];
                    if constexpr (KIND == 0) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(z[2 * q], z[2 * q + 1]);
                            hw[q] = *reinterpret_cast<const uint32_t*>(&h);
                            if constexpr (SPLIT) {
                                const float2 hf = __bfloat1622float2(h);
                                const __nv_bfloat162 l =
                                    __floats2bfloat162_rn(2.0f * (z[2 * q] - hf.x), 2.0f * (z[2 * q + 1] - hf.y));
                                lw[q] = *reinterpret_cast<const uint32_t*>(&l);
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            hw[q] = tf32_rna(z[q]);
                            if constexpr (SPLIT) lw[q] = __float_as_uint(2.0f * (z[q] - __uint_as_float(hw[q])));
                        }
                    }
                    const uint32_t hb = sbase + (uint32_t)s * NBUF * buf_bytes;
                    st_shared_v4(hb + row_off, hw[0], hw[1], hw[2], hw[3]);
                    if constexpr (SPLIT) st_shared_v4(hb + buf_bytes + row_off, lw[0], lw[1], lw[2], lw[3]);
                }
            }
            fence_proxy_async_shared();
            __syncthreads();
            if (s_abort) { ok = false; break; }
            if (tid == 0) {
                tc_fence_after();
                const uint32_t sbase = base + (uint32_t)stage * stage_bytes;
#pragma unroll 1
                for (int s = 0; s < SC; ++s) {
                    const uint32_t hb = sbase + (uint32_t)s * NBUF * buf_bytes;
                    const uint32_t d = tmem + (uint32_t)(s * Ncols);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = sw128_desc(hb + 32u * ks);
                        tc_mma<KIND>(d, ad, ad, idesc, (c == 0 && ks == 0) ? 0u : 1u);
                        if constexpr (SPLIT) tc_mma<KIND>(d, ad, sw128_desc(hb + buf_bytes + 32u * ks), idesc, 1u);
                    }
                }
                tc_commit(&s_mbar[stage]);
            }
            ++gc;
#pragma unroll
            for (int i = 0; i < SPC; ++i) cur[i] = nxt[i];
        }
        if (!ok) break;

        // ---- block epilogue: wait for the last MMAs, drain, write ----
        if (!mbar_wait_bounded(&s_mbar[(gc - 1) & 1], (uint32_t)(((gc - 1) >> 1) & 1), a.wait_limit)) {
            atomicOr(a.error, TVBX_DEVERR_TIMEOUT);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) { ok = false; break; }
        tc_fence_after();
        if (warp < 4) {
            const int row = warp * 32 + lane;
            for (int s = 0; s < SC; ++s) {
                for (int cb = 0; cb * 16 < N; ++cb) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * Ncols + cb * 16), v);
                    if (row < N) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int col = cb * 16 + q;
                            if (col < N) dmat[((int64_t)s * N + row) * (N + 1) + col] = v[q];
                        }
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        const int64_t stride_b = (int64_t)N * N + N;
        for (int idx = tid; idx < SC * N * N; idx += blockDim.x) {
            const int s = idx / (N * N);
            const int r = idx - s * N * N;
            const int i = r / N, jj = r - i * N;
            if (p0 + s < P) {
                const float* Ds = dmat + (int64_t)s * N * (N + 1);
                float g = 0.5f * (Ds[i * (N + 1) + jj] + Ds[jj * (N + 1) + i]);
                a.blocks[((p0 + s) * a.n_blocks + b) * stride_b + r] = g;
            }
        }
#pragma unroll
        for (int s = 0; s < SC; ++s) {
            float v = S[s] - C[s];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            if (loader && j == 0 && p0 + s < P)
                a.blocks[((p0 + s) * a.n_blocks + b) * stride_b + (int64_t)N * N + k] = v;
            S[s] = C[s] = 0.0f;
        }
        __syncthreads();   // the drain area is the next block's stage area
    }

    // leave: make sure no MMA is still running, then free tensor memory
    if (tid == 0 && gc > 0) {
        mbar_wait_bounded(&s_mbar[(gc - 1) & 1], (uint32_t)(((gc - 1) >> 1) & 1), a.wait_limit);
        if (gc > 1) mbar_wait_bounded(&s_mbar[gc & 1], (uint32_t)(((gc - 2) >> 1) & 1), a.wait_limit);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

// Geometry shared by the launcher and the host-side checks.
struct FcTcGeom {
    int SC, R, Ncols, threads;
    uint32_t tmem_cols;
    size_t smem;
};

static bool fc_tc_geom(int N, int prec, FcTcGeom& g)
{
    if (N < 1 || N > 128) return false;
    g.SC = N <= 72 ? 4 : 2;
    g.R = (N + 7) / 8 * 8;
    g.Ncols = (N + 15) / 16 * 16;
    int t = (8 * N + 31) / 32 * 32;
    g.threads = t < 128 ? 128 : t;
    const int nbuf = (prec == TVBX_FC_BF16X3 || prec == TVBX_FC_TF32X3) ? 2 : 1;
    const size_t buf = (size_t)g.R * 128;
    const size_t stage = (size_t)g.SC * nbuf * buf;
    const size_t main_bytes = 2 * stage + (size_t)(128 - g.R) * 128;
    const size_t drain = sizeof(float) * (size_t)g.SC * N * (N + 1);
    g.smem = 1024 + (main_bytes > drain ? main_bytes : drain);
    uint32_t need = (uint32_t)(g.SC * g.Ncols), cols = 32;
    while (cols < need) cols <<= 1;
    g.tmem_cols = cols;
    // more than half of the tensor memory: keep a second CTA off the SM (its
    // allocation would only wait for this one's release)
    if (cols > 256 && g.smem < 116 * 1024) g.smem = 116 * 1024;
    return cols <= 512 && g.smem <= 227 * 1024;
}

bool fc_tc_supported(int N, int prec)
{
    FcTcGeom g;
    return prec >= TVBX_FC_BF16 && prec <= TVBX_FC_TF32X3 && fc_tc_geom(N, prec, g);
}

template <int PREC, int SC, int MAXT>
static cudaError_t launch_one(const FcArgs& a, const FcTcGeom& g, int vec_ok, cudaStream_t s)
{
    auto kern = fc_tc_kernel<PREC, SC, MAXT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((a.P + SC - 1) / SC);
    note_launch();
    kern<<<grid, g.threads, g.smem, s>>>(a, g.R, g.Ncols, g.tmem_cols, vec_ok);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_prec(const FcArgs& a, const FcTcGeom& g, cudaStream_t s)
{
    const int vec_ok = (a.P % g.SC == 0) && ((uintptr_t)a.series % 16 == 0) ? 1 : 0;
    if (g.SC == 4) return launch_one<PREC, 4, 576>(a, g, vec_ok, s);
    return launch_one<PREC, 2, 1024>(a, g, vec_ok, s);
}

cudaError_t launch_fc_tc_moments(const FcArgs& a, int prec, cudaStream_t s)
{
    FcTcGeom g;
    if (!fc_tc_geom(a.N, prec, g) || !a.error) return cudaErrorInvalidValue;
    switch (prec) {
    case TVBX_FC_BF16: return launch_prec<TVBX_FC_BF16>(a, g, s);
    case TVBX_FC_BF16X3: return launch_prec<TVBX_FC_BF16X3>(a, g, s);
    case TVBX_FC_TF32: return launch_prec<TVBX_FC_TF32>(a, g, s);
    case TVBX_FC_TF32X3: return launch_prec<TVBX_FC_TF32X3>(a, g, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvbx

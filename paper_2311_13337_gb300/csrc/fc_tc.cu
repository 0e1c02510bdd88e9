// Tensor-core FC block moments (arXiv 2311.13337, Sec. "Output" and Eq. 6:
// the FC is the Pearson correlation of the simulated E series).
//
// For each set the Gram matrix of the shifted series, G = Z Z^T with
// Z[k][t] = x_k(t) - m_k, is a dense contraction over time, so it runs on the
// fifth-generation tensor cores (tcgen05) with the accumulator in tensor
// memory. Z is split into a high part H and a low part L (Z = H + L up to the
// rounding of L) in BF16 or TF32; the "x3" modes form the three-product
// split-precision Gram matrix
//   G = H H^T + H L^T + L H^T
// with three MMAs per K step. The L L^T term left out, like the rounding of L
// itself, is about 2^-16 of G in the BF16 forms (2^-22 in TF32), so the x3
// forms reach a few 1e-6 in the FC, not FP32 rounding. The single modes use
// G = H H^T. Both are symmetric up to the rounding
// of the accumulation, so readers take the upper triangle.
// Accumulation is FP32 throughout. The row sums s[k] = sum_t Z[k][t] use
// compensated (Kahan) FP32 summation in the loading threads.
//
// Output: the same block-moment format as the SIMT kernel,
// blocks[p][b][N*N + N] = (G_b, s_b) for the blocks of `blk` samples, so the
// finalize (Pearson, chi, mean FC) and FCD kernels are shared.
//
// Layout. A CTA owns SC consecutive sets (one 16- or 8-byte piece of every
// (t, k) row of the series: in the set-blocked layout the pieces of
// neighbouring regions are adjacent, so a warp's 4 regions x 8 sample groups
// read 8 segments of 64 bytes; in [T][N][P], 32 separate pieces) and all
// their samples. Per chunk of 128 bytes of K (64 BF16 or 32 TF32 samples)
// each loader thread (k, j) copies
// samples j*SPC .. j*SPC+SPC-1 of region k for the SC sets into its raw slot
// in shared memory (cp.async). Once chunk c has landed the thread reads its
// slot into registers and subtracts the shift, copies chunk c+1 into the same
// slot (in flight during the conversion), splits into registers (packed
// f32x2 arithmetic for the BF16 forms), and waits only for the MMAs of chunk
// c-2 to release the operand stage it writes (two stages, alternating by
// chunk), so the conversion of chunk c overlaps the MMAs of chunk c-1; it
// writes one 16-byte piece of row k of each operand buffer in the 128-byte
// swizzled K-major layout the MMA reads. One lane of the MMA warp issues the MMAs (M = 128 rows, of which the
// first N are regions; N_mma = N rounded up to 16) and commits them to the
// stage's mbarrier. Shared memory: the two operand stages, (128 - R) rows of
// 128 bytes (the A rows read beyond the last buffer), the raw slots. At the
// end of a block loader warps 0-3 read the accumulator rows out of tensor
// memory (lane = region) and write their diagonal and upper triangle to
// global memory, while the other loader warps already stage the next block's
// first chunk. Waits that may be long suspend in hardware (try_wait with a
// time hint) rather than poll.
//
// Rows N .. 127 of the A operand and N .. N_mma - 1 of the B operand are
// whatever follows the buffer in shared memory (in bounds by construction);
// they only reach accumulator rows and columns >= N, which are never read.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

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

// cp.async of `bytes` (4, 8 or 16) with zero fill: src_bytes = 0 writes zeros
// and reads nothing (src must still be a valid address).
template <int BYTES>
static __device__ __forceinline__ void cp_async_zfill(uint32_t dst, const void* src, uint32_t src_bytes)
{
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src), "n"(BYTES), "r"(src_bytes)
                     : "memory");
}

static __device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Two FP32 values in one 64-bit register pair, for the packed f32x2
// arithmetic of sm_100-class SMs (each lane rounds exactly like the scalar
// instruction, so packed and scalar forms give the same bits).
static __device__ __forceinline__ uint64_t pk2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};\n" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
static __device__ __forceinline__ float2 un2(uint64_t v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;\n" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
static __device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;\n" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
static __device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;\n" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// BF16 pair (lo, hi) rounded to nearest even, lo in the low half
static __device__ __forceinline__ uint32_t bf2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

}  // namespace

// Bounded wait that lets the hardware suspend the thread for up to ns
// nanoseconds per attempt (the suspend-time hint of try_wait: the thread
// resumes when the phase completes), instead of polling with sleeps in
// between. Returns false after limit attempts.
static __device__ __forceinline__ bool mbar_wait_hint(uint64_t* bar, uint32_t parity, uint32_t limit, uint32_t ns)
{
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

// Bounded wait by lane 0 of a warp, then the whole warp proceeds. After an
// expiry (or once any wait of the CTA has expired) the wait is skipped: the
// kernel then runs to its end without blocking and reports the error.
// sleep_ns != 0 marks a wait that may be long: its attempts are
// hardware-suspended for up to 1 us each (2^22 attempts bound it to seconds).
static __device__ __forceinline__ void warp_wait(uint64_t* bar, uint32_t parity, uint32_t limit,
                                                 volatile int* abort, uint32_t* error, uint32_t sleep_ns = 0)
{
    if ((threadIdx.x & 31) == 0 && !*abort &&
        !(sleep_ns ? mbar_wait_hint(bar, parity, limit, 1000u) : mbar_wait_bounded(bar, parity, limit))) {
        atomicOr(error, TVBX_DEVERR_TIMEOUT);
        *abort = 1;
    }
    __syncwarp();
}

// Accumulator rows of one lane quarter (the calling warp's) of every set
// to the block-moment rows in global memory (16-byte stores where the rows
// are 16-byte aligned, i.e. N a multiple of 4). Readers take the diagonal and
// the upper triangle only, so a row is written from the 16-column block that
// holds its diagonal on, and blocks below every row of the quarter are not
// read out of tensor memory.
template <int SC>
static __device__ __forceinline__ void drain_quarter(const FcArgs& a, uint32_t tmem, int quarter, int Ncols, int64_t p0,
                                                     int64_t b)
{
    const int N = a.N;
    const int64_t P = a.P;
    const int row = quarter * 32 + (threadIdx.x & 31);
    const int64_t stride_b = (int64_t)N * N + N;
    const bool vec = (N & 3) == 0;
    for (int s = 0; s < SC; ++s) {
        float* out = a.blocks + ((p0 + s) * a.n_blocks + b) * stride_b + (int64_t)row * N;
        const bool w_ok = row < N && p0 + s < P;
        for (int cb = quarter * 2; cb * 16 < N; ++cb) {   // columns from 32 * quarter on
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * Ncols + cb * 16), v);
            if (w_ok && cb * 16 + 16 > row) {
                if (vec && cb * 16 + 16 <= N) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4*>(out + cb * 16 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (cb * 16 + q < N) out[cb * 16 + q] = v[q];
                }
            }
        }
    }
}

// PREC: 1 BF16, 2 BF16x3, 3 TF32, 4 TF32x3 (the TVBX_FC_* values).
//
// Roles. Warps 0 .. NLW-1 load, shift, split and store (thread (k, j) =
// region k, 16-byte piece j of each 128-byte row); warp NLW issues the MMAs
// (one lane); loader warps 0 .. 3 also drain the accumulator of each finished
// block from tensor memory (warp w reads lanes 32 w ..). Hand-offs are
// mbarriers: full[stage] (one arrival per loader warp), empty[stage] (MMA commit), accf
// (MMA commit after a block's last chunk), drained (one arrival per draining
// warp) -- no CTA-wide barrier inside the loop.
template <int PREC, int SC, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
fc_tc_kernel(const __grid_constant__ FcArgs a, int32_t R, int32_t Ncols, uint32_t tmem_cols, int32_t vec_ok,
             int32_t n_loader_warps)
{
    constexpr int KIND = (PREC <= 2) ? 0 : 1;        // 0: kind::f16 (bf16), 1: kind::tf32
    constexpr bool SPLIT = (PREC == 2 || PREC == 4);
    constexpr int NBUF = SPLIT ? 2 : 1;
    constexpr int SPC = KIND == 0 ? 8 : 4;            // samples per 16-byte piece
    constexpr int KC = 8 * SPC;                       // samples per 128-byte chunk
    using V = typename LoadVec<SC>::T;

    extern __shared__ uint8_t dyn_smem[];
    __shared__ uint64_t s_full[2], s_empty[2], s_accf, s_drained;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int N = a.N;
    const int64_t P = a.P;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int NLW = n_loader_warps;
    const int64_t p0 = (int64_t)blockIdx.x * SC;
    const bool all_sets = p0 + SC <= P;
    const int64_t Tn = a.t_end - a.t_begin;
    const int64_t blk = a.blk > 0 ? (int64_t)a.blk : Tn;
    const int64_t NP = (int64_t)N * P;
    const int64_t n_blocks = a.n_blocks;
    const uint32_t buf_bytes = (uint32_t)R * 128u;
    const uint32_t stage_bytes = (uint32_t)SC * NBUF * buf_bytes;
    const uint32_t raw = smem_u32(dyn_smem);
    const uint32_t base = (raw + 1023u) & ~1023u;     // 1024-byte aligned operand stages
    volatile int* abort = &s_abort;

    if (warp == NLW) tmem_alloc(&s_tmem, tmem_cols);
    if (tid == 0) {
        mbar_init(&s_full[0], NLW);
        mbar_init(&s_full[1], NLW);
        mbar_init(&s_empty[0], 1);
        mbar_init(&s_empty[1], 1);
        mbar_init(&s_accf, 1);
        mbar_init(&s_drained, 4);
        s_abort = 0;
        fence_mbarrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // sample indices within the window fit in 32 bits (the launcher checks)
    const int T32 = (int)Tn, blk32 = (int)blk, nb32 = (int)n_blocks;
    auto block_len = [&](int b) { return ((b * blk32 + blk32 < T32) ? b * blk32 + blk32 : T32) - b * blk32; };

    if (warp < NLW) {
        // ------------------------------------------------------------ loaders
        const int k = tid >> 3, j = tid & 7;
        const bool loader = k < N;
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
        // sample t of region k for sets p0 ..: series_index(t, k, p0), consecutive samples st apart
        const float* src0 = a.series + series_index(a.sl, a.t_begin + (int64_t)j * SPC, k, p0);
        const int64_t st = a.sl.st;
        const bool fast_sets = loader && all_sets && vec_ok;
        // this thread's raw slot (q = 0): SPC pieces of SC floats, piece i at
        // raw_base + ((q * SPC + i) * NLT + tid) * 4 SC
        // (a warp's pieces are contiguous)
        constexpr int PBYTES = 4 * SC;
        const int NLT = 32 * NLW;
        const uint32_t raw_base = base + 2u * stage_bytes + (uint32_t)(128 - R) * 128u;
        // copy samples [ts, te) of this thread's piece into raw slot q; samples
        // outside and sets >= P are zero-filled
        auto issue_chunk = [&](int ts, int te, int q) {
            const float* src = src0 + (int64_t)ts * st;
            if (fast_sets && te - ts == KC) {
                const uint32_t dst0 = raw_base + (uint32_t)(q * SPC * NLT + tid) * PBYTES;
#pragma unroll
                for (int i = 0; i < SPC; ++i)
                    cp_async_zfill<PBYTES>(dst0 + (uint32_t)(i * NLT * PBYTES), src + i * st, PBYTES);
            } else if (all_sets && vec_ok) {
#pragma unroll
                for (int i = 0; i < SPC; ++i) {
                    const uint32_t dst = raw_base + (uint32_t)((q * SPC + i) * NLT + tid) * PBYTES;
                    const bool tv = loader && ts + j * SPC + i < te;
                    cp_async_zfill<PBYTES>(dst, tv ? (const void*)(src + i * st) : (const void*)a.series,
                                           tv ? PBYTES : 0u);
                }
            } else {   // sets not a multiple of SC or an unaligned series: 4-byte copies
#pragma unroll 1
                for (int i = 0; i < SPC; ++i) {
                    const uint32_t dst = raw_base + (uint32_t)((q * SPC + i) * NLT + tid) * PBYTES;
                    const bool tv = loader && ts + j * SPC + i < te;
#pragma unroll 1
                    for (int s = 0; s < SC; ++s) {
                        const bool ok_s = tv && p0 + s < P;
                        cp_async_zfill<4>(dst + 4 * s, ok_s ? (const void*)(src + i * st + s) : (const void*)a.series,
                                          ok_s ? 4u : 0u);
                    }
                }
            }
        };
        const uint32_t row_off = (uint32_t)(k >> 3) * 1024u + (uint32_t)(k & 7) * 128u +
                                 (uint32_t)((j ^ (k & 7)) << 4);
        float S[SC], C[SC];   // TF32 forms: row sums and their compensation
#pragma unroll
        for (int s = 0; s < SC; ++s) S[s] = C[s] = 0.0f;
        constexpr int NH = SC / 2;
        uint64_t S2[NH], C2[NH], shp[NH];   // BF16 forms: the same per set pair
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            S2[h] = C2[h] = pk2(0.0f, 0.0f);
            shp[h] = pk2(sh[2 * h], sh[2 * h + 1]);
        }
        // chunks are issued two ahead of the one being converted: the cursor
        // (ib, ic) is the next chunk to copy; an empty group keeps the count
        int ib = 0, ic = 0;
        auto issue_next = [&](int q) {
            if (ib < nb32) {
                const int b0 = ib * blk32, blen = block_len(ib);
                const int ts = b0 + ic * KC;
                issue_chunk(ts, (ts + KC < b0 + blen) ? ts + KC : b0 + blen, q);
                if (++ic * KC >= blen) { ic = 0; ++ib; }
            }
            cp_async_commit();
        };
        issue_next(0);
        int gc = 0;
        for (int b = 0; b < nb32; ++b) {
            const int b0 = b * blk32, blen = block_len(b);
            const int nck = (blen + KC - 1) / KC;
            for (int c = 0; c < nck; ++c) {
                const int ts = b0 + c * KC;
                const int te = (ts + KC < b0 + blen) ? ts + KC : b0 + blen;
                const int q = 0;                                          // the single raw slot
                const uint32_t st_q = (uint32_t)(gc & 1);                 // operand stage of this chunk
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // this chunk has landed
                // the chunk's samples to registers, shifted; padding samples and
                // missing sets are 0
                const bool full_chunk = fast_sets && te - ts == KC;
                const uint8_t* slot = dyn_smem + (raw_base - raw) + (size_t)(q * SPC * NLT + tid) * PBYTES;
                uint32_t hw[SC][4], lw[SC][4];
                if constexpr (KIND == 0) {
                    // sets 2h and 2h + 1 of every sample in one register pair
                    uint64_t zp[SPC][NH];
#pragma unroll
                    for (int i = 0; i < SPC; ++i) {
                        const V x = *reinterpret_cast<const V*>(slot + (size_t)i * NLT * PBYTES);
#pragma unroll
                        for (int h = 0; h < NH; ++h) zp[i][h] = sub2(pk2(lv(x, 2 * h), lv(x, 2 * h + 1)), shp[h]);
                    }
                    if (!full_chunk) {   // padding samples and missing sets are 0
#pragma unroll
                        for (int i = 0; i < SPC; ++i)
#pragma unroll
                            for (int h = 0; h < NH; ++h) {
                                float2 v = un2(zp[i][h]);
                                const bool tv = loader && ts + j * SPC + i < te;
                                if (!(tv && p0 + 2 * h < P)) v.x = 0.0f;
                                if (!(tv && p0 + 2 * h + 1 < P)) v.y = 0.0f;
                                zp[i][h] = pk2(v.x, v.y);
                            }
                    }
                    // the slot has been read (the values above depend on it): copy
                    // the next chunk into it while this one is split and the
                    // previous chunk's MMAs run
                    issue_next(q);
#pragma unroll
                    for (int h = 0; h < NH; ++h) {
                        uint64_t part[SPC];
#pragma unroll
                        for (int i = 0; i < SPC; ++i) part[i] = zp[i][h];
#pragma unroll
                        for (int w = SPC / 2; w > 0; w >>= 1)
#pragma unroll
                            for (int i = 0; i < w; ++i) part[i] = add2(part[i], part[i + w]);
                        const uint64_t y = sub2(part[0], C2[h]);   // compensated sum, both sets
                        const uint64_t t = add2(S2[h], y);
                        C2[h] = sub2(sub2(t, S2[h]), y);
                        S2[h] = t;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
#pragma unroll
                        for (int h = 0; h < NH; ++h) {
                            const float2 z0 = un2(zp[2 * u][h]), z1 = un2(zp[2 * u + 1][h]);
                            const uint32_t ha = bf2(z0.x, z1.x);   // set 2h, samples 2u and 2u + 1
                            const uint32_t hb = bf2(z0.y, z1.y);   // set 2h + 1
                            hw[2 * h][u] = ha;
                            hw[2 * h + 1][u] = hb;
                            if constexpr (SPLIT) {
                                // the high parts back in FP32 (exact), then the low parts
                                const uint64_t h0 = pk2(__uint_as_float(ha << 16), __uint_as_float(hb << 16));
                                const uint64_t h1 = pk2(__uint_as_float(ha & 0xffff0000u), __uint_as_float(hb & 0xffff0000u));
                                const float2 l0 = un2(sub2(zp[2 * u][h], h0)), l1 = un2(sub2(zp[2 * u + 1][h], h1));
                                lw[2 * h][u] = bf2(l0.x, l1.x);
                                lw[2 * h + 1][u] = bf2(l0.y, l1.y);
                            }
                        }
                    }
                } else {
                    float zz[SC][SPC];
#pragma unroll
                    for (int i = 0; i < SPC; ++i) {
                        const V x = *reinterpret_cast<const V*>(slot + (size_t)i * NLT * PBYTES);
#pragma unroll
                        for (int s = 0; s < SC; ++s) zz[s][i] = lv(x, s) - sh[s];
                    }
                    if (!full_chunk) {
#pragma unroll
                        for (int s = 0; s < SC; ++s)
#pragma unroll
                            for (int i = 0; i < SPC; ++i)
                                if (!(loader && ts + j * SPC + i < te && p0 + s < P)) zz[s][i] = 0.0f;
                    }
                    issue_next(q);
#pragma unroll
                    for (int s = 0; s < SC; ++s) {
                        const float* z = zz[s];
                        float part[SPC];
#pragma unroll
                        for (int i = 0; i < SPC; ++i) part[i] = z[i];
#pragma unroll
                        for (int w = SPC / 2; w > 0; w >>= 1)
#pragma unroll
                            for (int i = 0; i < w; ++i) part[i] += part[i + w];
                        kahan(S[s], C[s], part[0]);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            hw[s][u] = tf32_rna(z[u]);
                            if constexpr (SPLIT) lw[s][u] = __float_as_uint(z[u] - __uint_as_float(hw[s][u]));
                        }
                    }
                }
                // the operand stage is free once the previous chunk's MMAs completed
                if (gc >= 2) warp_wait(&s_empty[st_q], (uint32_t)(((gc >> 1) - 1) & 1), a.wait_limit, abort, a.error, 20);
                if (loader) {
#pragma unroll
                    for (int s = 0; s < SC; ++s) {
                        const uint32_t hb = base + st_q * stage_bytes + (uint32_t)s * NBUF * buf_bytes;
                        st_shared_v4(hb + row_off, hw[s][0], hw[s][1], hw[s][2], hw[s][3]);
                        if constexpr (SPLIT) st_shared_v4(hb + buf_bytes + row_off, lw[s][0], lw[s][1], lw[s][2], lw[s][3]);
                    }
                }
                fence_proxy_async_shared();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_full[st_q]);
                ++gc;
            }
            // this block's row sums
            const int64_t stride_b = (int64_t)N * N + N;
#pragma unroll
            for (int s = 0; s < SC; ++s) {
                float v;
                if constexpr (KIND == 0) {
                    const float2 d = un2(sub2(S2[s >> 1], C2[s >> 1]));
                    v = (s & 1) ? d.y : d.x;
                } else {
                    v = S[s] - C[s];
                }
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                if (loader && j == 0 && p0 + s < P)
                    a.blocks[((p0 + s) * n_blocks + b) * stride_b + (int64_t)N * N + k] = v;
                S[s] = C[s] = 0.0f;
            }
#pragma unroll
            for (int h = 0; h < NH; ++h) S2[h] = C2[h] = pk2(0.0f, 0.0f);
            // warps 0-3: drain block b (accumulator rows, lane = region) to global
            if (warp < 4) {
                warp_wait(&s_accf, (uint32_t)(b & 1), a.wait_limit, abort, a.error, 64);
                tc_fence_after();
                drain_quarter<SC>(a, tmem, warp, Ncols, p0, b);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_drained);
            }
        }
    } else {
        // ------------------------------------------------------- MMA issue
        const uint32_t idesc = tc_idesc(KIND == 0 ? 1u : 2u, 128u, (uint32_t)Ncols);
        int gc = 0;
        for (int b = 0; b < nb32; ++b) {
            const int nck = (block_len(b) + KC - 1) / KC;
            for (int c = 0; c < nck; ++c) {
                const uint32_t st_q = (uint32_t)(gc & 1);
                warp_wait(&s_full[st_q], (uint32_t)((gc >> 1) & 1), a.wait_limit, abort, a.error, 32);
                if (c == 0 && b > 0)   // the accumulator of block b-1 must have been read
                    warp_wait(&s_drained, (uint32_t)((b - 1) & 1), a.wait_limit, abort, a.error, 32);
                tc_fence_after();
                if (lane == 0) {
#pragma unroll 1
                    for (int s = 0; s < SC; ++s) {
                        const uint32_t hb = base + st_q * stage_bytes + (uint32_t)s * NBUF * buf_bytes;
                        const uint32_t d = tmem + (uint32_t)(s * Ncols);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = sw128_desc(hb + 32u * ks);
                            tc_mma<KIND>(d, ad, ad, idesc, (c == 0 && ks == 0) ? 0u : 1u);
                            if constexpr (SPLIT) {
                                const uint64_t ld = sw128_desc(hb + buf_bytes + 32u * ks);
                                tc_mma<KIND>(d, ad, ld, idesc, 1u);   // H L^T
                                tc_mma<KIND>(d, ld, ad, idesc, 1u);   // L H^T
                            }
                        }
                    }
                    tc_commit(&s_empty[st_q]);
                    if (c + 1 == nck) tc_commit(&s_accf);
                }
                __syncwarp();
                ++gc;
            }
        }
        // the last block's drain ends every MMA before tensor memory is freed
        if (n_blocks > 0) warp_wait(&s_drained, (uint32_t)((n_blocks - 1) & 1), a.wait_limit, abort, a.error, 64);
    }

    // every MMA has completed (its block was drained); free tensor memory
    tc_fence_before();
    __syncthreads();
    if (warp == NLW) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

// Geometry shared by the launcher and the host-side checks.
struct FcTcGeom {
    int SC, R, Ncols, threads, loader_warps;
    uint32_t tmem_cols;
    size_t smem;
};

static bool fc_tc_geom(int N, int prec, FcTcGeom& g)
{
    if (N < 1 || N > 112) return false;
    g.SC = N <= 68 ? 4 : 2;
    g.R = (N + 7) / 8 * 8;
    g.Ncols = (N + 15) / 16 * 16;
    g.loader_warps = std::max(4, (8 * N + 31) / 32);   // warps 0-3 also drain the accumulator
    g.threads = 32 * g.loader_warps + 32;
    const int nbuf = (prec == TVBX_FC_BF16X3 || prec == TVBX_FC_TF32X3) ? 2 : 1;
    const size_t buf = (size_t)g.R * 128;
    const size_t stage = (size_t)g.SC * nbuf * buf;
    const int spc = (prec == TVBX_FC_BF16 || prec == TVBX_FC_BF16X3) ? 8 : 4;
    g.smem = 1024 + 2 * stage + (size_t)(128 - g.R) * 128 + (size_t)32 * g.loader_warps * spc * 4 * g.SC;
    uint32_t need = (uint32_t)(g.SC * g.Ncols), cols = 32;
    while (cols < need) cols <<= 1;
    g.tmem_cols = cols;
    // more than half of the tensor memory: keep a second CTA off the SM (its
    // allocation would only wait for this one's release)
    if (cols > 256 && g.smem < 116 * 1024) g.smem = 116 * 1024;
    return cols <= 512 && g.smem <= 227 * 1024 && g.threads <= (g.SC == 4 ? 576 : 1024);
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
    kern<<<grid, g.threads, g.smem, s>>>(a, g.R, g.Ncols, g.tmem_cols, vec_ok, g.loader_warps);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_prec(const FcArgs& a, const FcTcGeom& g, cudaStream_t s)
{
    // whole 16- (8-) byte pieces: every group of sets is aligned in the set-blocked layout
    const int vec_ok = (a.sl.sk == 4 || a.P % g.SC == 0) && ((uintptr_t)a.series % 16 == 0) ? 1 : 0;
    if (g.SC == 4) return launch_one<PREC, 4, 576>(a, g, vec_ok, s);
    return launch_one<PREC, 2, 1024>(a, g, vec_ok, s);
}

cudaError_t launch_fc_tc_moments(const FcArgs& a, int prec, cudaStream_t s)
{
    FcTcGeom g;
    if (!fc_tc_geom(a.N, prec, g) || !a.error) return cudaErrorInvalidValue;
    if (a.t_end - a.t_begin > (int64_t)INT32_MAX - 4096) return cudaErrorInvalidValue;   // 32-bit sample indices
    switch (prec) {
    case TVBX_FC_BF16: return launch_prec<TVBX_FC_BF16>(a, g, s);
    case TVBX_FC_BF16X3: return launch_prec<TVBX_FC_BF16X3>(a, g, s);
    case TVBX_FC_TF32: return launch_prec<TVBX_FC_TF32>(a, g, s);
    case TVBX_FC_TF32X3: return launch_prec<TVBX_FC_TF32X3>(a, g, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvbx

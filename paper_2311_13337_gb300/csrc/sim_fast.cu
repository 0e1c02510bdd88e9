// Prefetching simulation kernels of the tvbx engine (arXiv 2311.13337, the
// lock-step integration of Eq. 1-5 with forward Euler).
//
// A CTA owns PB sets of one speed group and all N regions of each. A thread
// owns SPT adjacent sets and RPT regions (k = t / (PB/SPT) + i * kstride),
// with their state in registers across the whole chunk (tile_common.cuh).
//
// Delays are at least one step for every nonzero weight with a positive
// tract length, so the values the coupling needs at step n + 1,
// E_j(n + 1 - d_kj), are all in the ring buffer once step n - 1 has written
// E(n). Each CTA therefore copies the delayed rows of the next step (one
// PB-float row segment per delayed weight) into shared memory while the
// current step computes. Zero-delay entries (d = 0) sit at the end of each
// CSR row and read E_j(n) directly.
//
// Two kernels:
//  * sim_fast_kernel: 16-byte cp.async copies into one buffer; two CTA
//    barriers per step (buffer consumed, then refilled).
//  * sim_bulk_kernel: one TMA bulk copy (cp.async.bulk) per row into one of
//    two buffers, completion counted in bytes on an mbarrier per buffer; one
//    CTA barrier per step, and the copy for step n + 1 is issued before the
//    wait for step n. Every mbarrier wait is bounded: on expiry the kernel
//    records TVBX_DEVERR_TIMEOUT, finishes the step with whatever is in the
//    buffer, and all threads leave at the next barrier after waiting (again
//    bounded) for their copies.
//
// In the coupling sum, the SPT sets of a thread share one broadcast weight
// load and one vector load of the gathered row. CSR rows start at an index
// of the parity of their region (a zero-weight self entry pads) so that the
// rows read together by consecutive regions of a warp fall in opposite
// halves of the shared-memory banks.

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "model_device.cuh"
#include "ptx_async.cuh"
#include "tile_common.cuh"

namespace tvbx {

// Shared-memory layout common to both kernels after the gather buffer(s).
struct TileSmem {
    float* s_w;
    uint32_t* s_cd;
    int* s_row;
    int* s_mid;
    float* s_prm;
};

template <int PB>
static __device__ __forceinline__ TileSmem stage_tile(const SimArgs& a, const TileDev& tile, const GroupDev& grp,
                                                      float* after_buffers)
{
    const int N = a.N, nnz = grp.nnz;
    TileSmem t;
    t.s_w = after_buffers;
    t.s_cd = reinterpret_cast<uint32_t*>(t.s_w + nnz);
    t.s_row = reinterpret_cast<int*>(t.s_cd + nnz);
    t.s_mid = t.s_row + N + 1;
    t.s_prm = reinterpret_cast<float*>(t.s_mid + N);
    stage_set_params<PB>(a, tile, grp, t.s_prm);
    for (int i = threadIdx.x; i < nnz; i += blockDim.x) {
        t.s_cd[i] = grp.col_dly[i];
        t.s_w[i] = grp.w[i];
    }
    for (int i = threadIdx.x; i <= N; i += blockDim.x) t.s_row[i] = grp.row_ptr[i];
    for (int i = threadIdx.x; i < N; i += blockDim.x) t.s_mid[i] = grp.row_mid[i];
    return t;
}

// ---------------------------------------------------------------------------
// cp.async, one buffer
// ---------------------------------------------------------------------------
template <int PB, int SPT, int RPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
sim_fast_kernel(const __grid_constant__ SimArgs a)
{
    constexpr int TPR = PB / SPT;
    extern __shared__ __align__(128) float smem[];
    const TileDev tile = a.tiles[blockIdx.x];
    const GroupDev grp = a.groups[tile.group];
    const int N = a.N;
    float* gbuf = smem;   // [nnz][PB]
    const TileSmem sm = stage_tile<PB>(a, tile, grp, gbuf + (size_t)grp.nnz * PB);

    ThreadSlot ts;
    ts.kstride = blockDim.x / TPR;
    ts.qt = (threadIdx.x % TPR) * SPT;
    ts.kr = threadIdx.x / TPR;
    ts.col0 = grp.p_base + tile.q0;
    ThreadPairs<SPT, RPT> tp;
    load_pairs<SPT, RPT>(a, tile, ts, tp);
    __syncthreads();

    const int H = grp.H;
    const int64_t slot_stride = (int64_t)N * grp.stride;
    float* ring_cols = grp.ring + tile.q0;
    constexpr int CH = PB / 4;
    auto prefetch = [&](int64_t mstep) {
        const int slot_m = (int)(mstep % H);
        for (int idx = threadIdx.x; idx < grp.nnz * CH; idx += blockDim.x) {
            const int e = idx / CH, c = idx - e * CH;
            const uint32_t cd = sm.s_cd[e];
            const int d = (int)(cd >> 16);
            if (d == 0) continue;
            int sl = slot_m - d;
            sl += sl < 0 ? H : 0;
            cp_async16(gbuf + (size_t)e * PB + 4 * c,
                       ring_cols + sl * slot_stride + (int64_t)(cd & 0xffffu) * grp.stride + 4 * c);
        }
        cp_async_commit();
    };

    prefetch(a.n0);
    for (int step = 0; step < a.n_chunk; ++step) {
        const int64_t n = a.n0 + step;
        const int slot_n = (int)(n % H);
        const int slot_w = slot_n + 1 == H ? 0 : slot_n + 1;
        cp_async_wait_all();
        __syncthreads();
        float cpl[SPT * RPT];
        coupling_sums<PB, SPT, RPT>(ts, N, gbuf, sm.s_w, sm.s_cd, sm.s_row, sm.s_mid, ring_cols + slot_n * slot_stride,
                                    grp.stride, cpl);
        __syncthreads();
        if (step + 1 < a.n_chunk) prefetch(n + 1);
        advance_pairs<PB, SPT, RPT>(a, ts, sm.s_prm, tp, cpl, n, step, ring_cols + slot_w * slot_stride, grp.stride);
    }
    cp_async_wait_all();
    store_pairs<SPT, RPT>(a, ts, tp);
}

// ---------------------------------------------------------------------------
// TMA bulk copies, two buffers, one barrier per step
// ---------------------------------------------------------------------------
template <int PB, int SPT, int RPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
sim_bulk_kernel(const __grid_constant__ SimArgs a)
{
    constexpr int TPR = PB / SPT;
    extern __shared__ __align__(128) float smem[];
    const TileDev tile = a.tiles[blockIdx.x];
    const GroupDev grp = a.groups[tile.group];
    const int N = a.N;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);        // [2], first 32 bytes
    int* s_abort = reinterpret_cast<int*>(smem + 8);            // timeout flag of the CTA
    float* gbuf0 = smem + 32;                                   // [nnz][PB], 128-byte aligned
    float* gbuf1 = gbuf0 + (size_t)grp.nnz * PB;
    const TileSmem sm = stage_tile<PB>(a, tile, grp, gbuf1 + (size_t)grp.nnz * PB);
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        *s_abort = 0;
        fence_mbarrier_init();
    }

    ThreadSlot ts;
    ts.kstride = blockDim.x / TPR;
    ts.qt = (threadIdx.x % TPR) * SPT;
    ts.kr = threadIdx.x / TPR;
    ts.col0 = grp.p_base + tile.q0;
    ThreadPairs<SPT, RPT> tp;
    load_pairs<SPT, RPT>(a, tile, ts, tp);

    const int H = grp.H;
    const int64_t slot_stride = (int64_t)N * grp.stride;
    float* ring_cols = grp.ring + tile.q0;
    const uint32_t row_bytes = PB * sizeof(float);
    const uint32_t step_bytes = (uint32_t)grp.nnz_d * row_bytes;
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arm(&mbar[a.n0 & 1], step_bytes);
        if (a.n_chunk > 1) mbar_arm(&mbar[(a.n0 + 1) & 1], step_bytes);
    }
    __syncthreads();

    auto prefetch = [&](int64_t mstep) {
        if (mstep == a.withhold_step) return;   // failure-path test: nothing arrives
        const int b = (int)(mstep & 1);
        float* dst = b ? gbuf1 : gbuf0;
        const int slot_m = (int)(mstep % H);
        for (int e = threadIdx.x; e < grp.nnz; e += blockDim.x) {
            const uint32_t cd = sm.s_cd[e];
            const int d = (int)(cd >> 16);
            if (d == 0) continue;
            int sl = slot_m - d;
            sl += sl < 0 ? H : 0;
            bulk_g2s(dst + (size_t)e * PB, ring_cols + sl * slot_stride + (int64_t)(cd & 0xffffu) * grp.stride,
                     row_bytes, &mbar[b]);
        }
    };

    prefetch(a.n0);
    uint32_t parity[2] = {0u, 0u};
    for (int step = 0; step < a.n_chunk; ++step) {
        const int64_t n = a.n0 + step;
        const int b = (int)(n & 1);
        const int slot_n = (int)(n % H);
        const int slot_w = slot_n + 1 == H ? 0 : slot_n + 1;
        if (step > 0) {
            __syncthreads();   // step n-1 done: its reads of the other buffer and its ring writes
            if (*s_abort) break;
        }
        if (step + 1 < a.n_chunk) prefetch(n + 1);
        const bool arrived = mbar_wait_bounded(&mbar[b], parity[b], a.wait_limit);
        if (!arrived) {
            *s_abort = 1;
            atomicOr(a.error, TVBX_DEVERR_TIMEOUT);
        }
        parity[b] ^= 1u;
        float cpl[SPT * RPT];
        coupling_sums<PB, SPT, RPT>(ts, N, b ? gbuf1 : gbuf0, sm.s_w, sm.s_cd, sm.s_row, sm.s_mid,
                                    ring_cols + slot_n * slot_stride, grp.stride, cpl);
        advance_pairs<PB, SPT, RPT>(a, ts, sm.s_prm, tp, cpl, n, step, ring_cols + slot_w * slot_stride, grp.stride);
        fence_proxy_async_global();   // E(n+1) visible to the next bulk copies
        // re-arm only a phase this thread saw complete (never twice in one phase)
        if (threadIdx.x == 0 && arrived && step + 2 < a.n_chunk) mbar_arm(&mbar[b], step_bytes);
    }
    __syncthreads();
    if (*s_abort) {
        // let copies already in flight land before the CTA's shared memory is released
        mbar_wait_bounded(&mbar[0], parity[0], a.wait_limit);
        mbar_wait_bounded(&mbar[1], parity[1], a.wait_limit);
    }
    store_pairs<SPT, RPT>(a, ts, tp);
}

// ---------------------------------------------------------------------------
// Variants: (kernel, sets per CTA, sets per thread, regions per thread, max
// threads, min CTAs per SM).
// ---------------------------------------------------------------------------
struct FastVariant {
    int bulk, pb, spt, rpt, maxt, minb;
};
static const FastVariant kFast[] = {
    {0, 16, 2, 1, 576, 1},   // 0: cp.async, 16 sets, 2 sets x 1 region per thread
    {0, 32, 4, 1, 576, 1},   // 1: cp.async, 32 sets, 4 x 1
    {0, 16, 1, 2, 576, 1},   // 2: cp.async, 16 sets, 1 x 2
    {0, 16, 2, 2, 320, 1},   // 3: cp.async, 16 sets, 2 x 2
    {1, 16, 2, 1, 576, 1},   // 4: TMA bulk, double buffer, 16 sets, 2 x 1
    {1, 16, 1, 2, 576, 1},   // 5: TMA bulk, double buffer, 16 sets, 1 x 2
    {0, 8, 2, 1, 288, 2},    // 6: cp.async, 8 sets, 2 x 1, two CTAs per SM
    {0, 8, 1, 2, 288, 2},    // 7: cp.async, 8 sets, 1 x 2, two CTAs per SM
};
constexpr int kNumFast = (int)(sizeof kFast / sizeof kFast[0]);

static size_t tail_bytes(int N, int nnz, int pb) { return 8 * (size_t)nnz + 4 * (size_t)(2 * N + 1) + 4 * 11 * (size_t)pb; }

size_t sim_fast_smem_bytes(int variant, int N, int nnz)
{
    const FastVariant& v = kFast[variant];
    const size_t buf = sizeof(float) * (size_t)nnz * v.pb;
    return v.bulk ? 128 + 2 * buf + tail_bytes(N, nnz, v.pb) : buf + tail_bytes(N, nnz, v.pb);
}

bool sim_fast_fits(int variant, int N, int nnz_max)
{
    if (variant < 0 || variant >= kNumFast) return false;
    const FastVariant& v = kFast[variant];
    const int kstride = (N + v.rpt - 1) / v.rpt;
    if (kstride * (v.pb / v.spt) > v.maxt) return false;
    if (v.bulk && (size_t)nnz_max * v.pb * sizeof(float) >= (1u << 20)) return false;   // mbarrier tx-count range
    return sim_fast_smem_bytes(variant, N, nnz_max) * v.minb <= 220 * 1024;
}

int sim_fast_pb(int variant) { return kFast[variant].pb; }
int sim_fast_variants() { return kNumFast; }

template <int BULK, int PB, int SPT, int RPT, int MAXT, int MINB>
static cudaError_t launch_fast(const SimArgs& a, int variant, int32_t n_tiles, int nnz_max, cudaStream_t s)
{
    const int kstride = (a.N + RPT - 1) / RPT;
    const int threads = kstride * (PB / SPT);
    const size_t smem = sim_fast_smem_bytes(variant, a.N, nnz_max);
    auto kern = BULK ? sim_bulk_kernel<PB, SPT, RPT, MAXT, MINB> : sim_fast_kernel<PB, SPT, RPT, MAXT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    kern<<<n_tiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sim_fast(const SimArgs& a, int variant, int32_t n_tiles, int nnz_max, cudaStream_t s)
{
    if (n_tiles <= 0 || a.n_chunk <= 0) return cudaSuccess;
    switch (variant) {
    case 0: return launch_fast<0, 16, 2, 1, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 1: return launch_fast<0, 32, 4, 1, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 2: return launch_fast<0, 16, 1, 2, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 3: return launch_fast<0, 16, 2, 2, 320, 1>(a, variant, n_tiles, nnz_max, s);
    case 4: return launch_fast<1, 16, 2, 1, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 5: return launch_fast<1, 16, 1, 2, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 6: return launch_fast<0, 8, 2, 1, 288, 2>(a, variant, n_tiles, nnz_max, s);
    case 7: return launch_fast<0, 8, 1, 2, 288, 2>(a, variant, n_tiles, nnz_max, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvbx

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
    // 16-byte aligned (the packed kernel reads two sets' parameters as one
    // float2); formed as an offset from a shared-memory pointer, so that the
    // compiler keeps its loads in the shared state space
    float* prm = reinterpret_cast<float*>(t.s_mid + N);
    t.s_prm = prm + ((16u - (uint32_t)(reinterpret_cast<uintptr_t>(prm) & 15u)) & 15u) / 4u;
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
// cp.async into one buffer (two CTA barriers per step: rows visible, then
// consumed) or, with DB, into two (one barrier per step: the rows of step
// n + 1 go into the buffer step n - 1 read, requested once every thread has
// passed the barrier of step n)
// ---------------------------------------------------------------------------
template <int PB, int SPT, int RPT, int MAXT, int MINB, bool DB>
__global__ void __launch_bounds__(MAXT, MINB)
sim_fast_kernel(const __grid_constant__ SimArgs a)
{
    constexpr int TPR = PB / SPT;
    extern __shared__ __align__(128) float smem[];
    const TileDev tile = a.tiles[blockIdx.x];
    const GroupDev grp = a.groups[tile.group];
    const int N = a.N;
    float* gbuf0 = smem;   // [nnz][PB], and with DB a second buffer after it
    float* gbuf1 = gbuf0 + (DB ? (size_t)grp.nnz * PB : 0);
    const TileSmem sm = stage_tile<PB>(a, tile, grp, gbuf1 + (size_t)grp.nnz * PB);

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
    constexpr int CH = PB / 4;   // 16-byte chunks per row
    // this thread's chunk c0 of rows e0, e0 + estep, ... (blockDim is a
    // multiple of CH because a thread owns at most 4 sets)
    const int c0 = threadIdx.x % CH, e0 = threadIdx.x / CH, estep = blockDim.x / CH;
    auto prefetch = [&](int64_t mstep, float* dst) {
        const int slot_m = (int)(mstep % H);
        for (int e = e0; e < grp.nnz; e += estep) {
            const uint32_t cd = sm.s_cd[e];
            const int d = (int)(cd >> 16);
            if (d == 0) continue;
            int sl = slot_m - d;
            sl += sl < 0 ? H : 0;
            cp_async16(dst + (size_t)e * PB + 4 * c0,
                       ring_cols + sl * slot_stride + (int64_t)(cd & 0xffffu) * grp.stride + 4 * c0);
        }
        cp_async_commit();
    };

    prefetch(a.n0, gbuf0);
    for (int step = 0; step < a.n_chunk; ++step) {
        const int64_t n = a.n0 + step;
        const int slot_n = (int)(n % H);
        const int slot_w = slot_n + 1 == H ? 0 : slot_n + 1;
        const float* gbuf = (DB && (step & 1)) ? gbuf1 : gbuf0;
        cp_async_wait_all();
        __syncthreads();   // step n's rows visible (with DB: the other buffer free, E(n) written)
        if (DB && step + 1 < a.n_chunk) prefetch(n + 1, (step & 1) ? gbuf0 : gbuf1);
        float cpl[SPT * RPT];
        coupling_sums<PB, SPT, RPT>(ts, N, gbuf, sm.s_w, sm.s_cd, sm.s_row, sm.s_mid, ring_cols + slot_n * slot_stride,
                                    grp.stride, cpl);
        if (!DB) {
            __syncthreads();   // one buffer: every read of it done before it is refilled
            if (step + 1 < a.n_chunk) prefetch(n + 1, gbuf0);
        }
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
    uint32_t par0 = 0u, par1 = 0u;   // phase parity of each buffer's mbarrier
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
        const bool arrived = mbar_wait_bounded(&mbar[b], b ? par1 : par0, a.wait_limit);
        if (!arrived) {
            *s_abort = 1;
            atomicOr(a.error, TVBX_DEVERR_TIMEOUT);
        }
        if (b) par1 ^= 1u;
        else par0 ^= 1u;
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
        mbar_wait_bounded(&mbar[0], par0, a.wait_limit);
        mbar_wait_bounded(&mbar[1], par1, a.wait_limit);
    }
    store_pairs<SPT, RPT>(a, ts, tp);
}

// ---------------------------------------------------------------------------
// TMA bulk copies into one buffer, one CTA barrier per step. The wait on the
// buffer's mbarrier replaces the barrier before the coupling sums; after the
// barrier that follows them (every read of the buffer done, every ring write
// of the previous step made), one bulk copy per delayed row refills the
// buffer for the next step while this step's transfer functions run. The
// wait is bounded as in sim_bulk_kernel.
// ---------------------------------------------------------------------------
template <int PB, int SPT, int RPT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
sim_tma_kernel(const __grid_constant__ SimArgs a)
{
    constexpr int TPR = PB / SPT;
    extern __shared__ __align__(128) float smem[];
    const TileDev tile = a.tiles[blockIdx.x];
    const GroupDev grp = a.groups[tile.group];
    const int N = a.N;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);        // first 16 bytes
    int* s_abort = reinterpret_cast<int*>(smem + 8);            // timeout flag of the CTA
    float* gbuf = smem + 32;                                    // [nnz][PB], 128-byte aligned
    const TileSmem sm = stage_tile<PB>(a, tile, grp, gbuf + (size_t)grp.nnz * PB);
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
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

    // thread 0 arms the phase of step mstep, then every thread issues its copies
    auto prefetch = [&](int64_t mstep) {
        if (threadIdx.x == 0) mbar_arm(mbar, step_bytes);
        if (mstep == a.withhold_step) return;   // failure-path test: nothing arrives
        const int slot_m = (int)(mstep % H);
        for (int e = threadIdx.x; e < grp.nnz; e += blockDim.x) {
            const uint32_t cd = sm.s_cd[e];
            const int d = (int)(cd >> 16);
            if (d == 0) continue;
            int sl = slot_m - d;
            sl += sl < 0 ? H : 0;
            bulk_g2s(gbuf + (size_t)e * PB, ring_cols + sl * slot_stride + (int64_t)(cd & 0xffffu) * grp.stride,
                     row_bytes, mbar);
        }
    };

    prefetch(a.n0);
    uint32_t par = 0u;   // parity of the phase being waited for
    for (int step = 0; step < a.n_chunk; ++step) {
        const int64_t n = a.n0 + step;
        const int slot_n = (int)(n % H);
        const int slot_w = slot_n + 1 == H ? 0 : slot_n + 1;
        if (mbar_wait_bounded(mbar, par, a.wait_limit)) {
            par ^= 1u;
        } else {
            *s_abort = 1;
            atomicOr(a.error, TVBX_DEVERR_TIMEOUT);
        }
        float cpl[SPT * RPT];
        coupling_sums<PB, SPT, RPT>(ts, N, gbuf, sm.s_w, sm.s_cd, sm.s_row, sm.s_mid, ring_cols + slot_n * slot_stride,
                                    grp.stride, cpl);
        __syncthreads();   // the buffer is consumed; the ring writes of E(n) are done and fenced
        if (*s_abort) break;
        if (step + 1 < a.n_chunk) prefetch(n + 1);
        advance_pairs<PB, SPT, RPT>(a, ts, sm.s_prm, tp, cpl, n, step, ring_cols + slot_w * slot_stride, grp.stride);
        fence_proxy_async_global();   // E(n+1) visible to the next bulk copies
    }
    if (*s_abort) {
        // let copies already in flight land before the CTA's shared memory is released
        mbar_wait_bounded(mbar, par, a.wait_limit);
    }
    store_pairs<SPT, RPT>(a, ts, tp);
}

// OU values of two sets advanced by one step with their own normals (per-set
// noise), out of line to keep it off the integration's register budget.
static __device__ __noinline__ float2 ou_advance2(const DevModel& m, uint64_t seed, uint32_t n, uint32_t k,
                                                  uint32_t p0, uint32_t p1, float2 OU)
{
    const float x0 = std_normal(seed, n, k, p0), x1 = std_normal(seed, n, k, p1);
    return make_float2(fmaf(m.ou_a, m.ou_mu - OU.x, fmaf(m.ou_b, x0, OU.x)),
                       fmaf(m.ou_a, m.ou_mu - OU.y, fmaf(m.ou_b, x1, OU.y)));
}

// ---------------------------------------------------------------------------
// Packed kernel: a thread owns two adjacent sets of RPT regions and integrates
// both with FP32x2 instructions (the two sets in the halves of each register
// pair; the same rounding as one set per thread, see model_device.cuh).
// Delayed rows are copied with 16-byte cp.async into one of two buffers: at
// step n, after the CTA barrier that makes step n's rows visible and ends
// every use of the other buffer, the rows of step n + 1 are requested into
// it, so one barrier per step suffices. The thread count is a multiple of
// the chunks per row, so each thread's (row, chunk) split is fixed.
// Needs the reduced transfer function (tau_e == tau_i).
// ---------------------------------------------------------------------------
template <int PB, int RPT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
sim_pack_kernel(const __grid_constant__ SimArgs a)
{
    constexpr int TPR = PB / 2;
    constexpr int CH = PB / 4;   // 16-byte chunks per row
    extern __shared__ __align__(128) float smem[];
    const TileDev tile = a.tiles[blockIdx.x];
    const GroupDev grp = a.groups[tile.group];
    const DevModel& m = a.m;
    const int N = a.N;
    float* gbuf0 = smem;                                        // [nnz][PB] x 2
    float* gbuf1 = gbuf0 + (size_t)grp.nnz * PB;
    const TileSmem sm = stage_tile<PB>(a, tile, grp, gbuf1 + (size_t)grp.nnz * PB);

    // the thread's sets qt, qt + 1 (lanes x, y) and regions kr + r kstride
    const int qt = (threadIdx.x % TPR) * 2;
    const int kr = threadIdx.x / TPR;
    const int kstride = blockDim.x / TPR;
    const int64_t col0 = grp.p_base + tile.q0;
    const bool act0 = qt < tile.nq, act1 = qt + 1 < tile.nq;
    const int64_t NP = (int64_t)N * a.P;
    PairV<float2> x[RPT];
    float2 ou[RPT], accE[RPT], accI[RPT];
    uint32_t pn[2];
    pn[0] = act0 ? (uint32_t)(a.p_offset + a.ext_index[col0 + qt]) : 0u;
    pn[1] = act1 ? (uint32_t)(a.p_offset + a.ext_index[col0 + qt + 1]) : 0u;
    Track<float2> trk = track_init<float2>();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int k = kr + r * kstride;
        float v[SV_ACC_I + 1][2];
#pragma unroll
        for (int c = 0; c <= SV_ACC_I; ++c)
#pragma unroll
            for (int l = 0; l < 2; ++l)
                v[c][l] = (k < N && (l ? act1 : act0)) ? a.state[c * NP + (int64_t)k * a.P + col0 + qt + l] : 0.0f;
        float cw[2][2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const bool in = k < N && (l ? act1 : act0);
            const int64_t o = (int64_t)k * a.P + col0 + qt + l;
            cw[0][l] = in ? a.state[SV_CWE * NP + o] : 0.0f;
            cw[1][l] = in ? a.state[SV_CWI * NP + o] : 0.0f;
        }
        x[r] = PairV<float2>{make_float2(v[SV_E][0], v[SV_E][1]),     make_float2(v[SV_I][0], v[SV_I][1]),
                             make_float2(v[SV_CEE][0], v[SV_CEE][1]), make_float2(v[SV_CEI][0], v[SV_CEI][1]),
                             make_float2(v[SV_CII][0], v[SV_CII][1]), make_float2(v[SV_WE][0], v[SV_WE][1]),
                             make_float2(v[SV_WI][0], v[SV_WI][1]),   make_float2(cw[0][0], cw[0][1]),
                             make_float2(cw[1][0], cw[1][1])};
        ou[r] = make_float2(v[SV_OU][0], v[SV_OU][1]);
        accE[r] = make_float2(v[SV_ACC_E][0], v[SV_ACC_E][1]);
        accI[r] = make_float2(v[SV_ACC_I][0], v[SV_ACC_I][1]);
    }

    const int H = grp.H;
    const int64_t slot_stride = (int64_t)N * grp.stride;
    float* ring_cols = grp.ring + tile.q0;
    const float inv_ts = 1.0f / (float)a.ts;
    // this thread's chunk c0 of rows e0, e0 + estep, ... (blockDim is a multiple of CH)
    const int c0 = threadIdx.x % CH, e0 = threadIdx.x / CH, estep = blockDim.x / CH;
    auto prefetch = [&](int64_t mstep, float* dst) {
        const int slot_m = (int)(mstep % H);
        for (int e = e0; e < grp.nnz; e += estep) {
            const uint32_t cd = sm.s_cd[e];
            const int d = (int)(cd >> 16);
            if (d == 0) continue;
            int sl = slot_m - d;
            sl += sl < 0 ? H : 0;
            cp_async16(dst + (size_t)e * PB + 4 * c0,
                       ring_cols + sl * slot_stride + (int64_t)(cd & 0xffffu) * grp.stride + 4 * c0);
        }
        cp_async_commit();
    };

    __syncthreads();
    prefetch(a.n0, gbuf0);
    for (int step = 0; step < a.n_chunk; ++step) {
        const int64_t n = a.n0 + step;
        const int slot_n = (int)(n % H);
        const int slot_w = slot_n + 1 == H ? 0 : slot_n + 1;
        const float* gbuf = (step & 1) ? gbuf1 : gbuf0;
        cp_async_wait_all();
        __syncthreads();   // step n's rows visible; every read of the other buffer and every write of E(n) done
        if (step + 1 < a.n_chunk) prefetch(n + 1, (step & 1) ? gbuf0 : gbuf1);
        const float* ring_n = ring_cols + slot_n * slot_stride;
        float* ring_w = ring_cols + slot_w * slot_stride;
        const bool sample_now = ((n + 1) % a.ts) == 0;
        const int64_t t = (n + 1) / a.ts - 1;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int k = kr + r * kstride;
            if (k >= N) continue;
            // coupling sum_j u_kj E_j(n - d_kj) in CSR order, both sets at once
            float2 cpl = make_float2(0.0f, 0.0f);
            const int e_mid = sm.s_mid[k], e_end = sm.s_row[k + 1];
            int e = sm.s_row[k];
#pragma unroll 4
            for (; e < e_mid; ++e)
                cpl = vfma(vbc<float2>(sm.s_w[e]), *reinterpret_cast<const float2*>(gbuf + (size_t)e * PB + qt), cpl);
            for (; e < e_end; ++e)   // zero delay: E_j(n), written last step
                cpl = vfma(vbc<float2>(sm.s_w[e]),
                           *reinterpret_cast<const float2*>(ring_n + (int64_t)(sm.s_cd[e] & 0xffffu) * grp.stride + qt),
                           cpl);
            ParamsV<float2> sp;
            float2* f = reinterpret_cast<float2*>(&sp);
#pragma unroll
            for (int c = 0; c < 11; ++c) f[c] = *reinterpret_cast<const float2*>(sm.s_prm + c * PB + qt);
            const float2 OU = a.noise_per_set ? ou[r] : vbc<float2>(a.ou_table[(int64_t)step * N + k]);
            pair_step(m, sp, x[r], cpl, OU, trk);
            if (a.noise_per_set) ou[r] = ou_advance2(m, a.seed, (uint32_t)n, (uint32_t)k, pn[0], pn[1], OU);
            float* wr = ring_w + (int64_t)k * grp.stride + qt;
            if (act1) *reinterpret_cast<float2*>(wr) = x[r].E;
            else if (act0) wr[0] = x[r].E.x;
            accE[r] = vadd(accE[r], x[r].E);
            accI[r] = vadd(accI[r], x[r].I);
            if (sample_now) {
                if (t < a.T) {
                    const float2 xE = vmul(accE[r], vbc<float2>(inv_ts)), xI = vmul(accI[r], vbc<float2>(inv_ts));
                    const int64_t o = (int64_t)k * a.P + col0 + qt;
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        if (!(l ? act1 : act0)) continue;
                        const int64_t so = series_index(a.sl, t, k, col0 + qt + l);
                        a.series[so] = lane(xE, l);
                        if (a.series_i) a.series_i[so] = lane(xI, l);
                        if (t >= a.transient) {
                            float* st = a.state + o + l;
                            float sE = st[SV_SUM_E * NP], cE = st[SV_CMP_E * NP];
                            float sI = st[SV_SUM_I * NP], cI = st[SV_CMP_I * NP];
                            kahan_add(sE, cE, lane(xE, l));
                            kahan_add(sI, cI, lane(xI, l));
                            st[SV_SUM_E * NP] = sE;
                            st[SV_CMP_E * NP] = cE;
                            st[SV_SUM_I * NP] = sI;
                            st[SV_CMP_I * NP] = cI;
                        }
                    }
                }
                accE[r] = make_float2(0.0f, 0.0f);
                accI[r] = make_float2(0.0f, 0.0f);
            }
        }
    }
    cp_async_wait_all();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int k = kr + r * kstride;
        if (k >= N) continue;
        const float2 v[SV_ACC_I + 1] = {x[r].E, x[r].I, x[r].Cee, x[r].Cei, x[r].Cii, x[r].We, x[r].Wi,
                                        ou[r], accE[r], accI[r]};
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            if (!(l ? act1 : act0)) continue;
#pragma unroll
            for (int c = 0; c <= SV_ACC_I; ++c) a.state[c * NP + (int64_t)k * a.P + col0 + qt + l] = lane(v[c], l);
            a.state[SV_CWE * NP + (int64_t)k * a.P + col0 + qt + l] = lane(x[r].cWe, l);
            a.state[SV_CWI * NP + (int64_t)k * a.P + col0 + qt + l] = lane(x[r].cWi, l);
        }
    }
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const uint32_t fl = track_flags(m, trk, l);
        if ((l ? act1 : act0) && fl) atomicOr(a.status + col0 + qt + l, fl);
    }
}

// ---------------------------------------------------------------------------
// Variants: (kernel, sets per CTA, sets per thread, regions per thread, max
// threads, min CTAs per SM).
// ---------------------------------------------------------------------------
struct FastVariant {
    int bulk, pb, spt, rpt, maxt, minb;   // 0 cp.async, 1 TMA bulk x 2 buffers, 2 packed FP32x2 with
                                          // cp.async x 2 buffers, 3 TMA bulk x 1 buffer, 4 cp.async x 2
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
    {2, 12, 2, 1, 512, 1},   // 8: packed FP32x2, cp.async, two buffers, 12 sets, 2 x 1 (128 registers)
    {2, 16, 2, 1, 576, 1},   // 9: packed, 16 sets, 2 x 1 (96 registers)
    {2, 8, 2, 1, 288, 1},    // 10: packed, 8 sets, 2 x 1 (168 registers)
    {2, 16, 2, 2, 320, 1},   // 11: packed, 16 sets, 2 x 2 (168 registers)
    {3, 32, 4, 1, 576, 1},   // 12: TMA bulk, one buffer, 32 sets, 4 x 1
    {3, 16, 2, 1, 576, 1},   // 13: TMA bulk, one buffer, 16 sets, 2 x 1
    {3, 32, 2, 2, 576, 1},   // 14: TMA bulk, one buffer, 32 sets, 2 x 2
    {4, 16, 2, 1, 576, 1},   // 15: cp.async, two buffers, 16 sets, 2 x 1
    {4, 16, 1, 2, 576, 1},   // 16: cp.async, two buffers, 16 sets, 1 x 2
};
constexpr int kNumFast = (int)(sizeof kFast / sizeof kFast[0]);

static size_t tail_bytes(int N, int nnz, int pb)
{
    return 8 * (size_t)nnz + 4 * (size_t)(2 * N + 1) + 16 + 4 * 11 * (size_t)pb;   // + alignment of the parameters
}

size_t sim_fast_smem_bytes(int variant, int N, int nnz)
{
    const FastVariant& v = kFast[variant];
    const size_t buf = sizeof(float) * (size_t)nnz * v.pb;
    if (v.bulk == 3) return 128 + buf + tail_bytes(N, nnz, v.pb);
    if (v.bulk == 2 || v.bulk == 4) return 2 * buf + tail_bytes(N, nnz, v.pb);
    return v.bulk ? 128 + 2 * buf + tail_bytes(N, nnz, v.pb) : buf + tail_bytes(N, nnz, v.pb);
}

bool sim_fast_fits(int variant, int N, int nnz_max)
{
    if (variant < 0 || variant >= kNumFast) return false;
    const FastVariant& v = kFast[variant];
    const int kstride = (N + v.rpt - 1) / v.rpt;
    if (kstride * (v.pb / v.spt) > v.maxt) return false;
    if ((v.bulk == 1 || v.bulk == 3) && (size_t)nnz_max * v.pb * sizeof(float) >= (1u << 20))
        return false;   // mbarrier tx-count range
    if (v.bulk == 2 && (kstride * (v.pb / v.spt)) % (v.pb / 4) != 0) return false;   // fixed chunk per thread
    return sim_fast_smem_bytes(variant, N, nnz_max) * v.minb <= 220 * 1024;
}

int sim_fast_pb(int variant) { return kFast[variant].pb; }
bool sim_fast_packed(int variant) { return variant >= 0 && variant < kNumFast && kFast[variant].bulk == 2; }
int sim_fast_variants() { return kNumFast; }

template <int BULK, int PB, int SPT, int RPT, int MAXT, int MINB>
static cudaError_t launch_fast(const SimArgs& a, int variant, int32_t n_tiles, int nnz_max, cudaStream_t s)
{
    const int kstride = (a.N + RPT - 1) / RPT;
    const int threads = kstride * (PB / SPT);
    const size_t smem = sim_fast_smem_bytes(variant, a.N, nnz_max);
    void (*kern)(SimArgs);
    if constexpr (BULK == 4) kern = sim_fast_kernel<PB, SPT, RPT, MAXT, MINB, true>;
    else if constexpr (BULK == 3) kern = sim_tma_kernel<PB, SPT, RPT, MAXT>;
    else if constexpr (BULK == 2) kern = sim_pack_kernel<PB, RPT, MAXT>;
    else if constexpr (BULK == 1) kern = sim_bulk_kernel<PB, SPT, RPT, MAXT, MINB>;
    else kern = sim_fast_kernel<PB, SPT, RPT, MAXT, MINB, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // all of the unified L1 as shared memory, so that MINB CTAs fit on an SM
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
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
    case 8: return launch_fast<2, 12, 2, 1, 512, 1>(a, variant, n_tiles, nnz_max, s);
    case 9: return launch_fast<2, 16, 2, 1, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 10: return launch_fast<2, 8, 2, 1, 288, 1>(a, variant, n_tiles, nnz_max, s);
    case 11: return launch_fast<2, 16, 2, 2, 320, 1>(a, variant, n_tiles, nnz_max, s);
    case 12: return launch_fast<3, 32, 4, 1, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 13: return launch_fast<3, 16, 2, 1, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 14: return launch_fast<3, 32, 2, 2, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 15: return launch_fast<4, 16, 2, 1, 576, 1>(a, variant, n_tiles, nnz_max, s);
    case 16: return launch_fast<4, 16, 1, 2, 576, 1>(a, variant, n_tiles, nnz_max, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvbx

// Per-thread pieces shared by the tiled simulation kernels: a thread owns SPT
// adjacent sets and RPT regions of its CTA's tile and keeps their state in
// registers for a whole chunk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "model_device.cuh"

namespace tvbx {

template <int SPT> struct VecT;
template <> struct VecT<1> { using T = float; };
template <> struct VecT<2> { using T = float2; };
template <> struct VecT<4> { using T = float4; };

static __device__ __forceinline__ float vget(const float& v, int) { return v; }
static __device__ __forceinline__ float vget(const float2& v, int i) { return i == 0 ? v.x : v.y; }
static __device__ __forceinline__ float vget(const float4& v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Registers of one thread: SPT x RPT pairs.
template <int SPT, int RPT>
struct ThreadPairs {
    PairState x[SPT * RPT];
    float ou[SPT * RPT], accE[SPT * RPT], accI[SPT * RPT];
    uint32_t pn[SPT];     // noise counter of each set (per-set noise)
    bool act[SPT];        // set exists in the tile
    Track<float> trk[SPT];  // status events gathered during the chunk
};

// Tile geometry of the calling thread.
struct ThreadSlot {
    int qt;       // first set of the thread within the tile
    int kr;       // first region
    int kstride;  // region stride
    int64_t col0; // internal index of set 0 of the tile
};

// Stage the tile's set parameters into shared memory s_prm[11][PB] (PB = 0:
// the runtime width pb_rt).
template <int PB>
static __device__ __forceinline__ void stage_set_params(const SimArgs& a, const TileDev& tile, const GroupDev& grp,
                                                        float* s_prm, int pb_rt = 0)
{
    const int pbs = PB > 0 ? PB : pb_rt;
    for (int q = threadIdx.x; q < pbs; q += blockDim.x) {
        SetParams v{};
        if (q < tile.nq) v = load_set_params(a.prm, a.P, grp.p_base + tile.q0 + q);
        const float* f = reinterpret_cast<const float*>(&v);
        for (int c = 0; c < 11; ++c) s_prm[c * pbs + q] = f[c];
    }
}

template <int SPT, int RPT>
static __device__ __forceinline__ void load_pairs(const SimArgs& a, const TileDev& tile, const ThreadSlot& ts,
                                                  ThreadPairs<SPT, RPT>& tp)
{
    const int N = a.N;
    const int64_t NP = (int64_t)N * a.P;
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
        tp.act[s] = ts.qt + s < tile.nq;
        tp.pn[s] = tp.act[s] ? (uint32_t)(a.p_offset + a.ext_index[ts.col0 + ts.qt + s]) : 0u;
        tp.trk[s] = track_init<float>();
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int k = ts.kr + r * ts.kstride;
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int i = r * SPT + s;
            if (tp.act[s] && k < N) {
                const int64_t o = (int64_t)k * a.P + ts.col0 + ts.qt + s;
                tp.x[i] = PairState{a.state[SV_E * NP + o],   a.state[SV_I * NP + o],   a.state[SV_CEE * NP + o],
                                    a.state[SV_CEI * NP + o], a.state[SV_CII * NP + o], a.state[SV_WE * NP + o],
                                    a.state[SV_WI * NP + o],  a.state[SV_CWE * NP + o], a.state[SV_CWI * NP + o]};
                tp.ou[i] = a.state[SV_OU * NP + o];
                tp.accE[i] = a.state[SV_ACC_E * NP + o];
                tp.accI[i] = a.state[SV_ACC_I * NP + o];
            } else {
                tp.x[i] = PairState{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                tp.ou[i] = tp.accE[i] = tp.accI[i] = 0.0f;
            }
        }
    }
}

template <int SPT, int RPT>
static __device__ __forceinline__ void store_pairs(const SimArgs& a, const ThreadSlot& ts,
                                                   const ThreadPairs<SPT, RPT>& tp)
{
    const int N = a.N;
    const int64_t NP = (int64_t)N * a.P;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int k = ts.kr + r * ts.kstride;
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int i = r * SPT + s;
            if (tp.act[s] && k < N) {
                const int64_t o = (int64_t)k * a.P + ts.col0 + ts.qt + s;
                a.state[SV_E * NP + o] = tp.x[i].E;
                a.state[SV_I * NP + o] = tp.x[i].I;
                a.state[SV_CEE * NP + o] = tp.x[i].Cee;
                a.state[SV_CEI * NP + o] = tp.x[i].Cei;
                a.state[SV_CII * NP + o] = tp.x[i].Cii;
                a.state[SV_WE * NP + o] = tp.x[i].We;
                a.state[SV_WI * NP + o] = tp.x[i].Wi;
                a.state[SV_CWE * NP + o] = tp.x[i].cWe;
                a.state[SV_CWI * NP + o] = tp.x[i].cWi;
                a.state[SV_OU * NP + o] = tp.ou[i];
                a.state[SV_ACC_E * NP + o] = tp.accE[i];
                a.state[SV_ACC_I * NP + o] = tp.accI[i];
            }
        }
    }
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
        const uint32_t f = track_flags(a.m, tp.trk[s], 0);
        if (tp.act[s] && f) atomicOr(a.status + ts.col0 + ts.qt + s, f);
    }
}

// Coupling sums sum_j u_kj E_j(n - d_kj) of the thread's pairs: delayed
// entries from the gathered rows gbuf[e][PB], zero-delay entries (the tail of
// each row) straight from ring slot n.
template <int PB, int SPT, int RPT>
static __device__ __forceinline__ void coupling_sums(const ThreadSlot& ts, int N, const float* gbuf, const float* s_w,
                                                     const uint32_t* s_cd, const int* s_row, const int* s_mid,
                                                     const float* ring_slot_n, int64_t row_stride, float* cpl)
{
    using V = typename VecT<SPT>::T;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int k = ts.kr + r * ts.kstride;
        float acc[SPT];
#pragma unroll
        for (int s = 0; s < SPT; ++s) acc[s] = 0.0f;
        if (k < N) {
            const int e_mid = s_mid[k];
            const int e_end = s_row[k + 1];
            int e = s_row[k];
#pragma unroll 4
            for (; e < e_mid; ++e) {
                const float w = s_w[e];
                const V v = *reinterpret_cast<const V*>(gbuf + (size_t)e * PB + ts.qt);
#pragma unroll
                for (int s = 0; s < SPT; ++s) acc[s] = fmaf(w, vget(v, s), acc[s]);
            }
            for (; e < e_end; ++e) {   // zero delay: E_j(n), written last step
                const float w = s_w[e];
                const float* src = ring_slot_n + (int64_t)(s_cd[e] & 0xffffu) * row_stride + ts.qt;
#pragma unroll
                for (int s = 0; s < SPT; ++s) acc[s] = fmaf(w, src[s], acc[s]);
            }
        }
#pragma unroll
        for (int s = 0; s < SPT; ++s) cpl[r * SPT + s] = acc[s];
    }
}

// OU value of one set advanced by one step with its own normal (per-set
// noise), out of line to keep it off the integration's register budget.
static __device__ __noinline__ float ou_advance(const DevModel& m, uint64_t seed, uint32_t n, uint32_t k, uint32_t p,
                                                float OU)
{
    const float xi = std_normal(seed, n, k, p);
    return fmaf(m.ou_a, m.ou_mu - OU, fmaf(m.ou_b, xi, OU));
}

// One Euler step of the thread's pairs, the ring write of E(n+1) and the
// temporal average. ring_slot_w points at slot (n+1) mod H, column 0 of the
// tile; s_prm is [11][PB] (PB = 0: the runtime width pb_rt).
template <int PB, int SPT, int RPT>
static __device__ __forceinline__ void advance_pairs(const SimArgs& a, const ThreadSlot& ts, const float* s_prm,
                                                     ThreadPairs<SPT, RPT>& tp, const float* cpl, int64_t n,
                                                     int step, float* ring_slot_w, int64_t row_stride, int pb_rt = 0)
{
    const int pbs = PB > 0 ? PB : pb_rt;
    const DevModel& m = a.m;
    const int N = a.N;
    const int64_t NP = (int64_t)N * a.P;
    const bool sample_now = ((n + 1) % a.ts) == 0;
    const int64_t t = (n + 1) / a.ts - 1;
    const float inv_ts = 1.0f / (float)a.ts;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int k = ts.kr + r * ts.kstride;
        // the shared OU value of region k at this step (one load for the thread's sets)
        const float ou_k = (!a.noise_per_set && k < N) ? a.ou_table[(int64_t)step * N + k] : 0.0f;
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int i = r * SPT + s;
            if (!(tp.act[s] && k < N)) continue;
            const float OU = a.noise_per_set ? tp.ou[i] : ou_k;
            SetParams spv;
            float* f = reinterpret_cast<float*>(&spv);
#pragma unroll
            for (int c = 0; c < 11; ++c) f[c] = s_prm[c * pbs + ts.qt + s];
            pair_step(m, spv, tp.x[i], cpl[i], OU, tp.trk[s]);
            if (a.noise_per_set) tp.ou[i] = ou_advance(m, a.seed, (uint32_t)n, (uint32_t)k, tp.pn[s], OU);
            ring_slot_w[(int64_t)k * row_stride + ts.qt + s] = tp.x[i].E;
            tp.accE[i] += tp.x[i].E;
            tp.accI[i] += tp.x[i].I;
            if (sample_now) {
                if (t < a.T) {
                    const float xE = tp.accE[i] * inv_ts, xI = tp.accI[i] * inv_ts;
                    const int64_t o = (int64_t)k * a.P + ts.col0 + ts.qt + s;
                    const int64_t so = series_index(a.sl, t, k, ts.col0 + ts.qt + s);
                    a.series[so] = xE;
                    if (a.series_i) a.series_i[so] = xI;
                    if (t >= a.transient) {
                        float sE = a.state[SV_SUM_E * NP + o], cE = a.state[SV_CMP_E * NP + o];
                        float sI = a.state[SV_SUM_I * NP + o], cI = a.state[SV_CMP_I * NP + o];
                        kahan_add(sE, cE, xE);
                        kahan_add(sI, cI, xI);
                        a.state[SV_SUM_E * NP + o] = sE;
                        a.state[SV_CMP_E * NP + o] = cE;
                        a.state[SV_SUM_I * NP + o] = sI;
                        a.state[SV_CMP_I * NP + o] = cI;
                    }
                }
                tp.accE[i] = 0.0f;
                tp.accI[i] = 0.0f;
            }
        }
    }
}

}  // namespace tvbx

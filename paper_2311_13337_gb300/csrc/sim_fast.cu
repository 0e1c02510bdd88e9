// Prefetching simulation kernel of the tvbx engine (arXiv 2311.13337, the
// lock-step integration of Eq. 1-5 with forward Euler).
//
// A CTA owns PB sets of one speed group and all N regions of each. A thread
// owns SPT adjacent sets and RPT regions (k = t / (PB/SPT) + i * kstride),
// with their state in registers across the whole chunk.
//
// Delays are at least one step for every nonzero weight with a positive
// tract length, so the values the coupling needs at step n + 1,
// E_j(n + 1 - d_kj), are all in the ring buffer when step n begins. The CTA
// issues the whole gather of step n + 1 with 16-byte cp.async copies (one
// PB-float row segment per delayed weight, L2 only) into a shared buffer
// right after it has consumed the buffer for step n; the copies complete
// while step n's transfer functions are evaluated. Zero-delay entries
// (d = 0) sit at the end of each CSR row and read E_j(n) directly after the
// step barrier.
//
// In the coupling sum, the SPT sets of a thread share one broadcast weight
// load and one vector load of the gathered row. CSR rows start at an index
// of the same parity as their region (a zero-weight self entry pads when
// needed) so that the rows read at the same time by the two halves of a warp
// fall in opposite halves of the shared-memory banks.
//
// Shared memory: gather buffer [nnz][PB] floats, weights, CSR (j, d), row
// starts and the start of each row's zero-delay entries.

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "model_device.cuh"

namespace tvbx {

static __device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
static __device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

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

template <int PB, int SPT, int RPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
sim_fast_kernel(const __grid_constant__ SimArgs a)
{
    using V = typename VecT<SPT>::T;
    constexpr int TPR = PB / SPT;  // threads per region row
    constexpr int NP_T = SPT * RPT; // pairs per thread
    extern __shared__ __align__(16) float smem[];
    const TileDev tile = a.tiles[blockIdx.x];
    const GroupDev grp = a.groups[tile.group];
    const DevModel& m = a.m;
    const int N = a.N;
    const int P = a.P;
    const int nnz = grp.nnz;
    float* gbuf = smem;                                                    // [nnz][PB]
    float* s_w = gbuf + (size_t)nnz * PB;                                  // [nnz]
    uint32_t* s_cd = reinterpret_cast<uint32_t*>(s_w + nnz);               // [nnz] (d << 16) | j
    int* s_row = reinterpret_cast<int*>(s_cd + nnz);                       // [N + 1]
    int* s_mid = s_row + N + 1;                                            // [N] first zero-delay entry
    float* s_prm = reinterpret_cast<float*>(s_mid + N);                    // [11][PB] set parameters
    for (int q = threadIdx.x; q < PB; q += blockDim.x) {
        SetParams v{};
        if (q < tile.nq) v = load_set_params(a.prm, P, grp.p_base + tile.q0 + q);
        const float* f = reinterpret_cast<const float*>(&v);
        for (int c = 0; c < 11; ++c) s_prm[c * PB + q] = f[c];
    }
    for (int i = threadIdx.x; i < nnz; i += blockDim.x) {
        s_cd[i] = grp.col_dly[i];
        s_w[i] = grp.w[i];
    }
    for (int i = threadIdx.x; i <= N; i += blockDim.x) s_row[i] = grp.row_ptr[i];
    for (int i = threadIdx.x; i < N; i += blockDim.x) s_mid[i] = grp.row_mid[i];

    const int kstride = blockDim.x / TPR;
    const int qt = (threadIdx.x % TPR) * SPT;   // first set of this thread in the tile
    const int kr = threadIdx.x / TPR;
    const int64_t NP = (int64_t)N * P;
    uint32_t pn[SPT];
    bool act[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
        act[s] = qt + s < tile.nq;
        pn[s] = act[s] ? (uint32_t)(a.p_offset + a.ext_index[grp.p_base + tile.q0 + qt + s]) : 0u;
    }
    PairState x[NP_T];
    float ou[NP_T], accE[NP_T], accI[NP_T];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int k = kr + r * kstride;
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int i = r * SPT + s;
            if (act[s] && k < N) {
                const int64_t o = (int64_t)k * P + grp.p_base + tile.q0 + qt + s;
                x[i] = PairState{a.state[SV_E * NP + o], a.state[SV_I * NP + o], a.state[SV_CEE * NP + o],
                                 a.state[SV_CEI * NP + o], a.state[SV_CII * NP + o], a.state[SV_WE * NP + o],
                                 a.state[SV_WI * NP + o]};
                ou[i] = a.state[SV_OU * NP + o];
                accE[i] = a.state[SV_ACC_E * NP + o];
                accI[i] = a.state[SV_ACC_I * NP + o];
            } else {
                x[i] = PairState{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                ou[i] = accE[i] = accI[i] = 0.0f;
            }
        }
    }
    __syncthreads();

    const int H = grp.H;
    const int64_t slot_stride = (int64_t)N * grp.stride;
    float* ring_cols = grp.ring + tile.q0;
    constexpr int CH = PB / 4;  // 16-byte chunks per row segment

    // gather of step `mstep`'s delayed values (d >= 1) into gbuf
    auto prefetch = [&](int64_t mstep) {
        const int slot_m = (int)(mstep % H);
        for (int idx = threadIdx.x; idx < nnz * CH; idx += blockDim.x) {
            const int e = idx / CH, c = idx - e * CH;
            const uint32_t cd = s_cd[e];
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
    uint32_t flags[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) flags[s] = 0u;
    const float inv_ts = 1.0f / (float)a.ts;
    for (int step = 0; step < a.n_chunk; ++step) {
        const int64_t n = a.n0 + step;
        const int slot_n = (int)(n % H);
        const int slot_w = slot_n + 1 == H ? 0 : slot_n + 1;
        cp_async_wait_all();
        __syncthreads();
        float cpl[NP_T];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int k = kr + r * kstride;
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
                    const V v = *reinterpret_cast<const V*>(gbuf + (size_t)e * PB + qt);
#pragma unroll
                    for (int s = 0; s < SPT; ++s) acc[s] = fmaf(w, vget(v, s), acc[s]);
                }
                for (; e < e_end; ++e) {   // zero delay: E_j(n), written last step
                    const float w = s_w[e];
                    const float* src = ring_cols + slot_n * slot_stride + (int64_t)(s_cd[e] & 0xffffu) * grp.stride + qt;
#pragma unroll
                    for (int s = 0; s < SPT; ++s) acc[s] = fmaf(w, src[s], acc[s]);
                }
            }
#pragma unroll
            for (int s = 0; s < SPT; ++s) cpl[r * SPT + s] = acc[s];
        }
        __syncthreads();
        if (step + 1 < a.n_chunk) prefetch(n + 1);

        const bool sample_now = ((n + 1) % a.ts) == 0;
        const int64_t t = (n + 1) / a.ts - 1;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int k = kr + r * kstride;
#pragma unroll
            for (int s = 0; s < SPT; ++s) {
                const int i = r * SPT + s;
                if (!(act[s] && k < N)) continue;
                const float OU = a.noise_per_set ? ou[i] : a.ou_table[(int64_t)step * N + k];
                SetParams spv;
                float* f = reinterpret_cast<float*>(&spv);
#pragma unroll
                for (int c = 0; c < 11; ++c) f[c] = s_prm[c * PB + qt + s];
                euler_step(m, spv, x[i], cpl[i], OU, flags[s]);
                if (a.noise_per_set) {
                    const float xi = std_normal(a.seed, (uint32_t)n, (uint32_t)k, pn[s]);
                    ou[i] = fmaf(m.ou_a, m.ou_mu - OU, fmaf(m.ou_b, xi, OU));
                }
                ring_cols[slot_w * slot_stride + (int64_t)k * grp.stride + qt + s] = x[i].E;
                accE[i] += x[i].E;
                accI[i] += x[i].I;
                if (sample_now) {
                    if (t < a.T) {
                        const float xE = accE[i] * inv_ts, xI = accI[i] * inv_ts;
                        const int64_t o = (int64_t)k * P + grp.p_base + tile.q0 + qt + s;
                        a.series[t * NP + o] = xE;
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
                    accE[i] = 0.0f;
                    accI[i] = 0.0f;
                }
            }
        }
    }
    cp_async_wait_all();

#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int k = kr + r * kstride;
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
            const int i = r * SPT + s;
            if (act[s] && k < N) {
                const int64_t o = (int64_t)k * P + grp.p_base + tile.q0 + qt + s;
                a.state[SV_E * NP + o] = x[i].E;
                a.state[SV_I * NP + o] = x[i].I;
                a.state[SV_CEE * NP + o] = x[i].Cee;
                a.state[SV_CEI * NP + o] = x[i].Cei;
                a.state[SV_CII * NP + o] = x[i].Cii;
                a.state[SV_WE * NP + o] = x[i].We;
                a.state[SV_WI * NP + o] = x[i].Wi;
                a.state[SV_OU * NP + o] = ou[i];
                a.state[SV_ACC_E * NP + o] = accE[i];
                a.state[SV_ACC_I * NP + o] = accI[i];
            }
        }
    }
#pragma unroll
    for (int s = 0; s < SPT; ++s)
        if (act[s] && flags[s]) atomicOr(a.status + grp.p_base + tile.q0 + qt + s, flags[s]);
}

// ---------------------------------------------------------------------------
// Variants: (sets per CTA, sets per thread, regions per thread, max threads,
// min CTAs per SM).
// ---------------------------------------------------------------------------
struct FastVariant {
    int pb, spt, rpt, maxt, minb;
};
static const FastVariant kFast[] = {
    {16, 2, 1, 576, 1},   // 0: 16 sets, 2 sets x 1 region per thread
    {32, 4, 1, 576, 1},   // 1: 32 sets, 4 sets x 1 region per thread
    {16, 1, 2, 576, 1},   // 2: 16 sets, 1 set x 2 regions per thread
    {16, 2, 2, 320, 1},   // 3: 16 sets, 2 sets x 2 regions per thread
};
constexpr int kNumFast = (int)(sizeof kFast / sizeof kFast[0]);

size_t sim_fast_smem_bytes(int N, int nnz, int pb)
{
    return sizeof(float) * (size_t)nnz * pb + 8 * (size_t)nnz + 4 * (size_t)(2 * N + 1) + 4 * 11 * (size_t)pb;
}

bool sim_fast_fits(int variant, int N, int nnz_max)
{
    if (variant < 0 || variant >= kNumFast) return false;
    const FastVariant& v = kFast[variant];
    const int kstride = (N + v.rpt - 1) / v.rpt;
    if (kstride * (v.pb / v.spt) > v.maxt) return false;
    return sim_fast_smem_bytes(N, nnz_max, v.pb) * v.minb <= 220 * 1024;
}

int sim_fast_pb(int variant) { return kFast[variant].pb; }
int sim_fast_variants() { return kNumFast; }

template <int PB, int SPT, int RPT, int MAXT, int MINB>
static cudaError_t launch_fast(const SimArgs& a, int32_t n_tiles, int nnz_max, cudaStream_t s)
{
    const int kstride = (a.N + RPT - 1) / RPT;
    const int threads = kstride * (PB / SPT);
    const size_t smem = sim_fast_smem_bytes(a.N, nnz_max, PB);
    cudaError_t e = cudaFuncSetAttribute(sim_fast_kernel<PB, SPT, RPT, MAXT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    sim_fast_kernel<PB, SPT, RPT, MAXT, MINB><<<n_tiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sim_fast(const SimArgs& a, int variant, int32_t n_tiles, int nnz_max, cudaStream_t s)
{
    if (n_tiles <= 0 || a.n_chunk <= 0) return cudaSuccess;
    switch (variant) {
    case 0: return launch_fast<16, 2, 1, 576, 1>(a, n_tiles, nnz_max, s);
    case 1: return launch_fast<32, 4, 1, 576, 1>(a, n_tiles, nnz_max, s);
    case 2: return launch_fast<16, 1, 2, 576, 1>(a, n_tiles, nnz_max, s);
    case 3: return launch_fast<16, 2, 2, 320, 1>(a, n_tiles, nnz_max, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvbx

// Prefetching simulation kernel of the tvbx engine (arXiv 2311.13337, the
// lock-step integration of Eq. 1-5 with forward Euler).
//
// A CTA owns PB sets of one speed group and all N regions of each. Thread t
// handles set q = t % PB and regions k = t / PB + i * (blockDim / PB), i < R,
// with their state in registers across the whole chunk.
//
// Delays are at least one step for every nonzero weight with a positive
// tract length, so the values the coupling needs at step n + 1,
// E_j(n + 1 - d_kj), are all in the ring buffer when step n begins. The CTA
// therefore issues the whole gather of step n + 1 with 16-byte cp.async
// copies (one PB-float row segment per nonzero weight, L2 only) into a shared
// buffer right after it has consumed the buffer for step n, and the copies
// complete while step n's transfer functions are evaluated. Zero-delay
// entries (d = 0) read E_j(n) directly after the step barrier.
//
// Shared memory: gather buffer [nnz][PB] floats, CSR (j, d) and weights.

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

template <int PB, int R, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
sim_fast_kernel(const __grid_constant__ SimArgs a)
{
    extern __shared__ __align__(16) float smem[];
    const TileDev tile = a.tiles[blockIdx.x];
    const GroupDev grp = a.groups[tile.group];
    const DevModel& m = a.m;
    const int N = a.N;
    const int P = a.P;
    const int nnz = grp.nnz;
    float* gbuf = smem;                                                   // [nnz][PB]
    uint32_t* s_cd = reinterpret_cast<uint32_t*>(gbuf + (size_t)nnz * PB); // [nnz] (d << 16) | j
    float* s_w = reinterpret_cast<float*>(s_cd + nnz);                    // [nnz]
    int* s_row = reinterpret_cast<int*>(s_w + nnz);                       // [N + 1]
    for (int i = threadIdx.x; i < nnz; i += blockDim.x) {
        s_cd[i] = grp.col_dly[i];
        s_w[i] = grp.w[i];
    }
    for (int i = threadIdx.x; i <= N; i += blockDim.x) s_row[i] = grp.row_ptr[i];

    const int kstride = blockDim.x / PB;
    const int q = threadIdx.x % PB;
    const int kr = threadIdx.x / PB;
    const bool active = q < tile.nq;
    const int qg = tile.q0 + q;
    const int p = grp.p_base + qg;
    const int64_t NP = (int64_t)N * P;
    SetParams sp{};
    uint32_t pn = 0u;
    if (active) {
        sp = load_set_params(a.prm, P, p);
        pn = (uint32_t)(a.p_offset + a.ext_index[p]);
    }
    PairState x[R];
    float ou[R], accE[R], accI[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int k = kr + i * kstride;
        if (active && k < N) {
            const int64_t o = (int64_t)k * P + p;
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
    uint32_t flags = 0u;
    const float inv_ts = 1.0f / (float)a.ts;
    for (int s = 0; s < a.n_chunk; ++s) {
        const int64_t n = a.n0 + s;
        const int slot_n = (int)(n % H);
        const int slot_w = slot_n + 1 == H ? 0 : slot_n + 1;
        cp_async_wait_all();
        __syncthreads();
        float cpl[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int k = kr + i * kstride;
            float acc = 0.0f;
            if (k < N) {
                const int e1 = s_row[k + 1];
                for (int e = s_row[k]; e < e1; ++e) {
                    const uint32_t cd = s_cd[e];
                    const float v = (cd >> 16) ? gbuf[(size_t)e * PB + q]
                                               : ring_cols[slot_n * slot_stride + (int64_t)(cd & 0xffffu) * grp.stride + q];
                    acc = fmaf(s_w[e], v, acc);
                }
            }
            cpl[i] = acc;
        }
        __syncthreads();
        if (s + 1 < a.n_chunk) prefetch(n + 1);

        const bool sample_now = ((n + 1) % a.ts) == 0;
        const int64_t t = (n + 1) / a.ts - 1;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int k = kr + i * kstride;
            if (!(active && k < N)) continue;
            const float OU = a.noise_per_set ? ou[i] : a.ou_table[(int64_t)s * N + k];
            euler_step(m, sp, x[i], cpl[i], OU, flags);
            if (a.noise_per_set) {
                const float xi = std_normal(a.seed, (uint32_t)n, (uint32_t)k, pn);
                ou[i] = fmaf(m.ou_a, m.ou_mu - OU, fmaf(m.ou_b, xi, OU));
            }
            ring_cols[slot_w * slot_stride + (int64_t)k * grp.stride + q] = x[i].E;
            accE[i] += x[i].E;
            accI[i] += x[i].I;
            if (sample_now) {
                if (t < a.T) {
                    const float xE = accE[i] * inv_ts, xI = accI[i] * inv_ts;
                    const int64_t o = (int64_t)k * P + p;
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
    cp_async_wait_all();

#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int k = kr + i * kstride;
        if (active && k < N) {
            const int64_t o = (int64_t)k * P + p;
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
    if (active && flags) atomicOr(a.status + p, flags);
}

// ---------------------------------------------------------------------------
// Variants: (sets per CTA, regions per thread, max threads, min CTAs per SM).
// ---------------------------------------------------------------------------
struct FastVariant {
    int pb, r, maxt, minb;
};
static const FastVariant kFast[] = {{16, 4, 288, 2}, {32, 4, 576, 1}, {16, 2, 544, 1}, {16, 4, 288, 1}};
constexpr int kNumFast = (int)(sizeof kFast / sizeof kFast[0]);

size_t sim_fast_smem_bytes(int N, int nnz, int pb)
{
    return sizeof(float) * (size_t)nnz * pb + 8 * (size_t)nnz + 4 * (size_t)(N + 1);
}

bool sim_fast_fits(int variant, int N, int nnz_max)
{
    if (variant < 0 || variant >= kNumFast) return false;
    const FastVariant& v = kFast[variant];
    const int kstride = (N + v.r - 1) / v.r;
    if (kstride * v.pb > v.maxt) return false;
    return sim_fast_smem_bytes(N, nnz_max, v.pb) * v.minb <= 220 * 1024;
}

int sim_fast_pb(int variant) { return kFast[variant].pb; }
int sim_fast_variants() { return kNumFast; }

template <int PB, int R, int MAXT, int MINB>
static cudaError_t launch_fast(const SimArgs& a, int32_t n_tiles, int nnz_max, cudaStream_t s)
{
    const int kstride = (a.N + R - 1) / R;
    const int threads = kstride * PB;
    const size_t smem = sim_fast_smem_bytes(a.N, nnz_max, PB);
    cudaError_t e = cudaFuncSetAttribute(sim_fast_kernel<PB, R, MAXT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    sim_fast_kernel<PB, R, MAXT, MINB><<<n_tiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sim_fast(const SimArgs& a, int variant, int32_t n_tiles, int nnz_max, cudaStream_t s)
{
    if (n_tiles <= 0 || a.n_chunk <= 0) return cudaSuccess;
    switch (variant) {
    case 0: return launch_fast<16, 4, 288, 2>(a, n_tiles, nnz_max, s);
    case 1: return launch_fast<32, 4, 576, 1>(a, n_tiles, nnz_max, s);
    case 2: return launch_fast<16, 2, 544, 1>(a, n_tiles, nnz_max, s);
    case 3: return launch_fast<16, 4, 288, 1>(a, n_tiles, nnz_max, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvbx

// Simulation kernels of the tvbx engine (arXiv 2311.13337): state and ring
// initialisation, the shared OU table (Eq. 4), and the general chunked
// lock-step integration of all (set, region) pairs (forward Euler, Sec. "MPI"
// last paragraph; temporal average of the inner steps, Sec. "Output"). The
// model itself is in model_device.cuh.

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "model_device.cuh"
#include "tile_common.cuh"

namespace tvbx {

// ---------------------------------------------------------------------------
// Initial state: E = E0, I = I0, everything else 0 (OU starts at 0).
// ---------------------------------------------------------------------------
__global__ void init_state_kernel(float* __restrict__ state, uint32_t* __restrict__ status,
                                  const float* __restrict__ prm, int64_t NP, int64_t P, float E0, float I0)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NP * SV_COUNT;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / NP;
        state[i] = v == SV_E ? E0 : (v == SV_I ? I0 : 0.0f);
    }
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t st = 0u;   // a non-finite parameter marks the set from the start
        for (int a = 0; a < TVBX_N_AXES; ++a)
            if (!isfinite(prm[a * P + p])) st = TVBX_SET_NONFINITE;
        status[p] = st;
    }
}

__global__ void fill_kernel(float* __restrict__ x, int64_t n, float v)
{
    const int64_t n4 = n / 4;
    float4* x4 = reinterpret_cast<float4*>(x);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x)
        x4[i] = make_float4(v, v, v, v);
    for (int64_t i = n4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// ---------------------------------------------------------------------------
// Shared OU table for one chunk: table[s][k] = OU_k(n0 + s), the value used at
// step n0 + s. One block per region: the normals are drawn in parallel into
// shared memory, then one thread runs the Euler-Maruyama recursion.
// ---------------------------------------------------------------------------
constexpr int OU_TILE = 4096;

__global__ void ou_table_kernel(DevModel m, float* __restrict__ table, float* __restrict__ ou_state,
                                int32_t N, int64_t n0, int32_t n_chunk, uint64_t seed)
{
    __shared__ float xi[OU_TILE];
    const int k = blockIdx.x;
    float ou = ou_state[k];
    for (int s0 = 0; s0 < n_chunk; s0 += OU_TILE) {
        const int len = min(OU_TILE, n_chunk - s0);
        for (int i = threadIdx.x; i < len; i += blockDim.x)
            xi[i] = std_normal(seed, (uint32_t)(n0 + s0 + i), (uint32_t)k, 0u);
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 0; i < len; ++i) {
                table[(int64_t)(s0 + i) * N + k] = ou;
                ou = fmaf(m.ou_a, m.ou_mu - ou, fmaf(m.ou_b, xi[i], ou));
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) ou_state[k] = ou;
}

// ---------------------------------------------------------------------------
// One chunk of the lock-step integration. A CTA owns PB sets of one speed
// group (all N regions of each): thread t handles set q = t % PB and regions
// k = t / PB + i * (blockDim / PB). The per-pair state lives in shared memory
// for the duration of the chunk; E goes to the group's ring buffer
// [H][N][P_g] (sets fastest, so a warp's gather of one delayed value across
// its sets is one contiguous segment). A CTA barrier separates steps: all
// cross-region reads stay inside the CTA's own sets.
// ---------------------------------------------------------------------------
// One tile of PB sets (PB a template constant or, with PB = 0, the runtime
// width pb) for a.n_chunk steps from step a.n0. st: shared memory
// [SV_COUNT][N][pb].
template <int PB>
static __device__ __forceinline__ void chunk_body(const SimArgs& a, const TileDev tile, int pb_rt, float* st)
{
    const int pb = PB > 0 ? PB : pb_rt;
    const GroupDev grp = a.groups[tile.group];
    const DevModel& m = a.m;
    const int N = a.N;
    const int P = a.P;
    const int npairs = N * pb;

    for (int i = threadIdx.x; i < SV_COUNT * npairs; i += blockDim.x) {
        const int v = i / npairs, rem = i - v * npairs, k = rem / pb, q = rem - k * pb;
        st[i] = q < tile.nq ? a.state[((int64_t)v * N + k) * P + grp.p_base + tile.q0 + q] : 0.0f;
    }
    __syncthreads();

    const int q = threadIdx.x % pb;
    const int kstart = threadIdx.x / pb;
    const int kstride = blockDim.x / pb;
    const bool active = q < tile.nq;
    const int qg = tile.q0 + q;           // column in the group's ring
    const int p = grp.p_base + qg;        // internal set index
    SetParams sp{};
    uint32_t pn = 0u;
    if (active) {
        sp = load_set_params(a.prm, P, p);
        pn = (uint32_t)(a.p_offset + a.ext_index[p]);
    }
    Track<float> trk = track_init<float>();
    const int64_t slot_stride = (int64_t)N * grp.stride;
    const float inv_ts = 1.0f / (float)a.ts;

    for (int s = 0; s < a.n_chunk; ++s) {
        const int64_t n = a.n0 + s;
        const int slot_n = (int)(n % grp.H);
        const int slot_w = slot_n + 1 == grp.H ? 0 : slot_n + 1;
        const bool sample_now = ((n + 1) % a.ts) == 0;
        const int64_t t = (n + 1) / a.ts - 1;
        if (active) {
            for (int k = kstart; k < N; k += kstride) {
                // delayed coupling: sum_j u_kj E_j(n - d_kj)
                float acc = 0.0f;
                const int e1 = grp.row_ptr[k + 1];
                for (int e = grp.row_ptr[k]; e < e1; ++e) {
                    const uint32_t cd = __ldg(grp.col_dly + e);
                    const int j = (int)(cd & 0xffffu);
                    int sl = slot_n - (int)(cd >> 16);
                    sl += sl < 0 ? grp.H : 0;
                    acc = fmaf(__ldg(grp.w + e), grp.ring[sl * slot_stride + (int64_t)j * grp.stride + qg], acc);
                }
                float* sk = st + k * pb + q;
                PairState x{sk[SV_E * npairs],   sk[SV_I * npairs],  sk[SV_CEE * npairs],
                            sk[SV_CEI * npairs], sk[SV_CII * npairs], sk[SV_WE * npairs],
                            sk[SV_WI * npairs],  sk[SV_CWE * npairs], sk[SV_CWI * npairs]};
                const float OU = a.noise_per_set ? sk[SV_OU * npairs] : a.ou_table[(int64_t)s * N + k];
                pair_step(m, sp, x, acc, OU, trk);
                if (a.noise_per_set) {
                    const float xi = std_normal(a.seed, (uint32_t)n, (uint32_t)k, pn);
                    sk[SV_OU * npairs] = fmaf(m.ou_a, m.ou_mu - OU, fmaf(m.ou_b, xi, OU));
                }
                sk[SV_E * npairs] = x.E; sk[SV_I * npairs] = x.I;
                sk[SV_CEE * npairs] = x.Cee; sk[SV_CEI * npairs] = x.Cei; sk[SV_CII * npairs] = x.Cii;
                sk[SV_WE * npairs] = x.We; sk[SV_WI * npairs] = x.Wi;
                sk[SV_CWE * npairs] = x.cWe; sk[SV_CWI * npairs] = x.cWi;
                grp.ring[slot_w * slot_stride + (int64_t)k * grp.stride + qg] = x.E;

                // temporal average: block mean of ts consecutive post-step states
                float accE = sk[SV_ACC_E * npairs] + x.E;
                float accI = sk[SV_ACC_I * npairs] + x.I;
                if (sample_now) {
                    const float xE = accE * inv_ts, xI = accI * inv_ts;
                    if (t < a.T) {
                        const int64_t so = series_index(a.sl, t, k, p);
                        a.series[so] = xE;
                        if (a.series_i) a.series_i[so] = xI;
                        if (t >= a.transient) {
                            kahan_add(sk[SV_SUM_E * npairs], sk[SV_CMP_E * npairs], xE);
                            kahan_add(sk[SV_SUM_I * npairs], sk[SV_CMP_I * npairs], xI);
                        }
                    }
                    accE = 0.0f;
                    accI = 0.0f;
                }
                sk[SV_ACC_E * npairs] = accE;
                sk[SV_ACC_I * npairs] = accI;
            }
        }
        __syncthreads();
    }

    for (int i = threadIdx.x; i < SV_COUNT * npairs; i += blockDim.x) {
        const int v = i / npairs, rem = i - v * npairs, k = rem / pb, qq = rem - k * pb;
        if (qq < tile.nq) a.state[((int64_t)v * N + k) * P + grp.p_base + tile.q0 + qq] = st[i];
    }
    const uint32_t flags = track_flags(m, trk, 0);
    if (active && flags) atomicOr(a.status + p, flags);
}

template <int PB>
__global__ void __launch_bounds__(512)
sim_chunk_kernel(const __grid_constant__ SimArgs a)
{
    extern __shared__ float st[];  // [SV_COUNT][N][PB]
    chunk_body<PB>(a, a.tiles[blockIdx.x], PB, st);
}

// Row entries per group of delayed loads in the register-tile body (8 measured
// 2-3% faster than 4 or than the plain loop at 192 and 360 regions).
#ifndef TVBX_DIRECT_DG
#define TVBX_DIRECT_DG 8
#endif

// ---------------------------------------------------------------------------
// Register-tile body for connectomes whose delayed rows do not fit a
// shared-memory prefetch buffer. Thread (k, quad) keeps 4 adjacent sets of
// region k in registers for the whole chunk; the coupling reads each delayed
// value of its 4 sets with one 16-byte load from the ring (the CSR rows through
// the read-only cache), in groups of TVBX_DIRECT_DG row entries whose loads
// are all issued before their sums, and sums in CSR order, like the general
// body, so the results are bit-identical to it. One CTA barrier per step (after the ring
// writes of E(n+1)). pb: sets per tile, a multiple of 4, with N pb / 4 <=
// blockDim; s_prm: shared memory [11][pb].
// ---------------------------------------------------------------------------
static __device__ __forceinline__ void direct_body(const SimArgs& a, const TileDev& tile, int pb, float* s_prm)
{
    constexpr int SPT = 4;
    constexpr int DG = TVBX_DIRECT_DG;
    const GroupDev grp = a.groups[tile.group];
    const int N = a.N;
    const int nq = pb / SPT;
    stage_set_params<0>(a, tile, grp, s_prm, pb);
    const int kk = threadIdx.x / nq;   // >= N: an idle thread (it still takes the barriers)
    ThreadSlot ts;
    ts.qt = (threadIdx.x - kk * nq) * SPT;
    ts.kr = kk;
    ts.kstride = N;
    ts.col0 = grp.p_base + tile.q0;
    ThreadPairs<SPT, 1> tp;
    load_pairs<SPT, 1>(a, tile, ts, tp);
    __syncthreads();

    const int H = grp.H;
    const int64_t slot_stride = (int64_t)N * grp.stride;
    float* ring_cols = grp.ring + tile.q0;
    // a quad whose first set exists reads 16 bytes inside the ring row (the
    // row stride is a multiple of 32 sets and quads start at multiples of 4)
    const bool reads = kk < N && tp.act[0];
    const int e0 = reads ? __ldg(grp.row_ptr + kk) : 0, e1 = reads ? __ldg(grp.row_ptr + kk + 1) : 0;
    for (int step = 0; step < a.n_chunk; ++step) {
        const int64_t n = a.n0 + step;
        const int slot_n = (int)(n % H);
        const int slot_w = slot_n + 1 == H ? 0 : slot_n + 1;
        float cpl[SPT] = {0.0f, 0.0f, 0.0f, 0.0f};
        int e = e0;
        for (; e + DG <= e1; e += DG) {
            uint32_t cd[DG];
            float w[DG];
#pragma unroll
            for (int u = 0; u < DG; ++u) {
                cd[u] = __ldg(grp.col_dly + e + u);
                w[u] = __ldg(grp.w + e + u);
            }
            float4 v[DG];
#pragma unroll
            for (int u = 0; u < DG; ++u) {
                int sl = slot_n - (int)(cd[u] >> 16);
                sl += sl < 0 ? H : 0;
                v[u] = *reinterpret_cast<const float4*>(ring_cols + sl * slot_stride +
                                                        (int64_t)(cd[u] & 0xffffu) * grp.stride + ts.qt);
            }
#pragma unroll
            for (int u = 0; u < DG; ++u) {
                cpl[0] = fmaf(w[u], v[u].x, cpl[0]);
                cpl[1] = fmaf(w[u], v[u].y, cpl[1]);
                cpl[2] = fmaf(w[u], v[u].z, cpl[2]);
                cpl[3] = fmaf(w[u], v[u].w, cpl[3]);
            }
        }
        for (; e < e1; ++e) {
            const uint32_t cd = __ldg(grp.col_dly + e);
            const float w = __ldg(grp.w + e);
            int sl = slot_n - (int)(cd >> 16);
            sl += sl < 0 ? H : 0;
            const float4 v = *reinterpret_cast<const float4*>(ring_cols + sl * slot_stride +
                                                               (int64_t)(cd & 0xffffu) * grp.stride + ts.qt);
            cpl[0] = fmaf(w, v.x, cpl[0]);
            cpl[1] = fmaf(w, v.y, cpl[1]);
            cpl[2] = fmaf(w, v.z, cpl[2]);
            cpl[3] = fmaf(w, v.w, cpl[3]);
        }
        advance_pairs<0, SPT, 1>(a, ts, s_prm, tp, cpl, n, step, ring_cols + slot_w * slot_stride, grp.stride, pb);
        __syncthreads();
    }
    store_pairs<SPT, 1>(a, ts, tp);
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
sim_direct_kernel(const __grid_constant__ SimArgs a, int32_t pb)
{
    extern __shared__ float s_prm[];   // [11][pb]
    direct_body(a, a.tiles[blockIdx.x], pb, s_prm);
}

// Persistent kernel of a batch of sweeps (any region counts, durations and
// delay horizons): each CTA takes work items (job, tile) from a global
// counter, most expensive first, and integrates the tile over the job's
// whole duration (the job's SimArgs have n0 = 0, n_chunk = n_steps and an OU
// table for all steps). The tile width pb and the body (register tiles or the
// general body) are per job; ONLY_DIRECT instances (every job on register
// tiles) leave the general body out, which keeps its registers off the
// direct body's budget.
template <int MAXT, bool ONLY_DIRECT>
__global__ void __launch_bounds__(MAXT)
sim_batch_kernel(const BatchJob* __restrict__ jobs, const BatchItem* __restrict__ items, int32_t n_items,
                 int32_t* __restrict__ head)
{
    extern __shared__ float st[];
    __shared__ int s_item;
    __shared__ BatchJob s_job;   // the item's job descriptor, read once per item
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const BatchItem bi = items[it];
        static_assert(sizeof(BatchJob) % 4 == 0, "BatchJob copied as words");
        const uint32_t* src = reinterpret_cast<const uint32_t*>(jobs + bi.job);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&s_job);
        for (int w = threadIdx.x; w < (int)(sizeof(BatchJob) / 4); w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        if (ONLY_DIRECT || s_job.direct) direct_body(s_job.a, s_job.a.tiles[bi.tile], s_job.pb, st);
        else chunk_body<0>(s_job.a, s_job.a.tiles[bi.tile], s_job.pb, st);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Transfer function at explicit points (parity tests of the a3 step).
// ---------------------------------------------------------------------------
__global__ void tf_eval_kernel(DevModel m, int pop, int64_t n, const float* __restrict__ x_e,
                               const float* __restrict__ x_i, const float* __restrict__ W,
                               const float* __restrict__ E_L, const float* __restrict__ C,
                               float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        // F, its gradient, mu_V and the contracted term from the integrator's
        // code; the Hessian from the full second-order jets
        const float* P = pop == 0 ? m.P_e : m.P_i;
        float F[6], muV;
        transfer_x(m, P, E_L[i], W[i], x_e[i], x_i[i], F, muV);
        for (int c = 3; c < 6; ++c) out[i * 8 + c] = F[c];
        float L[4];
        transfer_integrator(m, pop, E_L[i], W[i], x_e[i], x_i[i], C ? C[3 * i] : 0.0f, C ? C[3 * i + 1] : 0.0f,
                            C ? C[3 * i + 2] : 0.0f, L, muV);
        for (int c = 0; c < 3; ++c) out[i * 8 + c] = L[c];
        out[i * 8 + 6] = muV;
        out[i * 8 + 7] = L[3];
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int sim_threads(int N, int pb)
{
    // regions per thread so that the CTA has at most 512 threads
    int kstride = N;
    while (kstride * pb > 512) kstride = (kstride + 1) / 2;
    return kstride * pb;
}

size_t sim_smem_bytes(int N, int pb) { return sizeof(float) * (size_t)SV_COUNT * N * pb; }

cudaError_t launch_init_state(const SimArgs& a, cudaStream_t s)
{
    const int64_t NP = (int64_t)a.N * a.P;
    note_launch();
    init_state_kernel<<<1024, 256, 0, s>>>(a.state, a.status, a.prm, NP, a.P, a.m.E0, a.m.I0);
    return cudaGetLastError();
}

cudaError_t launch_init_ring(float* ring, int64_t count, float value, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    note_launch();
    fill_kernel<<<2048, 256, 0, s>>>(ring, count, value);
    return cudaGetLastError();
}

cudaError_t launch_ou_table(const DevModel& m, float* table, float* ou_state, int32_t N,
                            int64_t n0, int32_t n_chunk, uint64_t seed, cudaStream_t s)
{
    if (n_chunk <= 0) return cudaSuccess;
    note_launch();
    ou_table_kernel<<<N, 256, 0, s>>>(m, table, ou_state, N, n0, n_chunk, seed);
    return cudaGetLastError();
}

template <int PB>
static cudaError_t launch_sim_pb(const SimArgs& a, int32_t n_tiles, cudaStream_t s)
{
    const int threads = sim_threads(a.N, PB);
    const size_t smem = sim_smem_bytes(a.N, PB);
    cudaError_t e = cudaFuncSetAttribute(sim_chunk_kernel<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    sim_chunk_kernel<PB><<<n_tiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sim_chunk(const SimArgs& a, int32_t n_tiles, int32_t pb, cudaStream_t s)
{
    if (n_tiles <= 0 || a.n_chunk <= 0) return cudaSuccess;
    switch (pb) {
    case 8: return launch_sim_pb<8>(a, n_tiles, s);
    case 16: return launch_sim_pb<16>(a, n_tiles, s);
    case 32: return launch_sim_pb<32>(a, n_tiles, s);
    default: return cudaErrorInvalidValue;
    }
}

int sim_direct_pb(int N)
{
    // the widest tile that fits 768 threads (wider tiles measured faster)
    for (int pb : {32, 16, 8, 4})
        if ((int64_t)N * (pb / 4) <= 768) return pb;
    return 0;
}

cudaError_t launch_sim_direct(const SimArgs& a, int32_t n_tiles, int32_t pb, cudaStream_t s)
{
    if (n_tiles <= 0 || a.n_chunk <= 0) return cudaSuccess;
    if (pb % 4 != 0 || pb < 4 || (int64_t)a.N * (pb / 4) > 768) return cudaErrorInvalidValue;
    const int threads = (a.N * (pb / 4) + 31) / 32 * 32;
    const size_t smem = sizeof(float) * 11 * (size_t)pb;
    note_launch();
    if (threads <= 384) sim_direct_kernel<384><<<n_tiles, threads, smem, s>>>(a, pb);
    else sim_direct_kernel<768><<<n_tiles, threads, smem, s>>>(a, pb);
    return cudaGetLastError();
}

static auto batch_kernel(int32_t threads, bool only_direct)
{
    if (only_direct) return threads <= 512 ? sim_batch_kernel<512, true> : sim_batch_kernel<768, true>;
    return threads <= 512 ? sim_batch_kernel<512, false> : sim_batch_kernel<768, false>;
}

cudaError_t launch_sim_batch(const BatchJob* jobs, const BatchItem* items, int32_t n_items, int32_t* head,
                             int32_t grid, int32_t threads, size_t smem, bool only_direct, cudaStream_t s)
{
    if (threads > 768) return cudaErrorInvalidValue;
    auto kern = batch_kernel(threads, only_direct);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    kern<<<grid, threads, smem, s>>>(jobs, items, n_items, head);
    return cudaGetLastError();
}

int sim_batch_ctas_per_sm(int32_t threads, size_t smem, bool only_direct)
{
    if (threads > 768) return 0;
    auto kern = batch_kernel(threads, only_direct);
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_tf_eval(const DevModel& m, int pop, int64_t n, const float* x_e, const float* x_i,
                           const float* W, const float* E_L, const float* C, float* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    note_launch();
    tf_eval_kernel<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(
        m, pop, n, x_e, x_i, W, E_L, C, out);
    return cudaGetLastError();
}

}  // namespace tvbx

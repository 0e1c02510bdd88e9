// FC fitness, FC-SC correlation and the grid search over a sweep
// (arXiv 2311.13337, Sec. "Output": the simulated FC is compared with an
// external reference FC and with the structural connectivity by the Pearson
// coefficient, Eq. 6; Sec. "MPI": the results are sorted and the ten fittest
// reported; Sec. "Validation using Functional Connectivity": the fitness is
// the Pearson correlation of the external and the computed FC).
//
// Fitness of set p against target t: the Pearson coefficient of the strict
// upper triangles (k < j) of FC_p and of the target. Each target is centred
// and scaled to unit norm once (FP64 sums), so a set needs its triangle's
// mean, sum of squared deviations and one dot product per target; a CTA per
// set makes two passes over the triangle (the second from L1/L2).
// A set whose triangle is constant (min == max) or not finite gets NaN.
//
// Grid search: the k largest finite values of a [n] vector, largest first,
// ties to the lower index. Every value becomes one 64-bit key, the value's
// order-preserving bit pattern above the complement of its index, so a
// descending sort of the keys is the wanted order; non-finite values become
// key 0 and sort last. A CTA sorts 4,096 keys in shared memory (bitonic) and
// keeps its first k; passes repeat on the survivors until one CTA remains.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"
#include "tvbx.h"

namespace tvbx {
namespace {

constexpr int FIT_THREADS = 256;
constexpr int FIT_MAX_TARGETS = 8;
constexpr int TK_CHUNK = 4096;
constexpr int TK_THREADS = 1024;
constexpr int TOPK_MAX = 1024;   // k <= CHUNK / 4: every pass shrinks the survivors 4x

template <int NW>
__device__ __forceinline__ double block_sum_d(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += red[w];
    return s;
}

template <int NW>
__device__ __forceinline__ float block_sum_f(float v, float* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.0f;
    for (int w = 0; w < NW; ++w) s += red[w];
    return s;
}

// Triangle index of (r, j), r < j, row by row.
__device__ __forceinline__ int tri_index(int r, int j, int N) { return r * N - r * (r + 1) / 2 + (j - r - 1); }

// One CTA per target: that[t][e] = (x_e - mean) / ||x - mean|| over the
// triangle; bad[t] = 1 if the triangle is constant or not finite.
__global__ void __launch_bounds__(FIT_THREADS)
fit_target_kernel(const float* __restrict__ tg, int N, float* __restrict__ that, int* __restrict__ bad)
{
    constexpr int NW = FIT_THREADS / 32;
    __shared__ double red[NW];
    __shared__ float redf[2 * NW];
    const int t = blockIdx.x;
    const float* A = tg + (int64_t)t * N * N;
    const int M = N * (N - 1) / 2;
    float* out = that + (int64_t)t * M;
    double s = 0.0;
    float lo = INFINITY, hi = -INFINITY;
    bool fin = true;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < N - 1; r += NW) {
        const int e0 = tri_index(r, r + 1, N) - (r + 1);
        for (int j = r + 1 + lane; j < N; j += 32) {
            const float x = A[(int64_t)r * N + j];
            out[e0 + j] = x;
            fin = fin && isfinite(x);
            s += x;
            lo = fminf(lo, x);
            hi = fmaxf(hi, x);
        }
    }
    __syncthreads();   // out[] is re-read below by other threads
    const double mean = block_sum_d<NW>(s, red) / (double)M;
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int all_fin = __syncthreads_and(fin);
    if ((threadIdx.x & 31) == 0) { redf[threadIdx.x >> 5] = lo; redf[NW + (threadIdx.x >> 5)] = hi; }
    __syncthreads();
    for (int w = 0; w < NW; ++w) { lo = fminf(lo, redf[w]); hi = fmaxf(hi, redf[NW + w]); }
    double ss = 0.0;
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const double d = (double)out[e] - mean;
        ss += d * d;
    }
    ss = block_sum_d<NW>(ss, red);
    const bool ok = all_fin && lo < hi && ss > 0.0;
    const double inv = ok ? 1.0 / sqrt(ss) : 0.0;
    for (int e = threadIdx.x; e < M; e += blockDim.x) out[e] = (float)(((double)out[e] - mean) * inv);
    if (threadIdx.x == 0) bad[t] = ok ? 0 : 1;
}

// One CTA per set: out[p][t] = sum_e (x_e - mean) that[t][e] / sqrt(sum_e (x_e - mean)^2).
__global__ void __launch_bounds__(FIT_THREADS)
fitness_kernel(const float* __restrict__ fc, int N, const float* __restrict__ that, int n_t, float* __restrict__ out)
{
    constexpr int NW = FIT_THREADS / 32;
    __shared__ float red[(FIT_MAX_TARGETS + 3) * NW];
    const int64_t p = blockIdx.x;
    const float* F = fc + p * N * N;
    const int M = N * (N - 1) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float s = 0.0f, lo = INFINITY, hi = -INFINITY;
    bool fin = true;
    for (int r = warp; r < N - 1; r += NW)
        for (int j = r + 1 + lane; j < N; j += 32) {
            const float x = F[(int64_t)r * N + j];
            fin = fin && isfinite(x);
            s += x;
            lo = fminf(lo, x);
            hi = fmaxf(hi, x);
        }
    const float mean = block_sum_f<NW>(s, red) / (float)M;
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int all_fin = __syncthreads_and(fin);
    float* rlo = red + FIT_MAX_TARGETS * NW;
    float* rhi = rlo + NW;
    if (lane == 0) { rlo[warp] = lo; rhi[warp] = hi; }
    __syncthreads();
    for (int w = 0; w < NW; ++w) { lo = fminf(lo, rlo[w]); hi = fmaxf(hi, rhi[w]); }
    float ss = 0.0f, dot[FIT_MAX_TARGETS];
#pragma unroll
    for (int t = 0; t < FIT_MAX_TARGETS; ++t) dot[t] = 0.0f;
    for (int r = warp; r < N - 1; r += NW) {
        const int e0 = tri_index(r, r + 1, N) - (r + 1);
        for (int j = r + 1 + lane; j < N; j += 32) {
            const float d = F[(int64_t)r * N + j] - mean;
            ss = fmaf(d, d, ss);
#pragma unroll
            for (int t = 0; t < FIT_MAX_TARGETS; ++t)
                if (t < n_t) dot[t] = fmaf(d, that[(int64_t)t * M + e0 + j], dot[t]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
#pragma unroll
        for (int t = 0; t < FIT_MAX_TARGETS; ++t) dot[t] += __shfl_xor_sync(0xffffffffu, dot[t], o);
    }
    __syncthreads();
    float* rss = red + (FIT_MAX_TARGETS + 2) * NW;
    if (lane == 0) {
        rss[warp] = ss;
#pragma unroll
        for (int t = 0; t < FIT_MAX_TARGETS; ++t) red[t * NW + warp] = dot[t];
    }
    __syncthreads();
    if (threadIdx.x < n_t) {
        const int t = threadIdx.x;
        float S = 0.0f, D = 0.0f;
        for (int w = 0; w < NW; ++w) { S += rss[w]; D += red[t * NW + w]; }
        const bool ok = all_fin && lo < hi && S > 0.0f;
        out[p * n_t + t] = ok ? D * rsqrtf(S) : __int_as_float(0x7fc00000);
    }
}

__device__ __forceinline__ uint64_t make_key(float x, int64_t i)
{
    if (!isfinite(x)) return 0ull;
    if (x == 0.0f) x = 0.0f;   // -0 ties with +0
    const uint32_t u = __float_as_uint(x);
    const uint32_t o = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((uint64_t)o << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)i);
}

__device__ __forceinline__ float key_value(uint64_t k)
{
    const uint32_t o = (uint32_t)(k >> 32);
    return __uint_as_float((o & 0x80000000u) ? (o ^ 0x80000000u) : ~o);
}

// One pass: CTA b sorts items [b*CHUNK, (b+1)*CHUNK) and keeps its first k.
// keys_in == nullptr: the items are the values v (key from value and index).
// idx_out != nullptr: single CTA, final outputs.
__global__ void __launch_bounds__(TK_THREADS)
topk_kernel(const float* __restrict__ v, const uint64_t* __restrict__ keys_in, int64_t n, int k,
            uint64_t* __restrict__ keys_out, int64_t* __restrict__ idx_out, float* __restrict__ val_out)
{
    __shared__ uint64_t s[TK_CHUNK];
    const int64_t base = (int64_t)blockIdx.x * TK_CHUNK;
    for (int i = threadIdx.x; i < TK_CHUNK; i += blockDim.x) {
        const int64_t g = base + i;
        uint64_t key = 0ull;
        if (g < n) key = keys_in ? keys_in[g] : make_key(v[g], g);
        s[i] = key;
    }
    __syncthreads();
    for (int size = 2; size <= TK_CHUNK; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < TK_CHUNK / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool desc = (lo & size) == 0;
                const uint64_t a = s[lo], b = s[hi];
                if (desc ? (a < b) : (a > b)) { s[lo] = b; s[hi] = a; }
            }
            __syncthreads();
        }
    }
    if (idx_out) {
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const uint64_t key = i < TK_CHUNK ? s[i] : 0ull;
            idx_out[i] = key ? (int64_t)(0xFFFFFFFFu - (uint32_t)key) : -1;
            val_out[i] = key ? key_value(key) : __int_as_float(0x7fc00000);
        }
    } else {
        for (int i = threadIdx.x; i < k; i += blockDim.x) keys_out[(int64_t)blockIdx.x * k + i] = s[i];
    }
}

#define FCK(call, what)                                                                              \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ == cudaErrorMemoryAllocation) return report_error(TVBX_E_OOM, "%s: out of memory", what); \
        if (e_ != cudaSuccess) return report_error(TVBX_E_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// Stream-ordered scratch freed when the call returns.
struct Scratch {
    void* p = nullptr;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    cudaError_t get(size_t bytes) { return cudaMallocAsync(&p, bytes ? bytes : 1, s); }
    ~Scratch()
    {
        if (p) cudaFreeAsync(p, s);
    }
};

}  // namespace
}  // namespace tvbx

using namespace tvbx;

extern "C" tvbx_status tvbx_fc_fitness(const float* fc, int64_t n_sets, int32_t n_regions, const float* targets,
                                       int32_t n_targets, float* out, void* cuda_stream)
{
    const int N = n_regions;
    const int64_t P = n_sets;
    if (!fc || !targets || !out) return report_error(TVBX_E_INVALID_ARG, "NULL fc, targets or out");
    if (N < 3 || N > 1024) return report_error(TVBX_E_INVALID_ARG, "need 3 <= n_regions <= 1024 (have %d)", N);
    if (P < 0 || P > (int64_t)INT32_MAX) return report_error(TVBX_E_INVALID_ARG, "need 0 <= n_sets < 2^31");
    if (n_targets < 1 || n_targets > FIT_MAX_TARGETS)
        return report_error(TVBX_E_INVALID_ARG, "need 1 <= n_targets <= %d", FIT_MAX_TARGETS);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t M = (size_t)N * (N - 1) / 2;
    const size_t sz_that = sizeof(float) * M * n_targets;
    Scratch scr(s);
    FCK(scr.get(sz_that + 64), "fitness scratch");
    float* that = static_cast<float*>(scr.p);
    int* bad = reinterpret_cast<int*>(static_cast<char*>(scr.p) + sz_that);
    note_launch();
    fit_target_kernel<<<n_targets, FIT_THREADS, 0, s>>>(targets, N, that, bad);
    FCK(cudaGetLastError(), "fitness target");
    int hbad[FIT_MAX_TARGETS];
    FCK(cudaMemcpyAsync(hbad, bad, sizeof(int) * n_targets, cudaMemcpyDeviceToHost, s), "fitness target");
    FCK(cudaStreamSynchronize(s), "fitness target");
    for (int t = 0; t < n_targets; ++t)
        if (hbad[t]) return report_error(TVBX_E_INVALID_ARG, "target %d: its upper triangle is constant or not finite", t);
    if (P == 0) return TVBX_OK;
    note_launch();
    fitness_kernel<<<(unsigned)P, FIT_THREADS, 0, s>>>(fc, N, that, n_targets, out);
    FCK(cudaGetLastError(), "fitness");
    return TVBX_OK;
}

extern "C" tvbx_status tvbx_top_k(const float* values, int64_t n, int32_t k, int64_t* idx_out, float* val_out,
                                  void* cuda_stream)
{
    if (!values || !idx_out || !val_out) return report_error(TVBX_E_INVALID_ARG, "NULL values, idx_out or val_out");
    if (n < 1 || n > (int64_t)INT32_MAX) return report_error(TVBX_E_INVALID_ARG, "need 1 <= n < 2^31");
    if (k < 1 || k > TOPK_MAX) return report_error(TVBX_E_INVALID_ARG, "need 1 <= k <= %d", TOPK_MAX);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // survivors after the first pass: blocks * k keys; two ping-pong buffers
    const int64_t blocks0 = (n + TK_CHUNK - 1) / TK_CHUNK;
    const size_t cap = (size_t)(blocks0 > 1 ? blocks0 : 0) * k;
    Scratch scr(s);
    FCK(scr.get(2 * sizeof(uint64_t) * cap), "top-k scratch");
    uint64_t* buf[2] = {static_cast<uint64_t*>(scr.p), static_cast<uint64_t*>(scr.p) + cap};
    const uint64_t* in = nullptr;
    int64_t m = n;
    int cur = 0;
    while (true) {
        const int64_t blocks = (m + TK_CHUNK - 1) / TK_CHUNK;
        note_launch();
        if (blocks == 1) {
            topk_kernel<<<1, TK_THREADS, 0, s>>>(values, in, m, k, nullptr, idx_out, val_out);
            FCK(cudaGetLastError(), "top-k");
            return TVBX_OK;
        }
        topk_kernel<<<(unsigned)blocks, TK_THREADS, 0, s>>>(values, in, m, k, buf[cur], nullptr, nullptr);
        FCK(cudaGetLastError(), "top-k");
        in = buf[cur];
        m = blocks * k;
        cur ^= 1;
    }
}

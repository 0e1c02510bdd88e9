// Functional-connectivity kernels of the tvbx engine (arXiv 2311.13337,
// Sec. "Output": the FC is obtained from the covariance of the simulated
// series; Eq. 6: Pearson correlation; Table 2 "mean_FC").
//
// The E series is read through a SeriesLayout: the engine's set-blocked
// [P/4][T][N][4] or the sets-fastest [T][N][P]. For each set the kernels
// form block moments over the samples [t_begin, t_end):
//   G_b[k][j] = sum_{t in block b} (x_k(t) - m_k)(x_j(t) - m_j),
//   s_b[k]    = sum_{t in block b} (x_k(t) - m_k),
// with the shift m_k = the running mean kept by the simulation, or a given
// shift (any shift is exact; a close one avoids cancellation). The covariance over a union of
// blocks of length L is sum G_b - (sum s_b)(sum s_b)^T / L. Every producer's
// G_b is symmetric up to FP32 rounding, so the readers take the diagonal and
// the upper triangle (k < j) and write the FC symmetric.

#include <algorithm>

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace tvbx {

constexpr int FC_SETS = 8;        // sets per CTA (one 32-byte sector per (t, k) row)
constexpr int FC_THREADS = 256;
constexpr int FC_TASKS_PER_THREAD = 5;

// Gram block moments. grid = (P / FC_SETS, task chunks). Each thread owns up to
// FC_TASKS_PER_THREAD 4x4 tiles (set q, row tile kb <= column tile jb).
__global__ void __launch_bounds__(FC_THREADS)
fc_moments_kernel(const __grid_constant__ FcArgs a, int32_t Npad, int32_t Tt, int32_t tasks_per_set,
                  int32_t tasks_per_chunk)
{
    extern __shared__ float xs[];             // [FC_SETS][Tt][Npad]
    __shared__ float shift[FC_SETS * 384];    // N <= 384
    const int N = a.N;
    const int p0 = blockIdx.x * FC_SETS;
    const int nsets = min(FC_SETS, a.P - p0);
    const int64_t Tn = a.t_end - a.t_begin;
    const int nb = Npad / 4;

    for (int i = threadIdx.x; i < FC_SETS * N; i += blockDim.x) {
        const int q = i / N, k = i - q * N;
        float mval = 0.0f;
        if (q < nsets && Tn > 0) {
            const int64_t p = p0 + q;
            if (a.state) mval = a.state[(int64_t)SV_SUM_E * N * a.P + (int64_t)k * a.P + p] / (float)Tn;
            else if (a.shift) mval = a.shift[(int64_t)k * a.P + p];
        }
        shift[q * N + k] = mval;
    }

    // this thread's tasks
    int tq[FC_TASKS_PER_THREAD], tk[FC_TASKS_PER_THREAD], tj[FC_TASKS_PER_THREAD];
    int ntask = 0;
    const int chunk0 = blockIdx.y * tasks_per_chunk;
    for (int i = 0; i < FC_TASKS_PER_THREAD; ++i) {
        const int task = chunk0 + threadIdx.x + i * FC_THREADS;
        tq[i] = -1;
        if (task < chunk0 + tasks_per_chunk && task < tasks_per_set * FC_SETS) {
            const int q = task / tasks_per_set;
            int r = task - q * tasks_per_set;
            int kb = 0;
            while (r >= nb - kb) { r -= nb - kb; ++kb; }
            if (q < nsets) { tq[i] = q; tk[i] = kb; tj[i] = kb + r; ntask = i + 1; }
        }
    }
    float acc[FC_TASKS_PER_THREAD][16];
    float rs[FC_TASKS_PER_THREAD][4];
#pragma unroll
    for (int i = 0; i < FC_TASKS_PER_THREAD; ++i) {
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[i][c] = 0.0f;
#pragma unroll
        for (int c = 0; c < 4; ++c) rs[i][c] = 0.0f;
    }
    const int64_t blk = a.blk > 0 ? a.blk : Tn;
    const int64_t stride_b = (int64_t)N * N + N;
    __syncthreads();

    for (int64_t t0 = 0; t0 < Tn; t0 += Tt) {
        const int len = (int)(Tn - t0 < (int64_t)Tt ? Tn - t0 : (int64_t)Tt);
        // stage rows x[t][k][p0 .. p0 + FC_SETS) minus the shift, transposed to [q][t][k]
        for (int i = threadIdx.x; i < len * Npad * FC_SETS; i += blockDim.x) {
            const int q = i % FC_SETS;
            const int rem = i / FC_SETS;
            const int k = rem % Npad;
            const int tt = rem / Npad;
            float v = 0.0f;
            if (k < N && q < nsets)
                v = a.series[series_index(a.sl, a.t_begin + t0 + tt, k, p0 + q)] - shift[q * N + k];
            xs[((int64_t)q * Tt + tt) * Npad + k] = v;
        }
        __syncthreads();
        for (int tt = 0; tt < len; ++tt) {
#pragma unroll
            for (int i = 0; i < FC_TASKS_PER_THREAD; ++i) {
                if (i < ntask && tq[i] >= 0) {
                    const float4 xk = *reinterpret_cast<const float4*>(xs + ((int64_t)tq[i] * Tt + tt) * Npad + 4 * tk[i]);
                    const float4 xj = *reinterpret_cast<const float4*>(xs + ((int64_t)tq[i] * Tt + tt) * Npad + 4 * tj[i]);
                    const float kv[4] = {xk.x, xk.y, xk.z, xk.w};
                    const float jv[4] = {xj.x, xj.y, xj.z, xj.w};
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[i][r * 4 + c] = fmaf(kv[r], jv[c], acc[i][r * 4 + c]);
                        rs[i][r] += kv[r];
                    }
                }
            }
            // end of a moment block: write it out and restart
            const int64_t tg = t0 + tt + 1;
            if (tg % blk == 0 || tg == Tn) {
                const int64_t b = (tg - 1) / blk;
#pragma unroll
                for (int i = 0; i < FC_TASKS_PER_THREAD; ++i) {
                    if (i < ntask && tq[i] >= 0) {
                        float* G = a.blocks + ((int64_t)(p0 + tq[i]) * a.n_blocks + b) * stride_b;
                        for (int r = 0; r < 4; ++r) {
                            const int k = 4 * tk[i] + r;
                            if (k >= N) continue;
                            for (int c = 0; c < 4; ++c) {
                                const int j = 4 * tj[i] + c;
                                if (j >= N) continue;
                                G[(int64_t)k * N + j] = acc[i][r * 4 + c];
                                G[(int64_t)j * N + k] = acc[i][r * 4 + c];
                            }
                            if (tk[i] == tj[i]) G[(int64_t)N * N + k] = rs[i][r];
                        }
#pragma unroll
                        for (int c = 0; c < 16; ++c) acc[i][c] = 0.0f;
#pragma unroll
                        for (int c = 0; c < 4; ++c) rs[i][c] = 0.0f;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Per set: FC of each window (blocks [w, w + m)), upper-triangle vectors, and
// the Pearson correlation between every pair of window vectors.
__global__ void fcd_kernel(const float* __restrict__ blocks, int32_t N, int32_t n_blocks,
                           int32_t m, int32_t nw, int64_t Lw, float* __restrict__ vec,
                           float* __restrict__ fcd)
{
    extern __shared__ float sm[];   // diag [N] + mom [nw] + red
    const int p = blockIdx.x;
    const int M = N * (N - 1) / 2;
    const int64_t stride_b = (int64_t)N * N + N;
    const float* B = blocks + (int64_t)p * n_blocks * stride_b;
    float* V = vec + (int64_t)p * nw * M;
    float* dg = sm;
    float* mom = sm + N;         // [nw] means then inverse norms
    float* red = mom + 2 * nw;
    const float invL = 1.0f / (float)Lw;
    for (int w = 0; w < nw; ++w) {
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            float g = 0.0f, s = 0.0f;
            for (int b = w; b < w + m; ++b) {
                g += B[b * stride_b + (int64_t)k * N + k];
                s += B[b * stride_b + (int64_t)N * N + k];
            }
            const float v = g - s * s * invL;
            dg[k] = v > 0.0f ? sqrtf(v) : 0.0f;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < M; idx += blockDim.x) {
            // idx -> (k, j), k < j, row by row
            int k = 0, r = idx;
            while (r >= N - 1 - k) { r -= N - 1 - k; ++k; }
            const int j = k + 1 + r;
            float g = 0.0f, sk = 0.0f, sj = 0.0f;
            for (int b = w; b < w + m; ++b) {
                g += B[b * stride_b + (int64_t)k * N + j];   // upper triangle (the matrices are symmetric)
                sk += B[b * stride_b + (int64_t)N * N + k];
                sj += B[b * stride_b + (int64_t)N * N + j];
            }
            const float c = g - sk * sj * invL;
            const float d = dg[k] * dg[j];
            V[(int64_t)w * M + idx] = d > 0.0f ? c / d : 0.0f;
        }
        __syncthreads();
    }
    // centre each window vector and normalise it
    for (int w = 0; w < nw; ++w) {
        float s = 0.0f;
        for (int i = threadIdx.x; i < M; i += blockDim.x) s += V[(int64_t)w * M + i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += red[q];
            mom[w] = t / (float)M;
        }
        __syncthreads();
        const float mu = mom[w];
        float ss = 0.0f;
        for (int i = threadIdx.x; i < M; i += blockDim.x) {
            const float v = V[(int64_t)w * M + i] - mu;
            V[(int64_t)w * M + i] = v;
            ss += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        __syncthreads();
        if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = ss;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += red[q];
            mom[nw + w] = t > 0.0f ? rsqrtf(t) : 0.0f;
        }
        __syncthreads();
    }
    for (int pair = 0; pair < nw * nw; ++pair) {
        const int u = pair / nw, v = pair - u * nw;
        if (v < u) continue;
        float s = 0.0f;
        for (int i = threadIdx.x; i < M; i += blockDim.x) s += V[(int64_t)u * M + i] * V[(int64_t)v * M + i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += red[q];
            float r = t * mom[nw + u] * mom[nw + v];
            if (u == v) r = 1.0f;
            fcd[((int64_t)p * nw + u) * nw + v] = r;
            fcd[((int64_t)p * nw + v) * nw + u] = r;
        }
        __syncthreads();
    }
}

__global__ void summary_kernel(const float* __restrict__ state, int32_t N, int32_t P, int64_t n_samples,
                               float* __restrict__ mean_e_hz, float* __restrict__ mean_i_hz)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    float se = 0.0f, si = 0.0f;
    for (int k = 0; k < N; ++k) {
        se += state[(int64_t)SV_SUM_E * N * P + (int64_t)k * P + p];
        si += state[(int64_t)SV_SUM_I * N * P + (int64_t)k * P + p];
    }
    const float scale = n_samples > 0 ? 1000.0f / ((float)N * (float)n_samples) : 0.0f;
    mean_e_hz[p] = se * scale;
    mean_i_hz[p] = si * scale;
}

cudaError_t launch_fc_moments(const FcArgs& a, cudaStream_t s)
{
    if (a.N > 384) return cudaErrorInvalidValue;
    const int Npad = (a.N + 3) / 4 * 4;
    const int nb = Npad / 4;
    const int tasks_per_set = nb * (nb + 1) / 2;
    const int total = tasks_per_set * FC_SETS;
    const int per_chunk = FC_THREADS * FC_TASKS_PER_THREAD;
    const int chunks = (total + per_chunk - 1) / per_chunk;
    int Tt = 16384 / (FC_SETS * Npad);
    Tt = Tt < 4 ? 4 : (Tt > 32 ? 32 : Tt);
    const size_t smem = sizeof(float) * (size_t)FC_SETS * Tt * Npad;
    cudaError_t e = cudaFuncSetAttribute(fc_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.P + FC_SETS - 1) / FC_SETS, chunks);
    note_launch();
    fc_moments_kernel<<<grid, FC_THREADS, smem, s>>>(a, Npad, Tt, tasks_per_set, per_chunk);
    return cudaGetLastError();
}

// Shift of each (region, set): mean of up to 64 evenly spaced samples of
// [t_begin, t_end). Any shift gives the same moments in exact arithmetic; one
// within a few standard deviations of the mean keeps the low-precision
// operands of the tensor-core path small relative to the fluctuations.
// Consecutive threads take consecutive elements of a sample: sets fastest in
// the [T][N][P] layout, (region, set within the group of 4) in the
// set-blocked one.
__global__ void fc_shift_kernel(const float* __restrict__ series, const SeriesLayout sl, int32_t N, int64_t P,
                                int64_t t_begin, int64_t t_end, float* __restrict__ shift)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t k, p;
    if (sl.sk == 4) {   // i = (group, region, set within the group)
        const int64_t g = i / (4 * (int64_t)N), q = i - g * 4 * (int64_t)N;
        k = q >> 2;
        p = 4 * g + (q & 3);
        if (p >= P) return;
    } else {            // i = (region, set)
        if (i >= (int64_t)N * P) return;
        k = i / P;
        p = i - k * P;
    }
    const int64_t o = k * P + p;   // shift[k][p]
    const int64_t Tn = t_end - t_begin;
    const int64_t n = Tn < 64 ? Tn : 64;
    float s = 0.0f;
    if (Tn <= (int64_t)(UINT32_MAX / 64)) {   // the same sample indices in 32-bit arithmetic
        const uint32_t tn = (uint32_t)Tn, nn = (uint32_t)n;
#pragma unroll 8
        for (uint32_t q = 0; q < nn; ++q) s += series[series_index(sl, t_begin + (q * tn) / nn, k, p)];
    } else {
        for (int64_t q = 0; q < n; ++q) s += series[series_index(sl, t_begin + (q * Tn) / n, k, p)];
    }
    shift[o] = n > 0 ? s / (float)n : 0.0f;
}

// acc += add over n floats: the block moments of one chunk of a streamed
// series folded into the moments of the run (the blocks of all chunks share
// one shift, so their sums add).
__global__ void fc_accumulate_kernel(const float* __restrict__ add, float* __restrict__ acc, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[i] += add[i];
}

cudaError_t launch_fc_accumulate(const float* add, float* acc, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    note_launch();
    fc_accumulate_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(add, acc, n);
    return cudaGetLastError();
}

cudaError_t launch_fc_shift(const float* series, const SeriesLayout& sl, int32_t N, int64_t P, int64_t t_begin,
                            int64_t t_end, float* shift, cudaStream_t s)
{
    // threads: N P, or N x (P rounded up to 4) in the set-blocked layout
    const int64_t n = (int64_t)N * (sl.sk == 4 ? (P + 3) / 4 * 4 : P);
    note_launch();
    fc_shift_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(series, sl, N, P, t_begin, t_end, shift);
    return cudaGetLastError();
}

// Per set, from the block moments: Pearson FC over all samples, chi, mean
// off-diagonal FC and, when nw > 0, the FCD over nw windows of m blocks
// (Lw samples each) in one pass. One CTA per set; one warp per FC row; the
// window FC vectors (upper triangles) stay in shared memory. MW > 0: m == MW
// and n_blocks <= FCR_MAXB, block values in registers with compile-time
// indices; MW == 0: any m and n_blocks, block values re-read.
//
// Every producer writes a Gram matrix that is symmetric up to FP32 rounding
// (the SIMT kernel exactly, the tensor-core forms as H H^T or
// H H^T + H L^T + L H^T), so only the upper triangle is read: row r from
// column r + 1 on, along the row (coalesced).
constexpr int RED_THREADS = 512;
constexpr int RED_WARPS = RED_THREADS / 32;
constexpr int FCR_MAXB = 12;

// Work items of the row pass: (row r, first column of a 32-column chunk right
// of the diagonal), row by row; their number is sum over L = 1 .. N-1 of
// ceil(L / 32).
static __host__ __device__ inline int fc_reduce_items(int N)
{
    const int Q = (N - 1) / 32, R = (N - 1) % 32;
    return N > 1 ? 16 * Q * (Q + 1) + R * (Q + 1) : 0;
}

static __device__ __forceinline__ float warp_sum(float x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int MW>
__global__ void __launch_bounds__(RED_THREADS)
fc_reduce_kernel(const __grid_constant__ FcArgs a, int32_t m, int32_t nw, int64_t Lw, float* __restrict__ fcd)
{
    extern __shared__ float sm[];
    const int N = a.N, nb = a.n_blocks;
    const int64_t p = blockIdx.x;
    const int M = N * (N - 1) / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int64_t stride_b = (int64_t)N * N + N;
    const float* B = a.blocks + p * nb * stride_b;
    const int64_t Tn = a.t_end - a.t_begin;
    float* sSf = sm;                        // [N] row sums over all blocks
    float* isd = sSf + N;                   // [N] 1 / sd over all samples (0 if sd = 0)
    float* cdg = isd + N;                   // [N] variance over all samples
    float* sSw = cdg + N;                   // [nw][N] window row sums
    float* isdw = sSw + nw * N;             // [nw][N] window 1 / sd
    float* V = isdw + nw * N;               // [nw][M] window FC upper triangles
    float* red = V + (size_t)nw * M;        // [48] sums, [nw] inverse norms
    int* items = reinterpret_cast<int*>(red + 48 + nw);   // row-pass items
    const int n_items = fc_reduce_items(N);
    const float invT = Tn > 0 ? 1.0f / (float)Tn : 0.0f;
    const float invL = Lw > 0 ? 1.0f / (float)Lw : 0.0f;

    if (tid == RED_THREADS - 1) {
        int q = 0;
        for (int r = 0; r + 1 < N; ++r)
            for (int c = r + 1; c < N; c += 32) items[q++] = (r << 16) | c;
    }
    for (int k = tid; k < N; k += blockDim.x) {
        const float* sk_b = B + (int64_t)N * N + k;
        const float* dk_b = B + (int64_t)k * N + k;
        float g = 0.0f, sk = 0.0f;
        for (int b = 0; b < nb; ++b) { g += dk_b[b * stride_b]; sk += sk_b[b * stride_b]; }
        const float v = g - sk * sk * invT;
        sSf[k] = sk;
        cdg[k] = v;
        isd[k] = v > 0.0f ? rsqrtf(v) : 0.0f;
        for (int w = 0; w < nw; ++w) {
            float gw = 0.0f, sw = 0.0f;
            for (int b = w; b < w + m; ++b) { gw += dk_b[b * stride_b]; sw += sk_b[b * stride_b]; }
            const float vw = gw - sw * sw * invL;
            sSw[w * N + k] = sw;
            isdw[w * N + k] = vw > 0.0f ? rsqrtf(vw) : 0.0f;
        }
    }
    __syncthreads();

    float s_all = 0.0f, s_diag = 0.0f, s_fc = 0.0f;
    bool zero = false;
    float* fc = a.fc ? a.fc + p * N * N : nullptr;
    for (int k = tid; k < N; k += blockDim.x) {
        s_all += cdg[k];
        s_diag += cdg[k];
        if (!(isd[k] > 0.0f)) zero = true;
        if (fc) fc[(int64_t)k * N + k] = 1.0f;
    }
    // the row pass: items (row, 32-column chunk) dealt to the warps in turn,
    // so every warp gets the same number of chunks up to one
    for (int it = warp; it < n_items; it += RED_WARPS) {
        const int r = items[it] >> 16, jj = (items[it] & 0xffff) + lane;
        const float sr = sSf[r], ir = isd[r];
        const int e0 = r * N - r * (r + 1) / 2 - r - 1;   // triangle index of (r, jj) is e0 + jj
        const float* Br = B + (int64_t)r * N;              // row r of block 0
        if (jj < N) {
            // the block matrices at (r, jj)
            float g = 0.0f;
            float pre[FCR_MAXB + 1];
            if constexpr (MW > 0) {
                pre[0] = 0.0f;
#pragma unroll
                for (int b = 0; b < FCR_MAXB; ++b) {
                    const float gb = b < nb ? Br[b * stride_b + jj] : 0.0f;
                    pre[b + 1] = pre[b] + gb;
                }
                g = pre[FCR_MAXB];
            } else {
                for (int b = 0; b < nb; ++b) g += Br[b * stride_b + jj];
            }
            const float c = g - sr * sSf[jj] * invT;
            const float f = c * ir * isd[jj];
            s_all += 2.0f * c;
            s_fc += 2.0f * f;
            if (fc) {
                fc[(int64_t)r * N + jj] = f;
                fc[(int64_t)jj * N + r] = f;
            }
            if constexpr (MW > 0) {
#pragma unroll
                for (int w = 0; w + MW <= FCR_MAXB; ++w) {
                    if (w < nw) {
                        const float gw = pre[w + MW] - pre[w];
                        const float cw = gw - sSw[w * N + r] * sSw[w * N + jj] * invL;
                        V[(size_t)w * M + e0 + jj] = cw * isdw[w * N + r] * isdw[w * N + jj];
                    }
                }
            } else {
                for (int w = 0; w < nw; ++w) {
                    float gw = 0.0f;
                    for (int b = w; b < w + m; ++b)
                        gw += Br[b * stride_b + jj];
                    const float cw = gw - sSw[w * N + r] * sSw[w * N + jj] * invL;
                    V[(size_t)w * M + e0 + jj] = cw * isdw[w * N + r] * isdw[w * N + jj];
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s_all += __shfl_xor_sync(0xffffffffu, s_all, o);
        s_diag += __shfl_xor_sync(0xffffffffu, s_diag, o);
        s_fc += __shfl_xor_sync(0xffffffffu, s_fc, o);
    }
    if (lane == 0) { red[warp] = s_all; red[16 + warp] = s_diag; red[32 + warp] = s_fc; }
    if (zero) atomicOr(a.status + p, TVBX_SET_ZERO_VAR);
    __syncthreads();
    if (tid == 0) {
        float A = 0.0f, D = 0.0f, F = 0.0f;
        for (int w = 0; w < nwarps; ++w) { A += red[w]; D += red[16 + w]; F += red[32 + w]; }
        const float num = A / ((float)N * (float)N), den = D / (float)N;
        a.chi[p] = den > 0.0f ? sqrtf(fmaxf(num / den, 0.0f)) : 0.0f;
        a.mean_fc[p] = N > 1 ? F / ((float)N * (float)(N - 1)) : 0.0f;
    }
    if (nw == 0) return;

    // FCD: centre and normalise each window vector (a warp per window), then
    // the products of window u with up to four windows v > u per warp item
    // (window u read once for all four)
    float* mom = red + 48;   // [nw] inverse norms
    for (int w = warp; w < nw; w += RED_WARPS) {
        float* v = V + (size_t)w * M;
        float sum = 0.0f;
        for (int i = lane; i < M; i += 32) sum += v[i];
        const float mean = warp_sum(sum) / (float)M;
        float ss = 0.0f;
        for (int i = lane; i < M; i += 32) {
            const float x = v[i] - mean;
            v[i] = x;
            ss += x * x;
        }
        ss = warp_sum(ss);
        if (lane == 0) {
            mom[w] = ss > 0.0f ? rsqrtf(ss) : 0.0f;
            fcd[(p * nw + w) * nw + w] = 1.0f;
        }
    }
    __syncthreads();
    int n_pitems = 0;   // items (u, first v) with v = u + 1, u + 5, ...
    for (int u = 0; u < nw; ++u) n_pitems += (nw - 1 - u + 3) / 4;
    for (int it = warp; it < n_pitems; it += RED_WARPS) {
        int u = 0, rem = it;
        while (rem >= (nw - 1 - u + 3) / 4) { rem -= (nw - 1 - u + 3) / 4; ++u; }
        const int v0 = u + 1 + 4 * rem, nv = nw - v0 < 4 ? nw - v0 : 4;
        const float* x = V + (size_t)u * M;
        const float* y0 = V + (size_t)v0 * M;
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int i = lane; i < M; i += 32) {
            const float xi = x[i];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < nv) acc[c] += xi * y0[(size_t)c * M + i];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c < nv) {
                const float dot = warp_sum(acc[c]);
                if (lane == 0) {
                    const int v2 = v0 + c;
                    const float r = dot * mom[u] * mom[v2];
                    fcd[(p * nw + u) * nw + v2] = r;
                    fcd[(p * nw + v2) * nw + u] = r;
                }
            }
        }
    }
}

static size_t fc_reduce_smem(int N, int nb, int nw)
{
    (void)nb;
    const size_t M = (size_t)N * (N - 1) / 2;
    return sizeof(float) * (3 * (size_t)N + 2 * (size_t)nw * N + (size_t)nw * M + 48 + (size_t)nw) +
           sizeof(int) * (size_t)fc_reduce_items(N);
}

template <int MW>
static cudaError_t launch_reduce_mw(const FcArgs& a, int32_t m, int32_t nw, int64_t Lw, float* fcd, size_t smem,
                                    cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(fc_reduce_kernel<MW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    fc_reduce_kernel<MW><<<a.P, RED_THREADS, smem, s>>>(a, m, nw, Lw, fcd);
    return cudaGetLastError();
}

cudaError_t launch_fc_reduce(const FcArgs& a, int32_t m, int32_t nw, int64_t Lw, float* vec_scratch, float* fcd,
                             cudaStream_t s)
{
    const size_t smem = fc_reduce_smem(a.N, a.n_blocks, nw);
    if (smem > 200 * 1024) {
        // window vectors too large for shared memory: the FC pass without
        // windows, then the FCD with the vectors in global scratch
        cudaError_t e = launch_fc_finalize(a, s);
        if (e != cudaSuccess) return e;
        return launch_fcd(a.blocks, a.P, a.N, a.n_blocks, m, nw, Lw, vec_scratch, fcd, s);
    }
    if (a.n_blocks <= FCR_MAXB) {
        const int mw = nw == 0 ? 1 : m;   // without windows only the block sum is used
        switch (mw) {
        case 1: return launch_reduce_mw<1>(a, m, nw, Lw, fcd, smem, s);
        case 2: return launch_reduce_mw<2>(a, m, nw, Lw, fcd, smem, s);
        case 3: return launch_reduce_mw<3>(a, m, nw, Lw, fcd, smem, s);
        case 4: return launch_reduce_mw<4>(a, m, nw, Lw, fcd, smem, s);
        default: break;
        }
    }
    return launch_reduce_mw<0>(a, m, nw, Lw, fcd, smem, s);
}

cudaError_t launch_fc_finalize(const FcArgs& a, cudaStream_t s)
{
    const size_t smem = fc_reduce_smem(a.N, a.n_blocks, 0);
    return a.n_blocks <= FCR_MAXB ? launch_reduce_mw<1>(a, 0, 0, 0, nullptr, smem, s)
                                  : launch_reduce_mw<0>(a, 0, 0, 0, nullptr, smem, s);
}

size_t fc_reduce_needs_vec_scratch(int N, int nb, int nw) { return fc_reduce_smem(N, nb, nw) > 200 * 1024; }

cudaError_t launch_fcd(const float* blocks, int32_t P, int32_t N, int32_t n_blocks,
                       int32_t blocks_per_window, int32_t n_windows, int64_t window_samples,
                       float* vec_scratch, float* fcd, cudaStream_t s)
{
    const size_t smem = sizeof(float) * ((size_t)N + 2 * n_windows + 64);
    note_launch();
    fcd_kernel<<<P, 256, smem, s>>>(blocks, N, n_blocks, blocks_per_window, n_windows, window_samples,
                                    vec_scratch, fcd);
    return cudaGetLastError();
}

cudaError_t launch_summary(const float* state, int32_t N, int32_t P, int64_t n_samples,
                           float* mean_e_hz, float* mean_i_hz, cudaStream_t s)
{
    note_launch();
    summary_kernel<<<(P + 255) / 256, 256, 0, s>>>(state, N, P, n_samples, mean_e_hz, mean_i_hz);
    return cudaGetLastError();
}

}  // namespace tvbx

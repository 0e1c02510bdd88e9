// Allocation-free variant of the FC computation (tvbx_fc_noalloc).
//
// Some callers cannot allocate device memory at the point where they need an
// FC: hosts that fix their device-memory budget at start-up and forbid later
// allocations (real-time or embedded services, plugins running under another
// framework's memory manager), or code paths where a cudaMalloc would
// synchronise the device and stall other work. This entry point takes the
// caller's series and output buffers and keeps its only scratch, the moments
// of each set, in a fixed array that the library reserves on every device
// that loads it.
//
// The scratch is a file-scope __device__ array. Its address in host code is a
// host-side stand-in, so the device address is obtained with
// cudaGetSymbolAddress (with the device current) and passed to the kernels.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "internal.h"
#include "tvbx.h"

namespace tvbx {

// 8 Mi floats = 32 MiB, held by every GPU that loads the library until exit.
constexpr int64_t FC_NOALLOC_FLOATS = (int64_t)8 << 20;
static __device__ __align__(256) float g_fc_noalloc_scratch[FC_NOALLOC_FLOATS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device. The first call
// on a device looks it up; every later call made outside stream capture
// looks it up again (cheap), so the address stays valid when the device has
// been reset and the module reloaded since. Under capture the cached address
// is used.
cudaError_t scratch_address(cudaStream_t s, float** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusActive;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();   // the query's own error is not the call's
        cs = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fc_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

// Per set: shift m_k = x_k(0) plus the mean of x_k - x_k(0) over up to 64
// evenly spaced samples (any shift is exact; one near the mean keeps the
// centred sums small, and a constant row gets exactly zero variance), then the
// upper triangle of G[k][j] = sum_t (x_k - m_k)(x_j - m_j) and
// s[k] = sum_t (x_k - m_k) into scratch [P][N*N + N] (both triangles
// written). The sums are compensated: each 32-sample tile is summed in FP32
// and the tile sums are added with a Kahan carry. One CTA of 512 threads per
// set, up to 8 (k <= j) pairs per thread; the series is [T][N][P].
constexpr int NOALLOC_THREADS = 512;
constexpr int NOALLOC_PAIRS = 8;

static __device__ __forceinline__ void noalloc_kahan(float& s, float& c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__global__ void __launch_bounds__(NOALLOC_THREADS)
fc_noalloc_moments_kernel(const float* __restrict__ X, int32_t N, int64_t P, int64_t T, float* __restrict__ scratch)
{
    extern __shared__ float sh[];   // shift [N], tile [32][N]
    const int64_t p = blockIdx.x;
    float* shift = sh;
    float* tile = sh + N;
    const int64_t NP = (int64_t)N * P;
    const int n_tri = N * (N + 1) / 2;
    const int ns = (int)(T < 64 ? T : 64);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        // x(0) plus the mean deviation from it: exactly x(0) for a constant row
        const float x0 = X[(int64_t)k * P + p];
        float m = 0.0f;
        for (int i = 0; i < ns; ++i) m += X[(i * T / ns) * NP + (int64_t)k * P + p] - x0;
        shift[k] = x0 + m / (float)ns;
    }
    int pk[NOALLOC_PAIRS], pj[NOALLOC_PAIRS];
    float acc[NOALLOC_PAIRS], cmp[NOALLOC_PAIRS];
#pragma unroll
    for (int c = 0; c < NOALLOC_PAIRS; ++c) {
        int r = threadIdx.x + c * NOALLOC_THREADS, k = 0;
        if (r < n_tri) {
            while (r >= N - k) { r -= N - k; ++k; }
            pk[c] = k;
            pj[c] = k + r;
        } else {
            pk[c] = pj[c] = -1;
        }
        acc[c] = 0.0f;
        cmp[c] = 0.0f;
    }
    float rs = 0.0f, rc = 0.0f;
    __syncthreads();
    for (int64_t t0 = 0; t0 < T; t0 += 32) {
        const int len = (int)(T - t0 < 32 ? T - t0 : 32);
        for (int i = threadIdx.x; i < len * N; i += blockDim.x) {
            const int tt = i / N, k = i - tt * N;
            tile[i] = X[(t0 + tt) * NP + (int64_t)k * P + p] - shift[k];
        }
        __syncthreads();
        float part[NOALLOC_PAIRS];
#pragma unroll
        for (int c = 0; c < NOALLOC_PAIRS; ++c) part[c] = 0.0f;
        float prs = 0.0f;
        for (int tt = 0; tt < len; ++tt) {
#pragma unroll
            for (int c = 0; c < NOALLOC_PAIRS; ++c)
                if (pk[c] >= 0) part[c] = fmaf(tile[tt * N + pk[c]], tile[tt * N + pj[c]], part[c]);
            if (threadIdx.x < N) prs += tile[tt * N + threadIdx.x];
        }
#pragma unroll
        for (int c = 0; c < NOALLOC_PAIRS; ++c) noalloc_kahan(acc[c], cmp[c], part[c]);
        noalloc_kahan(rs, rc, prs);
        __syncthreads();
    }
    float* out = scratch + p * (int64_t)(N * N + N);
#pragma unroll
    for (int c = 0; c < NOALLOC_PAIRS; ++c)
        if (pk[c] >= 0) {
            out[pk[c] * N + pj[c]] = acc[c];
            out[pj[c] * N + pk[c]] = acc[c];
        }
    if (threadIdx.x < N) out[N * N + threadIdx.x] = rs;
}

// Per set: covariance, Pearson FC, chi and mean off-diagonal FC (same
// definitions as tvbx_fc).
__global__ void fc_noalloc_finalize_kernel(const float* __restrict__ scratch, int32_t N, int64_t T,
                                           float* __restrict__ fc, float* __restrict__ chi,
                                           float* __restrict__ mean_fc)
{
    extern __shared__ float sh[];   // cov [N*N], sd [N], red [48]
    const int64_t p = blockIdx.x;
    const int NN = N * N;
    const float* G = scratch + p * (int64_t)(NN + N);
    float* cov = sh;
    float* sd = sh + NN;
    float* red = sd + N;
    const float invT = 1.0f / (float)T;
    for (int i = threadIdx.x; i < NN; i += blockDim.x) {
        const int k = i / N, j = i - k * N;
        cov[i] = G[i] - G[NN + k] * G[NN + j] * invT;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) sd[k] = cov[k * N + k] > 0.0f ? sqrtf(cov[k * N + k]) : 0.0f;
    __syncthreads();
    float s_all = 0.0f, s_diag = 0.0f, s_fc = 0.0f;
    for (int i = threadIdx.x; i < NN; i += blockDim.x) {
        const int k = i / N, j = i - k * N;
        s_all += cov[i];
        float f = 1.0f;
        if (k == j) {
            s_diag += cov[i];
        } else {
            const float d = sd[k] * sd[j];
            f = d > 0.0f ? cov[i] / d : 0.0f;
            s_fc += f;
        }
        fc[p * NN + i] = f;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s_all += __shfl_xor_sync(0xffffffffu, s_all, o);
        s_diag += __shfl_xor_sync(0xffffffffu, s_diag, o);
        s_fc += __shfl_xor_sync(0xffffffffu, s_fc, o);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) { red[warp] = s_all; red[16 + warp] = s_diag; red[32 + warp] = s_fc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float A = 0.0f, D = 0.0f, F = 0.0f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) { A += red[w]; D += red[16 + w]; F += red[32 + w]; }
        const float num = A / ((float)N * (float)N), den = D / (float)N;
        if (chi) chi[p] = den > 0.0f ? sqrtf(fmaxf(num / den, 0.0f)) : 0.0f;
        if (mean_fc) mean_fc[p] = N > 1 ? F / ((float)N * (float)(N - 1)) : 0.0f;
    }
}

}  // namespace tvbx

using namespace tvbx;

extern "C" tvbx_status tvbx_fc_noalloc(const float* series, int32_t n_regions, int64_t n_sets, int64_t n_samples,
                                       float* fc_out, float* chi, float* mean_fc, void* cuda_stream)
{
    // Argument and size checks come first; nothing below allocates.
    if (!series || !fc_out) return report_error(TVBX_E_INVALID_ARG, "NULL series or fc_out");
    if (n_regions < 1 || n_regions > 90 || n_sets < 1 || n_samples < 1)
        return report_error(TVBX_E_INVALID_ARG, "need 1 <= n_regions <= 90, n_sets >= 1, n_samples >= 1");
    if (n_sets > (int64_t)INT32_MAX) return report_error(TVBX_E_INVALID_ARG, "n_sets must be < 2^31");
    const int64_t need = n_sets * ((int64_t)n_regions * n_regions + n_regions);
    if (need > FC_NOALLOC_FLOATS)
        return report_error(TVBX_E_INVALID_ARG,
                                 "n_sets x (n_regions^2 + n_regions) = %lld floats exceeds the fixed scratch of %lld "
                                 "floats; split the sets into calls of at most %lld",
                                 (long long)need, (long long)FC_NOALLOC_FLOATS,
                                 (long long)(FC_NOALLOC_FLOATS / ((int64_t)n_regions * n_regions + n_regions)));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float* scratch = nullptr;
    cudaError_t e = scratch_address(s, &scratch);
    if (e != cudaSuccess) return report_error(TVBX_E_CUDA, "scratch address: %s", cudaGetErrorString(e));
    const size_t sm1 = sizeof(float) * ((size_t)n_regions + 32 * (size_t)n_regions);
    note_launch();
    fc_noalloc_moments_kernel<<<(unsigned)n_sets, NOALLOC_THREADS, sm1, s>>>(series, n_regions, n_sets, n_samples, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return report_error(TVBX_E_CUDA, "moments: %s", cudaGetErrorString(e));
    const size_t sm2 = sizeof(float) * ((size_t)n_regions * n_regions + n_regions + 48);
    if (sm2 > 48 * 1024) {
        e = cudaFuncSetAttribute(fc_noalloc_finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        if (e != cudaSuccess) return report_error(TVBX_E_CUDA, "finalize: %s", cudaGetErrorString(e));
    }
    note_launch();
    fc_noalloc_finalize_kernel<<<(unsigned)n_sets, NOALLOC_THREADS, sm2, s>>>(scratch, n_regions, n_samples, fc_out, chi, mean_fc);
    if ((e = cudaGetLastError()) != cudaSuccess) return report_error(TVBX_E_CUDA, "finalize: %s", cudaGetErrorString(e));
    return TVBX_OK;
}

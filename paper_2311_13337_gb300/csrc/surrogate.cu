// Surrogate network of the tvbx engine: an ensemble of multilayer perceptrons
// mapping sweep parameters to summary statistics, trained on the GPU by this
// file's own kernels (forward, backward, AdamW), used to propose where the
// sweep should be refined. The paper has no counterpart; it motivates guided
// exploration of the parameter space (Sec. "Discussion").
//
// Network: inputs normalised to [-1, 1] by the domain box; hidden layers
// a_l = max(0, a_{l-1} W_l^T + b_l); linear output layer predicting the
// standardised targets. Loss: mean squared error. Optimiser: AdamW
// (decoupled weight decay on the weight matrices; Adam moment estimates with
// bias corrections). Parameters: FP32 master copy, BF16 copy of the weights
// read by the forward and backward products, FP32 accumulation. The members
// of the ensemble differ by their initial weights and their shuffles and run
// as the z dimension of every launch.
//
// Layout of one member's parameters (also the flattened host layout):
// layer by layer, W_l [out][in] row-major, then b_l [out].

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "alloc.h"
#include "internal.h"
#include "gemm_simt.cuh"
#include "gemm_tc.cuh"
#include "model_device.cuh"
#include "tvbx.h"

namespace tvbx {
namespace {

// ---------------------------------------------------------------- kernels

static __device__ __forceinline__ float uniform01(uint32_t x) { return ((float)x + 0.5f) * 2.3283064365386963e-10f; }

// He-uniform weights, zero biases; bf16 copy.
__global__ void mlp_init_kernel(float* __restrict__ p, __nv_bfloat16* __restrict__ pb, const int64_t* __restrict__ seg,
                                int n_layers, int64_t n_par, int E, uint64_t seed)
{
    // seg[4 l + 0..3] = W offset, W count, b offset, fan_in
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_par * E) return;
    const int64_t j = idx % n_par;
    const uint32_t m = (uint32_t)(idx / n_par);
    float v = 0.0f;
    for (int l = 0; l < n_layers; ++l) {
        const int64_t wo = seg[4 * l], wc = seg[4 * l + 1];
        if (j >= wo && j < wo + wc) {
            const float a = sqrtf(6.0f / (float)seg[4 * l + 3]);
            const uint4 r = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32), m, 0x1417u), (uint32_t)seed,
                                          (uint32_t)(seed >> 32));
            v = a * (2.0f * uniform01(r.x) - 1.0f);
        }
    }
    p[idx] = v;
    pb[idx] = __float2bfloat16_rn(v);
}

// Pseudo-random permutation of [0, n) (4-round Feistel network on
// [0, 4^hb), keyed by Philox, with cycle walking into [0, n)).
static __device__ __forceinline__ uint32_t feistel(uint32_t x, int hb, uint32_t k0, uint32_t k1)
{
    const uint32_t mask = (1u << hb) - 1u;
    uint32_t L = x >> hb, R = x & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t F = philox4x32_10(make_uint4(R, (uint32_t)r, k0, 0x5u), k0, k1).x & mask;
        const uint32_t nL = R;
        R = L ^ F;
        L = nL;
    }
    return (L << hb) | R;
}
static __device__ __forceinline__ uint32_t permute(uint32_t i, uint32_t n, int hb, uint32_t k0, uint32_t k1)
{
    uint32_t x = i;
    const uint64_t dom = 1ull << (2 * hb);
    for (uint64_t guard = 0; guard < dom; ++guard) {
        x = feistel(x, hb, k0, k1);
        if (x < n) break;
    }
    return x;
}

// Batch rows r of every member: input normalised to [-1, 1], target
// standardised. Row index = perm_member(start + r) or start + r.
__global__ void mlp_batch_kernel(const float* __restrict__ X, const float* __restrict__ Y, int64_t n, int n_in,
                                 int n_out, int64_t start, int rows, int shuffle, int hb, uint64_t key,
                                 const float* __restrict__ lo, const float* __restrict__ hi,
                                 const float* __restrict__ mu, const float* __restrict__ sd, float* __restrict__ xb,
                                 float* __restrict__ tb)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (r >= rows) return;
    uint32_t src = (uint32_t)(start + r);
    if (shuffle) src = permute(src, (uint32_t)n, hb, (uint32_t)key ^ (0x9E3779B9u * (m + 1)), (uint32_t)(key >> 32));
    const int64_t ob = ((int64_t)m * rows + r);
    for (int i = 0; i < n_in; ++i)
        xb[ob * n_in + i] = 2.0f * (X[(int64_t)src * n_in + i] - lo[i]) / (hi[i] - lo[i]) - 1.0f;
    if (Y)
        for (int o = 0; o < n_out; ++o) tb[ob * n_out + o] = (Y[(int64_t)src * n_out + o] - mu[o]) / sd[o];
}

// dZ = 2 (Y - T) / (rows n_out); loss sum of squares per member (double).
__global__ void mlp_loss_kernel(const float* __restrict__ y, const float* __restrict__ t, int rows, int n_out,
                                float* __restrict__ dz, double* __restrict__ loss)
{
    const int m = blockIdx.y;
    const int64_t cnt = (int64_t)rows * n_out;
    const float scale = 2.0f / (float)cnt;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[m * cnt + i] - t[m * cnt + i];
        dz[m * cnt + i] = scale * d;
        acc += (double)d * d;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss + m, red[0] / (double)cnt);
}

// db[o] = sum over rows of dZ[row][o]; grid (ceil(n_out / 32), members).
__global__ void mlp_bias_grad_kernel(const float* __restrict__ dz, int rows, int n_out, float* __restrict__ g,
                                     int64_t g_mem)
{
    const int m = blockIdx.y;
    const int o = blockIdx.x * 32 + (threadIdx.x & 31);
    const int q = threadIdx.x >> 5;
    float s = 0.0f;
    if (o < n_out)
        for (int r = q; r < rows; r += 8) s += dz[((int64_t)m * rows + r) * n_out + o];
    __shared__ float red[8][33];
    red[q][threadIdx.x & 31] = s;
    __syncthreads();
    if (q == 0 && o < n_out) {
        float t = 0.0f;
        for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x & 31];
        g[m * g_mem + o] = t;
    }
}

// AdamW on every parameter of every member; decay[j] marks weight entries.
__global__ void mlp_adamw_kernel(float* __restrict__ p, __nv_bfloat16* __restrict__ pb, float* __restrict__ m1,
                                 float* __restrict__ m2, const float* __restrict__ g,
                                 const uint8_t* __restrict__ decay, int64_t n_par, int E, float lr, float wd,
                                 float b1, float b2, float eps, float bc1, float bc2)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_par * E) return;
    const int64_t j = idx % n_par;
    float x = p[idx];
    const float gr = g[idx];
    if (decay[j]) x *= 1.0f - lr * wd;
    const float a = b1 * m1[idx] + (1.0f - b1) * gr;
    const float b = b2 * m2[idx] + (1.0f - b2) * gr * gr;
    m1[idx] = a;
    m2[idx] = b;
    x -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
    p[idx] = x;
    pb[idx] = __float2bfloat16_rn(x);
}

// Per-output mean and population standard deviation of Y [n][n_out] (double
// sums), one block per output; sd 0 -> 1.
__global__ void mlp_moments_kernel(const float* __restrict__ Y, int64_t n, int n_out, float* __restrict__ mu,
                                   float* __restrict__ sd)
{
    const int o = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = Y[r * n_out + o];
        s += v;
        s2 += v * v;
    }
    __shared__ double r1[256], r2[256];
    r1[threadIdx.x] = s;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) { r1[threadIdx.x] += r1[threadIdx.x + k]; r2[threadIdx.x] += r2[threadIdx.x + k]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = r1[0] / (double)n;
        double var = r2[0] / (double)n - m * m;
        // second pass-free form; guard tiny negative values
        var = var > 0.0 ? var : 0.0;
        const double s_ = sqrt(var);
        mu[o] = (float)m;
        sd[o] = s_ > 0.0 ? (float)s_ : 1.0f;
    }
}

// Ensemble mean and variance of the (un-standardised) outputs.
__global__ void mlp_ensemble_kernel(const float* __restrict__ y, int rows, int n_out, int E,
                                    const float* __restrict__ mu, const float* __restrict__ sd,
                                    float* __restrict__ mean, float* __restrict__ var)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t cnt = (int64_t)rows * n_out;
    if (i >= cnt) return;
    const int o = (int)(i % n_out);
    float s = 0.0f;
    for (int m = 0; m < E; ++m) s += y[m * cnt + i];
    const float a = s / (float)E;
    float v = 0.0f;
    for (int m = 0; m < E; ++m) {
        const float d = y[m * cnt + i] - a;
        v += d * d;
    }
    mean[i] = mu[o] + sd[o] * a;
    if (var) var[i] = sd[o] * sd[o] * (v / (float)E);
}

// Uniform candidates in the box, from Philox(counter = (index, round, dim)).
__global__ void mlp_candidates_kernel(float* __restrict__ x, int64_t n, int n_in, const float* __restrict__ lo,
                                      const float* __restrict__ hi, uint64_t seed, uint64_t round)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int i = 0; i < n_in; ++i) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), (uint32_t)round, 0xCA00u + i),
                                      (uint32_t)seed, (uint32_t)(seed >> 32));
        x[c * n_in + i] = lo[i] + (hi[i] - lo[i]) * uniform01(r.x);
    }
}

// Proposal score of each candidate: closeness of output `o` to the threshold
// and ensemble spread, both in units of the output's training standard
// deviation: score = -|mean - threshold| / sd + var_weight sqrt(var) / sd.
__global__ void mlp_score_kernel(const float* __restrict__ mean, const float* __restrict__ var, int64_t n, int n_out,
                                 int o, float threshold, float var_weight, const float* __restrict__ sd,
                                 float* __restrict__ score)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n) return;
    const float so = sd[o] > 0.0f ? sd[o] : 1.0f;
    const float m = mean[c * n_out + o], v = var[c * n_out + o];
    float r = -fabsf(m - threshold) / so + var_weight * sqrtf(fmaxf(v, 0.0f)) / so;
    score[c] = r == r ? r : -INFINITY;
}

// Device array from the allocator in force when it grew (tvbx_set_allocator),
// released through the same one.
template <class T> struct Buf {
    T* p = nullptr;
    size_t n = 0;
    DevAllocator how;
    Buf() = default;
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    ~Buf() { release(); }
    cudaError_t ensure(size_t count)
    {
        if (count <= n && p) return cudaSuccess;
        release();
        void* q = nullptr;
        cudaError_t e = dev_alloc(&q, sizeof(T) * (count ? count : 1), &how);
        if (e == cudaSuccess) {
            p = static_cast<T*>(q);
            n = count;
        }
        return e;
    }
    void release()
    {
        dev_free(p, how);
        p = nullptr;
        n = 0;
    }
};

}  // namespace
}  // namespace tvbx

using namespace tvbx;

struct tvbx_surrogate {
    int n_in = 0, n_out = 0, E = 1;
    std::vector<int> dims;               // [n_in, h, ..., h, n_out]
    std::vector<int64_t> w_off, b_off;   // per layer
    int64_t n_par = 0;
    uint64_t seed = 0;
    int64_t step = 0;                    // AdamW steps taken
    bool scaled = false;                 // output standardisation set by a training call
    cudaStream_t stream = nullptr;
    Buf<float> p, m1, m2, g;             // [E][n_par]
    Buf<__nv_bfloat16> pb;               // [E][n_par]
    Buf<uint8_t> decay;                  // [n_par]
    Buf<int64_t> seg;                    // [4 L]
    Buf<float> lo, hi, mu, sd;           // box, output standardisation
    Buf<float> act, dz0, dz1, tb;        // work buffers
    Buf<float> splitk;                   // split-K partial products
    Buf<float> xin, yin, ymean, yvar, cand, score, cbox;
    Buf<double> loss;
    Buf<uint32_t> err;                   // device error word of the tensor-core products
    int work_rows = 0;
};

namespace {

tvbx_status sfail(tvbx_status code, const char* what, cudaError_t e = cudaSuccess)
{
    if (e == cudaErrorMemoryAllocation) return report_error(TVBX_E_OOM, "%s: device allocation failed", what);
    if (e != cudaSuccess) return report_error(TVBX_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return report_error(code, "%s", what);
}

#define SCK(call, what)                                                  \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return sfail(TVBX_E_CUDA, what, e_);      \
    } while (0)

int64_t act_offset(const tvbx_surrogate* s, int layer, int rows)
{
    // activations of layer l (0 = input) stored one after another, each [E][rows][dims[l]]
    int64_t o = 0;
    for (int l = 0; l < layer; ++l) o += (int64_t)s->E * rows * s->dims[l];
    return o;
}

cudaError_t ensure_work(tvbx_surrogate* s, int rows)
{
    if (rows <= s->work_rows) return cudaSuccess;
    int64_t total = 0, widest = 0;
    for (size_t l = 0; l < s->dims.size(); ++l) {
        total += (int64_t)s->E * rows * s->dims[l];
        widest = std::max<int64_t>(widest, (int64_t)s->E * rows * s->dims[l]);
    }
    cudaError_t e;
    if ((e = s->act.ensure(total)) != cudaSuccess) return e;
    if ((e = s->dz0.ensure(widest)) != cudaSuccess) return e;
    if ((e = s->dz1.ensure(widest)) != cudaSuccess) return e;
    if ((e = s->tb.ensure((size_t)s->E * rows * s->n_out)) != cudaSuccess) return e;
    // split-K partials of the weight gradients: up to 32 splits, at most 64 MB
    int64_t widest_w = 0;
    for (size_t l = 0; l + 1 < s->dims.size(); ++l)
        widest_w = std::max<int64_t>(widest_w, (int64_t)s->dims[l] * s->dims[l + 1]);
    if ((e = s->splitk.ensure((size_t)std::min<int64_t>(32 * s->E * widest_w, 1ll << 24))) != cudaSuccess) return e;
    s->work_rows = rows;
    return cudaSuccess;
}

// try_wait polls before a tensor-core product's wait gives up (seconds).
constexpr uint32_t kTcWait = 1u << 26;

// After a stream synchronisation: TVBX_E_TIMEOUT if a bounded wait of a
// tensor-core product expired since the last check (the word is cleared).
tvbx_status check_tc_error(tvbx_surrogate* s, const char* what)
{
    uint32_t w = 0;
    SCK(cudaMemcpy(&w, s->err.p, sizeof w, cudaMemcpyDeviceToHost), what);
    if (w) {
        SCK(cudaMemset(s->err.p, 0, sizeof w), what);
        return report_error(TVBX_E_TIMEOUT, "%s: a tensor-core product's bounded wait expired", what);
    }
    return TVBX_OK;
}

// Forward pass of rows already placed in the input activations.
cudaError_t forward(tvbx_surrogate* s, int rows)
{
    const int L = (int)s->dims.size() - 1;
    for (int l = 0; l < L; ++l) {
        const int I = s->dims[l], O = s->dims[l + 1];
        GemmArgs g{};
        g.A = s->act.p + act_offset(s, l, rows);
        g.sam = I; g.sak = 1; g.a_mem = (int64_t)rows * I;
        g.B = s->pb.p + s->w_off[l];
        g.sbn = I; g.sbk = 1; g.b_mem = s->n_par;
        g.C = s->act.p + act_offset(s, l + 1, rows);
        g.ldc = O; g.c_mem = (int64_t)rows * O;
        g.bias = s->p.p + s->b_off[l];
        g.bias_mem = s->n_par;
        g.M = rows; g.N = O; g.K = I;
        cudaError_t e = (l + 1 < L) ? gemm_tc<float, __nv_bfloat16, EPI_BIAS_RELU>(g, s->E, s->err.p, kTcWait, s->stream)
                                    : gemm_tc<float, __nv_bfloat16, EPI_BIAS>(g, s->E, s->err.p, kTcWait, s->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Loss and gradients of the batch in the input activations and s->tb.
cudaError_t backward(tvbx_surrogate* s, int rows)
{
    const int L = (int)s->dims.size() - 1;
    cudaError_t e;
    float* dz = s->dz0.p;
    float* dzn = s->dz1.p;
    {
        dim3 grid(std::min(64, (rows * s->n_out + 255) / 256), s->E);
        note_launch();
        mlp_loss_kernel<<<grid, 256, 0, s->stream>>>(s->act.p + act_offset(s, L, rows), s->tb.p, rows, s->n_out, dz,
                                                     s->loss.p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int l = L - 1; l >= 0; --l) {
        const int I = s->dims[l], O = s->dims[l + 1];
        const float* a_prev = s->act.p + act_offset(s, l, rows);
        // dW_l = dZ^T a_prev
        GemmArgs gw{};
        gw.A = dz; gw.sam = 1; gw.sak = O; gw.a_mem = (int64_t)rows * O;
        gw.B = a_prev; gw.sbn = 1; gw.sbk = I; gw.b_mem = (int64_t)rows * I;
        gw.C = s->g.p + s->w_off[l]; gw.ldc = I; gw.c_mem = s->n_par;
        gw.M = O; gw.N = I; gw.K = rows;
        if ((e = gemm_tc<float, float, EPI_STORE>(gw, s->E, s->err.p, kTcWait, s->stream, s->splitk.p, s->splitk.n)) !=
            cudaSuccess)
            return e;
        // db_l
        {
            dim3 grid((O + 31) / 32, s->E);
            note_launch();
            mlp_bias_grad_kernel<<<grid, 256, 0, s->stream>>>(dz, rows, O, s->g.p + s->b_off[l], s->n_par);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (l == 0) break;
        // dZ_{l-1} = (dZ W_l) masked by a_prev > 0
        GemmArgs gd{};
        gd.A = dz; gd.sam = O; gd.sak = 1; gd.a_mem = (int64_t)rows * O;
        gd.B = s->pb.p + s->w_off[l]; gd.sbn = 1; gd.sbk = I; gd.b_mem = s->n_par;
        gd.C = dzn; gd.ldc = I; gd.c_mem = (int64_t)rows * I;
        gd.mask = a_prev; gd.ldm = I; gd.mask_mem = (int64_t)rows * I;
        gd.M = rows; gd.N = I; gd.K = O;
        if ((e = gemm_tc<float, __nv_bfloat16, EPI_MASK>(gd, s->E, s->err.p, kTcWait, s->stream)) != cudaSuccess) return e;
        std::swap(dz, dzn);
    }
    return cudaSuccess;
}

int half_bits_for(int64_t n)
{
    int hb = 1;
    while ((1ll << (2 * hb)) < n) ++hb;
    return hb;
}

tvbx_status check_handle(const tvbx_surrogate* s)
{
    if (!s) return report_error(TVBX_E_INVALID_ARG, "NULL surrogate");
    return TVBX_OK;
}

// Copy caller rows (host or device) into a device buffer.
tvbx_status stage_rows(tvbx_surrogate* s, int32_t mem, const float* src, size_t count, Buf<float>& dst,
                       const float** out)
{
    if (mem == TVBX_MEM_DEVICE) {
        *out = src;
        return TVBX_OK;
    }
    SCK(dst.ensure(count), "surrogate staging buffer");
    SCK(cudaMemcpyAsync(dst.p, src, sizeof(float) * count, cudaMemcpyHostToDevice, s->stream), "surrogate input copy");
    *out = dst.p;
    return TVBX_OK;
}

}  // namespace

extern "C" {

tvbx_status tvbx_surrogate_create(const tvbx_surrogate_cfg* cfg, tvbx_surrogate** out)
{
    if (!cfg || !out) return report_error(TVBX_E_INVALID_ARG, "NULL cfg or out");
    *out = nullptr;
    if (cfg->n_in < 1 || cfg->n_in > 64 || cfg->n_out < 1 || cfg->n_out > 256 || cfg->n_hidden < 1 ||
        cfg->n_hidden > 1024 || cfg->n_layers < 1 || cfg->n_layers > 8 || cfg->n_members < 1 || cfg->n_members > 16)
        return report_error(TVBX_E_INVALID_ARG,
                            "need 1 <= n_in <= 64, 1 <= n_out <= 256, 1 <= n_hidden <= 1024, 1 <= n_layers <= 8, "
                            "1 <= n_members <= 16");
    if (!cfg->in_lo || !cfg->in_hi) return report_error(TVBX_E_INVALID_ARG, "NULL in_lo or in_hi");
    for (int i = 0; i < cfg->n_in; ++i)
        if (!(cfg->in_hi[i] > cfg->in_lo[i]) || !isfinite(cfg->in_lo[i]) || !isfinite(cfg->in_hi[i]))
            return report_error(TVBX_E_INVALID_ARG, "domain box: need finite in_lo[%d] < in_hi[%d]", i, i);
    auto* s = new tvbx_surrogate;
    s->n_in = cfg->n_in;
    s->n_out = cfg->n_out;
    s->E = cfg->n_members;
    s->seed = cfg->seed;
    s->dims.push_back(cfg->n_in);
    for (int l = 0; l < cfg->n_layers; ++l) s->dims.push_back(cfg->n_hidden);
    s->dims.push_back(cfg->n_out);
    const int L = (int)s->dims.size() - 1;
    std::vector<int64_t> seg(4 * L);
    std::vector<uint8_t> decay;
    for (int l = 0; l < L; ++l) {
        const int64_t I = s->dims[l], O = s->dims[l + 1];
        s->w_off.push_back(s->n_par);
        seg[4 * l] = s->n_par;
        seg[4 * l + 1] = I * O;
        seg[4 * l + 3] = I;
        s->n_par += I * O;
        decay.insert(decay.end(), (size_t)(I * O), 1);
        s->b_off.push_back(s->n_par);
        seg[4 * l + 2] = s->n_par;
        s->n_par += O;
        decay.insert(decay.end(), (size_t)O, 0);
    }
    auto fail_destroy = [&](cudaError_t e, const char* what) {
        tvbx_surrogate_destroy(s);
        return sfail(TVBX_E_CUDA, what, e);
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return fail_destroy(e, "surrogate stream");
    const size_t np = (size_t)s->n_par * s->E;
    if ((e = s->p.ensure(np)) || (e = s->m1.ensure(np)) || (e = s->m2.ensure(np)) || (e = s->g.ensure(np)) ||
        (e = s->pb.ensure(np)) || (e = s->decay.ensure((size_t)s->n_par)) || (e = s->seg.ensure(seg.size())) ||
        (e = s->lo.ensure(s->n_in)) || (e = s->hi.ensure(s->n_in)) || (e = s->mu.ensure(s->n_out)) ||
        (e = s->sd.ensure(s->n_out)) || (e = s->loss.ensure(s->E)) || (e = s->err.ensure(1)) ||
        (e = cudaMemsetAsync(s->err.p, 0, sizeof(uint32_t), s->stream)))
        return fail_destroy(e, "surrogate parameters");
    std::vector<float> lo(cfg->in_lo, cfg->in_lo + s->n_in), hi(cfg->in_hi, cfg->in_hi + s->n_in);
    std::vector<float> mu(s->n_out, 0.0f), sd(s->n_out, 1.0f);
    for (int i = 0; i < s->n_in; ++i) {
        lo[i] = (float)cfg->in_lo[i];
        hi[i] = (float)cfg->in_hi[i];
    }
    if ((e = cudaMemcpyAsync(s->decay.p, decay.data(), decay.size(), cudaMemcpyHostToDevice, s->stream)) ||
        (e = cudaMemcpyAsync(s->seg.p, seg.data(), sizeof(int64_t) * seg.size(), cudaMemcpyHostToDevice, s->stream)) ||
        (e = cudaMemcpyAsync(s->lo.p, lo.data(), sizeof(float) * s->n_in, cudaMemcpyHostToDevice, s->stream)) ||
        (e = cudaMemcpyAsync(s->hi.p, hi.data(), sizeof(float) * s->n_in, cudaMemcpyHostToDevice, s->stream)) ||
        (e = cudaMemcpyAsync(s->mu.p, mu.data(), sizeof(float) * s->n_out, cudaMemcpyHostToDevice, s->stream)) ||
        (e = cudaMemcpyAsync(s->sd.p, sd.data(), sizeof(float) * s->n_out, cudaMemcpyHostToDevice, s->stream)) ||
        (e = cudaMemsetAsync(s->m1.p, 0, sizeof(float) * np, s->stream)) ||
        (e = cudaMemsetAsync(s->m2.p, 0, sizeof(float) * np, s->stream)))
        return fail_destroy(e, "surrogate set-up");
    note_launch();
    mlp_init_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s->stream>>>(s->p.p, s->pb.p, s->seg.p, L, s->n_par, s->E,
                                                                        s->seed);
    if ((e = cudaGetLastError()) || (e = cudaStreamSynchronize(s->stream))) return fail_destroy(e, "surrogate init");
    *out = s;
    return TVBX_OK;
}

tvbx_status tvbx_surrogate_destroy(tvbx_surrogate* s)
{
    if (!s) return TVBX_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Buf<float>* b : {&s->p, &s->m1, &s->m2, &s->g, &s->lo, &s->hi, &s->mu, &s->sd, &s->act, &s->dz0, &s->dz1,
                          &s->tb, &s->splitk, &s->xin, &s->yin, &s->ymean, &s->yvar, &s->cand, &s->score, &s->cbox})
        b->release();
    s->pb.release();
    s->decay.release();
    s->seg.release();
    s->loss.release();
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return TVBX_OK;
}

tvbx_status tvbx_surrogate_info(const tvbx_surrogate* s, int64_t* n_params, int32_t* n_members)
{
    if (tvbx_status st = check_handle(s)) return st;
    if (n_params) *n_params = s->n_par;
    if (n_members) *n_members = s->E;
    return TVBX_OK;
}

tvbx_status tvbx_surrogate_params(tvbx_surrogate* s, int32_t member, float* get_out, const float* set_in)
{
    if (tvbx_status st = check_handle(s)) return st;
    if (member < 0 || member >= s->E) return report_error(TVBX_E_INVALID_ARG, "member out of range");
    const size_t off = (size_t)member * s->n_par;
    if (set_in) {
        std::vector<__nv_bfloat16> hb((size_t)s->n_par);
        for (int64_t j = 0; j < s->n_par; ++j) hb[j] = __float2bfloat16_rn(set_in[j]);
        SCK(cudaMemcpyAsync(s->p.p + off, set_in, sizeof(float) * s->n_par, cudaMemcpyHostToDevice, s->stream),
            "set params");
        SCK(cudaMemcpyAsync(s->pb.p + off, hb.data(), sizeof(__nv_bfloat16) * s->n_par, cudaMemcpyHostToDevice,
                            s->stream),
            "set params");
        SCK(cudaMemsetAsync(s->m1.p + off, 0, sizeof(float) * s->n_par, s->stream), "set params");
        SCK(cudaMemsetAsync(s->m2.p + off, 0, sizeof(float) * s->n_par, s->stream), "set params");
        s->step = 0;
    }
    if (get_out)
        SCK(cudaMemcpyAsync(get_out, s->p.p + off, sizeof(float) * s->n_par, cudaMemcpyDeviceToHost, s->stream),
            "get params");
    SCK(cudaStreamSynchronize(s->stream), "params");
    return TVBX_OK;
}

tvbx_status tvbx_surrogate_gradients(tvbx_surrogate* s, int32_t member, const float* X, const float* Y, int64_t n,
                                     float* loss, float* grads)
{
    if (tvbx_status st = check_handle(s)) return st;
    if (member < 0 || member >= s->E) return report_error(TVBX_E_INVALID_ARG, "member out of range");
    if (!X || !Y || n < 1 || n > (1 << 20)) return report_error(TVBX_E_INVALID_ARG, "need X, Y and 1 <= n <= 2^20");
    const int rows = (int)n;
    SCK(ensure_work(s, rows), "surrogate work buffers");
    const float *dX, *dY;
    if (tvbx_status st = stage_rows(s, TVBX_MEM_HOST, X, (size_t)n * s->n_in, s->xin, &dX)) return st;
    if (tvbx_status st = stage_rows(s, TVBX_MEM_HOST, Y, (size_t)n * s->n_out, s->yin, &dY)) return st;
    SCK(cudaMemsetAsync(s->loss.p, 0, sizeof(double) * s->E, s->stream), "loss");
    note_launch();
    mlp_batch_kernel<<<dim3((rows + 127) / 128, s->E), 128, 0, s->stream>>>(
        dX, dY, n, s->n_in, s->n_out, 0, rows, 0, 1, 0, s->lo.p, s->hi.p, s->mu.p, s->sd.p, s->act.p, s->tb.p);
    SCK(cudaGetLastError(), "batch");
    SCK(forward(s, rows), "forward");
    SCK(backward(s, rows), "backward");
    double hl[16];
    SCK(cudaMemcpyAsync(hl, s->loss.p, sizeof(double) * s->E, cudaMemcpyDeviceToHost, s->stream), "loss");
    if (grads)
        SCK(cudaMemcpyAsync(grads, s->g.p + (size_t)member * s->n_par, sizeof(float) * s->n_par,
                            cudaMemcpyDeviceToHost, s->stream),
            "gradients");
    SCK(cudaStreamSynchronize(s->stream), "gradients");
    if (tvbx_status st = check_tc_error(s, "gradients")) return st;
    if (loss) *loss = (float)hl[member];
    return TVBX_OK;
}

tvbx_status tvbx_surrogate_train(tvbx_surrogate* s, int32_t mem, const float* X, const float* Y, int64_t n,
                                 int32_t epochs, int32_t batch, float lr, float weight_decay, int32_t flags,
                                 float* loss_out)
{
    const int shuffle = (flags & TVBX_TRAIN_SHUFFLE) ? 1 : 0;
    if (tvbx_status st = check_handle(s)) return st;
    if (mem != TVBX_MEM_HOST && mem != TVBX_MEM_DEVICE) return report_error(TVBX_E_INVALID_ARG, "bad mem");
    if (!X || !Y || n < 1 || n > (1ll << 31) - 1) return report_error(TVBX_E_INVALID_ARG, "need X, Y and 1 <= n < 2^31");
    if (epochs < 1 || batch < 1 || batch > 65536 || !(lr > 0.0f) || !(weight_decay >= 0.0f))
        return report_error(TVBX_E_INVALID_ARG, "need epochs >= 1, 1 <= batch <= 65536, lr > 0, weight_decay >= 0");
    const int rows_max = (int)std::min<int64_t>(batch, n);
    SCK(ensure_work(s, rows_max), "surrogate work buffers");
    const float *dX, *dY;
    if (tvbx_status st = stage_rows(s, mem, X, (size_t)n * s->n_in, s->xin, &dX)) return st;
    if (tvbx_status st = stage_rows(s, mem, Y, (size_t)n * s->n_out, s->yin, &dY)) return st;
    // output standardisation from this training set, unless an earlier one is kept
    if (!(flags & TVBX_TRAIN_KEEP_SCALE) || !s->scaled) {
        note_launch();
        mlp_moments_kernel<<<s->n_out, 256, 0, s->stream>>>(dY, n, s->n_out, s->mu.p, s->sd.p);
        SCK(cudaGetLastError(), "output moments");
        s->scaled = true;
    }
    const int hb = half_bits_for(n);
    const size_t np = (size_t)s->n_par * s->E;
    const double b1 = 0.9, b2 = 0.999;
    std::vector<double> ep_loss((size_t)s->E);
    for (int ep = 0; ep < epochs; ++ep) {
        SCK(cudaMemsetAsync(s->loss.p, 0, sizeof(double) * s->E, s->stream), "loss");
        const uint64_t key = s->seed * 0x9E3779B97F4A7C15ull + (uint64_t)(s->step + 1) * 0xD1B54A32D192ED03ull;
        int n_batches = 0;
        for (int64_t start = 0; start < n; start += batch) {
            const int rows = (int)std::min<int64_t>(batch, n - start);
            note_launch();
            mlp_batch_kernel<<<dim3((rows + 127) / 128, s->E), 128, 0, s->stream>>>(
                dX, dY, n, s->n_in, s->n_out, start, rows, shuffle, hb, key, s->lo.p, s->hi.p, s->mu.p,
                s->sd.p, s->act.p, s->tb.p);
            SCK(cudaGetLastError(), "batch");
            SCK(forward(s, rows), "forward");
            SCK(backward(s, rows), "backward");
            s->step += 1;
            const double bc1 = 1.0 - pow(b1, (double)s->step), bc2 = 1.0 - pow(b2, (double)s->step);
            note_launch();
            mlp_adamw_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s->stream>>>(
                s->p.p, s->pb.p, s->m1.p, s->m2.p, s->g.p, s->decay.p, s->n_par, s->E, lr, weight_decay, (float)b1,
                (float)b2, 1e-8f, (float)bc1, (float)bc2);
            SCK(cudaGetLastError(), "AdamW");
            ++n_batches;
        }
        if (loss_out) {
            SCK(cudaMemcpyAsync(ep_loss.data(), s->loss.p, sizeof(double) * s->E, cudaMemcpyDeviceToHost, s->stream),
                "loss");
            SCK(cudaStreamSynchronize(s->stream), "loss");
            double t = 0.0;
            for (int m = 0; m < s->E; ++m) t += ep_loss[m];
            loss_out[ep] = (float)(t / (s->E * (double)n_batches));
        }
    }
    SCK(cudaStreamSynchronize(s->stream), "train");
    if (tvbx_status st = check_tc_error(s, "train")) return st;
    return TVBX_OK;
}

// Forward of n rows (device pointer, raw parameter units) in chunks; ensemble
// mean / variance to the device buffers mean, var.
static tvbx_status predict_device(tvbx_surrogate* s, const float* dX, int64_t n, float* mean, float* var)
{
    const int chunk = 16384;
    SCK(ensure_work(s, (int)std::min<int64_t>(chunk, n)), "surrogate work buffers");
    const int L = (int)s->dims.size() - 1;
    for (int64_t start = 0; start < n; start += chunk) {
        const int rows = (int)std::min<int64_t>(chunk, n - start);
        note_launch();
        mlp_batch_kernel<<<dim3((rows + 127) / 128, s->E), 128, 0, s->stream>>>(
            dX, nullptr, n, s->n_in, s->n_out, start, rows, 0, 1, 0, s->lo.p, s->hi.p, s->mu.p, s->sd.p, s->act.p,
            nullptr);
        SCK(cudaGetLastError(), "predict batch");
        SCK(forward(s, rows), "predict forward");
        const int64_t cnt = (int64_t)rows * s->n_out;
        note_launch();
        mlp_ensemble_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s->stream>>>(
            s->act.p + act_offset(s, L, rows), rows, s->n_out, s->E, s->mu.p, s->sd.p, mean + start * s->n_out,
            var ? var + start * s->n_out : nullptr);
        SCK(cudaGetLastError(), "ensemble");
    }
    return TVBX_OK;
}

// Proposal scores of the device candidates dX [n][n_in] (mlp_score_kernel)
// and the indices of the n_propose best that exclude (host, nullable) leaves
// open, best first, ties to the lower index. score receives all n scores.
static tvbx_status score_and_pick(tvbx_surrogate* s, const float* dX, int64_t n, const uint8_t* exclude, int32_t output,
                                  float threshold, float var_weight, int32_t n_propose, std::vector<float>& score,
                                  std::vector<int64_t>& idx)
{
    SCK(s->ymean.ensure((size_t)n * s->n_out), "candidate predictions");
    SCK(s->yvar.ensure((size_t)n * s->n_out), "candidate predictions");
    if (tvbx_status st = predict_device(s, dX, n, s->ymean.p, s->yvar.p)) return st;
    // scores on the device; the n_propose best on the host
    SCK(s->score.ensure((size_t)n), "scores");
    note_launch();
    mlp_score_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(s->ymean.p, s->yvar.p, n, s->n_out, output,
                                                                         threshold, var_weight, s->sd.p, s->score.p);
    SCK(cudaGetLastError(), "scores");
    score.resize((size_t)n);
    SCK(cudaMemcpyAsync(score.data(), s->score.p, sizeof(float) * n, cudaMemcpyDeviceToHost, s->stream), "scores");
    SCK(cudaStreamSynchronize(s->stream), "scores");
    if (tvbx_status st = check_tc_error(s, "ranking")) return st;
    idx.clear();
    idx.reserve((size_t)n);
    for (int64_t c = 0; c < n; ++c)
        if (!exclude || !exclude[c]) idx.push_back(c);
    if ((int64_t)idx.size() < n_propose)
        return report_error(TVBX_E_INVALID_ARG, "n_propose %d exceeds the %lld candidates not excluded", n_propose,
                            (long long)idx.size());
    auto better = [&](int64_t a, int64_t b) { return score[a] > score[b] || (score[a] == score[b] && a < b); };
    std::nth_element(idx.begin(), idx.begin() + (n_propose - 1), idx.end(), better);
    std::sort(idx.begin(), idx.begin() + n_propose, better);
    idx.resize((size_t)n_propose);
    return TVBX_OK;
}

tvbx_status tvbx_surrogate_predict(tvbx_surrogate* s, int32_t mem, const float* X, int64_t n, float* y_mean,
                                   float* y_var)
{
    if (tvbx_status st = check_handle(s)) return st;
    if (mem != TVBX_MEM_HOST && mem != TVBX_MEM_DEVICE) return report_error(TVBX_E_INVALID_ARG, "bad mem");
    if (!X || !y_mean || n < 1) return report_error(TVBX_E_INVALID_ARG, "need X, y_mean and n >= 1");
    const float* dX;
    if (tvbx_status st = stage_rows(s, mem, X, (size_t)n * s->n_in, s->xin, &dX)) return st;
    float *dm = y_mean, *dv = y_var;
    if (mem == TVBX_MEM_HOST) {
        SCK(s->ymean.ensure((size_t)n * s->n_out), "predict output");
        dm = s->ymean.p;
        if (y_var) {
            SCK(s->yvar.ensure((size_t)n * s->n_out), "predict output");
            dv = s->yvar.p;
        }
    }
    if (tvbx_status st = predict_device(s, dX, n, dm, dv)) return st;
    if (mem == TVBX_MEM_HOST) {
        SCK(cudaMemcpyAsync(y_mean, dm, sizeof(float) * n * s->n_out, cudaMemcpyDeviceToHost, s->stream), "predict");
        if (y_var)
            SCK(cudaMemcpyAsync(y_var, dv, sizeof(float) * n * s->n_out, cudaMemcpyDeviceToHost, s->stream), "predict");
    }
    SCK(cudaStreamSynchronize(s->stream), "predict");
    if (tvbx_status st = check_tc_error(s, "predict")) return st;
    return TVBX_OK;
}

tvbx_status tvbx_surrogate_propose(tvbx_surrogate* s, int64_t n_candidates, uint64_t round, int32_t output,
                                   float threshold, float var_weight, const double* cand_lo, const double* cand_hi,
                                   int32_t n_propose, float* points_out, float* scores_out)
{
    if (tvbx_status st = check_handle(s)) return st;
    if (n_candidates < 1 || n_candidates > (1ll << 26) || n_propose < 1 || n_propose > n_candidates || !points_out)
        return report_error(TVBX_E_INVALID_ARG, "need 1 <= n_propose <= n_candidates <= 2^26 and points_out");
    if (output < 0 || output >= s->n_out) return report_error(TVBX_E_INVALID_ARG, "output index out of range");
    if ((cand_lo == nullptr) != (cand_hi == nullptr))
        return report_error(TVBX_E_INVALID_ARG, "give both cand_lo and cand_hi or neither");
    const float *clo = s->lo.p, *chi = s->hi.p;
    if (cand_lo) {
        std::vector<float> b(2 * (size_t)s->n_in);
        for (int i = 0; i < s->n_in; ++i) {
            if (!(cand_lo[i] <= cand_hi[i]) || !isfinite(cand_lo[i]) || !isfinite(cand_hi[i]))
                return report_error(TVBX_E_INVALID_ARG, "candidate box: need finite cand_lo[%d] <= cand_hi[%d]", i, i);
            b[i] = (float)cand_lo[i];
            b[s->n_in + i] = (float)cand_hi[i];
        }
        SCK(s->cbox.ensure(b.size()), "candidate box");
        SCK(cudaMemcpyAsync(s->cbox.p, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice, s->stream),
            "candidate box");
        clo = s->cbox.p;
        chi = s->cbox.p + s->n_in;
    }
    SCK(s->cand.ensure((size_t)n_candidates * s->n_in), "candidates");
    SCK(s->ymean.ensure((size_t)n_candidates * s->n_out), "candidate predictions");
    SCK(s->yvar.ensure((size_t)n_candidates * s->n_out), "candidate predictions");
    note_launch();
    mlp_candidates_kernel<<<(unsigned)((n_candidates + 255) / 256), 256, 0, s->stream>>>(
        s->cand.p, n_candidates, s->n_in, clo, chi, s->seed, round);
    SCK(cudaGetLastError(), "candidates");
    std::vector<float> score;
    std::vector<int64_t> idx;
    if (tvbx_status st = score_and_pick(s, s->cand.p, n_candidates, nullptr, output, threshold, var_weight, n_propose,
                                        score, idx))
        return st;
    std::vector<float> pts((size_t)n_candidates * s->n_in);
    SCK(cudaMemcpyAsync(pts.data(), s->cand.p, sizeof(float) * pts.size(), cudaMemcpyDeviceToHost, s->stream),
        "candidate points");
    SCK(cudaStreamSynchronize(s->stream), "candidate points");
    for (int32_t r = 0; r < n_propose; ++r) {
        memcpy(points_out + (size_t)r * s->n_in, pts.data() + (size_t)idx[r] * s->n_in, sizeof(float) * s->n_in);
        if (scores_out) scores_out[r] = score[idx[r]];
    }
    return TVBX_OK;
}

tvbx_status tvbx_surrogate_rank(tvbx_surrogate* s, const float* X, int64_t n, const uint8_t* exclude, int32_t output,
                                float threshold, float var_weight, int32_t n_propose, int64_t* idx_out,
                                float* scores_out)
{
    if (tvbx_status st = check_handle(s)) return st;
    if (!X || !idx_out || n < 1 || n > (1ll << 26) || n_propose < 1 || n_propose > n)
        return report_error(TVBX_E_INVALID_ARG, "need X, idx_out and 1 <= n_propose <= n <= 2^26");
    if (output < 0 || output >= s->n_out) return report_error(TVBX_E_INVALID_ARG, "output index out of range");
    const float* dX;
    if (tvbx_status st = stage_rows(s, TVBX_MEM_HOST, X, (size_t)n * s->n_in, s->cand, &dX)) return st;
    std::vector<float> score;
    std::vector<int64_t> idx;
    if (tvbx_status st =
            score_and_pick(s, dX, n, exclude, output, threshold, var_weight, n_propose, score, idx))
        return st;
    for (int32_t r = 0; r < n_propose; ++r) {
        idx_out[r] = idx[r];
        if (scores_out) scores_out[r] = score[idx[r]];
    }
    return TVBX_OK;
}

}  // extern "C"
